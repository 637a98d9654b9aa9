// gpma_dev.cuh -- device-side types and helpers shared by the libgpma kernels.
//
// Data layout in HBM for one array of C = L * 2^h slots (nleaves = 2^h):
//   slots[C]        u64 keys, EMPTY = all ones (the packed memory array, Sec. 4.1)
//   cnt[nleaves]    u32 valid keys per leaf (level 0 of the count tree)
//   F[nleaves]      u64 smallest valid key of each leaf, EMPTY for an empty leaf
//                   (the pivots of the leaf search, Algorithm "GPMA+", line "BinarySearchLeafSegments")
//   tree[]          u32 counts of the segments at levels 1..h, level i at tree_off[i]
//                   (logical counts: valid keys + inserts still pending in this batch)
//   mark[]          u32 per segment of levels 1..h, set while a batch decides merges
//   row_end[V]      u32 slot of the guard of every vertex (CSR row offsets, Sec. 4.2)
//   deg[V]          u32 out-degree of every vertex, kept by the update kernels
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gpk {

constexpr uint64_t kEmpty = ~0ull;
constexpr int kMaxLv = 48;
constexpr uint32_t kNoLevel = 0xFFu;

// error bits of one call (Ctl::err); mutating kernels do nothing once set
constexpr uint32_t kErrKey = 1u;      // a key outside the vertex range
constexpr uint32_t kErrTimeout = 2u;  // a bounded spin gave up
constexpr uint32_t kErrInternal = 4u; // an internal bound was exceeded

struct Geo {
  uint64_t *slots;
  uint32_t *cnt;
  uint64_t *F;
  uint32_t *tree;
  uint32_t *mark;
  uint32_t *row_end;
  uint32_t *deg;  // out-degree of every vertex (stored edges, guards excluded)
  uint64_t C, nleaves;
  uint32_t L, logL, h, V, raw;
  uint32_t dual;              // deletion as the dual of insertion: lower bounds kept
  uint32_t leaf_warps;        // warps per block of the general level-0 pass (0: by shared memory)
  uint64_t tree_off[kMaxLv];  // offset of level i (1..h) inside tree/mark
  uint64_t maxc[kMaxLv];      // max_i: largest admissible count at level i
  uint64_t minc[kMaxLv];      // min_i: smallest admissible count at level i (dual mode)
};

// Level-0 test of a touched leaf holding c keys after its deletes and inserts:
// lazy mode merges a leaf with inserts iff c <= max_0; dual mode rewrites every
// touched leaf with min_0 <= c <= max_0 (a single-leaf array waives min_0).
__device__ __forceinline__ bool leaf_fits(const Geo &g, uint64_t c, uint32_t nins) {
  if (!g.dual) return nins > 0 && c <= g.maxc[0];
  return c <= g.maxc[0] && (c >= g.minc[0] || g.h == 0);
}

// Level test of an escalated segment of level i holding t keys (valid + pending):
// t <= max_i, and in dual mode t >= min_i below the root.
__device__ __forceinline__ bool level_admits(const Geo &g, uint32_t i, uint64_t t) {
  return t <= g.maxc[i] && (!g.dual || i == g.h || t >= g.minc[i]);
}

// Device control block of one handle: counters written by kernels, read by
// later kernels of the same batch and (at sync points) by the host.
struct Ctl {
  uint32_t err;       // this call
  uint32_t sticky;    // accumulated, cleared by gpma_status
  uint32_t n;         // raw batch size (inserts + deletes)
  uint32_t m;         // after unique + cancellation
  uint32_t nruns;     // distinct leaves among the m keys
  uint32_t npend;     // inserts left pending after the leaf pass
  uint32_t neruns;    // distinct leaves among the pending inserts
  uint32_t nsegs;     // maximal merged segments
  uint32_t nleafw;    // leaves covered by the maximal merged segments
  uint32_t nesc;      // runs whose inserts did not fit at level 0
  uint32_t nfail;     // pending runs that no level up to the root admits (root resize)
  uint32_t nlong;     // runs left by the 64-slot fast leaf pass to the general one
  uint32_t epoch;     // bumped per single-pass scan, tags look-back status words
  uint32_t ticket[16];
  uint64_t total;     // logical number of stored keys (guards included)
  uint64_t n_inserted, n_deleted;
  uint64_t st_cov_touched, st_l0_only, st_empties;
  uint64_t st_del_leaves;  // runs holding an applied delete
  uint32_t levels_climbed;
  uint32_t n_merged0;
  uint64_t merges[kMaxLv];
  uint64_t gen_count;  // general-purpose counter (exports)
  uint32_t resized;    // this call grew the array on the device (into the spare)
  uint32_t nvlong;     // runs longer than kLongRun, left to the chunked level-0 path
  uint32_t lm_miss;    // learned searches of this batch whose predicted window missed the leaf
  uint32_t spin_limit; // polls a bounded wait may make before it gives up (0: the built-in limits)
};

__device__ __forceinline__ bool is_guard(uint64_t k) {
  return k != kEmpty && (k & 0xFFFFFFFFull) == 0xFFFFFFFFull;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Block index seen by a kernel body: the launch's own grid (one handle), or one
// handle's share of a launch that serves many handles (blocks [0, n) of its own).
struct GridIdx {
  __device__ __forceinline__ uint32_t x() const { return blockIdx.x; }
  __device__ __forceinline__ uint32_t n() const { return gridDim.x; }
};
struct SubIdx {
  uint32_t bx, bn;
  __device__ __forceinline__ uint32_t x() const { return bx; }
  __device__ __forceinline__ uint32_t n() const { return bn; }
};

// add +1 / -1 to the out-degree of the source of every marked lane's key; lanes
// of one source (rows are contiguous) combine into one atomic
__device__ __forceinline__ void degree_delta(uint32_t *deg, bool active, uint64_t key, int d) {
  const uint32_t src = active ? (uint32_t)(key >> 32) : 0xFFFFFFFFu;
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, src);
  if (active && (threadIdx.x & 31u) == (uint32_t)(__ffs(peers) - 1))
    atomicAdd(&deg[src], (uint32_t)(d * __popc(peers)));
}
__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << lane_id()) - 1u; }

// Out-degree change of one run held in lanes [0, len) in ascending key order
// (lanes of one source are contiguous): d = +1 for an inserted edge, -1 for a
// deleted one, 0 otherwise.  One atomic per source, from its first lane.
__device__ __forceinline__ void run_degree_delta(uint32_t *deg, uint32_t len, uint64_t key, int d) {
  const uint32_t lane = lane_id();
  const bool act = lane < len;
  const uint32_t pos = __ballot_sync(0xFFFFFFFFu, act && d > 0), neg = __ballot_sync(0xFFFFFFFFu, act && d < 0);
  if (!(pos | neg)) return;  // the same on every lane
  const uint32_t src = (uint32_t)(key >> 32);
  const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, src, 1);
  const uint32_t heads = __ballot_sync(0xFFFFFFFFu, act && (lane == 0 || prev != src));
  if (act && ((heads >> lane) & 1u)) {
    const uint32_t later = heads & ~((2u << lane) - 1u);  // lane 31: 2u << 31 == 0, so none
    const uint32_t end = later ? (uint32_t)(__ffs(later) - 1) : len;
    const uint32_t seg = (end >= 32 ? 0xFFFFFFFFu : ((1u << end) - 1u)) & ~((1u << lane) - 1u);
    const int sum = __popc(pos & seg) - __popc(neg & seg);
    if (sum) atomicAdd(&deg[src], (uint32_t)sum);
  }
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if ((int)lane_id() >= o) v += t;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Exclusive scan of one u32 per thread over the block; wsum: 33 words of shared
// memory; *total = the block's sum.  Every thread of the block must call it.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *wsum, uint32_t *total) {
  const uint32_t lane = lane_id(), wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t inc = warp_incl_scan(v);
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const uint32_t x = lane < nw ? wsum[lane] : 0u;
    const uint32_t xi = warp_incl_scan(x);
    wsum[lane] = xi - x;
    if (lane == 31) wsum[32] = xi;
  }
  __syncthreads();
  const uint32_t r = wsum[wid] + inc - v;
  *total = wsum[32];
  __syncthreads();  // wsum is reused by the next scan
  return r;
}

// first index in a[0..n) with a[i] >= k (a sorted ascending)
template <typename T>
__device__ __forceinline__ uint32_t lower_bound_dev(const T *a, uint32_t n, T k) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < k) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Leaf of key k on the current array: the last leaf whose smallest valid key is
// <= k, leaf 0 if none.  With eff(j) = smallest valid key of the first non-empty
// leaf at or after j (+inf past the end), eff is non-decreasing and the leaf is
// p - 1 for p = the first j with eff(j) > k.  search_first_above finds p inside
// [lo, hi] given eff(lo - 1) <= k (or lo = 0) and eff(hi) > k (or hi = nleaves);
// empty leaves are skipped forward.
__device__ __forceinline__ uint64_t search_first_above(const uint64_t *__restrict__ F, uint64_t lo, uint64_t hi,
                                                       uint64_t k) {
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1, j = mid;
    uint64_t f = kEmpty;
    while (j < hi) {
      f = __ldg(F + j);
      if (f != kEmpty) break;
      ++j;
    }
    if (j >= hi || f > k) hi = mid;
    else lo = j + 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t leaf_search(const uint64_t *__restrict__ F, uint64_t nleaves, uint64_t k) {
  const uint64_t p = search_first_above(F, 0, nleaves, k);
  return p ? (uint32_t)(p - 1) : 0u;
}

// ---- learned leaf search (two-stage model over the pivots) -------------------------------------
// Pieces: the leaves are cut into kPieces equal ranges of 2^span leaves each (the
// density bounds keep the keys per range near-equal, so these are quantile buckets
// of the pivots).  Root: the piece of key k is the last piece whose boundary (its
// first training pivot) is <= k, found by a search over the 4096 boundaries, which
// stay in L1.  Piece: an FP32 linear model first + (k - kb) * slope over its own
// leaves, clamped to the piece's answer bracket [lo, hi], with training error err.
// The predicted window is checked against the current pivots and widened until it
// brackets the answer, so the result equals leaf_search exactly, whatever the
// model's staleness.
constexpr uint32_t kPieces = 4096;

struct Piece {
  uint64_t kb;      // boundary: pivot of the piece's first non-empty leaf (empty piece:
                    // the next non-empty piece's boundary, EMPTY at the end)
  uint32_t lo, hi;  // answer bracket at training time
  uint32_t first;   // first non-empty training leaf (kNoLeaf: none)
  uint32_t err;     // max |prediction - leaf| over the training leaves
  float slope;
  uint32_t pad;
};

struct ModelHead {
  uint32_t npieces;  // pieces in use (min(kPieces, leaves))
  uint32_t span;     // log2 leaves per piece
  uint32_t valid;
  uint32_t pad0;
  uint64_t drift;    // leaves rewritten by merges above level 0 since the model was trained
  uint64_t rbase;    // radix table over the boundaries: prefix(k) = min((k - rbase) >> rshift,
  uint32_t rshift;   // kRadix - 1) (0 for k < rbase)
  uint32_t done;     // blocks of the training kernel finished so far (0 between launches)
};

// Radix table of the root stage: rt[r] = first piece whose boundary has a prefix
// >= r (rt[kRadix] = npieces), so the piece of key k (the last piece whose
// boundary is <= k) is rt[r] - 1 or one of the pieces [rt[r], rt[r + 1]) for
// r = prefix(k).  It lives right after the pieces.
constexpr uint32_t kRadix = 4096;
constexpr uint32_t kModelPieces = kPieces + (uint32_t)(((kRadix + 1) * 4 + 31) / 32);  // Piece slots allocated
__device__ __forceinline__ const uint32_t *model_radix(const Piece *pieces) {
  return reinterpret_cast<const uint32_t *>(pieces + kPieces);
}
__device__ __forceinline__ uint32_t model_prefix(const ModelHead &m, uint64_t k) {
  if (k < m.rbase) return 0;
  const uint64_t r = (k - m.rbase) >> m.rshift;
  return r < kRadix - 1 ? (uint32_t)r : kRadix - 1;
}

constexpr uint32_t kNoLeaf = 0xFFFFFFFFu;

// last piece whose boundary is <= k, or -1 (the binary search runs over the
// pieces of k's radix-table entry only)
__device__ __forceinline__ int32_t model_route(const ModelHead &m, const Piece *__restrict__ pieces, uint64_t k) {
  const uint32_t *rt = model_radix(pieces);
  const uint32_t r = model_prefix(m, k);
  uint32_t a = __ldg(rt + r), b = __ldg(rt + r + 1);
  while (a < b) {
    const uint32_t mid = (a + b) >> 1;
    if (__ldg(&pieces[mid].kb) <= k) a = mid + 1;
    else b = mid;
  }
  return (int32_t)a - 1;
}

// model_route of Q keys at once (their dependent loads in flight together);
// bucket[q] = the piece, 0 when the key lies below every boundary or !act[q]
template <int Q>
__device__ __forceinline__ void model_route_lockstep(const ModelHead &m, const Piece *__restrict__ pieces,
                                                     const uint64_t (&k)[Q], const bool (&act)[Q],
                                                     uint32_t (&bucket)[Q]) {
  const uint32_t *rt = model_radix(pieces);
  uint32_t a[Q], b[Q];
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const uint32_t r = model_prefix(m, k[q]);
    a[q] = act[q] ? __ldg(rt + r) : 0u;
    b[q] = act[q] ? __ldg(rt + r + 1) : 0u;
  }
  for (;;) {
    uint32_t mid[Q];
    uint64_t kb[Q];
    bool any = false;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      mid[q] = (a[q] + b[q]) >> 1;
      kb[q] = 0;
      if (a[q] < b[q]) {
        kb[q] = __ldg(&pieces[mid[q]].kb);
        any = true;
      }
    }
    if (!any) break;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      if (a[q] >= b[q]) continue;
      if (kb[q] <= k[q]) a[q] = mid[q] + 1;
      else b[q] = mid[q];
    }
  }
#pragma unroll
  for (int q = 0; q < Q; q++) bucket[q] = a[q] ? a[q] - 1 : 0u;
}

// eff(j) <= k ?
__device__ __forceinline__ bool eff_at_most(const uint64_t *__restrict__ F, uint64_t nleaves, uint64_t j, uint64_t k) {
  for (; j < nleaves; ++j) {
    const uint64_t f = __ldg(F + j);
    if (f != kEmpty) return f <= k;
  }
  return false;
}

__device__ __forceinline__ uint32_t learned_leaf_search(const ModelHead &m, const Piece *__restrict__ pieces,
                                                        const uint64_t *__restrict__ F, uint64_t nleaves,
                                                        uint64_t k) {
  const int32_t pi = model_route(m, pieces, k);
  const Piece pc = pieces[pi < 0 ? 0 : pi];
  // candidate window for p (= answer + 1)
  int64_t pred = pi < 0 ? 0 : (int64_t)pc.lo;
  if (pi >= 0 && pc.first != kNoLeaf) {
    const float d = (float)(k > pc.kb ? k - pc.kb : 0ull) * pc.slope;
    pred = (int64_t)pc.first + (int64_t)d;
    if (pred < (int64_t)pc.lo) pred = pc.lo;
    if (pred > (int64_t)pc.hi) pred = pc.hi;
  }
  int64_t a = pred - (int64_t)pc.err, b = pred + (int64_t)pc.err + 2;
  if (a < 0) a = 0;
  if (a > (int64_t)nleaves) a = (int64_t)nleaves;  // a model trained on another geometry
  if (b > (int64_t)nleaves) b = (int64_t)nleaves;
  if (b < a) b = a;
  // widen until eff(a - 1) <= k (or a = 0) and eff(b) > k (or b = nleaves); the
  // first probe of both ends goes out together (no empty leaf: one load each)
  if (a > 0 && b < (int64_t)nleaves) {
    const uint64_t fa = __ldg(F + (a - 1)), fb = __ldg(F + b);
    if (fa != kEmpty && fb != kEmpty && fa <= k && fb > k) {
      const uint64_t p = search_first_above(F, (uint64_t)a, (uint64_t)b, k);
      return p ? (uint32_t)(p - 1) : 0u;
    }
  }
  uint64_t step = pc.err + 2;
  while (a > 0 && !eff_at_most(F, nleaves, (uint64_t)(a - 1), k)) {
    a = a > (int64_t)step ? a - (int64_t)step : 0;
    step <<= 1;
  }
  step = pc.err + 2;
  while (b < (int64_t)nleaves && eff_at_most(F, nleaves, (uint64_t)b, k)) {
    b = b + (int64_t)step < (int64_t)nleaves ? b + (int64_t)step : (int64_t)nleaves;
    step <<= 1;
  }
  const uint64_t p = search_first_above(F, (uint64_t)a, (uint64_t)b, k);
  return p ? (uint32_t)(p - 1) : 0u;
}

// ---- Q leaf searches in lock step ----------------------------------------------------------------
// search_first_above for Q keys at once, each inside its own [lo, hi): the Q
// bisections advance together, so their loads are in flight together.  out = the
// leaf (p - 1, or 0 for p = 0); keys with lo >= hi on entry get lo - 1 (or 0).
template <int Q>
__device__ __forceinline__ void bisect_lockstep(const uint64_t *__restrict__ F, uint64_t (&lo)[Q], uint64_t (&hi)[Q],
                                                const uint64_t (&k)[Q], uint32_t (&out)[Q]) {
  for (;;) {
    uint64_t mid[Q], f[Q];
    bool any = false;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      mid[q] = (lo[q] + hi[q]) >> 1;
      f[q] = kEmpty;
      if (lo[q] < hi[q]) {
        f[q] = __ldg(F + mid[q]);
        any = true;
      }
    }
    if (!any) break;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      if (lo[q] >= hi[q]) continue;
      uint64_t j = mid[q], fv = f[q];
      while (fv == kEmpty && ++j < hi[q]) fv = __ldg(F + j);  // empty leaves skipped forward
      if (j >= hi[q] || fv > k[q]) hi[q] = mid[q];
      else lo[q] = j + 1;
    }
  }
#pragma unroll
  for (int q = 0; q < Q; q++) out[q] = lo[q] ? (uint32_t)(lo[q] - 1) : 0u;
}

// leaf_search for Q keys (inactive keys get 0)
template <int Q>
__device__ __forceinline__ void leaf_search_lockstep(const uint64_t *__restrict__ F, uint64_t nleaves,
                                                     const uint64_t (&k)[Q], const bool (&act)[Q],
                                                     uint32_t (&out)[Q]) {
  uint64_t lo[Q], hi[Q];
#pragma unroll
  for (int q = 0; q < Q; q++) {
    lo[q] = 0;
    hi[q] = act[q] ? nleaves : 0;
  }
  bisect_lockstep<Q>(F, lo, hi, k, out);
}

// learned_leaf_search for Q keys in lock step: the route (radix table, then the
// pieces of the entry), the piece's prediction and its bracket check together;
// keys whose window is bracketed finish with one lock-step bisection inside it,
// the others (a stale model) take learned_leaf_search alone.  Same leaves.
// bucket (or nullptr): each key's bucket from model_route_lockstep (the sort by
// model piece routed the keys already); it fixes the route's result up to the keys
// before the first piece boundary, which share bucket 0 with the first piece.
template <int Q>
__device__ __forceinline__ uint32_t learned_search_lockstep(const ModelHead &m, const Piece *__restrict__ pieces,
                                                        const uint64_t *__restrict__ F, uint64_t nleaves,
                                                        const uint64_t (&k)[Q], const bool (&act)[Q],
                                                        uint32_t (&out)[Q], const uint16_t *bucket = nullptr) {
  const uint32_t *rt = model_radix(pieces);
  uint32_t a[Q], b[Q];  // a: pieces whose boundary is <= k, once a = b
#pragma unroll
  for (int q = 0; q < Q; q++) {
    if (bucket) {
      const uint32_t bq = bucket[q];
      a[q] = !act[q] ? 0u : (bq ? bq + 1u : (__ldg(&pieces[0].kb) <= k[q] ? 1u : 0u));
      b[q] = a[q];
    } else {
      const uint32_t r = model_prefix(m, k[q]);
      a[q] = act[q] ? __ldg(rt + r) : 0u;
      b[q] = act[q] ? __ldg(rt + r + 1) : 0u;
    }
  }
  for (;;) {  // last piece whose boundary is <= k
    uint32_t mid[Q];
    uint64_t kb[Q];
    bool any = false;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      mid[q] = (a[q] + b[q]) >> 1;
      kb[q] = 0;
      if (a[q] < b[q]) {
        kb[q] = __ldg(&pieces[mid[q]].kb);
        any = true;
      }
    }
    if (!any) break;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      if (a[q] >= b[q]) continue;
      if (kb[q] <= k[q]) a[q] = mid[q] + 1;
      else b[q] = mid[q];
    }
  }
  uint64_t lo[Q], hi[Q], fa[Q], fb[Q];
  bool ok[Q];
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const int32_t pi = (int32_t)a[q] - 1;
    const Piece pc = pieces[pi < 0 ? 0 : pi];
    int64_t pred = pi < 0 ? 0 : (int64_t)pc.lo;
    if (pi >= 0 && pc.first != kNoLeaf) {
      const float d = (float)(k[q] > pc.kb ? k[q] - pc.kb : 0ull) * pc.slope;
      pred = (int64_t)pc.first + (int64_t)d;
      if (pred < (int64_t)pc.lo) pred = pc.lo;
      if (pred > (int64_t)pc.hi) pred = pc.hi;
    }
    int64_t wa = pred - (int64_t)pc.err, wb = pred + (int64_t)pc.err + 2;
    if (wa < 0) wa = 0;
    if (wa > (int64_t)nleaves) wa = (int64_t)nleaves;
    if (wb > (int64_t)nleaves) wb = (int64_t)nleaves;
    if (wb < wa) wb = wa;
    lo[q] = (uint64_t)wa;
    hi[q] = (uint64_t)wb;
    ok[q] = act[q] && wa > 0 && wb < (int64_t)nleaves;
    fa[q] = ok[q] ? __ldg(F + (wa - 1)) : kEmpty;
    fb[q] = ok[q] ? __ldg(F + wb) : kEmpty;
  }
#pragma unroll
  for (int q = 0; q < Q; q++) {
    ok[q] = ok[q] && fa[q] != kEmpty && fb[q] != kEmpty && fa[q] <= k[q] && fb[q] > k[q];
    if (!ok[q]) lo[q] = hi[q] = 0;  // left to the single search below
  }
  bisect_lockstep<Q>(F, lo, hi, k, out);
  uint32_t miss = 0;
#pragma unroll
  for (int q = 0; q < Q; q++) {
    if (!act[q]) {
      out[q] = 0;
    } else if (!ok[q]) {
      out[q] = learned_leaf_search(m, pieces, F, nleaves, k[q]);
      ++miss;
    }
  }
  return miss;  // keys whose window missed (a model that has drifted)
}

// ---- single-pass look-back (tiles take tickets in launch order) -------------------
// Status word of one tile: [epoch:32][flag:2][value:30]; flag 1 = tile aggregate,
// flag 2 = inclusive prefix.  A spin is bounded; on give-up the call's error word
// gets kErrTimeout and the value read so far is used (the batch is then discarded).
constexpr uint64_t kFlagAgg = 1ull << 30;
constexpr uint64_t kFlagPre = 2ull << 30;
constexpr uint32_t kSpinLimit = 1u << 22;         // look-back waits
constexpr uint32_t kBarrierSpinLimit = 1u << 24;  // grid barriers

// the handle's wait limit, or `dflt` when none was set
__device__ __forceinline__ uint32_t spin_limit(const Ctl *ctl, uint32_t dflt) {
  const uint32_t v = ctl->spin_limit;
  return v ? v : dflt;
}

__device__ __forceinline__ uint64_t pack_status(uint32_t epoch, uint64_t flag, uint32_t v) {
  return ((uint64_t)epoch << 32) | flag | (uint64_t)(v & 0x3FFFFFFFu);
}

__device__ __forceinline__ void st_status(uint64_t *p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_status(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Exclusive prefix of `agg` over earlier tiles in column `col` of a status
// matrix laid out status[tile * stride + col].  Called by one thread per column.
// A wait that exceeds the handle's limit sets kErrTimeout in ctl->err.
__device__ __forceinline__ uint32_t lookback(uint64_t *status, uint32_t stride, uint32_t col,
                                             uint32_t tile, uint32_t agg, uint32_t epoch,
                                             Ctl *ctl) {
  if (tile == 0) {
    st_status(status + col, pack_status(epoch, kFlagPre, agg));
    return 0;
  }
  st_status(status + (uint64_t)tile * stride + col, pack_status(epoch, kFlagAgg, agg));
  uint32_t excl = 0;
  int64_t t = (int64_t)tile - 1;
  uint32_t spins = 0;
  const uint32_t limit = spin_limit(ctl, kSpinLimit);
  while (t >= 0) {
    uint64_t s = ld_status(status + (uint64_t)t * stride + col);
    if ((uint32_t)(s >> 32) != epoch || (s & (3ull << 30)) == 0) {
      if (++spins > limit) {
        atomicOr(&ctl->err, kErrTimeout);
        break;
      }
      __nanosleep(20);
      continue;
    }
    excl += (uint32_t)(s & 0x3FFFFFFFull);
    if (s & kFlagPre) break;
    --t;
  }
  st_status(status + (uint64_t)tile * stride + col, pack_status(epoch, kFlagPre, excl + agg));
  return excl;
}

}  // namespace gpk
