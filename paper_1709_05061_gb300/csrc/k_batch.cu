// k_batch.cu -- front end of one update batch (Algorithm "GPMA+ Segment-Oriented
// Insertion", Sec. 5.2, lines Sort(U) and BinarySearchLeafSegments(U)):
//   k_init_batch  reset the per-call control block and the radix histograms
//   k_prep        one sort tile per block: validate keys, compress (src, dst,
//                 insert/delete tag) into one sortable word, count the tile's
//                 first-pass digits and every pass's digits over the batch
//   per radix pass (stable LSD, reduce then scan: no chained waits between tiles)
//   k_rcolscan    per digit, the exclusive prefix of the per-tile counts plus the
//                 digit's global offset: where every tile's keys of that digit go
//   k_rscatter    one tile per block: rank the keys by digit, write them to their
//                 places, count the next pass's digits per destination tile
//   or, for a handle with a trained position model, the model-bucketed sort:
//   k_lprep       validate and compress as k_prep, route every key to its model
//                 piece (its bucket) and take its rank in the bucket; the last block
//                 turns the bucket counts into offsets
//   k_lscatter    every word to its bucket's offset plus its rank
//   k_lsort_warp  buckets of up to 512 words, one warp each, bitonic in registers
//   k_lsort       the larger buckets, a block each (shared memory, or in place)
//   then
//   k_rsearch     256 or 1024 sorted words per block: unique + insert/delete
//                 cancellation, the leaf search of every survivor (learned model when
//                 trained, else binary search; both give the same leaf), the block's
//                 survivor and run-head counts; the last block to finish turns them
//                 into every block's offsets
//   k_twrite      survivors and the heads of their runs of equal leaf to their places
//   k_small_front all of the above in one block for batches of at most
//                 kSmallBatch keys (bitonic sort in shared memory)
//   k_m_*         the same stages as one launch over many handles
#include "gpma_dev.cuh"
#include "gpma_launch.h"
#include "scan_dev.cuh"

namespace gpk {

constexpr int kSortThreads = 256;
// keys per thread of a sort tile (1024-key tiles: many small blocks resident at once)
constexpr int kSortItems = 4;
constexpr uint32_t kSortTile = kSortThreads * kSortItems;
// search and compaction: 256 threads a block, Q sorted words a thread (their leaf
// searches in lock step): Q = 4 from kSearchWideFrom keys on, else 1 (small
// batches need every thread they can get to hide the search latency)
constexpr uint32_t kSearchThreads = 256;
constexpr uint64_t kSearchWideFrom = 1ull << 19;
constexpr uint32_t kPrepDone = 7;       // Ctl::ticket slot counting finished prep blocks
constexpr uint32_t kSearchDone = 6;     // ... finished search blocks
constexpr uint32_t kLPrepDone = 5;      // ... finished blocks of the model-bucketed prep

// ---- key compression -----------------------------------------------------------------
// Graph mode: word = (src << db) | d with d = dst, or d = V for a guard (so a
// guard sorts after every edge of its row); db = bits(V) when guards may occur,
// else bits(V-1).  Raw mode: word = key.  The insert/delete tag rides in bit 63,
// outside the sorted digits: the sort is stable and inserts precede deletes in
// its input, so words of equal key keep inserts first.
constexpr uint64_t kTagBit = 1ull << 63;

__device__ __forceinline__ uint64_t compress(uint64_t key, uint32_t tag, const PrepArgs &a) {
  const uint64_t t = tag ? kTagBit : 0ull;
  if (a.raw) return key | t;
  uint64_t src = key >> 32, dst = key & 0xFFFFFFFFull;
  uint64_t d = (dst == 0xFFFFFFFFull) ? (uint64_t)a.V : dst;
  return ((src << a.db) | d) | t;
}

__device__ __forceinline__ uint64_t expand(uint64_t w, const PrepArgs &a) {
  w &= ~kTagBit;
  if (a.raw) return w;
  uint64_t d = w & ((1ull << a.db) - 1ull);
  uint64_t src = w >> a.db;
  uint64_t dst = (d == (uint64_t)a.V) ? 0xFFFFFFFFull : d;
  return (src << 32) | dst;
}

template <class Blk>
__device__ __forceinline__ void init_batch_body(const Blk &bk, Ctl *ctl, uint32_t *hist, uint32_t nhist, uint32_t n) {
  for (uint32_t i = threadIdx.x; i < nhist; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x == 0) {
    ctl->err = 0;
    ctl->n = n;
    ctl->epoch += kSlotsPerBatch;
    ctl->nesc = 0;
    ctl->nfail = 0;
    ctl->nlong = 0;
    ctl->nvlong = 0;
    ctl->resized = 0;
    ctl->m = ctl->nruns = ctl->npend = ctl->neruns = ctl->nsegs = ctl->nleafw = 0;
    for (int i = 0; i < 16; i++) ctl->ticket[i] = 0;
    ctl->n_inserted = ctl->n_deleted = 0;
    ctl->st_cov_touched = ctl->st_l0_only = ctl->st_empties = ctl->st_del_leaves = 0;
    ctl->lm_miss = 0;
    ctl->levels_climbed = 0;
    ctl->n_merged0 = 0;
    for (int i = 0; i < kMaxLv; i++) ctl->merges[i] = 0;
  }
}

__global__ void k_init_batch(Ctl *ctl, uint32_t *hist, uint32_t nhist, uint32_t n) {
  init_batch_body(GridIdx{}, ctl, hist, nhist, n);
}

// Sort tiles (blockDim * ITEMS keys) tile, tile + nblocks, ... of a block:
// validation, compression, each tile's first-pass digit counts (column-major:
// H0[d * T + tile]) and the batch's digit counts of every pass (hist[p * 256 + d]).
template <int ITEMS, class Blk>
__device__ __forceinline__ void prep_body(const Blk &bk, const PrepArgs &a, const uint64_t *__restrict__ ins,
                                          const uint64_t *__restrict__ del, uint64_t *__restrict__ out,
                                          uint32_t *__restrict__ hist, uint32_t *__restrict__ H0, uint32_t T,
                                          Ctl *ctl) {
  __shared__ uint32_t sh[8 * 256];
  const uint32_t n = a.n_ins + a.n_del;
  const uint32_t mask = (1u << a.dbits) - 1u;
  for (uint32_t tile = bk.x(); tile < T; tile += bk.n()) {
    for (uint32_t i = threadIdx.x; i < a.npass * 256u; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    bool bad = false;
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
      const uint32_t i = tile * (kSortThreads * ITEMS) + r * kSortThreads + threadIdx.x;
      if (i >= n) break;
      const uint32_t tag = i >= a.n_ins;
      const uint64_t key = tag ? del[i - a.n_ins] : ins[i];
      bool ok;
      if (a.raw) {
        ok = (key >> 63) == 0;
      } else {
        const uint64_t src = key >> 32, dst = key & 0xFFFFFFFFull;
        ok = src < a.V && (dst < a.V || (a.allow_guards && !tag && dst == 0xFFFFFFFFull));
      }
      bad |= !ok;
      const uint64_t w = ok ? compress(key, tag, a) : 0ull;
      out[i] = w;
      const uint64_t kw = w & ~kTagBit;
      for (uint32_t p = 0; p < a.npass; p++)
        atomicAdd(&sh[p * 256 + (uint32_t)((kw >> (p * a.dbits)) & mask)], 1u);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->err, kErrKey);
    for (uint32_t d = threadIdx.x; d <= mask; d += blockDim.x) H0[(uint64_t)d * T + tile] = sh[d];
    for (uint32_t i = threadIdx.x; i < a.npass * 256u; i += blockDim.x)
      if (sh[i]) atomicAdd(&hist[i], sh[i]);
    __syncthreads();
  }
  // the last block to finish turns the batch's digit counts of every pass into
  // digit offsets: hist[8 * 256 + p * 256 + d] = keys of pass p with a smaller digit
  __shared__ uint32_t s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&ctl->ticket[kPrepDone], 1u) == bk.n() - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const uint32_t w = threadIdx.x >> 5, lane = lane_id();
  for (uint32_t p = w; p < a.npass; p += blockDim.x >> 5) {  // one warp per pass
    uint32_t carry = 0;
    for (uint32_t c = 0; c < 256; c += 32) {
      const uint32_t v = __ldcg(&hist[p * 256 + c + lane]);
      const uint32_t inc = warp_incl_scan(v);
      hist[8 * 256 + p * 256 + c + lane] = carry + inc - v;
      carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
  }
}

template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_prep(PrepArgs a, const uint64_t *__restrict__ ins,
                                                       const uint64_t *__restrict__ del, uint64_t *__restrict__ out,
                                                       uint32_t *__restrict__ hist, uint32_t *__restrict__ H0,
                                                       uint32_t T, Ctl *ctl) {
  prep_body<ITEMS>(GridIdx{}, a, ins, del, out, hist, H0, T, ctl);
}

// Pass `pass`, digits d = block, block + nblocks, ... < radix: H[d * T + t] (keys
// of tile t with digit d) becomes the position of the tile's first such key: the
// digit's global offset (keys of smaller digits, from the batch histogram) plus the
// same digit's keys in earlier tiles.  Also zeroes the next pass's counts Hn (may be
// nullptr).
template <class Blk>
__device__ __forceinline__ void rcolscan_body(const Blk &bk, uint32_t *__restrict__ H, uint32_t *__restrict__ Hn,
                                              uint32_t T, const uint32_t *__restrict__ dbase, uint32_t radix,
                                              const Ctl *ctl) {
  __shared__ uint32_t wsum[33];
  if (ctl->err) return;
  for (uint32_t d = bk.x(); d < radix; d += bk.n()) {
    uint32_t carry = dbase[d];
    uint32_t *col = H + (uint64_t)d * T;
    constexpr uint32_t kPer = 8;
    for (uint32_t c = 0; c < T; c += 256 * kPer) {
      const uint32_t t0 = c + threadIdx.x * kPer;
      uint32_t v[kPer], loc = 0;
#pragma unroll
      for (uint32_t q = 0; q < kPer; q++) {
        v[q] = t0 + q < T ? col[t0 + q] : 0u;
        loc += v[q];
      }
      uint32_t total;
      uint32_t run = carry + block_excl_scan(loc, wsum, &total);
#pragma unroll
      for (uint32_t q = 0; q < kPer; q++) {
        if (t0 + q < T) col[t0 + q] = run;
        run += v[q];
      }
      carry += total;
    }
    if (Hn)
      for (uint32_t t = threadIdx.x; t < T; t += 256) Hn[(uint64_t)d * T + t] = 0;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_rcolscan(uint32_t *__restrict__ H, uint32_t *__restrict__ Hn, uint32_t T,
                                                  const uint32_t *__restrict__ dbase, const Ctl *ctl) {
  rcolscan_body(GridIdx{}, H, Hn, T, dbase, gridDim.x, ctl);
}

// One stable LSD pass over tile blockIdx.x (ITEMS rounds x 256 keys; warp w owns
// the contiguous sub-tile [w*32*ITEMS, (w+1)*32*ITEMS), so ranks inside a warp
// need no block barrier).  O[d * T + t]: where the tile's keys of digit d start.
// With Hn, every key also counts its next-pass digit in its destination tile.
template <int ITEMS, class Blk>
__device__ __forceinline__ void rscatter_body(const Blk &bk, const uint64_t *__restrict__ src,
                                              uint64_t *__restrict__ dst, const uint32_t *__restrict__ O,
                                              uint32_t *__restrict__ Hn, uint32_t T, uint32_t shift, uint32_t nshift,
                                              uint32_t dbits, const Ctl *ctl) {
  __shared__ uint32_t wcnt[kSortThreads / 32][256];
  __shared__ uint32_t gbase[256];
  __shared__ uint32_t ltile[256];  // digit totals of the tile, then their exclusive prefix
  __shared__ uint64_t skey[kSortThreads * ITEMS];
  if (ctl->err) return;
  const uint32_t n = ctl->n;
  const uint32_t w = threadIdx.x >> 5, lane = lane_id();
  const uint32_t radix = 1u << dbits, mask = radix - 1u;
  for (uint32_t tile = bk.x(); tile < T; tile += bk.n()) {
    for (uint32_t d = threadIdx.x; d < 256; d += kSortThreads) {
      for (int q = 0; q < kSortThreads / 32; q++) wcnt[q][d] = 0;
      gbase[d] = d < radix ? O[(uint64_t)d * T + tile] : 0u;
    }
    __syncthreads();
    const uint64_t base = (uint64_t)tile * (kSortThreads * ITEMS) + w * (ITEMS * 32);
    uint64_t key[ITEMS];
    uint32_t rank[ITEMS];
    uint32_t dig[ITEMS];
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
      const uint64_t idx = base + r * 32 + lane;
      const bool valid = idx < n;
      key[r] = valid ? src[idx] : 0ull;
      dig[r] = valid ? (uint32_t)(((key[r] & ~kTagBit) >> shift) & mask) : 0xFFFFu;
    }
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
      // lanes holding the same digit, from one ballot per digit bit (cheaper than match.any)
      uint32_t peers = 0xFFFFFFFFu;
      for (uint32_t b = 0; b < dbits; b++) {
        const bool bit = (dig[r] >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, bit);
        peers &= bit ? bal : ~bal;
      }
      {
        const bool inv = dig[r] == 0xFFFFu;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, inv);
        peers &= inv ? bal : ~bal;
      }
      uint32_t before = 0;
      if (dig[r] != 0xFFFFu) before = wcnt[w][dig[r]];
      rank[r] = before + __popc(peers & lanemask_lt());
      __syncwarp();
      if (dig[r] != 0xFFFFu && lane == (uint32_t)(__ffs(peers) - 1)) wcnt[w][dig[r]] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over the warps, and the tile's total
    for (uint32_t d = threadIdx.x; d < 256; d += kSortThreads) {
      uint32_t run = 0;
      for (int q = 0; q < kSortThreads / 32; q++) {
        const uint32_t c = wcnt[q][d];
        wcnt[q][d] = run;
        run += c;
      }
      ltile[d] = run;
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // digit offsets inside the tile
      uint32_t carry = 0;
      for (int c = 0; c < 256; c += 32) {
        const uint32_t v = ltile[c + lane];
        const uint32_t inc = warp_incl_scan(v);
        ltile[c + lane] = carry + inc - v;
        carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
      }
    }
    __syncthreads();
    // the tile sorted by digit in shared memory, then written out in digit runs
    // (consecutive keys of one digit go to consecutive addresses)
#pragma unroll
    for (int r = 0; r < ITEMS; r++)
      if (dig[r] != 0xFFFFu) skey[ltile[dig[r]] + wcnt[w][dig[r]] + rank[r]] = key[r];
    __syncthreads();
    const uint64_t t0 = (uint64_t)tile * (kSortThreads * ITEMS);
    const uint32_t cnt = t0 >= n ? 0u : (n - t0 < kSortThreads * ITEMS ? (uint32_t)(n - t0) : kSortThreads * ITEMS);
    for (uint32_t i0 = 0; i0 < cnt; i0 += kSortThreads) {
      const uint32_t i = i0 + threadIdx.x;
      uint32_t cell = 0xFFFFFFFFu;
      if (i < cnt) {
        const uint64_t k = skey[i];
        const uint32_t d = (uint32_t)(((k & ~kTagBit) >> shift) & mask);
        const uint32_t pos = gbase[d] + (i - ltile[d]);
        dst[pos] = k;
        cell = (uint32_t)(((k & ~kTagBit) >> nshift) & mask) * T + pos / (kSortThreads * ITEMS);
      }
      if (Hn) {
        // staged keys leave in order, so lanes of one warp often share a destination
        // tile and (for skewed keys) the next digit: one atomic per distinct cell
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, cell);
        if (cell != 0xFFFFFFFFu && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&Hn[cell], (uint32_t)__popc(peers));
      }
    }
    __syncthreads();
  }
}

template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_rscatter(const uint64_t *__restrict__ src,
                                                           uint64_t *__restrict__ dst, const uint32_t *__restrict__ O,
                                                           uint32_t *__restrict__ Hn, uint32_t T, uint32_t shift,
                                                           uint32_t nshift, uint32_t dbits, const Ctl *ctl) {
  rscatter_body<ITEMS>(GridIdx{}, src, dst, O, Hn, T, shift, nshift, dbits, ctl);
}

// ---- small batches: the whole front end in one block ---------------------------------------
// Sort word = (compressed key without tag) << 1 | tag.  Inserts (tag 0) order
// before deletes (tag 1) of the same key, and equal words are identical, so the
// sorted sequence equals the stable radix sort's.  Each thread owns `ipt`
// consecutive positions for the two compactions (survivors, run heads).

// Leaf search with a sampled first stage: S evenly spaced pivots F[i * stride]
// sit in shared memory, the non-empty ones compacted in order.  The last sampled
// pivot <= k and the first one > k bracket the answer (eff(lo - 1) <= k and
// eff(hi) > k), and search_first_above finishes inside that bracket, so the leaf
// equals leaf_search's.
__device__ __forceinline__ uint32_t sampled_leaf_search(const uint64_t *__restrict__ F, uint64_t nleaves,
                                                        const uint64_t *cv, const uint32_t *cpos, uint32_t cnt,
                                                        uint64_t k) {
  uint32_t a = 0, b = cnt;  // first compacted sample with value > k
  while (a < b) {
    const uint32_t mid = (a + b) >> 1;
    if (cv[mid] > k) b = mid; else a = mid + 1;
  }
  const uint64_t lo = a ? (uint64_t)cpos[a - 1] + 1 : 0;
  const uint64_t hi = a < cnt ? (uint64_t)cpos[a] : nleaves;
  const uint64_t p = search_first_above(F, lo, hi, k);
  return p ? (uint32_t)(p - 1) : 0u;
}

template <class Blk>
__device__ __forceinline__ void small_front_body(const Blk &bk, const PrepArgs &a, const uint64_t *__restrict__ ins,
                                                 const uint64_t *__restrict__ del, Ctl *ctl,
                                                 const uint64_t *__restrict__ F, uint64_t nleaves,
                                                 uint64_t *__restrict__ ukey, uint8_t *__restrict__ utag,
                                                 uint32_t *__restrict__ uleaf, uint32_t *__restrict__ run_start,
                                                 uint32_t *__restrict__ run_leaf, const ModelHead *mhead,
                                                 const Piece *__restrict__ mpieces, uint32_t P, uint32_t S) {
  extern __shared__ uint64_t sk[];           // P sort words
  uint64_t *sw = sk + P;                     // P survivor words
  uint64_t *cv = sw + P;                     // S compacted sampled pivots
  uint32_t *sleaf = (uint32_t *)(cv + S);    // P leaves of the survivors
  uint32_t *cpos = sleaf + P;                // S leaf indices of the compacted samples
  __shared__ uint32_t wsum[33];
  const uint32_t n = a.n_ins + a.n_del, t = threadIdx.x, nt = blockDim.x;
  const uint32_t ipt = (P + nt - 1) / nt, e0 = t * ipt;
  const uint32_t spt = (S + nt - 1) / nt, s0 = t * spt;
  const uint64_t stride = nleaves / S;
  if (t == 0) {
    ctl->err = 0;
    ctl->n = n;
    ctl->epoch += kSlotsPerBatch;
    ctl->nesc = ctl->nfail = ctl->nlong = ctl->nvlong = ctl->resized = 0;
    ctl->m = ctl->nruns = ctl->npend = ctl->neruns = ctl->nsegs = ctl->nleafw = 0;
    for (int i = 0; i < 16; i++) ctl->ticket[i] = 0;
    ctl->n_inserted = ctl->n_deleted = 0;
    ctl->st_cov_touched = ctl->st_l0_only = ctl->st_empties = ctl->st_del_leaves = 0;
    ctl->lm_miss = 0;
    ctl->levels_climbed = 0;
    ctl->n_merged0 = 0;
    for (int i = 0; i < kMaxLv; i++) ctl->merges[i] = 0;
  }
  bool bad = false;
  for (uint32_t i = t; i < P; i += nt) {
    uint64_t word = ~0ull;  // padding sorts last
    if (i < n) {
      const uint32_t tag = i >= a.n_ins;
      const uint64_t key = tag ? del[i - a.n_ins] : ins[i];
      bool ok;
      if (a.raw) {
        ok = (key >> 63) == 0;
      } else {
        const uint64_t src = key >> 32, dst = key & 0xFFFFFFFFull;
        ok = src < a.V && (dst < a.V || (a.allow_guards && !tag && dst == 0xFFFFFFFFull));
      }
      bad |= !ok;
      word = ok ? ((compress(key, 0, a) << 1) | tag) : 0ull;
    }
    sk[i] = word;
  }
  ModelHead hd;
  hd.valid = 0;
  if (mhead) hd = *mhead;
  const bool learned = hd.valid != 0;
  // sampled pivots (the stores land in cv; compacted in place below); a trained
  // model replaces them, so it skips the loads
  uint32_t nonempty = 0;
  for (uint32_t q = 0; q < spt && !learned; q++) {
    const uint32_t i = s0 + q;
    if (i >= S) break;
    const uint64_t f = __ldg(F + i * stride);
    cv[i] = f;
    nonempty += f != kEmpty;
  }
  if (__syncthreads_or(bad)) {
    if (t == 0) atomicOr(&ctl->err, kErrKey);
    return;  // nothing of the batch is applied
  }
  // bitonic sort, ascending
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = t; i < P / 2; i += nt) {
        const uint32_t lo = ((i & ~(j - 1)) << 1) | (i & (j - 1)), hi = lo + j;
        const uint64_t x = sk[lo], y = sk[hi];
        if ((x > y) == ((lo & k) == 0)) {
          sk[lo] = y;
          sk[hi] = x;
        }
      }
      __syncthreads();
    }
  }
  // compact the non-empty samples in order (read own values before the scan's barrier)
  uint64_t mine[8];
  for (uint32_t q = 0; q < spt && q < 8; q++) mine[q] = (!learned && s0 + q < S) ? cv[s0 + q] : kEmpty;
  uint32_t cnt;
  uint32_t co = block_excl_scan(nonempty, wsum, &cnt);
  for (uint32_t q = 0; q < spt && q < 8; q++) {
    if (mine[q] == kEmpty) continue;
    cv[co] = mine[q];
    cpos[co] = (uint32_t)((s0 + q) * stride);
    co++;
  }
  // unique + cancellation (reading R2) on positions [e0, e0 + ipt)
  uint32_t keep = 0;
  for (uint32_t q = 0; q < ipt; q++) {
    const uint32_t e = e0 + q;
    if (e >= n) break;
    const uint64_t k = sk[e] >> 1;
    const bool kept = (sk[e] & 1) ? (e == 0 || (sk[e - 1] >> 1) != k) : (e + 1 == n || (sk[e + 1] >> 1) != k);
    keep |= (uint32_t)kept << q;
  }
  uint32_t m;
  uint32_t off = block_excl_scan(__popc(keep), wsum, &m);
  for (uint32_t q = 0; q < ipt; q++)
    if ((keep >> q) & 1) sw[off++] = sk[e0 + q];
  __syncthreads();
  // the leaf of every survivor (reading R4), one survivor per thread at a time
  for (uint32_t e = t; e < m; e += nt) {
    const uint64_t w = sw[e];
    const uint64_t key = expand(w >> 1, a);
    const uint32_t leaf = learned ? learned_leaf_search(hd, mpieces, F, nleaves, key)
                                  : sampled_leaf_search(F, nleaves, cv, cpos, cnt, key);
    ukey[e] = key;
    utag[e] = (uint8_t)(w & 1);
    uleaf[e] = leaf;
    sleaf[e] = leaf;
  }
  __syncthreads();
  // run heads over the m survivors
  uint32_t head = 0;
  for (uint32_t q = 0; q < ipt; q++) {
    const uint32_t e = e0 + q;
    if (e >= m) break;
    head |= (uint32_t)(e == 0 || sleaf[e] != sleaf[e - 1]) << q;
  }
  uint32_t nr;
  uint32_t ro = block_excl_scan(__popc(head), wsum, &nr);
  for (uint32_t q = 0; q < ipt; q++) {
    if (!((head >> q) & 1)) continue;
    run_start[ro] = e0 + q;
    run_leaf[ro] = sleaf[e0 + q];
    ro++;
  }
  if (t == 0) {
    ctl->m = m;
    ctl->nruns = nr;
    run_start[nr] = m;
  }
}

__global__ void __launch_bounds__(1024) k_small_front(PrepArgs a, const uint64_t *__restrict__ ins,
                                                      const uint64_t *__restrict__ del, Ctl *ctl,
                                                      const uint64_t *__restrict__ F, uint64_t nleaves,
                                                      uint64_t *__restrict__ ukey, uint8_t *__restrict__ utag,
                                                      uint32_t *__restrict__ uleaf, uint32_t *__restrict__ run_start,
                                                      uint32_t *__restrict__ run_leaf, const ModelHead *mhead,
                                                      const Piece *__restrict__ mpieces, uint32_t P, uint32_t S) {
  small_front_body(GridIdx{}, a, ins, del, ctl, F, nleaves, ukey, utag, uleaf, run_start, run_leaf, mhead, mpieces, P,
                   S);
}

// ---- unique/cancel, leaf search, run heads and compaction (after the radix passes) ------------
// Per-block survivor summaries of the sorted words (256 Q words a block).
struct TileSums {
  uint32_t *surv;    // survivors of reading R2 in the block
  uint32_t *hin;     // run heads among them, not counting the block's first survivor
  uint32_t *first;   // leaf of the block's first / last survivor (kNoLeaf: none)
  uint32_t *last;
  uint32_t *soff;    // survivors before the block
  uint32_t *hoff;    // run heads before the block
  uint32_t *hfirst;  // 1 if the block's first survivor starts a run
};

// Q consecutive sorted words per thread: the survivor test of reading R2
// (an insert survives unless the next word has its key, a delete unless the
// previous one has), the leaf of every survivor (reading R4), and the block's
// summary.
template <int Q, class Blk>
__device__ __forceinline__ void rsearch_body(const Blk &bk, const PrepArgs &a, const uint64_t *__restrict__ sorted,
                                             uint32_t *__restrict__ lfull, const uint64_t *__restrict__ F,
                                             uint64_t nleaves, const TileSums &ts, uint32_t ntiles, Ctl *ctl,
                                             const ModelHead *mhead, const Piece *__restrict__ mpieces,
                                             const uint16_t *__restrict__ spiece) {
  __shared__ uint32_t sl[(kSearchThreads * Q)];
  __shared__ uint32_t s_surv, s_hin, s_first, s_last;
  if (ctl->err) return;
  const uint32_t n = ctl->n, t = threadIdx.x;
  for (uint32_t tile = bk.x(); tile < ntiles; tile += bk.n()) {
    const uint32_t e0 = tile * (kSearchThreads * Q) + t * Q;
    if (t == 0) {
      s_surv = 0;
      s_hin = 0;
      s_first = 0xFFFFFFFFu;
      s_last = 0;
    }
    ModelHead hd;
    hd.valid = 0;
    if (mhead) hd = *mhead;
    uint64_t w[Q + 2];  // words e0 - 1 .. e0 + Q
#pragma unroll
    for (int q = 0; q < Q + 2; q++) {
      const int64_t e = (int64_t)e0 - 1 + q;
      w[q] = (e >= 0 && e < (int64_t)n) ? sorted[e] : kEmpty;
    }
    uint64_t key[Q];
    bool kept[Q];
    uint32_t leaf[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const uint32_t e = e0 + q;
      const uint64_t wq = w[q + 1], kq = wq & ~kTagBit;
      kept[q] = e < n && ((wq & kTagBit) ? (e == 0 || (w[q] & ~kTagBit) != kq)
                                         : (e + 1 == n || (w[q + 2] & ~kTagBit) != kq));
      key[q] = kept[q] ? expand(wq, a) : 0ull;
    }
    uint32_t miss = 0;
    if (hd.valid && spiece) {  // sorted by model piece: each word's bucket is known
      uint16_t pb[Q];
#pragma unroll
      for (int q = 0; q < Q; q++) pb[q] = e0 + q < n ? spiece[e0 + q] : (uint16_t)0;
      miss = learned_search_lockstep<Q>(hd, mpieces, F, nleaves, key, kept, leaf, pb);
    } else if (hd.valid) {
      miss = learned_search_lockstep<Q>(hd, mpieces, F, nleaves, key, kept, leaf);
    } else {
      leaf_search_lockstep<Q>(F, nleaves, key, kept, leaf);
    }
#pragma unroll
    for (int q = 0; q < Q; q++)
      if (!kept[q]) leaf[q] = kNoLeaf;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      if (e0 + q < n) lfull[e0 + q] = leaf[q];
      sl[t * Q + q] = leaf[q];
    }
    __syncthreads();
    uint32_t hin = 0, surv = 0;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      if (leaf[q] == kNoLeaf) continue;
      const uint32_t i = t * Q + q;
      ++surv;
      int32_t j = (int32_t)i - 1;  // previous survivor of the block (dropped words are rare)
      while (j >= 0 && sl[j] == kNoLeaf) --j;
      if (j < 0) s_first = i;  // exactly one survivor has none before it
      else hin += sl[j] != leaf[q];
      atomicMax(&s_last, i);
    }
    surv = warp_sum(surv);
    hin = warp_sum(hin);
    miss = warp_sum(miss);
    if (lane_id() == 0) {
      if (surv) atomicAdd(&s_surv, surv);
      if (hin) atomicAdd(&s_hin, hin);
      if (miss) atomicAdd(&ctl->lm_miss, miss);
    }
    __syncthreads();
    if (t == 0) {
      ts.surv[tile] = s_surv;
      ts.hin[tile] = s_hin;
      ts.first[tile] = s_surv ? sl[s_first] : kNoLeaf;
      ts.last[tile] = s_surv ? sl[s_last] : kNoLeaf;
    }
    __syncthreads();
  }
}


// Survivor and run-head offsets of every block of k_rsearch: exclusive scans over
// the blocks; a block's first survivor starts a run unless the last survivor of
// the nearest earlier block with survivors has the same leaf.  One block of 1024.
template <class Blk>
__device__ __forceinline__ void toffsets_body(const Blk &bk, const TileSums &ts, uint32_t nt, Ctl *ctl,
                                              uint32_t *__restrict__ run_start) {
  __shared__ uint32_t wsum[33];
  __shared__ uint32_t s_last[1024];  // last survivor leaf of each thread's blocks
  __shared__ int32_t s_idx[1024];    // nearest thread <= t whose blocks hold a survivor, -1 if none
  __shared__ int32_t s_wmax[32];
  if (ctl->err) return;
  const uint32_t t = threadIdx.x, per = (nt + blockDim.x - 1) / blockDim.x, b0 = t * per;
  const uint32_t nw = blockDim.x >> 5;
  uint32_t sv = 0, lastleaf = kNoLeaf;
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t b = b0 + q;
    if (b >= nt) break;
    const uint32_t c = __ldcg(ts.surv + b);  // written by other blocks (L2, not this block's L1)
    if (c) {
      sv += c;
      lastleaf = __ldcg(ts.last + b);
    }
  }
  s_last[t] = lastleaf;
  // inclusive running maximum of (t if its blocks hold survivors, else -1)
  const uint32_t lane = lane_id(), wid = t >> 5;
  int32_t v = sv ? (int32_t)t : -1;
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v = u > v ? u : v;
  }
  if (lane == 31) s_wmax[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int32_t x = lane < nw ? s_wmax[lane] : -1;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x = u > x ? u : x;
    }
    s_wmax[lane] = x;
  }
  __syncthreads();
  if (wid) v = s_wmax[wid - 1] > v ? s_wmax[wid - 1] : v;
  s_idx[t] = v;
  __syncthreads();
  const int32_t pt = t ? s_idx[t - 1] : -1;
  uint32_t prevleaf = pt >= 0 ? s_last[pt] : kNoLeaf;
  uint32_t hc = 0;
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t b = b0 + q;
    if (b >= nt) break;
    if (!__ldcg(ts.surv + b)) continue;
    const uint32_t hf = (prevleaf == kNoLeaf || prevleaf != __ldcg(ts.first + b)) ? 1u : 0u;
    ts.hfirst[b] = hf;
    hc += __ldcg(ts.hin + b) + hf;
    prevleaf = __ldcg(ts.last + b);
  }
  uint32_t m, nr;
  uint32_t so = block_excl_scan(sv, wsum, &m);
  uint32_t ho = block_excl_scan(hc, wsum, &nr);
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t b = b0 + q;
    if (b >= nt) break;
    ts.soff[b] = so;
    ts.hoff[b] = ho;
    const uint32_t c = __ldcg(ts.surv + b);
    if (c) {
      so += c;
      ho += __ldcg(ts.hin + b) + ts.hfirst[b];
    }
  }
  if (t == 0) {
    ctl->m = m;
    ctl->nruns = nr;
    run_start[nr] = m;
  }
}

// Unique/cancel, leaf search and block summaries (rsearch_body); the last block to
// finish then computes every block's survivor and run-head offsets (toffsets_body,
// without a launch of its own).
template <int Q>
__global__ void __launch_bounds__(kSearchThreads) k_rsearch(PrepArgs a, const uint64_t *__restrict__ sorted,
                                                            uint32_t *__restrict__ lfull,
                                                            const uint64_t *__restrict__ F, uint64_t nleaves,
                                                            TileSums ts, Ctl *ctl, const ModelHead *mhead,
                                                            const Piece *__restrict__ mpieces,
                                                            const uint16_t *__restrict__ spiece,
                                                            uint32_t *__restrict__ run_start) {
  __shared__ uint32_t s_done;
  rsearch_body<Q>(GridIdx{}, a, sorted, lfull, F, nleaves, ts, gridDim.x, ctl, mhead, mpieces, spiece);
  if (ctl->err) return;  // the same for every block: nothing of the batch is applied
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_done = atomicAdd(&ctl->ticket[kSearchDone], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_done) return;
  __threadfence();
  toffsets_body(GridIdx{}, ts, gridDim.x, ctl, run_start);
}

// survivors and run heads of every block to their places, Q words per thread
template <int Q, class Blk>
__device__ __forceinline__ void twrite_body(const Blk &bk, const PrepArgs &a, const uint64_t *__restrict__ sorted,
                                            const uint32_t *__restrict__ lfull, const TileSums &ts, uint32_t ntiles,
                                            uint64_t *__restrict__ ukey, uint8_t *__restrict__ utag,
                                            uint32_t *__restrict__ uleaf, uint32_t *__restrict__ run_start,
                                            uint32_t *__restrict__ run_leaf, const Ctl *ctl) {
  __shared__ uint32_t wsum[33];
  __shared__ uint32_t sl[(kSearchThreads * Q)];
  if (ctl->err) return;
  const uint32_t t = threadIdx.x, n = ctl->n;
  for (uint32_t b = bk.x(); b < ntiles; b += bk.n()) {
    if (ts.surv[b] == 0) continue;  // the same for the whole block
    const uint32_t base = b * (kSearchThreads * Q);
    for (uint32_t i = t; i < (kSearchThreads * Q); i += kSearchThreads)
      sl[i] = base + i < n ? lfull[base + i] : kNoLeaf;
    __syncthreads();
    uint32_t keep = 0, head = 0;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const uint32_t i = t * Q + q, lf = sl[i];
      if (lf == kNoLeaf) continue;
      keep |= 1u << q;
      int32_t j = (int32_t)i - 1;  // previous survivor of the block
      while (j >= 0 && sl[j] == kNoLeaf) --j;
      if (j < 0 ? ts.hfirst[b] != 0 : sl[j] != lf) head |= 1u << q;
    }
    uint32_t nk, nh;
    uint32_t ko = ts.soff[b] + block_excl_scan(__popc(keep), wsum, &nk);
    uint32_t ho = ts.hoff[b] + block_excl_scan(__popc(head), wsum, &nh);
#pragma unroll
    for (int q = 0; q < Q; q++) {
      if (!((keep >> q) & 1u)) continue;
      const uint32_t i = t * Q + q;
      const uint64_t w = sorted[base + i];
      ukey[ko] = expand(w, a);
      utag[ko] = (uint8_t)(w >> 63);
      uleaf[ko] = sl[i];
      if ((head >> q) & 1u) {
        run_start[ho] = ko;
        run_leaf[ho] = sl[i];
        ++ho;
      }
      ++ko;
    }
    __syncthreads();
  }
}

template <int Q>
__global__ void __launch_bounds__(kSearchThreads) k_twrite(PrepArgs a, const uint64_t *__restrict__ sorted,
                                                           const uint32_t *__restrict__ lfull, TileSums ts,
                                                           uint64_t *__restrict__ ukey, uint8_t *__restrict__ utag,
                                                           uint32_t *__restrict__ uleaf,
                                                           uint32_t *__restrict__ run_start,
                                                           uint32_t *__restrict__ run_leaf, const Ctl *ctl) {
  twrite_body<Q>(GridIdx{}, a, sorted, lfull, ts, gridDim.x, ukey, utag, uleaf, run_start, run_leaf, ctl);
}

// ---- model-bucketed front end (learned handles) ----------------------------------------------
// The model's pieces split the keys into kPieces ordered ranges whose sizes follow
// the array's own key distribution: bucket(k) = the last piece whose boundary is
// <= k, a non-decreasing function of k.  Bucketing the batch by piece and sorting
// every bucket therefore sorts the batch, in one scatter instead of the radix
// passes.  Equal keys keep inserts before deletes (the bucket sort compares
// (key, tag)), so the sorted words equal the stable radix sort's.  Before the model
// is trained the bucket is the top bits of the compressed key, also non-decreasing.

// (key, tag) order of a sort word (tag in bit 63, at most 62 key bits)
__device__ __forceinline__ uint64_t word_order(uint64_t w) { return ((w & ~kTagBit) << 1) | (w >> 63); }

// validation and compression as in k_prep, the bucket of every key, and its rank
// among the keys of its bucket (the order of those ranks is arbitrary: the bucket
// is sorted afterwards); the last block turns the bucket counts into offsets.
// BLOCK_RANKS: ranks in two levels (shared-memory atomics inside the block, one
// global atomic per bucket the block touches) for large batches, where each block's
// keys fill many buckets; else one global atomic per key (measured, serialised:
// 33 against 38 us at 1e6 keys, 19 against 14 us at 1e5)
template <int ITEMS, bool BLOCK_RANKS>
__global__ void __launch_bounds__(kSortThreads) k_lprep(PrepArgs a, const uint64_t *__restrict__ ins,
                                                        const uint64_t *__restrict__ del, uint64_t *__restrict__ out,
                                                        uint16_t *__restrict__ bkt, uint32_t *__restrict__ rank,
                                                        uint32_t *__restrict__ cnt, Ctl *ctl,
                                                        const ModelHead *mhead, const Piece *__restrict__ mpieces) {
  const ModelHead hd = *mhead;
  const uint32_t top = a.sbits > 12 ? a.sbits - 12 : 0;  // key-bit buckets: kPieces = 2^12
  const uint32_t n = a.n_ins + a.n_del;
  uint64_t key[ITEMS], w[ITEMS];
  bool act[ITEMS];
  bool bad = false;
#pragma unroll
  for (int r = 0; r < ITEMS; r++) {
    const uint32_t i = blockIdx.x * (kSortThreads * ITEMS) + r * kSortThreads + threadIdx.x;
    act[r] = false;
    key[r] = 0;
    w[r] = 0;
    if (i >= n) continue;
    const uint32_t tag = i >= a.n_ins;
    key[r] = tag ? del[i - a.n_ins] : ins[i];
    const uint64_t src = key[r] >> 32, dst = key[r] & 0xFFFFFFFFull;
    const bool ok = src < a.V && dst < a.V;
    bad |= !ok;
    w[r] = ok ? compress(key[r], tag, a) : 0ull;
    out[i] = w[r];
    act[r] = ok;
  }
  uint32_t b[ITEMS];
  if (hd.valid) {
    model_route_lockstep<ITEMS>(hd, mpieces, key, act, b);
  } else {
#pragma unroll
    for (int r = 0; r < ITEMS; r++) b[r] = (uint32_t)((w[r] & ~kTagBit) >> top);
  }
  if (BLOCK_RANKS) {
    // inside the block by shared-memory atomics, then one global atomic per bucket
    // the block touches claims the block's range of that bucket
    __shared__ uint32_t s_cnt[kPieces];
    for (uint32_t q = threadIdx.x; q < kPieces; q += kSortThreads) s_cnt[q] = 0;
    __syncthreads();
    uint32_t lr[ITEMS];
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
      const uint32_t i = blockIdx.x * (kSortThreads * ITEMS) + r * kSortThreads + threadIdx.x;
      lr[r] = i < n ? atomicAdd(&s_cnt[b[r]], 1u) : 0u;
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < kPieces; q += kSortThreads) {
      const uint32_t c = s_cnt[q];
      if (c) s_cnt[q] = atomicAdd(&cnt[q], c);  // the block's first rank in bucket q
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
      const uint32_t i = blockIdx.x * (kSortThreads * ITEMS) + r * kSortThreads + threadIdx.x;
      if (i >= n) continue;
      bkt[i] = (uint16_t)b[r];
      rank[i] = s_cnt[b[r]] + lr[r];
    }
  } else {
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
      const uint32_t i = blockIdx.x * (kSortThreads * ITEMS) + r * kSortThreads + threadIdx.x;
      if (i >= n) continue;
      bkt[i] = (uint16_t)b[r];
      rank[i] = atomicAdd(&cnt[b[r]], 1u);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->err, kErrKey);
  // the last block to finish turns the counts into offsets (cnt[kPieces] = all keys)
  __shared__ uint32_t s_done;
  __shared__ uint32_t wsum[33];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_done = atomicAdd(&ctl->ticket[kLPrepDone], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_done) return;
  __threadfence();
  constexpr uint32_t kPer = kPieces / kSortThreads;
  const uint32_t t = threadIdx.x;
  uint32_t v[kPer], loc = 0;
#pragma unroll
  for (uint32_t q = 0; q < kPer; q++) {
    v[q] = __ldcg(cnt + t * kPer + q);
    loc += v[q];
  }
  uint32_t total;
  uint32_t run = block_excl_scan(loc, wsum, &total);
#pragma unroll
  for (uint32_t q = 0; q < kPer; q++) {
    cnt[t * kPer + q] = run;
    run += v[q];
  }
  if (t == 0) cnt[kPieces] = total;
}

// every word to its bucket's offset plus its rank
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_lscatter(const uint64_t *__restrict__ src,
                                                           const uint16_t *__restrict__ bkt,
                                                           const uint32_t *__restrict__ rank,
                                                           const uint32_t *__restrict__ off,
                                                           uint64_t *__restrict__ dst, Ctl *ctl) {
  if (ctl->err) return;
  const uint32_t n = ctl->n;
#pragma unroll
  for (int r = 0; r < ITEMS; r++) {
    const uint32_t i = blockIdx.x * (kSortThreads * ITEMS) + r * kSortThreads + threadIdx.x;
    if (i >= n) break;
    const uint32_t b = bkt[i];
    const uint32_t pos = b < kPieces ? off[b] + rank[i] : n;
    if (pos < n) dst[pos] = src[i];
    else atomicOr(&ctl->err, kErrInternal);  // cannot happen when the counts are consistent
  }
}

// Buckets of up to kLWarpMax words: one warp per bucket (eight a block). The warp
// holds the bucket padded to P = 32 E words, E consecutive words a lane (moved there
// through the warp's shared memory, so that the global loads and stores stay
// coalesced), and runs the bitonic network on registers: comparators inside a lane's
// E words directly, the others against the partner lane by shuffles, with no shared
// memory and no synchronisation inside the network.
constexpr uint32_t kLWarpMax = 512;
constexpr uint32_t kLWarpPad = kLWarpMax + kLWarpMax / 16;  // word i at i + i / E (E <= 16)

__device__ __forceinline__ uint64_t word_unorder(uint64_t sw) { return (sw >> 1) | ((sw & 1ull) << 63); }

template <uint32_t E>
__device__ __forceinline__ void lsort_warp_regs(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst,
                                                uint32_t nb, uint64_t *s, uint32_t lane) {
  constexpr uint32_t P = 32u * E;
  // the padding puts both the striped (32 r + lane) and the blocked (E lane + r) index
  // of one access on distinct bank pairs within each half warp (up to a 2-way overlap)
  uint64_t v[E];
  if (E == 1) {
    v[0] = lane < nb ? word_order(src[lane]) : ~0ull;  // padding sorts last
  } else {
#pragma unroll
    for (uint32_t r = 0; r < E; r++) {
      const uint32_t i = 32u * r + lane;
      s[i + i / E] = i < nb ? word_order(src[i]) : ~0ull;
    }
    __syncwarp();
#pragma unroll
    for (uint32_t r = 0; r < E; r++) {
      const uint32_t i = E * lane + r;
      v[r] = s[i + i / E];
    }
  }
  // element e = E lane + r; merge size k, stride j; of the pair (e, e ^ j) the element
  // with (e & j) == 0 keeps the smaller word when (e & k) == 0, else the larger
  for (uint32_t k = 2; k <= P; k <<= 1) {
    const bool asc_lane = ((E * lane) & k) == 0;
    for (uint32_t j = k >> 1; j >= E; j >>= 1) {  // partner in lane ^ (j / E), same r
      const uint32_t lm = j / E;
      const bool keep_min = ((lane & lm) == 0) == asc_lane;  // here k >= 2E: r adds no bit of k
#pragma unroll
      for (uint32_t r = 0; r < E; r++) {
        const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, v[r], lm);
        const bool less = o < v[r];
        v[r] = (less == keep_min) ? o : v[r];
      }
    }
#pragma unroll
    for (uint32_t j = E / 2; j > 0; j >>= 1) {  // partner r ^ j in the same lane
      if (j >= k) continue;
#pragma unroll
      for (uint32_t r = 0; r < E; r++) {
        if (r & j) continue;
        const bool asc = asc_lane && (r & k) == 0;
        const uint64_t x = v[r], y = v[r | j];
        const bool sw = (x > y) == asc;
        v[r] = sw ? y : x;
        v[r | j] = sw ? x : y;
      }
    }
  }
  if (E == 1) {
    if (lane < nb) dst[lane] = word_unorder(v[0]);
  } else {
    __syncwarp();  // every lane has read its words before they are overwritten
#pragma unroll
    for (uint32_t r = 0; r < E; r++) {
      const uint32_t i = E * lane + r;
      s[i + i / E] = v[r];
    }
    __syncwarp();
#pragma unroll
    for (uint32_t r = 0; r < E; r++) {
      const uint32_t i = 32u * r + lane;
      if (i < nb) dst[i] = word_unorder(s[i + i / E]);
    }
  }
}

__global__ void __launch_bounds__(256) k_lsort_warp(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst,
                                                    const uint32_t *__restrict__ off, uint16_t *__restrict__ spiece,
                                                    Ctl *ctl) {
  __shared__ uint64_t sk[8][kLWarpPad];
  if (ctl->err) return;
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  const uint32_t bucket = blockIdx.x * 8 + w;
  const uint32_t o0 = off[bucket], nb = off[bucket + 1] - o0;
  if (nb == 0 || nb > kLWarpMax) return;  // larger buckets: k_lsort
  if (o0 + nb > ctl->n) {                  // cannot happen: the offsets count the batch's words
    if (lane == 0) atomicOr(&ctl->err, kErrInternal);
    return;
  }
  for (uint32_t i = lane; i < nb; i += 32) spiece[o0 + i] = (uint16_t)bucket;  // for the leaf search
  const uint64_t *in = src + o0;
  uint64_t *out = dst + o0;
  if (nb <= 32) lsort_warp_regs<1>(in, out, nb, sk[w], lane);
  else if (nb <= 64) lsort_warp_regs<2>(in, out, nb, sk[w], lane);
  else if (nb <= 128) lsort_warp_regs<4>(in, out, nb, sk[w], lane);
  else if (nb <= 256) lsort_warp_regs<8>(in, out, nb, sk[w], lane);
  else lsort_warp_regs<16>(in, out, nb, sk[w], lane);
}

// Buckets above kLWarpMax words, a block per bucket (the grid strides over the
// buckets, most of which the warp sort has taken): bitonic sort in shared memory up
// to kLSortMax words; a larger bucket (many new edges of one row, or key-bit buckets)
// in place in dst with the bitonic network whose comparators all put the smaller word
// first, positions past the bucket counting as +infinity (so a comparator that reaches
// past it does nothing).
__global__ void __launch_bounds__(256) k_lsort(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst,
                                               const uint32_t *__restrict__ off, uint16_t *__restrict__ spiece,
                                               Ctl *ctl) {
  __shared__ uint64_t sk[kLSortMax];
  if (ctl->err) return;
  const uint32_t t = threadIdx.x, nt = blockDim.x;
  for (uint32_t bucket = blockIdx.x; bucket < kPieces; bucket += gridDim.x) {
    const uint32_t o0 = off[bucket], nb = off[bucket + 1] - o0;
    if (nb <= kLWarpMax) continue;  // sorted by k_lsort_warp
    if (o0 + nb > ctl->n) {         // cannot happen: the offsets count the batch's words
      if (t == 0) atomicOr(&ctl->err, kErrInternal);
      return;
    }
    for (uint32_t i = t; i < nb; i += nt) spiece[o0 + i] = (uint16_t)bucket;  // for the leaf search
    uint32_t P = 1;
    while (P < nb) P <<= 1;
    if (nb <= kLSortMax) {
      for (uint32_t i = t; i < P; i += nt) sk[i] = i < nb ? word_order(src[o0 + i]) : ~0ull;  // padding sorts last
      __syncthreads();
      for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
          for (uint32_t i = t; i < P / 2; i += nt) {
            const uint32_t lo = ((i & ~(j - 1)) << 1) | (i & (j - 1)), hi = lo + j;
            const uint64_t x = sk[lo], y = sk[hi];
            if ((x > y) == ((lo & k) == 0)) {
              sk[lo] = y;
              sk[hi] = x;
            }
          }
          __syncthreads();
        }
      }
      for (uint32_t i = t; i < nb; i += nt) dst[o0 + i] = word_unorder(sk[i]);
      __syncthreads();  // the next bucket overwrites sk
      continue;
    }
    uint64_t *d = dst + o0;
    if (src != dst)
      for (uint32_t i = t; i < nb; i += nt) d[i] = src[o0 + i];
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t i = t; i < P / 2; i += nt) {
          uint32_t lo, hi;
          if (j == (k >> 1)) {  // first step of a merge: mirror inside the block of k
            lo = (i / j) * k + (i % j);
            hi = (i / j) * k + k - 1 - (i % j);
          } else {
            lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
            hi = lo + j;
          }
          if (hi < nb) {
            const uint64_t x = d[lo], y = d[hi];
            if (word_order(x) > word_order(y)) {
              d[lo] = y;
              d[hi] = x;
            }
          }
        }
        __syncthreads();
      }
    }
  }
}

// ---- host launchers ----------------------------------------------------------------------
static uint32_t grid_for(uint64_t n, uint32_t per_block, uint32_t cap) {
  uint64_t g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (uint32_t)g;
}

uint32_t comp_tiles(uint64_t n) { return (uint32_t)((n + kScanTile - 1) / kScanTile); }

bool small_front(uint64_t n) { return n <= kSmallBatch; }

void launch_small_front(const FrontArgs &f, cudaStream_t s) {
  const PrepArgs &a = f.prep;
  const uint32_t n = a.n_ins + a.n_del;
  constexpr uint32_t kSamples = 2048;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_small_front, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kSmallBatch * 20 + kSamples * 12);
    attr = true;
  }
  uint32_t P = 64;
  while (P < n) P <<= 1;
  const uint32_t nt = P >= 2048 ? 1024 : 256;  // at most 4 positions and 8 samples per thread
  const uint64_t nl = f.geo->nleaves;
  const uint32_t S = nl < kSamples ? (uint32_t)nl : kSamples;  // nleaves is a power of two
  note_launch();
  k_small_front<<<1, nt, P * 20 + S * 12, s>>>(a, f.ins, f.del, f.ctl, f.geo->F, nl, f.ukey, f.utag, f.uleaf,
                                               f.run_start, f.run_leaf, f.mhead, f.mpieces, P, S);
}

uint32_t front_tiles(uint64_t nb) { return (uint32_t)((nb + kSortTile - 1) / kSortTile); }
static uint32_t search_per(uint64_t nb) { return nb >= kSearchWideFrom ? 4u : 1u; }
uint32_t search_tiles(uint64_t nb) {
  const uint64_t tile = (uint64_t)kSearchThreads * search_per(nb);
  return (uint32_t)((nb + tile - 1) / tile);
}

void launch_prep(const FrontArgs &f, uint64_t nb, cudaStream_t s) {
  const PrepArgs &a = f.prep;
  const uint64_t n = (uint64_t)a.n_ins + a.n_del;
  const uint32_t T = front_tiles(nb);
  note_launch();
  k_init_batch<<<1, 256, 0, s>>>(f.ctl, f.hist, a.npass * 256u, (uint32_t)n);
  note_launch();
  k_prep<kSortItems><<<T, kSortThreads, 0, s>>>(a, f.ins, f.del, f.bufA, f.hist, f.rs, T, f.ctl);
}

// the words after the radix passes (bufA for an even pass count, else bufB)
static uint64_t *sorted_words(const FrontArgs &f) { return (f.prep.npass & 1) ? f.bufB : f.bufA; }

void launch_front_radix(const FrontArgs &f, uint64_t nb, cudaStream_t s) {
  const PrepArgs &a = f.prep;
  const uint32_t T = front_tiles(nb), radix = 1u << a.dbits;
  uint32_t *H[2] = {f.rs, f.rs + (uint64_t)256 * T};
  uint64_t *src = f.bufA, *dst = f.bufB;
  for (uint32_t p = 0; p < a.npass; p++) {
    uint32_t *O = H[p & 1], *Hn = p + 1 < a.npass ? H[(p + 1) & 1] : nullptr;
    note_launch();
    k_rcolscan<<<radix, 256, 0, s>>>(O, Hn, T, f.hist + 8 * 256 + p * 256, f.ctl);
    const uint32_t shift = p * a.dbits, nshift = (p + 1) * a.dbits;
    note_launch();
    k_rscatter<kSortItems><<<T, kSortThreads, 0, s>>>(src, dst, O, Hn, T, shift, nshift, a.dbits, f.ctl);
    uint64_t *t = src; src = dst; dst = t;
  }
}

void launch_front_search(const FrontArgs &f, uint64_t nb, cudaStream_t s, const uint16_t *spiece) {
  const PrepArgs &a = f.prep;
  const uint32_t T = front_tiles(nb);
  const uint64_t *src = sorted_words(f);
  const uint32_t T1 = search_tiles(nb);
  uint32_t *q = f.rs + (uint64_t)512 * T;
  const uint32_t K = T1 + 1;
  TileSums ts{q, q + K, q + 2 * K, q + 3 * K, q + 4 * K, q + 5 * K, q + 6 * K};
  const bool wide = search_per(nb) == 4;
  note_launch();
  if (wide)
    k_rsearch<4><<<T1, kSearchThreads, 0, s>>>(a, src, f.lfull, f.geo->F, f.geo->nleaves, ts, f.ctl, f.mhead,
                                               f.mpieces, spiece, f.run_start);
  else
    k_rsearch<1><<<T1, kSearchThreads, 0, s>>>(a, src, f.lfull, f.geo->F, f.geo->nleaves, ts, f.ctl, f.mhead,
                                               f.mpieces, spiece, f.run_start);
  note_launch();
  if (wide)
    k_twrite<4><<<T1, kSearchThreads, 0, s>>>(a, src, f.lfull, ts, f.ukey, f.utag, f.uleaf, f.run_start,
                                              f.run_leaf, f.ctl);
  else
    k_twrite<1><<<T1, kSearchThreads, 0, s>>>(a, src, f.lfull, ts, f.ukey, f.utag, f.uleaf, f.run_start,
                                              f.run_leaf, f.ctl);
}

void launch_front(const FrontArgs &f, uint64_t nb, cudaStream_t s) {
  launch_front_radix(f, nb, s);
  launch_front_search(f, nb, s);
}

// sorted (key, tag) words need one bit more than the key: graph batches only
// (no guards, so at most 62 sorted bits), with a model, above the one-block size
bool learned_front(const PrepArgs &a, bool has_model, uint64_t n) {
  return !a.raw && !a.allow_guards && has_model && a.sbits <= 62 && !small_front(n);
}

void launch_lprep(const FrontArgs &f, uint16_t *bkt, uint32_t *rank, uint32_t *cnt, uint64_t nb, cudaStream_t s) {
  const PrepArgs &a = f.prep;
  const uint64_t n = (uint64_t)a.n_ins + a.n_del;
  cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (kPieces + 1), s);
  note_launch();
  k_init_batch<<<1, 256, 0, s>>>(f.ctl, f.hist, a.npass * 256u, (uint32_t)n);
  note_launch();
  if (n >= kSearchWideFrom)
    k_lprep<kSortItems, true><<<front_tiles(nb), kSortThreads, 0, s>>>(a, f.ins, f.del, f.bufA, bkt, rank, cnt,
                                                                        f.ctl, f.mhead, f.mpieces);
  else
    k_lprep<kSortItems, false><<<front_tiles(nb), kSortThreads, 0, s>>>(a, f.ins, f.del, f.bufA, bkt, rank, cnt,
                                                                         f.ctl, f.mhead, f.mpieces);
}

// seven blocks of k_lsort fit an SM (32 KB of shared memory each)
static uint32_t lsort_blocks() {
  static uint32_t nblk = 0;
  if (!nblk) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    nblk = sms > 0 ? 7u * (uint32_t)sms : 1024u;
    if (nblk > kPieces) nblk = kPieces;
  }
  return nblk;
}

void launch_lfront_sort(const FrontArgs &f, uint16_t *bkt, const uint32_t *rank, uint32_t *cnt, uint64_t nb,
                        cudaStream_t s) {
  note_launch();
  k_lscatter<kSortItems><<<front_tiles(nb), kSortThreads, 0, s>>>(f.bufA, bkt, rank, cnt, f.bufB, f.ctl);
  note_launch();
  // bkt, read by k_lscatter by batch position, then takes each sorted word's bucket
  k_lsort_warp<<<kPieces / 8, 256, 0, s>>>(f.bufB, sorted_words(f), cnt, bkt, f.ctl);
  note_launch();
  k_lsort<<<lsort_blocks(), 256, 0, s>>>(f.bufB, sorted_words(f), cnt, bkt, f.ctl);
}

bool search_wide(uint64_t n) { return search_per(n) == 4; }

// ---- many handles: one launch per stage over the work of all of them ---------------------------
// Each block finds its handle (and its block index within that handle's share)
// in the call's plan table and runs the same body as the single-handle kernel,
// with the handle's own sizes; blocks beyond what this call's batch needs return.
__device__ __forceinline__ TileSums tile_sums(uint32_t *rs, uint32_t T, uint32_t T1) {
  uint32_t *q = rs + (uint64_t)512 * T;
  const uint32_t K = T1 + 1;
  return TileSums{q, q + K, q + 2 * K, q + 3 * K, q + 4 * K, q + 5 * K, q + 6 * K};
}

__global__ void k_m_init(const ManyDesc *d, uint32_t plan) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb) || !it->active || it->small) return;
  init_batch_body(GridIdx{}, it->ctl, it->hist, it->prep.npass * 256u, it->prep.n_ins + it->prep.n_del);
}

__global__ void __launch_bounds__(1024) k_m_small_front(const ManyDesc *d, uint32_t plan) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb) || !it->active || !it->small) return;
  small_front_body(GridIdx{}, it->prep, it->ins, it->del, it->ctl, it->g.F, it->g.nleaves, it->w.ukey, it->w.utag,
                   it->w.uleaf, it->w.run_start, it->w.rleaf, it->mhead, it->mpieces, it->P, it->S);
}

__global__ void __launch_bounds__(kSortThreads) k_m_prep(const ManyDesc *d, uint32_t plan) {
  const ManyItem *it;
  uint32_t sub, nb;
  // every block of the handle takes the prep ticket: the plan gives it at most T blocks
  if (!many_block(d, plan, &it, &sub, &nb) || it->small) return;
  prep_body<kSortItems>(SubIdx{sub, nb}, it->prep, it->ins, it->del, it->bufA, it->hist, it->w.rs, it->T,
                        it->ctl);
}

__global__ void __launch_bounds__(256) k_m_rcolscan(const ManyDesc *d, uint32_t plan, uint32_t p) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb) || it->small || p >= it->prep.npass) return;
  const uint32_t T = it->T;
  uint32_t *H[2] = {it->w.rs, it->w.rs + (uint64_t)256 * T};
  rcolscan_body(SubIdx{sub, nb}, H[p & 1], p + 1 < it->prep.npass ? H[(p + 1) & 1] : nullptr, T,
                it->hist + 8 * 256 + p * 256, 1u << it->prep.dbits, it->ctl);
}

__global__ void __launch_bounds__(kSortThreads) k_m_rscatter(const ManyDesc *d, uint32_t plan, uint32_t p) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb) || it->small || p >= it->prep.npass) return;
  const uint32_t T = it->T, db = it->prep.dbits;
  uint32_t *H[2] = {it->w.rs, it->w.rs + (uint64_t)256 * T};
  const uint64_t *src = (p & 1) ? it->bufB : it->bufA;
  uint64_t *dst = (p & 1) ? it->bufA : it->bufB;
  rscatter_body<kSortItems>(SubIdx{sub, nb}, src, dst, H[p & 1], p + 1 < it->prep.npass ? H[(p + 1) & 1] : nullptr,
                            T, p * db, (p + 1) * db, db, it->ctl);
}

template <int Q>
__global__ void __launch_bounds__(kSearchThreads) k_m_rsearch(const ManyDesc *d, uint32_t plan) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb) || it->small || it->wide != (Q == 4 ? 1u : 0u)) return;
  const uint64_t *sorted = (it->prep.npass & 1) ? it->bufB : it->bufA;
  rsearch_body<Q>(SubIdx{sub, nb}, it->prep, sorted, it->w.pleaf, it->g.F, it->g.nleaves,
                  tile_sums(it->w.rs, it->T, it->T1), it->T1, it->ctl, it->mhead, it->mpieces,
                  nullptr);
}

__global__ void __launch_bounds__(1024) k_m_toffsets(const ManyDesc *d, uint32_t plan) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb) || !it->active || it->small) return;
  toffsets_body(GridIdx{}, tile_sums(it->w.rs, it->T, it->T1), it->T1, it->ctl, it->w.run_start);
}

template <int Q>
__global__ void __launch_bounds__(kSearchThreads) k_m_twrite(const ManyDesc *d, uint32_t plan) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb) || it->small || it->wide != (Q == 4 ? 1u : 0u)) return;
  const uint64_t *sorted = (it->prep.npass & 1) ? it->bufB : it->bufA;
  twrite_body<Q>(SubIdx{sub, nb}, it->prep, sorted, it->w.pleaf, tile_sums(it->w.rs, it->T, it->T1), it->T1,
                 it->w.ukey, it->w.utag, it->w.uleaf, it->w.run_start, it->w.rleaf, it->ctl);
}

void prepare_many_front() {
  cudaFuncSetAttribute(k_m_small_front, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallBatch * 20 + 2048 * 12);
}

void launch_many_front(const ManyDesc *d, const ManyPlans &pl, cudaStream_t s) {
  const uint32_t one = pl.total[pl.one];
  note_launch();
  k_m_small_front<<<one, 1024, kSmallBatch * 20 + 2048 * 12, s>>>(d, pl.one);
  if (!pl.total[pl.tiles]) return;  // no handle's work arrays can hold more than kSmallBatch keys
  note_launch();
  k_m_init<<<one, 256, 0, s>>>(d, pl.one);
  note_launch();
  k_m_prep<<<pl.total[pl.tiles], kSortThreads, 0, s>>>(d, pl.tiles);
  for (uint32_t p = 0; p < pl.maxpass; p++) {
    note_launch();
    k_m_rcolscan<<<pl.total[pl.radix], 256, 0, s>>>(d, pl.radix, p);
    note_launch();
    k_m_rscatter<<<pl.total[pl.tiles], kSortThreads, 0, s>>>(d, pl.tiles, p);
  }
  if (pl.total[pl.search[0]]) {
    note_launch();
    k_m_rsearch<1><<<pl.total[pl.search[0]], kSearchThreads, 0, s>>>(d, pl.search[0]);
  }
  if (pl.total[pl.search[1]]) {
    note_launch();
    k_m_rsearch<4><<<pl.total[pl.search[1]], kSearchThreads, 0, s>>>(d, pl.search[1]);
  }
  note_launch();
  k_m_toffsets<<<one, 1024, 0, s>>>(d, pl.one);
  if (pl.total[pl.search[0]]) {
    note_launch();
    k_m_twrite<1><<<pl.total[pl.search[0]], kSearchThreads, 0, s>>>(d, pl.search[0]);
  }
  if (pl.total[pl.search[1]]) {
    note_launch();
    k_m_twrite<4><<<pl.total[pl.search[1]], kSearchThreads, 0, s>>>(d, pl.search[1]);
  }
}

// enough for every batch of at most nb keys (one word a thread gives the most search blocks)
uint64_t front_scratch_words(uint64_t nb) {
  return (uint64_t)512 * front_tiles(nb) + 7ull * ((nb + kSearchThreads - 1) / kSearchThreads + 1);
}

}  // namespace gpk
