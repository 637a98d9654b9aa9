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
  uint32_t pad;
  uint64_t tree_off[kMaxLv];  // offset of level i (1..h) inside tree/mark
  uint64_t maxc[kMaxLv];      // max_i: largest admissible count at level i
};

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
  uint32_t levels_climbed;
  uint32_t n_merged0;
  uint64_t merges[kMaxLv];
  uint64_t gen_count;  // general-purpose counter (exports)
};

__device__ __forceinline__ bool is_guard(uint64_t k) {
  return k != kEmpty && (k & 0xFFFFFFFFull) == 0xFFFFFFFFull;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// add +1 / -1 to the out-degree of the source of every marked lane's key; lanes
// of one source (rows are contiguous) combine into one atomic
__device__ __forceinline__ void degree_delta(uint32_t *deg, bool active, uint64_t key, int d) {
  const uint32_t src = active ? (uint32_t)(key >> 32) : 0xFFFFFFFFu;
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, src);
  if (active && (threadIdx.x & 31u) == (uint32_t)(__ffs(peers) - 1))
    atomicAdd(&deg[src], (uint32_t)(d * __popc(peers)));
}
__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << lane_id()) - 1u; }

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
// <= k, leaf 0 if none.  Binary search over the pivots F with empty leaves
// skipped forward (an empty leaf takes the pivot of the next non-empty one).
__device__ __forceinline__ uint32_t leaf_search(const uint64_t *__restrict__ F, uint64_t nleaves,
                                                uint64_t k) {
  uint64_t lo = 0, hi = nleaves;  // find p = first leaf whose effective pivot is > k
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
  return lo ? (uint32_t)(lo - 1) : 0u;
}

// ---- single-pass look-back (tiles take tickets in launch order) -------------------
// Status word of one tile: [epoch:32][flag:2][value:30]; flag 1 = tile aggregate,
// flag 2 = inclusive prefix.  A spin is bounded; on give-up the call's error word
// gets kErrTimeout and the value read so far is used (the batch is then discarded).
constexpr uint64_t kFlagAgg = 1ull << 30;
constexpr uint64_t kFlagPre = 2ull << 30;
constexpr uint32_t kSpinLimit = 1u << 22;

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
__device__ __forceinline__ uint32_t lookback(uint64_t *status, uint32_t stride, uint32_t col,
                                             uint32_t tile, uint32_t agg, uint32_t epoch,
                                             uint32_t *err) {
  if (tile == 0) {
    st_status(status + col, pack_status(epoch, kFlagPre, agg));
    return 0;
  }
  st_status(status + (uint64_t)tile * stride + col, pack_status(epoch, kFlagAgg, agg));
  uint32_t excl = 0;
  int64_t t = (int64_t)tile - 1;
  uint32_t spins = 0;
  while (t >= 0) {
    uint64_t s = ld_status(status + (uint64_t)t * stride + col);
    if ((uint32_t)(s >> 32) != epoch || (s & (3ull << 30)) == 0) {
      if (++spins > kSpinLimit) {
        atomicOr(err, kErrTimeout);
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
