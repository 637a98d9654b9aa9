// scan_dev.cuh -- block-level building block of the single-pass scans and
// compactions: a tile of kScanItems rounds x 256 threads, element order
// (round, thread); the tile's exclusive prefix comes from a look-back over the
// tiles before it (tiles are numbered by ticket, so every awaited tile runs).
#pragma once
#include "gpma_dev.cuh"

namespace gpk {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

struct ScanSmem {
  uint32_t cnt[kScanItems][kScanThreads / 32];
  uint32_t excl;
  uint32_t tot;
  uint32_t tile;
};

__device__ __forceinline__ uint32_t take_ticket(Ctl *ctl, uint32_t slot, ScanSmem &sm) {
  if (threadIdx.x == 0) sm.tile = atomicAdd(&ctl->ticket[slot], 1u);
  __syncthreads();
  return sm.tile;
}

// Exclusive prefix (in element order) of per-item values v; values and the
// tile total must stay below 2^30.  Returns the running total after this tile.
__device__ __forceinline__ uint32_t tile_scan(const uint32_t (&v)[kScanItems], uint32_t (&off)[kScanItems],
                                              uint32_t tile, uint64_t *status, uint32_t stride, uint32_t col,
                                              uint32_t epoch, Ctl *ctl, ScanSmem &sm) {
  const uint32_t w = threadIdx.x >> 5, lane = lane_id();
  uint32_t inc[kScanItems];
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    inc[r] = warp_incl_scan(v[r]);
    if (lane == 31) sm.cnt[r][w] = inc[r];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // kScanItems * 8 = 64 warp totals, two per lane, in (round, warp) order
    const uint32_t i0 = 2 * lane, i1 = 2 * lane + 1;
    uint32_t a = sm.cnt[i0 / 8][i0 % 8], b = sm.cnt[i1 / 8][i1 % 8];
    uint32_t s = warp_incl_scan(a + b);
    uint32_t tot = __shfl_sync(0xFFFFFFFFu, s, 31);
    sm.cnt[i0 / 8][i0 % 8] = s - a - b;
    sm.cnt[i1 / 8][i1 % 8] = s - b;
    if (lane == 0) {
      sm.excl = lookback(status, stride, col, tile, tot, epoch, ctl);
      sm.tot = tot;
    }
  }
  __syncthreads();
  const uint32_t excl = sm.excl, total = sm.excl + sm.tot;
#pragma unroll
  for (int r = 0; r < kScanItems; r++) off[r] = excl + sm.cnt[r][w] + inc[r] - v[r];
  __syncthreads();  // sm reused by a second scan in the same kernel
  return total;
}

__device__ __forceinline__ uint64_t scan_elem(uint32_t tile, int r) {
  return (uint64_t)tile * kScanTile + (uint64_t)r * kScanThreads + threadIdx.x;
}

}  // namespace gpk
