// k_misc.cu -- index rebuild (import / restore), the device consistency checker,
// exports (sorted edges, CSR columns, per-vertex degrees) and a u32 -> u64 scan.
#include "gpma_dev.cuh"
#include "gpma_launch.h"
#include "scan_dev.cuh"

namespace gpk {

static uint32_t nblocks(uint64_t items, uint32_t per_block, uint32_t cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (uint32_t)b;
}

// ---- exclusive scan u32 -> u64 (reduce, scan of tile sums, down-sweep) -----------------------
constexpr int kTile = 4096;  // 256 threads x 16 values

__device__ __forceinline__ uint64_t dev_n(uint64_t n_bound, const uint32_t *n_dev) {
  if (!n_dev) return n_bound;
  uint64_t n = *n_dev;
  return n < n_bound ? n : n_bound;
}

__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t *__restrict__ in, uint64_t n_bound,
                                                     const uint32_t *n_dev, uint64_t *partials) {
  __shared__ uint64_t ws[8];
  const uint64_t n = dev_n(n_bound, n_dev);
  const uint64_t b0 = (uint64_t)blockIdx.x * kTile;
  if (b0 >= n && blockIdx.x > 0) return;
  uint64_t s = 0;
  for (uint32_t i = threadIdx.x; i < kTile; i += 256) {
    uint64_t e = b0 + i;
    if (e < n) s += in[e];
  }
  s = warp_sum(s);
  if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int q = 0; q < 8; q++) t += ws[q];
    partials[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_scan_partials(uint64_t *partials, uint64_t n_bound, const uint32_t *n_dev,
                                                        uint64_t *out) {
  __shared__ uint64_t ws[32];
  __shared__ uint64_t carry_s;
  const uint64_t n = dev_n(n_bound, n_dev);
  const uint64_t nb = n ? (n + kTile - 1) / kTile : 0;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (uint64_t c = 0; c < nb; c += 1024) {
    uint64_t i = c + threadIdx.x;
    uint64_t v = i < nb ? partials[i] : 0;
    uint64_t inc = warp_incl_scan(v);
    if (lane_id() == 31) ws[threadIdx.x >> 5] = inc;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint64_t x = ws[threadIdx.x];
      ws[threadIdx.x] = warp_incl_scan(x) - x;
    }
    __syncthreads();
    uint64_t ex = carry_s + ws[threadIdx.x >> 5] + inc - v;
    if (i < nb) partials[i] = ex;
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = ex + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry_s;
}

__global__ void __launch_bounds__(256) k_scan_down(const uint32_t *__restrict__ in, uint64_t *__restrict__ out,
                                                   uint64_t n_bound, const uint32_t *n_dev,
                                                   const uint64_t *partials) {
  __shared__ uint64_t ws[8];
  const uint64_t n = dev_n(n_bound, n_dev);
  const uint64_t b0 = (uint64_t)blockIdx.x * kTile;
  if (b0 >= n) return;
  // thread t owns 16 consecutive values
  const uint64_t e0 = b0 + (uint64_t)threadIdx.x * 16;
  uint32_t v[16];
  uint64_t s = 0;
#pragma unroll
  for (int q = 0; q < 16; q++) {
    v[q] = (e0 + q < n) ? in[e0 + q] : 0u;
    s += v[q];
  }
  uint64_t inc = warp_incl_scan(s);
  if (lane_id() == 31) ws[threadIdx.x >> 5] = inc;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint64_t x = threadIdx.x < 8 ? ws[threadIdx.x] : 0;
    uint64_t y = warp_incl_scan(x) - x;
    if (threadIdx.x < 8) ws[threadIdx.x] = y;
  }
  __syncthreads();
  uint64_t run = partials[blockIdx.x] + ws[threadIdx.x >> 5] + inc - s;
#pragma unroll
  for (int q = 0; q < 16; q++) {
    if (e0 + q < n) out[e0 + q] = run;
    run += v[q];
  }
}

uint64_t scan_partials(uint64_t n) { return (n + kTile - 1) / kTile + 1; }

void launch_scan_u32_u64(const uint32_t *in, uint64_t *out, uint64_t n_bound, uint64_t *partials, cudaStream_t s,
                         const uint32_t *n_dev) {
  const uint32_t nb = (uint32_t)((n_bound + kTile - 1) / kTile);
  const uint32_t g = nb ? nb : 1;
  note_launch();
  k_scan_reduce<<<g, 256, 0, s>>>(in, n_bound, n_dev, partials);
  note_launch();
  k_scan_partials<<<1, 1024, 0, s>>>(partials, n_bound, n_dev, out);
  note_launch();
  k_scan_down<<<g, 256, 0, s>>>(in, out, n_bound, n_dev, partials);
}

// ---- index rebuild: cnt, F, row_end, total, then the tree level by level -----------------------
__global__ void k_leaf_index(Geo g, Ctl *ctl) {
  const uint32_t lane = lane_id(), L = g.L;
  uint64_t acc = 0;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t j = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < g.nleaves; j += nw) {
    const uint64_t *p = g.slots + j * L;
    uint32_t c = 0;
    uint64_t first = kEmpty;
    for (uint32_t b = 0; b < L; b += 32) {
      uint64_t k = (b + lane < L) ? p[b + lane] : kEmpty;
      bool v = k != kEmpty;
      uint32_t bal = __ballot_sync(0xFFFFFFFFu, v);
      if (first == kEmpty && bal) first = __shfl_sync(0xFFFFFFFFu, k, __ffs(bal) - 1);
      c += __popc(bal);
      if (!g.raw && v && is_guard(k)) g.row_end[k >> 32] = (uint32_t)(j * L + b + lane);
    }
    if (lane == 0) {
      g.cnt[j] = c;
      g.F[j] = first;
    }
    acc += c;
  }
  if (lane == 0 && acc) atomicAdd((unsigned long long *)&ctl->total, (unsigned long long)acc);
}

__global__ void k_tree_level(Geo g, uint32_t i) {
  const uint64_t nodes = g.nleaves >> i;
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nodes; s += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t a, b;
    if (i == 1) {
      a = g.cnt[2 * s];
      b = g.cnt[2 * s + 1];
    } else {
      a = g.tree[g.tree_off[i - 1] + 2 * s];
      b = g.tree[g.tree_off[i - 1] + 2 * s + 1];
    }
    g.tree[g.tree_off[i] + s] = a + b;
  }
}

__global__ void k_zero_total(Ctl *ctl) { ctl->total = 0; }

void launch_rebuild_indexes(const Geo &g, Ctl *ctl, cudaStream_t s) {
  if (!g.raw) launch_degrees(g, g.deg, s);
  note_launch();
  k_zero_total<<<1, 1, 0, s>>>(ctl);
  note_launch();
  k_leaf_index<<<nblocks(g.nleaves, 8, 152 * 16), 256, 0, s>>>(g, ctl);
  for (uint32_t i = 1; i <= g.h; i++) {
    note_launch();
    k_tree_level<<<nblocks(g.nleaves >> i, 256, 152 * 8), 256, 0, s>>>(g, i);
  }
}

// ---- consistency checker -----------------------------------------------------------------------
__global__ void k_check_leaves(Geo g, uint32_t *code, unsigned long long *sum) {
  const uint32_t lane = lane_id(), L = g.L;
  uint32_t bad = 0;
  uint64_t acc = 0;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t j = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < g.nleaves; j += nw) {
    const uint64_t *p = g.slots + j * L;
    uint32_t c = 0;
    uint64_t first = kEmpty, last = 0;
    bool have_last = false;
    for (uint32_t b = 0; b < L; b += 32) {
      uint64_t k = (b + lane < L) ? p[b + lane] : kEmpty;
      bool v = k != kEmpty;
      uint32_t bal = __ballot_sync(0xFFFFFFFFu, v);
      // valid keys of the round in slot order, against the last key seen
      for (uint32_t q = bal; q; q &= q - 1) {
        int src = __ffs(q) - 1;
        uint64_t kk = __shfl_sync(0xFFFFFFFFu, k, src);
        if (have_last && kk <= last) bad |= 1;
        last = kk;
        have_last = true;
        if (first == kEmpty) first = kk;
      }
      c += __popc(bal);
      if (!g.raw && v && is_guard(k) && g.row_end[k >> 32] != (uint32_t)(j * L + b + lane)) bad |= 8;
    }
    if (c != g.cnt[j] || first != g.F[j]) bad |= 2;
    if (c > g.maxc[0]) bad |= 4;
    // dual mode: no deletion leaves a hole, every leaf is left-packed
    if (g.dual)
      for (uint32_t b = 0; b < L; b += 32)
        if (b + lane < L && ((p[b + lane] != kEmpty) != (b + lane < c))) bad |= 128;
    // the last key of this leaf is below the first key of the next non-empty leaf
    if (have_last) {
      for (uint64_t q = j + 1; q < g.nleaves; q++) {
        uint64_t f = g.F[q];
        if (f == kEmpty) continue;
        if (f <= last) bad |= 1;
        break;
      }
    }
    acc += c;
  }
  if (bad) atomicOr(code, bad);
  if (lane_id() == 0 && acc) atomicAdd(sum, (unsigned long long)acc);
}

// the merge marks are all clear between batches (the count tree itself is
// rebuilt whenever a batch needs it)
__global__ void k_check_tree(Geo g, uint32_t *code) {
  uint32_t bad = 0;
  const uint64_t total = g.nleaves > 1 ? g.nleaves - 1 : 0;
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < total; s += (uint64_t)gridDim.x * blockDim.x)
    if (g.mark[s] != 0) bad |= 16;
  if (bad) atomicOr(code, bad);
}

// every vertex's kept out-degree equals the stored edges of its row
__global__ void k_check_degrees(Geo g, uint32_t *code) {
  const uint32_t lane = lane_id();
  uint32_t bad = 0;
  const uint32_t nw = gridDim.x * (blockDim.x >> 5);
  for (uint32_t u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < g.V; u += nw) {
    const uint32_t r = g.row_end[u];
    const uint64_t beg = u ? (uint64_t)g.row_end[u - 1] + 1 : 0, end = r;
    if (end > g.C || beg > end) {
      bad |= 64;
      continue;
    }
    uint32_t c = 0;
    for (uint64_t e = beg + lane; e < end; e += 32) c += g.slots[e] != kEmpty;
    c = warp_sum(c);
    if (c != g.deg[u]) bad |= 64;
  }
  if (bad && lane == 0) atomicOr(code, bad);
}

// every vertex has its guard exactly where row_end says
__global__ void k_check_guards(Geo g, uint32_t *code) {
  uint32_t bad = 0;
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < g.V; u += gridDim.x * blockDim.x) {
    const uint32_t r = g.row_end[u];
    if ((uint64_t)r >= g.C || g.slots[r] != (((uint64_t)u << 32) | 0xFFFFFFFFull)) bad |= 8;
  }
  if (bad) atomicOr(code, bad);
}

__global__ void k_check_total(Ctl *ctl, uint32_t *code, const unsigned long long *sum) {
  if (*sum != ctl->total) atomicOr(code, 32u);
}

void launch_check(const Geo &g, Ctl *ctl, uint32_t *code, cudaStream_t s) {
  // code[0] = bits, code[1..2] = scratch sum (u64)
  cudaMemsetAsync(code, 0, 16, s);
  unsigned long long *sum = (unsigned long long *)(code + 2);
  note_launch();
  k_check_leaves<<<nblocks(g.nleaves, 8, 152 * 16), 256, 0, s>>>(g, code, sum);
  note_launch();
  k_check_tree<<<nblocks(g.nleaves / 2, 256, 152 * 8), 256, 0, s>>>(g, code);
  if (!g.raw) {
    note_launch();
    k_check_guards<<<nblocks(g.V, 256, 152 * 8), 256, 0, s>>>(g, code);
    note_launch();
    k_check_degrees<<<nblocks(g.V, 8, 152 * 16), 256, 0, s>>>(g, code);
  }
  note_launch();
  k_check_total<<<1, 1, 0, s>>>(ctl, code, sum);
}

// ---- exports -----------------------------------------------------------------------------------
// single-pass compaction of the valid non-guard keys (raw mode: every valid key)
__global__ void __launch_bounds__(kScanThreads) k_export(Geo g, Ctl *ctl, uint64_t *out_keys, uint32_t *out_cols,
                                                         uint64_t cap, uint64_t *status) {
  __shared__ ScanSmem sm;
  const uint32_t tile = take_ticket(ctl, kSlotMisc, sm);
  uint32_t flag[kScanItems];
  uint64_t k[kScanItems];
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    uint64_t e = scan_elem(tile, r);
    k[r] = e < g.C ? g.slots[e] : kEmpty;
    flag[r] = k[r] != kEmpty && (g.raw || !is_guard(k[r]));
  }
  uint32_t off[kScanItems];
  uint32_t total = tile_scan(flag, off, tile, status, 1, 0, ctl->epoch + kSlotMisc, ctl, sm);
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    if (!flag[r] || off[r] >= cap) continue;
    if (out_keys) out_keys[off[r]] = k[r];
    if (out_cols) out_cols[off[r]] = (uint32_t)(k[r] & 0xFFFFFFFFull);
  }
  if ((uint64_t)(tile + 1) * kScanTile >= g.C && threadIdx.x == 0) ctl->gen_count = total;
}

// starts an export: its own error word (a batch's error is already in sticky)
__global__ void k_export_prep(Ctl *ctl) {
  ctl->err = 0;
  ctl->epoch += kSlotsPerBatch;
  ctl->ticket[kSlotMisc] = 0;
  ctl->gen_count = 0;
}

void launch_export(const Geo &g, Ctl *ctl, uint64_t *out_keys, uint32_t *out_cols, uint64_t cap, uint64_t *status,
                   cudaStream_t s) {
  note_launch();
  k_export_prep<<<1, 1, 0, s>>>(ctl);
  note_launch();
  k_export<<<comp_tiles(g.C), kScanThreads, 0, s>>>(g, ctl, out_keys, out_cols, cap, status);
}

// out-degree of every vertex; rows are contiguous, so lanes of one row add once
__global__ void k_degrees(Geo g, uint32_t *deg) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ((g.C + 31) & ~31ull);
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = e < g.C ? g.slots[e] : kEmpty;
    bool v = k != kEmpty && !is_guard(k);
    uint32_t src = v ? (uint32_t)(k >> 32) : 0xFFFFFFFFu;
    uint32_t peers = __match_any_sync(0xFFFFFFFFu, src);
    if (v && lane_id() == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&deg[src], (uint32_t)__popc(peers));
  }
}

void launch_degrees(const Geo &g, uint32_t *deg, cudaStream_t s) {
  cudaMemsetAsync(deg, 0, sizeof(uint32_t) * g.V, s);
  note_launch();
  k_degrees<<<nblocks(g.C, 256, 152 * 16), 256, 0, s>>>(g, deg);
}

void launch_rowptr(const uint32_t *deg, uint64_t *rowptr, uint32_t V, uint64_t *partials, cudaStream_t s) {
  launch_scan_u32_u64(deg, rowptr, V, partials, s, nullptr);
}

}  // namespace gpk
