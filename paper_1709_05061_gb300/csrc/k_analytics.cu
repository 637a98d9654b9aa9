// k_analytics.cu -- graph analytics that read the gapped array in place
// (Sec. 4.2: every access tests IsEntryExist, i.e. skips EMPTY slots; guards
// delimit the rows).
//   PageRank  power iteration with a push SpMV over the slots (Sec. 6.1)
//   BFS       level-synchronous in one persistent cooperative kernel: a warp gathers
//             a frontier vertex's row for small frontiers, one pass over the array
//             for large ones
//   CC        lock-free union-find over the edges; a root is always the smallest
//             id of its tree, so the final label is the component's minimum id
#include "gpma_dev.cuh"
#include "gpma_launch.h"

namespace gpk {

static uint32_t nb(uint64_t items, uint32_t per_block, uint32_t cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (uint32_t)b;
}

// ---- PageRank -----------------------------------------------------------------------------------
// Sum of one double per thread over the grid: per-block partials, and the last
// block to finish adds them in block order (fixed order, one atomic per block).
__device__ __forceinline__ void grid_sum_double(double v, double *partials, unsigned *counter, double *out) {
  __shared__ double ws[32];
  __shared__ bool last;
  v = warp_sum(v);
  if (lane_id() == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (uint32_t q = 0; q < (blockDim.x >> 5); q++) b += ws[q];
    partials[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    double t = 0.0;
    const volatile double *vp = partials;
    for (uint32_t q = threadIdx.x; q < gridDim.x; q += blockDim.x) t += vp[q];
    t = warp_sum(t);
    if (lane_id() == 0) ws[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (uint32_t q = 0; q < (blockDim.x >> 5); q++) tot += ws[q];
      *out = tot;
      *counter = 0;
    }
  }
}

__global__ void k_pr_init(uint32_t V, const uint32_t *__restrict__ deg, float *__restrict__ x,
                          float *__restrict__ contrib, double *__restrict__ y, double *dsum0, double *partials,
                          unsigned *counter) {
  const float x0 = (float)(1.0 / (double)V);
  double dang = 0.0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
    const uint32_t d = deg[v];
    x[v] = x0;
    y[v] = 0.0;
    contrib[v] = d ? x0 / (float)d : 0.0f;
    if (!d) dang += (double)x0;
  }
  grid_sum_double(dang, partials, counter, dsum0);
}

// y[v] += x[u] / outdeg(u) for every stored edge u -> v.  Each thread owns two
// 16-byte slot pairs per step and loads the next step's pairs before it works on
// the current ones, so the HBM stream overlaps the gathers and the reductions.
__device__ __forceinline__ void pr_push(uint64_t k, const float *__restrict__ contrib, double *__restrict__ y) {
  if (k != kEmpty && !is_guard(k)) atomicAdd(&y[k & 0xFFFFFFFFull], (double)__ldg(contrib + (k >> 32)));
}

__global__ void __launch_bounds__(256) k_pr_scatter(Geo g, const float *__restrict__ contrib,
                                                    double *__restrict__ y) {
  const uint64_t npairs = g.C >> 1;
  const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(g.slots);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const ulonglong2 none = make_ulonglong2(kEmpty, kEmpty);
  uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  ulonglong2 a = p < npairs ? __ldcs(s2 + p) : none;
  ulonglong2 b = p + stride < npairs ? __ldcs(s2 + p + stride) : none;
  while (p < npairs) {
    const uint64_t q = p + 2 * stride;
    const ulonglong2 na = q < npairs ? __ldcs(s2 + q) : none;
    const ulonglong2 nb = q + stride < npairs ? __ldcs(s2 + q + stride) : none;
    pr_push(a.x, contrib, y);
    pr_push(a.y, contrib, y);
    pr_push(b.x, contrib, y);
    pr_push(b.y, contrib, y);
    a = na;
    b = nb;
    p = q;
  }
}

__global__ void k_pr_apply(uint32_t V, float damping, const uint32_t *__restrict__ deg, double *__restrict__ y,
                           float *__restrict__ x, float *__restrict__ contrib, const double *dsum_in,
                           double *dsum_out, double *partials, unsigned *counter) {
  const double base = (1.0 - (double)damping) / (double)V;
  const double dn = *dsum_in / (double)V;
  double dang = 0.0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
    const double nx = base + (double)damping * (y[v] + dn);
    const float xf = (float)nx;
    const uint32_t d = deg[v];
    x[v] = xf;
    y[v] = 0.0;
    contrib[v] = d ? xf / (float)d : 0.0f;
    if (!d) dang += (double)xf;
  }
  grid_sum_double(dang, partials, counter, dsum_out);
}

constexpr uint32_t kVecBlocks = 152 * 4;  // grid of the per-vertex kernels (and partials per sum)

void launch_pr_setup(const Geo &g, uint32_t iters, float *rank, uint32_t *deg, double *y, float *contrib,
                     double *dsum, double *partials, unsigned *counter, cudaStream_t s) {
  launch_degrees(g, deg, s);
  cudaMemsetAsync(dsum, 0, sizeof(double) * (iters + 1), s);
  cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  note_launch();
  k_pr_init<<<nb(g.V, 256, kVecBlocks), 256, 0, s>>>(g.V, deg, rank, contrib, y, dsum, partials, counter);
}

void launch_pr_scatter(const Geo &g, const float *contrib, double *y, cudaStream_t s) {
  note_launch();
  k_pr_scatter<<<nb(g.C >> 2, 256, 152 * 8), 256, 0, s>>>(g, contrib, y);
}

void launch_pr_apply(const Geo &g, float damping, float *rank, const uint32_t *deg, double *y, float *contrib,
                     const double *dsum_in, double *dsum_out, double *partials, unsigned *counter,
                     cudaStream_t s) {
  note_launch();
  k_pr_apply<<<nb(g.V, 256, kVecBlocks), 256, 0, s>>>(g.V, damping, deg, y, rank, contrib, dsum_in, dsum_out,
                                                         partials, counter);
}

// ---- BFS ----------------------------------------------------------------------------------------
// Small frontiers: top-down from a queue, one warp per frontier vertex's row
// (Algorithm "GPU-based BFS Neighbour Gathering", EMPTY slots skipped).  Large
// frontiers: one pass over the whole gapped array, each stored edge u -> v with
// depth[u] == level claiming v (no queue); the queue is rebuilt from the depth
// array when the frontier shrinks again.
// ---- BFS as one persistent kernel -----------------------------------------------------------
// All levels run inside one cooperative launch (every block resident), separated
// by a grid barrier whose waits are bounded: a barrier that gives up sets
// kErrTimeout and every block leaves.  Counters: cnt[0..2] rotate per level
// (frontier sizes), cnt[3] is the queue-rebuild counter, cnt[4] the level count.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, uint32_t *err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      uint32_t spins = 0;
      while (*gen == g0) {
        if (++spins > (1u << 24)) {
          atomicOr(err, kErrTimeout);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile uint32_t *)err == 0;
}

// claim the unvisited heads of stored edges in slots [beg, end) of one row
__device__ __forceinline__ void bfs_gather(const Geo &g, int32_t *depth, uint64_t beg, uint64_t end,
                                           uint32_t *qout, uint32_t *cnext, int32_t level) {
  const uint32_t lane = lane_id();
  for (uint64_t s = beg; s < end; s += 32) {
    const uint64_t e = s + lane;
    bool got = false;
    uint32_t v = 0;
    if (e < end) {
      const uint64_t k = __ldg(g.slots + e);
      if (k != kEmpty) {  // IsEntryExist
        v = (uint32_t)(k & 0xFFFFFFFFull);
        if (__ldcg(depth + v) < 0) got = atomicCAS(&depth[v], -1, level + 1) == -1;
      }
    }
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, got);
    if (bal) {
      uint32_t base = 0;
      if (lane == (uint32_t)(__ffs(bal) - 1)) base = atomicAdd(cnext, (uint32_t)__popc(bal));
      base = __shfl_sync(0xFFFFFFFFu, base, __ffs(bal) - 1);
      if (got) qout[base + __popc(bal & lanemask_lt())] = v;
    }
  }
}

constexpr uint64_t kBigRow = 1024, kRowChunk = 256;

// cnt[0..2]: frontier sizes (rotating), cnt[3]: queue rebuild, cnt[4]: levels,
// cnt[5]: long rows of the level (listed in `big`)
__global__ void __launch_bounds__(256) k_bfs_persist(Geo g, int32_t *depth, uint32_t *qa, uint32_t *qb,
                                                     uint32_t *big, uint32_t *cnt, unsigned *bar, uint32_t *err,
                                                     uint32_t scan_from) {
  const uint32_t lane = lane_id();
  const uint32_t warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(g.slots);
  const uint64_t npairs = g.C >> 1;
  uint32_t *qin = qa, *qout = qb;
  uint32_t nfront = 1;
  int32_t level = 0;
  bool have_queue = true;
  while (nfront) {
    uint32_t *cnext = cnt + (level + 1) % 3;
    if (tid == 0) cnt[(level + 2) % 3] = 0;
    const bool scan = nfront >= scan_from;
    if (scan) {
      // one pass over the array: edges u -> v with depth[u] == level claim v
      uint32_t found = 0;
      for (uint64_t p = tid; p < npairs; p += nthreads) {
        const ulonglong2 kk = __ldcs(s2 + p);
        const uint64_t ks[2] = {kk.x, kk.y};
#pragma unroll
        for (int q = 0; q < 2; q++) {
          const uint64_t k = ks[q];
          if (k == kEmpty || is_guard(k)) continue;
          if (__ldcg(depth + (k >> 32)) != level) continue;
          const uint32_t v = (uint32_t)(k & 0xFFFFFFFFull);
          if (__ldcg(depth + v) < 0 && atomicCAS(&depth[v], -1, level + 1) == -1) ++found;
        }
      }
      found = warp_sum(found);
      if (lane == 0 && found) atomicAdd(cnext, found);
    } else {
      if (!have_queue) {  // queue of this level from the depth array
        const uint32_t vend = (g.V + 31) & ~31u;
        for (uint32_t v = (uint32_t)tid; v < vend; v += (uint32_t)nthreads) {
          const bool hit = v < g.V && __ldcg(depth + v) == level;
          const uint32_t bal = __ballot_sync(0xFFFFFFFFu, hit);
          if (!bal) continue;
          uint32_t base = 0;
          if (lane == (uint32_t)(__ffs(bal) - 1)) base = atomicAdd(cnt + 3, (uint32_t)__popc(bal));
          base = __shfl_sync(0xFFFFFFFFu, base, __ffs(bal) - 1);
          if (hit) qin[base + __popc(bal & lanemask_lt())] = v;
        }
        if (!grid_barrier(bar, err)) return;
      }
      // top-down: a warp per short row; long rows are listed and split below
      for (uint32_t i = warp; i < nfront; i += nwarps) {
        const uint32_t u = __ldcg(qin + i);
        const uint64_t beg = u ? (uint64_t)__ldg(g.row_end + u - 1) + 1 : 0, end = __ldg(g.row_end + u);
        if (end - beg > kBigRow) {
          if (lane == 0) big[atomicAdd(cnt + 5, 1u)] = u;
          continue;
        }
        bfs_gather(g, depth, beg, end, qout, cnext, level);
      }
      if (!grid_barrier(bar, err)) return;
      const uint32_t nbig = *(volatile uint32_t *)(cnt + 5);
      for (uint32_t b = 0; b < nbig; b++) {
        const uint32_t u = __ldcg(big + b);
        const uint64_t beg = u ? (uint64_t)__ldg(g.row_end + u - 1) + 1 : 0, end = __ldg(g.row_end + u);
        const uint64_t chunks = (end - beg + kRowChunk - 1) / kRowChunk;
        for (uint64_t c = warp; c < chunks; c += nwarps) {
          const uint64_t a = beg + c * kRowChunk;
          bfs_gather(g, depth, a, a + kRowChunk < end ? a + kRowChunk : end, qout, cnext, level);
        }
      }
    }
    if (!grid_barrier(bar, err)) return;
    nfront = *(volatile uint32_t *)cnext;
    have_queue = !scan;
    if (!scan) {
      uint32_t *t = qin;
      qin = qout;
      qout = t;
    }
    if (tid == 0) {
      cnt[3] = 0;
      cnt[5] = 0;
    }
    ++level;
    // every block has read nfront and the queue pointers before anyone reuses them
    if (!grid_barrier(bar, err)) return;
  }
  if (tid == 0) cnt[4] = (uint32_t)level;
}

__global__ void k_bfs_setup(int32_t *depth, uint32_t src, uint32_t *q0, uint32_t *cnt, unsigned *bar) {
  depth[src] = 0;
  q0[0] = src;
  cnt[0] = 0;  // the level-0 frontier (src) is implicit; level L appends to cnt[(L + 1) % 3]
  cnt[1] = 0;
  cnt[2] = 0;
  cnt[3] = 0;
  cnt[4] = 0;
  cnt[5] = 0;
  bar[0] = 0;
  bar[1] = 0;
}

int run_bfs(const Geo &g, uint32_t src, int32_t *depth, uint32_t *q0, uint32_t *q1, uint32_t *q2,
            uint32_t *counter, uint32_t *h_counter, cudaStream_t s) {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_persist, 256, 0);
    grid = sms * (per_sm > 4 ? 4 : per_sm);
    if (grid < 1) grid = 1;
  }
  // counter layout: cnt[0..4], barrier words, error word
  uint32_t *cnt = counter;
  unsigned *bar = counter + 8;
  uint32_t *err = counter + 12;
  cudaMemsetAsync(depth, 0xFF, sizeof(int32_t) * g.V, s);
  cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
  note_launch();
  k_bfs_setup<<<1, 1, 0, s>>>(depth, src, q0, cnt, bar);
  const uint32_t scan_from = g.V / 32 > 64 ? g.V / 32 : 64;
  Geo gg = g;
  void *args[] = {(void *)&gg, (void *)&depth, (void *)&q0,  (void *)&q1,
                  (void *)&q2, (void *)&cnt,   (void *)&bar, (void *)&err, (void *)&scan_from};
  note_launch();
  if (cudaLaunchCooperativeKernel((const void *)k_bfs_persist, dim3(grid), dim3(256), args, 0, s) != cudaSuccess)
    return -1;
  cudaMemcpyAsync(h_counter, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  return *h_counter ? -2 : 0;  // -2: a bounded barrier wait gave up
}

// ---- connected components -------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cc_find(uint32_t *parent, uint32_t v) {
  volatile uint32_t *p = parent;
  uint32_t par = p[v];
  if (par != v) {
    uint32_t prev = v, next;
    while (par > (next = p[par])) {  // parents are never larger than their children
      p[prev] = next;                // path halving towards the root
      prev = par;
      par = next;
    }
  }
  return par;
}

__global__ void k_cc_init(uint32_t *label, uint32_t V) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) label[v] = v;
}

__global__ void __launch_bounds__(256) k_cc_hook(Geo g, uint32_t *label) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g.C; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = g.slots[e];
    if (k == kEmpty || is_guard(k)) continue;
    uint32_t a = (uint32_t)(k >> 32), b = (uint32_t)(k & 0xFFFFFFFFull);
    if (a == b) continue;
    for (;;) {
      a = cc_find(label, a);
      b = cc_find(label, b);
      if (a == b) break;
      if (a < b) {
        uint32_t t = a; a = b; b = t;
      }
      // hook the larger root under the smaller one
      const uint32_t old = atomicCAS(&label[a], a, b);
      if (old == a) break;
      a = old;
    }
  }
}

__global__ void k_cc_compress(uint32_t *label, uint32_t V) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x)
    label[v] = cc_find(label, v);
}

void launch_cc(const Geo &g, uint32_t *label, cudaStream_t s) {
  const uint32_t vb = nb(g.V, 256, 152 * 8);
  note_launch();
  k_cc_init<<<vb, 256, 0, s>>>(label, g.V);
  note_launch();
  k_cc_hook<<<nb(g.C, 256, 152 * 16), 256, 0, s>>>(g, label);
  note_launch();
  k_cc_compress<<<vb, 256, 0, s>>>(label, g.V);
}

}  // namespace gpk
