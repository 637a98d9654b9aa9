// k_analytics.cu -- graph analytics that read the gapped array in place
// (Sec. 4.2: every access tests IsEntryExist, i.e. skips EMPTY slots; guards
// delimit the rows).
//   PageRank  power iteration with a push SpMV over the slots (Sec. 6.1)
//   BFS       level-synchronous, one warp gathers one frontier vertex's row
//             (Algorithm "GPU-based BFS Neighbour Gathering"), ballot-compacted
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

// y[v] += x[u] / outdeg(u) for every stored edge u -> v; each thread keeps two
// 16-byte slot loads in flight
__global__ void __launch_bounds__(256) k_pr_scatter(Geo g, const float *__restrict__ contrib,
                                                    double *__restrict__ y) {
  const uint64_t npairs = g.C >> 1;
  const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(g.slots);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += 2 * stride) {
    const ulonglong2 k0 = __ldcs(s2 + p);
    const bool has1 = p + stride < npairs;
    const ulonglong2 k1 = has1 ? __ldcs(s2 + p + stride) : make_ulonglong2(kEmpty, kEmpty);
    const uint64_t ks[4] = {k0.x, k0.y, k1.x, k1.y};
#pragma unroll
    for (int q = 0; q < 4; q++)
      if (ks[q] != kEmpty && !is_guard(ks[q]))
        atomicAdd(&y[ks[q] & 0xFFFFFFFFull], (double)__ldg(contrib + (ks[q] >> 32)));
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
// Small frontiers: top-down from a queue, one warp per frontier vertex's row.
// Large frontiers: one pass over the whole gapped array, each stored edge u -> v
// with depth[u] == level claiming v (no queue); the queue is rebuilt from the
// depth array when the frontier shrinks again.
__global__ void k_bfs_init(int32_t *depth, uint32_t src, uint32_t *q0, uint32_t *counter) {
  depth[src] = 0;
  q0[0] = src;
  counter[0] = 1;
  counter[1] = 0;
}

__device__ __forceinline__ void block_count_add(uint32_t c, uint32_t *dst) {
  c = warp_sum(c);
  if (lane_id() == 0 && c) atomicAdd(dst, c);
}

// one warp per frontier vertex u: row u is (guard(u-1), guard(u)) in slot order
__global__ void __launch_bounds__(256) k_bfs_expand(Geo g, int32_t *__restrict__ depth, const uint32_t *__restrict__ qin,
                                                    const uint32_t *nin, uint32_t *__restrict__ qout, uint32_t *nout,
                                                    int32_t level) {
  const uint32_t lane = lane_id();
  const uint32_t nf = *nin;
  const uint32_t nw = gridDim.x * (blockDim.x >> 5);
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nf; i += nw) {
    const uint32_t u = qin[i];
    const uint64_t beg = u ? (uint64_t)g.row_end[u - 1] + 1 : 0, end = g.row_end[u];
    for (uint64_t s = beg; s < end; s += 32) {
      const uint64_t e = s + lane;
      bool got = false;
      uint32_t v = 0;
      if (e < end) {
        const uint64_t k = g.slots[e];
        if (k != kEmpty) {  // IsEntryExist
          v = (uint32_t)(k & 0xFFFFFFFFull);
          if (depth[v] < 0) got = atomicCAS(&depth[v], -1, level + 1) == -1;
        }
      }
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, got);
      if (bal) {
        uint32_t base = 0;
        if (lane == (uint32_t)(__ffs(bal) - 1)) base = atomicAdd(nout, (uint32_t)__popc(bal));
        base = __shfl_sync(0xFFFFFFFFu, base, __ffs(bal) - 1);
        if (got) qout[base + __popc(bal & lanemask_lt())] = v;
      }
    }
  }
}

// one pass over all slots for a large frontier; counts the newly reached vertices
__global__ void __launch_bounds__(256) k_bfs_scan(Geo g, int32_t *__restrict__ depth, uint32_t *nout, int32_t level) {
  const uint64_t npairs = g.C >> 1;
  const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(g.slots);
  uint32_t found = 0;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += (uint64_t)gridDim.x * blockDim.x) {
    const ulonglong2 kk = __ldcs(s2 + p);
    const uint64_t ks[2] = {kk.x, kk.y};
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const uint64_t k = ks[q];
      if (k == kEmpty || is_guard(k)) continue;
      if (__ldg(depth + (k >> 32)) != level) continue;
      const uint32_t v = (uint32_t)(k & 0xFFFFFFFFull);
      if (depth[v] < 0 && atomicCAS(&depth[v], -1, level + 1) == -1) ++found;
    }
  }
  block_count_add(found, nout);
}

// queue of the vertices at depth `level` (after a scan level)
__global__ void k_bfs_collect(const int32_t *__restrict__ depth, uint32_t V, int32_t level, uint32_t *q,
                              uint32_t *n) {
  const uint32_t vend = (V + 31) & ~31u;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < vend; v += gridDim.x * blockDim.x) {
    const bool hit = v < V && depth[v] == level;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, hit);
    if (!bal) continue;
    uint32_t base = 0;
    if (lane_id() == (uint32_t)(__ffs(bal) - 1)) base = atomicAdd(n, (uint32_t)__popc(bal));
    base = __shfl_sync(0xFFFFFFFFu, base, __ffs(bal) - 1);
    if (hit) q[base + __popc(bal & lanemask_lt())] = v;
  }
}

int run_bfs(const Geo &g, uint32_t src, int32_t *depth, uint32_t *q0, uint32_t *q1, uint32_t *counter,
            uint32_t *h_counter, cudaStream_t s) {
  cudaMemsetAsync(depth, 0xFF, sizeof(int32_t) * g.V, s);
  note_launch();
  k_bfs_init<<<1, 1, 0, s>>>(depth, src, q0, counter);
  // a pass over the array costs about C/2 warp loads; a frontier is expanded
  // top-down while it is small against that
  const uint64_t scan_from = g.V / 32 > 64 ? g.V / 32 : 64;
  uint32_t nfront = 1;
  int32_t level = 0;
  bool have_queue = true;
  uint32_t *qin = q0, *qout = q1;
  uint32_t *cin = counter, *cout = counter + 1;
  while (nfront) {
    cudaMemsetAsync(cout, 0, sizeof(uint32_t), s);
    const bool scan = nfront >= scan_from;
    if (scan) {
      note_launch();
      k_bfs_scan<<<nb(g.C >> 1, 256, 152 * 8), 256, 0, s>>>(g, depth, cout, level);
    } else {
      if (!have_queue) {
        cudaMemsetAsync(cin, 0, sizeof(uint32_t), s);
        note_launch();
        k_bfs_collect<<<nb(g.V, 256, 152 * 4), 256, 0, s>>>(depth, g.V, level, qin, cin);
      }
      note_launch();
      k_bfs_expand<<<nb(nfront, 8, 152 * 16), 256, 0, s>>>(g, depth, qin, cin, qout, cout, level);
    }
    cudaMemcpyAsync(h_counter, cout, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    nfront = *h_counter;
    have_queue = !scan;
    uint32_t *t = qin; qin = qout; qout = t;
    uint32_t *c = cin; cin = cout; cout = c;
    ++level;
  }
  return level;
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
