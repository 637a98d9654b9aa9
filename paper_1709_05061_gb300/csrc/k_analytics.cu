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
__device__ __forceinline__ void block_add_double(double v, double *dst) {
  __shared__ double ws[32];
  v = warp_sum(v);
  if (lane_id() == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    x = warp_sum(x);
    if (threadIdx.x == 0 && x != 0.0) atomicAdd(dst, x);
  }
  __syncthreads();
}

__global__ void k_pr_init(uint32_t V, const uint32_t *__restrict__ deg, float *__restrict__ x,
                          float *__restrict__ contrib, double *__restrict__ y, double *dsum0) {
  const float x0 = (float)(1.0 / (double)V);
  double dang = 0.0;
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t vend = (V + blockDim.x - 1) / blockDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < vend; v += stride) {
    if (v < V) {
      const uint32_t d = deg[v];
      x[v] = x0;
      y[v] = 0.0;
      contrib[v] = d ? x0 / (float)d : 0.0f;
      if (!d) dang += (double)x0;
    }
  }
  block_add_double(dang, dsum0);
}

// y[v] += x[u] / outdeg(u) for every stored edge u -> v (16-byte slot loads)
__global__ void __launch_bounds__(256) k_pr_scatter(Geo g, const float *__restrict__ contrib,
                                                    double *__restrict__ y) {
  const uint64_t npairs = g.C >> 1;
  const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(g.slots);
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += (uint64_t)gridDim.x * blockDim.x) {
    ulonglong2 kk = __ldcs(s2 + p);
    if (kk.x != kEmpty && !is_guard(kk.x))
      atomicAdd(&y[kk.x & 0xFFFFFFFFull], (double)__ldg(contrib + (kk.x >> 32)));
    if (kk.y != kEmpty && !is_guard(kk.y))
      atomicAdd(&y[kk.y & 0xFFFFFFFFull], (double)__ldg(contrib + (kk.y >> 32)));
  }
}

__global__ void k_pr_apply(uint32_t V, float damping, const uint32_t *__restrict__ deg, double *__restrict__ y,
                           float *__restrict__ x, float *__restrict__ contrib, const double *dsum_in,
                           double *dsum_out) {
  const double base = (1.0 - (double)damping) / (double)V;
  const double dn = *dsum_in / (double)V;
  double dang = 0.0;
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t vend = (V + blockDim.x - 1) / blockDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < vend; v += stride) {
    if (v < V) {
      const double nx = base + (double)damping * (y[v] + dn);
      const float xf = (float)nx;
      const uint32_t d = deg[v];
      x[v] = xf;
      y[v] = 0.0;
      contrib[v] = d ? xf / (float)d : 0.0f;
      if (!d) dang += (double)xf;
    }
  }
  block_add_double(dang, dsum_out);
}

void launch_pr_setup(const Geo &g, uint32_t iters, float *rank, uint32_t *deg, double *y, float *contrib,
                     double *dsum, cudaStream_t s) {
  launch_degrees(g, deg, s);
  cudaMemsetAsync(dsum, 0, sizeof(double) * (iters + 1), s);
  note_launch();
  k_pr_init<<<nb(g.V, 256, 152 * 8), 256, 0, s>>>(g.V, deg, rank, contrib, y, dsum);
}

void launch_pr_scatter(const Geo &g, const float *contrib, double *y, cudaStream_t s) {
  note_launch();
  k_pr_scatter<<<nb(g.C >> 1, 256, 152 * 16), 256, 0, s>>>(g, contrib, y);
}

void launch_pr_apply(const Geo &g, float damping, float *rank, const uint32_t *deg, double *y, float *contrib,
                     const double *dsum_in, double *dsum_out, cudaStream_t s) {
  note_launch();
  k_pr_apply<<<nb(g.V, 256, 152 * 8), 256, 0, s>>>(g.V, damping, deg, y, rank, contrib, dsum_in, dsum_out);
}

// ---- BFS ----------------------------------------------------------------------------------------
__global__ void k_bfs_init(int32_t *depth, uint32_t src, uint32_t *q0, uint32_t *counter) {
  depth[src] = 0;
  q0[0] = src;
  counter[0] = 1;
  counter[1] = 0;
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

int run_bfs(const Geo &g, uint32_t src, int32_t *depth, uint32_t *q0, uint32_t *q1, uint32_t *counter,
            uint32_t *h_counter, cudaStream_t s) {
  cudaMemsetAsync(depth, 0xFF, sizeof(int32_t) * g.V, s);
  note_launch();
  k_bfs_init<<<1, 1, 0, s>>>(depth, src, q0, counter);
  uint32_t nfront = 1;
  int32_t level = 0;
  uint32_t *qin = q0, *qout = q1;
  uint32_t *cin = counter, *cout = counter + 1;
  while (nfront) {
    cudaMemsetAsync(cout, 0, sizeof(uint32_t), s);
    note_launch();
    k_bfs_expand<<<nb(nfront, 8, 152 * 16), 256, 0, s>>>(g, depth, qin, cin, qout, cout, level);
    cudaMemcpyAsync(h_counter, cout, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    nfront = *h_counter;
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
