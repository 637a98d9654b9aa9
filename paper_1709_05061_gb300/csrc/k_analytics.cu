// k_analytics.cu -- graph analytics that read the gapped array in place
// (Sec. 4.2: every access tests IsEntryExist, i.e. skips EMPTY slots; guards
// delimit the rows).
//   PageRank  power iteration (Sec. 6.1) with exact fixed-point sums: by default
//             the edges are bucketed by head once per call and every iteration sums
//             each bucket in shared memory; or a push SpMV over the slots
//   BFS       level-synchronous in one persistent cooperative kernel: a warp gathers
//             a frontier vertex's row for small frontiers, one pass over the array
//             for large ones
//   CC        lock-free union-find (sampled first pass, then every edge); a root is
//             always the smallest id of its tree, so labels are component minima
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
// Sums are exact: every contribution x_u / outdeg(u) is formed in FP32 and
// rounded once to a 64-bit fixed-point number with 60 fractional bits (all ranks
// and sums are <= 1), and the scatter adds integers, so the result does not
// depend on the order in which the reductions land.  Ranks are FP32 and the
// per-vertex arithmetic stays in FP32 and integer units.

// Conversions between FP32 and the 2^60 fixed point use integer operations only
// (GB300's FP64 pipe is narrow and 64-bit int <-> float conversions run there).
// fx(v) = round(v * 2^60) for v in [0, 1]: mantissa shifted by its exponent.
__device__ __forceinline__ uint64_t to_fx(float v) {
  const uint32_t b = __float_as_uint(v);
  const int32_t ex = (int32_t)((b >> 23) & 0xFFu);
  if (ex == 0) return 0ull;  // zero (no subnormal contribution matters at 2^-60)
  const uint64_t m = (uint64_t)((b & 0x7FFFFFu) | 0x800000u);
  const int32_t sh = ex - 127 - 23 + 60;  // value = m * 2^(ex - 150); times 2^60
  if (sh >= 0) return m << sh;
  if (sh <= -64) return 0ull;
  return (m + (1ull << (-sh - 1))) >> (-sh);  // round half up
}

// y * 2^-60 as FP32 from the two 32-bit halves: hi * 2^-28 + lo * 2^-60
__device__ __forceinline__ float fx_to_float(uint64_t y) {
  return __uint2float_rn((uint32_t)(y >> 32)) * 3.7252902984619140625e-09f +
         __uint2float_rn((uint32_t)y) * 8.6736173798840354720e-19f;
}

// Sum of one u64 per thread over the grid: per-block partials, and the last
// block to finish adds them (integers: exact, any order).
__device__ __forceinline__ void grid_sum_u64(uint64_t v, uint64_t *partials, unsigned *counter, uint64_t *out) {
  __shared__ uint64_t ws[32];
  __shared__ bool last;
  v = warp_sum(v);
  if (lane_id() == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t b = 0;
    for (uint32_t q = 0; q < (blockDim.x >> 5); q++) b += ws[q];
    partials[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    uint64_t t = 0;
    const volatile uint64_t *vp = partials;
    for (uint32_t q = threadIdx.x; q < gridDim.x; q += blockDim.x) t += vp[q];
    t = warp_sum(t);
    if (lane_id() == 0) ws[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t tot = 0;
      for (uint32_t q = 0; q < (blockDim.x >> 5); q++) tot += ws[q];
      *out = tot;
      *counter = 0;
    }
  }
}

// Contributions x_u / outdeg(u) are kept as fixed point (push pass: cfx) or as
// the FP32 quotient (bucketed pass: cf, converted per edge), the same value either way.
__global__ void k_pr_init(uint32_t V, const uint32_t *__restrict__ deg, float *__restrict__ x,
                          uint64_t *__restrict__ cfx, float *__restrict__ cf, uint64_t *__restrict__ y,
                          uint64_t *dsum0, uint64_t *partials, unsigned *counter) {
  const float x0 = __fdiv_rn(1.0f, (float)V);
  uint64_t dang = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
    const uint32_t d = deg[v];
    x[v] = x0;
    const float q = d ? __fdiv_rn(x0, (float)d) : 0.0f;
    if (cf) {
      cf[v] = q;
    } else {
      y[v] = 0;
      cfx[v] = to_fx(q);
    }
    if (!d) dang += to_fx(x0);
  }
  grid_sum_u64(dang, partials, counter, dsum0);
}

// y[v] += fx(x_u / outdeg(u)) for every stored edge u -> v.  Each thread owns two
// 16-byte slot pairs per step and loads the next step's pairs before it works on
// the current ones.
__device__ __forceinline__ void pr_push(uint64_t k, const uint64_t *__restrict__ cfx, uint64_t *__restrict__ y) {
  if (k != kEmpty && !is_guard(k))
    atomicAdd((unsigned long long *)&y[k & 0xFFFFFFFFull], (unsigned long long)__ldg(cfx + (k >> 32)));
}

// 32-bit indices (C <= 2^32 slots) keep the pass at 32 registers: eight resident
// blocks per SM, four 16-byte slot loads in flight per thread
__global__ void __launch_bounds__(256, 8) k_pr_scatter(const ulonglong2 *__restrict__ s2, uint32_t npairs,
                                                       const uint64_t *__restrict__ cfx, uint64_t *__restrict__ y) {
  const uint32_t stride = gridDim.x * blockDim.x;
  const ulonglong2 none = make_ulonglong2(kEmpty, kEmpty);
  uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  ulonglong2 a = p < npairs ? __ldcs(s2 + p) : none;
  ulonglong2 b = p + stride < npairs ? __ldcs(s2 + p + stride) : none;
  while (p < npairs) {
    const uint32_t q = p + 2 * stride;
    const ulonglong2 na = q < npairs ? __ldcs(s2 + q) : none;
    const ulonglong2 nb = q + stride < npairs ? __ldcs(s2 + q + stride) : none;
    pr_push(a.x, cfx, y);
    pr_push(a.y, cfx, y);
    pr_push(b.x, cfx, y);
    pr_push(b.y, cfx, y);
    a = na;
    b = nb;
    p = q;
  }
}

__global__ void k_pr_apply(uint32_t V, float damping, const uint32_t *__restrict__ deg, uint64_t *__restrict__ y,
                           float *__restrict__ x, uint64_t *__restrict__ cfx, const uint64_t *dsum_in,
                           uint64_t *dsum_out, uint64_t *partials, unsigned *counter, int write_x) {
  // x' = (1 - d)/V + d * (y + dangling / V), all in FP32 (the sums themselves are exact)
  const float base = __fdiv_rn(1.0f - damping, (float)V);
  const float dn = __fdiv_rn(fx_to_float(*dsum_in), (float)V);
  uint64_t dang = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
    const uint32_t d = deg[v];
    const float xf = __fmaf_rn(damping, fx_to_float(y[v]) + dn, base);
    if (write_x) x[v] = xf;  // the ranks are read only after the last iteration
    y[v] = 0;
    cfx[v] = d ? to_fx(__fdiv_rn(xf, (float)d)) : 0ull;
    if (!d) dang += to_fx(xf);
  }
  grid_sum_u64(dang, partials, counter, dsum_out);
}

// ---- bucketed PageRank pass ----------------------------------------------------------------------
// Once per call the stored edges are copied into buckets by head (v >> 13, a
// counting sort by chunk of the array: per-chunk bucket counts, a scan, a
// placement pass).  Every iteration then gives each bucket a cluster of blocks;
// each block sums the contributions of its share of the bucket into an 8192-entry
// table in shared memory, and the cluster adds its tables through distributed
// shared memory and applies the update.  The random reductions of the push pass
// become shared-memory atomics.  The copy keeps the chunks in slot order, so
// within a bucket the tails (and the contribution loads) move forward through
// the array.  Each 64-bit sum is kept as two 32-bit words: the low word's atomic
// returns the old value, and a carry out of it is added to the high word with
// the high half, so the sum is exact modulo 2^64 whatever the order, as in the
// push pass.
__global__ void __launch_bounds__(256) k_pb_count(const ulonglong2 *__restrict__ s2, uint64_t npairs, uint64_t chunk,
                                                  uint32_t nb, uint32_t shift, uint32_t *__restrict__ cnt,
                                                  uint32_t *__restrict__ tot) {
  __shared__ uint32_t hist[kPbMaxBuckets];
  for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const uint64_t p0 = (uint64_t)blockIdx.x * chunk, p1 = p0 + chunk < npairs ? p0 + chunk : npairs;
  for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const ulonglong2 k = __ldcs(s2 + p);
    if (k.x != kEmpty && !is_guard(k.x)) atomicAdd(&hist[(uint32_t)k.x >> shift], 1u);
    if (k.y != kEmpty && !is_guard(k.y)) atomicAdd(&hist[(uint32_t)k.y >> shift], 1u);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
    cnt[(uint64_t)b * gridDim.x + blockIdx.x] = hist[b];
    if (hist[b]) atomicAdd(&tot[b], hist[b]);
  }
}

// Offsets of the bucketed copy: off[b * G + c] = edges of smaller buckets plus
// bucket b's edges in chunks before c (off[nb * G] = all edges).  One block per
// bucket; tot[b] = bucket b's edges.
__global__ void __launch_bounds__(256) k_pb_offsets(const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ tot,
                                                    uint64_t *__restrict__ off, uint32_t G, uint32_t nb) {
  __shared__ uint32_t wsum[33];
  __shared__ unsigned long long s_base;
  const uint32_t b = blockIdx.x;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  unsigned long long part = 0;
  for (uint32_t e = threadIdx.x; e < b; e += blockDim.x) part += tot[e];
  part = warp_sum(part);
  if (lane_id() == 0 && part) atomicAdd(&s_base, part);
  __syncthreads();
  uint64_t carry = s_base;
  const uint32_t *col = cnt + (uint64_t)b * G;
  uint64_t *o = off + (uint64_t)b * G;
  constexpr uint32_t kPer = 8;
  for (uint32_t c0 = 0; c0 < G; c0 += 256 * kPer) {
    const uint32_t t0 = c0 + threadIdx.x * kPer;
    uint32_t v[kPer], loc = 0;
#pragma unroll
    for (uint32_t q = 0; q < kPer; q++) {
      v[q] = t0 + q < G ? col[t0 + q] : 0u;
      loc += v[q];
    }
    uint32_t total;
    uint64_t run = carry + block_excl_scan(loc, wsum, &total);
#pragma unroll
    for (uint32_t q = 0; q < kPer; q++) {
      if (t0 + q < G) o[t0 + q] = run;
      run += v[q];
    }
    carry += total;
  }
  if (b + 1 == nb && threadIdx.x == 0) off[(uint64_t)nb * G] = carry;
}

// Placement, one tile of kPbTile slots at a time: the tile's edges are ranked
// within their bucket (shared-memory counters), the counts scanned, the edges
// staged in bucket order in shared memory, and then written out so that the
// edges of one bucket go to consecutive addresses.
__global__ void __launch_bounds__(kPbPlaceThreads, 3) k_pb_place(const ulonglong2 *__restrict__ s2, uint64_t npairs,
                                                              uint64_t chunk, uint32_t nb, uint32_t shift,
                                                              const uint64_t *__restrict__ off,
                                                              uint64_t *__restrict__ keys) {
  extern __shared__ uint64_t pb_smem[];
  uint64_t *stage = pb_smem;                                         // kPbTile keys
  uint32_t *toff = reinterpret_cast<uint32_t *>(stage + kPbTile);    // nb + 1: counts, then offsets
  uint32_t *cur = toff + nb + 1;                                     // nb: placed so far in this chunk
  __shared__ uint32_t wsum[33];
  constexpr uint32_t kPer = kPbTile / 2 / kPbPlaceThreads;           // slot pairs per thread per tile
  const uint32_t t = threadIdx.x;
  const uint32_t per = (nb + 1 + kPbPlaceThreads - 1) / kPbPlaceThreads;  // scan entries per thread
  for (uint32_t b = t; b < nb; b += kPbPlaceThreads) cur[b] = 0;
  const uint64_t p0 = (uint64_t)blockIdx.x * chunk, p1 = p0 + chunk < npairs ? p0 + chunk : npairs;
  for (uint64_t tp = p0; tp < p1; tp += kPbTile / 2) {
    for (uint32_t b = t; b <= nb; b += kPbPlaceThreads) toff[b] = 0;
    __syncthreads();
    uint64_t k[2 * kPer];
    uint32_t r[2 * kPer];
#pragma unroll
    for (uint32_t u = 0; u < kPer; u++) {
      const uint64_t p = tp + u * kPbPlaceThreads + t;
      const ulonglong2 v = p < p1 ? __ldcs(s2 + p) : make_ulonglong2(kEmpty, kEmpty);
      k[2 * u] = (v.x != kEmpty && !is_guard(v.x)) ? v.x : kEmpty;
      k[2 * u + 1] = (v.y != kEmpty && !is_guard(v.y)) ? v.y : kEmpty;
    }
#pragma unroll
    for (uint32_t j = 0; j < 2 * kPer; j++)
      if (k[j] != kEmpty) r[j] = atomicAdd(&toff[(uint32_t)k[j] >> shift], 1u);
    __syncthreads();
    // exclusive scan of the nb counts (toff[nb] = 0 before, the tile's total after)
    uint32_t loc = 0;
    for (uint32_t e = 0; e < per; e++) {
      const uint32_t b = t * per + e;
      if (b <= nb) loc += toff[b];
    }
    uint32_t total;
    uint32_t run = block_excl_scan(loc, wsum, &total);
    for (uint32_t e = 0; e < per; e++) {
      const uint32_t b = t * per + e;
      if (b <= nb) {
        const uint32_t c = toff[b];
        toff[b] = run;
        run += c;
      }
    }
    __syncthreads();
#pragma unroll
    for (uint32_t j = 0; j < 2 * kPer; j++)
      if (k[j] != kEmpty) stage[toff[(uint32_t)k[j] >> shift] + r[j]] = k[j];
    __syncthreads();
    const uint32_t n = toff[nb];
    for (uint32_t i = t; i < n; i += kPbPlaceThreads) {
      const uint64_t key = stage[i];
      const uint32_t b = (uint32_t)key >> shift;
      keys[__ldg(off + (uint64_t)b * gridDim.x + blockIdx.x) + cur[b] + (i - toff[b])] = key;
    }
    __syncthreads();
    for (uint32_t b = t; b < nb; b += kPbPlaceThreads) cur[b] += toff[b + 1] - toff[b];
    __syncthreads();
  }
}

// Placement without staging, for many buckets (a tile then holds about one edge
// per bucket, so staging would not group the writes): each edge goes straight to
// its bucket's next free position of this chunk.
__global__ void __launch_bounds__(256) k_pb_place_direct(const ulonglong2 *__restrict__ s2, uint64_t npairs,
                                                         uint64_t chunk, uint32_t nb, uint32_t shift,
                                                         const uint64_t *__restrict__ off,
                                                         uint64_t *__restrict__ keys) {
  __shared__ uint32_t cur[kPbMaxBuckets];
  __shared__ uint64_t base[kPbMaxBuckets];
  for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
    cur[b] = 0;
    base[b] = off[(uint64_t)b * gridDim.x + blockIdx.x];
  }
  __syncthreads();
  const uint64_t p0 = (uint64_t)blockIdx.x * chunk, p1 = p0 + chunk < npairs ? p0 + chunk : npairs;
  for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const ulonglong2 k = __ldcs(s2 + p);
    if (k.x != kEmpty && !is_guard(k.x)) {
      const uint32_t b = (uint32_t)k.x >> shift;
      keys[base[b] + atomicAdd(&cur[b], 1u)] = k.x;
    }
    if (k.y != kEmpty && !is_guard(k.y)) {
      const uint32_t b = (uint32_t)k.y >> shift;
      keys[base[b] + atomicAdd(&cur[b], 1u)] = k.y;
    }
  }
}

// Cluster primitives (sm_90+): a barrier over the blocks of a cluster that also
// orders their shared-memory writes, and 32-bit loads from another block's shared
// memory (distributed shared memory).
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_smem_addr(const void *p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// One PageRank iteration over the bucketed copy.  A cluster of nparts blocks owns
// bucket b; block q sums its share of the bucket's edges into its own table, then
// (after a cluster barrier) adds the nparts tables over its share of the bucket's
// heads through distributed shared memory and applies the update there:
// x'_v = (1-d)/V + d * (y_v + dangling/V), the next contribution x'_v/outdeg(v)
// into cf_out, and the dangling mass of the next iteration by a grid sum.
template <uint32_t TPB>
__global__ void __launch_bounds__(TPB) k_pb_iter(const uint64_t *__restrict__ keys,
                                                        const uint64_t *__restrict__ off, uint32_t G, uint32_t shift,
                                                        uint32_t nparts,
                                                        uint32_t V, float damping, const uint32_t *__restrict__ deg,
                                                        const float *__restrict__ cf_in, float *__restrict__ cf_out,
                                                        float *__restrict__ x, int write_x, const uint64_t *dsum_in,
                                                        uint64_t *dsum_out, uint64_t *partials, unsigned *counter) {
  extern __shared__ uint32_t pb_tab[];  // low words, then high words, 2^shift each
  const uint32_t bs = 1u << shift;
  uint32_t *lo = pb_tab, *hi = pb_tab + bs;
  const uint32_t b = blockIdx.x / nparts, q = blockIdx.x % nparts;  // q is the rank in the cluster
  for (uint32_t i = threadIdx.x; i < bs; i += TPB) lo[i] = hi[i] = 0;
  __syncthreads();
  const uint64_t e0 = off[(uint64_t)b * G], len = off[(uint64_t)(b + 1) * G] - e0;
  const uint64_t a = e0 + len * q / nparts, z = e0 + len * (q + 1) / nparts;
  for (uint64_t i0 = a; i0 < z; i0 += 4 * TPB) {
    uint64_t k[4];
    float c[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint64_t i = i0 + u * TPB + threadIdx.x;
      k[u] = i < z ? __ldcs(keys + i) : kEmpty;
    }
#pragma unroll
    for (int u = 0; u < 4; u++) c[u] = k[u] != kEmpty ? __ldg(cf_in + (k[u] >> 32)) : 0.0f;
#pragma unroll
    for (int u = 0; u < 4; u++) {
      if (k[u] == kEmpty) continue;
      const uint64_t fx = to_fx(c[u]);
      const uint32_t dl = (uint32_t)k[u] & (bs - 1), cl = (uint32_t)fx;
      const uint32_t old = atomicAdd(&lo[dl], cl);
      atomicAdd(&hi[dl], (uint32_t)(fx >> 32) + ((uint32_t)(old + cl) < old ? 1u : 0u));
    }
  }
  cluster_barrier();
  const float base = __fdiv_rn(1.0f - damping, (float)V);
  const float dn = __fdiv_rn(fx_to_float(*dsum_in), (float)V);
  uint64_t dang = 0;
  const uint32_t h0 = q * bs / nparts, h1 = (q + 1) * bs / nparts;
  for (uint32_t e = h0 + threadIdx.x; e < h1; e += TPB) {
    uint64_t y = 0;
    for (uint32_t r = 0; r < nparts; r++)
      y += ((uint64_t)ld_cluster_u32(cluster_smem_addr(hi + e, r)) << 32) | ld_cluster_u32(cluster_smem_addr(lo + e, r));
    const uint32_t v = b * bs + e;
    if (v < V) {
      const uint32_t d = deg[v];
      const float xf = __fmaf_rn(damping, fx_to_float(y) + dn, base);
      if (write_x) x[v] = xf;
      cf_out[v] = d ? __fdiv_rn(xf, (float)d) : 0.0f;
      if (!d) dang += to_fx(xf);
    }
  }
  cluster_barrier();  // no block leaves while another still reads its tables
  grid_sum_u64(dang, partials, counter, dsum_out);
}

constexpr uint32_t kVecBlocks = 152 * 8;  // grid of the per-vertex kernels (and partials per sum)

void launch_pr_setup(const Geo &g, uint32_t iters, float *rank, uint64_t *y, uint64_t *cfx, float *cf,
                     uint64_t *dsum, uint64_t *partials, unsigned *counter, cudaStream_t s) {
  cudaMemsetAsync(dsum, 0, sizeof(uint64_t) * (iters + 1), s);
  cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  note_launch();
  k_pr_init<<<nb(g.V, 256, kVecBlocks), 256, 0, s>>>(g.V, g.deg, rank, cfx, cf, y, dsum, partials, counter);
}

void launch_pr_scatter(const Geo &g, const uint64_t *cfx, uint64_t *y, cudaStream_t s) {
  note_launch();
  k_pr_scatter<<<nb(g.C >> 2, 256, 152 * 8), 256, 0, s>>>(reinterpret_cast<const ulonglong2 *>(g.slots),
                                                           (uint32_t)(g.C >> 1), cfx, y);
}

void launch_pr_apply(const Geo &g, float damping, float *rank, uint64_t *y, uint64_t *cfx,
                     const uint64_t *dsum_in, uint64_t *dsum_out, uint64_t *partials, unsigned *counter,
                     bool last, cudaStream_t s) {
  note_launch();
  k_pr_apply<<<nb(g.V, 256, kVecBlocks), 256, 0, s>>>(g.V, damping, g.deg, y, rank, cfx, dsum_in, dsum_out,
                                                         partials, counter, last ? 1 : 0);
}

PbPlan pb_plan(const Geo &g) {
  PbPlan p;
  // 8192 heads a bucket (a 64 KB table): a warp's 32 edges then span half as
  // many contribution lines as with 4096 heads (measured, one iteration at R-MAT
  // scale 20: 0.058 ms against 0.062 ms with 4096 heads and 0.097 ms with 16384)
  p.shift = kPbShift;
  p.nb = (uint32_t)((g.V + (1u << p.shift) - 1) >> p.shift);
  const uint64_t npairs = g.C >> 1;
  uint64_t G = (npairs + 2047) / 2048;
  if (G < 1) G = 1;
  if (G > kPbMaxChunks) G = kPbMaxChunks;
  p.G = (uint32_t)G;
  p.chunk = (npairs + G - 1) / G;
  // blocks per bucket: a power of two (the cluster size), at most kPbMaxParts, for
  // a grid of about kPbTargetBlocks blocks of 1024 threads: one wave at two blocks
  // an SM (measured at R-MAT scale 20, 8192-head buckets, one iteration alone:
  // 2 blocks a bucket 0.0565 ms, 4 blocks 0.0598 ms, 8 blocks 0.074 ms, 1 block
  // 0.068 ms; 512 threads with 4 blocks a bucket 0.072 ms)
  const uint32_t want = (kPbTargetBlocks + p.nb - 1) / p.nb;
  p.nparts = 1;
  while (p.nparts * 2 <= want && p.nparts * 2 <= kPbMaxParts) p.nparts *= 2;
  p.threads = 1024;
  return p;
}

void launch_pb_build(const Geo &g, const PbPlan &p, uint32_t *cnt, uint64_t *off, uint64_t *scan_tmp, uint64_t *keys,
                     cudaStream_t s) {
  const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(g.slots);
  uint32_t *tot = reinterpret_cast<uint32_t *>(scan_tmp);  // nb bucket totals
  cudaMemsetAsync(tot, 0, sizeof(uint32_t) * p.nb, s);
  note_launch();
  k_pb_count<<<p.G, 256, 0, s>>>(s2, g.C >> 1, p.chunk, p.nb, p.shift, cnt, tot);
  note_launch();
  k_pb_offsets<<<p.nb, 256, 0, s>>>(cnt, tot, off, p.G, p.nb);
  if (p.nb > kPbStageMax) {
    note_launch();
    k_pb_place_direct<<<p.G, 256, 0, s>>>(s2, g.C >> 1, p.chunk, p.nb, p.shift, off, keys);
    return;
  }
  const size_t smem = sizeof(uint64_t) * kPbTile + sizeof(uint32_t) * (2 * p.nb + 1);
  static bool big = false;
  if (!big) {
    cudaFuncSetAttribute(k_pb_place, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(uint64_t) * kPbTile + sizeof(uint32_t) * (2 * kPbMaxBuckets + 1)));
    big = true;
  }
  note_launch();
  k_pb_place<<<p.G, kPbPlaceThreads, smem, s>>>(s2, g.C >> 1, p.chunk, p.nb, p.shift, off, keys);
}

void launch_pb_iter(const Geo &g, const PbPlan &p, const uint64_t *keys, const uint64_t *off, float damping,
                    const float *cf_in, float *cf_out, float *rank, bool last, const uint64_t *dsum_in,
                    uint64_t *dsum_out, uint64_t *partials, unsigned *counter, cudaStream_t s) {
  static bool big = false;
  if (!big) {
    cudaFuncSetAttribute(k_pb_iter<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8u << kPbMaxShift));
    big = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.nb * p.nparts);
  cfg.blockDim = dim3(p.threads);
  cfg.dynamicSmemBytes = 8u << p.shift;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = p.nparts;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  note_launch();
  auto kern = k_pb_iter<1024>;
  cudaLaunchKernelEx(&cfg, kern, keys, off, p.G, p.shift, p.nparts, g.V, damping, (const uint32_t *)g.deg, cf_in, cf_out,
                     rank, last ? 1 : 0, dsum_in, dsum_out, partials, counter);
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
// (frontier sizes), cnt[3..4] are the queue-rebuild counters of even and odd
// levels, cnt[5] the level count.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, uint32_t *err, uint32_t limit) {
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
        if (++spins > limit) {
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

// cnt[0..2]: frontier sizes (rotating), cnt[3..4]: queue rebuild (by level parity),
// cnt[5]: levels, cnt[6..7] / cnt[8..9]: one u64 per level parity = (long rows
// listed << 32) | chunks of those rows.  A level zeroes the next level's counters
// when it starts (their last users finished before this level's first barrier),
// so a level needs no barrier after its last one.  `big` holds
// (row, first chunk) pairs
__global__ void __launch_bounds__(256) k_bfs_persist(Geo g, int32_t *depth, uint32_t *qa, uint32_t *qb,
                                                     uint32_t *big, uint32_t *cnt, unsigned *bar, uint32_t *err,
                                                     uint32_t scan_from, const Ctl *ctl) {
  const uint32_t lane = lane_id();
  const uint32_t limit = spin_limit(ctl, kBarrierSpinLimit);
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
    const uint32_t par = (uint32_t)level & 1u;
    if (tid == 0) {
      cnt[(level + 2) % 3] = 0;
      cnt[3 + (par ^ 1u)] = 0;      // next level's queue-rebuild counter
      cnt[6 + 2 * (par ^ 1u)] = 0;  // next level's long-row list
      cnt[7 + 2 * (par ^ 1u)] = 0;
    }
    const bool scan = nfront >= scan_from;
    if (scan) {
      // one pass over the array: edges u -> v with depth[u] == level claim v
      // four 16-byte loads in flight per thread, then the sources' depths together
      uint32_t found = 0;
      for (uint64_t p = tid; p < npairs; p += 4 * nthreads) {
        uint64_t ks[8];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const uint64_t pq = p + (uint64_t)q * nthreads;
          const ulonglong2 kk = pq < npairs ? __ldcs(s2 + pq) : make_ulonglong2(kEmpty, kEmpty);
          ks[2 * q] = kk.x;
          ks[2 * q + 1] = kk.y;
        }
        int32_t du[8];
#pragma unroll
        for (int q = 0; q < 8; q++)
          du[q] = (ks[q] != kEmpty && !is_guard(ks[q])) ? __ldcg(depth + (ks[q] >> 32)) : -2;
#pragma unroll
        for (int q = 0; q < 8; q++) {
          if (du[q] != level) continue;
          const uint32_t v = (uint32_t)(ks[q] & 0xFFFFFFFFull);
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
          if (lane == (uint32_t)(__ffs(bal) - 1)) base = atomicAdd(cnt + 3 + par, (uint32_t)__popc(bal));
          base = __shfl_sync(0xFFFFFFFFu, base, __ffs(bal) - 1);
          if (hit) qin[base + __popc(bal & lanemask_lt())] = v;
        }
        if (!grid_barrier(bar, err, limit)) return;
      }
      // top-down: a warp per short row; long rows are listed with the running
      // total of their 256-slot chunks (one packed 64-bit atomic keeps the list
      // order and the chunk bases consistent), then all warps share the chunks
      unsigned long long *bigctr = reinterpret_cast<unsigned long long *>(cnt + 6 + 2 * par);
      for (uint32_t i = warp; i < nfront; i += nwarps) {
        const uint32_t u = __ldcg(qin + i);
        const uint64_t beg = u ? (uint64_t)__ldg(g.row_end + u - 1) + 1 : 0, end = __ldg(g.row_end + u);
        if (end - beg > kBigRow) {
          if (lane == 0) {
            const uint32_t nch = (uint32_t)((end - beg + kRowChunk - 1) / kRowChunk);
            const unsigned long long old = atomicAdd(bigctr, (1ull << 32) | nch);
            big[2 * (old >> 32)] = u;
            big[2 * (old >> 32) + 1] = (uint32_t)old;  // first chunk of this row
          }
          continue;
        }
        bfs_gather(g, depth, beg, end, qout, cnext, level);
      }
      if (!grid_barrier(bar, err, limit)) return;
      const unsigned long long bc = *(volatile unsigned long long *)bigctr;
      const uint32_t nbig = (uint32_t)(bc >> 32), nchunks = (uint32_t)bc;
      for (uint32_t c = warp; c < nchunks; c += nwarps) {
        uint32_t lo = 0, hi = nbig;  // last listed row whose first chunk is <= c
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (__ldcg(big + 2 * mid + 1) <= c) lo = mid; else hi = mid;
        }
        const uint32_t u = __ldcg(big + 2 * lo);
        const uint64_t beg = u ? (uint64_t)__ldg(g.row_end + u - 1) + 1 : 0, end = __ldg(g.row_end + u);
        const uint64_t a = beg + (uint64_t)(c - __ldcg(big + 2 * lo + 1)) * kRowChunk;
        bfs_gather(g, depth, a, a + kRowChunk < end ? a + kRowChunk : end, qout, cnext, level);
      }
    }
    if (!grid_barrier(bar, err, limit)) return;
    nfront = *(volatile uint32_t *)cnext;
    have_queue = !scan;
    if (!scan) {
      uint32_t *t = qin;
      qin = qout;
      qout = t;
    }
    ++level;
  }
  if (tid == 0) cnt[5] = (uint32_t)level;
}

__global__ void k_bfs_setup(int32_t *depth, uint32_t src, uint32_t *q0, uint32_t *cnt, unsigned *bar) {
  depth[src] = 0;
  q0[0] = src;
  // the level-0 frontier (src) is implicit; level L appends to cnt[(L + 1) % 3]
  for (int i = 0; i < 16; i++) cnt[i] = 0;
  bar[0] = 0;
  bar[1] = 0;
}

// a barrier wait that gave up becomes the handle's sticky timeout error
__global__ void k_bfs_flag(const uint32_t *err, Ctl *ctl) {
  if (*err) atomicOr(&ctl->sticky, kErrTimeout);
}

// resident blocks of the persistent BFS kernel per SM (it holds them for the whole
// search, so it also sets how much of the GPU a concurrent PageRank keeps).
// Measured in the bench step (R-MAT scale 20, BFS and CC beside PageRank-20): 2
// blocks 2.26 ms per step against 2.39 with 4 and 2.29 with 1 (BFS alone takes
// longer with fewer blocks, but the PageRank bucketing beside it halves)
#ifndef GPMA_BFS_BLOCKS_PER_SM
#define GPMA_BFS_BLOCKS_PER_SM 2
#endif
constexpr int kBfsBlocksPerSm = GPMA_BFS_BLOCKS_PER_SM;

int run_bfs(const Geo &g, uint32_t src, int32_t *depth, uint32_t *q0, uint32_t *q1, uint32_t *q2,
            uint32_t *counter, Ctl *ctl, cudaStream_t s) {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_persist, 256, 0);
    const int want = kBfsBlocksPerSm;
    grid = sms * (per_sm > want ? want : per_sm);
    if (grid < 1) grid = 1;
  }
  // counter layout: cnt[0..15], barrier words, error word
  uint32_t *cnt = counter;
  unsigned *bar = counter + 16;
  uint32_t *err = counter + 20;
  cudaMemsetAsync(depth, 0xFF, sizeof(int32_t) * g.V, s);
  cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
  note_launch();
  k_bfs_setup<<<1, 1, 0, s>>>(depth, src, q0, cnt, bar);
  // frontiers of at least V/32 vertices take the full pass (measured at R-MAT scale 20:
  // V/8 0.583 ms per call, V/16 to V/128 within 5% of each other, the order depending on
  // the source; at scale 24 V/32 to V/128 are equal, 4.06 ms, and V/8 takes 7.6 ms)
  const uint32_t scan_from = g.V / 32 > 64 ? g.V / 32 : 64;
  Geo gg = g;
  void *args[] = {(void *)&gg, (void *)&depth, (void *)&q0,  (void *)&q1,
                  (void *)&q2, (void *)&cnt,   (void *)&bar, (void *)&err, (void *)&scan_from, (void *)&ctl};
  note_launch();
  if (cudaLaunchCooperativeKernel((const void *)k_bfs_persist, dim3(grid), dim3(256), args, 0, s) != cudaSuccess)
    return -1;
  note_launch();
  k_bfs_flag<<<1, 1, 0, s>>>(err, ctl);
  return 0;
}

// ---- connected components -------------------------------------------------------------------------
// Parents only ever point to smaller ids, so a root is the smallest id of its
// tree and any (even stale) chain of parent reads strictly decreases: finds use
// plain loads, the CAS that hooks a root checks freshness.
__device__ __forceinline__ uint32_t cc_find(uint32_t *parent, uint32_t v) {
  uint32_t par = parent[v];
  if (par != v) {
    uint32_t prev = v, next;
    while (par > (next = parent[par])) {
      parent[prev] = next;  // path halving towards the root
      prev = par;
      par = next;
    }
  }
  return par;
}

__device__ __forceinline__ void cc_link(uint32_t *label, uint32_t a, uint32_t b) {
  for (;;) {
    a = cc_find(label, a);
    b = cc_find(label, b);
    if (a == b) return;
    if (a < b) {
      uint32_t t = a; a = b; b = t;
    }
    // hook the larger root under the smaller one
    const uint32_t old = atomicCAS(&label[a], a, b);
    if (old == a) return;
    a = old;
  }
}

__global__ void k_cc_init(uint32_t *label, uint32_t V) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) label[v] = v;
}

// first pass: the first two stored out-edges of every row, which already joins
// most vertices into large, shallow trees before the pass over all edges.  One edge
// per row was measured faster on a freshly loaded graph but slower in a sliding
// window (0.46 against 0.29 ms per call at R-MAT scale 20): its longer parent chains
// cost the compression more than the first pass saves.
__global__ void k_cc_sample(Geo g, uint32_t *label) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < g.V; u += gridDim.x * blockDim.x) {
    const uint64_t beg = u ? (uint64_t)g.row_end[u - 1] + 1 : 0, end = g.row_end[u];
    uint32_t taken = 0;
    for (uint64_t e = beg; e < end && taken < 2; e++) {
      const uint64_t k = g.slots[e];
      if (k == kEmpty) continue;
      ++taken;
      const uint32_t v = (uint32_t)(k & 0xFFFFFFFFull);
      if (v != u) cc_link(label, u, v);
    }
  }
}

__global__ void __launch_bounds__(256) k_cc_hook(Geo g, uint32_t *label) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g.C; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = g.slots[e];
    if (k == kEmpty || is_guard(k)) continue;
    const uint32_t a = (uint32_t)(k >> 32), b = (uint32_t)(k & 0xFFFFFFFFull);
    // equal labels: already one tree (after the compression most edges end here)
    if (a != b && label[a] != label[b]) cc_link(label, a, b);
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
  k_cc_sample<<<vb, 256, 0, s>>>(g, label);
  note_launch();
  k_cc_compress<<<vb, 256, 0, s>>>(label, g.V);
  note_launch();
  k_cc_hook<<<nb(g.C, 256, 152 * 16), 256, 0, s>>>(g, label);
  note_launch();
  k_cc_compress<<<vb, 256, 0, s>>>(label, g.V);
}

}  // namespace gpk
