// k_model.cu -- training of the learned leaf search (a two-stage linear model
// over the leaf pivots; the search itself is learned_leaf_search in
// gpma_dev.cuh).  Everything runs on the device from the current pivots:
//   k_lm_init    reset the head and the per-piece first/last training leaf
//   k_lm_minmax  smallest and largest pivot (range of the root model)
//   k_lm_scale   root slope: pieces per key unit
//   k_lm_route   route every non-empty leaf's pivot to its piece
//   k_lm_fit     per piece: base key, slope, answer bracket (running max of the
//                last leaves of the pieces before it)
//   k_lm_err     per piece: largest |prediction - leaf| over its training leaves
//   k_lm_valid   publish the model
#include "gpma_dev.cuh"
#include "gpma_launch.h"

namespace gpk {

namespace {
uint32_t nblk(uint64_t items, uint32_t per_block, uint32_t cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (uint32_t)b;
}
}  // namespace

__global__ void k_lm_init(ModelHead *head, uint32_t *first, uint32_t *last) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    head->kmin = kEmpty;
    head->kmax = 0;
    head->valid = 0;
    head->rscale = 0.0f;
  }
  for (uint32_t p = t; p < kPieces; p += gridDim.x * blockDim.x) {
    first[p] = kNoLeaf;
    last[p] = 0;
  }
}

__global__ void k_lm_minmax(Geo g, ModelHead *head) {
  uint64_t mn = kEmpty, mx = 0;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < g.nleaves; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t f = g.F[j];
    if (f == kEmpty) continue;
    mn = f < mn ? f : mn;
    mx = f > mx ? f : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t a = __shfl_xor_sync(0xFFFFFFFFu, mn, o), b = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
    mn = a < mn ? a : mn;
    mx = b > mx ? b : mx;
  }
  if (lane_id() == 0) {
    if (mn != kEmpty) atomicMin((unsigned long long *)&head->kmin, (unsigned long long)mn);
    if (mx) atomicMax((unsigned long long *)&head->kmax, (unsigned long long)mx);
  }
}

__global__ void k_lm_scale(ModelHead *head) {
  if (head->kmin == kEmpty) return;  // no pivot: the model stays invalid
  const uint64_t span = head->kmax - head->kmin + 1;
  head->rscale = (float)kPieces / (float)span;
}

__global__ void k_lm_route(Geo g, const ModelHead *head, uint32_t *first, uint32_t *last) {
  const ModelHead m = *head;
  if (m.kmin == kEmpty) return;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < g.nleaves; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t f = g.F[j];
    if (f == kEmpty) continue;
    const uint32_t p = model_route(m, f);
    atomicMin(&first[p], (uint32_t)j);
    atomicMax(&last[p], (uint32_t)j);
  }
}

// one block: running maximum of the last training leaf over the pieces in order
__global__ void __launch_bounds__(1024) k_lm_fit(Geo g, const ModelHead *head, const uint32_t *first,
                                                 const uint32_t *last, Piece *pieces) {
  __shared__ uint32_t wmax[32];
  constexpr uint32_t kPer = kPieces / 1024;
  const uint32_t t = threadIdx.x, lane = lane_id(), wid = t >> 5;
  if (head->kmin == kEmpty) return;
  // pieces [t*kPer, (t+1)*kPer) per thread: local running max, then a block scan of maxima
  uint32_t lmax = 0;
  bool any = false;
  for (uint32_t q = 0; q < kPer; q++) {
    const uint32_t p = t * kPer + q;
    if (first[p] != kNoLeaf) {
      lmax = last[p] > lmax ? last[p] : lmax;
      any = true;
    }
  }
  // exclusive running max over threads (a leaf index + 1, 0 = none)
  uint32_t v = any ? lmax + 1 : 0, inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if ((int)lane >= o && u > inc) inc = u;
  }
  if (lane == 31) wmax[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t x = wmax[lane], xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, xi, o);
      if ((int)lane >= o && u > xi) xi = u;
    }
    wmax[lane] = xi;  // inclusive over warps
  }
  __syncthreads();
  uint32_t before = __shfl_up_sync(0xFFFFFFFFu, inc, 1);
  if (lane == 0) before = 0;
  if (wid > 0 && wmax[wid - 1] > before) before = wmax[wid - 1];
  // walk this thread's pieces in order
  uint32_t run = before;  // last leaf + 1 of the pieces before, 0 = none
  for (uint32_t q = 0; q < kPer; q++) {
    const uint32_t p = t * kPer + q;
    Piece pc;
    pc.lo = run ? run - 1 : 0;
    pc.err = 0;
    pc.pad = 0;
    if (first[p] != kNoLeaf) {
      const uint32_t a = first[p], b = last[p];
      pc.first = a;
      pc.kb = g.F[a];
      const uint64_t kspan = g.F[b] - g.F[a];
      pc.slope = (b > a && kspan) ? (float)(b - a) / (float)kspan : 0.0f;
      pc.hi = b > pc.lo ? b : pc.lo;
      run = b + 1 > run ? b + 1 : run;
    } else {
      pc.first = kNoLeaf;
      pc.kb = 0;
      pc.slope = 0.0f;
      pc.hi = pc.lo;
    }
    pieces[p] = pc;
  }
}

__global__ void k_lm_err(Geo g, const ModelHead *head, Piece *pieces) {
  const ModelHead m = *head;
  if (m.kmin == kEmpty) return;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < g.nleaves; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t f = g.F[j];
    if (f == kEmpty) continue;
    const uint32_t p = model_route(m, f);
    const Piece pc = pieces[p];
    const float d = (float)(f > pc.kb ? f - pc.kb : 0ull) * pc.slope;
    int64_t pred = (int64_t)pc.first + (int64_t)d;
    if (pred < (int64_t)pc.lo) pred = pc.lo;
    if (pred > (int64_t)pc.hi) pred = pc.hi;
    const int64_t e = pred > (int64_t)j ? pred - (int64_t)j : (int64_t)j - pred;
    atomicMax(&pieces[p].err, (uint32_t)e);
  }
}

__global__ void k_lm_valid(ModelHead *head) { head->valid = head->kmin != kEmpty; }

void launch_train_model(const Geo &g, ModelHead *head, Piece *pieces, uint32_t *tmp, cudaStream_t s) {
  uint32_t *first = tmp, *last = tmp + kPieces;
  note_launch();
  k_lm_init<<<16, 256, 0, s>>>(head, first, last);
  const uint32_t b = nblk(g.nleaves, 256, 152 * 8);
  note_launch();
  k_lm_minmax<<<b, 256, 0, s>>>(g, head);
  note_launch();
  k_lm_scale<<<1, 1, 0, s>>>(head);
  note_launch();
  k_lm_route<<<b, 256, 0, s>>>(g, head, first, last);
  note_launch();
  k_lm_fit<<<1, 1024, 0, s>>>(g, head, first, last, pieces);
  note_launch();
  k_lm_err<<<b, 256, 0, s>>>(g, head, pieces);
  note_launch();
  k_lm_valid<<<1, 1, 0, s>>>(head);
}

}  // namespace gpk
