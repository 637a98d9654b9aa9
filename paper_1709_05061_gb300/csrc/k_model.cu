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

__global__ void k_lm_decide(Geo g, ModelHead *head, const Ctl *ctl, int after_batch) {
  bool now = true;
  if (after_batch) {
    const uint64_t d = head->drift + (ctl->err == 0 ? ctl->nleafw : 0u);
    now = head->valid == 0 || d * 32 >= g.nleaves;
    head->drift = now ? 0 : d;
  } else {
    head->drift = 0;
  }
  head->train = now ? 1u : 0u;
}

__global__ void k_lm_init(ModelHead *head, uint32_t *first, uint32_t *last) {
  if (!head->train) return;
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

// the pivots of non-empty leaves increase with the leaf: the smallest is the
// first non-empty leaf's, the largest the last one's (warp 0 scans from the
// front, warp 1 from the back, 32 leaves at a time)
__global__ void k_lm_minmax(Geo g, ModelHead *head) {
  if (!head->train) return;
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  if (w > 1) return;
  for (uint64_t b = 0; b < g.nleaves; b += 32) {
    const uint64_t j = w == 0 ? b + lane : g.nleaves - 1 - (b + lane);
    const bool inb = b + lane < g.nleaves;
    const uint64_t f = inb ? g.F[j] : kEmpty;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, f != kEmpty);
    if (bal) {
      const uint64_t pick = __shfl_sync(0xFFFFFFFFu, f, __ffs(bal) - 1);
      if (lane == 0) {
        if (w == 0) head->kmin = pick; else head->kmax = pick;
      }
      return;
    }
  }
}

__global__ void k_lm_scale(ModelHead *head) {
  if (!head->train) return;
  if (head->kmin == kEmpty) return;  // no pivot: the model stays invalid
  const uint64_t span = head->kmax - head->kmin + 1;
  head->rscale = (float)kPieces / (float)span;
}

// neighbouring leaves mostly share a piece: lanes of one piece combine first
__global__ void k_lm_route(Geo g, const ModelHead *head, uint32_t *first, uint32_t *last) {
  if (!head->train) return;
  const ModelHead m = *head;
  if (m.kmin == kEmpty) return;
  const uint64_t n32 = (g.nleaves + 31) & ~31ull;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n32; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t f = j < g.nleaves ? g.F[j] : kEmpty;
    const uint32_t p = f != kEmpty ? model_route(m, f) : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, p);
    if (p == 0xFFFFFFFFu) continue;
    const uint32_t lo = __ffs(peers) - 1, hi = 31 - __clz(peers);
    if (lane_id() == lo) atomicMin(&first[p], (uint32_t)j);
    if (lane_id() == hi) atomicMax(&last[p], (uint32_t)j);
  }
}

// one block: running maximum of the last training leaf over the pieces in order
__global__ void __launch_bounds__(1024) k_lm_fit(Geo g, const ModelHead *head, const uint32_t *first,
                                                 const uint32_t *last, Piece *pieces) {
  __shared__ uint32_t wmax[32];
  constexpr uint32_t kPer = kPieces / 1024;
  const uint32_t t = threadIdx.x, lane = lane_id(), wid = t >> 5;
  if (!head->train) return;
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
  if (!head->train) return;
  const ModelHead m = *head;
  if (m.kmin == kEmpty) return;
  const uint64_t n32 = (g.nleaves + 31) & ~31ull;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n32; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t f = j < g.nleaves ? g.F[j] : kEmpty;
    uint32_t p = 0xFFFFFFFFu, e = 0;
    if (f != kEmpty) {
      p = model_route(m, f);
      const Piece pc = pieces[p];
      const float d = (float)(f > pc.kb ? f - pc.kb : 0ull) * pc.slope;
      int64_t pred = (int64_t)pc.first + (int64_t)d;
      if (pred < (int64_t)pc.lo) pred = pc.lo;
      if (pred > (int64_t)pc.hi) pred = pc.hi;
      e = (uint32_t)(pred > (int64_t)j ? pred - (int64_t)j : (int64_t)j - pred);
    }
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, p);
    uint32_t mx = e;
    for (uint32_t b = peers; b; b &= b - 1) {
      const uint32_t o = __shfl_sync(peers, e, __ffs(b) - 1);
      mx = o > mx ? o : mx;
    }
    if (p != 0xFFFFFFFFu && lane_id() == (uint32_t)(__ffs(peers) - 1) && mx) atomicMax(&pieces[p].err, mx);
  }
}

__global__ void k_lm_valid(ModelHead *head) {
  if (!head->train) return;
  head->valid = head->kmin != kEmpty;
}

void launch_train_model(const Geo &g, ModelHead *head, Piece *pieces, uint32_t *tmp, const Ctl *ctl,
                        bool after_batch, cudaStream_t s) {
  uint32_t *first = tmp, *last = tmp + kPieces;
  note_launch();
  k_lm_decide<<<1, 1, 0, s>>>(g, head, ctl, after_batch ? 1 : 0);
  note_launch();
  k_lm_init<<<16, 256, 0, s>>>(head, first, last);
  note_launch();
  k_lm_minmax<<<1, 64, 0, s>>>(g, head);
  note_launch();
  k_lm_scale<<<1, 1, 0, s>>>(head);
  const uint32_t b = nblk(g.nleaves, 256, 152 * 8);
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
