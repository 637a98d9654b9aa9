// k_model.cu -- training of the learned leaf search (the model and the search
// are in gpma_dev.cuh).  Everything runs on the device from the current pivots:
// one kernel, k_lm_train:
//   decide       retrain now?  Always after a resize or import and periodically;
//                after a batch only once merges above level 0 have rewritten an
//                eighth of the leaves since the last training, or a quarter of the
//                batch's searches missed their predicted window (a miss costs one
//                more search, a training about two search kernels; a level-0
//                merge moves keys only inside their leaf, and the search stays
//                exact whatever the staleness, only slower).  Every block takes
//                the same decision from the same inputs.
//   fit          one warp per piece (2^span consecutive leaves): its first and
//                last non-empty leaf, boundary, slope, answer bracket and the
//                largest prediction error over its leaves
//   publish      the last block to finish: empty pieces take the next boundary
//                (so the boundaries never decrease), the radix table of the root
//                stage over the boundaries, then the model is published (or,
//                without training, the drift is carried over)
#include "gpma_dev.cuh"
#include "gpma_launch.h"

namespace gpk {

__device__ __forceinline__ void lm_fit_piece(const Geo &g, uint32_t span, uint32_t p, Piece *pieces) {
  const uint32_t lane = lane_id();
  const uint64_t S = 1ull << span;
  const uint64_t j0 = (uint64_t)p << span;
  // first and last non-empty leaf of the piece
  uint64_t first = kEmpty, last = kEmpty;
  for (uint64_t b = 0; b < S; b += 32) {
    const uint64_t j = j0 + b + lane;
    const bool ne = b + lane < S && __ldg(g.F + j) != kEmpty;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, ne);
    if (bal) {
      if (first == kEmpty) first = j0 + b + (__ffs(bal) - 1);
      last = j0 + b + (31 - __clz(bal));
    }
  }
  Piece pc;
  pc.pad = 0;
  if (first == kEmpty) {
    pc.kb = kEmpty;  // filled in when the model is published
    pc.first = kNoLeaf;
    pc.lo = pc.hi = (uint32_t)j0;
    pc.slope = 0.0f;
    pc.err = 0;
  } else {
    pc.kb = __ldg(g.F + first);
    pc.first = (uint32_t)first;
    pc.lo = (uint32_t)first;
    pc.hi = (uint32_t)last;
    const uint64_t kspan = __ldg(g.F + last) - pc.kb;
    pc.slope = (last > first && kspan) ? (float)(last - first) / (float)kspan : 0.0f;
    // largest |prediction - leaf| over the non-empty leaves
    uint32_t e = 0;
    for (uint64_t b = 0; b < S; b += 32) {
      const uint64_t j = j0 + b + lane;
      const uint64_t f = b + lane < S ? __ldg(g.F + j) : kEmpty;
      if (f != kEmpty) {
        const float d = (float)(f - pc.kb) * pc.slope;
        int64_t pred = (int64_t)pc.first + (int64_t)d;
        if (pred < (int64_t)pc.lo) pred = pc.lo;
        if (pred > (int64_t)pc.hi) pred = pc.hi;
        const uint32_t ej = (uint32_t)(pred > (int64_t)j ? pred - (int64_t)j : (int64_t)j - pred);
        e = ej > e ? ej : e;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const uint32_t u = __shfl_xor_sync(0xFFFFFFFFu, e, o);
      e = u > e ? u : e;
    }
    pc.err = e;
  }
  if (lane == 0) pieces[p] = pc;
}

constexpr uint32_t kLmThreads = 1024;

// Publish (one block of kLmThreads): suffix minimum of the boundaries (an empty
// piece takes the next boundary), the radix table, the head fields, valid last.
__device__ void lm_publish(ModelHead *head, Piece *pieces, uint32_t np, uint32_t span) {
  __shared__ uint64_t wmin[kLmThreads / 32];
  __shared__ uint64_t s_max[kLmThreads / 32];
  __shared__ uint32_t any;
  __shared__ uint64_t s_base;
  __shared__ uint32_t s_shift;
  const uint32_t t = threadIdx.x, lane = lane_id(), w = t >> 5;
  constexpr uint32_t kW = kLmThreads / 32;
  constexpr uint32_t kPer = kPieces / kLmThreads;
  if (t == 0) any = 0;
  __syncthreads();
  // this thread's pieces [t*kPer, (t+1)*kPer), scanned from the right
  uint64_t v[kPer], run = kEmpty;
  bool mine = false;
  for (int q = (int)kPer - 1; q >= 0; q--) {
    const uint32_t p = t * kPer + q;
    const uint64_t kb = p < np ? pieces[p].kb : kEmpty;
    mine |= p < np && pieces[p].first != kNoLeaf;
    run = kb < run ? kb : run;
    v[q] = run;
  }
  // minimum over this thread and the threads after it: in the warp, then over warps
  uint64_t inc = run;
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t u = __shfl_down_sync(0xFFFFFFFFu, inc, o);
    if (lane + o < 32 && u < inc) inc = u;
  }
  if (lane == 0) wmin[w] = inc;
  if (mine) atomicOr(&any, 1u);
  __syncthreads();
  if (t == 0)  // minimum over warps w..kW-1, in place
    for (int i = (int)kW - 2; i >= 0; i--) wmin[i] = wmin[i + 1] < wmin[i] ? wmin[i + 1] : wmin[i];
  __syncthreads();
  uint64_t right = __shfl_down_sync(0xFFFFFFFFu, inc, 1);  // threads after this one in the warp
  if (lane == 31) right = kEmpty;
  if (w + 1 < kW && wmin[w + 1] < right) right = wmin[w + 1];
  uint64_t kmax = 0;  // largest boundary of a non-empty piece
  uint64_t kbf[kPer];  // the final boundaries of this thread's pieces
  for (uint32_t q = 0; q < kPer; q++) {
    const uint32_t p = t * kPer + q;
    kbf[q] = kEmpty;
    if (p >= np) continue;
    const uint64_t fill = v[q] < right ? v[q] : right;
    if (pieces[p].first == kNoLeaf) pieces[p].kb = fill;
    else kmax = pieces[p].kb > kmax ? pieces[p].kb : kmax;
    kbf[q] = pieces[p].first == kNoLeaf ? fill : pieces[p].kb;
  }
  // radix table: prefix(k) = min((k - rbase) >> rshift, kRadix - 1) with the
  // smallest shift that maps every boundary below kRadix; rt[r] = first piece with
  // prefix >= r, i.e. rt[r] = p for prefix(piece p - 1) < r <= prefix(piece p):
  // every thread writes the entries its pieces own (each entry once)
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t u = __shfl_xor_sync(0xFFFFFFFFu, kmax, o);
    kmax = u > kmax ? u : kmax;
  }
  if (lane == 0) s_max[w] = kmax;
  __syncthreads();
  if (t == 0) {
    uint64_t mx = 0;
    for (uint32_t i = 0; i < kW; i++) mx = s_max[i] > mx ? s_max[i] : mx;
    const uint64_t base = pieces[0].kb;
    const uint64_t range = (any && mx > base) ? mx - base : 0;
    uint32_t sh = 0;
    while ((range >> sh) >= kRadix) sh++;
    s_base = base;
    s_shift = sh;
  }
  __syncthreads();
  const uint64_t base = s_base;
  const uint32_t sh = s_shift;
  auto prefix = [&](uint64_t kb) -> int32_t {
    if (kb < base) return 0;
    const uint64_t r = (kb - base) >> sh;
    return r < kRadix - 1 ? (int32_t)r : (int32_t)(kRadix - 1);
  };
  uint32_t *rt = reinterpret_cast<uint32_t *>(pieces + kPieces);
  // prefix of the piece before this thread's first (-1 before piece 0)
  int32_t prev = -1;
  if (t > 0 && t * kPer <= np) prev = prefix(pieces[t * kPer - 1].kb);
  for (uint32_t q = 0; q < kPer; q++) {
    const uint32_t p = t * kPer + q;
    if (p >= np) break;
    const int32_t cur = prefix(kbf[q]);
    for (int32_t r = prev + 1; r <= cur; r++) rt[r] = p;
    prev = cur > prev ? cur : prev;
  }
  // entries above the last piece's prefix: npieces
  if ((t + 1) * kPer >= np && t * kPer < np) {
    for (int32_t r = prev + 1; r <= (int32_t)kRadix; r++) rt[r] = np;
  }
  if (t == 0 && np == 0)
    for (uint32_t r = 0; r <= kRadix; r++) rt[r] = 0;
  __syncthreads();
  if (t == 0) {
    head->span = span;
    head->npieces = np;
    head->rbase = s_base;
    head->rshift = s_shift;
    head->drift = 0;
    __threadfence();
    head->valid = any;
  }
}

__global__ void __launch_bounds__(kLmThreads) k_lm_train(Geo g, ModelHead *head, Piece *pieces, const Ctl *ctl,
                                                         int after_batch) {
  __shared__ uint32_t s_last;
  uint32_t span = 0;
  while ((g.nleaves >> span) > kPieces) span++;
  const uint32_t np = (uint32_t)(g.nleaves >> span);
  uint64_t d = 0;
  bool now = true;
  if (after_batch) {
    // retrain once merges above level 0 have rewritten an eighth of the leaves, or
    // when a quarter of this batch's searches missed their predicted window
    d = head->drift + (ctl->err == 0 ? ctl->nleafw : 0u);
    now = head->valid == 0 || d * 8 >= g.nleaves || (uint64_t)ctl->lm_miss * 4 > ctl->m;
  }
  if (now) {
    const uint32_t p = blockIdx.x * (kLmThreads / 32) + (threadIdx.x >> 5);
    if (p < np) lm_fit_piece(g, span, p, pieces);
  }
  // the last block to finish publishes (head->done counts finished blocks and is
  // reset by that block, ready for the next launch)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&head->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) head->done = 0;
  if (now) {
    if (threadIdx.x == 0) head->valid = 0;
    lm_publish(head, pieces, np, span);
  } else if (threadIdx.x == 0) {
    head->drift = d;
  }
}

void launch_train_model(const Geo &g, ModelHead *head, Piece *pieces, const Ctl *ctl, bool after_batch,
                        cudaStream_t s) {
  const uint64_t np = g.nleaves < kPieces ? g.nleaves : kPieces;
  note_launch();
  constexpr uint32_t kWarps = kLmThreads / 32;  // one piece per warp
  k_lm_train<<<(uint32_t)((np + kWarps - 1) / kWarps), kLmThreads, 0, s>>>(g, head, pieces, ctl, after_batch ? 1 : 0);
}

}  // namespace gpk
