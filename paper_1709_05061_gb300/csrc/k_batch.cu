// k_batch.cu -- front end of one update batch (Algorithm "GPMA+ Segment-Oriented
// Insertion", Sec. 5.2, lines Sort(U) and BinarySearchLeafSegments(U)):
//   k_init_batch  reset the per-call control block and histograms
//   k_prep        validate keys, compress (src, dst, insert/delete tag) into one
//                 sort word, count the words of every bucket (top bits)
//   k_bk_scan     bucket offsets; flags a bucket too large for shared memory
//   k_bk_scatter  every word to its bucket
//   k_bk_sort     one bucket per block: sort in shared memory, unique + insert/
//                 delete cancellation, the leaf search of every survivor (learned
//                 model when trained, else binary search; both give the same
//                 leaf), the bucket's survivor and run-head counts
//   k_bk_offsets  survivor and run-head offsets of every bucket (one block)
//   k_bk_write    survivors and run heads to their places
//   k_small_front all of the above in one block for batches of at most
//                 kSmallBatch keys (bitonic sort in shared memory)
// A batch with a bucket above kBkCap keys (a heavily skewed batch) takes the
// radix-sort path instead: k_bk_convert (radix histograms), k_sort_pass (one
// stable LSD pass with per-digit look-back) per digit, k_search_all (unique/
// cancel + leaf search, one word per thread) and k_compact (single-pass
// compaction of survivors and run heads).
#include "gpma_dev.cuh"
#include "gpma_launch.h"
#include "scan_dev.cuh"

namespace gpk {

constexpr int kSortThreads = 256;
// keys per thread per pass: 8 for small batches (more tiles in flight, fewer
// registers), 16 for large ones (half the tiles on the look-back chain)
constexpr int kSortItemsSmall = 8, kSortItemsLarge = 16;
constexpr uint64_t kSortLargeFrom = 1ull << 19;
constexpr int kSortTile = kSortThreads * kSortItemsSmall;  // status words are sized for the small tile

// ---- key compression -----------------------------------------------------------------
// Graph mode: word = (src << db) | d with d = dst, or d = V for a guard (so a
// guard sorts after every edge of its row); db = bits(V) when guards may occur,
// else bits(V-1).  Raw mode: word = key.  The insert/delete tag rides in bit 63,
// outside the sorted digits: the sort is stable and inserts precede deletes in
// its input, so words of equal key keep inserts first.
constexpr uint64_t kTagBit = 1ull << 63;

__device__ __forceinline__ uint64_t compress(uint64_t key, uint32_t tag, const PrepArgs &a) {
  const uint64_t t = tag ? kTagBit : 0ull;
  if (a.raw) return key | t;
  uint64_t src = key >> 32, dst = key & 0xFFFFFFFFull;
  uint64_t d = (dst == 0xFFFFFFFFull) ? (uint64_t)a.V : dst;
  return ((src << a.db) | d) | t;
}

__device__ __forceinline__ uint64_t expand(uint64_t w, const PrepArgs &a) {
  w &= ~kTagBit;
  if (a.raw) return w;
  uint64_t d = w & ((1ull << a.db) - 1ull);
  uint64_t src = w >> a.db;
  uint64_t dst = (d == (uint64_t)a.V) ? 0xFFFFFFFFull : d;
  return (src << 32) | dst;
}

__global__ void k_init_batch(Ctl *ctl, uint32_t *hist, uint32_t nhist, uint32_t *bcnt, uint32_t nbk, uint32_t n) {
  for (uint32_t i = threadIdx.x; i < nhist; i += blockDim.x) hist[i] = 0;
  for (uint32_t i = threadIdx.x; i < nbk; i += blockDim.x) bcnt[i] = 0;
  if (threadIdx.x == 0) {
    ctl->err = 0;
    ctl->n = n;
    ctl->epoch += kSlotsPerBatch;
    ctl->nesc = 0;
    ctl->nfail = 0;
    ctl->nlong = 0;
    ctl->nvlong = 0;
    ctl->resized = 0;
    ctl->m = ctl->nruns = ctl->npend = ctl->neruns = ctl->nsegs = ctl->nleafw = 0;
    for (int i = 0; i < 16; i++) ctl->ticket[i] = 0;
    ctl->n_inserted = ctl->n_deleted = 0;
    ctl->st_cov_touched = ctl->st_l0_only = ctl->st_empties = ctl->st_del_leaves = 0;
    ctl->levels_climbed = 0;
    ctl->n_merged0 = 0;
    for (int i = 0; i < kMaxLv; i++) ctl->merges[i] = 0;
    ctl->bkfall = ctl->nbigbk = 0;
  }
}

// validation, sort words (compressed key << 1 | tag) and bucket counts
__global__ void __launch_bounds__(256) k_prep(PrepArgs a, const uint64_t *__restrict__ ins,
                                              const uint64_t *__restrict__ del, uint64_t *__restrict__ out,
                                              uint32_t *__restrict__ bcnt, uint32_t shift, uint32_t nbk, Ctl *ctl) {
  extern __shared__ uint32_t bh[];  // nbk counts
  for (uint32_t i = threadIdx.x; i < nbk; i += blockDim.x) bh[i] = 0;
  __syncthreads();
  const uint32_t n = a.n_ins + a.n_del;
  bool bad = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t tag = i >= a.n_ins;
    const uint64_t key = tag ? del[i - a.n_ins] : ins[i];
    bool ok;
    if (a.raw) {
      ok = (key >> 63) == 0;
    } else {
      const uint64_t src = key >> 32, dst = key & 0xFFFFFFFFull;
      ok = src < a.V && (dst < a.V || (a.allow_guards && !tag && dst == 0xFFFFFFFFull));
    }
    bad |= !ok;
    const uint64_t w = ok ? ((compress(key, 0, a) << 1) | tag) : 0ull;
    out[i] = w;
    atomicAdd(&bh[(uint32_t)(w >> shift)], 1u);
  }
  if (__any_sync(0xFFFFFFFFu, bad) && lane_id() == 0) atomicOr(&ctl->err, kErrKey);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nbk; i += blockDim.x)
    if (bh[i]) atomicAdd(&bcnt[i], bh[i]);
}

// radix-sort path: sort words back to the radix layout (tag in bit 63) and the
// digit histograms of every pass
__global__ void __launch_bounds__(256) k_bk_convert(PrepArgs a, uint64_t *__restrict__ buf,
                                                    uint32_t *__restrict__ hist, Ctl *ctl, const uint32_t *gate) {
  if (gate && *gate == 0) return;
  __shared__ uint32_t sh[8 * 256];
  for (uint32_t i = threadIdx.x; i < a.npass * 256u; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const uint32_t n = ctl->n;
  const uint32_t mask = (1u << a.dbits) - 1u;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t w = buf[i];
    const uint64_t kw = w >> 1;
    buf[i] = kw | ((w & 1ull) << 63);
    for (uint32_t p = 0; p < a.npass; p++)
      atomicAdd(&sh[p * 256 + (uint32_t)((kw >> (p * a.dbits)) & mask)], 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < a.npass * 256u; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// One stable LSD pass.  A tile is ITEMS rounds x 256 keys; warp w owns the
// contiguous sub-tile [w*32*ITEMS, (w+1)*32*ITEMS) so ranks inside a warp need no
// block barrier; tiles are ordered by ticket and chained by a per-digit look-back.
template <int kSortItems>
__global__ void __launch_bounds__(kSortThreads) k_sort_pass(const uint64_t *__restrict__ src,
                                                            uint64_t *__restrict__ dst, const uint32_t *hist,
                                                            uint64_t *status, Ctl *ctl, uint32_t pass,
                                                            uint32_t shift, uint32_t dbits, const uint32_t *gate) {
  __shared__ uint32_t wcnt[kSortThreads / 32][256];
  __shared__ uint32_t gbase[256];
  __shared__ uint32_t ltile[256];  // digit totals of the tile, then their exclusive prefix
  __shared__ uint64_t skey[kSortThreads * kSortItems];
  __shared__ uint32_t hs[256];  // this pass's global digit counts, then their exclusive prefix
  __shared__ uint32_t s_tile;
  if (gate && *gate == 0) return;
  const uint32_t n = ctl->n;
  const uint32_t w = threadIdx.x >> 5, lane = lane_id();
  const uint32_t radix = 1u << dbits, mask = radix - 1u;
  for (uint32_t d = threadIdx.x; d < 256; d += kSortThreads) {
    for (int q = 0; q < kSortThreads / 32; q++) wcnt[q][d] = 0;
    hs[d] = d < radix ? hist[pass * 256 + d] : 0u;
  }
  if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->ticket[pass], 1u);
  __syncthreads();
  if (w == 0) {  // the global offsets, while the other warps rank their keys
    uint32_t carry = 0;
    for (int c = 0; c < 256; c += 32) {
      const uint32_t v = hs[c + lane];
      const uint32_t inc = warp_incl_scan(v);
      hs[c + lane] = carry + inc - v;
      carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
  }
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * (kSortThreads * kSortItems) + w * (kSortItems * 32);
  uint64_t key[kSortItems];
  uint32_t rank[kSortItems];
  uint32_t dig[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; r++) {
    uint64_t idx = base + r * 32 + lane;
    bool valid = idx < n;
    key[r] = valid ? src[idx] : 0ull;
    dig[r] = valid ? (uint32_t)(((key[r] & ~kTagBit) >> shift) & mask) : 0xFFFFu;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; r++) {
    // lanes holding the same digit, from one ballot per digit bit (cheaper than match.any)
    uint32_t peers = 0xFFFFFFFFu;
    for (uint32_t b = 0; b < dbits; b++) {
      const bool bit = (dig[r] >> b) & 1u;
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, bit);
      peers &= bit ? bal : ~bal;
    }
    {
      const bool inv = dig[r] == 0xFFFFu;
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, inv);
      peers &= inv ? bal : ~bal;
    }
    uint32_t before = 0;
    if (dig[r] != 0xFFFFu) before = wcnt[w][dig[r]];
    rank[r] = before + __popc(peers & lanemask_lt());
    __syncwarp();
    if (dig[r] != 0xFFFFu && lane == (uint32_t)(__ffs(peers) - 1)) wcnt[w][dig[r]] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, tile total, look-back, global base
  for (uint32_t d = threadIdx.x; d < radix; d += kSortThreads) {
    uint32_t run = 0;
    for (int q = 0; q < kSortThreads / 32; q++) {
      uint32_t c = wcnt[q][d];
      wcnt[q][d] = run;
      run += c;
    }
    ltile[d] = run;
    uint32_t excl = lookback(status, 256, d, tile, run, ctl->epoch + pass, ctl);
    gbase[d] = excl;
  }
  for (uint32_t d = radix + threadIdx.x; d < 256; d += kSortThreads) ltile[d] = 0;
  // exclusive scan of the global histogram of this pass
  __syncthreads();
  if (threadIdx.x < 32) {  // digit offsets inside the tile
    uint32_t carry = 0;
    for (int c = 0; c < 256; c += 32) {
      const uint32_t v = ltile[c + lane];
      const uint32_t inc = warp_incl_scan(v);
      ltile[c + lane] = carry + inc - v;
      carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
  }
  __syncthreads();
  // the tile sorted by digit in shared memory, then written out in digit runs
  // (consecutive keys of one digit go to consecutive addresses)
#pragma unroll
  for (int r = 0; r < kSortItems; r++)
    if (dig[r] != 0xFFFFu) skey[ltile[dig[r]] + wcnt[w][dig[r]] + rank[r]] = key[r];
  __syncthreads();
  const uint64_t t0 = (uint64_t)tile * (kSortThreads * kSortItems);
  const uint32_t cnt = t0 >= n ? 0u : (n - t0 < kSortThreads * kSortItems ? (uint32_t)(n - t0) : kSortThreads * kSortItems);
  for (uint32_t i = threadIdx.x; i < cnt; i += kSortThreads) {
    const uint64_t k = skey[i];
    const uint32_t d = (uint32_t)(((k & ~kTagBit) >> shift) & mask);
    const uint32_t pos = hs[d] + gbase[d] + (i - ltile[d]);
    if (pos < n) dst[pos] = k;  // always true unless a look-back gave up
  }
}

// ---- small batches: the whole front end in one block ---------------------------------------
// Sort word = (compressed key without tag) << 1 | tag.  Inserts (tag 0) order
// before deletes (tag 1) of the same key, and equal words are identical, so the
// sorted sequence equals the stable radix sort's.  Each thread owns `ipt`
// consecutive positions for the two compactions (survivors, run heads).

// Leaf search with a sampled first stage: S evenly spaced pivots F[i * stride]
// sit in shared memory, the non-empty ones compacted in order.  The last sampled
// pivot <= k and the first one > k bracket the answer (eff(lo - 1) <= k and
// eff(hi) > k), and search_first_above finishes inside that bracket, so the leaf
// equals leaf_search's.
__device__ __forceinline__ uint32_t sampled_leaf_search(const uint64_t *__restrict__ F, uint64_t nleaves,
                                                        const uint64_t *cv, const uint32_t *cpos, uint32_t cnt,
                                                        uint64_t k) {
  uint32_t a = 0, b = cnt;  // first compacted sample with value > k
  while (a < b) {
    const uint32_t mid = (a + b) >> 1;
    if (cv[mid] > k) b = mid; else a = mid + 1;
  }
  const uint64_t lo = a ? (uint64_t)cpos[a - 1] + 1 : 0;
  const uint64_t hi = a < cnt ? (uint64_t)cpos[a] : nleaves;
  const uint64_t p = search_first_above(F, lo, hi, k);
  return p ? (uint32_t)(p - 1) : 0u;
}

__global__ void __launch_bounds__(1024) k_small_front(PrepArgs a, const uint64_t *__restrict__ ins,
                                                      const uint64_t *__restrict__ del, Ctl *ctl,
                                                      const uint64_t *__restrict__ F, uint64_t nleaves,
                                                      uint64_t *__restrict__ ukey, uint8_t *__restrict__ utag,
                                                      uint32_t *__restrict__ uleaf, uint32_t *__restrict__ run_start,
                                                      uint32_t *__restrict__ run_leaf, const ModelHead *mhead,
                                                      const Piece *__restrict__ mpieces, uint32_t P, uint32_t S) {
  extern __shared__ uint64_t sk[];           // P sort words
  uint64_t *sw = sk + P;                     // P survivor words
  uint64_t *cv = sw + P;                     // S compacted sampled pivots
  uint32_t *sleaf = (uint32_t *)(cv + S);    // P leaves of the survivors
  uint32_t *cpos = sleaf + P;                // S leaf indices of the compacted samples
  __shared__ uint32_t wsum[33];
  const uint32_t n = a.n_ins + a.n_del, t = threadIdx.x, nt = blockDim.x;
  const uint32_t ipt = (P + nt - 1) / nt, e0 = t * ipt;
  const uint32_t spt = (S + nt - 1) / nt, s0 = t * spt;
  const uint64_t stride = nleaves / S;
  if (t == 0) {
    ctl->err = 0;
    ctl->n = n;
    ctl->epoch += kSlotsPerBatch;
    ctl->nesc = ctl->nfail = ctl->nlong = ctl->nvlong = ctl->resized = 0;
    ctl->m = ctl->nruns = ctl->npend = ctl->neruns = ctl->nsegs = ctl->nleafw = 0;
    for (int i = 0; i < 16; i++) ctl->ticket[i] = 0;
    ctl->n_inserted = ctl->n_deleted = 0;
    ctl->st_cov_touched = ctl->st_l0_only = ctl->st_empties = ctl->st_del_leaves = 0;
    ctl->levels_climbed = 0;
    ctl->n_merged0 = 0;
    for (int i = 0; i < kMaxLv; i++) ctl->merges[i] = 0;
  }
  bool bad = false;
  for (uint32_t i = t; i < P; i += nt) {
    uint64_t word = ~0ull;  // padding sorts last
    if (i < n) {
      const uint32_t tag = i >= a.n_ins;
      const uint64_t key = tag ? del[i - a.n_ins] : ins[i];
      bool ok;
      if (a.raw) {
        ok = (key >> 63) == 0;
      } else {
        const uint64_t src = key >> 32, dst = key & 0xFFFFFFFFull;
        ok = src < a.V && (dst < a.V || (a.allow_guards && !tag && dst == 0xFFFFFFFFull));
      }
      bad |= !ok;
      word = ok ? ((compress(key, 0, a) << 1) | tag) : 0ull;
    }
    sk[i] = word;
  }
  // sampled pivots (the stores land in cv; compacted in place below)
  uint32_t nonempty = 0;
  for (uint32_t q = 0; q < spt; q++) {
    const uint32_t i = s0 + q;
    if (i >= S) break;
    const uint64_t f = __ldg(F + i * stride);
    cv[i] = f;
    nonempty += f != kEmpty;
  }
  if (__syncthreads_or(bad)) {
    if (t == 0) atomicOr(&ctl->err, kErrKey);
    return;  // nothing of the batch is applied
  }
  // bitonic sort, ascending
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = t; i < P / 2; i += nt) {
        const uint32_t lo = ((i & ~(j - 1)) << 1) | (i & (j - 1)), hi = lo + j;
        const uint64_t x = sk[lo], y = sk[hi];
        if ((x > y) == ((lo & k) == 0)) {
          sk[lo] = y;
          sk[hi] = x;
        }
      }
      __syncthreads();
    }
  }
  // compact the non-empty samples in order (read own values before the scan's barrier)
  uint64_t mine[8];
  for (uint32_t q = 0; q < spt && q < 8; q++) mine[q] = s0 + q < S ? cv[s0 + q] : kEmpty;
  uint32_t cnt;
  uint32_t co = block_excl_scan(nonempty, wsum, &cnt);
  for (uint32_t q = 0; q < spt && q < 8; q++) {
    if (mine[q] == kEmpty) continue;
    cv[co] = mine[q];
    cpos[co] = (uint32_t)((s0 + q) * stride);
    co++;
  }
  // unique + cancellation (reading R2) on positions [e0, e0 + ipt)
  uint32_t keep = 0;
  for (uint32_t q = 0; q < ipt; q++) {
    const uint32_t e = e0 + q;
    if (e >= n) break;
    const uint64_t k = sk[e] >> 1;
    const bool kept = (sk[e] & 1) ? (e == 0 || (sk[e - 1] >> 1) != k) : (e + 1 == n || (sk[e + 1] >> 1) != k);
    keep |= (uint32_t)kept << q;
  }
  uint32_t m;
  uint32_t off = block_excl_scan(__popc(keep), wsum, &m);
  for (uint32_t q = 0; q < ipt; q++)
    if ((keep >> q) & 1) sw[off++] = sk[e0 + q];
  __syncthreads();
  // the leaf of every survivor (reading R4), one survivor per thread at a time
  ModelHead hd;
  hd.valid = 0;
  if (mhead) hd = *mhead;
  const bool learned = hd.valid != 0;
  for (uint32_t e = t; e < m; e += nt) {
    const uint64_t w = sw[e];
    const uint64_t key = expand(w >> 1, a);
    const uint32_t leaf = learned ? learned_leaf_search(hd, mpieces, F, nleaves, key)
                                  : sampled_leaf_search(F, nleaves, cv, cpos, cnt, key);
    ukey[e] = key;
    utag[e] = (uint8_t)(w & 1);
    uleaf[e] = leaf;
    sleaf[e] = leaf;
  }
  __syncthreads();
  // run heads over the m survivors
  uint32_t head = 0;
  for (uint32_t q = 0; q < ipt; q++) {
    const uint32_t e = e0 + q;
    if (e >= m) break;
    head |= (uint32_t)(e == 0 || sleaf[e] != sleaf[e - 1]) << q;
  }
  uint32_t nr;
  uint32_t ro = block_excl_scan(__popc(head), wsum, &nr);
  for (uint32_t q = 0; q < ipt; q++) {
    if (!((head >> q) & 1)) continue;
    run_start[ro] = e0 + q;
    run_leaf[ro] = sleaf[e0 + q];
    ro++;
  }
  if (t == 0) {
    ctl->m = m;
    ctl->nruns = nr;
    run_start[nr] = m;
  }
}

// ---- unique/cancel, leaf search and run heads in two kernels ---------------------------------
// k_search_all: one sorted word per thread: the survivor test of reading R2 and,
// for survivors, the leaf (reading R4); lfull[e] = kNoLeaf for dropped words.
// k_compact: one single-pass compaction with two counts (survivors, runs): a run
// starts at a survivor whose leaf differs from the previous survivor's.
__global__ void __launch_bounds__(256) k_search_all(PrepArgs a, const uint64_t *__restrict__ sorted,
                                                    uint32_t *__restrict__ lfull, const uint64_t *__restrict__ F,
                                                    uint64_t nleaves, const Ctl *ctl, const ModelHead *mhead,
                                                    const Piece *__restrict__ mpieces, const uint32_t *gate) {
  if (gate && *gate == 0) return;
  const uint32_t n = ctl->n;
  ModelHead hd;
  hd.valid = 0;
  if (mhead) hd = *mhead;
  const bool learned = hd.valid != 0;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const uint64_t w = sorted[e], k = w & ~kTagBit;
    const bool kept = (w & kTagBit) ? (e == 0 || (sorted[e - 1] & ~kTagBit) != k)
                                    : (e + 1 == n || (sorted[e + 1] & ~kTagBit) != k);
    uint32_t leaf = kNoLeaf;
    if (kept) {
      const uint64_t key = expand(w, a);
      leaf = learned ? learned_leaf_search(hd, mpieces, F, nleaves, key) : leaf_search(F, nleaves, key);
    }
    lfull[e] = leaf;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_compact(PrepArgs a, const uint64_t *__restrict__ sorted,
                                                          const uint32_t *__restrict__ lfull,
                                                          uint64_t *__restrict__ ukey, uint8_t *__restrict__ utag,
                                                          uint32_t *__restrict__ uleaf, uint32_t *__restrict__ run_start,
                                                          uint32_t *__restrict__ run_leaf, uint64_t *status, Ctl *ctl,
                                                          const uint32_t *gate) {
  __shared__ ScanSmem sm;
  if (gate && *gate == 0) return;
  const uint32_t tile = take_ticket(ctl, kSlotKeep, sm), n = ctl->n;
  uint32_t keep[kScanItems], head[kScanItems], lf[kScanItems];
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    const uint64_t e = scan_elem(tile, r);
    lf[r] = e < n ? lfull[e] : kNoLeaf;
    keep[r] = lf[r] != kNoLeaf;
    head[r] = 0;
    if (keep[r]) {
      int64_t j = (int64_t)e - 1;  // previous survivor (dropped words are rare)
      while (j >= 0 && lfull[j] == kNoLeaf) --j;
      head[r] = j < 0 || lfull[j] != lf[r];
    }
  }
  uint32_t koff[kScanItems], hoff[kScanItems];
  const uint32_t m = tile_scan(keep, koff, tile, status, 2, 0, ctl->epoch + kSlotKeep, ctl, sm);
  const uint32_t nr = tile_scan(head, hoff, tile, status, 2, 1, ctl->epoch + kSlotKeep, ctl, sm);
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    if (!keep[r] || koff[r] >= n) continue;
    const uint64_t w = sorted[scan_elem(tile, r)];
    ukey[koff[r]] = expand(w, a);
    utag[koff[r]] = (uint8_t)(w >> 63);
    uleaf[koff[r]] = lf[r];
    if (head[r]) {
      run_start[hoff[r]] = koff[r];
      run_leaf[hoff[r]] = lf[r];
    }
  }
  if ((uint64_t)(tile + 1) * kScanTile >= n && threadIdx.x == 0) {
    ctl->m = m;
    ctl->nruns = nr;
    run_start[nr] = m;
  }
}

// ---- bucketed front end (batches above kSmallBatch keys) ---------------------------------------
// Bucket offsets (exclusive scan of the counts, start[nbk] = n), the counts
// turned into scatter cursors, the list of buckets above kBkSmall keys, and the
// flag (and graph conditional) that sends the batch to the radix-sort path when
// a bucket exceeds kBkCap.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_bk_scan(BucketWork bk, uint32_t nbk, Ctl *ctl,
                                                  cudaGraphConditionalHandle fall, int set_fall) {
  __shared__ uint32_t wsum[33];
  __shared__ uint32_t s_big, s_fall, s_nbig;
  const uint32_t t = threadIdx.x, per = (nbk + 1023) / 1024, b0 = t * per;
  if (t == 0) {
    s_fall = 0;
    s_nbig = 0;
  }
  __syncthreads();
  uint32_t loc = 0, mx = 0;
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t b = b0 + q;
    if (b >= nbk) break;
    const uint32_t c = bk.cnt[b];
    loc += c;
    mx = c > mx ? c : mx;
  }
  uint32_t total;
  uint32_t run = block_excl_scan(loc, wsum, &total);
  if (mx > kBkCap) atomicOr(&s_fall, 1u);
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t b = b0 + q;
    if (b >= nbk) break;
    const uint32_t c = bk.cnt[b];
    bk.start[b] = run;
    bk.cnt[b] = run;  // scatter cursor
    if (c > kBkSmall && c <= kBkCap) bk.big[atomicAdd(&s_nbig, 1u)] = b;
    run += c;
  }
  __syncthreads();
  if (t == 0) {
    bk.start[nbk] = total;
    const uint32_t f = (ctl->err == 0 && s_fall) ? 1u : 0u;
    ctl->bkfall = f;
    ctl->nbigbk = s_nbig;
    if (set_fall) cudaGraphSetConditional(fall, f);
  }
}

__global__ void __launch_bounds__(256) k_bk_scatter(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst,
                                                    uint32_t *__restrict__ cursor, uint32_t shift, const Ctl *ctl) {
  if (ctl->err || ctl->bkfall) return;
  const uint32_t n = ctl->n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t w = src[i];
    dst[atomicAdd(&cursor[(uint32_t)(w >> shift)], 1u)] = w;
  }
}

struct BkSortArgs {
  PrepArgs a;
  uint64_t *words;   // bucketed sort words in; sorted radix-layout words out (same place)
  uint32_t *lfull;   // leaf of every sorted word (kNoLeaf: dropped by reading R2)
  BucketWork bk;
  const uint64_t *F;
  uint64_t nleaves;
  const ModelHead *mhead;
  const Piece *mpieces;
  const Ctl *ctl;
};

// Sort bucket b (at most CAP keys) in shared memory and summarise it: bitonic sort
// of the sort words (padded to a power of two with all-ones words, which sort
// last), the survivor test of reading R2 on neighbours (equal keys share a
// bucket), the leaf of every survivor (reading R4), and the bucket's survivor
// count, run heads after its first survivor, and first and last survivor leaves.
template <uint32_t TPB>
__device__ void bk_sort_one(const BkSortArgs &x, uint32_t b, uint64_t *sk, uint32_t *sl, const ModelHead &hd,
                            bool learned) {
  __shared__ uint32_t s_surv, s_hin, s_first, s_last;
  const uint32_t t = threadIdx.x;
  const uint32_t start = x.bk.start[b], nb = x.bk.start[b + 1] - start;
  uint32_t P = 1;
  while (P < nb) P <<= 1;
  if (t == 0) {
    s_surv = 0;
    s_hin = 0;
    s_first = 0xFFFFFFFFu;
    s_last = 0;
  }
  for (uint32_t i = t; i < P; i += TPB) sk[i] = i < nb ? x.words[start + i] : ~0ull;
  __syncthreads();
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = t; i < P / 2; i += TPB) {
        const uint32_t lo = ((i & ~(j - 1)) << 1) | (i & (j - 1)), hi = lo + j;
        const uint64_t u = sk[lo], v = sk[hi];
        if ((u > v) == ((lo & k) == 0)) {
          sk[lo] = v;
          sk[hi] = u;
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = t; i < nb; i += TPB) {
    const uint64_t w = sk[i], k = w >> 1;
    const bool kept = (w & 1) ? (i == 0 || (sk[i - 1] >> 1) != k) : (i + 1 == nb || (sk[i + 1] >> 1) != k);
    const uint64_t rw = k | ((w & 1ull) << 63);  // radix layout: tag in bit 63
    uint32_t leaf = kNoLeaf;
    if (kept) {
      const uint64_t key = expand(rw, x.a);
      leaf = learned ? learned_leaf_search(hd, x.mpieces, x.F, x.nleaves, key) : leaf_search(x.F, x.nleaves, key);
    }
    sl[i] = leaf;
    x.words[start + i] = rw;
    x.lfull[start + i] = leaf;
  }
  __syncthreads();
  uint32_t surv = 0, hin = 0;
  for (uint32_t i = t; i < nb; i += TPB) {
    if (sl[i] == kNoLeaf) continue;
    ++surv;
    int32_t j = (int32_t)i - 1;  // previous survivor (dropped words are rare)
    while (j >= 0 && sl[j] == kNoLeaf) --j;
    if (j < 0) atomicMin(&s_first, i);
    else if (sl[j] != sl[i]) ++hin;
    atomicMax(&s_last, i);
  }
  surv = warp_sum(surv);
  hin = warp_sum(hin);
  if (lane_id() == 0) {
    if (surv) atomicAdd(&s_surv, surv);
    if (hin) atomicAdd(&s_hin, hin);
  }
  __syncthreads();
  if (t == 0) {
    x.bk.surv[b] = s_surv;
    x.bk.hin[b] = s_hin;
    x.bk.first[b] = s_surv ? sl[s_first] : kNoLeaf;
    x.bk.last[b] = s_surv ? sl[s_last] : kNoLeaf;
  }
  __syncthreads();  // shared memory is reused by the block's next bucket
}

// one 256-thread block per bucket of at most kBkSmall keys
__global__ void __launch_bounds__(256) k_bk_sort(BkSortArgs x, uint32_t nbk) {
  __shared__ uint64_t sk[kBkSmall];
  __shared__ uint32_t sl[kBkSmall];
  const Ctl *ctl = x.ctl;
  if (ctl->err || ctl->bkfall) return;
  const uint32_t b = blockIdx.x;
  if (b >= nbk) return;
  const uint32_t nb = x.bk.start[b + 1] - x.bk.start[b];
  if (nb > kBkSmall) return;  // k_bk_sort_big
  ModelHead hd;
  hd.valid = 0;
  if (x.mhead) hd = *x.mhead;
  bk_sort_one<256>(x, b, sk, sl, hd, hd.valid != 0);
}

// 1024-thread blocks for the buckets of (kBkSmall, kBkCap] keys, from the list
__global__ void __launch_bounds__(1024) k_bk_sort_big(BkSortArgs x) {
  extern __shared__ uint64_t bsm[];
  uint64_t *sk = bsm;
  uint32_t *sl = reinterpret_cast<uint32_t *>(bsm + kBkCap);
  const Ctl *ctl = x.ctl;
  if (ctl->err || ctl->bkfall) return;
  ModelHead hd;
  hd.valid = 0;
  if (x.mhead) hd = *x.mhead;
  const uint32_t nbig = ctl->nbigbk;
  for (uint32_t i = blockIdx.x; i < nbig; i += gridDim.x) bk_sort_one<1024>(x, x.bk.big[i], sk, sl, hd, hd.valid != 0);
}

// Survivor and run-head offsets of every bucket: exclusive scans over the buckets;
// the first survivor of a bucket starts a run unless the last survivor of the
// nearest earlier bucket with survivors has the same leaf.  One block of 1024.
__global__ void __launch_bounds__(1024) k_bk_offsets(BucketWork bk, uint32_t nbk, Ctl *ctl,
                                                     uint32_t *__restrict__ run_start) {
  __shared__ uint32_t wsum[33];
  __shared__ uint32_t s_last[1024];   // last survivor leaf of each thread's buckets
  __shared__ int32_t s_idx[1024];     // thread index, -1 when its buckets hold no survivor
  if (ctl->err || ctl->bkfall) return;
  const uint32_t t = threadIdx.x, per = (nbk + 1023) / 1024, b0 = t * per;
  uint32_t sv = 0, lastleaf = kNoLeaf;
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t b = b0 + q;
    if (b >= nbk) break;
    if (bk.surv[b]) {
      sv += bk.surv[b];
      lastleaf = bk.last[b];
    }
  }
  s_last[t] = lastleaf;
  // nearest earlier thread whose buckets hold survivors: an inclusive running
  // maximum of (t if it has survivors, else -1), read at t - 1
  const uint32_t lane = lane_id(), wid = t >> 5;
  int32_t v = sv ? (int32_t)t : -1;
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v = u > v ? u : v;
  }
  __shared__ int32_t s_wmax[32];
  if (lane == 31) s_wmax[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int32_t x = s_wmax[lane];
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x = u > x ? u : x;
    }
    s_wmax[lane] = x;
  }
  __syncthreads();
  if (wid) v = s_wmax[wid - 1] > v ? s_wmax[wid - 1] : v;
  s_idx[t] = v;
  __syncthreads();
  const int32_t pt = t ? s_idx[t - 1] : -1;
  uint32_t prevleaf = pt >= 0 ? s_last[pt] : kNoLeaf;
  uint32_t hc = 0;
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t b = b0 + q;
    if (b >= nbk) break;
    if (!bk.surv[b]) continue;
    const uint32_t hf = (prevleaf == kNoLeaf || prevleaf != bk.first[b]) ? 1u : 0u;
    bk.hfirst[b] = hf;
    hc += bk.hin[b] + hf;
    prevleaf = bk.last[b];
  }
  uint32_t m, nr;
  uint32_t so = block_excl_scan(sv, wsum, &m);
  uint32_t ho = block_excl_scan(hc, wsum, &nr);
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t b = b0 + q;
    if (b >= nbk) break;
    bk.soff[b] = so;
    bk.hoff[b] = ho;
    if (bk.surv[b]) {
      so += bk.surv[b];
      ho += bk.hin[b] + bk.hfirst[b];
    }
  }
  if (t == 0) {
    ctl->m = m;
    ctl->nruns = nr;
    run_start[nr] = m;
  }
}

// survivors and run heads of every bucket to their places (one block per bucket,
// 256 positions at a time)
__global__ void __launch_bounds__(256) k_bk_write(PrepArgs a, const uint64_t *__restrict__ words,
                                                  const uint32_t *__restrict__ lfull, BucketWork bk, uint32_t nbk,
                                                  uint64_t *__restrict__ ukey, uint8_t *__restrict__ utag,
                                                  uint32_t *__restrict__ uleaf, uint32_t *__restrict__ run_start,
                                                  uint32_t *__restrict__ run_leaf, const Ctl *ctl) {
  __shared__ uint32_t wsum[33];
  if (ctl->err || ctl->bkfall) return;
  const uint32_t b = blockIdx.x;
  if (b >= nbk || bk.surv[b] == 0) return;
  const uint32_t start = bk.start[b], nb = bk.start[b + 1] - start;
  uint32_t so = bk.soff[b], ho = bk.hoff[b];
  const uint32_t hf = bk.hfirst[b];
  for (uint32_t base = 0; base < nb; base += 256) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t lf = i < nb ? lfull[start + i] : kNoLeaf;
    const uint32_t keep = lf != kNoLeaf;
    uint32_t head = 0;
    if (keep) {
      int32_t j = (int32_t)i - 1;  // previous survivor of the bucket
      while (j >= 0 && lfull[start + j] == kNoLeaf) --j;
      head = j < 0 ? hf : (lfull[start + j] != lf);
    }
    uint32_t nk, nh;
    const uint32_t ko = so + block_excl_scan(keep, wsum, &nk);
    const uint32_t hoi = ho + block_excl_scan(head, wsum, &nh);
    if (keep) {
      const uint64_t w = words[start + i];
      ukey[ko] = expand(w, a);
      utag[ko] = (uint8_t)(w >> 63);
      uleaf[ko] = lf;
      if (head) {
        run_start[hoi] = ko;
        run_leaf[hoi] = lf;
      }
    }
    so += nk;
    ho += nh;
  }
}

// ---- host launchers ----------------------------------------------------------------------
static uint32_t grid_for(uint64_t n, uint32_t per_block, uint32_t cap) {
  uint64_t g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (uint32_t)g;
}

uint32_t sort_tiles(uint64_t n) { return (uint32_t)((n + kSortTile - 1) / kSortTile); }
uint32_t comp_tiles(uint64_t n) { return (uint32_t)((n + kScanTile - 1) / kScanTile); }

bool small_front(uint64_t n) { return n <= kSmallBatch; }

void launch_small_front(const FrontArgs &f, cudaStream_t s) {
  const PrepArgs &a = f.prep;
  const uint32_t n = a.n_ins + a.n_del;
  constexpr uint32_t kSamples = 2048;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_small_front, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kSmallBatch * 20 + kSamples * 12);
    attr = true;
  }
  uint32_t P = 64;
  while (P < n) P <<= 1;
  const uint32_t nt = P >= 2048 ? 1024 : 256;  // at most 4 positions and 8 samples per thread
  const uint64_t nl = f.geo->nleaves;
  const uint32_t S = nl < kSamples ? (uint32_t)nl : kSamples;  // nleaves is a power of two
  note_launch();
  k_small_front<<<1, nt, P * 20 + S * 12, s>>>(a, f.ins, f.del, f.ctl, f.geo->F, nl, f.ukey, f.utag, f.uleaf,
                                               f.run_start, f.run_leaf, f.mhead, f.mpieces, P, S);
}

BkGeo bucket_geo(uint64_t n, uint32_t sbits) {
  uint64_t P = 1;
  while (P < n) P <<= 1;
  uint32_t lp = 0;
  while ((1ull << lp) < P) ++lp;
  // about 128 to 256 keys per bucket, 32 to kBkMax buckets
  int kb = (int)lp - 8;
  if (kb < 5) kb = 5;
  if (kb > 14) kb = 14;
  const uint32_t sb = sbits + 1;  // sort word: compressed key << 1 | tag
  if ((uint32_t)kb > sb) kb = (int)sb;
  BkGeo g;
  g.kb = (uint32_t)kb;
  g.shift = sb - g.kb;
  g.nbk = 1u << g.kb;
  return g;
}

// shared-memory opt-in of the bucket kernels (the prep histogram holds up to kBkMax
// counts, the large-bucket sort kBkCap keys and their leaves)
static void bucket_attrs() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kBkMax * sizeof(uint32_t)));
  cudaFuncSetAttribute(k_bk_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(kBkCap * (sizeof(uint64_t) + sizeof(uint32_t))));
  done = true;
}

void launch_prep(const FrontArgs &f, cudaStream_t s) {
  bucket_attrs();
  const PrepArgs &a = f.prep;
  const uint64_t n = (uint64_t)a.n_ins + a.n_del;
  const BkGeo bg = bucket_geo(n, a.sbits);
  note_launch();
  k_init_batch<<<1, 256, 0, s>>>(f.ctl, f.hist, a.npass * 256u, f.bk.cnt, bg.nbk, (uint32_t)n);
  note_launch();
  k_prep<<<grid_for(n, 256, 4 * 152), 256, bg.nbk * sizeof(uint32_t), s>>>(a, f.ins, f.del, f.bufA, f.bk.cnt,
                                                                          bg.shift, bg.nbk, f.ctl);
}

void launch_front_buckets(const FrontArgs &f, uint64_t nb, cudaStream_t s, const cudaGraphConditionalHandle *fall) {
  const PrepArgs &a = f.prep;
  const BkGeo bg = bucket_geo(nb, a.sbits);
  bucket_attrs();
  note_launch();
  k_bk_scan<<<1, 1024, 0, s>>>(f.bk, bg.nbk, f.ctl, fall ? *fall : cudaGraphConditionalHandle(), fall ? 1 : 0);
  note_launch();
  k_bk_scatter<<<grid_for(nb, 256 * 8, 152 * 8), 256, 0, s>>>(f.bufA, f.bufB, f.bk.cnt, bg.shift, f.ctl);
  BkSortArgs x;
  x.a = a;
  x.words = f.bufB;
  x.lfull = f.lfull;
  x.bk = f.bk;
  x.F = f.geo->F;
  x.nleaves = f.geo->nleaves;
  x.mhead = f.mhead;
  x.mpieces = f.mpieces;
  x.ctl = f.ctl;
  note_launch();
  k_bk_sort<<<bg.nbk, 256, 0, s>>>(x, bg.nbk);
  note_launch();
  k_bk_sort_big<<<152, 1024, kBkCap * (sizeof(uint64_t) + sizeof(uint32_t)), s>>>(x);
  note_launch();
  k_bk_offsets<<<1, 1024, 0, s>>>(f.bk, bg.nbk, f.ctl, f.run_start);
  note_launch();
  k_bk_write<<<bg.nbk, 256, 0, s>>>(a, f.bufB, f.lfull, f.bk, bg.nbk, f.ukey, f.utag, f.uleaf, f.run_start,
                                     f.run_leaf, f.ctl);
}

// grids sized for `nb` keys (>= the batch); the kernels read the batch size from ctl
void launch_front_fallback(const FrontArgs &f, uint64_t nb, cudaStream_t s, bool gated) {
  const PrepArgs &a = f.prep;
  const uint32_t *gate = gated ? &f.ctl->bkfall : nullptr;
  note_launch();
  k_bk_convert<<<grid_for(nb, 256, 4 * 152), 256, 0, s>>>(a, f.bufA, f.hist, f.ctl, gate);
  uint64_t *src = f.bufA, *dst = f.bufB;
  const bool large = nb >= kSortLargeFrom;
  const uint32_t st = large ? (uint32_t)((nb + kSortThreads * kSortItemsLarge - 1) / (kSortThreads * kSortItemsLarge))
                            : sort_tiles(nb);
  for (uint32_t p = 0; p < a.npass; p++) {
    note_launch();
    if (large)
      k_sort_pass<kSortItemsLarge><<<st, kSortThreads, 0, s>>>(src, dst, f.hist, f.status, f.ctl, p, p * a.dbits,
                                                               a.dbits, gate);
    else
      k_sort_pass<kSortItemsSmall><<<st, kSortThreads, 0, s>>>(src, dst, f.hist, f.status, f.ctl, p, p * a.dbits,
                                                               a.dbits, gate);
    uint64_t *t = src; src = dst; dst = t;
  }
  // look-back epochs: pass p uses epoch + p, then the fixed slots of gpma_launch.h
  const uint32_t ct = comp_tiles(nb);
  note_launch();
  k_search_all<<<grid_for(nb, 256, 152 * 16), 256, 0, s>>>(a, src, f.lfull, f.geo->F, f.geo->nleaves, f.ctl, f.mhead,
                                                           f.mpieces, gate);
  note_launch();
  k_compact<<<ct, kScanThreads, 0, s>>>(a, src, f.lfull, f.ukey, f.utag, f.uleaf, f.run_start, f.run_leaf, f.status,
                                        f.ctl, gate);
}

}  // namespace gpk
