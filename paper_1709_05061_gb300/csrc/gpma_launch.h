// gpma_launch.h -- host-side launch interface between the libgpma translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "gpma_dev.cuh"

namespace gpk {

// process-wide count of kernel launches issued by the library
void note_launch();
uint64_t launch_count();
void unnote_launches(uint64_t k);  // launches recorded while capturing a graph
void allow_big_smem();

// ticket / look-back epoch slots of one batch (Ctl::ticket, Ctl::epoch + slot)
constexpr uint32_t kSlotKeep = 8, kSlotRuns = 9, kSlotPend = 10, kSlotERuns = 11, kSlotSegs = 12,
                   kSlotMisc = 13, kSlotsPerBatch = 16;

struct PrepArgs {
  uint32_t n_ins, n_del;
  uint32_t V, db, raw, allow_guards;
  uint32_t npass, dbits;
  uint32_t sbits;  // sorted bits of the compressed key (the tag is not among them)
};

struct FrontArgs {
  PrepArgs prep;
  const ModelHead *mhead;  // learned leaf search (nullptr: plain binary search)
  const Piece *mpieces;
  const uint64_t *ins, *del;
  uint64_t *bufA, *bufB;  // sort ping-pong
  uint32_t *hist;         // npass * 256
  uint64_t *status;       // look-back status words
  Ctl *ctl;
  const Geo *geo;
  uint64_t *ukey;
  uint8_t *utag;
  uint32_t *uleaf;
  uint32_t *run_start;
  uint32_t *run_leaf;
  uint32_t *lfull;        // leaf of every sorted word (kNoLeaf if dropped), before compaction
  uint32_t *rs;           // front_scratch_words(nb) words: per-tile digit counts, block summaries
};

// per-batch work arrays of the update kernels
struct Work {
  uint64_t *ukey;
  uint8_t *utag;
  uint32_t *uleaf;
  uint32_t *run_start;
  uint8_t *eflag;     // per key: 0 no effect, 1 applied, 2 pending insert
  uint32_t *rleaf;    // per run: its leaf (written with the run heads)
  int32_t *rdelta;
  uint8_t *rinfo;     // 1 merged at level 0, 2 escalated
  uint32_t *rdel;
  uint64_t *pkey;     // pending inserts (sorted) and their leaves
  uint32_t *pleaf;
  uint32_t *erun;     // per escalated run: its first pending insert (+ end)
  uint32_t *eleaf;    // per escalated run: its leaf
  uint8_t *elvl;      // merge level of each pending run
  uint8_t *etop;      // top merged ancestor of each pending run
  uint32_t *seg_node; // maximal merged segments: node, level, first pending, leaf prefix
  uint8_t *seg_top;
  uint32_t *seg_pstart;
  uint32_t *seg_lpre;
  uint64_t *status;
  uint32_t *rs;       // front_scratch_words(cap) words for the radix front end
  uint16_t *lbkt;     // model-bucketed front end: bucket (model piece) of every key
  uint32_t *lcnt;     // kPieces + 1 bucket counts, then offsets
  uint32_t *lrank;    // rank of every key among the keys of its bucket
  uint32_t cap;       // capacity of the per-key arrays
};

uint32_t comp_tiles(uint64_t n);
// k_init_batch + k_prep (take the batch's own pointers and sizes)
// runs longer than this (bulk loads) take the chunked level-0 path: many warps
// share one run's presence filter and deletes, one warp per run finishes it
constexpr uint32_t kLongRun = 1024;
// batches of at most kSmallBatch keys: validation .. run heads in one block
constexpr uint32_t kSmallBatch = 4096;
bool small_front(uint64_t n);
void launch_small_front(const FrontArgs &f, cudaStream_t s);
// Batches of more than kSmallBatch keys; `nb` (>= the batch, the same in the two
// calls) sizes the grids, the kernels read the batch size from ctl.
// k_init_batch + k_prep: validation, sort words, first-pass counts per tile
void launch_prep(const FrontArgs &f, uint64_t nb, cudaStream_t s);
// the radix passes, unique/cancel + leaf search, survivors and run heads
void launch_front(const FrontArgs &f, uint64_t nb, cudaStream_t s);
uint64_t front_scratch_words(uint64_t nb);  // size of FrontArgs::rs for batches of up to nb keys
// The model-bucketed front end of a learned handle (large batches, inside a captured
// graph): launch_lprep (direct, reads the batch) validates and compresses every key
// and counts it in its bucket (the model piece its key routes to; the top key bits
// before the model is trained), keeping its rank there, and turns the counts into
// offsets; in the graph, launch_lfront_sort places every word at its bucket's offset
// plus its rank, sorts every bucket (in registers up to 512 words, in shared memory up
// to kLSortMax, else in place) and leaves each sorted word's bucket in bkt;
// launch_front_search (given bkt) then finishes as after the radix passes
// (launch_front_radix), which plain handles keep.
constexpr uint32_t kLSortMax = 4096;  // words of the largest bucket sorted in shared memory
bool learned_front(const PrepArgs &a, bool has_model, uint64_t n);
void launch_lprep(const FrontArgs &f, uint16_t *bkt, uint32_t *rank, uint32_t *cnt, uint64_t nb, cudaStream_t s);
void launch_lfront_sort(const FrontArgs &f, uint16_t *bkt, const uint32_t *rank, uint32_t *cnt, uint64_t nb,
                        cudaStream_t s);
void launch_front_radix(const FrontArgs &f, uint64_t nb, cudaStream_t s);
// spiece: each sorted word's model piece (the model-bucketed sort leaves it in its
// bucket array), or nullptr: the learned search then routes every key itself
void launch_front_search(const FrontArgs &f, uint64_t nb, cudaStream_t s, const uint16_t *spiece = nullptr);

// k_update.cu
// level 0: k_leaf64 (L = 64, runs of at most 32 keys), then the general pass (the
// other runs; with rest_only the fast path handled the short ones) and the chunked
// path for runs above kLongRun keys, then the batch's out-degree changes
void launch_leaf_pass(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s);
void launch_leaf64(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s);
void launch_leaf_rest(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, bool rest_only, cudaStream_t s);
void launch_degrees_batch(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s);
// levels 1..h of the count tree from the leaf counts and this batch's pending
// inserts (run after launch_pending; does nothing when no insert is pending)
void launch_tree_rebuild(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s);
void launch_pending(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s);
// merge level of every pending run; with may_fail a run no level admits is counted in
// Ctl::nfail instead of being an error
void launch_esc_level(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, bool may_fail, cudaStream_t s);
void launch_esc_top(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s);
void launch_unmark(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s);
void launch_segments(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s);
void launch_stats(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s);
// merge of maximal segments (escalation) or of the whole array into a new one (resize):
// gathers valid keys of `src` over the segments' leaves into `scratch` (leaf offsets in
// `voff`, nleafw + 1 entries), then writes `dst`.
void launch_segment_merge(const Geo &src, const Geo &dst, Ctl *ctl, const Work &w, uint64_t scratch_cap,
                          uint64_t nleafw_bound, uint64_t *scratch, uint32_t *voff, uint64_t *partials,
                          bool whole, cudaStream_t s);

// k_model.cu: train the learned leaf search on the current pivots (tmp >= 2 * kPieces);
// with after_batch the model is retrained only once merges above level 0 have
// rewritten enough leaves since the last training (decided on the device)
void launch_train_model(const Geo &g, ModelHead *head, Piece *pieces, const Ctl *ctl, bool after_batch,
                        cudaStream_t s);

// k_misc.cu
void launch_rebuild_indexes(const Geo &g, Ctl *ctl, cudaStream_t s);  // cnt, F, tree, row_end, total
void launch_check(const Geo &g, Ctl *ctl, uint32_t *code, cudaStream_t s);
// valid non-guard keys (or their dst ids) in slot order; count in ctl->gen_count
void launch_export(const Geo &g, Ctl *ctl, uint64_t *out_keys, uint32_t *out_cols, uint64_t cap, uint64_t *status,
                   cudaStream_t s);
void launch_degrees(const Geo &g, uint32_t *deg, cudaStream_t s);
void launch_rowptr(const uint32_t *deg, uint64_t *rowptr, uint32_t V, uint64_t *partials, cudaStream_t s);
// exclusive scan of u32 values into u64 (out[n] = total); partials >= scan_partials(n)
uint64_t scan_partials(uint64_t n);
// n_dev (optional): device-side element count, at most n_bound
void launch_scan_u32_u64(const uint32_t *in, uint64_t *out, uint64_t n_bound, uint64_t *partials, cudaStream_t s,
                         const uint32_t *n_dev = nullptr);

// k_analytics.cu
// PageRank: x0 (setup), then per iteration one sum pass and one apply.  y, cfx:
// u64[V] fixed point (2^60); cf: FP32 contributions of the first iteration
// (bucketed pass, else nullptr); dsum: u64[iters + 1]; partials >= 152 * 16;
// counter one unsigned (zeroed by setup, re-zeroed by each sum)
void launch_pr_setup(const Geo &g, uint32_t iters, float *rank, uint64_t *y, uint64_t *cfx, float *cf,
                     uint64_t *dsum, uint64_t *partials, unsigned *counter, cudaStream_t s);
void launch_pr_scatter(const Geo &g, const uint64_t *cfx, uint64_t *y, cudaStream_t s);
void launch_pr_apply(const Geo &g, float damping, float *rank, uint64_t *y, uint64_t *cfx,
                     const uint64_t *dsum_in, uint64_t *dsum_out, uint64_t *partials, unsigned *counter, bool last,
                     cudaStream_t s);
// Bucketed pass: buckets of kPbBucket heads, G chunks of the slot array, a
// cluster of nparts blocks per bucket.  cnt: u32[nb * G]; off: u64[nb * G + 1]
// (off[nb*G] = edges); scan_tmp: nb u32 bucket totals; keys:
// u64[edges] (<= C).  One iteration reads cf_in and writes cf_out (FP32 x/outdeg,
// V each), the ranks when last, and dsum_out; partials >= nb * nparts.
constexpr uint32_t kPbShift = 13, kPbMaxShift = 14;
constexpr uint32_t kPbMaxBuckets = 4096;  // heads < kPbMaxBuckets << shift
constexpr uint32_t kPbMaxChunks = 152 * 8, kPbTargetBlocks = 256, kPbMaxParts = 8;
// placement: slots per tile, threads (4096-slot tiles at 40 registers fit three blocks
// an SM; measured at R-MAT scale 20 against 8192-slot tiles at two blocks an SM:
// 0.38-0.41 against 0.42-0.45 ms of bucketing per call in the bench step)
constexpr uint32_t kPbTile = 4096, kPbPlaceThreads = 512;
// more buckets than this: placement without staging (a staged tile of 4096 slots,
// about half of them edges, then holds fewer than 8 edges of each bucket, too few to
// group the writes)
constexpr uint32_t kPbStageMax = 256;
struct PbPlan {
  uint32_t shift, nb, G, nparts, threads;  // 2^shift heads per bucket; threads per iteration block
  uint64_t chunk;  // slot pairs per chunk
};
PbPlan pb_plan(const Geo &g);
void launch_pb_build(const Geo &g, const PbPlan &p, uint32_t *cnt, uint64_t *off, uint64_t *scan_tmp, uint64_t *keys,
                     cudaStream_t s);
void launch_pb_iter(const Geo &g, const PbPlan &p, const uint64_t *keys, const uint64_t *off, float damping,
                    const float *cf_in, float *cf_out, float *rank, bool last, const uint64_t *dsum_in,
                    uint64_t *dsum_out, uint64_t *partials, unsigned *counter, cudaStream_t s);
// BFS in one cooperative launch; counter >= 16 u32, h_counter pinned; waits for the
// stream; returns 0, -1 on a CUDA error, -2 when a bounded barrier wait gave up
int run_bfs(const Geo &g, uint32_t src, int32_t *depth, uint32_t *q0, uint32_t *q1, uint32_t *q2,
            uint32_t *counter, Ctl *ctl, cudaStream_t s);
void launch_cc(const Geo &g, uint32_t *label, cudaStream_t s);

// per-warp shared memory of the leaf kernels: three key buffers of L, a u16
// index array of L+1 and a byte mask of L
__host__ __device__ inline uint32_t leaf_smem_bytes(uint32_t L) {
  return 24u * L + ((2u * (L + 1u) + 15u) & ~15u) + ((L + 15u) & ~15u);
}

// ---- many handles in one launch per stage (gpma_update_many) ------------------------------
constexpr uint32_t kMaxMany = 128;  // handles of one batched launch
constexpr uint32_t kMaxPlans = 32;  // batched launches with their own block ranges

// One handle of a batched update: the arguments its own front end and level-0
// pass take, and this call's sizes.
struct ManyItem {
  PrepArgs prep;
  const uint64_t *ins, *del;
  uint64_t *bufA, *bufB;  // radix ping-pong (the sorted words end in bufB after an odd pass count)
  uint32_t *hist;
  Ctl *ctl;
  const ModelHead *mhead;
  const Piece *mpieces;
  uint32_t active;        // this call updates the handle here (else: no kernel touches it)
  uint32_t small;         // the whole front end in one block (at most kSmallBatch keys)
  uint32_t T, T1, wide;   // sort tiles, search blocks, four sorted words a search thread
  uint32_t P, S;          // one-block front end: padded batch, sampled pivots
  uint32_t per_warp;      // general level-0 pass: shared memory of a warp
  Geo g;
  Work w;
};

// Block ranges of one batched launch: item[k] runs on blocks [start[k], start[k+1]),
// k < n (handles without blocks in the launch are left out).
struct ManyPlan {
  uint32_t n;
  uint32_t item[kMaxMany];
  uint32_t start[kMaxMany + 1];
};

struct ManyDesc {
  uint32_t count;
  ManyPlan plan[kMaxPlans];
  ManyItem item[kMaxMany];  // last: a call uploads the first `count` only
};

// The handle and its own block index of this block of launch `plan` (false: no work)
__device__ __forceinline__ bool many_block(const ManyDesc *d, uint32_t plan, const ManyItem **it, uint32_t *sub,
                                           uint32_t *nblk) {
  const ManyPlan &p = d->plan[plan];
  const uint32_t b = blockIdx.x, n = p.n;
  if (n == 0 || b >= p.start[n]) return false;
  uint32_t lo = 0, hi = n;  // the last k with start[k] <= b
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (p.start[mid] <= b) lo = mid;
    else hi = mid;
  }
  *it = &d->item[p.item[lo]];
  *sub = b - p.start[lo];
  *nblk = p.start[lo + 1] - p.start[lo];
  return true;
}

// Plans of a batched update, by stage; the general level-0 pass has one launch
// per group of handles sharing its block shape (leaf size, warps per block).
struct ManyPlans {
  uint32_t one;        // one block a handle
  uint32_t tiles;      // sort tiles at the handle's work capacity
  uint32_t radix;      // digits of the handle's radix passes
  uint32_t search[2];  // search blocks at one / four sorted words a thread
  uint32_t leaf64;     // 64-slot level-0 pass
  uint32_t deg;        // out-degree changes
  uint32_t ngroups;
  struct Group {  // handles whose one-warp-per-leaf pass has wpb warps per block
    uint32_t rest, long_a, long_b;  // plans (long_a == ~0u: no handle of the group has long runs)
    uint32_t wpb, per_warp;         // per_warp: the largest shared memory a warp of the group takes
  } group[8];
  uint32_t maxpass;
  uint32_t total[kMaxPlans];  // blocks of each plan's launch
};
// k_batch.cu / k_update.cu: the batched stages (kernels read d, which the call uploaded);
// prepare_* set the kernels' shared-memory limits (once, outside any stream capture)
void prepare_many_front();
void prepare_many_leaf();
void launch_many_front(const ManyDesc *d, const ManyPlans &pl, cudaStream_t s);
void launch_many_leaf(const ManyDesc *d, const ManyPlans &pl, cudaStream_t s);
uint32_t search_tiles(uint64_t nb);
uint32_t front_tiles(uint64_t nb);
bool search_wide(uint64_t n);
uint32_t leaf_pass_warps(uint32_t L, uint32_t want);  // warps per block of the general level-0 pass

// read-only view of a handle (defined beside the handle in gpma_api.cu)
struct HandleView {
  const Geo *geo;
  Ctl *ctl;
  Ctl *h_ctl;
  int poisoned;
};

}  // namespace gpk

struct gpma;
namespace gpk {
HandleView handle_view(struct gpma *h, cudaStream_t s);  // waits for a pending device resize
int poison_handle(struct gpma *h, int code);             // every later call returns `code`
// status of an export from the control block read back after it: a look-back
// wait that gave up poisons the handle with GPMA_ETIMEOUT
int export_status(struct gpma *h, uint32_t err);
}  // namespace gpk
