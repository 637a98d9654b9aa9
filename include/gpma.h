/*
 * gpma.h -- C ABI of libgpma: a dynamic graph stored on one GB300 GPU as a GPMA+
 * packed memory array (Sha, Li, He, Tan, "Accelerating Dynamic Graph Analytics on
 * GPUs").
 *
 * Storage (Sec. 4.1 "Background of PMA", Sec. 4.2 Example 4): a sorted array of
 * 64-bit keys (src << 32 | dst) with gaps (EMPTY = all ones), cut into leaf
 * segments of L slots; a segment at height i spans L * 2^i slots.  Every vertex
 * u owns a guard key (u << 32 | 0xFFFFFFFF) that sits right after its row, so
 * the array doubles as CSR: row u is the valid, non-guard slots between the
 * guard of u-1 and the guard of u.
 *
 * Conventions for every call:
 *  - pointers named d_* are DEVICE pointers owned by the caller; they must stay
 *    valid until the work enqueued on `stream` has finished;
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream); all work is stream-ordered on it;
 *  - the library owns the array and its scratch memory (allocated through the
 *    allocator given at create, else cudaMallocAsync on the call's stream);
 *  - every call returns a status code; no exception, abort or exit crosses the
 *    ABI.  GPMA_ETIMEOUT and GPMA_EDEVICE poison the handle: every later call
 *    on it returns the same code.  A handle is not thread safe; distinct
 *    handles are independent.
 *  - calls on one handle issued from one thread on DIFFERENT streams: the
 *    caller orders them with events, except that gpma_bfs, gpma_cc and
 *    gpma_pagerank only read the array and keep separate buffers, so one of
 *    each may run concurrently on separate streams once the first call of each
 *    kind has completed (first calls allocate).  Updates, exports and two calls
 *    of the same kind must not overlap.
 */
#ifndef GPMA_H
#define GPMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gpma *gpma_t;

#define GPMA_OK 0
#define GPMA_EINVAL 1   /* bad argument or key; the batch was not applied */
#define GPMA_ENOMEM 2   /* an allocation failed; the handle is unchanged, except when the
                           new array of a root resize was refused (the batch had begun
                           to apply): the handle is then poisoned */
#define GPMA_ECAP 3     /* output buffer too small; *n_out holds the size needed */
#define GPMA_ETIMEOUT 4 /* a bounded device-side wait gave up (handle poisoned) */
#define GPMA_EDEVICE 5  /* a CUDA runtime error (handle poisoned) */

#define GPMA_EMPTY 0xFFFFFFFFFFFFFFFFull
#define GPMA_RAW_KEYS 1u   /* keys are opaque integers < 2^63: no guards, no analytics */
#define GPMA_PLAIN_SEARCH 2u /* find leaves by binary search only (default: a learned two-stage
                                linear model over the leaf pivots narrows the search; both
                                give the same leaf, hence the same array) */
#define GPMA_DUAL_DELETE 4u /* deletion as the dual of insertion (Sec. 4.1): a touched leaf or
                                a merged segment must end within [min_i, max_i]; deletes leave
                                no holes; an underfull root halves.  Default: lazy deletion
                                (Sec. 6.1), slots become EMPTY in place */
#define GPMA_PUSH_PAGERANK 8u /* PageRank sums by one push pass over the slots per iteration
                                (a reduction per edge into the L2).  Default, for graphs
                                of at most 2^25 vertices: the edges are bucketed by head
                                once per call and each iteration sums every bucket in
                                shared memory.  Both give the same ranks, bit for bit */

#define GPMA_MAX_LEVELS 48

/* Create-time parameters; a zero field takes the default.  Densities are whole
 * percentages: tau_0 (leaf upper bound, default 92), tau_h (root upper bound, 80),
 * rho_0 (8) and rho_h (40), the running example of Sec. 4.1 / Fig. 3.  The
 * per-level bound is the largest count n with n < tau_i * L * 2^i, tau_i linear
 * in the level between tau_0 and tau_h, clamped to twice the child bound. */
typedef struct {
  uint32_t leaf_size; /* L: power of two in [2, 1024]; default 64 */
  uint32_t tau0_pct, tauh_pct, rho0_pct, rhoh_pct;
  uint32_t flags;     /* GPMA_RAW_KEYS | GPMA_PLAIN_SEARCH | GPMA_DUAL_DELETE |
                         GPMA_PUSH_PAGERANK, or 0 */
  uint32_t leaf_warps; /* warps per block of the level-0 pass that gives one warp to
                          each touched leaf (the pass for leaves other than 64 slots and
                          for the runs the 64-slot pass leaves over): 1, 2, 4 or 8, fewer
                          when a leaf's shared memory does not fit; 0 = the largest
                          count that fits 96 KB of shared memory, at most 8 (App. A: the
                          threads given to one segment are a tuning choice) */
} gpma_params;

/* Optional device allocator.  alloc returns NULL on failure; both receive the
 * cudaStream_t of the call as void*.  NULL allocator => cudaMallocAsync. */
typedef struct {
  void *(*alloc)(size_t bytes, void *stream, void *ctx);
  void (*free)(void *ptr, void *stream, void *ctx);
  void *ctx;
} gpma_allocator;

/* Per-batch statistics (filled only when a non-NULL pointer is passed, which
 * makes the call wait for the batch). */
typedef struct {
  uint64_t n_inserted;     /* inserts that took effect */
  uint64_t n_deleted;      /* deletes that took effect */
  uint64_t n_ignored;      /* raw inputs with no effect: duplicates, cancelled pairs,
                              inserts of stored keys, deletes of absent keys */
  uint32_t levels_climbed; /* highest level at which a segment merged; old h + 1 on a resize */
  uint32_t resized;        /* 1 if the capacity grew, 2 if it shrank (GPMA_DUAL_DELETE) */
  uint64_t alg_bytes;      /* algorithmic bytes of the batch: 8 per raw key, 8L per touched leaf
                              (read), 8L per covered leaf (write), 8L per covered leaf not
                              touched (read), 8 per EMPTY written outside covered leaves; on a
                              resize 8 per raw key + 8L per touched leaf + 8 (C_old + C_new) */
  uint64_t touched_leaves; /* distinct leaves holding an update after cancellation */
  uint64_t covered_leaves; /* leaves rewritten by merges (0 on a resize) */
  uint64_t merges[GPMA_MAX_LEVELS]; /* segments merged at each level, Sec. 5.2 level order */
  uint64_t delete_leaves;  /* distinct leaves holding a delete that took effect */
  uint32_t model_sorted;   /* 1: the batch was sorted by bucketing its keys on the learned
                              model's pieces and sorting each bucket (learned handles); 0:
                              by the radix passes (plain handles, small batches, no trained
                              model yet, or a bucket too large for shared memory).  Either
                              way the sorted batch, and so every result, is the same */
  uint32_t pad;
} gpma_stats;

/* Create an array for vertices [0, n_vertices) (n_vertices in [1, 2^31]; ignored
 * with GPMA_RAW_KEYS) and load one guard per vertex through the update path
 * (bulk load = update, Sec. 5.2).  params may be NULL.  On success *out owns the
 * handle; the call waits for the stream. */
int gpma_create(uint32_t n_vertices, const gpma_params *params, const gpma_allocator *alloc,
                void *stream, gpma_t *out);

/* Free the handle and all library memory (waits for the handle's last stream). */
int gpma_destroy(gpma_t h);

/* Apply one batch of edge insertions and deletions (Algorithm "GPMA+
 * Segment-Oriented Insertion", Sec. 5.2, with lazy deletion, Sec. 6.1, or with
 * the lower bounds kept when the handle was created with GPMA_DUAL_DELETE).
 * d_ins[n_ins], d_del[n_del]: device arrays of keys (src << 32 | dst), in any
 * order, duplicates allowed.  Semantics: each list is made unique; a key in both
 * lists is dropped from both; inserts of stored keys and deletes of absent keys
 * are ignored; deletes empty their slot in place; inserts go to their leaf (the
 * last leaf whose smallest key is <= the key, before the batch) and every
 * segment holding pending inserts merges and re-spreads evenly at the lowest
 * level whose bound admits it; above the root the capacity doubles until all
 * keys fit.  Every key must have src, dst < n_vertices (raw mode: key < 2^63),
 * else GPMA_EINVAL and nothing changes.  n_ins + n_del < 2^30.
 * With stats == NULL the call returns after enqueueing; a batch that might
 * overflow the root grows the array on the device into a preallocated spare of
 * twice the capacity, and the next call on the handle first waits for that batch
 * to learn the geometry.  Only a batch that might need more than one doubling
 * (a bulk load) waits inside the call.  A device-detected
 * GPMA_EINVAL is then reported by the next gpma_status().  With stats != NULL
 * the call waits and returns the batch's status. */
int gpma_update_batch(gpma_t h, const uint64_t *d_ins, uint64_t n_ins, const uint64_t *d_del,
                      uint64_t n_del, void *stream, gpma_stats *stats);

/* Apply one batch to each of `count` distinct handles: the update of Sec. 5.2
 * applied to many independent graphs at once.  d_ins[i][n_ins[i]] and
 * d_del[i][n_del[i]] go to handles[i] with exactly the semantics of
 * gpma_update_batch; each handle ends as if its batch had been applied alone.
 * Batches that cannot overflow their root run together: every stage of the front
 * end (validation, radix passes, unique/cancel + leaf search, run heads) and of the
 * level-0 pass is one kernel launch over the work of all those handles, each block
 * finding its handle in a table uploaded by the call; a handle whose inserts did not
 * all fit their leaves runs its merge levels in its own branch of the same CUDA
 * graph, taken only then (a conditional node).  The graph is captured once per set
 * of handles and sizes and replayed by later calls.  The other batches (a possible
 * root resize, dual deletion) take gpma_update_batch's path on side streams forked
 * from `stream`.  Work enqueued on `stream` afterwards sees every batch applied.
 * Returns the first host-detected error; device-detected GPMA_EINVAL is reported per
 * handle by gpma_status().  The handles must not be in use on other streams
 * meanwhile; calls from several host threads are serialised. */
int gpma_update_many(gpma_t const *handles, const uint64_t *const *d_ins, const uint64_t *n_ins,
                     const uint64_t *const *d_del, const uint64_t *n_del, uint32_t count, void *stream);

/* Wait for `stream` and return (then clear) the first device-side error of the
 * batches enqueued without stats. */
int gpma_status(gpma_t h, void *stream);

/* Breadth-first search from src over out-edges (Algorithm "BFS", Sec. 4.2, with
 * the gap test of Algorithm "GPU-based BFS Neighbour Gathering").  d_depth[V]
 * receives the hop count, -1 where unreachable.  Asynchronous: one cooperative
 * kernel whose grid barriers are bounded; a barrier that gave up is reported as
 * GPMA_ETIMEOUT by the next gpma_status (the depths are then not valid). */
int gpma_bfs(gpma_t h, uint32_t src, int32_t *d_depth, void *stream);

/* Weakly connected components (the Connected Component application of Sec. 6.1
 * on the directed graph read as undirected).  d_label[V] receives, for every
 * vertex, the smallest vertex id of its component.  Stream-ordered. */
int gpma_cc(gpma_t h, uint32_t *d_label, void *stream);

/* PageRank by power iteration (Sec. 6.1): x0 = 1/V and `iters` steps of
 * x'_v = (1-d)/V + d * (sum_{u->v} x_u / outdeg(u) + (sum of x over vertices
 * without out-edges) / V).  d_rank[V] receives FP32 ranks.  Each quotient
 * x_u / outdeg(u) is formed in FP32 and rounded once to fixed point with 60
 * fractional bits; the sums over edges are exact integer sums, so the ranks do not
 * depend on the order of the edges or of the reductions.  The first call
 * allocates the pass's buffers (with the bucketed pass: an edge copy as large as
 * the slot array).  Stream-ordered. */
int gpma_pagerank(gpma_t h, uint32_t iters, float damping, float *d_rank, void *stream);

/* PageRank in two steps, so that updates need not wait for the iterations (the
 * stream of Sec. 3 keeps flowing while a query runs).  gpma_pagerank_snapshot takes
 * a snapshot of the graph on `stream`: the stored edges bucketed by head and the
 * out-degrees, in buffers of the handle.  gpma_pagerank_run then iterates exactly
 * as gpma_pagerank does, but over the last snapshot only: once the snapshot's work
 * has completed (an event recorded after it), updates may run on other streams
 * while the iterations run, and the ranks are those of the graph at snapshot time.
 * A new snapshot, or a gpma_pagerank call (which rebuilds the same buffers and
 * discards the snapshot), must not start before the runs on the previous one have
 * finished; runs share their scratch with each other and with gpma_pagerank, so
 * they must not overlap on the GPU either.  gpma_pagerank_snapshot returns
 * GPMA_EINVAL for a handle that sums by the push pass (GPMA_PUSH_PAGERANK, or more
 * than 2^25 vertices), which reads the array itself; gpma_pagerank_run returns
 * GPMA_EINVAL without a snapshot. */
int gpma_pagerank_snapshot(gpma_t h, void *stream);
int gpma_pagerank_run(gpma_t h, uint32_t iters, float damping, float *d_rank, void *stream);

/* Copy the stored edges (no guards) in ascending key order into d_out[cap]:
 * the edge set a query of the stream model sees (Sec. 3, "Graph Streams" and the
 * query buffer of Fig. 1), read off the gapped array in slot order.  *n_out =
 * number of edges.  GPMA_ECAP (nothing written past cap) if cap is too small;
 * GPMA_ETIMEOUT (handle poisoned) if a look-back wait of the compaction gave up.
 * Waits for the stream. */
int gpma_export_sorted(gpma_t h, uint64_t *d_out, uint64_t cap, uint64_t *n_out, void *stream);

/* Same result as gpma_export_sorted, but the call allocates no device memory:
 * the paper has no counterpart.  It is meant for callers that must not allocate
 * while they query the graph, for instance a serving loop that has handed all
 * free device memory to its own pool, or latency-bound code that cannot accept
 * the synchronisation an allocation may bring.  The scratch words of its
 * single-pass compaction live in one fixed array inside the library (about
 * 512 KiB per GPU, kept until the process exits), so the array may hold at most 2^27 slots
 * (GPMA_EINVAL otherwise).  The first call on each device looks up that array's
 * device address; make that first call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU (other streams, other handles)
 * race and must not be issued.  A look-back wait that gave up returns
 * GPMA_ETIMEOUT and a CUDA error GPMA_EDEVICE; both poison the handle.  Waits
 * for the stream. */
int gpma_export_sorted_noalloc(gpma_t h, uint64_t *d_out, uint64_t cap, uint64_t *n_out, void *stream);

/* CSR view (Sec. 4.2, Fig. 5): d_rowptr[V+1] row offsets, d_col[cap] column ids
 * (dst).  *n_out = number of edges; GPMA_ECAP if cap is too small.  Waits. */
int gpma_export_csr(gpma_t h, uint64_t *d_rowptr, uint32_t *d_col, uint64_t cap,
                    uint64_t *n_out, void *stream);

/* Copy the raw array (EMPTY slots and guards included) into d_slots[cap]: the
 * packed memory array itself, leaf segments of L slots with their gaps (Sec. 4.1,
 * Fig. 3; guards as in Sec. 4.2, Fig. 5).  *capacity_out = number of slots.
 * GPMA_ECAP if cap is too small. */
int gpma_export_layout(gpma_t h, uint64_t *d_slots, uint64_t cap, uint64_t *capacity_out,
                       void *stream);

/* Replace the array with d_slots[capacity] (capacity = L * 2^k; valid keys
 * strictly increasing; in graph mode one guard per vertex): a layout of the
 * packed memory array of Sec. 4.1 as gpma_export_layout writes it, every leaf
 * within its bound and the CSR guards of Sec. 4.2 in place.  Used to restore a
 * snapshot and by tests.  GPMA_EINVAL if the capacity is not L * 2^k or the
 * layout fails the device checker (the handle is then unchanged). Waits. */
int gpma_import_layout(gpma_t h, const uint64_t *d_slots, uint64_t capacity, void *stream);

/* d_row_end[V] = slot index of the guard of each vertex.  Stream-ordered. */
int gpma_row_end(gpma_t h, uint32_t *d_row_end, void *stream);

/* Number of stored edges (guards excluded; raw mode: keys): |E| of the graph
 * the stream has built so far (Sec. 3).  Waits. */
int gpma_num_edges(gpma_t h, uint64_t *out, void *stream);

/* Current number of slots, L * 2^h: the capacity of the root segment, which
 * doubles when the root exceeds its upper density bound (Sec. 4.1, and the root
 * case of Algorithm "GPMA+ Segment-Oriented Insertion", Sec. 5.2). */
int gpma_capacity(gpma_t h, uint64_t *out);

/* Device-side consistency check of the array and its indexes.  *code = 0 when
 * all hold, else a bit set: 1 keys not strictly increasing, 2 a leaf count or
 * first-key index is stale, 4 a leaf above its bound, 8 a guard index is stale,
 * 16 a merge mark was left set, 32 the total count is stale, 64 an out-degree is
 * stale, 128 a leaf has a hole (GPMA_DUAL_DELETE only).  Waits. */
int gpma_check(gpma_t h, uint32_t *code, void *stream);

/* Bound every device-side wait of this handle (look-back of the single-pass
 * sorts, scans and exports; grid barriers of gpma_bfs) to `polls` polls of the
 * awaited word; 0 restores the built-in limits (about a second).  A wait that
 * runs out makes its kernel return; the call (or the next gpma_status, for calls
 * that return before the work ends) reports GPMA_ETIMEOUT and poisons the handle.
 * The paper has no counterpart: this is failure detection for callers that would
 * rather give up than wait.  Stream-ordered: calls enqueued later on `stream`
 * use the new limit. */
int gpma_set_wait_limit(gpma_t h, uint32_t polls, void *stream);

/* ---- measurement ------------------------------------------------------------
 * Optional per-phase timing.  While enabled, every call records a pair of CUDA
 * events on its own stream around each phase below (one pair per PageRank push
 * pass), so the times are device times of the work actually enqueued. */
#define GPMA_PROF_SORT 0       /* validation, radix sort, unique/cancel, leaf search, runs */
#define GPMA_PROF_LEAF 1       /* leaf pass (presence, deletes, level-0 merges) + count tree */
#define GPMA_PROF_ESCALATE 2   /* pending inserts, merge levels, outer segment merges */
#define GPMA_PROF_RESIZE 3     /* root resize */
#define GPMA_PROF_PR_SCATTER 4 /* one PageRank sum pass (bucketed, or push over the slots) */
#define GPMA_PROF_PAGERANK 5   /* one whole gpma_pagerank call */
#define GPMA_PROF_BFS 6        /* one whole gpma_bfs call */
#define GPMA_PROF_CC 7         /* one whole gpma_cc call */
#define GPMA_PROF_UPDATE 8     /* one whole gpma_update_batch call (replayed batches run as one
                                  CUDA graph: then only this phase is recorded) */
#define GPMA_PROF_PR_BUCKET 9  /* bucketing the edges by head, once per gpma_pagerank call */
#define GPMA_PROF_N 10

typedef struct {
  double ms[GPMA_PROF_N];         /* summed device time */
  uint64_t count[GPMA_PROF_N];    /* timed occurrences */
  uint64_t launches[GPMA_PROF_N]; /* kernel launches inside those occurrences */
} gpma_profile;

/* Turn per-phase event recording on (on != 0) or off. */
int gpma_profile_enable(gpma_t h, int on);

/* Wait for the recorded events and sum them into *out; reset != 0 clears the
 * accumulated record afterwards. */
int gpma_profile_read(gpma_t h, gpma_profile *out, int reset);

/* Number of kernels this library has launched in this process (all handles). */
uint64_t gpma_launch_count(void);

/* Static text for a status code. */
const char *gpma_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* GPMA_H */
