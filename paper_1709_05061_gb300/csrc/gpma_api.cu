// gpma_api.cu -- the C ABI of include/gpma.h: handle, memory, and the order in
// which one batch's kernels are enqueued.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "gpma.h"
#include "gpma_launch.h"

using namespace gpk;

namespace {
std::atomic<uint64_t> g_launches{0};
}  // namespace

namespace gpk {
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void unnote_launches(uint64_t k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }
}  // namespace gpk

namespace {

// Threshold reading (Sec. 4.1 and the Fig. 3 table): tau_i and rho_i interpolate
// linearly in the level between leaf and root in whole hundredths; max_i is the
// largest count below tau_i * L * 2^i, clamped to twice the level below.
void level_bounds(uint32_t L, uint32_t h, uint32_t t0, uint32_t th, uint64_t *mx) {
  for (uint32_t i = 0; i <= h; i++) {
    const uint64_t seg = (uint64_t)L << i;
    uint64_t num, den;
    if (h == 0) {
      num = (uint64_t)t0 * seg;
      den = 100;
    } else {
      num = ((uint64_t)th * h + (uint64_t)(t0 - th) * (h - i)) * seg;
      den = 100ull * h;
    }
    uint64_t b = (num - 1) / den;
    if (i > 0 && b > 2 * mx[i - 1]) b = 2 * mx[i - 1];
    mx[i] = b;
  }
}

// min_i = floor(rho_i * c_i) + 1 clamped to 2 min_{i-1}, rho_i linear in the
// level between rho_0 (leaf) and rho_h (root), in exact integer hundredths
void level_min_bounds(uint32_t L, uint32_t h, uint32_t r0, uint32_t rh, uint64_t *mn) {
  for (uint32_t i = 0; i <= h; i++) {
    const uint64_t seg = (uint64_t)L << i;
    uint64_t num, den;
    if (h == 0) {
      num = (uint64_t)r0 * seg;
      den = 100;
    } else {
      num = ((uint64_t)rh * h - (uint64_t)(rh - r0) * (h - i)) * seg;
      den = 100ull * h;
    }
    uint64_t b = num / den + 1;
    if (i > 0 && b > 2 * mn[i - 1]) b = 2 * mn[i - 1];
    mn[i] = b;
  }
}

uint32_t bits_for(uint64_t x) {
  uint32_t b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

}  // namespace

// event pairs recorded around phases while profiling is on
struct Prof {
  bool on = false;
  struct Pair {
    cudaEvent_t a, b;
    int phase;
    uint64_t launches;
  };
  std::vector<Pair> pairs;
  std::vector<cudaEvent_t> pool;
  double ms[GPMA_PROF_N] = {};
  uint64_t count[GPMA_PROF_N] = {};
  uint64_t launches[GPMA_PROF_N] = {};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  ~Prof() {
    for (auto &p : pairs) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// brackets one phase of one call with events on the call's stream
struct Phase {
  Prof *p;
  int phase;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  uint64_t l0 = 0;
  bool open = false;
  Phase(Prof *p_, int ph, cudaStream_t s_) : p(p_), phase(ph), s(s_) {
    if (p && p->on) {
      a = p->get();
      cudaEventRecord(a, s);
      l0 = gpk::launch_count();
      open = true;
    }
  }
  void end() {
    if (!open) return;
    cudaEvent_t b = p->get();
    cudaEventRecord(b, s);
    p->pairs.push_back({a, b, phase, gpk::launch_count() - l0});
    open = false;
  }
  ~Phase() { end(); }
};

// Instantiated CUDA graphs of the post-prep part of a batch, one per batch-size
// bucket (and stats flag).  A graph bakes in device pointers, so every
// (re)allocation of an array it touches bumps the handle's alloc epoch and
// retires the graphs captured before.
struct GraphCache {
  struct Entry {
    cudaGraphExec_t exec = nullptr;
    uint64_t bucket = 0, epoch = 0, used = 0;
    bool stats = false;
    uint64_t kernels = 0;
  };
  static constexpr int kEntries = 8;
  Entry e[kEntries];
  cudaStream_t cap = nullptr, cap2 = nullptr;
  uint64_t tick = 0;
  bool enabled = true;
  Entry *find(uint64_t bucket, uint64_t epoch, bool stats) {
    for (auto &x : e)
      if (x.exec && x.bucket == bucket && x.epoch == epoch && x.stats == stats) {
        x.used = ++tick;
        return &x;
      }
    return nullptr;
  }
  Entry *victim() {
    Entry *v = &e[0];
    for (auto &x : e) {
      if (!x.exec) return &x;
      if (x.used < v->used) v = &x;
    }
    cudaGraphExecDestroy(v->exec);
    v->exec = nullptr;
    return v;
  }
  ~GraphCache() {
    for (auto &x : e)
      if (x.exec) cudaGraphExecDestroy(x.exec);
    if (cap) cudaStreamDestroy(cap);
    if (cap2) cudaStreamDestroy(cap2);
  }
};

struct gpma {
  uint32_t V, L, logL, raw;
  uint32_t tau0, tauh, rho0, rhoh;
  gpma_allocator alloc;
  bool has_alloc;
  Geo geo;
  Ctl *ctl;
  Ctl *h_ctl;
  // per-batch work arrays
  Work w;
  uint64_t *bufA, *bufB;
  uint32_t *hist;
  uint64_t status_cap;
  uint32_t cap;  // key capacity of the work arrays
  // segment merge scratch
  uint64_t *scratch;
  uint64_t scratch_cap;
  uint32_t *vbuf;
  uint64_t vbuf_leaves;
  uint64_t *partials;
  uint64_t partials_cap;
  // analytics
  uint64_t *y;    // PageRank sums, fixed point
  uint64_t *cfx;  // PageRank contributions x/outdeg, fixed point
  uint64_t *dsum;
  uint32_t dsum_cap;
  uint32_t *q0, *q1, *q2, *counter, *h_counter;
  uint64_t *pr_partials;
  unsigned *pr_counter;
  // bucketed PageRank: per-chunk bucket counts and their scan, the edges by head
  // bucket (as many slots as the array, grown with it), per-block dangling sums
  bool push_pr;  // GPMA_PUSH_PAGERANK
  uint32_t *pb_cnt;
  uint64_t *pb_off, *pb_scan, *pb_keys, *pb_dang;
  uint64_t pb_keys_cap;
  // the snapshot the iterations read: the bucketed copy above plus the out-degrees
  // at snapshot time, and the plan it was built with
  uint32_t *pb_deg;
  PbPlan snap_plan;
  bool snap_valid;
  uint32_t *check_buf;
  uint64_t *guards;
  uint64_t count_ub;
  uint64_t count_lb;  // a lower bound of the stored key count (dual mode: root underflow check)
  uint32_t dual;      // GPMA_DUAL_DELETE
  int poisoned;
  int host_sticky;
  Prof *prof;
  GraphCache *graphs;
  uint64_t alloc_epoch;
  // learned leaf search (nullptr with GPMA_PLAIN_SEARCH)
  ModelHead *mhead;
  Piece *mpieces;
  uint32_t since_train;
  // device-side root resize: the array of height h+1 a batch may grow into, and
  // the control block such a batch sends back (read before the next call)
  Geo spare;
  bool has_spare;
  Ctl *h_mirror;
  cudaEvent_t ev_mirror;
  bool mirror_pending;
  uint32_t leaf_warps;  // warps per block of the general level-0 pass (0: by shared memory)
  uint64_t uid;         // unique per handle created in the process (keys of batched graphs)
  uint64_t spare_epochs;  // the alloc_epoch steps that only allocated a spare (batched graphs ignore them)
};

namespace {

void *dmalloc(gpma *h, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  if (h->has_alloc) {
    p = h->alloc.alloc(bytes, (void *)s, h->alloc.ctx);
  } else if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

void dfree(gpma *h, void *p, cudaStream_t s) {
  if (!p) return;
  if (h->has_alloc) h->alloc.free(p, (void *)s, h->alloc.ctx);
  else cudaFreeAsync(p, s);
}

template <typename T>
bool dalloc(gpma *h, T **p, size_t count, cudaStream_t s) {
  *p = (T *)dmalloc(h, sizeof(T) * count, s);
  return *p != nullptr;
}

int poison(gpma *h, int code) {
  if (!h->poisoned) h->poisoned = code;
  return code;
}

int cuda_ok(gpma *h) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "libgpma: CUDA error %s\n", cudaGetErrorString(e));
    return poison(h, GPMA_EDEVICE);
  }
  return GPMA_OK;
}

// geometry of an array of height hh (device pointers not set)
void make_geo(gpma *h, uint32_t hh, Geo *g) {
  memset(g, 0, sizeof(Geo));
  g->L = h->L;
  g->logL = h->logL;
  g->h = hh;
  g->V = h->V;
  g->raw = h->raw;
  g->nleaves = 1ull << hh;
  g->C = (uint64_t)h->L << hh;
  uint64_t off = 0;
  for (uint32_t i = 1; i <= hh; i++) {
    g->tree_off[i] = off;
    off += g->nleaves >> i;
  }
  level_bounds(h->L, hh, h->tau0, h->tauh, g->maxc);
  level_min_bounds(h->L, hh, h->rho0, h->rhoh, g->minc);
  g->dual = h->dual;
  g->leaf_warps = h->leaf_warps;
}

bool alloc_arrays(gpma *h, Geo *g, cudaStream_t s) {
  const uint64_t tn = g->nleaves > 1 ? g->nleaves - 1 : 1;
  g->slots = nullptr;
  g->cnt = nullptr;
  g->F = nullptr;
  g->tree = nullptr;
  g->mark = nullptr;
  bool ok = dalloc(h, &g->slots, g->C, s) && dalloc(h, &g->cnt, g->nleaves, s) && dalloc(h, &g->F, g->nleaves, s) &&
            dalloc(h, &g->tree, tn, s) && dalloc(h, &g->mark, tn, s);
  if (ok) ok = cudaMemsetAsync(g->mark, 0, sizeof(uint32_t) * tn, s) == cudaSuccess;
  return ok;
}

void free_arrays(gpma *h, Geo *g, cudaStream_t s) {
  dfree(h, g->slots, s);
  dfree(h, g->cnt, s);
  dfree(h, g->F, s);
  dfree(h, g->tree, s);
  dfree(h, g->mark, s);
  g->slots = nullptr;
  g->cnt = nullptr;
  g->F = nullptr;
  g->tree = nullptr;
  g->mark = nullptr;
}

void free_work(gpma *h, cudaStream_t s) {
  Work &w = h->w;
  void *ptrs[] = {h->bufA,   h->bufB,     w.ukey,  w.utag,     w.uleaf,   w.run_start, w.eflag,
                  w.rleaf,   w.rdelta,    w.rinfo, w.rdel,     w.pkey,    w.pleaf,     w.erun, w.eleaf,
                  w.elvl,    w.etop,      w.seg_node, w.seg_top, w.seg_pstart, w.seg_lpre, w.status, w.rs,
                  w.lbkt,    w.lcnt,      w.lrank};
  for (void *p : ptrs) dfree(h, p, s);
  memset(&h->w, 0, sizeof(Work));
  h->bufA = h->bufB = nullptr;
  h->cap = 0;
  h->status_cap = 0;
}

// work arrays for batches of up to n keys (grown geometrically)
int ensure_work(gpma *h, uint64_t n, cudaStream_t s) {
  if (n <= h->cap && h->w.status) return GPMA_OK;
  uint64_t cap = h->cap ? h->cap : 4096;
  while (cap < n) cap *= 2;
  free_work(h, s);
  Work &w = h->w;
  const uint64_t c1 = cap + 1;
  const uint64_t st = (uint64_t)comp_tiles(cap) * 2 + 64;
  bool ok = dalloc(h, &h->bufA, cap, s) && dalloc(h, &h->bufB, cap, s) && dalloc(h, &w.ukey, cap, s) &&
            dalloc(h, &w.utag, cap, s) && dalloc(h, &w.uleaf, cap, s) && dalloc(h, &w.run_start, c1, s) &&
            dalloc(h, &w.eflag, cap, s) && dalloc(h, &w.rleaf, cap, s) && dalloc(h, &w.rdelta, cap, s) &&
            dalloc(h, &w.rinfo, cap, s) && dalloc(h, &w.rdel, cap, s) && dalloc(h, &w.pkey, cap, s) &&
            dalloc(h, &w.pleaf, cap, s) && dalloc(h, &w.erun, c1, s) && dalloc(h, &w.eleaf, cap, s) && dalloc(h, &w.elvl, cap, s) &&
            dalloc(h, &w.etop, cap, s) && dalloc(h, &w.seg_node, c1, s) && dalloc(h, &w.seg_top, c1, s) &&
            dalloc(h, &w.seg_pstart, c1, s) && dalloc(h, &w.seg_lpre, c1, s) && dalloc(h, &w.status, st, s) &&
            dalloc(h, &w.rs, front_scratch_words(cap), s) && dalloc(h, &w.lbkt, cap, s) &&
            dalloc(h, &w.lcnt, (uint64_t)kPieces + 1, s) && dalloc(h, &w.lrank, cap, s);
  if (!ok) {
    free_work(h, s);
    return GPMA_ENOMEM;
  }
  cudaMemsetAsync(w.status, 0, sizeof(uint64_t) * st, s);
  h->alloc_epoch++;
  h->cap = (uint32_t)cap;
  h->status_cap = st;
  w.cap = (uint32_t)cap;
  return GPMA_OK;
}

// look-back status words for a scan over n elements (exports over the whole array)
int ensure_status(gpma *h, uint64_t n, cudaStream_t s) {
  const uint64_t need = (uint64_t)comp_tiles(n) * 2 + 64;
  if (need <= h->status_cap) return GPMA_OK;
  dfree(h, h->w.status, s);
  if (!dalloc(h, &h->w.status, need, s)) {
    h->status_cap = 0;
    return GPMA_ENOMEM;
  }
  cudaMemsetAsync(h->w.status, 0, sizeof(uint64_t) * need, s);
  h->alloc_epoch++;
  h->status_cap = need;
  return GPMA_OK;
}

// scratch of the segment merge: gathered keys (up to C) and per-leaf offsets
int ensure_merge_scratch(gpma *h, cudaStream_t s) {
  const Geo &g = h->geo;
  if (h->scratch_cap < g.C) {
    dfree(h, h->scratch, s);
    if (!dalloc(h, &h->scratch, g.C, s)) {
      h->scratch_cap = 0;
      return GPMA_ENOMEM;
    }
    h->scratch_cap = g.C;
    h->alloc_epoch++;
  }
  if (h->vbuf_leaves < g.nleaves) {
    dfree(h, h->vbuf, s);
    dfree(h, h->partials, s);
    const uint64_t bytes = (g.nleaves + 1) * 4 + 16 + (g.nleaves + 1) * 8;
    h->vbuf = (uint32_t *)dmalloc(h, bytes, s);
    h->partials_cap = scan_partials(g.nleaves + 1) + 1;
    h->partials = (uint64_t *)dmalloc(h, h->partials_cap * 8, s);
    if (!h->vbuf || !h->partials) {
      h->vbuf_leaves = 0;
      return GPMA_ENOMEM;
    }
    h->vbuf_leaves = g.nleaves;
    h->alloc_epoch++;
  }
  return GPMA_OK;
}

__global__ void k_finish(Ctl *ctl) { ctl->sticky |= ctl->err; }

__global__ void k_set_wait_limit(Ctl *ctl, uint32_t polls) { ctl->spin_limit = polls; }

__global__ void k_make_guards(uint64_t *g, uint32_t V) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < V; u += gridDim.x * blockDim.x)
    g[u] = ((uint64_t)u << 32) | 0xFFFFFFFFull;
}

int err_to_status(uint32_t err) {
  if (err & kErrTimeout) return GPMA_ETIMEOUT;
  if (err & kErrInternal) return GPMA_EDEVICE;
  if (err & kErrKey) return GPMA_EINVAL;
  return GPMA_OK;
}

int read_ctl(gpma *h, cudaStream_t s) {
  cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return poison(h, GPMA_EDEVICE);
  return GPMA_OK;
}

void train_model(gpma *h, cudaStream_t s, bool after_batch = false) {
  if (!h->mhead) return;
  launch_train_model(h->geo, h->mhead, h->mpieces, h->ctl, after_batch, s);
  if (!after_batch) h->since_train = 0;
}

// Rebuild the whole array at height h2: every valid key and every pending insert
// of the batch spread evenly over the new array (segment merge in whole mode).
int rebuild_at(gpma *h, uint32_t h2, cudaStream_t s) {
  Geo &old = h->geo;
  int rc = ensure_merge_scratch(h, s);
  if (rc) return poison(h, rc);
  Geo g2;
  make_geo(h, h2, &g2);
  g2.row_end = old.row_end;
  g2.deg = old.deg;
  if (!alloc_arrays(h, &g2, s)) {
    free_arrays(h, &g2, s);
    return poison(h, GPMA_ENOMEM);
  }
  launch_segment_merge(old, g2, h->ctl, h->w, h->scratch_cap, old.nleaves, h->scratch, h->vbuf, h->partials,
                       true, s);
  free_arrays(h, &old, s);
  h->geo = g2;
  h->alloc_epoch++;
  train_model(h, s);
  return cuda_ok(h);
}

// smallest height whose root bound holds `total` keys, searching from h0 upwards
// (0 when none below the limits: the caller checks against the current height)
uint32_t smallest_height(const gpma *h, uint64_t total, uint32_t h0) {
  uint64_t mx[kMaxLv];
  for (uint32_t h2 = h0;; h2++) {
    if (h2 >= kMaxLv - 1 || ((uint64_t)h->L << h2) > (1ull << 32) || (1ull << h2) >= (1ull << 30)) return kMaxLv;
    level_bounds(h->L, h2, h->tau0, h->tauh, mx);
    if (total <= mx[h2]) return h2;
  }
}

// root resize (reading R7): the smallest taller array whose root bound holds
// every valid key and every pending insert
int do_resize(gpma *h, uint64_t total, cudaStream_t s) {
  const uint32_t h2 = smallest_height(h, total, h->geo.h + 1);
  if (h2 >= kMaxLv) return poison(h, GPMA_ENOMEM);
  return rebuild_at(h, h2, s);
}

// dual deletion: a root below min_h is rebuilt at the smallest height that holds
// its keys, if that is lower (nothing is pending: the batch is complete)
int maybe_shrink(gpma *h, uint64_t total, cudaStream_t s, bool *shrunk) {
  *shrunk = false;
  if (h->geo.h == 0 || total >= h->geo.minc[h->geo.h]) return GPMA_OK;
  const uint32_t h2 = smallest_height(h, total, 0);
  if (h2 >= h->geo.h) return GPMA_OK;
  if (cudaMemsetAsync(&h->ctl->npend, 0, sizeof(uint32_t), s) != cudaSuccess) return poison(h, GPMA_EDEVICE);
  *shrunk = true;
  return rebuild_at(h, h2, s);
}

__global__ void k_gate(const Ctl *ctl, cudaGraphConditionalHandle cond) {
  cudaGraphSetConditional(cond, (ctl->err == 0 && ctl->nesc > 0) ? 1u : 0u);
}

// after the merge levels of a batch that may overflow the root: either some
// pending run fits no level (grow into the spare array) or the usual merges run
__global__ void k_gate_grow(Ctl *ctl, cudaGraphConditionalHandle grow, cudaGraphConditionalHandle merge) {
  const bool esc = ctl->err == 0 && ctl->nesc > 0;
  const bool g = esc && ctl->nfail > 0;
  ctl->resized = g ? 1u : 0u;
  cudaGraphSetConditional(grow, g ? 1u : 0u);
  cudaGraphSetConditional(merge, (esc && !g) ? 1u : 0u);
}

// Append an IF node on `cond` to the graph being captured on `cap`, and capture
// `body` (launches on the stream it is given) into the node's body graph.
template <typename Body>
bool capture_if(cudaStream_t cap, cudaStream_t cap2, cudaGraphConditionalHandle cond, Body body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  if (cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cg, &deps, nullptr, &ndeps) != cudaSuccess) return false;
  // zero-initialised storage: the parameter union has no default constructor
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)] = {};
  cudaGraphNodeParams *p = reinterpret_cast<cudaGraphNodeParams *>(raw);
  p->type = cudaGraphNodeTypeConditional;
  p->conditional.handle = cond;
  p->conditional.type = cudaGraphCondTypeIf;
  p->conditional.size = 1;
  cudaGraphNode_t cnode = nullptr;
  if (cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, p) != cudaSuccess) return false;
  cudaGraph_t bgraph = p->conditional.phGraph_out[0];
  if (cudaStreamUpdateCaptureDependencies(cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    return false;
  if (cudaStreamBeginCaptureToGraph(cap2, bgraph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess)
    return false;
  body(cap2);
  cudaGraph_t out = nullptr;
  return cudaStreamEndCapture(cap2, &out) == cudaSuccess;
}

// Capture the part of a batch after k_prep as one graph, grids sized for `nb`
// keys.  The escalation (pending inserts, count tree, merge levels, outermost
// segments, segment merge) sits in the body of an IF node that runs only when
// some leaf could not take its inserts, which a sliding window rarely produces.
// With `grow` (the batch might overflow the root, reading R7) the merge levels
// also count the runs no level admits, and two more IF nodes follow: the root
// resize into the preallocated spare array of height h+1, or the usual merges.
bool capture_update(gpma *h, FrontArgs &f, uint32_t nb, bool stats, bool grow, GraphCache::Entry **out) {
  GraphCache &gc = *h->graphs;
  if (!gc.cap && cudaStreamCreateWithFlags(&gc.cap, cudaStreamNonBlocking) != cudaSuccess) return false;
  if (!gc.cap2 && cudaStreamCreateWithFlags(&gc.cap2, cudaStreamNonBlocking) != cudaSuccess) return false;
  cudaGraph_t graph = nullptr;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return false;
  cudaGraphConditionalHandle cond, cgrow, cmerge;
  bool ok = cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  if (grow) {
    ok = ok && cudaGraphConditionalHandleCreate(&cgrow, graph, 0, cudaGraphCondAssignDefault) == cudaSuccess &&
         cudaGraphConditionalHandleCreate(&cmerge, graph, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  }
  const uint64_t l0 = launch_count();
  ok = ok && cudaStreamBeginCaptureToGraph(gc.cap, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                 cudaSuccess;
  if (!ok) {
    cudaGraphDestroy(graph);
    return false;
  }
  const Geo &g = h->geo;
  auto merges = [&](cudaStream_t t) {
    launch_esc_top(g, h->ctl, h->w, nb, t);
    launch_segments(g, h->ctl, h->w, nb, t);
    launch_segment_merge(g, g, h->ctl, h->w, h->scratch_cap, g.nleaves, h->scratch, h->vbuf, h->partials, false,
                         t);
    if (h->mhead) launch_train_model(g, h->mhead, h->mpieces, h->ctl, true, t);
  };
  if (learned_front(f.prep, h->mhead != nullptr, nb)) {  // sorted by bucketing on the model's pieces
    launch_lfront_sort(f, h->w.lbkt, h->w.lrank, h->w.lcnt, nb, gc.cap);
    launch_front_search(f, nb, gc.cap, h->w.lbkt);
  } else if (!small_front(nb)) {
    launch_front(f, nb, gc.cap);
  }
  // (an IF node around the general pass, which a sliding window rarely needs,
  // measured slower than its three kernels returning at once)
  launch_leaf_pass(g, h->ctl, h->w, nb, gc.cap);
  note_launch();
  k_gate<<<1, 1, 0, gc.cap>>>(h->ctl, cond);
  ok = ok && capture_if(gc.cap, gc.cap2, cond, [&](cudaStream_t t) {
    launch_pending(g, h->ctl, h->w, nb, t);
    launch_tree_rebuild(g, h->ctl, h->w, nb, t);
    launch_esc_level(g, h->ctl, h->w, nb, grow, t);
    if (!grow) merges(t);
  });
  if (ok && grow) {
    note_launch();
    k_gate_grow<<<1, 1, 0, gc.cap>>>(h->ctl, cgrow, cmerge);
    ok = capture_if(gc.cap, gc.cap2, cgrow, [&](cudaStream_t t) {
      const Geo &g2 = h->spare;
      launch_unmark(g, h->ctl, h->w, nb, t);
      launch_segment_merge(g, g2, h->ctl, h->w, h->scratch_cap, g.nleaves, h->scratch, h->vbuf, h->partials,
                           true, t);
      if (h->mhead) launch_train_model(g2, h->mhead, h->mpieces, h->ctl, false, t);
    });
    ok = ok && capture_if(gc.cap, gc.cap2, cmerge, merges);
  }
  if (stats) launch_stats(g, h->ctl, h->w, nb, gc.cap);
  note_launch();
  k_finish<<<1, 1, 0, gc.cap>>>(h->ctl);
  cudaGraph_t done = nullptr;
  const bool ended = cudaStreamEndCapture(gc.cap, &done) == cudaSuccess;
  const uint64_t kernels = launch_count() - l0;
  unnote_launches(kernels);
  if (!ok || !ended) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return false;
  }
  GraphCache::Entry *ge = gc.victim();
  const cudaError_t ie = cudaGraphInstantiate(&ge->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    ge->exec = nullptr;
    return false;
  }
  ge->bucket = 0;
  ge->epoch = h->alloc_epoch;
  ge->stats = stats;
  ge->kernels = kernels;  // an upper bound: the IF bodies run only when needed
  ge->used = ++gc.tick;
  *out = ge;
  return true;
}

// The spare array of height h+1 that a batch captured with `grow` resizes into.
int ensure_spare(gpma *h, cudaStream_t s) {
  if (h->has_spare && h->spare.h == h->geo.h + 1) return GPMA_OK;
  if (h->has_spare) free_arrays(h, &h->spare, s);
  h->has_spare = false;
  make_geo(h, h->geo.h + 1, &h->spare);
  h->spare.row_end = h->geo.row_end;
  h->spare.deg = h->geo.deg;
  if (!alloc_arrays(h, &h->spare, s)) {
    free_arrays(h, &h->spare, s);
    return GPMA_ENOMEM;
  }
  h->has_spare = true;
  h->alloc_epoch++;
  h->spare_epochs++;
  return GPMA_OK;
}

// A batch that may have grown the array on the device left its control block
// on its way to the host; before anything else uses the geometry, wait for it
// and, if the array grew, switch to the spare.
int settle(gpma *h, cudaStream_t s) {
  if (!h->mirror_pending) return GPMA_OK;
  h->mirror_pending = false;
  if (cudaEventSynchronize(h->ev_mirror) != cudaSuccess) return poison(h, GPMA_EDEVICE);
  const Ctl &c = *h->h_mirror;
  if (c.resized) {
    free_arrays(h, &h->geo, s);
    h->geo = h->spare;
    memset(&h->spare, 0, sizeof(Geo));
    h->has_spare = false;
    h->alloc_epoch++;
    h->since_train = 0;
  }
  h->count_ub = h->count_lb = c.total;
  return cuda_ok(h);
}

// Front-end arguments of a batch: sizes and the compressed key's bits and passes
PrepArgs make_prep(const gpma *h, uint64_t n_ins, uint64_t n_del, bool allow_guards) {
  PrepArgs pa;
  memset(&pa, 0, sizeof(pa));
  pa.n_ins = (uint32_t)n_ins;
  pa.n_del = (uint32_t)n_del;
  pa.V = h->V;
  pa.raw = h->raw;
  pa.allow_guards = allow_guards ? 1 : 0;
  uint32_t bits;  // sorted bits of the compressed key (the tag is not sorted on)
  if (h->raw) {
    bits = 63;
  } else {
    uint32_t sb = bits_for(h->V - 1);
    if (sb < 1) sb = 1;
    pa.db = allow_guards ? bits_for(h->V) : (bits_for(h->V - 1) ? bits_for(h->V - 1) : 1);
    bits = sb + pa.db;
  }
  pa.npass = (bits + 7) / 8;
  pa.dbits = (bits + pa.npass - 1) / pa.npass;
  pa.sbits = bits;
  return pa;
}

int update(gpma *h, const uint64_t *ins, uint64_t n_ins, const uint64_t *del, uint64_t n_del, cudaStream_t s,
           gpma_stats *stats, bool allow_guards) {
  if (h->poisoned) return h->poisoned;
  if (stats) memset(stats, 0, sizeof(*stats));
  const uint64_t n = n_ins + n_del;
  if (n >= (1ull << 30) || (n_ins && !ins) || (n_del && !del)) return GPMA_EINVAL;
  if (n == 0) return GPMA_OK;
  int rc = settle(h, s);
  if (rc) return rc;
  rc = ensure_work(h, n, s);
  if (rc) return rc;
  if ((rc = ensure_merge_scratch(h, s))) return rc;
  const uint32_t h_old = h->geo.h;
  const uint64_t C_old = h->geo.C;

  const PrepArgs pa = make_prep(h, n_ins, n_del, allow_guards);

  FrontArgs f;
  f.prep = pa;
  f.mhead = h->mhead;
  f.mpieces = h->mpieces;
  f.ins = ins;
  f.del = del;
  f.bufA = h->bufA;
  f.bufB = h->bufB;
  f.hist = h->hist;
  f.status = h->w.status;
  f.ctl = h->ctl;
  f.geo = &h->geo;
  f.ukey = h->w.ukey;
  f.utag = h->w.utag;
  f.uleaf = h->w.uleaf;
  f.run_start = h->w.run_start;
  f.run_leaf = h->w.rleaf;
  f.lfull = h->w.pleaf;  // free until the escalation compacts pending inserts
  f.rs = h->w.rs;
  const uint32_t n32 = (uint32_t)n;
  Phase whole(h->prof, GPMA_PROF_UPDATE, s);
  // level-0 merges move pivots only inside their leaves and the search widens
  // its window when the model has drifted; retrain now and then all the same
  if (h->mhead && ++h->since_train >= 64) train_model(h, s);
  // one batch-size bucket (a power of two) sizes the front end's grids and tiles,
  // in a replayed graph and in directly launched kernels alike
  uint64_t nb_front = kSmallBatch;
  while (nb_front < n) nb_front <<= 1;
  // the root can only refuse inserts when the count might exceed its bound
  const bool may_fail = h->count_ub + n_ins > h->geo.maxc[h->geo.h];
  // such a batch still replays a graph (no host wait) when one level of growth
  // surely suffices: it resizes on the device into a preallocated spare array
  bool grow = false;
  if (may_fail && !stats && h->graphs->enabled && h->ev_mirror && h->geo.h + 2 < kMaxLv &&
      ((uint64_t)h->L << (h->geo.h + 1)) <= (1ull << 32)) {
    uint64_t mx[kMaxLv];
    level_bounds(h->L, h->geo.h + 1, h->tau0, h->tauh, mx);
    grow = h->count_ub + n_ins <= mx[h->geo.h + 1] && ensure_spare(h, s) == GPMA_OK;
  }
  const bool replay = (!may_fail || grow) && h->graphs->enabled;
  // the model-bucketed sort for every batch that cannot need more than one doubling
  // (replayed, or launched directly when graphs are off); a bulk load keeps the radix
  // passes (a model trained on a nearly empty array gives very uneven buckets)
  const bool by_model = (!may_fail || grow) && learned_front(pa, h->mhead != nullptr, n);
  if (small_front(n)) launch_small_front(f, s);
  else if (by_model) launch_lprep(f, h->w.lbkt, h->w.lrank, h->w.lcnt, nb_front, s);  // buckets by model piece
  else launch_prep(f, nb_front, s);
  bool resized = false;
  if (replay) {
    // replay: sort .. segment merge as one graph, grids sized for the bucket
    const uint64_t bucket = nb_front;  // one graph serves every batch of the fused front end
    const uint32_t nb = (uint32_t)bucket;
    // the key layout of a guard batch differs: never share its graph
    const uint64_t key = h->alloc_epoch + (allow_guards ? (1ull << 62) : 0) + (grow ? (1ull << 61) : 0);
    GraphCache::Entry *ge = h->graphs->find(bucket, key, stats != nullptr);
    if (!ge) {
      if (!capture_update(h, f, nb, stats != nullptr, grow, &ge)) return poison(h, GPMA_EDEVICE);
      ge->bucket = bucket;
      ge->epoch = key;
    }
    if (cudaGraphLaunch(ge->exec, s) != cudaSuccess) return poison(h, GPMA_EDEVICE);
    for (uint64_t k = 0; k < ge->kernels; k++) note_launch();
    h->count_ub += n_ins;
    if (grow) {
      cudaMemcpyAsync(h->h_mirror, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
      if (cudaEventRecord(h->ev_mirror, s) != cudaSuccess) return poison(h, GPMA_EDEVICE);
      h->mirror_pending = true;
    }
  } else {
    {
      Phase ph(h->prof, GPMA_PROF_SORT, s);
      if (by_model) {
        launch_lfront_sort(f, h->w.lbkt, h->w.lrank, h->w.lcnt, nb_front, s);
        launch_front_search(f, nb_front, s, h->w.lbkt);
      } else if (!small_front(n)) {
        launch_front(f, nb_front, s);
      }
    }
    {
      Phase ph(h->prof, GPMA_PROF_LEAF, s);
      launch_leaf_pass(h->geo, h->ctl, h->w, n32, s);
    }
    Phase esc(h->prof, GPMA_PROF_ESCALATE, s);
    launch_pending(h->geo, h->ctl, h->w, n32, s);
    launch_tree_rebuild(h->geo, h->ctl, h->w, n32, s);
    launch_esc_level(h->geo, h->ctl, h->w, n32, may_fail, s);
    if ((rc = cuda_ok(h))) return rc;
    if (may_fail) {
      if ((rc = read_ctl(h, s))) return rc;
      if (h->h_ctl->err) {
        note_launch();
        k_finish<<<1, 1, 0, s>>>(h->ctl);
        int st = err_to_status(h->h_ctl->err);
        if (st != GPMA_EINVAL) poison(h, st);
        return st;
      }
      h->count_ub = h->count_lb = h->h_ctl->total;
      if (h->h_ctl->nfail) {
        esc.end();
        Phase ph(h->prof, GPMA_PROF_RESIZE, s);
        launch_unmark(h->geo, h->ctl, h->w, n32, s);
        if ((rc = do_resize(h, h->h_ctl->total, s))) return rc;
        resized = true;
        if (stats) launch_stats(h->geo, h->ctl, h->w, n32, s);  // touched leaves with a delete
      }
    } else {
      h->count_ub += n_ins;
    }
    if (!resized) {
      launch_esc_top(h->geo, h->ctl, h->w, n32, s);
      launch_segments(h->geo, h->ctl, h->w, n32, s);
      launch_segment_merge(h->geo, h->geo, h->ctl, h->w, h->scratch_cap, h->geo.nleaves, h->scratch, h->vbuf,
                           h->partials, false, s);
      esc.end();
      if (stats) launch_stats(h->geo, h->ctl, h->w, n32, s);
      train_model(h, s, true);
    }
    note_launch();
    k_finish<<<1, 1, 0, s>>>(h->ctl);
  }
  whole.end();
  if ((rc = cuda_ok(h))) return rc;
  bool shrunk = false;
  if (h->dual && !resized) {
    // deletes can only lower the count: look only when the root might be underfull
    h->count_lb = h->count_lb > n_del ? h->count_lb - n_del : 0;
    if (h->count_lb < h->geo.minc[h->geo.h]) {
      if ((rc = settle(h, s)) || (rc = read_ctl(h, s))) return rc;
      if (h->h_ctl->err == 0) {
        h->count_ub = h->count_lb = h->h_ctl->total;
        Phase ph(h->prof, GPMA_PROF_RESIZE, s);
        if ((rc = maybe_shrink(h, h->h_ctl->total, s, &shrunk))) return rc;
      }
    }
  }
  if (!stats) return GPMA_OK;

  if ((rc = read_ctl(h, s))) return rc;
  const Ctl &c = *h->h_ctl;
  int st = err_to_status(c.err);
  if (st) {
    if (st != GPMA_EINVAL) poison(h, st);
    return st;
  }
  h->count_ub = h->count_lb = c.total;
  const uint64_t L = h->L;
  stats->n_inserted = c.n_inserted;
  stats->n_deleted = c.n_deleted;
  stats->n_ignored = n - c.n_inserted - c.n_deleted;
  stats->touched_leaves = c.nruns;
  stats->delete_leaves = c.st_del_leaves;
  stats->model_sorted = by_model ? 1u : 0u;
  stats->resized = resized ? 1 : (shrunk ? 2 : 0);
  for (int i = 0; i < GPMA_MAX_LEVELS && i < kMaxLv; i++) stats->merges[i] = c.merges[i];
  stats->merges[0] = c.n_merged0;
  uint32_t climbed = c.levels_climbed;
  if (resized) climbed = h_old + 1;
  stats->levels_climbed = climbed;
  if (resized || shrunk) {
    stats->covered_leaves = 0;
    stats->alg_bytes = 8 * n + 8 * L * c.nruns + 8 * C_old + 8 * h->geo.C;
  } else {
    const uint64_t cov = (uint64_t)c.nleafw + c.st_l0_only;
    stats->covered_leaves = cov;
    stats->alg_bytes = 8 * n + 8 * L * c.nruns + 8 * L * cov + 8 * L * (cov - c.st_cov_touched) + 8 * c.st_empties;
  }
  return GPMA_OK;
}

int ensure_analytics(gpma *h, uint32_t iters, cudaStream_t s) {
  if (!h->y) {
    if (!dalloc(h, &h->y, h->V, s) || !dalloc(h, &h->cfx, h->V, s) ||
        !dalloc(h, &h->q0, h->V, s) || !dalloc(h, &h->q1, h->V, s) || !dalloc(h, &h->q2, 2ull * h->V, s) || !dalloc(h, &h->counter, 32, s) ||
        !dalloc(h, &h->pr_partials, 152 * 16, s) || !dalloc(h, &h->pr_counter, 4, s))
      return GPMA_ENOMEM;
  }
  if (iters + 1 > h->dsum_cap) {
    dfree(h, h->dsum, s);
    h->dsum_cap = iters + 1 < 64 ? 64 : iters + 1;
    if (!dalloc(h, &h->dsum, h->dsum_cap, s)) {
      h->dsum_cap = 0;
      return GPMA_ENOMEM;
    }
  }
  return GPMA_OK;
}

// Buffers of the bucketed PageRank pass; false (nothing changed that matters)
// when the heads do not fit its bucket table or memory is short: the caller then
// takes the push pass.
bool ensure_pb(gpma *h, const PbPlan &p, cudaStream_t s) {
  if (h->push_pr || p.nb > kPbMaxBuckets) return false;
  if (!h->pb_cnt) {
    const uint64_t n = (uint64_t)p.nb * kPbMaxChunks;
    if (!dalloc(h, &h->pb_cnt, n, s) || !dalloc(h, &h->pb_off, n + 1, s) ||
        !dalloc(h, &h->pb_scan, (uint64_t)kPbMaxBuckets / 2 + 16, s) ||  // bucket totals (u32)
        !dalloc(h, &h->pb_dang, (uint64_t)p.nparts * p.nb, s)) {
      dfree(h, h->pb_cnt, s);
      dfree(h, h->pb_off, s);
      dfree(h, h->pb_scan, s);
      dfree(h, h->pb_dang, s);
      h->pb_cnt = nullptr;
      h->pb_off = h->pb_scan = h->pb_dang = nullptr;
      return false;
    }
  }
  if (h->pb_keys_cap < h->geo.C) {
    dfree(h, h->pb_keys, s);
    h->pb_keys_cap = 0;
    if (!dalloc(h, &h->pb_keys, h->geo.C, s)) {
      h->pb_keys = nullptr;
      return false;
    }
    h->pb_keys_cap = h->geo.C;
  }
  return true;
}

// The PageRank snapshot: the stored edges bucketed by head and, with `own_deg`,
// a copy of the out-degrees as they are now (bucketed pass only; *bucketed = false
// when the handle sums by the push pass, which reads the array itself).
int pr_snapshot(gpma *h, cudaStream_t s, bool own_deg, bool *bucketed) {
  *bucketed = false;
  const PbPlan plan = pb_plan(h->geo);
  if (!ensure_pb(h, plan, s)) return GPMA_OK;
  if (own_deg && !h->pb_deg && !dalloc(h, &h->pb_deg, h->V, s)) return GPMA_ENOMEM;
  {
    Phase ph(h->prof, GPMA_PROF_PR_BUCKET, s);
    launch_pb_build(h->geo, plan, h->pb_cnt, h->pb_off, h->pb_scan, h->pb_keys, s);
    if (own_deg) cudaMemcpyAsync(h->pb_deg, h->geo.deg, sizeof(uint32_t) * h->V, cudaMemcpyDeviceToDevice, s);
  }
  h->snap_plan = plan;
  h->snap_valid = own_deg;  // only a snapshot with its own degrees outlives the call
  *bucketed = true;
  return cuda_ok(h);
}

// iterations over the bucketed copy (with `own_deg`, over the snapshot alone: the
// live array may change meanwhile)
int pr_run(gpma *h, uint32_t iters, float damping, float *d_rank, bool own_deg, cudaStream_t s) {
  Geo gs = h->geo;
  if (own_deg) gs.deg = h->pb_deg;
  // bucketed: the two halves of cfx hold the FP32 contributions of alternate iterations
  float *cf[2] = {reinterpret_cast<float *>(h->cfx), reinterpret_cast<float *>(h->cfx) + h->V};
  launch_pr_setup(gs, iters, d_rank, h->y, h->cfx, cf[0], h->dsum, h->pr_partials, h->pr_counter, s);
  for (uint32_t it = 0; it < iters; it++) {
    Phase ph(h->prof, GPMA_PROF_PR_SCATTER, s);
    launch_pb_iter(gs, h->snap_plan, h->pb_keys, h->pb_off, damping, cf[it & 1], cf[(it + 1) & 1], d_rank,
                   it + 1 == iters, h->dsum + it, h->dsum + it + 1, h->pb_dang, h->pr_counter, s);
  }
  return cuda_ok(h);
}

// ---- batched update of many handles (gpma_update_many) -----------------------------------------
__global__ void k_m_gate(const ManyDesc *d, const cudaGraphConditionalHandle *cond) {
  const uint32_t k = threadIdx.x;
  if (k >= d->count) return;
  const Ctl *ctl = d->item[k].ctl;
  cudaGraphSetConditional(cond[k], (d->item[k].active && ctl->err == 0 && ctl->nesc > 0) ? 1u : 0u);
}

__global__ void k_m_finish(const ManyDesc *d) {
  const uint32_t k = threadIdx.x;
  if (k < d->count && d->item[k].active) d->item[k].ctl->sticky |= d->item[k].ctl->err;
}

// Process-wide state of the batched update: the plan table on the device (read by
// every batched kernel), pinned staging copies of it, side streams, and captured
// graphs keyed by the handles they serve.
struct ManyCtx {
  static constexpr int kStage = 4, kGraphs = 4;
  std::mutex mu;
  ManyDesc *d_desc = nullptr;
  ManyDesc *h_desc[kStage] = {};
  cudaEvent_t up[kStage] = {};
  uint32_t next_stage = 0;
  cudaEvent_t done = nullptr, fork = nullptr, cfork = nullptr;
  std::vector<cudaStream_t> side, cside;  // lone batches; branches of a graph being captured
  std::vector<cudaEvent_t> join, cjoin;
  cudaStream_t cap = nullptr, cap2 = nullptr;
  struct Graph {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle *d_cond = nullptr;
    uint64_t kernels = 0, used = 0;
  } graphs[kGraphs];
  uint64_t tick = 0;
  bool graphs_on = true;

  bool init() {
    if (d_desc) return true;
    const char *ng = getenv("GPMA_NO_GRAPHS");
    graphs_on = !(ng && ng[0] == '1');
    prepare_many_front();
    prepare_many_leaf();
    allow_big_smem();
    if (cudaMalloc(&d_desc, sizeof(ManyDesc)) != cudaSuccess) return false;
    for (int i = 0; i < kStage; i++)
      if (cudaMallocHost(&h_desc[i], sizeof(ManyDesc)) != cudaSuccess ||
          cudaEventCreateWithFlags(&up[i], cudaEventDisableTiming) != cudaSuccess)
        return false;
    return cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&cfork, cudaEventDisableTiming) == cudaSuccess &&
           cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess &&
           cudaStreamCreateWithFlags(&cap2, cudaStreamNonBlocking) == cudaSuccess;
  }
  static bool grow(std::vector<cudaStream_t> &ss, std::vector<cudaEvent_t> &es, uint32_t n) {
    while (ss.size() < n) {
      cudaStream_t t = nullptr;
      cudaEvent_t e = nullptr;
      if (cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
        return false;
      ss.push_back(t);
      es.push_back(e);
    }
    return true;
  }
  bool ensure_streams(uint32_t n) { return init() && grow(side, join, n); }
  bool ensure_branches(uint32_t n) { return init() && grow(cside, cjoin, n); }
};

ManyCtx &many_ctx() {
  static ManyCtx *c = new ManyCtx;  // lives until the process exits
  return *c;
}

// Blocks of one batched launch: a grid of G blocks (fixed when the graph is
// captured) shared among the handles with work, each getting at least one block
// and otherwise in proportion to its work, never more than cap[k].
uint32_t add_plan(ManyDesc &D, ManyPlans &pl, uint32_t &nplans, uint32_t G, const std::vector<uint64_t> &work,
                  const std::vector<uint32_t> &cap) {
  const uint32_t id = nplans++;
  ManyPlan &p = D.plan[id];
  uint64_t tot = 0;
  uint32_t nw = 0;
  for (size_t k = 0; k < work.size(); k++)
    if (work[k]) {
      tot += work[k];
      nw++;
    }
  p.n = 0;
  uint32_t start = 0;
  for (size_t k = 0; k < work.size(); k++) {
    if (!work[k]) continue;
    uint64_t b = 1 + (uint64_t)(G - nw) * work[k] / tot;
    if (b > cap[k]) b = cap[k];
    if (b < 1) b = 1;
    p.item[p.n] = (uint32_t)k;
    p.start[p.n] = start;
    start += (uint32_t)b;
    p.n++;
  }
  p.start[p.n] = start;
  pl.total[id] = G;
  return id;
}

uint32_t ceil_div(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

// One handle's merge levels (the IF-node body of its branch): the same launches as
// gpma_update_batch's escalation, grids sized for the handle's work capacity.
void many_escalation(gpma *h, cudaStream_t t) {
  const Geo &g = h->geo;
  const uint32_t nb = h->cap;
  launch_pending(g, h->ctl, h->w, nb, t);
  launch_tree_rebuild(g, h->ctl, h->w, nb, t);
  launch_esc_level(g, h->ctl, h->w, nb, false, t);
  launch_esc_top(g, h->ctl, h->w, nb, t);
  launch_segments(g, h->ctl, h->w, nb, t);
  launch_segment_merge(g, g, h->ctl, h->w, h->scratch_cap, g.nleaves, h->scratch, h->vbuf, h->partials, false, t);
  if (h->mhead) launch_train_model(g, h->mhead, h->mpieces, h->ctl, true, t);
}

bool capture_many(ManyCtx &mc, const std::vector<gpma *> &hs, const ManyPlans &pl, ManyCtx::Graph *ge) {
  const uint32_t nb = (uint32_t)hs.size();
  if (!mc.ensure_branches(nb)) return false;
  cudaGraph_t graph = nullptr;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return false;
  std::vector<cudaGraphConditionalHandle> cond(nb);
  bool ok = true;
  for (uint32_t k = 0; k < nb && ok; k++)
    ok = cudaGraphConditionalHandleCreate(&cond[k], graph, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok && !ge->d_cond) ok = cudaMalloc(&ge->d_cond, sizeof(cudaGraphConditionalHandle) * kMaxMany) == cudaSuccess;
  ok = ok && cudaMemcpy(ge->d_cond, cond.data(), sizeof(cudaGraphConditionalHandle) * nb, cudaMemcpyHostToDevice) ==
                 cudaSuccess;
  const uint64_t l0 = launch_count();
  ok = ok && cudaStreamBeginCaptureToGraph(mc.cap, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                 cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return false;
  }
  launch_many_front(mc.d_desc, pl, mc.cap);
  launch_many_leaf(mc.d_desc, pl, mc.cap);
  note_launch();
  k_m_gate<<<1, nb, 0, mc.cap>>>(mc.d_desc, ge->d_cond);
  // one branch per handle, its merge levels behind its own IF node
  ok = cudaEventRecord(mc.cfork, mc.cap) == cudaSuccess;
  for (uint32_t k = 0; k < nb && ok; k++) {
    ok = cudaStreamWaitEvent(mc.cside[k], mc.cfork, 0) == cudaSuccess &&
         capture_if(mc.cside[k], mc.cap2, cond[k], [&](cudaStream_t t) { many_escalation(hs[k], t); }) &&
         cudaEventRecord(mc.cjoin[k], mc.cside[k]) == cudaSuccess &&
         cudaStreamWaitEvent(mc.cap, mc.cjoin[k], 0) == cudaSuccess;
  }
  note_launch();
  k_m_finish<<<1, nb, 0, mc.cap>>>(mc.d_desc);
  cudaGraph_t done = nullptr;
  const bool ended = cudaStreamEndCapture(mc.cap, &done) == cudaSuccess;
  const uint64_t kernels = launch_count() - l0;
  unnote_launches(kernels);
  if (!ok || !ended) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return false;
  }
  const cudaError_t ie = cudaGraphInstantiate(&ge->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    ge->exec = nullptr;
    return false;
  }
  ge->kernels = kernels;
  return true;
}

// The handles `sel` of a call as one batched graph; act[k]: sel[k] is updated by this
// call (the others keep their place in the graph, which is then reused as long as
// the same handles come back, and are left alone by every kernel).
int run_many(ManyCtx &mc, gpma_t const *handles, const uint64_t *const *d_ins, const uint64_t *n_ins,
             const uint64_t *const *d_del, const uint64_t *n_del, const std::vector<uint32_t> &sel,
             const std::vector<uint8_t> &act, cudaStream_t s) {
  if (!mc.init()) return GPMA_EDEVICE;
  const uint32_t nb = (uint32_t)sel.size();
  std::vector<gpma *> hs(nb);
  for (uint32_t k = 0; k < nb; k++) hs[k] = handles[sel[k]];
  // level-0 merges move pivots only inside their leaves; retrain now and then all the same
  for (uint32_t k = 0; k < nb; k++)
    if (act[k] && hs[k]->mhead && ++hs[k]->since_train >= 64) train_model(hs[k], s);
  // the staging copy this call fills (waits only when every copy is still in flight)
  const uint32_t st = mc.next_stage;
  mc.next_stage = (st + 1) % ManyCtx::kStage;
  if (cudaEventSynchronize(mc.up[st]) != cudaSuccess) return GPMA_EDEVICE;
  ManyDesc &D = *mc.h_desc[st];
  D.count = nb;
  std::vector<uint64_t> n(nb), wt(nb), wr(nb), w1(nb), w4(nb), w64(nb), wdeg(nb);
  std::vector<uint32_t> ct(nb), cr(nb), c1(nb), c4(nb), c64(nb), cdeg(nb), one(nb, 1);
  uint32_t maxpass = 0;
  for (uint32_t k = 0; k < nb; k++) {
    gpma *h = hs[k];
    const uint32_t i = sel[k];
    ManyItem &it = D.item[k];
    it.active = act[k];
    n[k] = act[k] ? n_ins[i] + n_del[i] : 0;
    it.prep = make_prep(h, act[k] ? n_ins[i] : 0, act[k] ? n_del[i] : 0, false);
    it.ins = d_ins ? d_ins[i] : nullptr;
    it.del = d_del ? d_del[i] : nullptr;
    it.bufA = h->bufA;
    it.bufB = h->bufB;
    it.hist = h->hist;
    it.ctl = h->ctl;
    it.mhead = h->mhead;
    it.mpieces = h->mpieces;
    it.small = small_front(n[k]) ? 1u : 0u;
    it.T = front_tiles(n[k]);
    it.wide = search_wide(n[k]) ? 1u : 0u;
    it.T1 = search_tiles(n[k]);
    it.P = 64;
    while (it.P < n[k]) it.P <<= 1;
    it.S = h->geo.nleaves < 2048 ? (uint32_t)h->geo.nleaves : 2048u;
    it.per_warp = leaf_smem_bytes(h->L);
    it.g = h->geo;
    it.w = h->w;
    if (it.prep.npass > maxpass) maxpass = it.prep.npass;
    const uint32_t radix = 1u << it.prep.dbits;
    wt[k] = it.small ? 0 : it.T;
    ct[k] = it.T;
    wr[k] = it.small ? 0 : (uint64_t)radix * it.T;
    cr[k] = radix;
    w1[k] = (!it.small && !it.wide) ? it.T1 : 0;
    c1[k] = it.T1;
    w4[k] = (!it.small && it.wide) ? it.T1 : 0;
    c4[k] = it.T1;
    w64[k] = h->L == 64 ? n[k] : 0;
    c64[k] = ceil_div(n[k], 8);
    wdeg[k] = h->raw ? 0 : n[k];
    cdeg[k] = ceil_div(n[k], 256);
  }
  // plans: the grid of every launch depends only on the set of handles
  ManyPlans pl;
  memset(&pl, 0, sizeof(pl));
  uint32_t np = 0;
  pl.one = add_plan(D, pl, np, nb, std::vector<uint64_t>(nb, 1), one);  // every handle: kernels test `active`
  pl.tiles = add_plan(D, pl, np, 1216 + nb, wt, ct);
  pl.radix = add_plan(D, pl, np, 2432 + nb, wr, cr);
  pl.search[0] = add_plan(D, pl, np, 2432 + nb, w1, c1);
  pl.search[1] = add_plan(D, pl, np, 1216 + nb, w4, c4);
  pl.leaf64 = add_plan(D, pl, np, 608 + nb, w64, c64);
  pl.deg = add_plan(D, pl, np, 1216 + nb, wdeg, cdeg);
  pl.maxpass = maxpass;
  // the one-warp-per-leaf pass: one launch per block size (warps per block, 1..8);
  // a block's warps use its own handle's shared-memory stride, and the launch
  // reserves the group's largest
  std::vector<uint64_t> key;
  key.reserve(4 * nb + 2);
  key.push_back(nb);
  for (uint32_t k = 0; k < nb; k++) {
    gpma *h = hs[k];
    const uint32_t wpb = leaf_pass_warps(h->L, h->leaf_warps);
    uint32_t gi = 0;
    while (gi < pl.ngroups && pl.group[gi].wpb != wpb) gi++;
    if (gi == pl.ngroups) {
      pl.group[gi].wpb = wpb;
      pl.group[gi].per_warp = 0;
      pl.ngroups++;
    }
    if (leaf_smem_bytes(h->L) > pl.group[gi].per_warp) pl.group[gi].per_warp = leaf_smem_bytes(h->L);
    key.push_back(h->uid);
    key.push_back(h->alloc_epoch - h->spare_epochs);  // a batched graph never uses the spare array
    key.push_back(((uint64_t)gi << 32) | ((uint64_t)(h->cap > kLongRun) << 16) | (h->mhead ? 1u : 0u));
  }
  for (uint32_t gi = 0; gi < pl.ngroups; gi++) {
    ManyPlans::Group &gr = pl.group[gi];
    std::vector<uint64_t> wrest(nb, 0), wla(nb, 0), wlb(nb, 0);
    std::vector<uint32_t> crest(nb), cla(nb), clb(nb);
    bool any_long = false;
    for (uint32_t k = 0; k < nb; k++) {
      gpma *h = hs[k];
      if (leaf_pass_warps(h->L, h->leaf_warps) != gr.wpb) continue;
      wrest[k] = n[k];
      crest[k] = ceil_div(n[k], gr.wpb);
      any_long |= h->cap > kLongRun;
      if (n[k] > kLongRun) {
        wla[k] = wlb[k] = n[k];
        cla[k] = ceil_div(ceil_div(n[k], 32), gr.wpb);
        clb[k] = ceil_div(n[k] / kLongRun + 1, gr.wpb);
      }
    }
    gr.rest = add_plan(D, pl, np, 2432 + nb, wrest, crest);
    gr.long_a = gr.long_b = ~0u;
    if (any_long) {
      gr.long_a = add_plan(D, pl, np, 2432 + nb, wla, cla);
      gr.long_b = add_plan(D, pl, np, 2432 + nb, wlb, clb);
    }
  }
  // upload after the previous batched call has finished reading the table
  const size_t bytes = offsetof(ManyDesc, item) + sizeof(ManyItem) * nb;
  if (cudaStreamWaitEvent(s, mc.done, 0) != cudaSuccess ||
      cudaMemcpyAsync(mc.d_desc, &D, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaEventRecord(mc.up[st], s) != cudaSuccess)
    return GPMA_EDEVICE;
  if (mc.graphs_on) {
    ManyCtx::Graph *ge = nullptr;
    for (auto &g : mc.graphs)
      if (g.exec && g.key == key) ge = &g;
    if (!ge) {
      ge = &mc.graphs[0];
      for (auto &g : mc.graphs) {
        if (!g.exec) {
          ge = &g;
          break;
        }
        if (g.used < ge->used) ge = &g;
      }
      if (ge->exec) cudaGraphExecDestroy(ge->exec);
      ge->exec = nullptr;
      if (!capture_many(mc, hs, pl, ge)) return GPMA_EDEVICE;
      ge->key = key;
    }
    ge->used = ++mc.tick;
    if (cudaGraphLaunch(ge->exec, s) != cudaSuccess) return GPMA_EDEVICE;
    for (uint64_t k = 0; k < ge->kernels; k++) note_launch();
  } else {
    // direct launches (profilers see every kernel): every updated handle's merge
    // levels run and return at once when nothing is pending
    launch_many_front(mc.d_desc, pl, s);
    launch_many_leaf(mc.d_desc, pl, s);
    for (uint32_t k = 0; k < nb; k++)
      if (act[k]) many_escalation(hs[k], s);
    note_launch();
    k_m_finish<<<1, nb, 0, s>>>(mc.d_desc);
  }
  if (cudaEventRecord(mc.done, s) != cudaSuccess) return GPMA_EDEVICE;
  for (uint32_t k = 0; k < nb; k++)
    if (act[k]) hs[k]->count_ub += n_ins[sel[k]];
  return GPMA_OK;
}

}  // namespace

namespace gpk {
// Read-only view of a handle for entry points defined in other files.
HandleView handle_view(gpma_t h, cudaStream_t s) {
  HandleView v;
  if (!h->poisoned) settle(h, s);
  v.geo = &h->geo;
  v.ctl = h->ctl;
  v.h_ctl = h->h_ctl;
  v.poisoned = h->poisoned;
  return v;
}
int poison_handle(gpma_t h, int code) { return poison(h, code); }
int export_status(gpma_t h, uint32_t err) {
  const int st = err_to_status(err);
  return st ? poison(h, st) : GPMA_OK;
}
}  // namespace gpk

extern "C" {

const char *gpma_strerror(int status) {
  switch (status) {
    case GPMA_OK: return "ok";
    case GPMA_EINVAL: return "invalid argument or key (nothing applied)";
    case GPMA_ENOMEM: return "out of device memory";
    case GPMA_ECAP: return "output buffer too small";
    case GPMA_ETIMEOUT: return "a bounded device-side wait gave up (handle poisoned)";
    case GPMA_EDEVICE: return "CUDA runtime error (handle poisoned)";
    default: return "unknown status";
  }
}

int gpma_create(uint32_t n_vertices, const gpma_params *params, const gpma_allocator *alloc, void *stream,
                gpma_t *out) {
  if (!out) return GPMA_EINVAL;
  *out = nullptr;
  gpma_params p;
  memset(&p, 0, sizeof(p));
  if (params) p = *params;
  if (!p.leaf_size) p.leaf_size = 64;
  if (!p.tau0_pct) p.tau0_pct = 92;
  if (!p.tauh_pct) p.tauh_pct = 80;
  if (!p.rho0_pct) p.rho0_pct = 8;
  if (!p.rhoh_pct) p.rhoh_pct = 40;
  const uint32_t L = p.leaf_size;
  if (L < 2 || L > 1024 || (L & (L - 1))) return GPMA_EINVAL;
  if (p.leaf_warps != 0 && p.leaf_warps != 1 && p.leaf_warps != 2 && p.leaf_warps != 4 && p.leaf_warps != 8)
    return GPMA_EINVAL;
  if (!(p.tauh_pct <= p.tau0_pct && p.tau0_pct <= 100 && p.rho0_pct <= p.rhoh_pct && p.rhoh_pct < p.tauh_pct))
    return GPMA_EINVAL;
  const bool raw = (p.flags & GPMA_RAW_KEYS) != 0;
  if (!raw && (n_vertices == 0 || n_vertices > (1u << 31))) return GPMA_EINVAL;
  if (alloc && (!alloc->alloc || !alloc->free)) return GPMA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;

  gpma *h = new (std::nothrow) gpma;
  if (!h) return GPMA_ENOMEM;
  memset(h, 0, sizeof(gpma));
  h->prof = new (std::nothrow) Prof;
  h->graphs = new (std::nothrow) GraphCache;
  if (!h->prof || !h->graphs) {
    delete h->prof;
    delete h->graphs;
    delete h;
    return GPMA_ENOMEM;
  }
  allow_big_smem();
  // GPMA_NO_GRAPHS=1 launches every kernel of a batch directly (profilers then
  // see each launch; the results are the same)
  const char *ng = getenv("GPMA_NO_GRAPHS");
  if (ng && ng[0] == '1') h->graphs->enabled = false;
  h->V = raw ? 0 : n_vertices;
  h->L = L;
  h->leaf_warps = p.leaf_warps;
  static std::atomic<uint64_t> next_uid{1};
  h->uid = next_uid.fetch_add(1);
  h->logL = bits_for(L) - 1;
  h->raw = raw ? 1 : 0;
  h->dual = (p.flags & GPMA_DUAL_DELETE) ? 1 : 0;
  h->push_pr = (p.flags & GPMA_PUSH_PAGERANK) != 0;
  h->tau0 = p.tau0_pct;
  h->tauh = p.tauh_pct;
  h->rho0 = p.rho0_pct;
  h->rhoh = p.rhoh_pct;
  if (alloc) {
    h->alloc = *alloc;
    h->has_alloc = true;
  }
  make_geo(h, 0, &h->geo);
  bool ok = alloc_arrays(h, &h->geo, s) && dalloc(h, &h->ctl, 1, s) && dalloc(h, &h->hist, 16 * 256, s) &&
            dalloc(h, &h->check_buf, 4, s);
  if (ok && !(p.flags & GPMA_PLAIN_SEARCH)) {
    ok = dalloc(h, &h->mhead, 1, s) && dalloc(h, &h->mpieces, kModelPieces, s);
    if (ok) ok = cudaMemsetAsync(h->mhead, 0, sizeof(ModelHead), s) == cudaSuccess;
  }
  if (ok && !raw) ok = dalloc(h, &h->geo.row_end, h->V, s) && dalloc(h, &h->geo.deg, h->V, s);
  if (ok && !raw) ok = cudaMemsetAsync(h->geo.deg, 0, sizeof(uint32_t) * h->V, s) == cudaSuccess;
  if (ok) ok = cudaMallocHost(&h->h_ctl, sizeof(Ctl)) == cudaSuccess && cudaMallocHost(&h->h_counter, 16) == cudaSuccess;
  if (ok) ok = cudaMallocHost(&h->h_mirror, sizeof(Ctl)) == cudaSuccess;
  if (ok) ok = cudaEventCreateWithFlags(&h->ev_mirror, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    gpma_destroy(h);
    return GPMA_ENOMEM;
  }
  cudaMemsetAsync(h->geo.slots, 0xFF, sizeof(uint64_t) * h->geo.C, s);
  cudaMemsetAsync(h->geo.F, 0xFF, sizeof(uint64_t) * h->geo.nleaves, s);
  cudaMemsetAsync(h->geo.cnt, 0, sizeof(uint32_t) * h->geo.nleaves, s);
  cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), s);
  int rc = GPMA_OK;
  if (!raw) {
    if (!dalloc(h, &h->guards, h->V, s)) rc = GPMA_ENOMEM;
    if (!rc) {
      note_launch();
      note_launch();
      k_make_guards<<<(h->V + 255) / 256 < 4096 ? (h->V + 255) / 256 : 4096, 256, 0, s>>>(h->guards, h->V);
      gpma_stats st;
      rc = update(h, h->guards, h->V, nullptr, 0, s, &st, true);
      dfree(h, h->guards, s);
      h->guards = nullptr;
    }
  }
  if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = GPMA_EDEVICE;
  if (rc) {
    gpma_destroy(h);
    return rc;
  }
  *out = h;
  return GPMA_OK;
}

int gpma_destroy(gpma_t h) {
  if (!h) return GPMA_EINVAL;
  cudaStream_t s = 0;
  cudaDeviceSynchronize();
  free_arrays(h, &h->geo, s);
  if (h->has_spare) free_arrays(h, &h->spare, s);
  dfree(h, h->geo.row_end, s);
  dfree(h, h->geo.deg, s);
  free_work(h, s);
  void *ptrs[] = {h->mhead, h->mpieces, h->ctl, h->hist, h->scratch, h->vbuf, h->partials, h->cfx, h->y,
                  h->dsum, h->q0,  h->q1,  h->q2,    h->counter, h->check_buf, h->guards, h->pr_partials,
                  h->pr_counter, h->pb_cnt, h->pb_off, h->pb_scan, h->pb_keys, h->pb_dang, h->pb_deg};
  for (void *p : ptrs) dfree(h, p, s);
  cudaStreamSynchronize(s);
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  if (h->h_counter) cudaFreeHost(h->h_counter);
  if (h->h_mirror) cudaFreeHost(h->h_mirror);
  if (h->ev_mirror) cudaEventDestroy(h->ev_mirror);
  delete h->prof;
  delete h->graphs;
  cudaGetLastError();
  delete h;
  return GPMA_OK;
}

int gpma_update_batch(gpma_t h, const uint64_t *d_ins, uint64_t n_ins, const uint64_t *d_del, uint64_t n_del,
                      void *stream, gpma_stats *stats) {
  if (!h) return GPMA_EINVAL;
  return update(h, d_ins, n_ins, d_del, n_del, (cudaStream_t)stream, stats, false);
}

int gpma_status(gpma_t h, void *stream) {
  if (!h) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = read_ctl(h, s);
  if (rc) return rc;
  uint32_t sticky = h->h_ctl->sticky;
  cudaMemsetAsync(&h->ctl->sticky, 0, sizeof(uint32_t), s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return poison(h, GPMA_EDEVICE);
  int st = err_to_status(sticky);
  if (st != GPMA_OK && st != GPMA_EINVAL) poison(h, st);
  return st;
}

int gpma_bfs(gpma_t h, uint32_t src, int32_t *d_depth, void *stream) {
  if (!h || !d_depth || h->raw || src >= h->V) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  cudaStream_t s = (cudaStream_t)stream;
  if (ensure_analytics(h, 1, s)) return GPMA_ENOMEM;
  Phase ph(h->prof, GPMA_PROF_BFS, s);
  if (run_bfs(h->geo, src, d_depth, h->q0, h->q1, h->q2, h->counter, h->ctl, s) < 0) return poison(h, GPMA_EDEVICE);
  return cuda_ok(h);
}

int gpma_cc(gpma_t h, uint32_t *d_label, void *stream) {
  if (!h || !d_label || h->raw) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  Phase ph(h->prof, GPMA_PROF_CC, (cudaStream_t)stream);
  launch_cc(h->geo, d_label, (cudaStream_t)stream);
  return cuda_ok(h);
}

int gpma_pagerank(gpma_t h, uint32_t iters, float damping, float *d_rank, void *stream) {
  if (!h || !d_rank || h->raw || !(damping >= 0.0f && damping <= 1.0f)) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  cudaStream_t s = (cudaStream_t)stream;
  if (ensure_analytics(h, iters, s)) return GPMA_ENOMEM;
  Phase all(h->prof, GPMA_PROF_PAGERANK, s);
  bool bucketed = false;
  if (iters > 0) {
    const int rc = pr_snapshot(h, s, false, &bucketed);
    if (rc) return rc;
  }
  if (bucketed) return pr_run(h, iters, damping, d_rank, false, s);
  // push pass: every iteration reads the array itself
  launch_pr_setup(h->geo, iters, d_rank, h->y, h->cfx, nullptr, h->dsum, h->pr_partials, h->pr_counter, s);
  for (uint32_t it = 0; it < iters; it++) {
    Phase ph(h->prof, GPMA_PROF_PR_SCATTER, s);
    launch_pr_scatter(h->geo, h->cfx, h->y, s);
    ph.end();
    launch_pr_apply(h->geo, damping, d_rank, h->y, h->cfx, h->dsum + it, h->dsum + it + 1, h->pr_partials,
                    h->pr_counter, it + 1 == iters, s);
  }
  all.end();
  return cuda_ok(h);
}

int gpma_pagerank_snapshot(gpma_t h, void *stream) {
  if (!h || h->raw) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  bool bucketed = false;
  const int rc = pr_snapshot(h, (cudaStream_t)stream, true, &bucketed);
  if (rc) return rc;
  return bucketed ? GPMA_OK : GPMA_EINVAL;  // the push pass reads the array itself
}

int gpma_pagerank_run(gpma_t h, uint32_t iters, float damping, float *d_rank, void *stream) {
  if (!h || !d_rank || h->raw || !(damping >= 0.0f && damping <= 1.0f) || !h->snap_valid) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  cudaStream_t s = (cudaStream_t)stream;
  if (ensure_analytics(h, iters, s)) return GPMA_ENOMEM;
  Phase all(h->prof, GPMA_PROF_PAGERANK, s);
  return pr_run(h, iters, damping, d_rank, true, s);
}

int gpma_export_sorted(gpma_t h, uint64_t *d_out, uint64_t cap, uint64_t *n_out, void *stream) {
  if (!h || !n_out || (cap && !d_out)) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  cudaStream_t s = (cudaStream_t)stream;
  if (ensure_status(h, h->geo.C, s)) return GPMA_ENOMEM;
  launch_export(h->geo, h->ctl, d_out, nullptr, cap, h->w.status, s);
  int rc = read_ctl(h, s);
  if (rc) return rc;
  if ((rc = export_status(h, h->h_ctl->err))) return rc;
  *n_out = h->h_ctl->gen_count;
  return *n_out > cap ? GPMA_ECAP : cuda_ok(h);
}

int gpma_export_csr(gpma_t h, uint64_t *d_rowptr, uint32_t *d_col, uint64_t cap, uint64_t *n_out, void *stream) {
  if (!h || !n_out || !d_rowptr || (cap && !d_col) || h->raw) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  cudaStream_t s = (cudaStream_t)stream;
  if (ensure_analytics(h, 1, s) || ensure_status(h, h->geo.C, s)) return GPMA_ENOMEM;
  uint64_t *partials = (uint64_t *)dmalloc(h, scan_partials(h->V + 1) * 8 + 8, s);
  if (!partials) return GPMA_ENOMEM;
  launch_rowptr(h->geo.deg, d_rowptr, h->V, partials, s);
  launch_export(h->geo, h->ctl, nullptr, d_col, cap, h->w.status, s);
  dfree(h, partials, s);
  int rc = read_ctl(h, s);
  if (rc) return rc;
  if ((rc = export_status(h, h->h_ctl->err))) return rc;
  *n_out = h->h_ctl->gen_count;
  return *n_out > cap ? GPMA_ECAP : cuda_ok(h);
}

int gpma_export_layout(gpma_t h, uint64_t *d_slots, uint64_t cap, uint64_t *capacity_out, void *stream) {
  if (!h || !capacity_out) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  *capacity_out = h->geo.C;
  if (cap < h->geo.C) return GPMA_ECAP;
  if (!d_slots) return GPMA_EINVAL;
  cudaMemcpyAsync(d_slots, h->geo.slots, sizeof(uint64_t) * h->geo.C, cudaMemcpyDeviceToDevice,
                  (cudaStream_t)stream);
  return cuda_ok(h);
}

int gpma_import_layout(gpma_t h, const uint64_t *d_slots, uint64_t capacity, void *stream) {
  if (!h || !d_slots) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  uint32_t hh = 0;
  while (((uint64_t)h->L << hh) < capacity && hh < kMaxLv - 2) hh++;
  if (((uint64_t)h->L << hh) != capacity || capacity > (1ull << 32)) return GPMA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Geo g2;
  make_geo(h, hh, &g2);
  g2.row_end = h->geo.row_end;
  g2.deg = h->geo.deg;
  if (!alloc_arrays(h, &g2, s)) {
    free_arrays(h, &g2, s);
    return GPMA_ENOMEM;
  }
  // keep the old guard index and degrees in case the import is rejected
  uint32_t *old_re = nullptr;
  if (!h->raw) {
    if (!dalloc(h, &old_re, 2ull * h->V, s)) {
      free_arrays(h, &g2, s);
      return GPMA_ENOMEM;
    }
    cudaMemcpyAsync(old_re, h->geo.row_end, sizeof(uint32_t) * h->V, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(old_re + h->V, h->geo.deg, sizeof(uint32_t) * h->V, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(h->geo.row_end, 0xFF, sizeof(uint32_t) * h->V, s);
  }
  const uint64_t old_total_ub = h->count_ub;
  Ctl saved;
  if (read_ctl(h, s)) return h->poisoned;
  saved = *h->h_ctl;
  cudaMemcpyAsync(g2.slots, d_slots, sizeof(uint64_t) * capacity, cudaMemcpyDeviceToDevice, s);
  launch_rebuild_indexes(g2, h->ctl, s);
  launch_check(g2, h->ctl, h->check_buf, s);
  uint32_t code[4] = {0, 0, 0, 0};
  cudaMemcpyAsync(code, h->check_buf, 16, cudaMemcpyDeviceToHost, s);
  if (read_ctl(h, s)) return h->poisoned;
  if (code[0]) {
    free_arrays(h, &g2, s);
    if (old_re) {
      cudaMemcpyAsync(h->geo.row_end, old_re, sizeof(uint32_t) * h->V, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(h->geo.deg, old_re + h->V, sizeof(uint32_t) * h->V, cudaMemcpyDeviceToDevice, s);
      dfree(h, old_re, s);
    }
    cudaMemcpyAsync(&h->ctl->total, &saved.total, sizeof(uint64_t), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    h->count_ub = old_total_ub;
    h->count_lb = saved.total;
    return GPMA_EINVAL;
  }
  if (old_re) dfree(h, old_re, s);
  free_arrays(h, &h->geo, s);
  h->geo = g2;
  h->alloc_epoch++;
  h->count_ub = h->count_lb = h->h_ctl->total;
  train_model(h, s);
  return cuda_ok(h);
}

int gpma_row_end(gpma_t h, uint32_t *d_row_end, void *stream) {
  if (!h || !d_row_end || h->raw) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  cudaMemcpyAsync(d_row_end, h->geo.row_end, sizeof(uint32_t) * h->V, cudaMemcpyDeviceToDevice,
                  (cudaStream_t)stream);
  return cuda_ok(h);
}

int gpma_num_edges(gpma_t h, uint64_t *out, void *stream) {
  if (!h || !out) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  int rc = read_ctl(h, (cudaStream_t)stream);
  if (rc) return rc;
  *out = h->h_ctl->total - (h->raw ? 0 : h->V);
  return GPMA_OK;
}

int gpma_capacity(gpma_t h, uint64_t *out) {
  if (!h || !out) return GPMA_EINVAL;
  if (int rs = settle(h, nullptr)) return rs;
  *out = h->geo.C;
  return GPMA_OK;
}

int gpma_check(gpma_t h, uint32_t *code, void *stream) {
  if (!h || !code) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  cudaStream_t s = (cudaStream_t)stream;
  launch_check(h->geo, h->ctl, h->check_buf, s);
  uint32_t buf[4];
  cudaMemcpyAsync(buf, h->check_buf, 16, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return poison(h, GPMA_EDEVICE);
  *code = buf[0];
  return cuda_ok(h);
}

int gpma_update_many(gpma_t const *handles, const uint64_t *const *d_ins, const uint64_t *n_ins,
                     const uint64_t *const *d_del, const uint64_t *n_del, uint32_t count, void *stream) {
  if (!handles || (count && (!n_ins || !n_del))) return GPMA_EINVAL;
  for (uint32_t i = 0; i < count; i++) {
    if (!handles[i]) return GPMA_EINVAL;
    for (uint32_t j = 0; j < i; j++)
      if (handles[j] == handles[i]) return GPMA_EINVAL;  // one batch per handle
  }
  ManyCtx &mc = many_ctx();
  std::lock_guard<std::mutex> lock(mc.mu);
  cudaStream_t s = (cudaStream_t)stream;
  int first_err = GPMA_OK;
  auto note_err = [&](int rc) {
    if (rc && !first_err) first_err = rc;
  };
  // batches that cannot overflow their root run batched; the others alone.  The
  // batched graph holds the call's first kMaxMany handles whatever they do this time
  const uint32_t ng = count < kMaxMany ? count : kMaxMany;
  std::vector<uint32_t> graph_sel(ng), alone;
  std::vector<uint8_t> act(ng, 0);
  bool any = false;
  for (uint32_t i = 0; i < ng; i++) graph_sel[i] = i;
  for (uint32_t i = 0; i < count; i++) {
    gpma *h = handles[i];
    const uint64_t ni = n_ins[i], nd = n_del[i], n = ni + nd;
    const uint64_t *ins = d_ins ? d_ins[i] : nullptr, *del = d_del ? d_del[i] : nullptr;
    if (h->poisoned) {
      note_err(h->poisoned);
      continue;
    }
    if (n == 0) continue;
    if (n >= (1ull << 30) || (ni && !ins) || (nd && !del)) {
      note_err(GPMA_EINVAL);
      continue;
    }
    int rc = settle(h, s);
    if (!rc) rc = ensure_work(h, n, s);
    if (!rc) rc = ensure_merge_scratch(h, s);
    if (rc) {
      note_err(rc);
      continue;
    }
    const bool may_fail = h->count_ub + ni > h->geo.maxc[h->geo.h];
    if (may_fail || h->dual || i >= ng) {
      alone.push_back(i);
    } else {
      act[i] = 1;
      any = true;
    }
  }
  // the lone batches: gpma_update_batch's path, forked onto side streams
  if (!alone.empty()) {
    if (!mc.ensure_streams((uint32_t)alone.size())) return GPMA_EDEVICE;
    if (cudaEventRecord(mc.fork, s) != cudaSuccess) return GPMA_EDEVICE;
    for (size_t k = 0; k < alone.size(); k++) {
      const uint32_t i = alone[k];
      cudaStreamWaitEvent(mc.side[k], mc.fork, 0);
      note_err(update(handles[i], d_ins ? d_ins[i] : nullptr, n_ins[i], d_del ? d_del[i] : nullptr, n_del[i],
                      mc.side[k], nullptr, false));
      cudaEventRecord(mc.join[k], mc.side[k]);
    }
  }
  if (any) note_err(run_many(mc, handles, d_ins, n_ins, d_del, n_del, graph_sel, act, s));
  for (size_t k = 0; k < alone.size(); k++) cudaStreamWaitEvent(s, mc.join[k], 0);
  if (cudaGetLastError() != cudaSuccess) note_err(GPMA_EDEVICE);
  return first_err;
}

int gpma_set_wait_limit(gpma_t h, uint32_t polls, void *stream) {
  if (!h) return GPMA_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (int rs = settle(h, (cudaStream_t)stream)) return rs;
  note_launch();
  k_set_wait_limit<<<1, 1, 0, (cudaStream_t)stream>>>(h->ctl, polls);
  return cuda_ok(h);
}

int gpma_profile_enable(gpma_t h, int on) {
  if (!h) return GPMA_EINVAL;
  h->prof->on = on != 0;
  return GPMA_OK;
}

int gpma_profile_read(gpma_t h, gpma_profile *out, int reset) {
  if (!h || !out) return GPMA_EINVAL;
  Prof &p = *h->prof;
  for (auto &pr : p.pairs) {
    if (cudaEventSynchronize(pr.b) != cudaSuccess) return poison(h, GPMA_EDEVICE);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, pr.a, pr.b);
    p.ms[pr.phase] += ms;
    p.count[pr.phase] += 1;
    p.launches[pr.phase] += pr.launches;
    p.pool.push_back(pr.a);
    p.pool.push_back(pr.b);
  }
  p.pairs.clear();
  for (int i = 0; i < GPMA_PROF_N; i++) {
    out->ms[i] = p.ms[i];
    out->count[i] = p.count[i];
    out->launches[i] = p.launches[i];
  }
  if (reset) {
    for (int i = 0; i < GPMA_PROF_N; i++) {
      p.ms[i] = 0;
      p.count[i] = 0;
      p.launches[i] = 0;
    }
  }
  return cuda_ok(h);
}

uint64_t gpma_launch_count(void) { return gpk::launch_count(); }

}  // extern "C"
