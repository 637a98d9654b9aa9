/*
 * gpma_oracle.c -- plain, slow, single-threaded CPU oracle of GPMA+.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by the smoke check and by the
 * CPU-baseline leg of bench.py.  It shares no code with the CUDA library.
 *
 * Paper: Sha, Li, He, Tan, "Accelerating Dynamic Graph Analytics on GPUs".
 *
 * Readings taken where the paper is silent, ambiguous or garbled (each one is
 * also used by the CUDA library, which implements it independently):
 *  T  thresholds (Sec. 4.1, Fig. 3 table): tau_i and rho_i interpolate
 *     linearly between the leaf (height 0) and the root (height h) in exact
 *     integer hundredths; max_i is the largest count n with n < tau_i * c_i,
 *     clamped to 2 * max_{i-1}; min_i = floor(rho_i * c_i) + 1 clamped to
 *     2 * min_{i-1}.  With L=4, h=3 this reproduces the Fig. 3 table row for
 *     row.  h = 0 uses tau_0 / rho_0.
 *  R1 inputs: src, dst < n_vertices (RAW mode: key < 2^63); a bad key rejects
 *     the whole batch and nothing changes.
 *  R2 inserts and deletes are each made sorted and unique; a key present in
 *     both is removed from both (net no-op).
 *  R3 inserts of keys already stored and deletes of keys not stored are
 *     dropped.
 *  R4 leaf of a key k = the last leaf whose smallest valid key is <= k, taken
 *     on the state before the batch; leaf 0 when there is none.
 *  R5 deletion is lazy (Sec. 6.1): the slot becomes EMPTY, nothing moves.
 *  R6 level loop of Algorithm "GPMA+ Segment-Oriented Insertion" (Sec. 5.2):
 *     at level i every segment holding pending inserts merges them iff
 *     n_s + |U_s| <= max_i (the strict "< tau" of TryInsert+ as an integer).
 *  R7 if inserts remain above the root, the capacity is doubled until
 *     everything fits under the new root bound ("double the space of the old
 *     root segment", read as repeated doubling), and all keys are spread over
 *     the new array.
 *  D  dual deletion (OR_DUAL_DELETE; Sec. 4.1: deletions are the dual of
 *     insertions, the density must stay inside (rho_i, tau_i)).  After the
 *     deletes and inserts of a batch, a touched leaf whose count c lies in
 *     [min_0, max_0] is rewritten left-packed at level 0 (the whole array being
 *     one leaf waives min_0).  Every other touched leaf is a pending unit; at
 *     level i a segment holding pending units merges iff
 *     min_i <= n_s + |U_s| <= max_i, the root waiving min_h.  If the root
 *     cannot take them (count > max_h) the array grows as in R7.  After the
 *     batch, a root holding fewer than min_h keys is rebuilt at the smallest
 *     height whose root bound holds them when that height is lower (halving,
 *     possibly repeated).
 *  RD "re-dispatch evenly": a segment of m leaves receiving n sorted keys
 *     gives leaf t the ranks [floor(n t / m), floor(n (t+1) / m)), stored at
 *     the front of the leaf; the rest of the leaf is EMPTY.
 *  G  CSR on the array (Sec. 4.2, Example 4): vertex u owns a guard key
 *     (u << 32 | 0xFFFFFFFF) after its row; columns are dst.
 */
#include "gpma_oracle.h"

#include <stdlib.h>
#include <string.h>

struct or_pma {
  uint32_t V, L, tau0, tauh, rho0, rhoh, flags;
  uint32_t h;
  uint64_t C;
  uint64_t *slots;
  uint64_t maxc[OR_MAX_LEVELS], minc[OR_MAX_LEVELS];
};

static uint64_t guard_of(uint32_t u) { return ((uint64_t)u << 32) | 0xFFFFFFFFull; }
static int is_guard(uint64_t k) { return k != OR_EMPTY && (k & 0xFFFFFFFFull) == 0xFFFFFFFFull; }

/* ---- thresholds (reading T) ------------------------------------------------ */
void or_thresholds(uint32_t L, uint32_t h, uint32_t tau0, uint32_t tauh, uint32_t rho0,
                   uint32_t rhoh, uint64_t *max_out, uint64_t *min_out) {
  for (uint32_t i = 0; i <= h; i++) {
    uint64_t c = (uint64_t)L << i;
    uint64_t num_tau, num_rho, den;
    if (h == 0) {
      num_tau = (uint64_t)tau0 * c;
      num_rho = (uint64_t)rho0 * c;
      den = 100;
    } else {
      /* tau_i = tau_h + (tau_0 - tau_h)(h - i)/h ;  rho_i = rho_h - (rho_h - rho_0)(h - i)/h */
      num_tau = ((uint64_t)tauh * h + (uint64_t)(tau0 - tauh) * (h - i)) * c;
      num_rho = ((uint64_t)rhoh * h - (uint64_t)(rhoh - rho0) * (h - i)) * c;
      den = 100ull * h;
    }
    uint64_t up = num_tau ? (num_tau - 1) / den : 0; /* largest n with n < tau_i c_i */
    uint64_t lo = num_rho / den + 1;                 /* floor(rho_i c_i) + 1 */
    if (i > 0) {
      if (up > 2 * max_out[i - 1]) up = 2 * max_out[i - 1];
      if (lo > 2 * min_out[i - 1]) lo = 2 * min_out[i - 1];
    }
    max_out[i] = up;
    min_out[i] = lo;
  }
}

static void set_height(or_pma *p, uint32_t h) {
  p->h = h;
  or_thresholds(p->L, h, p->tau0, p->tauh, p->rho0, p->rhoh, p->maxc, p->minc);
}

/* ---- small helpers ----------------------------------------------------------- */
static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* sort and drop duplicates in place; returns the new length */
static uint64_t sort_unique(uint64_t *a, uint64_t n) {
  if (n == 0) return 0;
  qsort(a, n, sizeof(uint64_t), cmp_u64);
  uint64_t w = 1;
  for (uint64_t r = 1; r < n; r++)
    if (a[r] != a[w - 1]) a[w++] = a[r];
  return w;
}

/* "re-dispatch entries evenly" (reading RD) over m leaves starting at dst */
static void redistribute(uint64_t *dst, uint32_t L, uint64_t m, const uint64_t *keys, uint64_t n) {
  for (uint64_t t = 0; t < m; t++) {
    uint64_t a = (uint64_t)(((unsigned __int128)n * t) / m);
    uint64_t b = (uint64_t)(((unsigned __int128)n * (t + 1)) / m);
    for (uint64_t o = 0; o < L; o++) dst[t * L + o] = (o < b - a) ? keys[a + o] : OR_EMPTY;
  }
}

/* merge two sorted key lists with no common key */
static uint64_t merge2(const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb, uint64_t *out) {
  uint64_t i = 0, j = 0, k = 0;
  while (i < na && j < nb) out[k++] = (a[i] < b[j]) ? a[i++] : b[j++];
  while (i < na) out[k++] = a[i++];
  while (j < nb) out[k++] = b[j++];
  return k;
}

/* ---- pivots of the pre-batch state (reading R4) ------------------------------ */
typedef struct {
  uint64_t n;
  uint64_t *minkey; /* smallest valid key of each non-empty leaf, ascending */
  uint64_t *leaf;   /* that leaf's index */
} pivots;

static int build_pivots(const or_pma *p, pivots *pv) {
  uint64_t nleaves = p->C / p->L;
  pv->minkey = (uint64_t *)malloc(sizeof(uint64_t) * (nleaves ? nleaves : 1));
  pv->leaf = (uint64_t *)malloc(sizeof(uint64_t) * (nleaves ? nleaves : 1));
  if (!pv->minkey || !pv->leaf) return OR_ENOMEM;
  pv->n = 0;
  for (uint64_t j = 0; j < nleaves; j++) {
    for (uint64_t o = 0; o < p->L; o++) {
      uint64_t k = p->slots[j * p->L + o];
      if (k != OR_EMPTY) {
        pv->minkey[pv->n] = k;
        pv->leaf[pv->n] = j;
        pv->n++;
        break;
      }
    }
  }
  return OR_OK;
}

static void free_pivots(pivots *pv) {
  free(pv->minkey);
  free(pv->leaf);
}

/* last leaf whose smallest valid key is <= k; leaf 0 if none */
static uint64_t leaf_of(const pivots *pv, uint64_t k) {
  uint64_t lo = 0, hi = pv->n; /* first index with minkey > k */
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (pv->minkey[mid] > k) hi = mid; else lo = mid + 1;
  }
  return lo == 0 ? 0 : pv->leaf[lo - 1];
}

/* slot holding k inside leaf j, or -1 */
static int64_t find_in_leaf(const or_pma *p, uint64_t j, uint64_t k) {
  for (uint64_t o = 0; o < p->L; o++)
    if (p->slots[j * p->L + o] == k) return (int64_t)(j * p->L + o);
  return -1;
}

/* ---- create / destroy --------------------------------------------------------- */
static int apply_batch(or_pma *p, uint64_t *I, uint64_t nI, uint64_t *D, uint64_t nD,
                       uint64_t n_raw, or_stats *st);

or_pma *or_create(uint32_t n_vertices, uint32_t L, uint32_t tau0, uint32_t tauh,
                  uint32_t rho0, uint32_t rhoh, uint32_t flags) {
  if (L < 2 || L > (1u << 20) || (L & (L - 1))) return NULL;
  if (!(tauh > 0 && tauh <= tau0 && tau0 <= 100 && rho0 <= rhoh && rhoh < tauh)) return NULL;
  if (!(flags & OR_RAW_KEYS) && (n_vertices == 0 || n_vertices > (1u << 31))) return NULL;
  or_pma *p = (or_pma *)calloc(1, sizeof(or_pma));
  if (!p) return NULL;
  p->V = n_vertices; p->L = L; p->tau0 = tau0; p->tauh = tauh;
  p->rho0 = rho0; p->rhoh = rhoh; p->flags = flags;
  p->C = L;
  p->slots = (uint64_t *)malloc(sizeof(uint64_t) * L);
  if (!p->slots) { free(p); return NULL; }
  for (uint64_t s = 0; s < L; s++) p->slots[s] = OR_EMPTY;
  set_height(p, 0);
  if (!(flags & OR_RAW_KEYS)) {
    /* the guards enter through the ordinary update path (bulk load = update) */
    uint64_t *g = (uint64_t *)malloc(sizeof(uint64_t) * n_vertices);
    if (!g) { or_destroy(p); return NULL; }
    for (uint32_t u = 0; u < n_vertices; u++) g[u] = guard_of(u);
    int rc = apply_batch(p, g, n_vertices, NULL, 0, n_vertices, NULL);
    free(g);
    if (rc) { or_destroy(p); return NULL; }
  }
  return p;
}

void or_destroy(or_pma *p) {
  if (!p) return;
  free(p->slots);
  free(p);
}

uint64_t or_capacity(const or_pma *p) { return p->C; }
uint32_t or_height(const or_pma *p) { return p->h; }

uint64_t or_num_valid(const or_pma *p) {
  uint64_t n = 0;
  for (uint64_t s = 0; s < p->C; s++) n += p->slots[s] != OR_EMPTY;
  return n;
}

void or_layout(const or_pma *p, uint64_t *out) { memcpy(out, p->slots, sizeof(uint64_t) * p->C); }

int or_import_layout(or_pma *p, const uint64_t *slots, uint64_t capacity) {
  uint32_t h = 0;
  while (((uint64_t)p->L << h) < capacity && h < OR_MAX_LEVELS - 1) h++;
  if (((uint64_t)p->L << h) != capacity) return OR_EINVAL;
  uint64_t *ns = (uint64_t *)malloc(sizeof(uint64_t) * capacity);
  if (!ns) return OR_ENOMEM;
  memcpy(ns, slots, sizeof(uint64_t) * capacity);
  free(p->slots);
  p->slots = ns;
  p->C = capacity;
  set_height(p, h);
  return OR_OK;
}

/* ---- the batch update --------------------------------------------------------- */
static int key_ok(const or_pma *p, uint64_t k) {
  if (p->flags & OR_RAW_KEYS) return k < (1ull << 63);
  return (k >> 32) < p->V && (k & 0xFFFFFFFFull) < p->V;
}

int or_update(or_pma *p, const uint64_t *ins, uint64_t n_ins, const uint64_t *del,
              uint64_t n_del, or_stats *st) {
  if (st) memset(st, 0, sizeof(*st));
  /* R1: validate everything before touching anything */
  for (uint64_t i = 0; i < n_ins; i++) if (!key_ok(p, ins[i])) return OR_EINVAL;
  for (uint64_t i = 0; i < n_del; i++) if (!key_ok(p, del[i])) return OR_EINVAL;
  /* R2: sort + unique each side, then cancel keys present on both sides */
  uint64_t *I = (uint64_t *)malloc(sizeof(uint64_t) * (n_ins ? n_ins : 1));
  uint64_t *D = (uint64_t *)malloc(sizeof(uint64_t) * (n_del ? n_del : 1));
  if (!I || !D) { free(I); free(D); return OR_ENOMEM; }
  if (n_ins) memcpy(I, ins, sizeof(uint64_t) * n_ins);
  if (n_del) memcpy(D, del, sizeof(uint64_t) * n_del);
  uint64_t nI = sort_unique(I, n_ins), nD = sort_unique(D, n_del);
  uint64_t a = 0, b = 0, wi = 0, wd = 0;
  while (a < nI || b < nD) {
    if (b >= nD || (a < nI && I[a] < D[b])) I[wi++] = I[a++];
    else if (a >= nI || D[b] < I[a]) D[wd++] = D[b++];
    else { a++; b++; } /* in both: net no-op */
  }
  int rc = apply_batch(p, I, wi, D, wd, n_ins + n_del, st);
  free(I);
  free(D);
  return rc;
}

/* Reading D, levels 0..h: pending units are touched leaves out of bounds.  On
   return *npend counts the inserts still pending and *nunits the leaves still
   pending (both nonzero only if the root could not take them). */
static int level_loop_dual(or_pma *p, const uint64_t *I, const uint64_t *leafI, uint64_t nI, uint8_t *pend,
                           const uint8_t *touched, int8_t *cover, uint64_t *merges, uint32_t *climbed,
                           uint64_t *npend, uint8_t **unit_out, uint64_t *nunits_out) {
  const uint32_t L = p->L;
  const uint64_t nleaves = p->C / L;
  uint8_t *unit = (uint8_t *)calloc(nleaves, 1);
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (p->C + nI + 1));
  uint64_t *ins = (uint64_t *)malloc(sizeof(uint64_t) * (nI + 1));
  uint64_t *mrg = (uint64_t *)malloc(sizeof(uint64_t) * (p->C + nI + 1));
  *unit_out = unit;
  if (!unit || !keys || !ins || !mrg) { free(keys); free(ins); free(mrg); return OR_ENOMEM; }
  uint64_t nunits = 0;
  /* level 0: every touched leaf, with its inserts (contiguous in I, leaves ascending) */
  uint64_t a = 0;
  for (uint64_t j = 0; j < nleaves; j++) {
    uint64_t b = a;
    while (b < nI && leafI[b] == j) b++;
    if (touched[j]) {
      uint64_t nv = 0;
      for (uint64_t o = 0; o < L; o++) if (p->slots[j * L + o] != OR_EMPTY) keys[nv++] = p->slots[j * L + o];
      uint64_t c = nv + (b - a);
      if (c <= p->maxc[0] && (c >= p->minc[0] || p->h == 0)) {
        uint64_t n = merge2(keys, nv, I + a, b - a, mrg);
        redistribute(p->slots + j * L, L, 1, mrg, n);
        for (uint64_t x = a; x < b; x++) pend[x] = 0;
        *npend -= b - a;
        merges[0]++;
        cover[j] = 0;
      } else {
        unit[j] = 1;
        nunits++;
      }
    }
    a = b;
  }
  /* levels 1..h: segments holding pending units */
  for (uint32_t lvl = 1; lvl <= p->h && nunits > 0; lvl++) {
    const uint64_t span = (uint64_t)1 << lvl;
    for (uint64_t s = 0; s < nleaves >> lvl; s++) {
      uint64_t j0 = s * span, u_units = 0;
      for (uint64_t j = j0; j < j0 + span; j++) u_units += unit[j];
      if (!u_units) continue;
      uint64_t nv = 0, q = 0;
      for (uint64_t x = j0 * L; x < (j0 + span) * L; x++) if (p->slots[x] != OR_EMPTY) keys[nv++] = p->slots[x];
      for (uint64_t x = 0; x < nI; x++)
        if (pend[x] && (leafI[x] >> lvl) == s) ins[q++] = I[x];
      uint64_t t = nv + q;
      if (t <= p->maxc[lvl] && (t >= p->minc[lvl] || lvl == p->h)) {
        uint64_t n = merge2(keys, nv, ins, q, mrg);
        redistribute(p->slots + j0 * L, L, span, mrg, n);
        for (uint64_t x = 0; x < nI; x++)
          if (pend[x] && (leafI[x] >> lvl) == s) pend[x] = 0;
        *npend -= q;
        for (uint64_t j = j0; j < j0 + span; j++) {
          nunits -= unit[j];
          unit[j] = 0;
          cover[j] = (int8_t)lvl;
        }
        merges[lvl]++;
        *climbed = lvl;
      }
    }
  }
  *nunits_out = nunits;
  free(keys); free(ins); free(mrg);
  return OR_OK;
}

/* R3..R7 on sorted, unique, disjoint I and D */
static int apply_batch(or_pma *p, uint64_t *I, uint64_t nI, uint64_t *D, uint64_t nD,
                       uint64_t n_raw, or_stats *st) {
  const uint32_t L = p->L;
  const uint64_t nleaves = p->C / L;
  const uint64_t C_old = p->C;
  const uint32_t h_old = p->h;
  pivots pv;
  if (build_pivots(p, &pv)) { free_pivots(&pv); return OR_ENOMEM; }

  uint64_t *leafI = (uint64_t *)malloc(sizeof(uint64_t) * (nI ? nI : 1));
  uint64_t *leafD = (uint64_t *)malloc(sizeof(uint64_t) * (nD ? nD : 1));
  uint8_t *touched = (uint8_t *)calloc(nleaves, 1);
  int8_t *cover = (int8_t *)malloc(nleaves);
  uint8_t *pend = (uint8_t *)malloc(nI ? nI : 1);
  if (!leafI || !leafD || !touched || !cover || !pend) {
    free(leafI); free(leafD); free(touched); free(cover); free(pend); free_pivots(&pv);
    return OR_ENOMEM;
  }
  memset(cover, -1, nleaves);

  /* R4 on the pre-batch state, for every key that survived R2 */
  for (uint64_t i = 0; i < nI; i++) { leafI[i] = leaf_of(&pv, I[i]); touched[leafI[i]] = 1; }
  for (uint64_t i = 0; i < nD; i++) { leafD[i] = leaf_of(&pv, D[i]); touched[leafD[i]] = 1; }

  /* R3: drop inserts already stored and deletes not stored */
  uint64_t w = 0;
  for (uint64_t i = 0; i < nI; i++)
    if (find_in_leaf(p, leafI[i], I[i]) < 0) { I[w] = I[i]; leafI[w] = leafI[i]; w++; }
  nI = w;
  w = 0;
  int64_t *slotD = (int64_t *)malloc(sizeof(int64_t) * (nD ? nD : 1));
  if (!slotD) { free(leafI); free(leafD); free(touched); free(cover); free(pend); free_pivots(&pv); return OR_ENOMEM; }
  for (uint64_t i = 0; i < nD; i++) {
    int64_t s = find_in_leaf(p, leafD[i], D[i]);
    if (s >= 0) { D[w] = D[i]; leafD[w] = leafD[i]; slotD[w] = s; w++; }
  }
  nD = w;

  /* R5: lazy deletion */
  for (uint64_t i = 0; i < nD; i++) p->slots[slotD[i]] = OR_EMPTY;

  /* R6: bottom-up level loop (Algorithm "GPMA+ Segment-Oriented Insertion") */
  uint64_t npend = nI;
  for (uint64_t i = 0; i < nI; i++) pend[i] = 1;
  uint64_t *buf = NULL, *mrg = NULL, *ub = NULL;
  uint64_t cap_buf = 0;
  uint32_t climbed = 0;
  uint64_t merges[OR_MAX_LEVELS];
  memset(merges, 0, sizeof(merges));
  int rc = OR_OK;
  const int dual = (p->flags & OR_DUAL_DELETE) != 0;
  uint64_t nunits = 0;
  uint8_t *unit = NULL;
  if (dual) {
    rc = level_loop_dual(p, I, leafI, nI, pend, touched, cover, merges, &climbed, &npend, &unit, &nunits);
    if (rc) goto done;
  }
  for (uint32_t lvl = 0; lvl <= p->h && npend > 0 && !dual; lvl++) {
    const uint64_t seg_slots = (uint64_t)L << lvl;
    uint64_t a = 0;
    while (a < nI) {
      if (!pend[a]) { a++; continue; }
      /* UniqueSegments: the pending inserts of segment s = leaf >> lvl are contiguous */
      uint64_t s = leafI[a] >> lvl, b = a, u = 0;
      while (b < nI && (leafI[b] >> lvl) == s) { u += pend[b]; b++; }
      /* TryInsert+: CountSegment + CountUpdatesInSegment */
      uint64_t lo = s * seg_slots, nv = 0;
      for (uint64_t x = lo; x < lo + seg_slots; x++) nv += p->slots[x] != OR_EMPTY;
      if (nv + u <= p->maxc[lvl]) {
        if (cap_buf < nv + u) {
          cap_buf = nv + u;
          free(buf); free(mrg); free(ub);
          buf = (uint64_t *)malloc(sizeof(uint64_t) * cap_buf);
          mrg = (uint64_t *)malloc(sizeof(uint64_t) * cap_buf);
          ub = (uint64_t *)malloc(sizeof(uint64_t) * cap_buf);
          if (!buf || !mrg || !ub) { rc = OR_ENOMEM; goto done; }
        }
        uint64_t k = 0;
        for (uint64_t x = lo; x < lo + seg_slots; x++)
          if (p->slots[x] != OR_EMPTY) buf[k++] = p->slots[x];
        uint64_t q = 0;
        for (uint64_t x = a; x < b; x++)
          if (pend[x]) { ub[q++] = I[x]; pend[x] = 0; }
        uint64_t n = merge2(buf, nv, ub, u, mrg); /* Merge(s, U_s) */
        redistribute(p->slots + lo, L, (uint64_t)1 << lvl, mrg, n); /* re-dispatch evenly */
        npend -= u;
        merges[lvl]++;
        climbed = lvl;
        for (uint64_t j = s << lvl; j < (s + 1) << lvl; j++) cover[j] = (int8_t)lvl;
      }
      a = b;
    }
  }

  /* R7: the root could not take the rest -- grow and spread everything */
  int resized = 0;
  if (npend > 0 || nunits > 0) {
    uint64_t nv = 0;
    for (uint64_t x = 0; x < p->C; x++) nv += p->slots[x] != OR_EMPTY;
    uint64_t *all = (uint64_t *)malloc(sizeof(uint64_t) * (nv ? nv : 1));
    uint64_t *rest = (uint64_t *)malloc(sizeof(uint64_t) * (npend ? npend : 1));
    uint64_t *mer = (uint64_t *)malloc(sizeof(uint64_t) * (nv + npend));
    if (!all || !rest || !mer) { free(all); free(rest); free(mer); rc = OR_ENOMEM; goto done; }
    uint64_t k = 0;
    for (uint64_t x = 0; x < p->C; x++) if (p->slots[x] != OR_EMPTY) all[k++] = p->slots[x];
    uint64_t q = 0;
    for (uint64_t x = 0; x < nI; x++) if (pend[x]) rest[q++] = I[x];
    uint64_t n = merge2(all, nv, rest, npend, mer);
    uint32_t h2 = p->h + 1;
    uint64_t mx[OR_MAX_LEVELS], mn[OR_MAX_LEVELS];
    for (;;) {
      if (h2 >= OR_MAX_LEVELS - 1) { free(all); free(rest); free(mer); rc = OR_ENOMEM; goto done; }
      or_thresholds(L, h2, p->tau0, p->tauh, p->rho0, p->rhoh, mx, mn);
      if (n <= mx[h2]) break;
      h2++;
    }
    uint64_t C2 = (uint64_t)L << h2;
    uint64_t *ns = (uint64_t *)malloc(sizeof(uint64_t) * C2);
    if (!ns) { free(all); free(rest); free(mer); rc = OR_ENOMEM; goto done; }
    redistribute(ns, L, (uint64_t)1 << h2, mer, n);
    free(p->slots);
    p->slots = ns;
    p->C = C2;
    set_height(p, h2);
    free(all); free(rest); free(mer);
    npend = 0;
    resized = 1;
    climbed = h_old + 1;
  } else if (dual && p->h > 0) {
    /* D: a root below min_h is rebuilt at the smallest height that holds it */
    uint64_t nv = 0;
    for (uint64_t x = 0; x < p->C; x++) nv += p->slots[x] != OR_EMPTY;
    if (nv < p->minc[p->h]) {
      uint32_t h2 = 0;
      uint64_t mx[OR_MAX_LEVELS], mn[OR_MAX_LEVELS];
      for (;; h2++) {
        or_thresholds(L, h2, p->tau0, p->tauh, p->rho0, p->rhoh, mx, mn);
        if (nv <= mx[h2]) break;
      }
      if (h2 < p->h) {
        uint64_t *all = (uint64_t *)malloc(sizeof(uint64_t) * (nv ? nv : 1));
        uint64_t C2 = (uint64_t)L << h2;
        uint64_t *ns = (uint64_t *)malloc(sizeof(uint64_t) * C2);
        if (!all || !ns) { free(all); free(ns); rc = OR_ENOMEM; goto done; }
        uint64_t k = 0;
        for (uint64_t x = 0; x < p->C; x++) if (p->slots[x] != OR_EMPTY) all[k++] = p->slots[x];
        redistribute(ns, L, (uint64_t)1 << h2, all, nv);
        free(all);
        free(p->slots);
        p->slots = ns;
        p->C = C2;
        set_height(p, h2);
        resized = 2;
      }
    }
  }

  if (st) {
    /* algorithmic bytes: read every raw update key once; read every touched
       leaf once (presence / delete / merge); read the untouched part and write
       all of each final merged segment; 8 B per EMPTY written outside them;
       a resize reads the old array and writes the new one instead. */
    uint64_t nt = 0, ncov = 0, ncov_untouched = 0, empties = 0;
    for (uint64_t j = 0; j < nleaves; j++) {
      nt += touched[j];
      if (cover[j] >= 0) { ncov++; ncov_untouched += !touched[j]; }
    }
    for (uint64_t i = 0; i < nD; i++) empties += cover[leafD[i]] < 0;
    uint64_t ndl = 0;  /* leafD is non-decreasing: D is sorted */
    for (uint64_t i = 0; i < nD; i++) ndl += i == 0 || leafD[i] != leafD[i - 1];
    st->delete_leaves = ndl;
    st->n_inserted = nI;
    st->n_deleted = nD;
    st->n_ignored = n_raw - nI - nD;
    st->levels_climbed = climbed;
    st->resized = (uint32_t)resized;
    st->touched_leaves = nt;
    st->covered_leaves = resized ? 0 : ncov;
    if (resized)
      st->alg_bytes = 8 * n_raw + 8ull * L * nt + 8 * C_old + 8 * p->C;
    else
      st->alg_bytes = 8 * n_raw + 8ull * L * nt + 8ull * L * ncov + 8ull * L * ncov_untouched + 8 * empties;
    for (uint32_t i = 0; i < OR_MAX_LEVELS; i++) st->merges[i] = merges[i];
  }
done:
  free(unit);
  free(buf); free(mrg); free(ub);
  free(leafI); free(leafD); free(touched); free(cover); free(pend); free(slotD);
  free_pivots(&pv);
  return rc;
}

/* ---- exports ---------------------------------------------------------------- */
uint64_t or_export_sorted(const or_pma *p, uint64_t *out) {
  uint64_t n = 0;
  for (uint64_t s = 0; s < p->C; s++) {
    uint64_t k = p->slots[s];
    if (k == OR_EMPTY) continue;
    if (!(p->flags & OR_RAW_KEYS) && is_guard(k)) continue;
    if (out) out[n] = k;
    n++;
  }
  return n;
}

uint64_t or_export_csr(const or_pma *p, uint64_t *rowptr, uint32_t *col) {
  for (uint64_t u = 0; u <= p->V; u++) rowptr[u] = 0;
  uint64_t e = 0;
  for (uint64_t s = 0; s < p->C; s++) {
    uint64_t k = p->slots[s];
    if (k == OR_EMPTY || is_guard(k)) continue;
    rowptr[(k >> 32) + 1]++;
    if (col) col[e] = (uint32_t)(k & 0xFFFFFFFFull);
    e++;
  }
  for (uint64_t u = 0; u < p->V; u++) rowptr[u + 1] += rowptr[u];
  return e;
}

void or_row_end(const or_pma *p, uint32_t *row_end) {
  for (uint64_t s = 0; s < p->C; s++)
    if (is_guard(p->slots[s])) row_end[p->slots[s] >> 32] = (uint32_t)s;
}

/* ---- analytics (Sec. 4.2 and Sec. 6.1 "Applications") ------------------------ */
/* BFS (Algorithm "BFS"): hop depth from src along out-edges, -1 if unreachable */
/* The three analytics below read a plain array of keys: the slot array of a PMA
   (EMPTY slots and guards are skipped) or a list of edges (src << 32 | dst) in any
   order.  Every src and dst must be below V. */
static int keys_in_range(uint32_t V, const uint64_t *keys, uint64_t n) {
  for (uint64_t i = 0; i < n; i++) {
    uint64_t k = keys[i];
    if (k == OR_EMPTY || is_guard(k)) continue;
    if ((k >> 32) >= V || (k & 0xFFFFFFFFull) >= V) return 0;
  }
  return 1;
}

/* breadth-first search from src over out-edges (Algorithm "BFS", Sec. 4.2):
   out-neighbour lists by a counting pass, then a FIFO queue; -1 = unreachable */
static int bfs_keys(uint32_t V, const uint64_t *keys, uint64_t n, uint32_t src, int32_t *depth) {
  if (src >= V || !keys_in_range(V, keys, n)) return OR_EINVAL;
  uint64_t *rp = (uint64_t *)calloc((uint64_t)V + 1, sizeof(uint64_t));
  uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * ((uint64_t)V + 1));
  uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * ((uint64_t)V + 1));
  if (!rp || !cur || !queue) { free(rp); free(cur); free(queue); return OR_ENOMEM; }
  for (uint64_t i = 0; i < n; i++) {
    uint64_t k = keys[i];
    if (k != OR_EMPTY && !is_guard(k)) rp[(k >> 32) + 1]++;
  }
  for (uint64_t u = 0; u < V; u++) rp[u + 1] += rp[u];
  uint32_t *col = (uint32_t *)malloc(sizeof(uint32_t) * (rp[V] ? rp[V] : 1));
  if (!col) { free(rp); free(cur); free(queue); return OR_ENOMEM; }
  for (uint64_t u = 0; u < V; u++) cur[u] = rp[u];
  for (uint64_t i = 0; i < n; i++) {
    uint64_t k = keys[i];
    if (k != OR_EMPTY && !is_guard(k)) col[cur[k >> 32]++] = (uint32_t)(k & 0xFFFFFFFFull);
  }
  for (uint32_t v = 0; v < V; v++) depth[v] = -1;
  uint64_t head = 0, tail = 0;
  depth[src] = 0;
  queue[tail++] = src;
  while (head < tail) {
    uint32_t u = queue[head++];
    for (uint64_t e = rp[u]; e < rp[u + 1]; e++) {
      uint32_t v = col[e];
      if (depth[v] < 0) { depth[v] = depth[u] + 1; queue[tail++] = v; }
    }
  }
  free(queue); free(rp); free(cur); free(col);
  return OR_OK;
}

int or_bfs(const or_pma *p, uint32_t src, int32_t *depth) {
  if (p->flags & OR_RAW_KEYS) return OR_EINVAL;
  return bfs_keys(p->V, p->slots, p->C, src, depth);
}

int or_bfs_edges(uint32_t V, const uint64_t *keys, uint64_t n, uint32_t src, int32_t *depth) {
  return bfs_keys(V, keys, n, src, depth);
}

/* weakly connected components; every vertex is labelled with the smallest
   vertex id of its component (union-find, the smaller root always wins) */
static uint32_t uf_find(uint32_t *parent, uint32_t x) {
  while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
  return x;
}

static int cc_keys(uint32_t V, const uint64_t *keys, uint64_t n, uint32_t *label) {
  if (!keys_in_range(V, keys, n)) return OR_EINVAL;
  for (uint32_t v = 0; v < V; v++) label[v] = v;
  for (uint64_t i = 0; i < n; i++) {
    uint64_t k = keys[i];
    if (k == OR_EMPTY || is_guard(k)) continue;
    uint32_t a = uf_find(label, (uint32_t)(k >> 32)), b = uf_find(label, (uint32_t)(k & 0xFFFFFFFFu));
    if (a < b) label[b] = a; else if (b < a) label[a] = b;
  }
  for (uint32_t v = 0; v < V; v++) label[v] = uf_find(label, v);
  return OR_OK;
}

int or_cc(const or_pma *p, uint32_t *label) {
  if (p->flags & OR_RAW_KEYS) return OR_EINVAL;
  return cc_keys(p->V, p->slots, p->C, label);
}

int or_cc_edges(uint32_t V, const uint64_t *keys, uint64_t n, uint32_t *label) {
  return cc_keys(V, keys, n, label);
}

/* PageRank by power iteration (Sec. 6.1): x0 = 1/N,
   x'_v = (1-d)/N + d * ( sum_{u->v} x_u / outdeg(u) + sum_{outdeg(w)=0} x_w / N ),
   a fixed number of iterations, in double precision. */
static int pagerank_keys(uint32_t V, const uint64_t *keys, uint64_t n, uint32_t iters, double damping,
                         double *rank) {
  if (!keys_in_range(V, keys, n)) return OR_EINVAL;
  uint64_t N = V;
  double *y = (double *)malloc(sizeof(double) * (N ? N : 1));
  uint64_t *deg = (uint64_t *)calloc(N ? N : 1, sizeof(uint64_t));
  if (!y || !deg) { free(y); free(deg); return OR_ENOMEM; }
  for (uint64_t i = 0; i < n; i++) {
    uint64_t k = keys[i];
    if (k != OR_EMPTY && !is_guard(k)) deg[k >> 32]++;
  }
  for (uint64_t v = 0; v < N; v++) rank[v] = 1.0 / (double)N;
  for (uint32_t it = 0; it < iters; it++) {
    double dangling = 0.0;
    for (uint64_t v = 0; v < N; v++) { y[v] = 0.0; if (deg[v] == 0) dangling += rank[v]; }
    for (uint64_t i = 0; i < n; i++) {
      uint64_t k = keys[i];
      if (k == OR_EMPTY || is_guard(k)) continue;
      uint64_t u = k >> 32, v = k & 0xFFFFFFFFull;
      y[v] += rank[u] / (double)deg[u];
    }
    for (uint64_t v = 0; v < N; v++)
      rank[v] = (1.0 - damping) / (double)N + damping * (y[v] + dangling / (double)N);
  }
  free(y); free(deg);
  return OR_OK;
}

int or_pagerank(const or_pma *p, uint32_t iters, double damping, double *rank) {
  if (p->flags & OR_RAW_KEYS) return OR_EINVAL;
  return pagerank_keys(p->V, p->slots, p->C, iters, damping, rank);
}

int or_pagerank_edges(uint32_t V, const uint64_t *keys, uint64_t n, uint32_t iters, double damping,
                      double *rank) {
  return pagerank_keys(V, keys, n, iters, damping, rank);
}

/* ---- invariants ----------------------------------------------------------------
   1 valid keys not strictly increasing; 2 a leaf holds more than max_0;
   3 capacity is not L*2^h; 4 a key outside the vertex range or a guard missing. */
int or_check_invariants(const or_pma *p) {
  if (((uint64_t)p->L << p->h) != p->C) return 3;
  uint64_t prev = 0;
  int have = 0;
  for (uint64_t s = 0; s < p->C; s++) {
    uint64_t k = p->slots[s];
    if (k == OR_EMPTY) continue;
    if (have && k <= prev) return 1;
    prev = k; have = 1;
  }
  for (uint64_t j = 0; j < p->C / p->L; j++) {
    uint64_t c = 0;
    for (uint64_t o = 0; o < p->L; o++) c += p->slots[j * p->L + o] != OR_EMPTY;
    if (c > p->maxc[0]) return 2;
    if (p->flags & OR_DUAL_DELETE) /* no deletion leaves a hole: leaves stay left-packed */
      for (uint64_t o = 0; o < p->L; o++)
        if ((p->slots[j * p->L + o] != OR_EMPTY) != (o < c)) return 5;
  }
  if (!(p->flags & OR_RAW_KEYS)) {
    uint64_t guards = 0;
    for (uint64_t s = 0; s < p->C; s++) {
      uint64_t k = p->slots[s];
      if (k == OR_EMPTY) continue;
      if ((k >> 32) >= p->V) return 4;
      if (is_guard(k)) guards++;
      else if ((k & 0xFFFFFFFFull) >= p->V) return 4;
    }
    if (guards != p->V) return 4;
  }
  return 0;
}
