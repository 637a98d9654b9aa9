// k_update.cu -- the level loop of Algorithm "GPMA+ Segment-Oriented Insertion"
// (Sec. 5.2) with lazy deletion (Sec. 6.1), organised for one GB300.
//
// Fact used throughout: for a segment s of level i the test of TryInsert+ compares
// n_s + |U_s| with max_i, where n_s counts the valid keys of s after the deletes and
// after the merges of lower levels, and U_s are the inserts of s still pending.
// Every insert of s is either merged below (and counted in n_s) or pending (and
// counted in U_s), so n_s + |U_s| = (valid keys of s after the deletes) + (all
// surviving inserts of s): the test does not depend on the order of the merges.
// The level at which an insert merges is therefore the lowest level whose
// segment passes that test, computable from a count tree, and the final layout
// is fixed by the outermost merged segments alone (a merge re-spreads its whole
// segment, erasing any merge inside it).  So:
//   k_leaf_pass    one warp per touched leaf: presence filter, lazy deletes, and the
//                  level-0 TryInsert+ (merge + even re-dispatch inside the leaf)
//   k_pending / k_eruns / k_tree_* / k_esc_level / k_esc_top / k_segs
//                  inserts that did not fit their leaf (only then): rebuild the
//                  count tree, find their merge level, the outermost merged
//                  segments and their pending inserts
//   segment merge  gather valid keys of those segments, merge with the pending
//                  inserts (merge path), re-dispatch evenly, rewrite the counts
#include "gpma_dev.cuh"
#include "gpma_launch.h"
#include "scan_dev.cuh"

namespace gpk {


struct WarpBufs {
  uint64_t *a, *b, *out;
  uint16_t *pos;
  uint8_t *mark;
};

__device__ __forceinline__ WarpBufs warp_bufs(unsigned char *smem, uint32_t per_warp, uint32_t L) {
  unsigned char *base = smem + (threadIdx.x >> 5) * per_warp;
  WarpBufs b;
  b.a = (uint64_t *)base;
  b.b = b.a + L;
  b.out = b.b + L;
  b.pos = (uint16_t *)(b.out + L);
  b.mark = base + 24u * L + ((2u * (L + 1u) + 15u) & ~15u);
  return b;
}

// ---- level 0: one warp per touched leaf ------------------------------------------------------
template <class Blk>
__device__ __forceinline__ void leaf_pass_body(const Blk &bk, const Geo &g, Ctl *ctl, const Work &w, uint32_t per_warp,
                                               int rest_only) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (ctl->err) return;
  if (rest_only && ctl->nlong == 0) return;
  const uint32_t L = g.L, lane = lane_id();
  const uint32_t wpb = blockDim.x >> 5;
  WarpBufs B = warp_bufs(smem, per_warp, L);
  uint64_t *vkeys = B.a, *ins = B.b, *out = B.out;
  uint16_t *vpos = B.pos;
  uint8_t *dmark = B.mark;
  const uint32_t nruns = ctl->nruns;
  uint64_t acc_ins = 0, acc_del = 0;
  uint32_t acc_m0 = 0, acc_esc = 0;
  for (uint32_t r = bk.x() * wpb + (threadIdx.x >> 5); r < nruns; r += bk.n() * wpb) {
    const uint32_t rs = w.run_start[r], re = w.run_start[r + 1];
    if (rest_only && re - rs <= 32) continue;  // done by the 64-slot fast path
    if (re - rs > kLongRun) {  // done by the chunked path: reset its accumulators
      if (lane == 0) {
        w.rdelta[r] = 0;
        w.rdel[r] = 0;
        atomicAdd(&ctl->nvlong, 1u);
      }
      continue;
    }
    const uint32_t j = w.rleaf[r];
    uint64_t *leaf = g.slots + (uint64_t)j * L;
    // the leaf's valid keys, compacted, with their slot offsets
    uint32_t nv = 0;
    for (uint32_t b = 0; b < L; b += 32) {
      uint32_t o = b + lane;
      uint64_t k = o < L ? leaf[o] : kEmpty;
      bool v = k != kEmpty;
      uint32_t bal = __ballot_sync(0xFFFFFFFFu, v);
      if (v) {
        uint32_t idx = nv + __popc(bal & lanemask_lt());
        vkeys[idx] = k;
        vpos[idx] = (uint16_t)o;
        dmark[idx] = 0;
      }
      nv += __popc(bal);
    }
    __syncwarp();
    // presence filter (reading R3) and lazy deletes (R5); surviving inserts in order
    uint32_t nins = 0, ndel = 0;
    for (uint32_t c = rs; c < re; c += 32) {
      const uint32_t e = c + lane;
      const bool act = e < re;
      uint64_t key = act ? w.ukey[e] : 0ull;
      uint32_t tag = act ? w.utag[e] : 0u;
      uint32_t idx = act ? lower_bound_dev(vkeys, nv, key) : 0u;
      bool found = act && idx < nv && vkeys[idx] == key;
      bool dl = act && tag && found;
      bool sv = act && !tag && !found;
      if (dl) dmark[idx] = 1;
      uint32_t bs = __ballot_sync(0xFFFFFFFFu, sv);
      if (sv) {
        uint32_t p = nins + __popc(bs & lanemask_lt());
        if (p < L) ins[p] = key;
      }
      nins += __popc(bs);
      ndel += __popc(__ballot_sync(0xFFFFFFFFu, dl));
      if (act) w.eflag[e] = dl ? 1 : (sv ? 2 : 0);
    }
    __syncwarp();
    const uint32_t cnt_del = nv - ndel;
    const bool fits = leaf_fits(g, (uint64_t)cnt_del + nins, nins);
    if (fits) {
      // TryInsert+ at level 0: merge the kept keys with the inserts, left-packed
      uint32_t run = 0;
      for (uint32_t b = 0; b < nv; b += 32) {
        uint32_t a = b + lane;
        bool kp = a < nv && !dmark[a];
        uint32_t bal = __ballot_sync(0xFFFFFFFFu, kp);
        if (a < nv) vpos[a] = (uint16_t)(run + __popc(bal & lanemask_lt()));  // kept keys before a
        run += __popc(bal);
      }
      if (lane == 0) vpos[nv] = (uint16_t)run;
      __syncwarp();
      for (uint32_t a = lane; a < nv; a += 32)
        if (!dmark[a]) out[vpos[a] + lower_bound_dev(ins, nins, vkeys[a])] = vkeys[a];
      for (uint32_t b = lane; b < nins; b += 32) out[b + vpos[lower_bound_dev(vkeys, nv, ins[b])]] = ins[b];
      __syncwarp();
      const uint32_t n = cnt_del + nins;
      for (uint32_t o = lane; o < L; o += 32) {
        uint64_t k = o < n ? out[o] : kEmpty;
        leaf[o] = k;
        if (!g.raw && o < n && is_guard(k)) g.row_end[k >> 32] = (uint32_t)((uint64_t)j * L + o);
      }
      if (lane == 0) {
        g.F[j] = n ? out[0] : kEmpty;  // n = 0 only for a single-leaf array in dual mode
        g.cnt[j] = n;
      }
      for (uint32_t c = rs + lane; c < re; c += 32)
        if (w.eflag[c] == 2) w.eflag[c] = 1;
    } else {
      for (uint32_t a = lane; a < nv; a += 32)
        if (dmark[a]) leaf[vpos[a]] = kEmpty;
      uint32_t first = nv;
      for (uint32_t b = 0; b < nv; b += 32) {
        uint32_t a = b + lane;
        uint32_t bal = __ballot_sync(0xFFFFFFFFu, a < nv && !dmark[a]);
        if (bal) {
          first = b + __ffs(bal) - 1;
          break;
        }
      }
      if (lane == 0) {
        g.F[j] = first < nv ? vkeys[first] : kEmpty;
        g.cnt[j] = cnt_del;
      }
    }
    if (lane == 0) {
      w.rdelta[r] = (int32_t)nins - (int32_t)ndel;
      w.rinfo[r] = fits ? 1 : ((nins || g.dual) ? 2 : 0);
      w.rdel[r] = ndel;
    }
    acc_ins += nins;
    acc_del += ndel;
    acc_m0 += fits;
    acc_esc += !fits && (nins || g.dual);
    __syncwarp();
  }
  if (lane == 0) {
    if (acc_ins) atomicAdd((unsigned long long *)&ctl->n_inserted, (unsigned long long)acc_ins);
    if (acc_del) atomicAdd((unsigned long long *)&ctl->n_deleted, (unsigned long long)acc_del);
    if (acc_ins != acc_del)  // logical key count (pending inserts included), two's complement
      atomicAdd((unsigned long long *)&ctl->total, (unsigned long long)(acc_ins - acc_del));
    if (acc_m0) atomicAdd(&ctl->n_merged0, acc_m0);
    if (acc_esc) atomicAdd(&ctl->nesc, acc_esc);
  }
}

__global__ void k_leaf_pass(Geo g, Ctl *ctl, Work w, uint32_t per_warp, int rest_only) {
  leaf_pass_body(GridIdx{}, g, ctl, w, per_warp, rest_only);
}

// ---- level 0 for runs longer than kLongRun (bulk loads) -----------------------------------------
// Phase A, a warp per 32 consecutive keys: the presence filter against the
// leaf's valid keys, deletes made EMPTY in place (distinct slots), surviving
// inserts marked pending and counted per run; the first L surviving inserts of
// a run are recorded (a run can only settle at level 0 with fewer than L).
// Phase B, a warp per long run: with the run's counts, the level-0 test, and the
// merge of the recorded inserts when it passes.
__device__ __forceinline__ uint32_t run_of(const uint32_t *run_start, uint32_t nruns, uint32_t e) {
  uint32_t lo = 0, hi = nruns;  // last run starting at or before e
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (run_start[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// the leaf's valid keys compacted into vkeys (with their slot offsets); returns how many
__device__ __forceinline__ uint32_t load_leaf(const uint64_t *leaf, uint32_t L, uint64_t *vkeys, uint16_t *vpos) {
  const uint32_t lane = lane_id();
  uint32_t nv = 0;
  for (uint32_t b = 0; b < L; b += 32) {
    const uint32_t o = b + lane;
    const uint64_t k = o < L ? leaf[o] : kEmpty;
    const bool v = k != kEmpty;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, v);
    if (v) {
      vkeys[nv + __popc(bal & lanemask_lt())] = k;
      if (vpos) vpos[nv + __popc(bal & lanemask_lt())] = (uint16_t)o;
    }
    nv += __popc(bal);
  }
  __syncwarp();
  return nv;
}

template <class Blk>
__device__ __forceinline__ void long_a_body(const Blk &bk, const Geo &g, Ctl *ctl, const Work &w, uint32_t per_warp) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (ctl->err || ctl->nvlong == 0) return;
  const uint32_t L = g.L, lane = lane_id(), wpb = blockDim.x >> 5;
  WarpBufs B = warp_bufs(smem, per_warp, L);
  const uint32_t m = ctl->m, nruns = ctl->nruns;
  for (uint32_t c = (bk.x() * wpb + (threadIdx.x >> 5)) * 32; c < m; c += bk.n() * wpb * 32) {
    // the keys [c, c+32) span at most two runs: the run of the first key, then the next
    const uint32_t r0 = run_of(w.run_start, nruns, c);
    for (uint32_t r = r0; r < nruns && w.run_start[r] < c + 32 && w.run_start[r] < m; r++) {
      const uint32_t rs = w.run_start[r], re = w.run_start[r + 1];
      if (re - rs <= kLongRun) continue;
      const uint32_t j = w.rleaf[r];
      uint64_t *leaf = g.slots + (uint64_t)j * L;
      const uint32_t nv = load_leaf(leaf, L, B.a, B.pos);
      const uint32_t e = c + lane;
      const bool act = e >= rs && e < re && e < m;
      const uint64_t key = act ? w.ukey[e] : 0ull;
      const uint32_t tag = act ? (uint32_t)w.utag[e] : 0u;
      const uint32_t idx = act ? lower_bound_dev(B.a, nv, key) : 0u;
      const bool found = act && idx < nv && B.a[idx] == key;
      const bool dl = act && tag && found, sv = act && !tag && !found;
      if (dl) leaf[B.pos[idx]] = kEmpty;
      if (act) w.eflag[e] = dl ? 1 : (sv ? 2 : 0);
      const uint32_t svb = __ballot_sync(0xFFFFFFFFu, sv), dlb = __ballot_sync(0xFFFFFFFFu, dl);
      uint32_t base = 0;
      if (lane == 0 && svb) base = (uint32_t)atomicAdd(&w.rdelta[r], (int32_t)__popc(svb));
      if (lane == 0 && dlb) atomicAdd(&w.rdel[r], __popc(dlb));
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      const uint32_t slot = base + __popc(svb & lanemask_lt());
      if (sv && slot < L) {  // record (a level-0 merge takes fewer than L; the run has more than L keys)
        w.pkey[rs + slot] = key;
        w.pleaf[rs + slot] = e;
      }
      __syncwarp();
    }
  }
}

__global__ void k_long_a(Geo g, Ctl *ctl, Work w, uint32_t per_warp) { long_a_body(GridIdx{}, g, ctl, w, per_warp); }

template <class Blk>
__device__ __forceinline__ void long_b_body(const Blk &bk, const Geo &g, Ctl *ctl, const Work &w, uint32_t per_warp) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (ctl->err || ctl->nvlong == 0) return;
  const uint32_t L = g.L, lane = lane_id(), wpb = blockDim.x >> 5;
  WarpBufs B = warp_bufs(smem, per_warp, L);
  uint64_t *vkeys = B.a, *ins = B.b, *out = B.out;
  const uint32_t nruns = ctl->nruns;
  uint64_t acc_ins = 0, acc_del = 0;
  uint32_t acc_m0 = 0, acc_esc = 0;
  for (uint32_t r = bk.x() * wpb + (threadIdx.x >> 5); r < nruns; r += bk.n() * wpb) {
    const uint32_t rs = w.run_start[r], re = w.run_start[r + 1];
    if (re - rs <= kLongRun) continue;
    const uint32_t j = w.rleaf[r];
    uint64_t *leaf = g.slots + (uint64_t)j * L;
    const uint32_t nins = (uint32_t)w.rdelta[r], ndel = w.rdel[r];
    const uint32_t nv = load_leaf(leaf, L, vkeys, nullptr);  // deletes already EMPTY
    const bool fits = nins < L && leaf_fits(g, (uint64_t)nv + nins, nins);
    if (fits) {
      // the recorded inserts, sorted by rank (distinct keys), merged with the kept keys
      for (uint32_t t = lane; t < nins; t += 32) {
        const uint64_t k = w.pkey[rs + t];
        uint32_t rk = 0;
        for (uint32_t u = 0; u < nins; u++) rk += w.pkey[rs + u] < k;
        ins[rk] = k;
        w.eflag[w.pleaf[rs + t]] = 1;
      }
      __syncwarp();
      for (uint32_t a = lane; a < nv; a += 32) out[a + lower_bound_dev(ins, nins, vkeys[a])] = vkeys[a];
      for (uint32_t b = lane; b < nins; b += 32) out[b + lower_bound_dev(vkeys, nv, ins[b])] = ins[b];
      __syncwarp();
      const uint32_t n = nv + nins;
      for (uint32_t o = lane; o < L; o += 32) {
        const uint64_t k = o < n ? out[o] : kEmpty;
        leaf[o] = k;
        if (!g.raw && o < n && is_guard(k)) g.row_end[k >> 32] = (uint32_t)((uint64_t)j * L + o);
      }
      if (lane == 0) {
        g.F[j] = n ? out[0] : kEmpty;
        g.cnt[j] = n;
      }
    } else if (lane == 0) {
      g.F[j] = nv ? vkeys[0] : kEmpty;
      g.cnt[j] = nv;
    }
    if (lane == 0) {
      w.rdelta[r] = (int32_t)nins - (int32_t)ndel;
      w.rinfo[r] = fits ? 1 : ((nins || g.dual) ? 2 : 0);
      acc_ins += nins;
      acc_del += ndel;
      acc_m0 += fits;
      acc_esc += !fits && (nins || g.dual);
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (acc_ins) atomicAdd((unsigned long long *)&ctl->n_inserted, (unsigned long long)acc_ins);
    if (acc_del) atomicAdd((unsigned long long *)&ctl->n_deleted, (unsigned long long)acc_del);
    if (acc_ins != acc_del)
      atomicAdd((unsigned long long *)&ctl->total, (unsigned long long)(acc_ins - acc_del));
    if (acc_m0) atomicAdd(&ctl->n_merged0, acc_m0);
    if (acc_esc) atomicAdd(&ctl->nesc, acc_esc);
  }
}

__global__ void k_long_b(Geo g, Ctl *ctl, Work w, uint32_t per_warp) { long_b_body(GridIdx{}, g, ctl, w, per_warp); }

// ---- level 0, fast path for 64-slot leaves and runs of at most 32 updates ---------------------
// Lane l holds slots 2l and 2l+1 of the leaf in registers (one 16-byte load),
// lane i < len holds update i of the run; presence, deletes and ranks are warp
// ballots.  The next run's leaf is loaded before the current one is processed.
// 4 blocks of 256 threads an SM (64 registers)
template <class Blk>
__device__ __forceinline__ void leaf64_body(const Blk &bk, const Geo &g, Ctl *ctl, const Work &w) {
  __shared__ uint64_t sout[8][64];
  if (ctl->err) return;
  const uint32_t lane = lane_id(), wib = threadIdx.x >> 5;
  const uint32_t nruns = ctl->nruns;
  const uint32_t nw = bk.n() * 8;
  ulonglong2 *s2 = reinterpret_cast<ulonglong2 *>(g.slots);
  uint64_t acc_ins = 0, acc_del = 0;
  uint32_t acc_m0 = 0, acc_esc = 0, acc_long = 0;
  uint32_t r = bk.x() * 8 + wib;
  // a run's leaf and updates are loaded one run ahead, its leaf index and bounds two
  // runs ahead, so that no load of an iteration waits on another
  uint32_t jn = 0, rsn = 0, ren = 0, jm = 0, rsm = 0, rem = 0, tagn = 0;
  uint64_t keyn = 0;
  ulonglong2 kn = make_ulonglong2(kEmpty, kEmpty);
  if (r < nruns) {
    jn = w.rleaf[r];
    rsn = w.run_start[r];
    ren = w.run_start[r + 1];
    kn = __ldcg(s2 + (uint64_t)jn * 32 + lane);
    if (lane < ren - rsn) {
      keyn = w.ukey[rsn + lane];
      tagn = w.utag[rsn + lane];
    }
  }
  if (r + nw < nruns) {
    jm = w.rleaf[r + nw];
    rsm = w.run_start[r + nw];
    rem = w.run_start[r + nw + 1];
  }
  for (; r < nruns; r += nw) {
    const uint32_t j = jn, rs = rsn, re = ren;
    const uint64_t k0 = kn.x, k1 = kn.y;
    const uint64_t ukey = keyn;  // update `lane` of the run (lanes below its length)
    const uint32_t utag = tagn;
    const uint32_t rn = r + nw;
    if (rn < nruns) {  // the next run's leaf (a different leaf: runs are distinct) and updates
      jn = jm;
      rsn = rsm;
      ren = rem;
      kn = __ldcg(s2 + (uint64_t)jn * 32 + lane);
      keyn = 0;
      tagn = 0;
      if (lane < ren - rsn) {
        keyn = w.ukey[rsn + lane];
        tagn = w.utag[rsn + lane];
      }
      if (rn + nw < nruns) {
        jm = w.rleaf[rn + nw];
        rsm = w.run_start[rn + nw];
        rem = w.run_start[rn + nw + 1];
      }
    }
    const uint32_t len = re - rs;
    if (len > 32) {
      acc_long++;
      continue;
    }
    if (len == 1 && !g.dual) {
      // one update (most runs of a large batch over a large array): every lane
      // reads it, no loop over the run; the same result as the general case below
      const uint64_t ku = __shfl_sync(0xFFFFFFFFu, ukey, 0);
      const bool del = __shfl_sync(0xFFFFFFFFu, utag, 0) != 0;
      const bool m0 = k0 == ku, m1 = k1 == ku;
      const bool found = __any_sync(0xFFFFFFFFu, m0 || m1);
      const bool d0 = del && m0, d1 = del && m1;
      const bool kp0 = k0 != kEmpty && !d0, kp1 = k1 != kEmpty && !d1;
      const uint32_t kb0 = __ballot_sync(0xFFFFFFFFu, kp0), kb1 = __ballot_sync(0xFFFFFFFFu, kp1);
      const uint32_t nkept = __popc(kb0) + __popc(kb1);
      const uint32_t nins = (!del && !found) ? 1u : 0u, ndel = (del && found) ? 1u : 0u;
      const bool fits = nins && nkept + 1 <= g.maxc[0];
      if (fits) {
        // TryInsert+ at level 0: the kept keys and the insert, left-packed
        const uint32_t lt_mask = lanemask_lt();
        const uint32_t before = __popc(kb0 & lt_mask) + __popc(kb1 & lt_mask);
        const uint32_t pk = __popc(__ballot_sync(0xFFFFFFFFu, kp0 && k0 < ku)) +
                            __popc(__ballot_sync(0xFFFFFFFFu, kp1 && k1 < ku));
        if (kp0) sout[wib][before + (ku < k0)] = k0;
        if (kp1) sout[wib][before + kp0 + (ku < k1)] = k1;
        if (lane == 0) sout[wib][pk] = ku;
        __syncwarp();
        const uint32_t n = nkept + 1;
        const uint32_t o = 2 * lane;
        const uint64_t a = o < n ? sout[wib][o] : kEmpty, b = o + 1 < n ? sout[wib][o + 1] : kEmpty;
        s2[(uint64_t)j * 32 + lane] = make_ulonglong2(a, b);
        if (!g.raw) {
          if (o < n && is_guard(a)) g.row_end[a >> 32] = j * 64u + o;
          if (o + 1 < n && is_guard(b)) g.row_end[b >> 32] = j * 64u + o + 1;
        }
        if (lane == 0) {
          g.F[j] = sout[wib][0];
          g.cnt[j] = n;
        }
        __syncwarp();
      } else if (ndel) {
        if (d0 || d1) s2[(uint64_t)j * 32 + lane] = make_ulonglong2(d0 ? kEmpty : k0, d1 ? kEmpty : k1);
        const uint32_t fb = kb0 | kb1;
        const uint32_t fl = fb ? __ffs(fb) - 1 : 0;
        const uint64_t fk = __shfl_sync(0xFFFFFFFFu, ((kb0 >> fl) & 1u) ? k0 : k1, fl);
        if (lane == 0) {
          g.F[j] = fb ? fk : kEmpty;
          g.cnt[j] = nkept;
        }
      }
      if (lane == 0) {
        w.eflag[rs] = ndel ? 1 : (nins ? (fits ? 1 : 2) : 0);
        w.rdelta[r] = (int32_t)nins - (int32_t)ndel;
        w.rinfo[r] = fits ? 1 : (nins ? 2 : 0);
        w.rdel[r] = ndel;
      }
      acc_ins += nins;
      acc_del += ndel;
      acc_m0 += fits;
      acc_esc += !fits && nins;
      continue;
    }
    const bool act = lane < len;
    const uint64_t key = act ? ukey : 0ull;
    const uint32_t tag = act ? utag : 0u;
    const bool v0 = k0 != kEmpty, v1 = k1 != kEmpty;
    const uint32_t tbal = __ballot_sync(0xFFFFFFFFu, tag != 0);  // deletes of the run
    bool d0 = false, d1 = false;
    uint32_t fbal = 0;  // run keys present in the leaf
    for (uint32_t i = 0; i < len; i++) {
      const uint64_t ki = __shfl_sync(0xFFFFFFFFu, key, i);
      const bool m0 = k0 == ki, m1 = k1 == ki;
      if (__ballot_sync(0xFFFFFFFFu, m0 || m1)) fbal |= 1u << i;
      if ((tbal >> i) & 1u) {
        d0 |= m0;
        d1 |= m1;
      }
    }
    const bool found = (fbal >> lane) & 1u;
    const bool sv = act && !tag && !found;  // surviving insert (sorted in lane order)
    const uint32_t svbal = __ballot_sync(0xFFFFFFFFu, sv);
    const uint32_t nins = __popc(svbal);
    const uint32_t ndel = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)d0 + (uint32_t)d1);
    const bool kp0 = v0 && !d0, kp1 = v1 && !d1;
    const uint32_t kb0 = __ballot_sync(0xFFFFFFFFu, kp0), kb1 = __ballot_sync(0xFFFFFFFFu, kp1);
    const uint32_t nkept = __popc(kb0) + __popc(kb1);
    const bool fits = leaf_fits(g, (uint64_t)nkept + nins, nins);
    if (fits) {
      // TryInsert+ at level 0: rank-merge kept keys with the surviving inserts
      const uint32_t lt_mask = lanemask_lt();
      const uint32_t before = __popc(kb0 & lt_mask) + __popc(kb1 & lt_mask);
      uint32_t lt0 = 0, lt1 = 0, my_pos = 0;
      for (uint32_t bits = svbal; bits; bits &= bits - 1) {
        const uint32_t b = __ffs(bits) - 1;
        const uint64_t ik = __shfl_sync(0xFFFFFFFFu, key, b);
        lt0 += ik < k0;
        lt1 += ik < k1;
        const uint32_t below = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)(kp0 && k0 < ik) + (uint32_t)(kp1 && k1 < ik));
        if (lane == b) my_pos = __popc(svbal & lt_mask) + below;
      }
      if (kp0) sout[wib][before + lt0] = k0;
      if (kp1) sout[wib][before + kp0 + lt1] = k1;
      if (sv) sout[wib][my_pos] = key;
      __syncwarp();
      const uint32_t n = nkept + nins;
      const uint32_t o = 2 * lane;
      const uint64_t a = o < n ? sout[wib][o] : kEmpty, b = o + 1 < n ? sout[wib][o + 1] : kEmpty;
      s2[(uint64_t)j * 32 + lane] = make_ulonglong2(a, b);
      if (!g.raw) {
        if (o < n && is_guard(a)) g.row_end[a >> 32] = j * 64u + o;
        if (o + 1 < n && is_guard(b)) g.row_end[b >> 32] = j * 64u + o + 1;
      }
      if (lane == 0) {
        g.F[j] = n ? sout[wib][0] : kEmpty;
        g.cnt[j] = n;
      }
      __syncwarp();
    } else {
      if (d0 || d1) s2[(uint64_t)j * 32 + lane] = make_ulonglong2(d0 ? kEmpty : k0, d1 ? kEmpty : k1);
      const uint32_t fb = __ballot_sync(0xFFFFFFFFu, kp0 || kp1);
      const uint32_t fl = fb ? __ffs(fb) - 1 : 0;
      const uint64_t fk = __shfl_sync(0xFFFFFFFFu, kp0 ? k0 : k1, fl);
      if (lane == 0) {
        g.F[j] = fb ? fk : kEmpty;
        g.cnt[j] = nkept;
      }
    }
    const bool dl = act && tag && found;
    if (act) w.eflag[rs + lane] = dl ? 1 : (sv ? (fits ? 1 : 2) : 0);
    if (lane == 0) {
      w.rdelta[r] = (int32_t)nins - (int32_t)ndel;
      w.rinfo[r] = fits ? 1 : ((nins || g.dual) ? 2 : 0);
      w.rdel[r] = ndel;
    }
    acc_ins += nins;
    acc_del += ndel;
    acc_m0 += fits;
    acc_esc += !fits && (nins || g.dual);
  }
  if (lane == 0) {
    if (acc_ins) atomicAdd((unsigned long long *)&ctl->n_inserted, (unsigned long long)acc_ins);
    if (acc_del) atomicAdd((unsigned long long *)&ctl->n_deleted, (unsigned long long)acc_del);
    if (acc_ins != acc_del)  // logical key count (pending inserts included), two's complement
      atomicAdd((unsigned long long *)&ctl->total, (unsigned long long)(acc_ins - acc_del));
    if (acc_m0) atomicAdd(&ctl->n_merged0, acc_m0);
    if (acc_esc) atomicAdd(&ctl->nesc, acc_esc);
    if (acc_long) atomicAdd(&ctl->nlong, acc_long);
  }
}

__global__ void __launch_bounds__(256, 4) k_leaf64(Geo g, Ctl *ctl, Work w) { leaf64_body(GridIdx{}, g, ctl, w); }

// ---- count tree, rebuilt only when some inserts did not fit their leaf ----------------------
// Levels 1..h of the tree hold logical counts for the merge-level test: valid
// keys of every segment plus the inserts still pending in this batch.  Stage A:
// one block per 4096 leaves builds the levels inside its range in shared memory;
// stage B: one block builds the levels above from the block sums; then every
// pending run adds its inserts to its ancestors.
constexpr uint32_t kTreeSpan = 4096;

__global__ void __launch_bounds__(1024) k_tree_a(Geo g, Ctl *ctl) {
  __shared__ uint32_t sv[kTreeSpan];
  if (ctl->err || ctl->nesc == 0) return;
  const uint64_t span = g.nleaves < kTreeSpan ? g.nleaves : kTreeSpan;
  const uint64_t base = (uint64_t)blockIdx.x * span;
  for (uint32_t t = threadIdx.x; t < span; t += blockDim.x) sv[t] = g.cnt[base + t];
  __syncthreads();
  uint32_t i = 1;
  for (uint64_t nodes = span >> 1; nodes >= 1 && i <= g.h; nodes >>= 1, ++i) {
    uint32_t v[4];
    uint32_t k = 0;
    for (uint32_t t = threadIdx.x; t < nodes; t += blockDim.x) v[k++] = sv[2 * t] + sv[2 * t + 1];
    __syncthreads();
    k = 0;
    for (uint32_t t = threadIdx.x; t < nodes; t += blockDim.x) {
      sv[t] = v[k];
      g.tree[g.tree_off[i] + (base >> i) + t] = v[k];
      ++k;
    }
    __syncthreads();
  }
}

// levels above the blocks' span, one level at a time through global memory
__global__ void __launch_bounds__(1024) k_tree_b(Geo g, Ctl *ctl) {
  if (ctl->err || ctl->nesc == 0) return;
  uint32_t first = 0;  // first level above a block's span
  while ((1ull << first) < kTreeSpan && first < g.h) ++first;
  for (uint32_t i = first + 1; i <= g.h; i++) {
    const uint64_t nodes = g.nleaves >> i;
    for (uint64_t t = threadIdx.x; t < nodes; t += blockDim.x)
      g.tree[g.tree_off[i] + t] = g.tree[g.tree_off[i - 1] + 2 * t] + g.tree[g.tree_off[i - 1] + 2 * t + 1];
    __syncthreads();
  }
}

__global__ void k_tree_pend(Geo g, Ctl *ctl, Work w) {
  if (ctl->err) return;
  const uint32_t ner = ctl->neruns;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < ner; r += gridDim.x * blockDim.x) {
    const uint32_t j = w.eleaf[r];
    const uint32_t c = w.erun[r + 1] - w.erun[r];
    for (uint32_t i = 1; i <= g.h; i++) atomicAdd(&g.tree[g.tree_off[i] + (j >> i)], c);
  }
}

// ---- escalation: inserts that did not fit their leaf -----------------------------------------
__global__ void __launch_bounds__(kScanThreads) k_pending(Ctl *ctl, Work w) {
  __shared__ ScanSmem sm;
  if (ctl->err || ctl->nesc == 0) return;
  const uint32_t tile = take_ticket(ctl, kSlotPend, sm), m = ctl->m;
  if ((uint64_t)tile * kScanTile >= m && tile > 0) return;
  uint32_t flag[kScanItems];
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    uint64_t e = scan_elem(tile, r);
    flag[r] = e < m && w.eflag[e] == 2;
  }
  uint32_t off[kScanItems];
  uint32_t total = tile_scan(flag, off, tile, w.status, 1, 0, ctl->epoch + kSlotPend, ctl, sm);
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    if (!flag[r] || off[r] >= m) continue;
    uint64_t e = scan_elem(tile, r);
    w.pkey[off[r]] = w.ukey[e];
    w.pleaf[off[r]] = w.uleaf[e];
  }
  if ((uint64_t)(tile + 1) * kScanTile >= m && threadIdx.x == 0) ctl->npend = total;
}

// escalated runs (leaves that did not settle at level 0), in leaf order, with the
// first of their pending inserts (those are contiguous and in the same order)
__global__ void __launch_bounds__(kScanThreads) k_eruns(Ctl *ctl, Work w) {
  __shared__ ScanSmem sm;
  if (ctl->err || ctl->nesc == 0) return;
  const uint32_t tile = take_ticket(ctl, kSlotERuns, sm), nr = ctl->nruns;
  if ((uint64_t)tile * kScanTile >= nr && tile > 0) return;
  uint32_t flag[kScanItems], pc[kScanItems];
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    const uint64_t q = scan_elem(tile, r);
    flag[r] = q < nr && w.rinfo[q] == 2;
    pc[r] = flag[r] ? (uint32_t)(w.rdelta[q] + (int32_t)w.rdel[q]) : 0u;  // its surviving inserts
  }
  uint32_t off[kScanItems], poff[kScanItems];
  const uint32_t total = tile_scan(flag, off, tile, w.status, 2, 0, ctl->epoch + kSlotERuns, ctl, sm);
  const uint32_t ptotal = tile_scan(pc, poff, tile, w.status, 2, 1, ctl->epoch + kSlotERuns, ctl, sm);
#pragma unroll
  for (int r = 0; r < kScanItems; r++)
    if (flag[r] && off[r] < nr) {
      w.erun[off[r]] = poff[r];
      w.eleaf[off[r]] = w.rleaf[scan_elem(tile, r)];
    }
  if ((uint64_t)(tile + 1) * kScanTile >= nr && threadIdx.x == 0) {
    ctl->neruns = total;
    w.erun[total] = ptotal;
  }
}

// merge level of every pending run: the lowest level whose segment passes the test.
// With may_fail set, a run that no level admits is counted in nfail (root resize).
__global__ void k_esc_level(Geo g, Ctl *ctl, Work w, int resize) {  // resize = may_fail
  if (ctl->err) return;
  const uint32_t ner = ctl->neruns;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < ner; r += gridDim.x * blockDim.x) {
    const uint32_t j = w.eleaf[r];
    uint32_t lvl = kNoLevel;
    for (uint32_t i = 1; i <= g.h; i++) {
      if (level_admits(g, i, g.tree[g.tree_off[i] + (j >> i)])) {
        lvl = i;
        break;
      }
    }
    w.elvl[r] = (uint8_t)lvl;
    if (lvl != kNoLevel) {
      uint32_t old = atomicExch(&g.mark[g.tree_off[lvl] + (j >> lvl)], 1u);
      if (!old) atomicAdd((unsigned long long *)&ctl->merges[lvl], 1ull);
      atomicMax(&ctl->levels_climbed, lvl);
    } else if (resize) {
      atomicAdd(&ctl->nfail, 1u);
    } else {
      atomicOr(&ctl->err, kErrInternal);
    }
  }
}

// outermost merged segment above every pending run
__global__ void k_esc_top(Geo g, Ctl *ctl, Work w) {
  if (ctl->err) return;
  const uint32_t ner = ctl->neruns;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < ner; r += gridDim.x * blockDim.x) {
    const uint32_t lvl = w.elvl[r];
    const uint32_t j = w.eleaf[r];
    uint32_t top = lvl;
    for (uint32_t i = lvl + 1; i <= g.h; i++)
      if (g.mark[g.tree_off[i] + (j >> i)]) top = i;
    w.etop[r] = (uint8_t)top;
  }
}

__global__ void k_unmark(Geo g, Ctl *ctl, Work w) {
  const uint32_t ner = ctl->neruns;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < ner; r += gridDim.x * blockDim.x) {
    const uint32_t lvl = w.elvl[r];
    if (lvl == kNoLevel) continue;
    g.mark[g.tree_off[lvl] + (w.eleaf[r] >> lvl)] = 0;
  }
}

// runs sharing an outermost segment are consecutive: one entry per segment, with
// its first pending insert and the prefix of covered leaves; clears the marks
__global__ void __launch_bounds__(kScanThreads) k_segs(Geo g, Ctl *ctl, Work w) {
  __shared__ ScanSmem sm;
  if (ctl->err || ctl->neruns == 0) return;
  const uint32_t tile = take_ticket(ctl, kSlotSegs, sm), ner = ctl->neruns;
  if ((uint64_t)tile * kScanTile >= ner && tile > 0) return;
  uint32_t flag[kScanItems], lv[kScanItems];
  uint32_t top[kScanItems], node[kScanItems];
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    uint64_t q = scan_elem(tile, r);
    flag[r] = 0;
    lv[r] = 0;
    top[r] = 0;
    node[r] = 0;
    if (q < ner) {
      top[r] = w.etop[q];
      node[r] = w.eleaf[q] >> top[r];
      if (q == 0) {
        flag[r] = 1;
      } else {
        uint32_t pt = w.etop[q - 1];
        uint32_t pn = w.eleaf[q - 1] >> pt;
        flag[r] = (pt != top[r]) || (pn != node[r]);
      }
      lv[r] = flag[r] ? (1u << top[r]) : 0u;
    }
  }
  uint32_t off[kScanItems], loff[kScanItems];
  uint32_t total = tile_scan(flag, off, tile, w.status, 2, 0, ctl->epoch + kSlotSegs, ctl, sm);
  uint32_t ltotal = tile_scan(lv, loff, tile, w.status, 2, 1, ctl->epoch + kSlotSegs, ctl, sm);
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    uint64_t q = scan_elem(tile, r);
    if (q >= ner) continue;
    const uint32_t lvl = w.elvl[q];
    g.mark[g.tree_off[lvl] + (w.eleaf[q] >> lvl)] = 0;
    if (!flag[r] || off[r] >= ner) continue;
    w.seg_top[off[r]] = (uint8_t)top[r];
    w.seg_node[off[r]] = node[r];
    w.seg_pstart[off[r]] = w.erun[q];
    w.seg_lpre[off[r]] = loff[r];
  }
  if ((uint64_t)(tile + 1) * kScanTile >= ner && threadIdx.x == 0) {
    ctl->nsegs = total;
    ctl->nleafw = ltotal;
    w.seg_pstart[total] = ctl->npend;
    w.seg_lpre[total] = ltotal;
  }
}

// ---- merge of segments: gather, merge path, even re-dispatch ---------------------------------
struct SegArgs {
  int whole;            // 1: the whole source array into a new array (root resize)
  uint32_t whole_top;   // height of the new array
  uint64_t src_nleaves; // leaves of the source array (whole mode)
};

__device__ __forceinline__ uint32_t seg_of(const uint32_t *lpre, uint32_t nsegs, uint32_t wl) {
  uint32_t lo = 0, hi = nsegs;  // last k with lpre[k] <= wl
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (lpre[mid] <= wl) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_seg_vcnt(Geo src, Ctl *ctl, Work w, uint32_t *vcnt) {
  if (ctl->err) return;
  const uint32_t nsegs = ctl->nsegs, nlw = ctl->nleafw;
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < nlw; x += gridDim.x * blockDim.x) {
    uint32_t k = seg_of(w.seg_lpre, nsegs, x);
    uint32_t top = w.seg_top[k];
    uint64_t leaf = ((uint64_t)w.seg_node[k] << top) + (x - w.seg_lpre[k]);
    vcnt[x] = src.cnt[leaf];
  }
}

// one warp per source leaf: its valid keys go to scratch[voff[x] ...] in order
__global__ void k_seg_gather(Geo src, Ctl *ctl, Work w, SegArgs sa, const uint64_t *voff, uint64_t *scratch,
                             uint64_t scratch_cap) {
  if (ctl->err) return;
  const uint32_t lane = lane_id(), L = src.L;
  const uint64_t nlw = sa.whole ? sa.src_nleaves : ctl->nleafw;
  const uint32_t nsegs = ctl->nsegs;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t x = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); x < nlw; x += nw) {
    uint64_t leaf = x;
    if (!sa.whole) {
      uint32_t k = seg_of(w.seg_lpre, nsegs, (uint32_t)x);
      leaf = ((uint64_t)w.seg_node[k] << w.seg_top[k]) + (x - w.seg_lpre[k]);
    }
    const uint64_t *p = src.slots + leaf * L;
    uint64_t o = voff[x];
    for (uint32_t b = 0; b < L; b += 32) {
      uint64_t k = (b + lane < L) ? p[b + lane] : kEmpty;
      bool v = k != kEmpty;
      uint32_t bal = __ballot_sync(0xFFFFFFFFu, v);
      const uint64_t at = o + __popc(bal & lanemask_lt());
      if (v && at < scratch_cap) scratch[at] = k;
      o += __popc(bal);
    }
  }
}

// number of A elements among the first r of merge(A, B) (keys distinct)
__device__ __forceinline__ uint64_t co_rank(const uint64_t *A, uint64_t na, const uint64_t *B, uint64_t nb,
                                            uint64_t r) {
  uint64_t lo = r > nb ? r - nb : 0, hi = r < na ? r : na;
  while (lo < hi) {
    uint64_t i = (lo + hi) >> 1;
    if (A[i] < B[r - i - 1]) lo = i + 1; else hi = i;
  }
  return lo;
}

struct SegGeom {
  uint64_t dleaf;     // destination leaf
  uint64_t t, top;    // leaf index inside the segment, segment height
  uint64_t abase, na; // valid keys of the segment in scratch
  uint64_t bbase, nb; // pending inserts of the segment
};

__device__ __forceinline__ SegGeom seg_geom(const Work &w, SegArgs sa, const uint64_t *voff, Ctl *ctl,
                                            uint64_t x) {
  SegGeom s;
  if (sa.whole) {
    s.dleaf = x;
    s.t = x;
    s.top = sa.whole_top;
    s.abase = 0;
    s.na = voff[sa.src_nleaves];
    s.bbase = 0;
    s.nb = ctl->npend;
  } else {
    uint32_t k = seg_of(w.seg_lpre, ctl->nsegs, (uint32_t)x);
    s.top = w.seg_top[k];
    s.t = x - w.seg_lpre[k];
    s.dleaf = ((uint64_t)w.seg_node[k] << s.top) + s.t;
    s.abase = voff[w.seg_lpre[k]];
    s.na = voff[w.seg_lpre[k + 1]] - s.abase;
    s.bbase = w.seg_pstart[k];
    s.nb = w.seg_pstart[k + 1] - s.bbase;
  }
  return s;
}

// one warp per destination leaf: its share [n t / m, n (t+1) / m) of the merged keys
__global__ void k_seg_write(Geo dst, Ctl *ctl, Work w, SegArgs sa, const uint64_t *voff,
                            const uint64_t *scratch, uint32_t per_warp) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (ctl->err) return;
  const uint32_t lane = lane_id(), L = dst.L;
  WarpBufs Bf = warp_bufs(smem, per_warp, L);
  uint64_t *sa_ = Bf.a, *sb_ = Bf.b, *out = Bf.out;
  const uint64_t nlw = sa.whole ? dst.nleaves : ctl->nleafw;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t x = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); x < nlw; x += nw) {
    const SegGeom s = seg_geom(w, sa, voff, ctl, x);
    const uint64_t n = s.na + s.nb;
    const uint64_t a = (n * s.t) >> s.top, b = (n * (s.t + 1)) >> s.top;
    if (b - a > L) {  // cannot happen when the counts are consistent
      if (lane == 0) atomicOr(&ctl->err, kErrInternal);
      break;
    }
    const uint64_t *A = scratch + s.abase, *Bk = w.pkey + s.bbase;
    uint64_t i0 = 0, i1 = 0;
    if (lane == 0) {
      i0 = co_rank(A, s.na, Bk, s.nb, a);
      i1 = co_rank(A, s.na, Bk, s.nb, b);
    }
    i0 = __shfl_sync(0xFFFFFFFFu, i0, 0);
    i1 = __shfl_sync(0xFFFFFFFFu, i1, 0);
    const uint32_t na = (uint32_t)(i1 - i0), nb = (uint32_t)((b - a) - na);
    const uint64_t j0 = a - i0;
    for (uint32_t q = lane; q < na; q += 32) sa_[q] = A[i0 + q];
    for (uint32_t q = lane; q < nb; q += 32) sb_[q] = Bk[j0 + q];
    __syncwarp();
    for (uint32_t q = lane; q < na; q += 32) out[q + lower_bound_dev(sb_, nb, sa_[q])] = sa_[q];
    for (uint32_t q = lane; q < nb; q += 32) out[q + lower_bound_dev(sa_, na, sb_[q])] = sb_[q];
    __syncwarp();
    const uint32_t cntl = na + nb;
    uint64_t *leaf = dst.slots + s.dleaf * L;
    for (uint32_t o = lane; o < L; o += 32) {
      uint64_t k = o < cntl ? out[o] : kEmpty;
      leaf[o] = k;
      if (!dst.raw && o < cntl && is_guard(k)) dst.row_end[k >> 32] = (uint32_t)(s.dleaf * L + o);
    }
    if (lane == 0) {
      dst.cnt[s.dleaf] = cntl;
      dst.F[s.dleaf] = cntl ? out[0] : kEmpty;
    }
    __syncwarp();
  }
}

// ---- statistics (only when the caller asks for them) -------------------------------------------
__global__ void k_stats(Ctl *ctl, Work w) {
  const uint32_t nruns = ctl->nruns, nsegs = ctl->nsegs;
  uint64_t cov = 0, emp = 0, l0 = 0, dl = 0;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nruns; r += gridDim.x * blockDim.x) {
    dl += w.rdel[r] != 0;
    const uint32_t leaf = w.rleaf[r], info = w.rinfo[r];
    bool in = false;
    if (nsegs) {
      uint32_t lo = 0, hi = nsegs;  // last segment starting at or before leaf
      while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (((uint64_t)w.seg_node[mid] << w.seg_top[mid]) <= leaf) lo = mid; else hi = mid;
      }
      uint64_t st = (uint64_t)w.seg_node[lo] << w.seg_top[lo];
      in = leaf >= st && leaf < st + (1ull << w.seg_top[lo]);
    }
    const bool covered = info == 1 || in;
    cov += covered;
    emp += covered ? 0 : w.rdel[r];
    l0 += (info == 1 && !in);
  }
  cov = warp_sum(cov);
  emp = warp_sum(emp);
  l0 = warp_sum(l0);
  dl = warp_sum(dl);
  if (lane_id() == 0) {
    if (dl) atomicAdd((unsigned long long *)&ctl->st_del_leaves, (unsigned long long)dl);
    if (cov) atomicAdd((unsigned long long *)&ctl->st_cov_touched, (unsigned long long)cov);
    if (emp) atomicAdd((unsigned long long *)&ctl->st_empties, (unsigned long long)emp);
    if (l0) atomicAdd((unsigned long long *)&ctl->st_l0_only, (unsigned long long)l0);
  }
}

// ---- host launchers ------------------------------------------------------------------------------
static uint32_t blocks_for(uint64_t items, uint32_t per_block, uint32_t cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (uint32_t)b;
}

// warps per block of the one-warp-per-leaf kernels: as many as fit 96 KB of
// shared memory, at most 8, or `want` (a tuned choice) when that fits
static uint32_t warps_per_block(uint32_t L, uint32_t want = 0) {
  uint32_t pw = leaf_smem_bytes(L);
  uint32_t wpb = (96u * 1024u) / pw;
  if (wpb > 8) wpb = 8;
  if (wpb < 1) wpb = 1;
  if (want && want < wpb) wpb = want;
  return wpb;
}
uint32_t leaf_pass_warps(uint32_t L, uint32_t want) { return warps_per_block(L, want); }

void allow_big_smem() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_leaf_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_seg_write, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_long_a, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_long_b, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  done = true;
}

// Out-degree change of the batch, one key per thread after the level-0 passes
// (every surviving insert ends up stored, pending ones by the merges of this
// batch; guards are not edges): lanes of one source (keys are sorted, so they
// are adjacent) add once.
template <class Blk>
__device__ __forceinline__ void deg_batch_body(const Blk &bk, const Geo &g, const Ctl *ctl, const Work &w) {
  if (ctl->err) return;
  const uint32_t m = ctl->m;
  for (uint32_t b = bk.x() * blockDim.x; b < m; b += bk.n() * blockDim.x) {
    const uint32_t e = b + threadIdx.x;
    int d = 0;
    uint64_t key = 0;
    if (e < m) {
      key = w.ukey[e];
      const uint8_t f = w.eflag[e];
      if (w.utag[e]) d = f == 1 ? -1 : 0;
      else d = (f != 0 && !is_guard(key)) ? 1 : 0;
    }
    const uint32_t src = d ? (uint32_t)(key >> 32) : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, src);
    const uint32_t pos = __ballot_sync(0xFFFFFFFFu, d > 0), neg = __ballot_sync(0xFFFFFFFFu, d < 0);
    const int sum = __popc(peers & pos) - __popc(peers & neg);
    if (d && lane_id() == (uint32_t)(__ffs(peers) - 1) && sum) atomicAdd(&g.deg[src], (uint32_t)sum);
  }
}

__global__ void __launch_bounds__(256) k_deg_batch(Geo g, const Ctl *ctl, Work w) {
  deg_batch_body(GridIdx{}, g, ctl, w);
}

void launch_leaf64(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s) {
  note_launch();
  k_leaf64<<<blocks_for(n, 8, 152 * 4), 256, 0, s>>>(g, ctl, w);  // one wave of resident blocks
}

void launch_leaf_rest(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, bool rest_only, cudaStream_t s) {
  allow_big_smem();
  const uint32_t pw = leaf_smem_bytes(g.L), wpb = warps_per_block(g.L, g.leaf_warps);
  note_launch();
  k_leaf_pass<<<blocks_for(n, wpb, 152 * 16), wpb * 32, wpb * pw, s>>>(g, ctl, w, pw, rest_only ? 1 : 0);
  if (n > kLongRun) {  // only a batch this large can hold a run this long
    note_launch();
    k_long_a<<<blocks_for((n + 31) / 32, wpb, 152 * 16), wpb * 32, wpb * pw, s>>>(g, ctl, w, pw);
    note_launch();
    k_long_b<<<blocks_for(n / kLongRun + 1, wpb, 152 * 16), wpb * 32, wpb * pw, s>>>(g, ctl, w, pw);
  }
}

void launch_degrees_batch(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s) {
  if (g.raw) return;
  note_launch();
  k_deg_batch<<<blocks_for(n, 256, 152 * 8), 256, 0, s>>>(g, ctl, w);
}

void launch_leaf_pass(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s) {
  const bool fast = g.L == 64;
  if (fast) launch_leaf64(g, ctl, w, n, s);
  launch_leaf_rest(g, ctl, w, n, fast, s);
  launch_degrees_batch(g, ctl, w, n, s);
}

// ---- many handles: the level-0 stages as one launch over all of them ---------------------------
__global__ void __launch_bounds__(256, 4) k_m_leaf64(const ManyDesc *d, uint32_t plan) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb)) return;
  leaf64_body(SubIdx{sub, nb}, it->g, it->ctl, it->w);
}

__global__ void k_m_leaf_pass(const ManyDesc *d, uint32_t plan) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb)) return;
  leaf_pass_body(SubIdx{sub, nb}, it->g, it->ctl, it->w, it->per_warp, it->g.L == 64 ? 1 : 0);
}

__global__ void k_m_long_a(const ManyDesc *d, uint32_t plan) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb)) return;
  long_a_body(SubIdx{sub, nb}, it->g, it->ctl, it->w, it->per_warp);
}

__global__ void k_m_long_b(const ManyDesc *d, uint32_t plan) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb)) return;
  long_b_body(SubIdx{sub, nb}, it->g, it->ctl, it->w, it->per_warp);
}

__global__ void __launch_bounds__(256) k_m_deg_batch(const ManyDesc *d, uint32_t plan) {
  const ManyItem *it;
  uint32_t sub, nb;
  if (!many_block(d, plan, &it, &sub, &nb)) return;
  deg_batch_body(SubIdx{sub, nb}, it->g, it->ctl, it->w);
}

void prepare_many_leaf() {
  cudaFuncSetAttribute(k_m_leaf_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_m_long_a, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_m_long_b, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void launch_many_leaf(const ManyDesc *d, const ManyPlans &pl, cudaStream_t s) {
  if (pl.total[pl.leaf64]) {
    note_launch();
    k_m_leaf64<<<pl.total[pl.leaf64], 256, 0, s>>>(d, pl.leaf64);
  }
  for (uint32_t k = 0; k < pl.ngroups; k++) {
    const ManyPlans::Group &gr = pl.group[k];
    const uint32_t smem = gr.wpb * gr.per_warp;
    note_launch();
    k_m_leaf_pass<<<pl.total[gr.rest], gr.wpb * 32, smem, s>>>(d, gr.rest);
    if (gr.long_a != ~0u) {
      note_launch();
      k_m_long_a<<<pl.total[gr.long_a], gr.wpb * 32, smem, s>>>(d, gr.long_a);
      note_launch();
      k_m_long_b<<<pl.total[gr.long_b], gr.wpb * 32, smem, s>>>(d, gr.long_b);
    }
  }
  if (pl.total[pl.deg]) {
    note_launch();
    k_m_deg_batch<<<pl.total[pl.deg], 256, 0, s>>>(d, pl.deg);
  }
}

void launch_tree_rebuild(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s) {
  if (g.h == 0) return;
  const uint64_t span = g.nleaves < kTreeSpan ? g.nleaves : kTreeSpan;
  note_launch();
  k_tree_a<<<(uint32_t)(g.nleaves / span), 1024, 0, s>>>(g, ctl);
  if ((1ull << g.h) > kTreeSpan) {
    note_launch();
    k_tree_b<<<1, 1024, 0, s>>>(g, ctl);
  }
  note_launch();
  k_tree_pend<<<blocks_for(n, 256, 152 * 8), 256, 0, s>>>(g, ctl, w);
}

void launch_pending(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s) {
  (void)g;
  const uint32_t ct = comp_tiles(n);
  note_launch();
  k_pending<<<ct, kScanThreads, 0, s>>>(ctl, w);
  note_launch();
  k_eruns<<<ct, kScanThreads, 0, s>>>(ctl, w);
}

void launch_esc_level(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, bool may_fail, cudaStream_t s) {
  note_launch();
  k_esc_level<<<blocks_for(n, 256, 152 * 8), 256, 0, s>>>(g, ctl, w, may_fail ? 1 : 0);
}

void launch_esc_top(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s) {
  note_launch();
  k_esc_top<<<blocks_for(n, 256, 152 * 8), 256, 0, s>>>(g, ctl, w);
}

void launch_unmark(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s) {
  note_launch();
  k_unmark<<<blocks_for(n, 256, 152 * 8), 256, 0, s>>>(g, ctl, w);
}

void launch_segments(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s) {
  note_launch();
  k_segs<<<comp_tiles(n), kScanThreads, 0, s>>>(g, ctl, w);
}

void launch_stats(const Geo &g, Ctl *ctl, const Work &w, uint32_t n, cudaStream_t s) {
  (void)g;
  note_launch();
  k_stats<<<blocks_for(n, 256, 152 * 8), 256, 0, s>>>(ctl, w);
}

void launch_segment_merge(const Geo &src, const Geo &dst, Ctl *ctl, const Work &w, uint64_t scratch_cap,
                          uint64_t nleafw_bound, uint64_t *scratch, uint32_t *voff_u32tmp, uint64_t *partials,
                          bool whole, cudaStream_t s) {
  allow_big_smem();
  SegArgs sa;
  sa.whole = whole ? 1 : 0;
  sa.whole_top = dst.h;
  sa.src_nleaves = src.nleaves;
  // voff (u64, nleafw + 1 entries) lives right after the u32 counts in the same buffer
  uint32_t *vcnt = voff_u32tmp;
  uint64_t *voff = (uint64_t *)(((uintptr_t)(vcnt + nleafw_bound + 1) + 15) & ~(uintptr_t)15);
  const uint32_t *cnt_in = vcnt;
  if (whole) {
    cnt_in = src.cnt;
  } else {
    note_launch();
    k_seg_vcnt<<<blocks_for(nleafw_bound, 256, 152 * 8), 256, 0, s>>>(src, ctl, w, vcnt);
  }
  launch_scan_u32_u64(cnt_in, voff, whole ? src.nleaves : nleafw_bound, partials, s,
                      whole ? nullptr : &ctl->nleafw);
  note_launch();
  k_seg_gather<<<blocks_for(nleafw_bound, 8, 152 * 16), 256, 0, s>>>(src, ctl, w, sa, voff, scratch, scratch_cap);
  const uint32_t pw = leaf_smem_bytes(dst.L), wpb = warps_per_block(dst.L);
  const uint64_t dst_bound = whole ? dst.nleaves : nleafw_bound;
  note_launch();
  k_seg_write<<<blocks_for(dst_bound, wpb, 152 * 16), wpb * 32, wpb * pw, s>>>(dst, ctl, w, sa, voff, scratch, pw);
}

}  // namespace gpk
