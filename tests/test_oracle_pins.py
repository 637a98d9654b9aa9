"""Pins of the CPU oracle against things other than itself: the paper's printed
examples (tests/golden/), closed forms, invariants and brute force."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from helpers import (EMPTY, apply_set_semantics, check_layout, edges_of, floats, ints,
                     parse_leaves, read_golden)


# ---- Fig. 3 threshold table -------------------------------------------------------
def test_fig3_threshold_table():
    g = read_golden("fig3_thresholds.txt")
    L, h = int(g["L"]), int(g["h"])
    mx, mn = oracle.thresholds(L, h)
    assert list(mx) == ints(g["max_entries"])
    assert list(mn) == ints(g["min_entries"])


def test_fig3_densities_follow_linear_reading():
    """The printed tau/rho rows are the linear interpolation between leaf and root."""
    g = read_golden("fig3_thresholds.txt")
    h = int(g["h"])
    tau, rho = ints(g["tau_pct"]), ints(g["rho_pct"])
    for i in range(h + 1):
        t = Fraction(tau[-1]) + Fraction(tau[0] - tau[-1]) * (h - i) / h
        r = Fraction(rho[-1]) - Fraction(rho[-1] - rho[0]) * (h - i) / h
        assert round(t) == tau[i] and round(r) == rho[i]


def test_threshold_bound_is_nested():
    """Even re-dispatch of max_i keys never overfills a child: ceil(max_i/2) <= max_{i-1}."""
    for L in (4, 32, 64, 256):
        for h in range(0, 24):
            mx, mn = oracle.thresholds(L, h)
            for i in range(1, h + 1):
                assert (int(mx[i]) + 1) // 2 <= int(mx[i - 1])
                assert int(mx[i]) < 0.92 * (L << i)


# ---- worked examples (Sec. 4.1 Ex. 1, Sec. 5.2 Ex. 3) ------------------------------
def _w_instance():
    g = read_golden("example_w.txt")
    L = int(g["L"])
    o = oracle.OraclePMA(0, L=L, raw_keys=True)
    assert o.import_layout(parse_leaves(g["initial"], L)) == 0
    assert o.height == 3
    return g, L, o


@pytest.mark.parametrize("ex", ["ex3", "ex1"])
def test_worked_examples(ex):
    g, L, o = _w_instance()
    rc, st = o.update(ints(g[f"{ex}_insert"]))
    assert rc == 0
    assert np.array_equal(o.layout(), parse_leaves(g[f"{ex}_final"], L))
    assert st["merges"][:4] == ints(g[f"{ex}_merges_per_level"])
    assert st["resized"] == 0


def test_example3_algorithmic_bytes():
    g, L, o = _w_instance()
    rc, st = o.update(ints(g["ex3_insert"]))
    # 5 raw keys * 8 B; touched leaves {0,1,4,5}: 4 * 8L; both level-2 segments are
    # rewritten: 8 leaves * 8L written + untouched leaves {2,3,6,7} read: 4 * 8L.
    assert st["alg_bytes"] == 5 * 8 + 4 * 8 * L + 8 * 8 * L + 4 * 8 * L
    assert st["touched_leaves"] == 4 and st["covered_leaves"] == 8


# ---- Fig. 5 CSR with guard entries ------------------------------------------------
@pytest.mark.parametrize("L", [2, 4, 8, 64])
def test_fig5_csr(L):
    g = read_golden("fig5_csr.txt")
    V = int(g["n_vertices"])
    rp, col = ints(g["row_offset"]), ints(g["column_index"])
    edges = [(u << 32) | col[e] for u in range(V) for e in range(rp[u], rp[u + 1])]
    o = oracle.OraclePMA(V, L=L)
    rng = np.random.default_rng(L)
    rc, _ = o.update(rng.permutation(np.array(edges, np.uint64)))
    assert rc == 0
    rowptr, c = o.export_csr()
    assert list(rowptr) == rp and list(c) == col
    check_layout(o.layout(), L, V)
    # the guard of u sits right after row u
    re = o.row_end()
    lay = o.layout()
    for u in range(V):
        assert lay[re[u]] == np.uint64((u << 32) | 0xFFFFFFFF)


# ---- brute force against the set definition ----------------------------------------
def _random_batch(rng, V, live, n):
    live_l = list(live)
    ins = list(rng.integers(0, V, (n, 2)))
    ins = [(int(a) << 32) | int(b) for a, b in ins]
    if live_l:
        ins += [live_l[i] for i in rng.integers(0, len(live_l), n // 4)]  # already present
    ins += ins[: n // 8]  # duplicates
    dels = []
    if live_l:
        dels += [live_l[i] for i in rng.integers(0, len(live_l), n)]
    dels += [(int(a) << 32) | int(b) for a, b in rng.integers(0, V, (n // 4, 2))]  # mostly absent
    dels += ins[: n // 8]  # cancelling pairs
    return (rng.permutation(np.array(ins, np.uint64)) if ins else np.zeros(0, np.uint64),
            rng.permutation(np.array(dels, np.uint64)) if dels else np.zeros(0, np.uint64))


@pytest.mark.parametrize("V,L,seed", [(40, 4, 0), (200, 8, 1), (300, 64, 2), (1000, 16, 3)])
def test_bruteforce_stream(V, L, seed):
    rng = np.random.default_rng(seed)
    o = oracle.OraclePMA(V, L=L)
    live = set()
    for it in range(30):
        n = int(rng.integers(0, 3 * V if it % 7 else 8 * V))
        ins, dels = _random_batch(rng, V, live, n)
        before = o.layout()
        rc, st = o.update(ins, dels)
        assert rc == 0
        new_live = apply_set_semantics(live, ins, dels)
        got = edges_of(o.layout())
        assert np.array_equal(got, np.array(sorted(new_live), np.uint64))
        assert st["n_inserted"] == len(new_live - live)
        assert st["n_deleted"] == len(live - new_live)
        assert st["n_ignored"] == ins.size + dels.size - st["n_inserted"] - st["n_deleted"]
        check_layout(o.layout(), L, V)
        assert o.check_invariants() == 0
        if st["resized"]:
            assert o.capacity > before.size
        live = new_live


def test_rejects_bad_ids_and_changes_nothing():
    o = oracle.OraclePMA(10, L=4)
    o.update([(1 << 32) | 2, (3 << 32) | 4])
    before = o.layout()
    for bad in ([(10 << 32) | 1], [(1 << 32) | 10], [(1 << 32) | 0xFFFFFFFF]):
        rc, _ = o.update([(2 << 32) | 3] + bad)
        assert rc == 1
        assert np.array_equal(o.layout(), before)
    rc, _ = o.update([], [(1 << 32) | 0xFFFFFFFF])  # a guard cannot be deleted
    assert rc == 1 and np.array_equal(o.layout(), before)


def test_cancel_before_presence():
    """A key in both lists is a no-op even when it is stored (cancellation precedes
    the presence filter)."""
    o = oracle.OraclePMA(8, L=4)
    k = (1 << 32) | 2
    o.update([k])
    rc, st = o.update([k], [k])
    assert rc == 0 and k in set(int(x) for x in edges_of(o.layout()))
    assert st["n_ignored"] == 2 and st["n_inserted"] == 0 and st["n_deleted"] == 0


def test_lazy_delete_is_in_place():
    """Sec. 6.1: deletion only marks the slot; nothing else moves."""
    rng = np.random.default_rng(5)
    o = oracle.OraclePMA(300, L=16)
    o.update(np.unique(rng.integers(0, 300, 3000) * (1 << 32) + rng.integers(0, 300, 3000)).astype(np.uint64))
    before = o.layout()
    e = edges_of(before)
    d = rng.choice(e, 200, replace=False)
    rc, st = o.update([], d)
    after = o.layout()
    changed = np.nonzero(before != after)[0]
    assert set(before[changed].tolist()) == set(int(x) for x in d)
    assert np.all(after[changed] == np.uint64(EMPTY))
    assert st["merges"][0] == 0 and st["resized"] == 0
    # the leaves holding a delete, counted from the slots that changed
    assert st["delete_leaves"] == len(set((changed // 16).tolist()))


def test_bulk_load_closed_form():
    """Loading n sorted keys into an empty array takes the smallest height whose root
    bound holds n, and spreads rank r into leaf t = floor(n t/m)..floor(n(t+1)/m)."""
    for L, n in [(8, 1), (8, 1000), (4, 37), (64, 5000)]:
        o = oracle.OraclePMA(0, L=L, raw_keys=True)
        keys = np.arange(1, n + 1, dtype=np.uint64) * np.uint64(3)
        rc, st = o.update(keys[::-1])
        assert rc == 0
        h = o.height
        assert int(oracle.thresholds(L, h)[0][h]) >= n
        assert h == 0 or int(oracle.thresholds(L, h - 1)[0][h - 1]) < n or h == 1
        m = o.capacity // L
        lay = o.layout().reshape(m, L)
        for t in range(m):
            a, b = n * t // m, n * (t + 1) // m
            assert list(lay[t, : b - a]) == list(keys[a:b])
            assert np.all(lay[t, b - a:] == np.uint64(EMPTY))


def test_single_insert_with_room_touches_one_leaf():
    o = oracle.OraclePMA(0, L=8, raw_keys=True)
    o.update(np.arange(10, 400, 10, dtype=np.uint64))
    before = o.layout()
    rc, st = o.update([155])
    after = o.layout()
    diff_leaves = np.nonzero((before != after).reshape(-1, 8).any(axis=1))[0]
    assert len(diff_leaves) == 1 and st["merges"][0] == 1
    leaf = after.reshape(-1, 8)[diff_leaves[0]]
    vals = leaf[leaf != np.uint64(EMPTY)]
    assert np.all(vals[1:] > vals[:-1]) and 155 in vals.tolist()
    assert np.all(leaf[: vals.size] != np.uint64(EMPTY))  # left-packed


# ---- analytics ----------------------------------------------------------------------
def _graph(V, edges, L=8):
    o = oracle.OraclePMA(V, L=L)
    rc, _ = o.update(np.array([(u << 32) | v for u, v in edges], np.uint64))
    assert rc == 0
    return o


def test_bfs_closed_forms():
    V = 12
    path = _graph(V, [(i, i + 1) for i in range(V - 1)])
    assert list(path.bfs(0)) == list(range(V))
    assert list(path.bfs(5)) == [-1] * 5 + list(range(V - 5))
    star = _graph(V, [(0, i) for i in range(1, V)] + [(3, 3)])
    assert list(star.bfs(0)) == [0] + [1] * (V - 1)


def test_cc_closed_forms():
    cliques = [(a, b) for base in (0, 4, 9) for a in range(base, base + 3) for b in range(base, base + 3) if a != b]
    o = _graph(13, cliques)
    lab = o.cc()
    exp = [0, 0, 0, 3, 4, 4, 4, 7, 8, 9, 9, 9, 12]
    assert list(lab) == exp


def test_analytics_vs_networkx():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(11)
    for V, E in [(60, 90), (300, 1200), (500, 400)]:
        ed = set()
        while len(ed) < E:
            u, v = (int(x) for x in rng.integers(0, V, 2))
            ed.add((u, v))
        o = _graph(V, sorted(ed), L=16)
        G = nx.DiGraph()
        G.add_nodes_from(range(V))
        G.add_edges_from(ed)
        for s in (0, V // 2):
            d = nx.single_source_shortest_path_length(G, s)
            exp = [d.get(v, -1) for v in range(V)]
            assert list(o.bfs(s)) == exp
        lab = o.cc()
        for comp in nx.weakly_connected_components(G):
            m = min(comp)
            assert all(lab[v] == m for v in comp)
        x = o.pagerank(iters=300)
        pr = nx.pagerank(G, alpha=0.85, tol=1e-15, max_iter=10000)
        assert np.allclose(x, [pr[v] for v in range(V)], rtol=1e-9, atol=0)
        assert abs(o.pagerank(iters=7).sum() - 1.0) < 1e-12
        # the edge-list forms (for graphs too large for the oracle's PMA), fed the
        # edges in a shuffled order, against networkx directly
        el = rng.permutation(np.array([(u << 32) | v for u, v in ed], np.uint64))
        for s in (0, V // 2):
            d = nx.single_source_shortest_path_length(G, s)
            assert list(oracle.bfs_edges(V, el, s)) == [d.get(v, -1) for v in range(V)]
        lab_e = oracle.cc_edges(V, el)
        for comp in nx.weakly_connected_components(G):
            assert all(lab_e[v] == min(comp) for v in comp)
        assert np.allclose(oracle.pagerank_edges(V, el, 300), [pr[v] for v in range(V)], rtol=1e-9, atol=0)


def test_edge_list_analytics_reject_out_of_range_ids():
    with pytest.raises(ValueError):
        oracle.bfs_edges(4, np.array([(1 << 32) | 4], np.uint64), 0)
    with pytest.raises(ValueError):
        oracle.cc_edges(4, np.array([(4 << 32) | 1], np.uint64))
    with pytest.raises(ValueError):
        oracle.pagerank_edges(4, np.array([(0 << 32) | 9], np.uint64), 3)


def test_pagerank_two_vertex_hand_computed():
    g = read_golden("pagerank_two_vertex.txt")
    o = _graph(2, [(0, 1)], L=4)
    assert np.allclose(o.pagerank(1), floats(g["iters_1"]), rtol=0, atol=1e-15)
    assert np.allclose(o.pagerank(2), floats(g["iters_2"]), rtol=0, atol=1e-15)


def test_pagerank_cycle_uniform_and_eigenvector():
    V = 9
    o = _graph(V, [(i, (i + 1) % V) for i in range(V)])
    assert np.allclose(o.pagerank(13), 1.0 / V, rtol=0, atol=1e-15)
    # random graph: the fixed point is the Perron vector of the Google matrix
    rng = np.random.default_rng(3)
    V = 40
    ed = {(int(a), int(b)) for a, b in rng.integers(0, V, (120, 2))}
    o = _graph(V, sorted(ed))
    A = np.zeros((V, V))
    for u, v in ed:
        A[v, u] += 1.0
    deg = A.sum(axis=0)
    M = np.where(deg > 0, A / np.where(deg > 0, deg, 1), 1.0 / V)
    G = 0.85 * M + 0.15 / V
    w, vecs = np.linalg.eig(G)
    pv = np.real(vecs[:, np.argmax(np.real(w))])
    pv /= pv.sum()
    assert np.allclose(o.pagerank(400), pv, rtol=1e-9)


# ---- dual deletion (reading D): hand-computed cases, set semantics, bounds ------------
@pytest.mark.parametrize("case", ["d1", "d2", "d3", "d4"])
def test_dual_worked_examples(case):
    g = read_golden("dual_w.txt")
    L = int(g["L"])
    o = oracle.OraclePMA(0, L=L, raw_keys=True, dual=True)
    assert o.import_layout(parse_leaves(g["initial"], L)) == 0
    rc, st = o.update(ints(g[f"{case}_insert"]), ints(g[f"{case}_delete"]))
    assert rc == 0
    assert o.capacity == int(g[f"{case}_capacity"])
    assert np.array_equal(o.layout(), parse_leaves(g[f"{case}_final"], L))
    assert st["merges"][:4] == ints(g[f"{case}_merges_per_level"])
    assert st["resized"] == (2 if o.capacity < 32 else 0)
    assert o.check_invariants() == 0


def test_dual_lazy_differs_only_in_layout():
    """The same deletes in lazy mode leave holes and keep the capacity (R5)."""
    g = read_golden("dual_w.txt")
    L = int(g["L"])
    o = oracle.OraclePMA(0, L=L, raw_keys=True)
    o.import_layout(parse_leaves(g["initial"], L))
    o.update([], ints(g["d3_delete"]))
    assert o.capacity == 32 and sorted(edges_of(o.layout()).tolist()) == [3, 5, 7]


def _leaf_counts(lay, L):
    return (lay.reshape(-1, L) != EMPTY).sum(axis=1)


@pytest.mark.parametrize("V,L,seed", [(60, 4, 10), (300, 8, 11), (2000, 64, 12), (800, 16, 13)])
def test_dual_bruteforce_stream_and_bounds(V, L, seed):
    """Set semantics; no holes; leaves written by a batch hold at least the even-split
    lower bound min_i / 2^i (some level i >= 1) once the root holds min_h; the capacity
    shrinks to the smallest height whose root bound holds the keys."""
    rng = np.random.default_rng(seed)
    o = oracle.OraclePMA(V, L=L, dual=True)
    live = set()
    for it in range(40):
        grow = it < 15 or it % 9 == 0
        n = int(rng.integers(1, 3 * V))
        ins, dels = _random_batch(rng, V, live, n)
        if not grow:  # mostly deletes: shrink the graph
            ins = ins[: ins.size // 8]
            dels = np.concatenate([dels, np.array(list(live), np.uint64)[: len(live) // 2]])
        before = o.layout()
        rc, st = o.update(ins, dels)
        assert rc == 0
        new_live = apply_set_semantics(live, ins, dels)
        lay = o.layout()
        assert np.array_equal(edges_of(lay), np.array(sorted(new_live), np.uint64))
        check_layout(lay, L, V)
        assert o.check_invariants() == 0
        h, total = o.height, len(new_live) + V
        mx, mn = oracle.thresholds(L, h)
        if h > 0 and total >= mn[h]:
            lmin = min(int(mn[i]) // (1 << i) for i in range(1, h + 1))
            cnt = _leaf_counts(lay, L)
            changed = np.ones(cnt.size, bool) if lay.size != before.size else \
                (lay.reshape(-1, L) != before.reshape(-1, L)).any(axis=1)
            assert np.all(cnt[changed] >= lmin), (it, lmin, cnt[changed].min())
        # the array is never taller than needed while the root is underfull
        if h > 0 and total < mn[h]:
            mx1, _ = oracle.thresholds(L, h - 1)
            assert total > mx1[h - 1]
        if st["resized"] == 2:
            assert o.capacity < before.size
        live = new_live


# ---- negative pins of the invariant checker -----------------------------------------
def _broken(o, mutate, **kw):
    """A copy of o's layout with one property broken, imported into a fresh oracle
    of the same parameters (import does no checking of its own)."""
    lay = o.layout().copy()
    mutate(lay)
    b = oracle.OraclePMA(o.n_vertices, L=o.L, dual=o.dual, **kw)
    assert b.import_layout(lay) == 0
    return b


@pytest.mark.parametrize("dual", [False, True])
def test_check_invariants_flags_each_broken_property(dual):
    """The checker returns 0 on a valid layout and the code of the property that a
    hand-made layout breaks: 1 keys not strictly increasing, 2 a leaf above max_0,
    5 a hole inside a leaf (dual deletion only; lazy deletion leaves holes by
    design).  Raw keys 100, 200, ... leave room for keys in between."""
    L = 8
    E = np.uint64(EMPTY)
    o = oracle.OraclePMA(0, L=L, raw_keys=True, dual=dual)
    assert o.update(np.arange(1, 61, dtype=np.uint64) * np.uint64(100))[0] == 0
    assert o.check_invariants() == 0
    lay = o.layout()
    valid = np.nonzero(lay != E)[0]
    max0 = int(oracle.thresholds(L, o.height)[0][0])
    assert max0 == 7

    def swap_two_keys(a):
        i, j = valid[3], valid[4]
        a[i], a[j] = a[j], a[i]
    assert _broken(o, swap_two_keys, raw_keys=True).check_invariants() == 1

    def duplicate_key(a):
        a[valid[4]] = a[valid[3]]
    assert _broken(o, duplicate_key, raw_keys=True).check_invariants() == 1

    def overfill_leaf(a):
        # leaf 1 gets max_0 + 1 keys, all between the keys of leaves 0 and 2
        lo = max(int(x) for x in a[:L] if x != E)
        a[L:2 * L] = np.arange(lo + 1, lo + 1 + L, dtype=np.uint64)
    assert _broken(o, overfill_leaf, raw_keys=True).check_invariants() == 2

    def hole(a):  # the first slot of a leaf holding two keys or more becomes EMPTY
        per = (a.reshape(-1, L) != E).sum(axis=1)
        j = int(np.nonzero(per >= 2)[0][0])
        a[j * L] = E
    assert _broken(o, hole, raw_keys=True).check_invariants() == (5 if dual else 0)
    # code 3 (capacity not L * 2^h) cannot be imported: the import refuses it
    assert oracle.OraclePMA(0, L=L, raw_keys=True, dual=dual).import_layout(lay[:3 * L]) != 0


def test_check_invariants_flags_bad_vertices_and_guards():
    """Graph mode adds code 4: a vertex id >= V, or not exactly one guard per vertex."""
    V, L = 16, 8
    E = np.uint64(EMPTY)
    o = oracle.OraclePMA(V, L=L)
    edges = [(u << 32) | ((u + 1) % V) for u in range(V)] + [(u << 32) | ((u + 5) % V) for u in range(V)]
    assert o.update(np.array(edges, np.uint64))[0] == 0
    assert o.check_invariants() == 0
    lay = o.layout()
    guard_slots = [i for i in np.nonzero(lay != E)[0] if (int(lay[i]) & 0xFFFFFFFF) == 0xFFFFFFFF]
    assert len(guard_slots) == V

    def dst_out_of_range(a):  # the last edge of row V-1 gets dst = V (still below the guard)
        i = guard_slots[-1] - 1
        while a[i] == E:
            i -= 1
        a[i] = np.uint64(((V - 1) << 32) | V)
    assert _broken(o, dst_out_of_range).check_invariants() == 4

    def drop_a_guard(a):
        a[guard_slots[V // 2]] = E
    assert _broken(o, drop_a_guard).check_invariants() == 4
