"""Test helpers: golden-fixture parsing and checks written independently of the oracle."""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
EMPTY = 0xFFFFFFFFFFFFFFFF


def read_golden(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.strip()
    return out


def ints(s: str):
    return [int(x) for x in s.split()]


def floats(s: str):
    return [float(x) for x in s.split()]


def parse_leaves(s: str, L: int) -> np.ndarray:
    """'3 . . . | 5 7 8 .' -> uint64 slots with EMPTY for '.'."""
    slots = []
    for leaf in s.split("|"):
        toks = leaf.split()
        assert len(toks) == L, (leaf, L)
        slots += [EMPTY if t == "." else int(t) for t in toks]
    return np.array(slots, dtype=np.uint64)


def leaf_bound(L: int, tau0_pct: int = 92) -> int:
    """Largest count n with n < tau_0 * L (the leaf bound of Sec. 4.1)."""
    lim = Fraction(tau0_pct, 100) * L
    n = int(lim)
    return n - 1 if n == lim else n


def check_layout(slots: np.ndarray, L: int, n_vertices: int | None = None, tau0_pct: int = 92):
    """Structural properties every layout must have: capacity L * 2^h, valid keys
    strictly increasing, every leaf within the leaf bound, one guard per vertex."""
    slots = np.asarray(slots, dtype=np.uint64)
    C = slots.size
    assert C % L == 0 and (C // L) & (C // L - 1) == 0, C
    valid = slots[slots != np.uint64(EMPTY)]
    assert np.all(valid[1:] > valid[:-1]), "valid keys not strictly increasing"
    per_leaf = (slots.reshape(-1, L) != np.uint64(EMPTY)).sum(axis=1)
    assert per_leaf.max(initial=0) <= leaf_bound(L, tau0_pct), per_leaf.max()
    if n_vertices is not None:
        guards = valid[(valid & np.uint64(0xFFFFFFFF)) == np.uint64(0xFFFFFFFF)]
        assert np.array_equal(guards >> np.uint64(32), np.arange(n_vertices, dtype=np.uint64))


def edges_of(slots: np.ndarray) -> np.ndarray:
    slots = np.asarray(slots, dtype=np.uint64)
    valid = slots[slots != np.uint64(EMPTY)]
    return valid[(valid & np.uint64(0xFFFFFFFF)) != np.uint64(0xFFFFFFFF)]


def apply_set_semantics(live: set, ins, dels) -> set:
    """Plain definition of the edge set after a batch: keys in both lists cancel,
    the other inserts are added and the other deletes removed."""
    I, D = set(int(x) for x in ins), set(int(x) for x in dels)
    X = I & D
    return (live | (I - X)) - (D - X)
