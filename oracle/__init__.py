"""CPU oracle of GPMA+ (Sha, Li, He, Tan, "Accelerating Dynamic Graph Analytics on GPUs").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_1709_05061_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``gpma_oracle.c`` (plain single-threaded C following the
paper's steps in order); this module only compiles it with gcc and marshals
numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
RAW_KEYS = 1
DUAL_DELETE = 2
MAX_LEVELS = 48


def build(force: bool = False) -> str:
    """Compile gpma_oracle.c into _build/liboracle.so (plain -O2, no vector flags)."""
    src = os.path.join(_HERE, "gpma_oracle.c")
    hdr = os.path.join(_HERE, "gpma_oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall",
                           "-o", tmp, src])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Stats(C.Structure):
    _fields_ = [
        ("n_inserted", C.c_uint64), ("n_deleted", C.c_uint64), ("n_ignored", C.c_uint64),
        ("levels_climbed", C.c_uint32), ("resized", C.c_uint32),
        ("alg_bytes", C.c_uint64), ("touched_leaves", C.c_uint64),
        ("covered_leaves", C.c_uint64), ("merges", C.c_uint64 * MAX_LEVELS),
        ("delete_leaves", C.c_uint64),
    ]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "merges"}
        d["merges"] = list(self.merges)
        return d


def lib():
    global _lib
    if _lib is None:
        build()
        l = C.CDLL(_LIB_PATH)
        u32, u64, vp = C.c_uint32, C.c_uint64, C.c_void_p
        l.or_thresholds.argtypes = [u32, u32, u32, u32, u32, u32, vp, vp]
        l.or_create.argtypes = [u32, u32, u32, u32, u32, u32, u32]
        l.or_create.restype = vp
        l.or_destroy.argtypes = [vp]
        l.or_update.argtypes = [vp, vp, u64, vp, u64, C.POINTER(Stats)]
        l.or_update.restype = C.c_int
        l.or_capacity.argtypes = [vp]; l.or_capacity.restype = u64
        l.or_height.argtypes = [vp]; l.or_height.restype = u32
        l.or_num_valid.argtypes = [vp]; l.or_num_valid.restype = u64
        l.or_layout.argtypes = [vp, vp]
        l.or_import_layout.argtypes = [vp, vp, u64]; l.or_import_layout.restype = C.c_int
        l.or_export_sorted.argtypes = [vp, vp]; l.or_export_sorted.restype = u64
        l.or_export_csr.argtypes = [vp, vp, vp]; l.or_export_csr.restype = u64
        l.or_row_end.argtypes = [vp, vp]
        l.or_bfs.argtypes = [vp, u32, vp]; l.or_bfs.restype = C.c_int
        l.or_cc.argtypes = [vp, vp]; l.or_cc.restype = C.c_int
        l.or_pagerank.argtypes = [vp, u32, C.c_double, vp]; l.or_pagerank.restype = C.c_int
        l.or_check_invariants.argtypes = [vp]; l.or_check_invariants.restype = C.c_int
        l.or_bfs_edges.argtypes = [u32, vp, u64, u32, vp]; l.or_bfs_edges.restype = C.c_int
        l.or_cc_edges.argtypes = [u32, vp, u64, vp]; l.or_cc_edges.restype = C.c_int
        l.or_pagerank_edges.argtypes = [u32, vp, u64, u32, C.c_double, vp]
        l.or_pagerank_edges.restype = C.c_int
        _lib = l
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def thresholds(L: int, h: int, tau0=92, tauh=80, rho0=8, rhoh=40):
    """Per-level (max, min) entry counts for a tree of height h (reading T)."""
    mx = np.zeros(h + 1, np.uint64)
    mn = np.zeros(h + 1, np.uint64)
    lib().or_thresholds(L, h, tau0, tauh, rho0, rhoh, _ptr(mx), _ptr(mn))
    return mx, mn


def _edges(keys) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(keys, dtype=np.uint64))


def bfs_edges(n_vertices: int, keys, src: int) -> np.ndarray:
    """BFS depths over a plain edge list (src << 32 | dst, any order)."""
    k = _edges(keys)
    out = np.empty(n_vertices, np.int32)
    rc = lib().or_bfs_edges(n_vertices, _ptr(k), k.size, src, _ptr(out))
    if rc:
        raise ValueError(f"oracle bfs_edges rc={rc}")
    return out


def cc_edges(n_vertices: int, keys) -> np.ndarray:
    """Weakly connected component labels (smallest vertex id) of a plain edge list."""
    k = _edges(keys)
    out = np.empty(n_vertices, np.uint32)
    rc = lib().or_cc_edges(n_vertices, _ptr(k), k.size, _ptr(out))
    if rc:
        raise ValueError(f"oracle cc_edges rc={rc}")
    return out


def pagerank_edges(n_vertices: int, keys, iters: int = 20, damping: float = 0.85) -> np.ndarray:
    """FP64 PageRank (the oracle's definition) over a plain edge list."""
    k = _edges(keys)
    out = np.empty(n_vertices, np.float64)
    rc = lib().or_pagerank_edges(n_vertices, _ptr(k), k.size, iters, damping, _ptr(out))
    if rc:
        raise ValueError(f"oracle pagerank_edges rc={rc}")
    return out


class OraclePMA:
    """One packed memory array holding a dynamic graph (or raw keys)."""

    def __init__(self, n_vertices: int, L: int = 64, tau0=92, tauh=80, rho0=8, rhoh=40,
                 raw_keys: bool = False, dual: bool = False):
        self.n_vertices = int(n_vertices)
        self.L = L
        self.raw = raw_keys
        self.dual = dual
        self.params = (tau0, tauh, rho0, rhoh)
        self._p = lib().or_create(self.n_vertices, L, tau0, tauh, rho0, rhoh,
                                  (RAW_KEYS if raw_keys else 0) | (DUAL_DELETE if dual else 0))
        if not self._p:
            raise ValueError("oracle: invalid parameters")

    def __del__(self):
        p = getattr(self, "_p", None)
        if p:
            lib().or_destroy(p)
            self._p = None

    def update(self, ins, dels=None) -> tuple[int, dict]:
        ins = np.ascontiguousarray(np.asarray(ins if ins is not None else [], dtype=np.uint64))
        dels = np.ascontiguousarray(np.asarray(dels if dels is not None else [], dtype=np.uint64))
        st = Stats()
        rc = lib().or_update(self._p, _ptr(ins), ins.size, _ptr(dels), dels.size, C.byref(st))
        return rc, st.as_dict()

    @property
    def capacity(self) -> int:
        return int(lib().or_capacity(self._p))

    @property
    def height(self) -> int:
        return int(lib().or_height(self._p))

    def layout(self) -> np.ndarray:
        out = np.empty(self.capacity, np.uint64)
        lib().or_layout(self._p, _ptr(out))
        return out

    def import_layout(self, slots) -> int:
        slots = np.ascontiguousarray(np.asarray(slots, dtype=np.uint64))
        return lib().or_import_layout(self._p, _ptr(slots), slots.size)

    def export_sorted(self) -> np.ndarray:
        n = lib().or_export_sorted(self._p, None)
        out = np.empty(n, np.uint64)
        lib().or_export_sorted(self._p, _ptr(out))
        return out

    def export_csr(self):
        n = lib().or_export_sorted(self._p, None)
        rowptr = np.empty(self.n_vertices + 1, np.uint64)
        col = np.empty(max(n, 1), np.uint32)
        e = lib().or_export_csr(self._p, _ptr(rowptr), _ptr(col))
        return rowptr, col[:e]

    def row_end(self) -> np.ndarray:
        out = np.empty(self.n_vertices, np.uint32)
        lib().or_row_end(self._p, _ptr(out))
        return out

    def bfs(self, src: int) -> np.ndarray:
        out = np.empty(self.n_vertices, np.int32)
        rc = lib().or_bfs(self._p, src, _ptr(out))
        if rc:
            raise ValueError(f"oracle bfs rc={rc}")
        return out

    def cc(self) -> np.ndarray:
        out = np.empty(self.n_vertices, np.uint32)
        rc = lib().or_cc(self._p, _ptr(out))
        if rc:
            raise ValueError(f"oracle cc rc={rc}")
        return out

    def pagerank(self, iters: int = 20, damping: float = 0.85) -> np.ndarray:
        out = np.empty(self.n_vertices, np.float64)
        rc = lib().or_pagerank(self._p, iters, damping, _ptr(out))
        if rc:
            raise ValueError(f"oracle pagerank rc={rc}")
        return out

    def check_invariants(self) -> int:
        return int(lib().or_check_invariants(self._p))
