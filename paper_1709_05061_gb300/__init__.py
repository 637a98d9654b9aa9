"""GPMA+ dynamic graph store on one GB300 GPU -- thin Python binding of libgpma.

Every function below has the name of the C entry point it calls (include/gpma.h)
and only marshals arguments: device tensors (torch, CUDA) are passed by pointer,
the current torch stream is passed as the cudaStream_t, and status codes become
``GpmaError``.  All work runs in the library's kernels.  There is no fallback:
if ``libgpma.so`` has not been built, ``lib()`` raises.

Keys are 64-bit ``(src << 32) | dst``; torch tensors of dtype int64 or uint64
are accepted (int64 is read as the same bits).
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build_mod

GPMA_OK, GPMA_EINVAL, GPMA_ENOMEM, GPMA_ECAP, GPMA_ETIMEOUT, GPMA_EDEVICE = range(6)
GPMA_RAW_KEYS = 1
GPMA_PLAIN_SEARCH = 2
GPMA_DUAL_DELETE = 4
GPMA_PUSH_PAGERANK = 8
GPMA_MAX_LEVELS = 48
EMPTY = 0xFFFFFFFFFFFFFFFF

_lib = None


class GpmaError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().gpma_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (status {code})")


class gpma_params(C.Structure):
    _fields_ = [("leaf_size", C.c_uint32), ("tau0_pct", C.c_uint32), ("tauh_pct", C.c_uint32),
                ("rho0_pct", C.c_uint32), ("rhoh_pct", C.c_uint32), ("flags", C.c_uint32),
                ("leaf_warps", C.c_uint32)]


class gpma_stats(C.Structure):
    _fields_ = [
        ("n_inserted", C.c_uint64), ("n_deleted", C.c_uint64), ("n_ignored", C.c_uint64),
        ("levels_climbed", C.c_uint32), ("resized", C.c_uint32), ("alg_bytes", C.c_uint64),
        ("touched_leaves", C.c_uint64), ("covered_leaves", C.c_uint64),
        ("merges", C.c_uint64 * GPMA_MAX_LEVELS), ("delete_leaves", C.c_uint64),
        ("model_sorted", C.c_uint32), ("pad", C.c_uint32),
    ]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "merges"}
        d["merges"] = list(self.merges)
        return d


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class gpma_allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", C.c_void_p)]


class Allocator:
    """Device memory of a handle from two Python callables (the ``gpma_allocator``
    of include/gpma.h): ``alloc(nbytes, stream) -> int`` returns a device pointer,
    0 on failure; ``free(ptr, stream)`` releases one.  ``stream`` is the call's
    cudaStream_t as an int (0 = the legacy default stream).  Keep the object alive
    as long as the handle (``Graph`` does)."""

    def __init__(self, alloc, free):
        def _a(nbytes, stream, ctx):
            try:
                return int(alloc(int(nbytes), int(stream or 0)) or 0) or None
            except Exception:  # an exception must not cross the C ABI: report a failed allocation
                return None

        def _f(ptr, stream, ctx):
            try:
                free(int(ptr or 0), int(stream or 0))
            except Exception:
                pass

        self._cb = (_ALLOC_FN(_a), _FREE_FN(_f))
        self.struct = gpma_allocator(self._cb[0], self._cb[1], None)


def torch_allocator() -> Allocator:
    """An Allocator over torch's caching allocator (library memory then shows up
    in torch's memory statistics and is reused from its pool)."""
    torch = _torch()

    def alloc(nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(nbytes, stream=stream)
        except RuntimeError:  # torch's out-of-memory error
            return 0

    def free(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    return Allocator(alloc, free)


GPMA_PROF_NAMES = ("sort", "leaf", "escalate", "resize", "pr_scatter", "pagerank", "bfs", "cc", "update",
                   "pr_bucket")
GPMA_PROF_N = len(GPMA_PROF_NAMES)


class gpma_profile(C.Structure):
    _fields_ = [("ms", C.c_double * GPMA_PROF_N), ("count", C.c_uint64 * GPMA_PROF_N),
                ("launches", C.c_uint64 * GPMA_PROF_N)]

    def as_dict(self) -> dict:
        return {n: {"ms": self.ms[i], "count": self.count[i], "launches": self.launches[i]}
                for i, n in enumerate(GPMA_PROF_NAMES)}


def build(force: bool = False, verbose: bool = False) -> str:
    return _build_mod.build(force=force, verbose=verbose)


def lib_path() -> str:
    return _build_mod.LIB


def lib():
    """Load libgpma.so (built in-tree).  Raises when it is missing."""
    global _lib
    if _lib is None:
        path = _build_mod.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libgpma.so is not built ({path}); run paper_1709_05061_gb300.build()")
        l = C.CDLL(path)
        vp, u32, u64, i = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
        P = C.POINTER
        sig = {
            "gpma_create": ([u32, P(gpma_params), P(gpma_allocator), vp, P(vp)], i),
            "gpma_destroy": ([vp], i),
            "gpma_update_batch": ([vp, vp, u64, vp, u64, vp, P(gpma_stats)], i),
            "gpma_status": ([vp, vp], i),
            "gpma_update_many": ([P(vp), P(vp), P(u64), P(vp), P(u64), u32, vp], i),
            "gpma_bfs": ([vp, u32, vp, vp], i),
            "gpma_cc": ([vp, vp, vp], i),
            "gpma_pagerank": ([vp, u32, C.c_float, vp, vp], i),
            "gpma_pagerank_snapshot": ([vp, vp], i),
            "gpma_pagerank_run": ([vp, u32, C.c_float, vp, vp], i),
            "gpma_export_sorted": ([vp, vp, u64, P(u64), vp], i),
            "gpma_export_sorted_noalloc": ([vp, vp, u64, P(u64), vp], i),
            "gpma_export_csr": ([vp, vp, vp, u64, P(u64), vp], i),
            "gpma_export_layout": ([vp, vp, u64, P(u64), vp], i),
            "gpma_import_layout": ([vp, vp, u64, vp], i),
            "gpma_row_end": ([vp, vp, vp], i),
            "gpma_num_edges": ([vp, P(u64), vp], i),
            "gpma_capacity": ([vp, P(u64)], i),
            "gpma_check": ([vp, P(u32), vp], i),
            "gpma_strerror": ([i], C.c_char_p),
            "gpma_profile_enable": ([vp, i], i),
            "gpma_profile_read": ([vp, P(gpma_profile), i], i),
            "gpma_launch_count": ([], u64),
            "gpma_set_wait_limit": ([vp, u32, vp], i),
        }
        for name, (args, res) in sig.items():
            f = getattr(l, name)
            f.argtypes = args
            f.restype = res
        _lib = l
    return _lib


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def _keys(t):
    torch = _torch()
    if t is None:
        return torch.empty(0, dtype=torch.int64, device="cuda")
    if not t.is_cuda or t.dtype not in (torch.int64, torch.uint64) or not t.is_contiguous():
        raise ValueError("keys must be a contiguous CUDA int64/uint64 tensor")
    return t


def _check(rc: int, where: str):
    if rc != GPMA_OK:
        raise GpmaError(rc, where)


# ---- the C entry points, one to one --------------------------------------------------------
def gpma_create(n_vertices: int, leaf_size: int = 64, tau0: int = 92, tauh: int = 80, rho0: int = 8,
                rhoh: int = 40, raw_keys: bool = False, plain_search: bool = False, dual: bool = False,
                push_pagerank: bool = False, leaf_warps: int = 0, stream=None,
                allocator: "Allocator | None" = None) -> int:
    flags = ((GPMA_RAW_KEYS if raw_keys else 0) | (GPMA_PLAIN_SEARCH if plain_search else 0) |
             (GPMA_DUAL_DELETE if dual else 0) | (GPMA_PUSH_PAGERANK if push_pagerank else 0))
    p = gpma_params(leaf_size, tau0, tauh, rho0, rhoh, flags, leaf_warps)
    h = C.c_void_p()
    a = C.byref(allocator.struct) if allocator is not None else None
    _check(lib().gpma_create(n_vertices, C.byref(p), a, _stream(stream), C.byref(h)), "gpma_create")
    return h.value


def gpma_destroy(h: int):
    _check(lib().gpma_destroy(C.c_void_p(h)), "gpma_destroy")


def gpma_update_batch(h: int, ins, dels, stream=None, stats: bool = False):
    ins, dels = _keys(ins), _keys(dels)
    st = gpma_stats() if stats else None
    rc = lib().gpma_update_batch(C.c_void_p(h), _ptr(ins), ins.numel(), _ptr(dels), dels.numel(),
                                 _stream(stream), C.byref(st) if st is not None else None)
    _check(rc, "gpma_update_batch")
    return st.as_dict() if st is not None else None


def gpma_update_many(handles, ins_list, del_list, stream=None):
    """One batch per handle; the batches run as one launch per stage (see include/gpma.h)."""
    n = len(handles)
    ins_list = [_keys(x) for x in ins_list]
    del_list = [_keys(x) for x in del_list]
    H = (C.c_void_p * n)(*handles)
    PI = (C.c_void_p * n)(*[_ptr(x).value for x in ins_list])
    PD = (C.c_void_p * n)(*[_ptr(x).value for x in del_list])
    NI = (C.c_uint64 * n)(*[x.numel() for x in ins_list])
    ND = (C.c_uint64 * n)(*[x.numel() for x in del_list])
    _check(lib().gpma_update_many(H, PI, NI, PD, ND, n, _stream(stream)), "gpma_update_many")


def gpma_status(h: int, stream=None):
    _check(lib().gpma_status(C.c_void_p(h), _stream(stream)), "gpma_status")


def gpma_bfs(h: int, src: int, out, stream=None):
    _check(lib().gpma_bfs(C.c_void_p(h), src, _ptr(out), _stream(stream)), "gpma_bfs")
    return out


def gpma_cc(h: int, out, stream=None):
    _check(lib().gpma_cc(C.c_void_p(h), _ptr(out), _stream(stream)), "gpma_cc")
    return out


def gpma_pagerank(h: int, iters: int, damping: float, out, stream=None):
    _check(lib().gpma_pagerank(C.c_void_p(h), iters, damping, _ptr(out), _stream(stream)), "gpma_pagerank")
    return out


def gpma_pagerank_snapshot(h: int, stream=None) -> bool:
    """True when a snapshot was taken; False for a handle that sums by the push pass."""
    rc = lib().gpma_pagerank_snapshot(C.c_void_p(h), _stream(stream))
    if rc == GPMA_EINVAL:
        return False
    _check(rc, "gpma_pagerank_snapshot")
    return True


def gpma_pagerank_run(h: int, iters: int, damping: float, out, stream=None):
    _check(lib().gpma_pagerank_run(C.c_void_p(h), iters, damping, _ptr(out), _stream(stream)), "gpma_pagerank_run")
    return out


def gpma_export_sorted(h: int, out, stream=None) -> int:
    n = C.c_uint64()
    rc = lib().gpma_export_sorted(C.c_void_p(h), _ptr(out), out.numel() if out is not None else 0, C.byref(n),
                                  _stream(stream))
    if rc not in (GPMA_OK, GPMA_ECAP):
        _check(rc, "gpma_export_sorted")
    return n.value if rc == GPMA_OK else -n.value - 1


def gpma_export_sorted_noalloc(h: int, out, stream=None) -> int:
    n = C.c_uint64()
    rc = lib().gpma_export_sorted_noalloc(C.c_void_p(h), _ptr(out), out.numel() if out is not None else 0,
                                          C.byref(n), _stream(stream))
    if rc not in (GPMA_OK, GPMA_ECAP):
        _check(rc, "gpma_export_sorted_noalloc")
    return n.value if rc == GPMA_OK else -n.value - 1


def gpma_export_csr(h: int, rowptr, col, stream=None) -> int:
    n = C.c_uint64()
    rc = lib().gpma_export_csr(C.c_void_p(h), _ptr(rowptr), _ptr(col), col.numel() if col is not None else 0,
                               C.byref(n), _stream(stream))
    if rc not in (GPMA_OK, GPMA_ECAP):
        _check(rc, "gpma_export_csr")
    return n.value if rc == GPMA_OK else -n.value - 1


def gpma_export_layout(h: int, out, stream=None) -> int:
    n = C.c_uint64()
    rc = lib().gpma_export_layout(C.c_void_p(h), _ptr(out), out.numel() if out is not None else 0, C.byref(n),
                                  _stream(stream))
    if rc not in (GPMA_OK, GPMA_ECAP):
        _check(rc, "gpma_export_layout")
    return n.value if rc == GPMA_OK else -n.value - 1


def gpma_import_layout(h: int, slots, stream=None):
    _check(lib().gpma_import_layout(C.c_void_p(h), _ptr(slots), slots.numel(), _stream(stream)),
           "gpma_import_layout")


def gpma_row_end(h: int, out, stream=None):
    _check(lib().gpma_row_end(C.c_void_p(h), _ptr(out), _stream(stream)), "gpma_row_end")
    return out


def gpma_num_edges(h: int, stream=None) -> int:
    n = C.c_uint64()
    _check(lib().gpma_num_edges(C.c_void_p(h), C.byref(n), _stream(stream)), "gpma_num_edges")
    return n.value


def gpma_capacity(h: int) -> int:
    n = C.c_uint64()
    _check(lib().gpma_capacity(C.c_void_p(h), C.byref(n)), "gpma_capacity")
    return n.value


def gpma_check(h: int, stream=None) -> int:
    c = C.c_uint32()
    _check(lib().gpma_check(C.c_void_p(h), C.byref(c), _stream(stream)), "gpma_check")
    return c.value


def gpma_set_wait_limit(h: int, polls: int, stream=None):
    _check(lib().gpma_set_wait_limit(C.c_void_p(h), polls, _stream(stream)), "gpma_set_wait_limit")


def gpma_strerror(code: int) -> str:
    return lib().gpma_strerror(code).decode()


def gpma_profile_enable(h: int, on: bool = True):
    _check(lib().gpma_profile_enable(C.c_void_p(h), 1 if on else 0), "gpma_profile_enable")


def gpma_profile_read(h: int, reset: bool = True) -> dict:
    p = gpma_profile()
    _check(lib().gpma_profile_read(C.c_void_p(h), C.byref(p), 1 if reset else 0), "gpma_profile_read")
    return p.as_dict()


def gpma_launch_count() -> int:
    return int(lib().gpma_launch_count())


# ---- convenience object over the same calls -------------------------------------------------
class Graph:
    """A GPMA+ array on the current CUDA device (owns one libgpma handle).

    Flags (include/gpma.h): ``raw_keys`` (opaque keys, no guards or queries),
    ``plain_search`` (binary leaf search only), ``dual`` (deletion as the dual of
    insertion), ``push_pagerank`` (PageRank by the push pass instead of the bucketed
    pass; same ranks).  ``leaf_warps`` (1, 2, 4, 8; 0 = the library's choice) sets the
    warps per block of the one-warp-per-leaf level-0 pass.  Extra keywords ``tau0``,
    ``tauh``, ``rho0``, ``rhoh`` set the density bounds in whole percent.  ``allocator``
    (an ``Allocator``, e.g. ``torch_allocator()``) supplies the library's device
    memory; default cudaMallocAsync."""

    def __init__(self, n_vertices: int, leaf_size: int = 64, raw_keys: bool = False, plain_search: bool = False,
                 dual: bool = False, push_pagerank: bool = False, leaf_warps: int = 0, stream=None,
                 allocator: Allocator | None = None, **dens):
        self.n_vertices = 0 if raw_keys else int(n_vertices)
        self.raw = raw_keys
        self.allocator = allocator  # the callbacks must outlive the handle
        self.h = None
        self.h = gpma_create(n_vertices, leaf_size=leaf_size, raw_keys=raw_keys, plain_search=plain_search,
                             dual=dual, push_pagerank=push_pagerank, leaf_warps=leaf_warps, stream=stream,
                             allocator=allocator, **dens)

    def close(self):
        if getattr(self, "h", None):
            gpma_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, ins=None, dels=None, stats: bool = False, stream=None):
        return gpma_update_batch(self.h, ins, dels, stream=stream, stats=stats)

    @staticmethod
    def update_many(graphs, ins_list, del_list, stream=None):
        """Apply ins_list[i] / del_list[i] to graphs[i], all batches in one batched call."""
        gpma_update_many([g.h for g in graphs], ins_list, del_list, stream=stream)

    def status(self, stream=None):
        gpma_status(self.h, stream)

    def bfs(self, src: int, stream=None):
        torch = _torch()
        out = torch.empty(self.n_vertices, dtype=torch.int32, device="cuda")
        return gpma_bfs(self.h, src, out, stream)

    def cc(self, stream=None):
        torch = _torch()
        out = torch.empty(self.n_vertices, dtype=torch.int32, device="cuda")
        return gpma_cc(self.h, out, stream)

    def pagerank(self, iters: int = 20, damping: float = 0.85, stream=None):
        torch = _torch()
        out = torch.empty(self.n_vertices, dtype=torch.float32, device="cuda")
        return gpma_pagerank(self.h, iters, damping, out, stream)

    def export_sorted(self, stream=None):
        torch = _torch()
        n = self.num_edges(stream)
        out = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        got = gpma_export_sorted(self.h, out, stream)
        if got < 0:
            raise GpmaError(GPMA_ECAP, "export_sorted")
        return out[:got]

    def export_csr(self, stream=None):
        torch = _torch()
        n = self.num_edges(stream)
        rowptr = torch.empty(self.n_vertices + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        got = gpma_export_csr(self.h, rowptr, col, stream)
        if got < 0:
            raise GpmaError(GPMA_ECAP, "export_csr")
        return rowptr, col[:got]

    def layout(self, stream=None):
        torch = _torch()
        out = torch.empty(self.capacity, dtype=torch.int64, device="cuda")
        gpma_export_layout(self.h, out, stream)
        return out

    def import_layout(self, slots, stream=None):
        gpma_import_layout(self.h, _keys(slots), stream)

    def row_end(self, stream=None):
        torch = _torch()
        out = torch.empty(self.n_vertices, dtype=torch.int32, device="cuda")
        return gpma_row_end(self.h, out, stream)

    def num_edges(self, stream=None) -> int:
        return gpma_num_edges(self.h, stream)

    @property
    def capacity(self) -> int:
        return gpma_capacity(self.h)

    def check(self, stream=None) -> int:
        return gpma_check(self.h, stream)
