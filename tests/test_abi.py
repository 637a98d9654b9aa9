"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/gpma.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_1709_05061_gb300 as gp

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gpma.h")


@pytest.fixture(scope="module")
def lib():
    gp.build()
    return gp.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gpma_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for n in ["gpma_create", "gpma_destroy", "gpma_update_batch", "gpma_bfs", "gpma_cc", "gpma_pagerank",
              "gpma_export_sorted", "gpma_export_csr", "gpma_export_layout", "gpma_import_layout",
              "gpma_num_edges", "gpma_capacity", "gpma_strerror", "gpma_status", "gpma_check", "gpma_row_end"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_strerror_without_gpu(lib):
    for code in range(6):
        assert gp.gpma_strerror(code)
    assert "unknown" in gp.gpma_strerror(99)


def test_argument_errors_without_gpu(lib):
    # rejected on the host before any CUDA call
    assert lib.gpma_destroy(None) == gp.GPMA_EINVAL
    assert lib.gpma_capacity(None, None) == gp.GPMA_EINVAL
    out = ctypes.c_void_p()
    p = gp.gpma_params(3, 0, 0, 0, 0, 0)  # leaf size not a power of two
    assert lib.gpma_create(10, ctypes.byref(p), None, None, ctypes.byref(out)) == gp.GPMA_EINVAL
    p = gp.gpma_params(64, 50, 80, 0, 0, 0)  # tau_0 below tau_h
    assert lib.gpma_create(10, ctypes.byref(p), None, None, ctypes.byref(out)) == gp.GPMA_EINVAL
    p = gp.gpma_params(64, 0, 0, 0, 0, 0)
    assert lib.gpma_create(0, ctypes.byref(p), None, None, ctypes.byref(out)) == gp.GPMA_EINVAL
    p = gp.gpma_params(64, 0, 0, 0, 0, 0, 3)  # warps per leaf-pass block not 1, 2, 4 or 8
    assert lib.gpma_create(10, ctypes.byref(p), None, None, ctypes.byref(out)) == gp.GPMA_EINVAL
    # gpma_update_many: a missing handle array, a null handle
    n = ctypes.c_uint64(1)
    assert lib.gpma_update_many(None, None, ctypes.byref(n), None, ctypes.byref(n), 1, None) == gp.GPMA_EINVAL
    H = (ctypes.c_void_p * 1)(None)
    assert lib.gpma_update_many(H, None, ctypes.byref(n), None, ctypes.byref(n), 1, None) == gp.GPMA_EINVAL


def header_defines():
    text = open(HEADER).read()
    return {m.group(1): m.group(2) for m in re.finditer(r"#define\s+(GPMA_[A-Z0-9_]+)\s+(\S+)", text)}


def test_binding_constants_match_the_header():
    """The binding's flag values and profile layout follow include/gpma.h (a
    mismatch in the profile struct would let the library write past it)."""
    d = header_defines()
    assert int(d["GPMA_PROF_N"]) == gp.GPMA_PROF_N == len(gp.GPMA_PROF_NAMES)
    assert ctypes.sizeof(gp.gpma_profile) == 3 * 8 * int(d["GPMA_PROF_N"])
    for i, n in enumerate(gp.GPMA_PROF_NAMES):
        assert int(d["GPMA_PROF_" + n.upper()]) == i, n
    for name in ("GPMA_RAW_KEYS", "GPMA_PLAIN_SEARCH", "GPMA_DUAL_DELETE", "GPMA_PUSH_PAGERANK"):
        assert int(d[name].rstrip("u")) == getattr(gp, name), name


def test_allocator_failure_without_gpu(lib):
    """A caller-supplied allocator that refuses the first request: gpma_create
    returns GPMA_ENOMEM, hands out no handle and frees nothing it did not get."""
    asked, freed = [], []
    A = gp.Allocator(lambda n, s: asked.append(n) or 0, lambda p, s: freed.append(p))
    out = ctypes.c_void_p()
    p = gp.gpma_params(64, 0, 0, 0, 0, 0)
    rc = lib.gpma_create(1000, ctypes.byref(p), ctypes.byref(A.struct), None, ctypes.byref(out))
    assert rc == gp.GPMA_ENOMEM
    assert not out.value
    assert asked and not freed
    # an allocator without both functions is rejected before any allocation
    bad = gp.gpma_allocator()
    assert lib.gpma_create(1000, ctypes.byref(p), ctypes.byref(bad), None, ctypes.byref(out)) == gp.GPMA_EINVAL
