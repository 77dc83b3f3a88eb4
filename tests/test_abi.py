"""CPU checks of the C ABI boundary: the library loads, exports every entry
point declared in include/ugks.h, and its host-only workspace query and
argument validation work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2604_09984_gb300 import ugks as U
from paper_2604_09984_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "ugks.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ugks_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(U.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return U.load()


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(U.SYMBOLS), set(names) ^ set(U.SYMBOLS)


def test_workspace_query_host_only(lib):
    case = wl.channel(ni=16, nj=8, nv=10)
    n32 = U.workspace_bytes(case, U.FP32)
    n64 = U.workspace_bytes(case, U.FP64)
    nbf = U.workspace_bytes(case, U.BF16F)
    assert n64 > n32 > nbf > 0
    assert n32 - nbf >= 4 * 16 * 8 * 100       # f alone shrinks by 4 bytes a cell-velocity
    # f, level-n term and sweep increments dominate: >= 3 copies of f
    assert n64 >= 3 * 16 * 16 * 8 * 100
    big = wl.mems(nv=32)
    assert U.workspace_bytes(big, U.FP32) > 3 * 8 * 36864 * 1024


def test_argument_validation(lib):
    case = wl.channel(ni=4, nj=4, nv=6)
    p = U.make_params(case, U.FP64)
    descs, keep = U.make_blocks(case)
    n = ctypes.c_size_t(0)
    descs[0].nj = 1
    assert lib.ugks_workspace_query(ctypes.byref(p), 1, descs, ctypes.byref(n)) == -1
    descs[0].nj = 4
    descs[0].bc[0] = 1          # periodic block with an i-side wall
    assert lib.ugks_workspace_query(ctypes.byref(p), 1, descs, ctypes.byref(n)) == -1
    descs[0].bc[0] = 0
    p.precision = 7
    assert lib.ugks_workspace_query(ctypes.byref(p), 1, descs, ctypes.byref(n)) == -1
    p.precision = 0
    assert lib.ugks_workspace_query(ctypes.byref(p), 1, descs, ctypes.byref(n)) == 0
    # misaligned workspace is rejected before any CUDA call
    ctx = ctypes.c_void_p()
    assert lib.ugks_create(ctypes.byref(p), ctypes.c_void_p(8), 100, None, ctypes.byref(ctx)) == -6


def test_batch_argument_validation(lib):
    """ugks_advance_batch checks its arguments before touching any context or
    the device: an empty batch is a no-op, a negative count or missing arrays
    are rejected."""
    failed = ctypes.c_int(7)
    assert lib.ugks_advance_batch(None, 0, None, None, 10, ctypes.byref(failed)) == 0
    assert failed.value == -1
    assert lib.ugks_advance_batch(None, -1, None, None, 10, ctypes.byref(failed)) == -1
    ctxs = (ctypes.c_void_p * 1)(None)
    assert lib.ugks_advance_batch(ctxs, 1, None, None, 10, None) == -1
    t = (ctypes.c_double * 1)(1.0)
    aff = (ctypes.POINTER(ctypes.c_double) * 1)()
    assert lib.ugks_advance_batch(ctxs, 1, t, aff, 10, ctypes.byref(failed)) == -7
    assert failed.value == 0


def test_null_context_is_rejected_without_cuda(lib):
    """The checkpoint, metrics and graph entry points check their context
    before any CUDA call: a null context is an argument or ordering error."""
    t = ctypes.c_double(0.0)
    m = U.StepMetrics()
    assert lib.ugks_get_checkpoint(None, ctypes.byref(t), None, None) == -7
    assert lib.ugks_set_checkpoint(None, 0.0, None, None) == -7
    assert lib.ugks_set_metrics(None, 1) == -1
    assert lib.ugks_get_metrics(None, ctypes.byref(m)) == -7
    assert lib.ugks_set_graphs(None, 1) == -1
    c, r = ctypes.c_int64(), ctypes.c_int64()
    assert lib.ugks_graph_stats(None, ctypes.byref(c), ctypes.byref(r)) == -1
