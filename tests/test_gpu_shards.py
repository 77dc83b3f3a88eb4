"""Velocity-space sharding on one GPU: the velocity grid split into 2 or 3
shards of whole velocity rows, each a context of its own, stepped together
with the shards' partial velocity sums added in shard order at the two
exchange points of every inner iteration (the face sums of the velocity
reduction, the step-7 moment sums).  The sharded run equals the run on one
context holding the whole grid: f velocity by velocity, W, q and the wall
loads (FP64 to 1e-12; FP32 to 1e-6, the FP32 velocity sums being grouped
differently) -- the data path of a multi-GPU run with the collective
replaced by an in-process sum."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2604_09984_gb300 import ugks as U  # noqa: E402
from paper_2604_09984_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(U.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    U.load()


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("prec,tol", [(U.FP64, 1e-12), (U.FP32, 1e-6)])
@pytest.mark.parametrize("nshards", [2, 3])
def test_velocity_shards_match_single_context(prec, tol, nshards):
    case = wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=2)
    prim = wl.random_prim(case, 31, amp_rho=0.05, amp_u=0.05, amp_T=0.05)
    one = U.Solver(case, prec, prim=prim)
    sh = U.ShardSet(case, prec, nshards, prim=prim)
    assert [s.nv for s in sh.solvers] == [case.nvx * (b - a) for a, b in sh.rows]
    for _ in range(2):
        one.advance()
        sh.advance()
    W1, q1, st1, wall1 = one.moments()
    for s in sh.solvers:                    # every shard holds the same macroscopic state
        W, q, st, wall = s.moments()
        assert np.array_equal(st, st1)
        assert rel(W, W1) < tol and rel(q, q1) < 10 * tol and rel(wall, wall1) < 10 * tol
    assert np.array_equal(sh.solvers[0].moments()[0], sh.solvers[-1].moments()[0])
    f1 = one.get_state()[0].cpu().numpy()
    fs = sh.get_f().cpu().numpy()
    assert fs.shape == f1.shape
    assert rel(fs, f1) < tol


def test_sharded_context_needs_its_exchange():
    case = wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=1)
    s = U.Solver(case, U.FP64, shard=(0, 4))
    with pytest.raises(U.UgksError) as err:
        s.advance()
    assert err.value.code == -7              # UGKS_ERR_ORDER: no exchange function set
    whole = U.Solver(case, U.FP64)
    with pytest.raises(U.UgksError):
        whole.set_exchange(lambda which: None)    # not a sharded context
