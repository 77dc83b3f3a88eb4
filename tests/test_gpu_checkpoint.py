"""Checkpoint and resume (GPU).  A context restored from a checkpoint taken
between two physical steps (f, W, q, t, the node coordinates at t and the cell
status of the last assembly) continues bit for bit as the context it was
taken from: an overset MEMS case with a moving body, whose assembly changes
the status of some cells every step, on the FP32 and FP64 paths.  The
restored context hands back the checkpoint it was given.  A checkpoint is
refused while a move is pending."""
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


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_resume_continues_bit_for_bit(prec):
    case = wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=2)
    prim = wl.random_prim(case, 43, amp_rho=0.05, amp_u=0.05, amp_T=0.05)
    a = U.Solver(case, prec, prim=prim)
    b = U.Solver(case, prec, prim=prim)
    for _ in range(3):
        a.advance()
        b.advance()
    ck = b.checkpoint()
    del b
    # a context started from another state, then restored
    c = U.Solver(case, prec, prim=wl.random_prim(case, 7, amp_rho=0.05, amp_u=0.05, amp_T=0.05))
    c.restore(ck)
    assert c.t == a.t
    back = c.checkpoint()
    assert back["t"] == ck["t"]
    for k in ("W", "q", "nodes", "status"):
        assert np.array_equal(back[k], ck[k]), k
    assert torch.equal(back["f"], ck["f"])
    for _ in range(3):
        a.advance()
        c.advance()
        assert a.last_stats == c.last_stats
    for x, y in zip(a.moments(), c.moments()):
        assert np.array_equal(x, y)
    assert torch.equal(a.get_state()[0], c.get_state()[0])
    ka, kc = a.checkpoint(), c.checkpoint()
    assert ka["t"] == kc["t"]
    assert np.array_equal(ka["nodes"], kc["nodes"])
    assert np.array_equal(ka["status"], kc["status"])


def test_checkpoint_refused_while_a_move_is_pending():
    case = wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=1)
    s = U.Solver(case, U.FP32)
    ck = s.checkpoint()
    s.move_mesh(s.t + case.dt)
    with pytest.raises(U.UgksError) as e:
        s.checkpoint()
    assert e.value.code == -7
    with pytest.raises(U.UgksError):
        s.restore(ck)
