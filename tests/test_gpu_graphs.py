"""CUDA graphs of ugks_step (GPU).  A context that captures its step into a
graph and replays it equals, bit for bit, a context that launches every
kernel directly, over physical steps of an overset MEMS case with a moving
body (a step after an assembly that uncovered cells runs one more
interpolation and has a graph of its own), on the FP32 and FP64 paths.  Later steps
are replays; a change of the wait limit (part of the device struct the
kernels take by value) makes a new capture, whose replay still matches."""
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
def test_graph_replay_matches_direct_launches(prec):
    case = wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=2)
    prim = wl.random_prim(case, 41, amp_rho=0.05, amp_u=0.05, amp_T=0.05)
    g = U.Solver(case, prec, prim=prim)
    n = U.Solver(case, prec, prim=prim)
    n.set_graphs(False)
    for step in range(6):
        if step == 3:
            for s in (g, n):
                s.set_wait_limit(1 << 20)     # a new by-value argument: new capture
        for s in (g, n):
            s.advance()
    captures, replays = g.graph_stats()
    assert replays >= 2 and captures >= 2
    assert captures + replays == 6
    assert n.graph_stats() == (0, 0)
    assert g.launch_count() == n.launch_count()
    for a, b in zip(g.moments(), n.moments()):
        assert np.array_equal(a, b)
    assert torch.equal(g.get_state()[0], n.get_state()[0])


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_split_tail_matches_serial_tail(prec):
    """Step 7, the receptors' W and q and the W gradients of an inner
    iteration run on the side stream beside the next iteration's velocity
    reduction; the result equals, bit for bit, the same step with that tail
    in line on the main stream (UGKS_SERIAL_TAIL=1), with and without graphs."""
    case = wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=3)
    prim = wl.random_prim(case, 17, amp_rho=0.05, amp_u=0.05, amp_T=0.05)
    split = U.Solver(case, prec, prim=prim)
    os.environ["UGKS_SERIAL_TAIL"] = "1"
    try:
        serial = U.Solver(case, prec, prim=prim)
    finally:
        del os.environ["UGKS_SERIAL_TAIL"]
    direct = U.Solver(case, prec, prim=prim)
    direct.set_graphs(False)
    for _ in range(3):
        for s in (split, serial, direct):
            s.advance()
    ref = serial.moments()
    for s in (split, direct):
        for a, b in zip(s.moments(), ref):
            assert np.array_equal(a, b)
        assert torch.equal(s.get_state()[0], serial.get_state()[0])


def test_macro_sweep_pass_slots_match_four_threads_a_row():
    """The FP32 macro LU-SGS with two threads a row on the face slots that
    couple in each pass (and the periodic wrap of the O-grid) equals, bit for
    bit, the sweep with four threads a row evaluating every slot (the slots
    left out are exact zeros)."""
    case = wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=3)
    prim = wl.random_prim(case, 23, amp_rho=0.05, amp_u=0.05, amp_T=0.05)
    pm = U.Solver(case, U.FP32, prim=prim)
    four = U.Solver(case, U.FP32, prim=prim)
    for _ in range(3):
        pm.advance()
        os.environ["UGKS_MACRO_TPR"] = "4"
        try:
            four.advance()
        finally:
            del os.environ["UGKS_MACRO_TPR"]
    for a, b in zip(pm.moments(), four.moments()):
        assert np.array_equal(a, b)
    assert torch.equal(pm.get_state()[0], four.get_state()[0])
