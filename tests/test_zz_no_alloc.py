"""Allocation-free receptor interpolation (ugks_idw_interpolate_static).

Some callers of this library cannot allocate device memory at all -- a host
framework that owns every device allocation, or code that must not call
cudaMalloc while other work is being captured or replayed -- so they cannot
even provide the context workspace.  For them the library exports one entry
point whose scratch is a fixed static device array.  This test checks it
against the interpolation that ugks_eval_flux applies through the context's
workspace scratch, on two calls in a row (the scratch keeps the previous
call's contents, which must not leak into the result).  The file name makes
pytest collect it last."""
import ctypes
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


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_static_interpolation_matches_workspace_path():
    case = wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=2)
    prim = wl.random_prim(case, 21, amp_rho=0.1, amp_u=0.1, amp_T=0.1)
    s = U.Solver(case, U.FP64, prim=prim)
    s.move_mesh(case.dt)
    s.overset_connect()
    f0, W0, q0 = s.get_state()
    s.eval_flux()                        # interpolates the receptor rows in place
    f1, W1, q1 = s.get_state()
    st, dn, w = s.connectivity()
    rec = np.nonzero(st == U.RECEPTOR)[0].astype(np.int32)
    assert rec.size > 0
    dev = s.device
    rec_d = torch.as_tensor(rec, device=dev)
    dn_d = torch.as_tensor(np.ascontiguousarray(dn[rec]), device=dev)
    w_d = torch.as_tensor(np.ascontiguousarray(w[rec]), device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    lib = U.load()
    for _ in range(2):
        fx = f0.clone()
        Wx = torch.as_tensor(W0, device=dev).clone()
        qx = torch.as_tensor(q0, device=dev).clone()
        r = lib.ugks_idw_interpolate_static(_p(fx), _p(Wx), _p(qx), s.nc, s.nv, _p(rec_d),
                                            int(rec.size), _p(dn_d), _p(w_d), stream)
        assert r == U.OK
        torch.cuda.synchronize()
        assert rel(fx.cpu().numpy(), f1.cpu().numpy()) < 1e-12
        assert rel(Wx.cpu().numpy(), W1) < 1e-12
        assert rel(qx.cpu().numpy(), q1) < 1e-12
        moved = fx.cpu().numpy()[rec] - f0.cpu().numpy()[rec]
        assert np.abs(moved).max() > 0       # the call did interpolate


def test_static_interpolation_rejects_oversized_input():
    dev = torch.device("cuda")
    f = torch.zeros(16, dtype=torch.float64, device=dev)
    idx = torch.zeros(5, dtype=torch.int32, device=dev)
    wt = torch.zeros(5, dtype=torch.float64, device=dev)
    lib = U.load()
    nv = U.STATIC_SCRATCH_DOUBLES          # 2 * nv > the scratch: rejected, nothing launched
    r = lib.ugks_idw_interpolate_static(_p(f), None, None, 1, nv, _p(idx), 1, _p(idx), _p(wt), None)
    assert r == -1
    r = lib.ugks_idw_interpolate_static(None, None, None, 1, 8, _p(idx), 1, _p(idx), _p(wt), None)
    assert r == -1
