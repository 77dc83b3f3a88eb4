"""Allocation-free receptor interpolation (ugks_idw_interpolate_static).

Some callers of this library cannot allocate device memory at all -- a host
framework that owns every device allocation, or code that must not call
cudaMalloc while other work is being captured or replayed -- so they cannot
even provide the context workspace.  For them the library exports one entry
point whose scratch is a fixed static device array.  This test checks it
against the interpolation that ugks_eval_flux applies through the context's
workspace, and against the inverse-distance sums written out on the host,
on two calls in a row with different inputs and receptor orders (the
scratch keeps the previous call's contents, which must not leak into the
result), with an odd velocity count, an orphan row and a row naming a donor
outside the mesh.  The file name makes pytest collect it last."""
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


def host_idw(f, W, q, rec, dn, w, nc):
    """phi_r = sum_j w_rj phi_j over the valid donors of each row (weights
    renormalised when a donor outside the mesh was dropped); orphan rows and
    rows without a valid donor keep their values; donors read the values
    from before the call."""
    f2, W2, q2 = f.copy(), W.copy(), q.copy()
    for r, c in enumerate(rec):
        if dn[r, 0] < 0 or not 0 <= c < nc:
            continue
        valid = (dn[r] >= 0) & (dn[r] < nc)
        wv = np.where(valid, w[r], 0.0)
        tot = wv.sum()
        if tot == 0.0:
            continue
        if ((dn[r] != -1) & ~valid).any():
            wv = wv / tot
        ids = np.where(valid, dn[r], 0)
        f2[c] = np.tensordot(wv, f[ids], axes=1)
        W2[c] = wv @ W[ids]
        q2[c] = wv @ q[ids]
    return f2, W2, q2


def test_static_interpolation_matches_workspace_path():
    # 5x5 velocities: an odd count, one ragged chunk of the kernels
    case = wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=5, stretch=1.15, n_inner=2)
    prim = wl.random_prim(case, 21, amp_rho=0.1, amp_u=0.1, amp_T=0.1)
    s = U.Solver(case, U.FP64, prim=prim)
    s.move_mesh(case.dt)
    s.overset_connect()
    f0, W0, q0 = s.get_state()
    st, dn, w = s.connectivity()
    nc = s.nc
    rec = np.nonzero(st == U.RECEPTOR)[0].astype(np.int32)
    assert rec.size > 0
    field = np.nonzero(st == U.FIELD)[0]
    # extra rows: an orphan (first donor -1) and a row with a donor id past
    # the last cell, on two field cells the assembly did not touch
    orphan, bad = int(field[0]), int(field[1])
    d_bad = np.array([[int(field[2]), nc + 7, int(field[3]), -1, -1]], dtype=np.int32)
    w_bad = np.array([[0.5, 0.3, 0.2, 0.0, 0.0]])
    rec_all = np.concatenate([rec, [orphan, bad]]).astype(np.int32)
    dn_all = np.concatenate([dn[rec], [[-1, -1, -1, -1, -1]], d_bad]).astype(np.int32)
    w_all = np.concatenate([w[rec], [[0.0] * 5], w_bad])
    dev = s.device
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    lib = U.load()
    rng = np.random.default_rng(5)
    scales = [(1.0, 1.0, 1.0), (1.7, 0.9, 1.3)]
    for call, (sf, sW, sq) in enumerate(scales):
        order = np.arange(rec_all.size) if call == 0 else rng.permutation(rec_all.size)
        fin = f0 * sf
        Win, qin = W0 * sW, q0 * sq
        # the workspace path on the same input
        s.set_state(fin, Win, qin)
        s.eval_flux()
        fw, Ww, qw = s.get_state()
        fx = fin.clone()
        Wx = torch.as_tensor(Win, device=dev).clone()
        qx = torch.as_tensor(qin, device=dev).clone()
        rec_d = torch.as_tensor(rec_all[order], device=dev)
        dn_d = torch.as_tensor(np.ascontiguousarray(dn_all[order]), device=dev)
        w_d = torch.as_tensor(np.ascontiguousarray(w_all[order]), device=dev)
        r = lib.ugks_idw_interpolate_static(_p(fx), _p(Wx), _p(qx), nc, s.nv, _p(rec_d),
                                            int(rec_all.size), _p(dn_d), _p(w_d), stream)
        assert r == U.OK
        torch.cuda.synchronize()
        fx, Wx, qx = fx.cpu().numpy(), Wx.cpu().numpy(), qx.cpu().numpy()
        # assembly rows: as the workspace path; all rows: the host sums
        assert rel(fx[rec], fw.cpu().numpy()[rec]) < 1e-12
        assert rel(Wx[rec], Ww[rec]) < 1e-12 and rel(qx[rec], qw[rec]) < 1e-12
        fh, Wh, qh = host_idw(fin.cpu().numpy(), Win, qin, rec_all, dn_all, w_all, nc)
        assert rel(fx, fh) < 1e-12 and rel(Wx, Wh) < 1e-12 and rel(qx, qh) < 1e-12
        assert np.array_equal(fx[orphan], fin.cpu().numpy()[orphan])    # orphan row unchanged
        assert np.abs(fx[bad] - fin.cpu().numpy()[bad]).max() > 0        # the bad row was interpolated
        moved = fx[rec] - fin.cpu().numpy()[rec]
        assert np.abs(moved).max() > 0


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
