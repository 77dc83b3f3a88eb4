"""GPU parity at the shape the bench times (32x32 velocities on [-6, 6],
overset MEMS meshes, micro-sweep tiles picked by the autotuner), one flux
evaluation on a random non-equilibrium state at the full bench size compared
output by output, and bit-exact overset connectivity at the full MEMS and
two-body sizes.

The field comparison scales every component of W and q by that component's
own largest magnitude (a global maximum would hide errors in the small
components: the velocity near rest, the heat flux)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import kinetic as kn  # noqa: E402
from oracle import overset  # noqa: E402
from oracle import ugks as ou  # noqa: E402
from oracle.run import Run  # noqa: E402
from paper_2604_09984_gb300 import ugks as U  # noqa: E402
from paper_2604_09984_gb300 import workloads as wl  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(U.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    U.load()


def rel_per_component(a, b):
    """max over components m of max_cells |a_m - b_m| / max_cells |b_m|."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = []
    for m in range(b.shape[1]):
        s = np.abs(b[:, m]).max()
        out.append(np.abs(a[:, m] - b[:, m]).max() / s if s > 0 else np.abs(a[:, m]).max())
    return max(out), out


def test_fp32_bench_velocity_grid_after_autotune():
    """FP32-mixed path on the MEMS geometry at 96x48 + 64x16 cells with the
    bench's 32x32 velocity grid on [-6, 6] (32 velocity chunks of 32), the
    sweep tile chosen by ugks_autotune after the first step as the bench
    does: after two physical steps every component of W is within 1e-5 of
    the FP64 oracle relative to its own magnitude, and q within 1e-4."""
    case = wl.mems(nbi=96, nbj=48, noi=64, noj=16, nv=32, n_inner=2)
    assert case.nvx == 32 and case.vbox == (-6.0, 6.0, -6.0, 6.0)
    s = U.Solver(case, U.FP32)
    r = Run(case)
    s.advance()
    tiles = s.autotune(reps=1)
    assert tiles[1] in (2, 4) and tiles[0] == 32 * tiles[1] and tiles[4] in (8, 16, 32) and tiles[5] in (1, 2)
    s.advance()
    r.step()
    r.step()
    W, q, st, _ = s.moments()
    assert np.array_equal(st, r.status)
    field = r.status == 0
    eW, cw = rel_per_component(W[field], r.state.W[field])
    eq, cq = rel_per_component(q[field], r.state.q[field])
    print("\nW per component", ["%.2e" % v for v in cw], "q", ["%.2e" % v for v in cq], "tiles", tiles)
    assert eW < 1e-5, cw
    assert eq < 1e-4, cq


def _load_golden(name):
    path = os.path.join(GOLDEN, "connect_%s.npz" % name)
    return np.load(path)


@pytest.mark.parametrize("name", ["mems", "tsto"])
def test_connectivity_full_size_bit_exact(name):
    """Sec. 3.1 assembly at the full bench sizes (MEMS 256x128 + 128x32,
    two bodies 512x256 + 2x192x48): status, stencils and the bits of the
    inverse-distance weights equal the oracle's (stored by
    tests/golden/make_connect_golden.py) at t = 0 and after a move to t1."""
    g = _load_golden(name)
    case = wl.mems() if name == "mems" else wl.tsto()
    s = U.Solver(case, U.FP32)
    for tag in ("t0", "t1"):
        if tag == "t1":
            s.move_mesh(float(g["t1"]))
            stats = s.overset_connect()
            assert stats["n_fresh"] == g["t1_fresh"].size
            assert stats["n_orphan"] == int(g["t1_n_orphan"]) == 0
        st, dn, w = s.connectivity()
        assert np.array_equal(st, g[tag + "_status"].astype(np.int32))
        rec = g[tag + "_receptors"]
        assert np.array_equal(np.nonzero(st == U.RECEPTOR)[0], rec)
        assert np.array_equal(dn[rec], g[tag + "_donors"])
        assert np.array_equal(w[rec].view(np.int64), g[tag + "_weight_bits"])


@pytest.fixture(scope="module")
def full_size_flux():
    """The oracle's flux evaluation (Eqs. microscopicFlux, macroscopicFlux, the
    wall condition) on the full MEMS bench mesh (256x128 + 128x32 cells, 32x32
    velocities) in a random non-equilibrium state (Maxwellians of perturbed
    primitives times seeded noise on f), with the receptors interpolated from
    the assembly at t = 0 and the geometry of the move to t = dt."""
    case = wl.mems()
    prim = wl.random_prim(case, 7, amp_rho=0.1, amp_u=0.1, amp_T=0.1)
    r = Run(case, prim)
    rng = np.random.Generator(np.random.PCG64(8))
    st = r.state
    st.f = st.f * (1.0 + rng.uniform(-0.05, 0.05, st.f.shape))
    st.W = kn.moments(st.f, r.dvs)
    rho, Vx, Vy, lam = kn.primitive(st.W, r.gas)
    st.q = kn.heat_flux(st.f, Vx, Vy, r.dvs)
    f0, W0, q0 = st.f.copy(), st.W.copy(), st.q.copy()
    conn = r.conn
    overset.interpolate(st, conn.receptors, conn.donors, conn.weights)
    geo = r.geometry(0.0, case.dt)
    wS = ou.normal_velocity(r.setup, geo)
    dts = ou.explicit_dt(r.setup, geo, wS)
    fl = ou.flux(r.setup, geo, st, r.status, dts, wS)
    wall = np.zeros((len(case.blocks), 4))
    for n, f in enumerate(fl.wall_face):
        wall[r.setup.topo.face_block[f]] += geo.S[f] * fl.wall_F[n]
    return case, prim, (f0, W0, q0), r.status, fl, wall


@pytest.mark.parametrize("prec,tol", [(U.FP64, 1e-11), (U.FP32, 2e-5)])
def test_flux_full_size_matches_oracle(full_size_flux, prec, tol):
    """At the full bench size, every (cell, velocity) of the flux divergence
    D, every cell's macro flux F and every block's wall loads equal the
    oracle's (FP64 to 1e-11, FP32-mixed to 2e-5 of the largest magnitude)."""
    case, prim, (f0, W0, q0), status, fl, wall_ref = full_size_flux
    s = U.Solver(case, prec, prim=prim)
    st, _, _ = s.connectivity()
    assert np.array_equal(st, status.astype(np.int32))
    s.set_state(torch.as_tensor(f0), W0, q0)
    s.move_mesh(case.dt)
    D, F = s.eval_flux()
    field = status == 0
    Dg = D.cpu().numpy()
    assert np.abs(Dg[field] - fl.D[field]).max() / np.abs(fl.D[field]).max() < tol
    assert np.abs(F[field] - fl.F[field]).max() / np.abs(fl.F[field]).max() < tol
    _, _, _, wall = s.moments()
    assert np.abs(wall - wall_ref).max() / np.abs(wall_ref).max() < tol
    del D
