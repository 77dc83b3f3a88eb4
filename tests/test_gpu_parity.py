"""GPU parity of libugks (through the C ABI) against the FP64 oracle on
small seeded cases that span several velocity tiles and a ragged tail.

Tolerances: FP64 path 1e-11 relative (max-norm) after several steps; FP32
mixed path 1e-5 relative on the macroscopic fields; overset connectivity
bit-exact."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import kinetic as kn  # noqa: E402
from oracle import mesh, overset  # noqa: E402
from oracle import ugks as ou  # noqa: E402
from oracle.run import Run  # noqa: E402
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


def perturbed_state(run, seed, amp=0.05):
    """Non-equilibrium f (Maxwellians times seeded noise), W and q from f."""
    rng = np.random.Generator(np.random.PCG64(seed))
    st = run.state
    st.f = st.f * (1.0 + rng.uniform(-amp, amp, st.f.shape))
    st.W = kn.moments(st.f, run.dvs)
    rho, Vx, Vy, lam = kn.primitive(st.W, run.gas)
    st.q = kn.heat_flux(st.f, Vx, Vy, run.dvs)
    return st


def small_channel(**kw):
    args = dict(ni=12, nj=7, nv=10, n_inner=3, n_steps=3)
    args.update(kw)
    return wl.channel(**args)


def small_mems(**kw):
    args = dict(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=2)
    args.update(kw)
    return wl.mems(**args)


@pytest.mark.parametrize("which", ["channel", "mems"])
def test_geometry_matches_oracle(which):
    case = small_channel() if which == "channel" else small_mems()
    s = U.Solver(case, U.FP64)
    s.move_mesh(case.dt)
    g = s.geometry()
    topo = mesh.Topology(case.blocks)
    ref = mesh.geometry(topo, case.nodes_at(0.0), case.nodes_at(case.dt), case.dt)
    assert rel(g["vol_old"], ref.vol_old) < 1e-14
    assert rel(g["vol_new"], ref.vol_new) < 1e-14
    assert rel(g["xc"], ref.xc) < 1e-14
    assert rel(g["Sn"], ref.Sn) < 1e-14
    assert np.abs(g["SUn"] - ref.SUn).max() < 1e-14 * np.abs(ref.Sn).max() * max(np.abs(ref.Uf).max(), 1.0)
    r = Run(case)
    wS = ou.normal_velocity(r.setup, ref)
    dts = ou.explicit_dt(r.setup, ref, wS)
    assert rel(g["dts"], dts) < 1e-13


@pytest.mark.parametrize("prec,tol", [(U.FP64, 1e-12), (U.FP32, 2e-5)])
def test_flux_random_state(prec, tol):
    """Eqs. microscopicFlux / macroscopicFlux on a random non-equilibrium
    state with a moving wall and a periodic seam."""
    case = small_channel()
    prim = wl.random_prim(case, 3, amp_rho=0.2, amp_u=0.3, amp_T=0.2)
    r = Run(case, prim)
    st = perturbed_state(r, 4)
    s = U.Solver(case, prec, prim=prim)
    s.set_state(st.f, st.W, st.q)
    s.move_mesh(case.dt)
    D, F = s.eval_flux()
    geo = r.geometry(0.0, case.dt)
    wS = ou.normal_velocity(r.setup, geo)
    dts = ou.explicit_dt(r.setup, geo, wS)
    fl = ou.flux(r.setup, geo, st, r.status, dts, wS)
    assert rel(D.cpu().numpy(), fl.D) < tol
    assert rel(F, fl.F) < tol
    # wall loads: per block, sum over its wall faces of S times the wall
    # macro flux (Eq. macroscopicFlux at the wall faces, reading R5)
    _, _, _, wall = s.moments()
    topo = r.setup.topo
    exp = np.zeros((len(case.blocks), 4))
    for n, f in enumerate(fl.wall_face):
        exp[topo.face_block[f]] += geo.S[f] * fl.wall_F[n]
    assert fl.wall_face.size > 0
    assert rel(wall, exp) < tol


def test_step_fp64_channel():
    """Several implicit steps (Sec. 2.2 Steps 1-8) on the deforming channel:
    f, W and q agree with the oracle."""
    case = small_channel()
    prim = wl.random_prim(case, 5, amp_rho=0.1, amp_u=0.1, amp_T=0.1)
    s = U.Solver(case, U.FP64, prim=prim)
    r = Run(case, prim)
    for _ in range(case.n_steps):
        s.advance()
        r.step()
    f, W, q = s.get_state()
    assert rel(W, r.state.W) < 1e-11
    assert rel(q, r.state.q) < 1e-9 * max(1.0, 1.0)
    assert rel(f.cpu().numpy(), r.state.f) < 1e-11


def test_step_fp32_channel_macro_tolerance():
    """Mixed precision: macroscopic fields within 1e-5 relative of FP64."""
    case = small_channel()
    prim = wl.random_prim(case, 5, amp_rho=0.1, amp_u=0.1, amp_T=0.1)
    s = U.Solver(case, U.FP32, prim=prim)
    r = Run(case, prim)
    for _ in range(case.n_steps):
        s.advance()
        r.step()
    W, q, st, wall = s.moments()
    assert rel(W, r.state.W) < 1e-5


@pytest.mark.parametrize("nv,ni,nj", [(7, 5, 3), (13, 9, 4), (6, 2, 3)])
def test_step_ragged_sizes(nv, ni, nj):
    """Velocity counts that leave a ragged last tile and a padded stride,
    minimal periodic width (ni = 2 makes both i-faces join the same pair)."""
    case = wl.channel(ni=ni, nj=nj, nv=nv, n_inner=2)
    prim = wl.random_prim(case, 11)
    s = U.Solver(case, U.FP64, prim=prim)
    r = Run(case, prim)
    for _ in range(2):
        s.advance()
        r.step()
    _, W, _ = s.get_state()
    assert rel(W, r.state.W) < 1e-11


@pytest.mark.parametrize("prec", [U.FP64, U.FP32])
@pytest.mark.parametrize("nj", [150, 300, 450, 512])
def test_step_tall_blocks(prec, nj):
    """Block heights that select the other sweep layouts: two and one threads
    per row in the macro sweep, shallower rings, records read straight from
    memory (nj > 427 in FP32), and the widest micro-sweep CTAs."""
    case = wl.channel(ni=3, nj=nj, nv=4, n_inner=2)
    prim = wl.random_prim(case, 12)
    s = U.Solver(case, prec, prim=prim)
    r = Run(case, prim)
    for _ in range(2):
        s.advance()
        r.step()
    W, _, _, _ = s.moments()
    assert rel(W, r.state.W) < (1e-11 if prec == U.FP64 else 1e-5)


def test_overset_connectivity_bit_exact():
    """Sec. 3.1 assembly: status, donor stencils and IDW weights identical
    bit for bit to the oracle, at several positions of the plate."""
    case = small_mems()
    s = U.Solver(case, U.FP64)
    topo = mesh.Topology(case.blocks)
    conn = overset.connect(topo, case.nodes_at(0.0))
    st, dn, w = s.connectivity()
    assert np.array_equal(st, conn.status)
    prev = conn.status
    t = 0.0
    for n in range(4):
        t1 = t + 0.7 / case.meta["freq"] / 4
        s.move_mesh(t1)
        stats = s.overset_connect()
        conn = overset.connect(topo, case.nodes_at(t1), prev)
        st, dn, w = s.connectivity()
        assert np.array_equal(st, conn.status)
        rec = conn.receptors
        assert np.array_equal(dn[rec], conn.donors)
        assert np.array_equal(w[rec].view(np.int64), conn.weights.view(np.int64))
        assert stats["n_fresh"] == conn.fresh.size
        assert stats["n_orphan"] == conn.n_orphan == 0
        prev = conn.status
        s.step(t1 - t, 1)
        t = t1


def test_step_fp64_overset():
    case = small_mems()
    prim = wl.random_prim(case, 9, amp_rho=0.05, amp_u=0.05, amp_T=0.05)
    s = U.Solver(case, U.FP64, prim=prim)
    r = Run(case, prim)
    for _ in range(2):
        s.advance()
        r.step()
    _, W, q = s.get_state()
    field = r.status == 0
    assert rel(W[field], r.state.W[field]) < 1e-11
    Wm, qm, stm, wall = s.moments()
    assert np.array_equal(stm, r.status)


def small_tsto(**kw):
    """Two-body separation at reduced size: K = 2 gas (Pr 0.72, omega 0.74),
    Mach 8 stream entering a gas at rest, three blocks, a pitching wedge and
    a translating cylinder, connectivity recomputed every step, CFL 10 on the
    smallest cell.  22^2 velocities on [-15, 15] (a ragged last tile); the
    background (1/40) is fine enough that its buffer receptors around the
    holes stay inside the body grids (no orphans)."""
    args = dict(nbi=80, nbj=40, noi=24, noj=10, nv=22, n_inner=2)
    args.update(kw)
    return wl.tsto(**args)


@pytest.mark.parametrize("prec,tol", [(U.FP64, 1e-11), (U.FP32, 1e-5)])
def test_step_two_bodies(prec, tol):
    case = small_tsto()
    s = U.Solver(case, prec)
    s.advance()
    W, q, st, wall = s.moments()
    ref_status, ref_W = _two_body_oracle()
    assert np.array_equal(st, ref_status)
    field = ref_status == 0
    assert np.isfinite(ref_W).all()
    assert rel(W[field], ref_W[field]) < tol


_TWO_BODY = {}


def _two_body_oracle():
    """One oracle step of the reduced two-body case (shared by both precisions)."""
    if not _TWO_BODY:
        r = Run(small_tsto())
        r.step()
        _TWO_BODY["v"] = (r.status.copy(), r.state.W.copy())
    return _TWO_BODY["v"]


@pytest.mark.parametrize("prec,tol", [(U.FP64, 1e-11), (U.FP32, 1e-5)])
def test_batch_matches_separate_runs(prec, tol):
    """Batched serving: independent instances of uneven mesh sizes, velocity
    grids, Knudsen numbers and wall temperatures, each on its own stream,
    advanced together through ugks_advance_batch.  Every instance matches
    the oracle and a separate run of the same instance."""
    cases = wl.mems_batch(n=3, seed=1, n_inner=2, ni_range=(32, 48), ntheta_range=(32, 40),
                          nv_range=(6, 9))
    assert len({c.nv for c in cases}) > 1 and len({c.ncells for c in cases}) > 1
    streams = [torch.cuda.Stream() for _ in cases]
    batch = [U.Solver(c, prec, stream=st) for c, st in zip(cases, streams)]
    single = [U.Solver(c, prec) for c in cases]
    runs = [Run(c) for c in cases]
    for _ in range(2):
        U.advance_batch(batch)
        for s, r in zip(single, runs):
            s.advance()
            r.step()
    for b, s, r in zip(batch, single, runs):
        Wb, _, stb, _ = b.moments()
        Ws, _, sts, _ = s.moments()
        assert np.array_equal(stb, r.status)
        assert np.array_equal(sts, r.status)
        field = r.status == 0
        assert rel(Wb[field], r.state.W[field]) < tol
        assert rel(Wb, Ws) < (1e-13 if prec == U.FP64 else 1e-6)


def test_autotune_restores_state_and_changes_no_result():
    """The sweep autotuner times every candidate (velocities per lane,
    prefetch ring depth) on the live state, restores f bit for bit, and every
    candidate computes the same sweeps: runs on the tuned choice and on the
    shallowest ring match the default one."""
    case = small_mems()
    prim = wl.random_prim(case, 21, amp_rho=0.05, amp_u=0.05, amp_T=0.05)
    a = U.Solver(case, U.FP64, prim=prim)
    b = U.Solver(case, U.FP64, prim=prim)
    with pytest.raises(U.UgksError):
        a.autotune(reps=1)                      # needs a step first
    os.environ["UGKS_SWEEP_NS"] = "2"
    try:
        c = U.Solver(case, U.FP64, prim=prim)
    finally:
        del os.environ["UGKS_SWEEP_NS"]
    for s in (a, b, c):
        s.advance()
    f0, _, _ = a.get_state()
    items, vpt, ring_f, ring_b, fvk, fnh = a.autotune(reps=1)
    assert vpt == 2 and items == 64 and ring_f in (1, 2, 4, 6) and ring_b in (1, 2, 4, 6)
    assert (fvk, fnh) == (8, 2)
    f1, _, _ = a.get_state()
    assert torch.equal(f0, f1)
    for _ in range(2):
        for s in (a, b, c):
            s.advance()
    Wb = b.moments()[0]
    assert rel(a.moments()[0], Wb) < 1e-13
    assert rel(c.moments()[0], Wb) < 1e-13


def test_batch_defers_orphan_report_to_next_sync():
    """ugks_advance_batch never waits on the device: an assembly that leaves
    receptors without donor (the body grid pushed half out of the box)
    returns UGKS_OK at once and surfaces as UGKS_ERR_ORPHAN at the next
    synchronising call; the oracle finds orphans for the same placement."""
    import ctypes
    case = wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=1, amp=0.5)
    s = U.Solver(case, U.FP64, stream=torch.cuda.Stream())
    t1 = 0.25 / case.meta["freq"]
    A = np.ascontiguousarray(case.motion(t1), dtype=np.float64)
    ctxs = (ctypes.c_void_p * 1)(s.ctx.value)
    tn = (ctypes.c_double * 1)(t1)
    aff = (ctypes.POINTER(ctypes.c_double) * 1)(A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    failed = ctypes.c_int(7)
    assert U.load().ugks_advance_batch(ctxs, 1, tn, aff, 1, ctypes.byref(failed)) == U.OK
    assert failed.value == -1
    with pytest.raises(U.UgksError) as err:
        s.moments()
    assert err.value.code == -4
    topo = mesh.Topology(case.blocks)
    c0 = overset.connect(topo, case.nodes_at(0.0))
    c1 = overset.connect(topo, case.nodes_at(t1), c0.status)
    assert c1.n_orphan > 0


@pytest.mark.parametrize("tile", range(3))
def test_face_tile_shapes_agree(tile):
    """Every tile shape the autotuner may give the FP32 face kernels
    (velocities per chunk x threads per face slot) computes the same step up
    to the rounding of the face sums, and matches the oracle."""
    case = small_mems(nv=12)
    prim = wl.random_prim(case, 29, amp_rho=0.05, amp_u=0.05, amp_T=0.05)
    b = U.Solver(case, U.FP32, prim=prim)
    os.environ["UGKS_FACE_TILE"] = str(tile)
    try:
        c = U.Solver(case, U.FP32, prim=prim)
    finally:
        del os.environ["UGKS_FACE_TILE"]
    r = Run(case, prim)
    for _ in range(2):
        b.advance()
        c.advance()
        r.step()
    Wc = c.moments()[0]
    field = r.status == 0
    assert rel(Wc, b.moments()[0]) < 1e-6
    assert rel(Wc[field], r.state.W[field]) < 1e-5


@pytest.mark.parametrize("prec", [U.FP32, U.BF16F])
def test_four_velocities_per_sweep_thread(prec):
    """The FP32 sweeps with four velocities per lane (a choice the autotuner
    may make) compute what the default two compute."""
    case = small_mems(nv=10)
    prim = wl.random_prim(case, 23, amp_rho=0.05, amp_u=0.05, amp_T=0.05)
    b = U.Solver(case, prec, prim=prim)
    os.environ["UGKS_SWEEP_VPT"] = "4"
    try:
        c = U.Solver(case, prec, prim=prim)
    finally:
        del os.environ["UGKS_SWEEP_VPT"]
    for _ in range(2):
        b.advance()
        c.advance()
    Wb = b.moments()[0]
    assert rel(c.moments()[0], Wb) < 1e-6
    if prec == U.FP32:
        r = Run(case, prim)
        r.step()
        r.step()
        field = r.status == 0
        assert rel(c.moments()[0][field], r.state.W[field]) < 1e-5


@pytest.mark.parametrize("u0,omega0", [((0.3, 0.1), 0.0), ((0.0, 0.0), 2.0)])
def test_free_particle_coupled_motion(u0, omega0):
    """Newton-Euler coupling (Sec. 3 Step 1): a rigid particle moved by the
    wall force and torque from the library (ugks_moments, ugks_wall_torque)
    follows the oracle's coupled run -- same trajectory, connectivity and
    field after three physical steps."""
    from oracle import coupling
    case = wl.particle(nbi=48, nbj=24, noi=32, noj=10, nv=8, r_out=0.3, n_inner=2, u0=u0,
                       omega0=omega0)
    m = case.meta
    body = U.RigidBody(m["body_block"], m["mass"], m["inertia"], m["center"], m["u0"], m["omega0"])
    ref_body = coupling.Body(m["body_block"], m["mass"], m["inertia"], m["center"], velocity=m["u0"],
                             omega=m["omega0"])
    s = U.Solver(case, U.FP64)
    r = coupling.CoupledRun(case, [ref_body])
    for _ in range(3):
        s.advance_coupled([body])
        r.step_coupled()
    assert np.allclose(body.vel, ref_body.V, rtol=1e-10, atol=1e-13)
    assert abs(body.omega - ref_body.w) < 1e-10 * max(abs(ref_body.w), 1e-3)
    assert np.allclose(body.disp, ref_body.d, rtol=1e-10, atol=1e-14)
    assert abs(body.angle - ref_body.a) < 1e-12
    W, q, st, wall = s.moments()
    assert np.array_equal(st, r.status)
    field = r.status == 0
    assert rel(W[field], r.state.W[field]) < 1e-11


@pytest.mark.parametrize("which", ["mems", "tsto"])
def test_full_size_rest_state_stays_at_rest(which):
    """At the full sizes and launch configuration the bench times (tiled
    flux, sweep tiles, overset assembly and interpolation of every block):
    a Maxwellian at rest with walls at the gas temperature and no motion is
    a steady solution, so after two physical steps the FP32 path keeps rho,
    T = 1 and V = 0 up to the velocity quadrature defect and FP32 rounding
    (a property that holds at any size, checked where the oracle cannot
    run)."""
    case = wl.mems(mach=0.0, Tw=1.0) if which == "mems" else wl.tsto(mach=0.0, pitch_rate=0.0)
    s = U.Solver(case, U.FP32)
    for _ in range(2):
        s.advance()
    W, q, st, wall = s.moments()
    field = st == 0
    rho = W[field, 0]
    V = W[field, 1:3] / rho[:, None]
    e = W[field, 3] / rho - 0.5 * (V * V).sum(1)
    T = 2.0 * e / (3.0 + case.K)
    assert np.isfinite(W).all()
    assert np.abs(rho - 1.0).max() < 1e-5
    assert np.abs(T - 1.0).max() < 1e-5
    assert np.abs(V).max() < 1e-5


def test_second_move_replaces_the_pending_one():
    """Moving twice before a step keeps the old level at t: the geometry
    equals that of the second move alone (discrete GCL intact)."""
    case = small_mems()
    a = U.Solver(case, U.FP64)
    b = U.Solver(case, U.FP64)
    t1, t2 = 0.3 * case.dt, case.dt
    a.move_mesh(t1)
    a.move_mesh(t2)
    b.move_mesh(t2)
    ga, gb = a.geometry(), b.geometry()
    for k in ("vol_old", "vol_new", "Sn", "SUn", "dts"):
        assert np.array_equal(ga[k], gb[k]), k


def test_channel_full_configuration_fp64():
    """The plain-FP64 channel configuration at its full size (64x32 cells,
    24x24 velocities on [-5, 5], 10 inner iterations, seeded density noise,
    oscillating top wall): one physical step agrees with the oracle field by
    field."""
    case = wl.channel()
    s = U.Solver(case, U.FP64)
    r = Run(case)
    s.advance()
    r.step()
    f, W, q = s.get_state()
    assert rel(W, r.state.W) < 1e-11
    assert rel(f.cpu().numpy(), r.state.f) < 1e-11
