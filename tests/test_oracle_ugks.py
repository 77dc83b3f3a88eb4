"""Pins of the oracle's implicit UGKS step (Sec. 2) on small grids (CPU only):
geometric conservation, free-stream and rest-state preservation, zero wall
penetration, conservative flux form, LU-SGS against a dense solve,
conservation at dual-time convergence, free-molecular and continuum limits."""
import math

import numpy as np
import pytest

from oracle import kinetic as kn
from oracle import mesh, ugks
from paper_2604_09984_gb300 import workloads as wl


def block(ni, nj, periodic=True, bc=(0, 0, wl.BC_WALL, wl.BC_WALL), Tw=(0, 0, 1.0, 1.0),
          L=2.0, H=1.0):
    return wl.BlockSpec(ni, nj, periodic, bc, Tw, wl.cartesian_nodes(ni, nj, 0.0, L, 0.0, H))


def deform(X, t, amp=0.04, walls_fixed=True):
    """Smooth non-affine node motion; x-periodic in [0, 2], vanishing on
    y = 0, 1 when walls_fixed."""
    x, y = X[..., 0], X[..., 1]
    Y = np.sin(math.pi * y) if walls_fixed else 1.0 + 0.3 * y
    out = X.copy()
    out[..., 0] = x + amp * math.sin(3.0 * t + 0.4) * np.sin(math.pi * x) ** 2 * Y
    out[..., 1] = y + amp * math.sin(2.0 * t) * np.cos(math.pi * x) * Y * 0.5
    return out


def make_setup(blocks, gas, dvs, farfield=(1.0, 0.0, 0.0, 1.0)):
    topo = mesh.Topology(blocks)
    r, ux, uy, T = farfield
    Winf = kn.conservative(r, ux, uy, 1.0 / (2.0 * T), gas)
    return ugks.Setup(topo, gas, dvs, Winf)


GAS = kn.Gas(0, 2.0 / 3.0, 0.81, 0.05 * 1.0339)
WIDE = kn.make_dvs(44, 44, -10, 10, -10, 10)
SMALL = kn.make_dvs(12, 12, -5, 5, -5, 5)


def uniform_prim(nc, rho=1.0, ux=0.0, uy=0.0, T=1.0):
    p = np.empty((nc, 4))
    p[:] = (rho, ux, uy, T)
    return p


def test_gcl_nonaffine():
    """Omega^{n+1} - Omega^n = dt sum_faces S U.n, and sum_faces S n = 0 per
    cell, for a non-affine deformation (discrete GCL of the mid-time /
    swept-area geometry)."""
    b = block(7, 5)
    topo = mesh.Topology([b])
    dt = 0.3
    geo = mesh.geometry(topo, [deform(b.x_ref, 0.0)], [deform(b.x_ref, dt)], dt)
    sgn = topo.cell_face_sign
    fsum = (sgn * geo.SUn[topo.cell_faces]).sum(1)
    np.testing.assert_allclose(geo.vol_new - geo.vol_old, dt * fsum, rtol=0, atol=1e-15)
    Ssum = (sgn[..., None] * geo.Sn[topo.cell_faces]).sum(1)
    np.testing.assert_allclose(Ssum, 0.0, atol=1e-15)
    assert np.all(geo.vol_new > 0) and abs(geo.vol_new.sum() - 2.0) < 1e-13


def test_free_stream_preserved_on_deforming_mesh():
    """A uniform equilibrium flow stays uniform on a non-affinely deforming,
    periodic mesh with far-field sides (free-stream preservation)."""
    bc = (0, 0, wl.BC_FARFIELD, wl.BC_FARFIELD)
    b = block(6, 5, True, bc, (0, 0, 0, 0))
    ff = (1.0, 0.3, -0.2, 1.0)
    setup = make_setup([b], GAS, WIDE, ff)
    st = ugks.initial_state(setup, uniform_prim(30, *ff))
    dt = 0.2
    geo = mesh.geometry(setup.topo, [deform(b.x_ref, 0.0, walls_fixed=False)],
                        [deform(b.x_ref, dt, walls_fixed=False)], dt)
    new, _ = ugks.implicit_step(setup, geo, st, dt, 3)
    np.testing.assert_allclose(new.W, st.W, rtol=0, atol=1e-12)
    np.testing.assert_allclose(new.f, st.f, rtol=0, atol=1e-12)


def test_rest_maxwellian_stationary():
    """A Maxwellian at rest with walls at the gas temperature is a steady
    state, also while the interior mesh deforms."""
    b = block(6, 5)
    setup = make_setup([b], GAS, WIDE)
    st = ugks.initial_state(setup, uniform_prim(30))
    dt = 0.25
    for t0 in (0.0, dt):
        geo = mesh.geometry(setup.topo, [deform(b.x_ref, t0)], [deform(b.x_ref, t0 + dt)], dt)
        st2, _ = ugks.implicit_step(setup, geo, st, dt, 3)
        np.testing.assert_allclose(st2.f, st.f, rtol=0, atol=1e-12)
        np.testing.assert_allclose(st2.W, st.W, rtol=0, atol=1e-12)


def random_state(setup, seed, amp=0.15):
    rng = np.random.default_rng(seed)
    nc = setup.topo.nc
    p = uniform_prim(nc)
    p[:, 0] *= 1 + rng.uniform(-amp, amp, nc)
    p[:, 1] += rng.uniform(-amp, amp, nc)
    p[:, 2] += rng.uniform(-amp, amp, nc)
    p[:, 3] *= 1 + rng.uniform(-amp, amp, nc)
    st = ugks.initial_state(setup, p)
    st.f *= 1 + rng.uniform(-0.05, 0.05, st.f.shape)     # non-equilibrium part
    st.W = kn.moments(st.f, setup.dvs)
    rho, Vx, Vy, lam = kn.primitive(st.W, setup.gas)
    st.q = kn.heat_flux(st.f, Vx, Vy, setup.dvs)
    return st


def moving_channel_geo(b, dt, t=0.3):
    case = wl.channel(ni=b.ni, nj=b.nj)
    return mesh.geometry(mesh.Topology([b]), case.nodes_at(t), case.nodes_at(t + dt), dt)


def test_wall_zero_penetration_and_telescoping():
    """Eq. maxWalldes: no net mass crosses any wall face (moving top wall);
    conservative form: interior face fluxes cancel, so the sum of the cell
    divergences equals the sum of wall fluxes (mass: zero)."""
    b = block(6, 5)
    setup = make_setup([b], GAS, SMALL)
    st = random_state(setup, 1)
    geo = moving_channel_geo(b, 0.1)
    wS = ugks.normal_velocity(setup, geo)
    dts = ugks.explicit_dt(setup, geo, wS)
    fl = ugks.flux(setup, geo, st, np.zeros(30, dtype=np.int64), dts, wS)
    scale = np.abs(fl.wall_F).max()
    np.testing.assert_allclose(fl.wall_F[:, 0], 0.0, atol=1e-14 * scale)
    walls = (geo.S[fl.wall_face][:, None] * fl.wall_F).sum(0)
    np.testing.assert_allclose(fl.F.sum(0), walls, atol=1e-13 * np.abs(fl.F).max())
    assert abs(fl.F[:, 0].sum()) < 1e-13 * np.abs(fl.F[:, 0]).max()
    # micro level: interior faces cancel velocity by velocity
    Dsum = fl.D.sum(0)
    assert np.isfinite(Dsum).all()


def _dense_micro(setup, wS, diag, status, k):
    topo = setup.topo
    nc = topo.nc
    Dm = np.diag(diag[:, k])
    Lm = np.zeros((nc, nc))
    Um = np.zeros((nc, nc))
    for c in range(nc):
        for d in range(4):
            fid = topo.cell_faces[c, d]
            sgn = topo.cell_face_sign[c, d]
            nb = topo.face_R[fid] if sgn > 0 else topo.face_L[fid]
            if nb < 0:
                continue
            coef = 0.5 * min(sgn * wS[fid, k], 0.0)
            if nb < c:
                Lm[c, nb] += coef
            elif nb > c:
                Um[c, nb] += coef
    return Dm, Lm, Um


def test_micro_lusgs_equals_dense_factorisation():
    """The sweeps solve (D + L) D^-1 (D + U) x = r with L/U the lower/upper
    lexicographic neighbour couplings (1/2) S min(w_out, 0) of Sec. 2.2."""
    b = block(4, 3)
    setup = make_setup([b], GAS, SMALL)
    geo = moving_channel_geo(b, 0.2)
    wS = ugks.normal_velocity(setup, geo)
    rng = np.random.default_rng(2)
    nc, nv = 12, SMALL.nv
    rhs = rng.normal(size=(nc, nv, 2))
    diag = 5.0 + rng.uniform(0, 1, (nc, nv))
    status = np.zeros(nc, dtype=np.int64)
    d = ugks.micro_lusgs(setup, wS, rhs, diag, status)
    for k in (0, 5, nv - 1):
        Dm, Lm, Um = _dense_micro(setup, wS, diag, status, k)
        A = (Dm + Lm) @ np.linalg.inv(Dm) @ (Dm + Um)
        for comp in range(2):
            np.testing.assert_allclose(d[:, k, comp], np.linalg.solve(A, rhs[:, k, comp]),
                                       rtol=1e-12, atol=1e-14)


def test_macro_lusgs_linear_regime():
    """For small increments the macro sweeps solve (D+L) D^-1 (D+U) dW = R
    with the blocks (1/4) S (J_j - Gamma I), J_j the Jacobian of the ALE
    Euler flux (by finite differences)."""
    b = block(3, 3)
    setup = make_setup([b], GAS, SMALL)
    topo = setup.topo
    geo = moving_channel_geo(b, 0.2)
    st = random_state(setup, 4)
    Gam = ugks.face_gamma(setup, geo, st.W)
    nc = topo.nc
    diag = np.full(nc, 40.0)
    rng = np.random.default_rng(5)
    R = 1e-7 * rng.normal(size=(nc, 4))
    status = np.zeros(nc, dtype=np.int64)
    dW = ugks.macro_lusgs(setup, geo, st.W, R, diag, Gam, status)
    Dm = np.kron(np.diag(diag), np.eye(4))
    Lm = np.zeros((4 * nc, 4 * nc))
    Um = np.zeros((4 * nc, 4 * nc))
    for c in range(nc):
        for d in range(4):
            fid = topo.cell_faces[c, d]
            sgn = topo.cell_face_sign[c, d]
            nb = topo.face_R[fid] if sgn > 0 else topo.face_L[fid]
            if nb < 0:
                continue
            nx, ny = sgn * geo.n[fid]
            un = sgn * geo.SUn[fid] / geo.S[fid]
            J = np.zeros((4, 4))
            for m in range(4):
                e = np.zeros(4)
                e[m] = 1e-6
                J[:, m] = (ugks.euler_flux(st.W[nb] + e, nx, ny, un, GAS)
                           - ugks.euler_flux(st.W[nb] - e, nx, ny, un, GAS)) / 2e-6
            blk = 0.25 * geo.S[fid] * (J - Gam[fid] * np.eye(4))
            tgt = Lm if nb < c else Um
            tgt[4 * c:4 * c + 4, 4 * nb:4 * nb + 4] += blk
    A = (Dm + Lm) @ np.linalg.inv(Dm) @ (Dm + Um)
    ref = np.linalg.solve(A, R.ravel()).reshape(nc, 4)
    np.testing.assert_allclose(dW, ref, rtol=1e-6, atol=1e-15)


def _total(setup, geo_vol, st):
    return (geo_vol[:, None] * st.W).sum(0)


def test_conservation_at_dual_time_convergence():
    """Sum of Omega W is conserved by a physical step once the inner
    iterations converge (Sec. 2.2); walls exchange no mass (Eq. maxWalldes),
    so total mass is conserved on a periodic channel with moving walls."""
    b = block(5, 4)
    gas = kn.Gas(0, 2 / 3, 0.81, 0.1)
    setup = make_setup([b], gas, kn.make_dvs(36, 36, -9, 9, -9, 9))
    st = random_state(setup, 7, amp=0.1)
    geo = moving_channel_geo(b, 0.05)
    m0 = (geo.vol_old * st.W[:, 0]).sum()
    defects = []
    for n_inner in (3, 40):
        st2, _ = ugks.implicit_step(setup, geo, st, 0.05, n_inner)
        defects.append(abs((geo.vol_new * st2.W[:, 0]).sum() - m0) / m0)
    assert defects[1] < 1e-11
    assert defects[1] < defects[0]


def test_dual_time_fixed_point():
    """The inner iteration converges: one more inner step changes nothing
    (its fixed point is the Crank-Nicolson solution of Sec. 2.2)."""
    b = block(4, 3)
    setup = make_setup([b], GAS, SMALL)
    st = random_state(setup, 8, amp=0.05)
    geo = moving_channel_geo(b, 0.05)
    a, _ = ugks.implicit_step(setup, geo, st, 0.05, 50)
    c, _ = ugks.implicit_step(setup, geo, st, 0.05, 51)
    np.testing.assert_allclose(c.f, a.f, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(c.W, a.W, rtol=1e-11, atol=1e-14)


def test_free_molecular_couette_closed_form():
    """Kn -> inf, planar Couette between diffuse walls moving at -U/2 and +U/2:
    the discrete steady state is the half-range wall Maxwellians with equal
    densities (zero net mass flux), uniform in space; it is a fixed point of
    the scheme, and its shear stress matches the continuous free-molecular
    value rho_w U sqrt(RT/(2 pi)) within the velocity quadrature error
    (RT = 1)."""
    U = 0.4
    ni, nj = 2, 6
    X = wl.cartesian_nodes(ni, nj, 0.0, 1.0, 0.0, 1.0)
    b = wl.BlockSpec(ni, nj, True, (0, 0, wl.BC_WALL, wl.BC_WALL), (0, 0, 1.0, 1.0), X)
    gas = kn.Gas(0, 2 / 3, 0.81, 1e12)
    dvs = kn.make_dvs(28, 160, -7, 7, -7, 7)
    setup = make_setup([b], gas, dvs)
    topo = setup.topo
    # walls move tangentially: node x-velocity -U/2 at y = 0, +U/2 at y = 1
    dt = 0.05

    def nodes(t):
        Y = X.copy()
        Y[..., 0] = X[..., 0] + t * U * (X[..., 1] - 0.5)
        return Y

    geo = mesh.geometry(topo, [nodes(0.0)], [nodes(dt)], dt)
    # only the wall faces should move: rebuild with static interior, moving walls
    geo.Uf[:] = 0.0
    geo.SUn[:] = 0.0
    bot = topo.face_side == 2
    top = topo.face_side == 3
    geo.Uf[bot, 0] = -U / 2
    geo.Uf[top, 0] = U / 2
    geo.xc[:] = mesh.vertex_centre(*(topo.concat_nodes([X])[topo.cell_nodes[:, i]] for i in range(4)))
    geo.xf[:] = 0.5 * (topo.concat_nodes([X])[topo.face_a] + topo.concat_nodes([X])[topo.face_b])
    geo.vol_old[:] = geo.vol_new[:] = 1.0 / (ni * nj)
    e = topo.concat_nodes([X])[topo.face_b] - topo.concat_nodes([X])[topo.face_a]
    geo.Sn[:] = np.stack([e[:, 1], -e[:, 0]], -1)
    geo.S[:] = np.hypot(e[:, 0], e[:, 1])
    geo.n[:] = geo.Sn / geo.S[:, None]
    Hb = kn.maxwellian(1.0, -U / 2, 0.0, 0.5, dvs, gas)
    Ht = kn.maxwellian(1.0, U / 2, 0.0, 0.5, dvs, gas)
    up = (dvs.vy > 0)[:, None]
    f = np.where(up, Hb, Ht)
    st = ugks.State(np.repeat(f[None], topo.nc, 0), None, None)
    st.W = kn.moments(st.f, dvs)
    rho, Vx, Vy, lam = kn.primitive(st.W, gas)
    st.q = kn.heat_flux(st.f, Vx, Vy, dvs)
    new, info = ugks.implicit_step(setup, geo, st, dt, 4)
    np.testing.assert_allclose(new.f, st.f, rtol=0, atol=1e-10)
    np.testing.assert_allclose(info.flux_n.wall_rho, 1.0, rtol=1e-12)
    sxy = (dvs.w * dvs.vx * dvs.vy * f[:, 0]).sum()
    # half-range sums converge at second order in the v_y spacing
    assert sxy == pytest.approx(-1.0 * U * math.sqrt(1.0 / (2 * math.pi)), rel=2e-3)


@pytest.mark.parametrize("which", ["shear", "heat"])
def test_continuum_navier_stokes_fluxes(which):
    """Kn -> 0 (dts >> tau): on a linear velocity (temperature) profile the
    UGKS interface flux carries the Navier-Stokes shear stress mu du/dy
    (Fourier heat flux kappa dT/dy, kappa = mu c_p / Pr, c_p = 5/2 R) through
    interior faces; the free-transport weight of the (equilibrium) initial f
    is tau/dts ~ 0.3%."""
    nj = 16
    X = wl.cartesian_nodes(2, nj, 0.0, 1.0, 0.0, 1.0)
    b = wl.BlockSpec(2, nj, True, (0, 0, wl.BC_WALL, wl.BC_WALL), (0, 0, 1.0, 1.0), X)
    mu = 1e-5                           # dts/tau ~ 350: continuum regime
    gas = kn.Gas(0, 2 / 3, 0.0, mu)          # omega = 0: constant viscosity
    dvs = kn.make_dvs(40, 40, -8, 8, -8, 8)
    setup = make_setup([b], gas, dvs)
    topo = setup.topo
    geo = mesh.geometry(topo, [X], [X], 1.0)
    y = geo.xc[:, 1]
    p = uniform_prim(topo.nc)
    G = 0.05
    if which == "shear":
        p[:, 1] = G * (y - 0.5)
    else:
        p[:, 3] = 1.0 + G * (y - 0.5)
        p[:, 0] = 1.0 / p[:, 3]          # uniform pressure
    st = ugks.initial_state(setup, p)
    if which == "heat":
        # cells carry the Navier-Stokes heat flux; the interface Shakhov term
        # (1 - Pr) q0 then lifts the BGK conductivity mu c_p to mu c_p / Pr
        st.q[:, 1] = -mu * 2.5 / gas.Pr * G
    wS = ugks.normal_velocity(setup, geo)
    dts = ugks.explicit_dt(setup, geo, wS)
    # flux through one interior j-face in the middle: isolate it
    fmask = np.zeros(topo.nf, dtype=bool)
    jf = np.nonzero((topo.face_R >= 0) & (np.abs(geo.n[:, 1]) > 0.5)
                    & (np.abs(geo.xf[:, 1] - 0.5) < 1e-12))[0][0]
    fmask[jf] = True
    fl = ugks.flux(setup, geo, st, np.zeros(topo.nc, dtype=np.int64), dts, wS, faces=fmask)
    L = topo.face_L[jf]
    Fface = fl.F[L] / geo.S[jf]       # outward from L (+y)
    if which == "shear":
        # momentum flux of x-momentum through a +y face = -mu du/dy
        assert Fface[1] == pytest.approx(-mu * G, rel=0.02)
    else:
        kappa = mu * 2.5 / gas.Pr
        assert Fface[3] == pytest.approx(-kappa * G, rel=0.02)


def test_step_metrics_vanish_at_rest_and_at_dual_time_convergence():
    """The step metrics (Sec. 2.2): at a rest Maxwellian every residual and
    the moment fix are zero; on a moving channel the macro residual R, the
    micro residual r and the Step-7 fix shrink with the inner iterations and
    vanish at the fixed point (the iteration drives exactly these quantities
    to zero, so a wrong sign or a dropped term in either leaves a finite
    norm), and the field total of Omega^{n+1} rho equals the level-n mass there
    (the conservation of the converged step)."""
    b = block(6, 5)
    setup = make_setup([b], GAS, WIDE)
    st = ugks.initial_state(setup, uniform_prim(30))
    geo = mesh.geometry(setup.topo, [deform(b.x_ref, 0.0)], [deform(b.x_ref, 0.25)], 0.25)
    st2, info = ugks.implicit_step(setup, geo, st, 0.25, 2)
    m = ugks.step_metrics(geo, st2, info, np.zeros(30, dtype=np.int64))
    assert m["res_macro_sq"] < 1e-24 and m["res_micro_sq"] < 1e-24 and m["fix_sq"] < 1e-24
    np.testing.assert_allclose(m["total"], (geo.vol_new[:, None] * st.W).sum(axis=0), rtol=1e-13, atol=1e-14)

    b = block(5, 4)
    gas = kn.Gas(0, 2 / 3, 0.81, 0.1)
    setup = make_setup([b], gas, kn.make_dvs(36, 36, -9, 9, -9, 9))
    st = random_state(setup, 7, amp=0.1)
    geo = moving_channel_geo(b, 0.05)
    status = np.zeros(setup.topo.nc, dtype=np.int64)
    ms = []
    for n_inner in (1, 4, 40):
        st2, info = ugks.implicit_step(setup, geo, st, 0.05, n_inner)
        ms.append(ugks.step_metrics(geo, st2, info, status))
    for k in ("res_macro_sq", "res_micro_sq", "fix_sq"):
        v = [m[k] for m in ms]
        assert v[0] > 0 and v[1] < v[0] and v[2] < 1e-20 * v[0], (k, v)
    m0 = (geo.vol_old * st.W[:, 0]).sum()
    assert abs(ms[2]["total"][0] - m0) < 1e-11 * m0
    assert abs(ms[0]["total"][0] - m0) > abs(ms[2]["total"][0] - m0)
