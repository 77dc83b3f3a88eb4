"""Pins of what the oracle's inner iteration converges TO (Sec. 2.2) and of
its reconstruction limiter (Sec. 2.1, reading R1), CPU only.

* the dual-time fixed point satisfies the Crank-Nicolson equations of the
  physical step, assembled here independently from single flux and Shakhov
  evaluations (backward Euler or a dropped 1/2 fails it);
* a spatially uniform non-equilibrium perturbation relaxes by the
  Crank-Nicolson amplification factor (1 - dt/2tau)/(1 + dt/2tau);
* the limited slope is the van Leer mean 2ab/(a+b) of the two one-sided
  differences, zero at an extremum, one-sided next to a missing neighbour.
"""
import numpy as np
import pytest

from oracle import kinetic as kn
from oracle import mesh, ugks
from paper_2604_09984_gb300 import workloads as wl

GAS = kn.Gas(0, 2.0 / 3.0, 0.81, 0.05 * 1.0339)


def _setup(blocks, gas, dvs, W_inf):
    return ugks.Setup(mesh.Topology(blocks), gas, dvs, np.asarray(W_inf, dtype=np.float64))


def _random_state(setup, seed, amp=0.1):
    rng = np.random.default_rng(seed)
    nc = setup.topo.nc
    p = np.empty((nc, 4))
    p[:] = (1.0, 0.0, 0.0, 1.0)
    p[:, 0] *= 1 + rng.uniform(-amp, amp, nc)
    p[:, 1] += rng.uniform(-amp, amp, nc)
    p[:, 2] += rng.uniform(-amp, amp, nc)
    p[:, 3] *= 1 + rng.uniform(-amp, amp, nc)
    st = ugks.initial_state(setup, p)
    st.f *= 1 + rng.uniform(-0.05, 0.05, st.f.shape)
    st.W = kn.moments(st.f, setup.dvs)
    _, Vx, Vy, _ = kn.primitive(st.W, setup.gas)
    st.q = kn.heat_flux(st.f, Vx, Vy, setup.dvs)
    return st


def _collision(setup, f, W, q):
    """Q = (f+(W, q) - f) / tau(W)  (Sec. 2.1, Shakhov relaxation term)."""
    rho, _, _, lam = kn.primitive(W, setup.gas)
    tau = kn.collision_time(rho, lam, setup.gas)
    return (kn.shakhov_equilibrium(W, q, setup.dvs, setup.gas) - f) / tau[:, None, None]


def test_fixed_point_solves_crank_nicolson_system():
    """Sec. 2.2: at dual-time convergence the step solves
    (Om1 f1 - Om0 f0)/dt + (D1 + D0)/2 - (Om1 Q1 + Om0 Q0)/2 = 0
    with D the flux divergence and Q the collision term of each level, the
    macroscopic state W1 = sum V Psi f1 and q1 the heat flux of f1 about the
    velocity of W1 (reading R7).  Moving, deforming mesh; 3x2 cells."""
    ni, nj = 3, 2
    case = wl.channel(ni=ni, nj=nj, nv=8, Kn=0.05)
    blk = case.blocks[0]
    # spacing 0.5 on [-10, 10]: the trapezoid moments of the Maxwellians are
    # exact to round-off, so the fixed point is the one of the moment system
    dvs = kn.make_dvs(41, 41, -10.0, 10.0, -10.0, 10.0)
    setup = _setup([blk], GAS, dvs, kn.conservative(1.0, 0.0, 0.0, 0.5, GAS))
    topo = setup.topo
    st0 = _random_state(setup, 11)
    dt, t = 0.05, 0.3
    geo = mesh.geometry(topo, case.nodes_at(t), case.nodes_at(t + dt), dt)
    assert np.abs(geo.SUn).max() > 1e-3            # the mesh really moves
    st1, info = ugks.implicit_step(setup, geo, st0, dt, 300)
    status = np.zeros(topo.nc, dtype=np.int64)
    wS = ugks.normal_velocity(setup, geo)
    dts = ugks.explicit_dt(setup, geo, wS)
    D0 = ugks.flux(setup, geo, st0, status, dts, wS).D
    D1 = ugks.flux(setup, geo, st1, status, dts, wS).D
    # the converged state is consistent: W1 are the moments of f1, q1 its
    # heat flux about V1
    np.testing.assert_allclose(st1.W, kn.moments(st1.f, dvs), rtol=1e-12, atol=1e-13)
    _, V1x, V1y, _ = kn.primitive(st1.W, GAS)
    np.testing.assert_allclose(st1.q, kn.heat_flux(st1.f, V1x, V1y, dvs), rtol=1e-10, atol=1e-12)
    Q0 = _collision(setup, st0.f, st0.W, st0.q)
    Q1 = _collision(setup, st1.f, st1.W, st1.q)
    om0 = geo.vol_old[:, None, None]
    om1 = geo.vol_new[:, None, None]
    tdiff = (om1 * st1.f - om0 * st0.f) / dt
    scale = np.abs(tdiff).max() + np.abs(D0).max() + np.abs(om0 * Q0).max()
    cn = tdiff + 0.5 * (D1 + D0) - 0.5 * (om1 * Q1 + om0 * Q0)
    assert np.abs(cn).max() < 1e-12 * scale
    # the same state violates backward Euler and a CN without the 1/2
    be = tdiff + D1 - om1 * Q1
    half = tdiff + (D1 + D0) - (om1 * Q1 + om0 * Q0)
    assert np.abs(be).max() > 1e-4 * scale
    assert np.abs(half).max() > 1e-4 * scale


def _row_perturbation(dvs, eps):
    """delta on the v_y = 0 row of the velocity grid only, even in v_x, with
    zero mass, energy and heat flux (the odd moments vanish by symmetry):
    delta_h = eps e^{-vx^2/2} (vx^2 - c), delta_b = -vx^2 delta_h."""
    row = np.abs(dvs.vy) < 1e-14
    vx = dvs.vx[row]
    w = dvs.w[row]
    e = np.exp(-0.5 * vx * vx)
    c = (w * e * vx * vx).sum() / (w * e).sum()
    d = np.zeros((dvs.nv, 2))
    d[row, 0] = eps * e * (vx * vx - c)
    d[row, 1] = -vx * vx * d[row, 0]
    return d


@pytest.mark.parametrize("dt_over_tau", [0.5, 2.0, 6.0])
def test_uniform_relaxation_crank_nicolson_factor(dt_over_tau):
    """Sec. 2.2 on a spatially uniform state: with no transport (D = 0) the
    Crank-Nicolson step gives f1 - g = r (f0 - g), r = (1 - dt/2tau) /
    (1 + dt/2tau), for a perturbation delta carrying no collision invariant
    and no heat flux (backward Euler would give 1/(1 + dt/tau)).  The
    perturbation lives on the v_y = 0 velocity row, which never crosses the
    far-field j-faces of the x-periodic block, so the boundaries see g only."""
    ni, nj = 4, 3
    blk = wl.BlockSpec(ni, nj, True, (0, 0, wl.BC_FARFIELD, wl.BC_FARFIELD), (0, 0, 0, 0),
                       wl.cartesian_nodes(ni, nj, 0.0, 2.0, 0.0, 1.0))
    dvs = kn.make_dvs(41, 41, -10.0, 10.0, -10.0, 10.0)   # v_y = 0 is a grid row
    W = kn.conservative(1.0, 0.0, 0.0, 0.5, GAS)
    setup = _setup([blk], GAS, dvs, W)
    topo = setup.topo
    X = blk.x_ref
    dt = 0.05
    geo = mesh.geometry(topo, [X], [X], dt)
    rho, _, _, lam = kn.primitive(W, GAS)
    tau = kn.collision_time(rho, lam, GAS)
    gas = kn.Gas(0, GAS.Pr, GAS.omega, GAS.mu_ref * dt / (dt_over_tau * tau))
    setup = _setup([blk], gas, dvs, W)
    tau = kn.collision_time(rho, lam, gas)
    assert tau == pytest.approx(dt / dt_over_tau, rel=1e-14)
    g = kn.maxwellian(1.0, 0.0, 0.0, 0.5, dvs, gas)
    delta = _row_perturbation(dvs, 1e-3)
    np.testing.assert_allclose(kn.moments(delta, dvs), 0.0, atol=1e-18)
    np.testing.assert_allclose(kn.heat_flux(delta, 0.0, 0.0, dvs), 0.0, atol=1e-18)
    f0 = np.repeat((g + delta)[None], topo.nc, 0)
    Wd = kn.moments(f0, dvs)
    st = ugks.State(f0, Wd, np.zeros((topo.nc, 2)))
    setup.farfield_W = Wd[0].copy()
    st1, _ = ugks.implicit_step(setup, geo, st, dt, 60)
    r = (1.0 - 0.5 * dt / tau) / (1.0 + 0.5 * dt / tau)
    g_d = kn.maxwellian(*kn.primitive(Wd[0], gas), dvs, gas)
    expect = g_d + r * (f0[0] - g_d)
    np.testing.assert_allclose(st1.f, np.repeat(expect[None], topo.nc, 0), rtol=0,
                               atol=1e-12 * np.abs(delta).max())
    be = 1.0 / (1.0 + dt / tau)
    assert abs(be - r) * np.abs(delta).max() > 1e-6


def test_limiter_is_van_leer():
    """Reading R1 on a Cartesian row (spacing h): the limited slope of cell i
    is 2ab/((a+b) h) with a, b the backward and forward differences when they
    share a sign, zero at an extremum, and the one-sided difference where a
    side has no neighbour (wall or hole).  Minmod (min(a, b)/h) or an
    unlimited centre difference ((a+b)/2h) would fail."""
    ni, nj = 7, 1
    h = 2.0 / ni
    blk = wl.BlockSpec(ni, nj, False, (wl.BC_WALL, wl.BC_WALL, wl.BC_WALL, wl.BC_WALL), (1, 1, 1, 1),
                       wl.cartesian_nodes(ni, nj, 0.0, 2.0, 0.0, 1.0))
    dvs = kn.make_dvs(4, 4, -1, 1, -1, 1)
    setup = _setup([blk], GAS, dvs, kn.conservative(1.0, 0.0, 0.0, 0.5, GAS))
    topo = setup.topo
    X = blk.x_ref
    geo = mesh.geometry(topo, [X], [X], 1.0)
    # kinked, with a maximum at cell 4
    phi = np.array([0.0, 1.0, 3.0, 3.5, 4.0, 2.0, 1.5])
    status = np.zeros(topo.nc, dtype=np.int64)
    gr = ugks.gradients(setup, geo, phi[:, None], np.zeros((topo.nf, 1)), status)[:, 0, :]
    for i in range(ni):
        if i == 0:
            want = (phi[1] - phi[0]) / h
        elif i == ni - 1:
            want = (phi[i] - phi[i - 1]) / h
        else:
            a, b = phi[i] - phi[i - 1], phi[i + 1] - phi[i]
            want = 2.0 * a * b / ((a + b) * h) if a * b > 0 else 0.0
        assert gr[i, 0] == pytest.approx(want, rel=1e-13, abs=1e-14)
        assert abs(gr[i, 1]) < 1e-14
    # a hole on one side makes the slope one-sided
    status[3] = ugks.HOLE
    gr = ugks.gradients(setup, geo, phi[:, None], np.zeros((topo.nf, 1)), status)[:, 0, :]
    assert gr[2, 0] == pytest.approx((phi[2] - phi[1]) / h, rel=1e-13)
    assert gr[4, 0] == pytest.approx((phi[5] - phi[4]) / h, rel=1e-13)
