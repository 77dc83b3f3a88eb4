"""Pins of the oracle's kinetic model against quantities the paper and the
mathematics fix independently of the oracle's own formulas (CPU only)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import kinetic as kn

pytestmark = pytest.mark.cpu


def wide_dvs(n=64, L=10.0):
    return kn.make_dvs(n, n, -L, L, -L, L)


GASES = [kn.Gas(0, 2.0 / 3.0, 0.81, 0.05), kn.Gas(2, 0.72, 0.74, 0.02)]


@pytest.mark.parametrize("gas", GASES)
def test_maxwellian_discrete_moments(gas):
    """Trapezoid moments of the reduced Maxwellian on a wide grid reproduce W
    (spectral accuracy) and give zero heat flux (Sec. 2.1, W = int Psi f)."""
    dvs = wide_dvs()
    rho, Vx, Vy, lam = 1.3, 0.4, -0.7, 0.45
    g = kn.maxwellian(rho, Vx, Vy, lam, dvs, gas)
    W = kn.moments(g, dvs)
    Wref = kn.conservative(rho, Vx, Vy, lam, gas)
    np.testing.assert_allclose(W, Wref, rtol=1e-13, atol=1e-13)
    q = kn.heat_flux(g, Vx, Vy, dvs)
    np.testing.assert_allclose(q, 0.0, atol=1e-13)
    # rho E = rho|V|^2/2 + (D + Keff) p / 2  <=>  gamma = (K+5)/(K+3)
    assert gas.gamma == pytest.approx((gas.K + 5.0) / (gas.K + 3.0), rel=1e-15)


def test_shakhov_reduction_bruteforce():
    """Integrating the full Shakhov f+ = g[1 + (1-Pr) c.q (c^2/RT - 5)/(5pRT)]
    (Sec. 2.1) over the internal variable (K = 0: the out-of-plane velocity,
    Keff = 1) by brute-force quadrature gives the printed reduced H+ and B+."""
    gas = GASES[0]
    rho, Vx, Vy, lam = 0.9, 0.2, -0.3, 0.7
    qx, qy = 0.05, -0.08
    T = 1.0 / (2.0 * lam)
    p = rho * T
    rng = np.random.default_rng(3)
    vx = rng.uniform(-3, 3, 7)
    vy = rng.uniform(-3, 3, 7)
    dvs = kn.Dvs(vx, vy, np.ones(7))
    got = kn.maxwellian(rho, Vx, Vy, lam, dvs, gas) + kn.shakhov_part(
        rho, Vx, Vy, lam, qx, qy, dvs, gas)
    xi = np.linspace(-14 * math.sqrt(T), 14 * math.sqrt(T), 20001)
    for k in range(7):
        cx, cy = vx[k] - Vx, vy[k] - Vy
        c2 = cx * cx + cy * cy + xi * xi
        g = rho * (lam / math.pi) ** 1.5 * np.exp(-lam * c2)
        fp = g * (1.0 + (1.0 - gas.Pr) * (cx * qx + cy * qy) * (c2 / T - 5.0) / (5.0 * p * T))
        Hb = integrate.trapezoid(fp, xi)
        Bb = integrate.trapezoid(xi * xi * fp, xi)
        assert got[k, 0] == pytest.approx(Hb, rel=1e-11)
        assert got[k, 1] == pytest.approx(Bb, rel=1e-11)


@pytest.mark.parametrize("gas", GASES)
def test_shakhov_part_moments(gas):
    """g+ carries no mass, momentum or energy and its heat flux is (1-Pr) q,
    the Shakhov model's defining property, for K = 0 and K = 2 with the
    printed reduced B+ (Sec. 2.1)."""
    dvs = wide_dvs()
    rho, Vx, Vy, lam = 1.1, -0.3, 0.5, 0.6
    qx, qy = 0.07, -0.04
    gp = kn.shakhov_part(rho, Vx, Vy, lam, qx, qy, dvs, gas)
    np.testing.assert_allclose(kn.moments(gp, dvs), 0.0, atol=1e-13)
    q = kn.heat_flux(gp, Vx, Vy, dvs)
    np.testing.assert_allclose(q, [(1 - gas.Pr) * qx, (1 - gas.Pr) * qy], rtol=1e-11)


@pytest.mark.parametrize("gas", GASES)
def test_micro_slope_is_directional_derivative(gas):
    """g (a.Psi) with a = M^-1 dW equals the derivative of the reduced
    Maxwellian along dW, by central finite differences of H and B."""
    dvs = kn.make_dvs(9, 9, -3, 3, -3, 3)
    W = kn.conservative(1.2, 0.3, -0.2, 0.55, gas)
    dW = np.array([0.3, -0.2, 0.15, 0.4])
    a = kn.micro_slope(W, dW, gas)
    rho, Vx, Vy, lam = kn.primitive(W, gas)
    g = kn.maxwellian(rho, Vx, Vy, lam, dvs, gas)
    ga = kn.slope_times_g(a, g, lam, dvs, gas)
    eps = 1e-6

    def gm(Wx):
        return kn.maxwellian(*kn.primitive(Wx, gas), dvs, gas)

    fd = (gm(W + eps * dW) - gm(W - eps * dW)) / (2 * eps)
    np.testing.assert_allclose(ga, fd, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("gas", GASES)
def test_time_slope_compatibility(gas):
    """A from compatibility: sum_k V_k Psi_k [(a.Psi) w.grad + (A.Psi)] g = 0
    on a wide discrete grid, with w = v - U for a moving face."""
    dvs = wide_dvs()
    W = kn.conservative(0.8, 0.5, 0.1, 0.4, gas)
    ax = kn.micro_slope(W, np.array([0.1, 0.2, -0.1, 0.3]), gas)
    ay = kn.micro_slope(W, np.array([-0.2, 0.05, 0.1, -0.1]), gas)
    Ux, Uy = 0.3, -0.6
    A = kn.time_slope(W, ax, ay, Ux, Uy, gas)
    rho, Vx, Vy, lam = kn.primitive(W, gas)
    g = kn.maxwellian(rho, Vx, Vy, lam, dvs, gas)
    wx = (dvs.vx - Ux)[:, None]
    wy = (dvs.vy - Uy)[:, None]
    tot = (wx * kn.slope_times_g(ax, g, lam, dvs, gas) + wy * kn.slope_times_g(ay, g, lam, dvs, gas)
           + kn.slope_times_g(A, g, lam, dvs, gas))
    np.testing.assert_allclose(kn.moments(tot, dvs), 0.0, atol=1e-12)


@pytest.mark.parametrize("x", [1e-9, 1e-4, 0.3, 0.999, 1.001, 4.0, 80.0])
def test_time_integrals_quadrature(x):
    """q_m = int_0^dts c_m(t) dt of the coefficients of Eq. fullSolution, by
    adaptive quadrature."""
    dts = 0.37
    tau = dts / x
    c = [lambda t: math.exp(-t / tau), lambda t: -t * math.exp(-t / tau),
         lambda t: -math.expm1(-t / tau), lambda t: t * math.exp(-t / tau) + tau * math.expm1(-t / tau),
         lambda t: t + tau * math.expm1(-t / tau)]
    q = kn.time_integrals(dts, tau)
    for m in range(5):
        ref, err = integrate.quad(c[m], 0.0, dts, epsabs=1e-17, epsrel=1e-13, limit=200)
        scale = dts if m in (0, 2) else dts * dts
        assert abs(float(q[m]) - ref) <= 1e-13 * scale, (m, float(q[m]), ref)


def test_time_integrals_limits():
    """tau -> inf (free transport): q1 -> dts, q2 -> -dts^2/2, others -> 0;
    tau -> 0 (continuum): q3 -> dts, q5 -> dts^2/2, q1, q2, q4 -> 0."""
    dts = 0.2
    q = kn.time_integrals(dts, 1e14)
    np.testing.assert_allclose([float(v) for v in q], [dts, -dts * dts / 2, 0, 0, 0], atol=1e-14)
    q = kn.time_integrals(dts, 1e-14)
    np.testing.assert_allclose([float(v) for v in q], [0, 0, dts, 0, dts * dts / 2], atol=1e-13)
    # sum of the f and g weights is the step: q1 + q3 = dts
    for x in (1e-3, 0.5, 3.0):
        q = kn.time_integrals(dts, dts / x)
        assert float(q[0] + q[2]) == pytest.approx(dts, rel=1e-15)


def test_collision_time_vhs():
    """tau = mu/p with mu = mu_ref T^omega (VHS); a Maxwellian at T = 1,
    rho = 1 relaxes with tau = mu_ref."""
    gas = kn.Gas(0, 2 / 3, 0.81, 0.123)
    assert float(kn.collision_time(1.0, 0.5, gas)) == pytest.approx(0.123, rel=1e-15)
    assert float(kn.collision_time(2.0, 0.25, gas)) == pytest.approx(0.123 * 2 ** 0.81 / 4, rel=1e-14)
