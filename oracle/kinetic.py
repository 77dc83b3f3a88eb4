"""Kinetic model of the oracle (test infrastructure; see ``oracle/__init__``).

Plain FP64 numpy.  Notation: D = 2 spatial dimensions, K internal degrees of
freedom, Keff = 3 - D + K the number of components of the internal variable
xi that the reduced distributions h = int f dxi and b = int xi^2 f dxi
integrate out (Sec. 2.1, reduced distributions).  R = 1.
Particle velocity v, gas (macroscopic) velocity V, mesh/face velocity U,
relative velocity w = v - U.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

D = 2


@dataclass(frozen=True)
class Gas:
    """Gas model constants (Sec. 2.1: Shakhov model; VHS viscosity law)."""
    K: int          # internal degrees of freedom
    Pr: float       # Prandtl number
    omega: float    # viscosity exponent mu = mu_ref T^omega
    mu_ref: float   # viscosity at T = 1

    @property
    def Keff(self) -> int:
        # Sec. 2.1, reduced Maxwellian: B = (3 - D + K)/(2 lambda) H
        return 3 - D + self.K

    @property
    def gamma(self) -> float:
        n = D + self.Keff
        return (n + 2.0) / n


@dataclass(frozen=True)
class Dvs:
    """Discrete velocity space: nodes v_k and weights V_k (Sec. 2.1, the
    velocity cells delta v_k with weight V_k).  Tensor-product uniform grid,
    trapezoid weights, index k = iy * nvx + ix."""
    vx: np.ndarray
    vy: np.ndarray
    w: np.ndarray

    @property
    def nv(self) -> int:
        return self.vx.size


def make_dvs(nvx, nvy, xmin, xmax, ymin, ymax) -> Dvs:
    ux = np.array([xmin + (xmax - xmin) * i / (nvx - 1) for i in range(nvx)])
    uy = np.array([ymin + (ymax - ymin) * i / (nvy - 1) for i in range(nvy)])
    wx = np.full(nvx, (xmax - xmin) / (nvx - 1))
    wy = np.full(nvy, (ymax - ymin) / (nvy - 1))
    wx[0] *= 0.5
    wx[-1] *= 0.5
    wy[0] *= 0.5
    wy[-1] *= 0.5
    vx = np.tile(ux, nvy)
    vy = np.repeat(uy, nvx)
    w = np.outer(wy, wx).ravel()
    return Dvs(vx, vy, w)


# ---------------------------------------------------------------- primitives
def primitive(W, gas: Gas):
    """(rho, Vx, Vy, lambda) from W = (rho, rho V, rho E) (Sec. 2.1, W and
    lambda = m/(2 k_B T)); rho E = rho |V|^2/2 + (D + Keff) rho/(4 lambda)."""
    W = np.asarray(W, dtype=np.float64)
    rho = W[..., 0]
    Vx = W[..., 1] / rho
    Vy = W[..., 2] / rho
    eint = W[..., 3] - 0.5 * rho * (Vx * Vx + Vy * Vy)
    lam = (D + gas.Keff) * rho / (4.0 * eint)
    return rho, Vx, Vy, lam


def conservative(rho, Vx, Vy, lam, gas: Gas):
    rho = np.asarray(rho, dtype=np.float64)
    E = 0.5 * rho * (Vx * Vx + Vy * Vy) + (D + gas.Keff) * rho / (4.0 * lam)
    return np.stack([rho, rho * Vx, rho * Vy, E], axis=-1)


def pressure(W, gas: Gas):
    rho, Vx, Vy, lam = primitive(W, gas)
    return rho / (2.0 * lam)


def collision_time(rho, lam, gas: Gas):
    """tau = mu(T)/p with mu = mu_ref T^omega, T = 1/(2 lambda), p = rho T."""
    T = 1.0 / (2.0 * lam)
    return gas.mu_ref * T ** gas.omega / (rho * T)


# ----------------------------------------------------------- equilibria
def maxwellian(rho, Vx, Vy, lam, dvs: Dvs, gas: Gas):
    """Reduced Maxwellian (Sec. 2.1): H = rho (lam/pi)^{D/2} exp(-lam |v-V|^2),
    B = Keff/(2 lam) H.  Broadcasts parameters of shape S to S + (nv,);
    returns an array S + (nv, 2) holding (H, B)."""
    rho, Vx, Vy, lam = (np.asarray(a, dtype=np.float64)[..., None]
                        for a in (rho, Vx, Vy, lam))
    cx = dvs.vx - Vx
    cy = dvs.vy - Vy
    H = rho * (lam / np.pi) * np.exp(-lam * (cx * cx + cy * cy))
    B = gas.Keff / (2.0 * lam) * H
    return np.stack([H, B], axis=-1)


def shakhov_part(rho, Vx, Vy, lam, qx, qy, dvs: Dvs, gas: Gas):
    """Reduced Shakhov correction (H+, B+) exactly as printed in Sec. 2.1:
    H+ = 4(1-Pr) lam^2/(5 rho) (c.q) (2 lam c^2 - 2 - D) H,
    B+ = 4(1-Pr) lam^2/(5 rho) (c.q) {[2 lam c^2 - D](3-D+K) - 2K} H/(2 lam),
    with c = v - V the peculiar velocity (gas velocity V)."""
    rho, Vx, Vy, lam, qx, qy = (np.asarray(a, dtype=np.float64)[..., None]
                                for a in (rho, Vx, Vy, lam, qx, qy))
    cx = dvs.vx - Vx
    cy = dvs.vy - Vy
    c2 = cx * cx + cy * cy
    H = rho * (lam / np.pi) * np.exp(-lam * c2)
    P = 4.0 * (1.0 - gas.Pr) * lam * lam / (5.0 * rho)
    cq = cx * qx + cy * qy
    Hp = P * cq * (2.0 * lam * c2 - 2.0 - D) * H
    Bp = P * cq * ((2.0 * lam * c2 - D) * gas.Keff - 2.0 * gas.K) * H / (2.0 * lam)
    return np.stack([Hp, Bp], axis=-1)


def shakhov_equilibrium(W, q, dvs: Dvs, gas: Gas):
    """f+ = g + g+ (Sec. 2.1) in reduced form, from W and heat flux q."""
    rho, Vx, Vy, lam = primitive(W, gas)
    q = np.asarray(q, dtype=np.float64)
    return (maxwellian(rho, Vx, Vy, lam, dvs, gas)
            + shakhov_part(rho, Vx, Vy, lam, q[..., 0], q[..., 1], dvs, gas))


# ---------------------------------------------------------------- moments
def moments(f, dvs: Dvs):
    """W = sum_k V_k Psi_k f_k with Psi = (1, v, (v^2 + xi^2)/2) in reduced
    form: (sum h, sum vx h, sum vy h, sum (|v|^2 h + b)/2)  (Sec. 2.1 and
    Eq. macroscopicFlux).  f has shape S + (nv, 2)."""
    h = f[..., 0]
    b = f[..., 1]
    w = dvs.w
    return np.stack([
        (w * h).sum(-1),
        (w * dvs.vx * h).sum(-1),
        (w * dvs.vy * h).sum(-1),
        (w * 0.5 * ((dvs.vx ** 2 + dvs.vy ** 2) * h + b)).sum(-1),
    ], axis=-1)


def heat_flux(f, Vx, Vy, dvs: Dvs):
    """q = (1/2) sum_k V_k c (|c|^2 h + b), c = v - V (Sec. 2.1)."""
    Vx = np.asarray(Vx, dtype=np.float64)[..., None]
    Vy = np.asarray(Vy, dtype=np.float64)[..., None]
    cx = dvs.vx - Vx
    cy = dvs.vy - Vy
    c2 = cx * cx + cy * cy
    e = c2 * f[..., 0] + f[..., 1]
    return np.stack([0.5 * (dvs.w * cx * e).sum(-1),
                     0.5 * (dvs.w * cy * e).sum(-1)], axis=-1)


# --------------------------------------------- continuous Gaussian moments
_GH_S, _GH_W = np.polynomial.hermite.hermgauss(8)


def _gaussian_expectations(Vx, Vy, lam, Keff):
    """Expectation operator of the normalised Gaussian g/rho over (u, v, xi):
    u, v ~ N(V, 1/(2 lam)), Z = |xi|^2 with E Z = Keff/(2 lam),
    E Z^2 = Keff (Keff + 2)/(4 lam^2).  Returns (U, Vv, wt, EZ, EZ2) so that
    E[p0 + p1 Z + p2 Z^2] = sum wt (p0 + p1 EZ + p2 EZ2) for polynomials p_i
    in (u, v) evaluated on the tensor Gauss-Hermite grid (exact to degree 15).
    Parameters of shape S give grids of shape S + (8, 8)."""
    Vx, Vy, lam = (np.asarray(a, dtype=np.float64)[..., None, None] for a in (Vx, Vy, lam))
    r = 1.0 / np.sqrt(lam)
    U = Vx + _GH_S[:, None] * r
    Vv = Vy + _GH_S[None, :] * r
    U, Vv = np.broadcast_arrays(U, Vv)
    wt = np.outer(_GH_W, _GH_W) / math.pi
    EZ = Keff / (2.0 * lam)
    EZ2 = Keff * (Keff + 2.0) / (4.0 * lam * lam)
    return U, Vv, wt, EZ, EZ2


def moment_matrices(rho, Vx, Vy, lam, gas: Gas):
    """M_ab = int Psi_a Psi_b g,  Nx_ab = int u Psi_a Psi_b g,
    Ny_ab = int v Psi_a Psi_b g  over (u, v, xi).  Parameters of shape S give
    matrices of shape S + (4, 4)."""
    U, Vv, wt, EZ, EZ2 = _gaussian_expectations(Vx, Vy, lam, gas.Keff)
    rho = np.asarray(rho, dtype=np.float64)
    one = np.ones_like(U)
    zero = np.zeros_like(U)
    # Psi_a = c0 + c1 Z
    psi = [(one, zero), (U, zero), (Vv, zero), (0.5 * (U * U + Vv * Vv), 0.5 * one)]

    def expect(p0, p1, p2):
        return (wt * (p0 + p1 * EZ + p2 * EZ2)).sum(axis=(-2, -1))

    shape = rho.shape + (4, 4)
    M = np.empty(shape)
    Nx = np.empty(shape)
    Ny = np.empty(shape)
    for a in range(4):
        for b in range(4):
            a0, a1 = psi[a]
            b0, b1 = psi[b]
            p0 = a0 * b0
            p1 = a0 * b1 + a1 * b0
            p2 = a1 * b1
            M[..., a, b] = rho * expect(p0, p1, p2)
            Nx[..., a, b] = rho * expect(U * p0, U * p1, U * p2)
            Ny[..., a, b] = rho * expect(Vv * p0, Vv * p1, Vv * p2)
    return M, Nx, Ny


def _solve(M, r):
    return np.linalg.solve(M, r[..., None])[..., 0]


def micro_slope(W0, dW, gas: Gas):
    """Micro-slope a with int Psi (a.Psi) g0 = dW (the spatial derivative of
    the interface equilibrium, Sec. 2.1 'equilibrium state is approximated',
    standard UGKS construction).  W0: (..., 4); dW: (..., 4)."""
    rho, Vx, Vy, lam = primitive(W0, gas)
    M, _, _ = moment_matrices(rho, Vx, Vy, lam, gas)
    return _solve(M, np.asarray(dW, dtype=np.float64))


def time_slope(W0, ax, ay, Ux, Uy, gas: Gas):
    """A from the compatibility condition int Psi (a.w + A) g0 = 0 with the
    relative velocity w = v - U (moving-frame kinetic equation, Eq. BGK):
    M A = -[(Nx - Ux M) ax + (Ny - Uy M) ay]."""
    rho, Vx, Vy, lam = primitive(W0, gas)
    M, Nx, Ny = moment_matrices(rho, Vx, Vy, lam, gas)
    Ux = np.asarray(Ux, dtype=np.float64)[..., None, None]
    Uy = np.asarray(Uy, dtype=np.float64)[..., None, None]
    rhs = (((Nx - Ux * M) @ np.asarray(ax)[..., None])[..., 0]
           + ((Ny - Uy * M) @ np.asarray(ay)[..., None])[..., 0])
    return -_solve(M, rhs)


def slope_times_g(a, g, lam, dvs: Dvs, gas: Gas):
    """Reduced form of g (a.Psi): integrate g (a0 + a1 u + a2 v +
    a3 (u^2+v^2+xi^2)/2) over xi, and xi^2 times it:
      h part: H [a0 + a1 vx + a2 vy + a3 (|v|^2 + Keff/(2 lam))/2]
      b part: B [a0 + a1 vx + a2 vy + a3 (|v|^2 + (Keff+2)/(2 lam))/2]
    (uses int xi^4 g dxi = (Keff+2)/(2 lam) B).  a: (..., 4); g: (..., nv, 2)."""
    a = np.asarray(a, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)[..., None]
    a0, a1, a2, a3 = (a[..., i][..., None] for i in range(4))
    v2 = dvs.vx ** 2 + dvs.vy ** 2
    base = a0 + a1 * dvs.vx + a2 * dvs.vy + 0.5 * a3 * v2
    sh = base + 0.5 * a3 * gas.Keff / (2.0 * lam)
    sb = base + 0.5 * a3 * (gas.Keff + 2.0) / (2.0 * lam)
    return np.stack([g[..., 0] * sh, g[..., 1] * sb], axis=-1)


# ------------------------------------------------------- time coefficients
def time_integrals(dts, tau, nterms: int = 40):
    """q_m = int_0^{dts} c_m(t) dt for the coefficients of Eq. fullSolution:
      c1 = e^{-t/tau}, c2 = -t e^{-t/tau}, c3 = 1 - e^{-t/tau},
      c4 = t e^{-t/tau} - tau (1 - e^{-t/tau}), c5 = t - tau (1 - e^{-t/tau}).
    Closed forms (x = dts/tau, E = e^{-x}):
      q1 = tau(1-E), q2 = tau(dts+tau)E - tau^2, q3 = dts - tau(1-E),
      q4 = -tau dts (1+E) + 2 tau^2 (1-E), q5 = dts^2/2 - tau dts + tau^2 (1-E);
    for x < 1 the same quantities from their Taylor series in x (the closed
    forms cancel catastrophically there).  Scalars or arrays."""
    dts = np.asarray(dts, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    x = dts / tau
    # closed forms
    E = np.exp(-x)
    em = -np.expm1(-x)
    q1c = tau * em
    q2c = tau * (dts + tau) * E - tau * tau
    q3c = dts - tau * em
    q4c = -tau * dts * (1.0 + E) + 2.0 * tau * tau * em
    q5c = 0.5 * dts * dts - tau * dts + tau * tau * em
    # series: q1 = dts sum_{m>=1} (-1)^{m+1} x^{m-1}/m!
    #         q2 = dts^2 sum_{m>=2} (-1)^{m-1} (m-1) x^{m-2}/m!
    #         q4 = dts^2 sum_{m>=3} (-1)^{m+1} (2-m) x^{m-2}/m!
    #         q5 = dts^2 sum_{m>=3} (-1)^{m+1} x^{m-2}/m!
    xs = np.minimum(x, 1.0)
    s1 = np.zeros_like(xs)
    s2 = np.zeros_like(xs)
    s4 = np.zeros_like(xs)
    s5 = np.zeros_like(xs)
    for m in range(1, nterms):
        fac = math.factorial(m)
        sgn = (-1.0) ** (m + 1)
        s1 = s1 + sgn * xs ** (m - 1) / fac
        if m >= 2:
            s2 = s2 + sgn * (m - 1) * xs ** (m - 2) / fac
        if m >= 3:
            s4 = s4 + sgn * (2 - m) * xs ** (m - 2) / fac
            s5 = s5 + sgn * xs ** (m - 2) / fac
    small = x < 1.0
    q1 = np.where(small, dts * s1, q1c)
    q2 = np.where(small, dts * dts * s2, q2c)
    q3 = np.where(small, dts - dts * s1, q3c)
    q4 = np.where(small, dts * dts * s4, q4c)
    q5 = np.where(small, dts * dts * s5, q5c)
    return q1, q2, q3, q4, q5
