"""Transposes of the linear operators of the implicit step (test infrastructure;
see ``oracle/__init__``): the first pieces of a discrete adjoint of one step
(Sec. 2.2 and 3.2), written from the forward operators of ``oracle.ugks`` and
``oracle.overset``.  Plain FP64 numpy, no blocking or reordering beyond the
definitions below.

For cotangents y of the outputs these return the cotangents of the inputs,
i.e. A^T y for the linear map A the forward call applies:

  micro_lusgs_transpose  the micro LU-SGS solve d = M^{-1} r of Eq.
                         dualTimeStepping_micro, M = (D + L) D^{-1} (D + U)
                         with the upwind couplings (1/2) min(sgn w_S, 0), per
                         velocity on the solved cells.  M^{-T} = (D + L)^{-T}
                         D (D + U)^{-T}: (D + U)^T is lower triangular (solved
                         in increasing cell order with the couplings a
                         neighbour holds to the cell), (D + L)^T upper
                         (decreasing order).
  interpolate_transpose  the receptor overwrite of Sec. 3.2, phi_r <-
                         sum_j w_rj phi_j (Jacobi: donors read before the
                         pass), identity on every other cell: the receptor's
                         cotangent goes to its donors with the same weights
                         and the receptor keeps none.
  moments_transpose      the velocity moments sum_k V_k Psi_k f_k of the
                         reduced pair (Psi = 1, v, |v|^2/2 on h and 1/2 on b),
                         the linear part of the Step-7 fix.

  euler_flux_jacobian    dF_E/dW of the ALE Euler flux along a face (Sec.
                         2.2, the flux variation of the macro LU-SGS).
  macro_lusgs_tangent,   the macro LU-SGS of Eq. dualTimeStepping_macro as a
  macro_lusgs_adjoint    map R -> dW (W, Gamma, diag fixed) is nonlinear
                         through F_E(W_j + dW_j); linearised at its solution
                         it is (D + U')^{-1} D (D + L')^{-1}, with L' and U'
                         the blocks (1/4) S (A_E(W_j + dW_j) - Gamma I) of
                         the forward (at the forward increments) and the
                         backward pass (at the final increments).  The
                         tangent applies it to dR, the adjoint its transpose
                         (D + L')^{-T} D (D + U')^{-T} to a cotangent of dW.

  moment_fix,            Step 7, W^{s+1} = W' + sum V Psi (f^{s+1} - g(W')),
  moment_fix_tangent,    as a map of (W', f^{s+1}); the derivative of g(W')
  moment_fix_adjoint     along dW' is (a.Psi) g with the micro slope a of
                         int Psi (a.Psi) g = dW' (exact for the Maxwellian),
                         so the tangent is dW' + sum V Psi (df - (a.Psi) g)
                         and the adjoint returns (Wbar - G^T Wbar, the
                         moments' transpose of Wbar) with G the 4 x 4 map
                         dW' -> sum V Psi (a.Psi) g of each cell.

The flux, the interface state and the geometry have no transpose here.
"""
from __future__ import annotations

import numpy as np

from . import kinetic as kn
from .ugks import FIELD, Setup, _cell_links


def micro_lusgs_transpose(setup: Setup, wS, ybar, diag, status):
    """M^{-T} ybar for the micro LU-SGS of ``oracle.ugks.micro_lusgs`` with the
    same (wS, diag, status); arrays (nc, nv, 2), zero on unsolved cells."""
    topo = setup.topo
    cells = [c for c in range(topo.nc) if status[c] == FIELD]
    solved = np.zeros(topo.nc, dtype=bool)
    solved[cells] = True
    links = {c: _cell_links(topo, c) for c in cells}

    def coupling(nb, c):
        """Coupling of cell nb's row to cell c: (1/2) min(sgn_nb w_S, 0) over
        the face they share, sgn_nb the face's sign seen from nb."""
        acc = 0.0
        for fid, sgn, other in links[nb]:
            if other == c:
                acc = acc + 0.5 * np.minimum(sgn * wS[fid], 0.0)
        return acc

    # (D + U)^T a = ybar: U holds the couplings of a row to larger cells, so
    # row c of U^T gathers the rows nb < c that couple to c
    # (a neighbour reached across two faces -- a periodic row of two cells --
    # is one column: coupling() sums its faces)
    nbs = {c: sorted({nb for _, _, nb in links[c] if nb >= 0 and solved[nb]}) for c in cells}
    a = np.zeros_like(ybar)
    for c in cells:
        acc = ybar[c].copy()
        for nb in nbs[c]:
            if nb < c:
                acc -= coupling(nb, c)[:, None] * a[nb]
        a[c] = acc / diag[c][:, None]
    b = a * diag[:, :, None]
    # (D + L)^T z = b: L holds the couplings to smaller cells, so row c of
    # L^T gathers the rows nb > c that couple to c
    z = np.zeros_like(ybar)
    for c in reversed(cells):
        acc = b[c].copy()
        for nb in nbs[c]:
            if nb > c:
                acc -= coupling(nb, c)[:, None] * z[nb]
        z[c] = acc / diag[c][:, None]
    return z


def interpolate_transpose(phibar, cells, donors, weights):
    """Cotangent of the cell values before ``oracle.overset.interpolate`` given
    the cotangent phibar after it (one field: shape (nc, ...)); orphan rows
    (first donor < 0) keep their values, so their cotangent stays."""
    out = phibar.copy()
    for r, c in enumerate(cells):
        if donors[r, 0] < 0:
            continue
        out[c] = 0.0
    for r, c in enumerate(cells):
        if donors[r, 0] < 0:
            continue
        for k in range(donors.shape[1]):
            d = donors[r, k]
            if d < 0:
                continue
            out[d] = out[d] + weights[r, k] * phibar[c]
    return out


def moments_transpose(Wbar, dvs):
    """Cotangent of f (nc, nv, 2) for the moments W = sum_k V_k Psi_k f_k given
    the cotangent Wbar (nc, 4)."""
    v2 = 0.5 * (dvs.vx * dvs.vx + dvs.vy * dvs.vy)
    fbar = np.zeros((Wbar.shape[0], dvs.nv, 2))
    fbar[:, :, 0] = dvs.w[None, :] * (Wbar[:, 0, None] + dvs.vx[None, :] * Wbar[:, 1, None]
                                      + dvs.vy[None, :] * Wbar[:, 2, None] + v2[None, :] * Wbar[:, 3, None])
    fbar[:, :, 1] = dvs.w[None, :] * 0.5 * Wbar[:, 3, None]
    return fbar


def euler_flux_jacobian(W, nx, ny, un, gas):
    """A_E = dF_E/dW (4 x 4) of the Euler flux through a moving face, F_E =
    (rho v_n, m v_n + p n, E v_n + p V.n) with v_n = V.n - U.n and
    p = (gamma - 1)(E - |m|^2 / (2 rho)), written out from the chain rule;
    W of shape (4,)."""
    rho, m1, m2, E = W
    u, v = m1 / rho, m2 / rho
    g1 = gas.gamma - 1.0
    p = g1 * (E - 0.5 * (m1 * m1 + m2 * m2) / rho)
    vabs = u * nx + v * ny
    vn = vabs - un
    dp = np.array([0.5 * g1 * (u * u + v * v), -g1 * u, -g1 * v, g1])
    dvabs = np.array([-vabs / rho, nx / rho, ny / rho, 0.0])
    A = np.zeros((4, 4))
    A[0] = np.array([-un, nx, ny, 0.0])
    A[1] = m1 * dvabs + vn * np.array([0.0, 1.0, 0.0, 0.0]) + nx * dp
    A[2] = m2 * dvabs + vn * np.array([0.0, 0.0, 1.0, 0.0]) + ny * dp
    A[3] = E * dvabs + vn * np.array([0.0, 0.0, 0.0, 1.0]) + vabs * dp + p * dvabs
    return A


def _macro_links(setup, geo, W, Gam, status):
    topo = setup.topo
    cells = [c for c in range(topo.nc) if status[c] == FIELD]
    solved = np.zeros(topo.nc, dtype=bool)
    solved[cells] = True
    links = {c: [(fid, sgn, nb) for fid, sgn, nb in _cell_links(topo, c) if nb >= 0 and solved[nb]]
             for c in cells}
    return cells, links


def _coupling_jacobian(setup, geo, W, Gam, c, fid, sgn, nb, dW):
    """d/d(dW) of the coupling (1/4) S (F_E(W_nb + dW) - F_E(W_nb) - Gamma dW)
    of cell c to its neighbour nb across face fid (outward normal of c)."""
    nx, ny = sgn * geo.n[fid]
    un = sgn * geo.SUn[fid] / geo.S[fid]
    A = euler_flux_jacobian(W[nb] + dW, nx, ny, un, setup.gas)
    return 0.25 * geo.S[fid] * (A - Gam[fid] * np.eye(4))


def _macro_passes(setup, geo, W, R, diag, Gam, status):
    """The forward increments d* and the final increments d of the macro
    LU-SGS, in the order of ``oracle.ugks.macro_lusgs``."""
    from .ugks import euler_flux
    cells, links = _macro_links(setup, geo, W, Gam, status)

    def off(fid, sgn, nb, dW):
        nx, ny = sgn * geo.n[fid]
        un = sgn * geo.SUn[fid] / geo.S[fid]
        dF = euler_flux(W[nb] + dW, nx, ny, un, setup.gas) - euler_flux(W[nb], nx, ny, un, setup.gas)
        return 0.25 * geo.S[fid] * (dF - Gam[fid] * dW)

    dstar = np.zeros_like(R)
    for c in cells:
        acc = R[c].copy()
        for fid, sgn, nb in links[c]:
            if nb < c:
                acc -= off(fid, sgn, nb, dstar[nb])
        dstar[c] = acc / diag[c]
    d = dstar.copy()
    for c in reversed(cells):
        acc = np.zeros(4)
        for fid, sgn, nb in links[c]:
            if nb > c:
                acc += off(fid, sgn, nb, d[nb])
        d[c] = d[c] - acc / diag[c]
    return cells, links, dstar, d


def macro_lusgs_tangent(setup, geo, W, R, diag, Gam, status, dR):
    """Derivative of the macro LU-SGS solution with respect to its right-hand
    side R in the direction dR (W, diag, Gamma and the geometry fixed)."""
    cells, links, dstar, d = _macro_passes(setup, geo, W, R, diag, Gam, status)
    x = np.zeros_like(dR)
    for c in cells:
        acc = dR[c].copy()
        for fid, sgn, nb in links[c]:
            if nb < c:
                acc -= _coupling_jacobian(setup, geo, W, Gam, c, fid, sgn, nb, dstar[nb]) @ x[nb]
        x[c] = acc / diag[c]
    y = x.copy()
    for c in reversed(cells):
        acc = np.zeros(4)
        for fid, sgn, nb in links[c]:
            if nb > c:
                acc += _coupling_jacobian(setup, geo, W, Gam, c, fid, sgn, nb, d[nb]) @ y[nb]
        y[c] = y[c] - acc / diag[c]
    return y


def macro_lusgs_adjoint(setup, geo, W, R, diag, Gam, status, ybar):
    """Cotangent of R for a cotangent ybar of the macro LU-SGS solution: the
    transpose of ``macro_lusgs_tangent`` at the same point."""
    cells, links, dstar, d = _macro_passes(setup, geo, W, R, diag, Gam, status)
    solved = set(cells)
    # rows nb that couple to column c in each pass, with their Jacobian blocks
    upper_to = {c: [] for c in cells}       # backward pass: row nb < c holds a block for c
    lower_to = {c: [] for c in cells}       # forward pass: row nb > c holds a block for c
    for nb in cells:
        for fid, sgn, c in links[nb]:
            if c in solved and c > nb:
                upper_to[c].append((nb, _coupling_jacobian(setup, geo, W, Gam, nb, fid, sgn, c, d[c])))
            elif c in solved and c < nb:
                lower_to[c].append((nb, _coupling_jacobian(setup, geo, W, Gam, nb, fid, sgn, c, dstar[c])))
    # (D + U')^T a = ybar, increasing order
    a = np.zeros_like(ybar)
    for c in cells:
        acc = ybar[c].copy()
        for nb, J in upper_to[c]:
            acc -= J.T @ a[nb]
        a[c] = acc / diag[c]
    b = a * diag[:, None]
    # (D + L')^T z = b, decreasing order
    z = np.zeros_like(ybar)
    for c in reversed(cells):
        acc = b[c].copy()
        for nb, J in lower_to[c]:
            acc -= J.T @ z[nb]
        z[c] = acc / diag[c]
    return z


def moment_fix(setup, Wp, f):
    """Step 7 of the oracle's step as a function: W' + sum V Psi (f - g(W'))."""
    gas, dvs = setup.gas, setup.dvs
    rho, Vx, Vy, lam = kn.primitive(Wp, gas)
    g = kn.maxwellian(rho, Vx, Vy, lam, dvs, gas)
    return Wp + kn.moments(f - g, dvs)


def _fix_dg(setup, Wp, dWp):
    gas, dvs = setup.gas, setup.dvs
    rho, Vx, Vy, lam = kn.primitive(Wp, gas)
    g = kn.maxwellian(rho, Vx, Vy, lam, dvs, gas)
    return kn.slope_times_g(kn.micro_slope(Wp, dWp, gas), g, lam, dvs, gas)


def moment_fix_tangent(setup, Wp, dWp, df):
    """Derivative of ``moment_fix`` at (Wp, f) in the direction (dWp, df)."""
    return dWp + kn.moments(df - _fix_dg(setup, Wp, dWp), setup.dvs)


def moment_fix_adjoint(setup, Wp, Wbar):
    """Cotangents (of W', of f) of ``moment_fix`` for a cotangent Wbar of its
    result."""
    nc = Wp.shape[0]
    G = np.zeros((nc, 4, 4))
    for j in range(4):
        e = np.zeros((nc, 4))
        e[:, j] = 1.0
        G[:, :, j] = kn.moments(_fix_dg(setup, Wp, e), setup.dvs)
    Wpbar = Wbar - np.einsum("cij,ci->cj", G, Wbar)
    return Wpbar, moments_transpose(Wbar, setup.dvs)
