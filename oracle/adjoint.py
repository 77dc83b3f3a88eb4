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

The nonlinear parts of the step (flux, interface state, macro LU-SGS,
geometry) have no transpose here.
"""
from __future__ import annotations

import numpy as np

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
