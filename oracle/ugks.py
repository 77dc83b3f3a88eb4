"""Implicit unsteady UGKS step on moving structured blocks (test infrastructure).

Plain FP64 numpy restatement of Sec. 2 of the paper; see ``oracle/__init__``.
Arrays: f (nc, nv, 2) holds the reduced pair (h, b); W (nc, 4); q (nc, 2).

Readings where the paper is silent:
  R1 reconstruction: per logical direction a van Leer limited slope of the
     cell-centre differences (one-sided where a side has no neighbour cell,
     ghost cells count as neighbours, holes do not), mapped to Cartesian
     components with the 2x2 Jacobian of the same centre differences.
  R2 interface equilibrium (Sec. 2.1, details "in earlier work"): W0 from the
     upwind face values of both sides; q0 = mean of the two cells' heat
     fluxes; one face gradient of W (mean of the cell gradients with the
     component along x_R - x_L replaced by the centre difference); micro
     slopes from the continuous moment system; A from compatibility with the
     relative velocity w = v - U_f.
  R3 time-averaged flux (Sec. 2.2) over the per-face explicit step
     dts = min of the two cells' dts_i = cfl_s Omega_i / max_k sum_faces
     S max(w_n,out, 0).
  R4 ALE Crank-Nicolson in conservative (extensive) form:
     (Omega^{n+1} f^{n+1} - Omega^n f^n)/dt = -1/2 sum S (F^{n+1} + F^n)
                                              + 1/2 (Omega^{n+1} Q^{n+1} + Omega^n Q^n);
     with a static mesh this is exactly the paper's r_{i,k}.
  R5 walls: incident part from the interior cell extrapolated to the face
     (f, and W for g_in), reflected part a wall Maxwellian at the face
     velocity with rho_w from zero net mass flux (Eq. maxWalldes) over dts.
  R6 far field / outflow: ghost cell at the mirror point holding the
     Maxwellian of W_inf / of the interior W, zero gradients, q = 0.
  R7 heat flux of a cell after an inner step: taken about the predictor
     velocity V' (Step 4) from f^{s+1}.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np

from . import kinetic as kn
from .mesh import IM, IP, JM, JP, NB_CELL, NB_GHOST, Geometry, Topology
from paper_2604_09984_gb300.workloads import BC_FARFIELD, BC_OUTFLOW, BC_WALL

FIELD, RECEPTOR, HOLE = 0, 1, 2


@dataclass
class Setup:
    topo: Topology
    gas: kn.Gas
    dvs: kn.Dvs
    farfield_W: np.ndarray
    cfl_s: float = 0.5
    cfl_pseudo: float = 100.0


@dataclass
class State:
    f: np.ndarray
    W: np.ndarray
    q: np.ndarray

    def copy(self):
        return State(self.f.copy(), self.W.copy(), self.q.copy())


def initial_state(setup: Setup, prim) -> State:
    """f = Maxwellian of the initial primitive field, q from f."""
    gas, dvs = setup.gas, setup.dvs
    prim = np.asarray(prim, dtype=np.float64)
    lam = 1.0 / (2.0 * prim[:, 3])
    W = kn.conservative(prim[:, 0], prim[:, 1], prim[:, 2], lam, gas)
    f = kn.maxwellian(prim[:, 0], prim[:, 1], prim[:, 2], lam, dvs, gas)
    q = kn.heat_flux(f, prim[:, 1], prim[:, 2], dvs)
    return State(f, W, q)


# ------------------------------------------------------------ explicit step
def normal_velocity(setup: Setup, geo: Geometry):
    """S w_n = S v_k.n - S U.n for every face and velocity (nf, nv)."""
    dvs = setup.dvs
    return (geo.Sn[:, 0, None] * dvs.vx[None, :] + geo.Sn[:, 1, None] * dvs.vy[None, :]
            - geo.SUn[:, None])


def explicit_dt(setup: Setup, geo: Geometry, wS):
    """Reading R3: dts_i = cfl_s Omega_i^{n+1} / max_k sum_j S max(w_out, 0)."""
    topo = setup.topo
    out = np.zeros((topo.nc, setup.dvs.nv))
    for d in range(4):
        fid = topo.cell_faces[:, d]
        sgn = topo.cell_face_sign[:, d]
        out += np.maximum(sgn[:, None] * wS[fid], 0.0)
    return setup.cfl_s * geo.vol_new / out.max(axis=1)


# ---------------------------------------------------------- reconstruction
def _vanleer(a, b):
    prod = a * b
    safe = np.where(prod > 0.0, a + b, 1.0)
    return np.where(prod > 0.0, 2.0 * prod / safe, 0.0)


def ghost_W(setup: Setup, W):
    """Ghost conservative state per face (nf, 4): far field W_inf, outflow the
    interior W (reading R6); zero elsewhere."""
    topo = setup.topo
    gW = np.zeros((topo.nf, 4))
    ff = topo.face_kind == BC_FARFIELD
    of = topo.face_kind == BC_OUTFLOW
    gW[ff] = setup.farfield_W
    gW[of] = W[topo.face_L[of]]
    return gW


def ghost_f(setup: Setup, gW):
    topo = setup.topo
    gf = np.zeros((topo.nf, setup.dvs.nv, 2))
    m = (topo.face_kind == BC_FARFIELD) | (topo.face_kind == BC_OUTFLOW)
    if m.any():
        rho, Vx, Vy, lam = kn.primitive(gW[m], setup.gas)
        gf[m] = kn.maxwellian(rho, Vx, Vy, lam, setup.dvs, setup.gas)
    return gf


def mirror(xc, xf, n):
    """Mirror image of the point xc across the line through xf with normal n."""
    d = ((xf - xc) * n).sum(-1, keepdims=True)
    return xc + 2.0 * d * n


def gradients(setup: Setup, geo: Geometry, phi, ghost, status):
    """Reading R1: limited Cartesian gradient of the cell field phi
    (nc, ...) -> (nc, ..., 2); ghost (nf, ...) holds ghost-cell values."""
    topo = setup.topo
    nc = topo.nc
    extra = phi.shape[1:]
    ex = (slice(None),) + (None,) * len(extra)
    cell = np.arange(nc)
    dphi = []
    dx = []
    for dm, dp in ((IM, IP), (JM, JP)):
        vals, pos, has = [], [], []
        for d in (dm, dp):
            kind = topo.nb_kind[:, d]
            nid = topo.nb_id[:, d]
            v = np.zeros_like(phi)
            p = np.zeros((nc, 2))
            h = np.zeros(nc, dtype=bool)
            mc = kind == NB_CELL
            ids = nid[mc]
            v[mc] = phi[ids]
            p[mc] = geo.xc[ids] + topo.nb_shift[mc, d][:, None] * geo.period[mc]
            h[mc] = status[ids] != HOLE
            mg = kind == NB_GHOST
            fids = nid[mg]
            v[mg] = ghost[fids]
            p[mg] = mirror(geo.xc[mg], geo.xf[fids], geo.n[fids])
            h[mg] = True
            vals.append(v)
            pos.append(p)
            has.append(h)
        (vm, vp), (pm, pp), (hm, hp) = vals, pos, has
        both = hm & hp
        only_p = hp & ~hm
        only_m = hm & ~hp
        s = np.zeros_like(phi)
        s = np.where(both[ex], _vanleer(phi - vm, vp - phi), s)
        s = np.where(only_p[ex], vp - phi, s)
        s = np.where(only_m[ex], phi - vm, s)
        # geometric derivative of the same differences
        fm = geo.xf[topo.cell_faces[:, dm]]
        fp = geo.xf[topo.cell_faces[:, dp]]
        g = fp - fm
        g = np.where(both[:, None], 0.5 * (pp - pm), g)
        g = np.where(only_p[:, None], pp - geo.xc, g)
        g = np.where(only_m[:, None], geo.xc - pm, g)
        dphi.append(s)
        dx.append(g)
    (sx, se), (gx, ge) = dphi, dx
    # [x_xi y_xi; x_eta y_eta] [phi_x; phi_y] = [phi_xi; phi_eta]
    a11, a12 = gx[:, 0], gx[:, 1]
    a21, a22 = ge[:, 0], ge[:, 1]
    det = a11 * a22 - a12 * a21
    px = (sx * a22[ex] - se * a12[ex]) / det[ex]
    py = (se * a11[ex] - sx * a21[ex]) / det[ex]
    return np.stack([px, py], axis=-1)


def _dot_grad(dx, grad):
    """dx (n, 2) . grad (n, ..., 2) -> (n, ...)."""
    sh = (slice(None),) + (None,) * (grad.ndim - 2)
    return dx[:, 0][sh] * grad[..., 0] + dx[:, 1][sh] * grad[..., 1]


# ------------------------------------------------------------------- flux
@dataclass
class FluxResult:
    D: np.ndarray          # (nc, nv, 2) sum_faces S F_hat (outward positive)
    F: np.ndarray          # (nc, 4) macro flux divergence sum_k V_k Psi_k D_k
    wall_face: np.ndarray  # wall face ids
    wall_rho: np.ndarray   # rho_w per wall face
    wall_F: np.ndarray     # (nwall, 4) macro flux per unit length (outward)


def _interface_terms(setup, geo, F, ff, gup, W0, gradW0, q0, dts, Uf):
    """Time-integrated interface distribution of Eq. fullSolution for the
    faces F: returns int_0^{dts} f dt (nF, nv, 2)."""
    gas, dvs = setup.gas, setup.dvs
    rho0, Vx0, Vy0, lam0 = kn.primitive(W0, gas)
    ax = kn.micro_slope(W0, gradW0[..., 0], gas)
    ay = kn.micro_slope(W0, gradW0[..., 1], gas)
    A = kn.time_slope(W0, ax, ay, Uf[:, 0], Uf[:, 1], gas)
    tau0 = kn.collision_time(rho0, lam0, gas)
    q1, q2, q3, q4, q5 = kn.time_integrals(dts, tau0)
    g0 = kn.maxwellian(rho0, Vx0, Vy0, lam0, dvs, gas)
    g0p = kn.shakhov_part(rho0, Vx0, Vy0, lam0, q0[:, 0], q0[:, 1], dvs, gas)
    gax = kn.slope_times_g(ax, g0, lam0, dvs, gas)
    gay = kn.slope_times_g(ay, g0, lam0, dvs, gas)
    gA = kn.slope_times_g(A, g0, lam0, dvs, gas)
    wx = (dvs.vx[None, :] - Uf[:, 0, None])[..., None]
    wy = (dvs.vy[None, :] - Uf[:, 1, None])[..., None]
    wgf = wx * gup[..., 0] + wy * gup[..., 1]
    c = lambda q: q[:, None, None]
    return (c(q1) * ff + c(q2) * wgf + c(q3) * (g0 + g0p)
            + c(q4) * (wx * gax + wy * gay) + c(q5) * gA)


def flux(setup: Setup, geo: Geometry, st: State, status, dts_cell, wS=None,
         faces=None) -> FluxResult:
    """Time-averaged interface fluxes (Eqs. microscopicFlux, fullSolution,
    Sec. 2.2) summed per cell: D_i = sum_j S_ij F_hat_ij (outward positive),
    and the macroscopic divergence F_i = sum_k V_k Psi_k D_ik
    (Eq. macroscopicFlux).  `faces` optionally restricts the faces evaluated
    (boolean mask); by default every face touching a FIELD cell."""
    topo, gas, dvs = setup.topo, setup.gas, setup.dvs
    nc, nv = topo.nc, dvs.nv
    if wS is None:
        wS = normal_velocity(setup, geo)
    gW = ghost_W(setup, st.W)
    gf = ghost_f(setup, gW)
    gradf = gradients(setup, geo, st.f, gf, status)
    gradW = gradients(setup, geo, st.W, gW, status)
    L, R, kind = topo.face_L, topo.face_R, topo.face_kind
    fieldL = status[L] == FIELD
    fieldR = np.where(R >= 0, status[np.maximum(R, 0)] == FIELD, False)
    need = fieldL | fieldR
    if faces is not None:
        need &= faces
    D = np.zeros((nc, nv, 2))

    # ---- two-sided faces: interior and ghost (far field / outflow)
    two = need & ((R >= 0) | (kind == BC_FARFIELD) | (kind == BC_OUTFLOW))
    F2 = np.nonzero(two)[0]
    if F2.size:
        l = L[F2]
        isint = R[F2] >= 0
        r = np.where(isint, R[F2], 0)
        xf, n = geo.xf[F2], geo.n[F2]
        xL = geo.xc[l] + topo.face_shiftL[F2][:, None] * geo.period[l]
        xR = np.where(isint[:, None], geo.xc[r], mirror(xL, xf, n))
        fL = st.f[l] + _dot_grad(xf - xL, gradf[l])
        fR = np.where(isint[:, None, None], st.f[r] + _dot_grad(xf - xR, gradf[r]), gf[F2])
        gL = gradf[l]
        gR = np.where(isint[:, None, None, None], gradf[r], 0.0)
        WL = st.W[l]
        WR = np.where(isint[:, None], st.W[r], gW[F2])
        dWL = gradW[l]
        dWR = np.where(isint[:, None, None], gradW[r], 0.0)
        qL = st.q[l]
        qR = np.where(isint[:, None], st.q[r], 0.0)
        dts = np.where(isint, np.minimum(dts_cell[l], dts_cell[r]), dts_cell[l])
        w = wS[F2]
        pos = (w > 0.0)[..., None]
        neg = (w < 0.0)[..., None]
        ff = np.where(pos, fL, np.where(neg, fR, 0.5 * (fL + fR)))
        gup = np.where(pos[..., None], gL, np.where(neg[..., None], gR, 0.5 * (gL + gR)))
        W0 = kn.moments(ff, dvs)
        q0 = 0.5 * (qL + qR)
        t = xR - xL
        avg = 0.5 * (dWL + dWR)
        jump = (WR - WL) - (avg[..., 0] * t[:, None, 0] + avg[..., 1] * t[:, None, 1])
        t2 = (t * t).sum(-1)
        gradW0 = avg + jump[..., None] * (t / t2[:, None])[:, None, :]
        integ = _interface_terms(setup, geo, F2, ff, gup, W0, gradW0, q0, dts, geo.Uf[F2])
        wn = w / geo.S[F2][:, None]
        SF = (geo.S[F2] / dts)[:, None, None] * wn[..., None] * integ
        np.add.at(D, l, SF)
        np.add.at(D, r[isint], -SF[isint])

    # ---- wall faces (reading R5)
    Fw = np.nonzero(need & (kind == BC_WALL))[0]
    wall_rho = np.zeros(Fw.size)
    wall_F = np.zeros((Fw.size, 4))
    if Fw.size:
        c = L[Fw]
        xf = geo.xf[Fw]
        dx = xf - geo.xc[c]
        ff = st.f[c] + _dot_grad(dx, gradf[c])
        gup = gradf[c]
        Win = st.W[c] + _dot_grad(dx, gradW[c])
        integ = _interface_terms(setup, geo, Fw, ff, gup, Win, gradW[c], st.q[c],
                                 dts_cell[c], geo.Uf[Fw])
        w = wS[Fw]
        wn = w / geo.S[Fw][:, None]
        inc = w > 0.0
        Tw = topo.face_Tw[Fw]
        lamw = 1.0 / (2.0 * Tw)
        Uf = geo.Uf[Fw]
        cx = dvs.vx[None, :] - Uf[:, 0, None]
        cy = dvs.vy[None, :] - Uf[:, 1, None]
        Hw = (lamw / np.pi)[:, None] * np.exp(-lamw[:, None] * (cx * cx + cy * cy))
        dts = dts_cell[c]
        num = (np.where(inc, dvs.w * wn * integ[..., 0], 0.0)).sum(-1)
        den = dts * (np.where(inc, 0.0, dvs.w * wn * Hw)).sum(-1)
        rho_w = -num / den
        refl = np.stack([Hw, gas.Keff / (2.0 * lamw)[:, None] * Hw], axis=-1) * rho_w[:, None, None]
        Fhat = np.where(inc[..., None], (wn / dts[:, None])[..., None] * integ,
                        wn[..., None] * refl)
        np.add.at(D, c, geo.S[Fw][:, None, None] * Fhat)
        wall_rho = rho_w
        wall_F = kn.moments(Fhat, dvs)
    F = kn.moments(D, dvs)
    return FluxResult(D, F, Fw, wall_rho, wall_F)


# ------------------------------------------------------------ LU-SGS sweeps
def _cell_links(topo: Topology, c):
    """(face id, sign, neighbour cell) for the four faces of cell c; the
    neighbour is -1 across boundary faces."""
    out = []
    for d in range(4):
        fid = topo.cell_faces[c, d]
        sgn = topo.cell_face_sign[c, d]
        nb = topo.face_R[fid] if sgn > 0 else topo.face_L[fid]
        out.append((fid, sgn, nb))
    return out


def micro_lusgs(setup: Setup, wS, rhs, diag, status):
    """LU-SGS (Yoon-Jameson) for Eq. dualTimeStepping_micro with the upwind
    flux variation of Sec. 2.2:  (D + L) d* = rhs,  (D + U) d = D d*, where
    the off-diagonal coupling to neighbour j is (1/2) S min(w_out, 0) and
    lower/upper means a smaller/larger lexicographic cell index in the same
    block (i fastest).  Only FIELD cells are solved; others have d = 0.
    All arrays extensive (multiplied by Omega^{n+1})."""
    topo = setup.topo
    d = np.zeros_like(rhs)
    cells = [c for c in range(topo.nc) if status[c] == FIELD]
    links = {c: _cell_links(topo, c) for c in cells}
    for c in cells:
        acc = rhs[c].copy()
        for fid, sgn, nb in links[c]:
            if nb >= 0 and nb < c and status[nb] == FIELD:
                acc -= 0.5 * np.minimum(sgn * wS[fid], 0.0)[:, None] * d[nb]
        d[c] = acc / diag[c][:, None]
    for c in reversed(cells):
        acc = np.zeros_like(rhs[c])
        for fid, sgn, nb in links[c]:
            if nb > c and status[nb] == FIELD:
                acc += 0.5 * np.minimum(sgn * wS[fid], 0.0)[:, None] * d[nb]
        d[c] = d[c] - acc / diag[c][:, None]
    return d


def euler_flux(W, nx, ny, un, gas):
    """Euler flux through a moving face: rho v_n, rho V v_n + p n,
    rho E v_n + p V.n with v_n = V.n - U.n (Sec. 2.2 Euler-based variation)."""
    rho, Vx, Vy, lam = kn.primitive(W, gas)
    p = rho / (2.0 * lam)
    vabs = Vx * nx + Vy * ny
    vn = vabs - un
    return np.stack([rho * vn, W[..., 1] * vn + p * nx, W[..., 2] * vn + p * ny,
                     W[..., 3] * vn + p * vabs], axis=-1)


def spectral_radius(W, nx, ny, un, gas):
    """Gamma = |(V - U).n| + a (Sec. 2.2)."""
    rho, Vx, Vy, lam = kn.primitive(W, gas)
    p = rho / (2.0 * lam)
    a = np.sqrt(gas.gamma * p / rho)
    return np.abs(Vx * nx + Vy * ny - un) + a


def macro_lusgs(setup: Setup, geo: Geometry, W, R, diag, Gam, status):
    """LU-SGS for Eq. dualTimeStepping_macro with the Euler-flux variation
    (1/2)[dF_E,i + dF_E,j + Gamma (dW_i - dW_j)]; the dF_E,i part is dropped
    into the diagonal as usual, leaving the off-diagonal coupling
    (1/4) S (dF_E,j - Gamma dW_j), dF_E,j = F_E(W_j + dW_j) - F_E(W_j) along the
    outward normal of cell i.  Extensive arrays (times Omega^{n+1})."""
    topo, gas = setup.topo, setup.gas
    d = np.zeros_like(R)
    cells = [c for c in range(topo.nc) if status[c] == FIELD]
    links = {c: _cell_links(topo, c) for c in cells}

    def off(c, fid, sgn, nb, dW):
        nx, ny = sgn * geo.n[fid]
        un = sgn * geo.SUn[fid] / geo.S[fid]
        dF = euler_flux(W[nb] + dW, nx, ny, un, gas) - euler_flux(W[nb], nx, ny, un, gas)
        return 0.25 * geo.S[fid] * (dF - Gam[fid] * dW)

    for c in cells:
        acc = R[c].copy()
        for fid, sgn, nb in links[c]:
            if nb >= 0 and nb < c and status[nb] == FIELD:
                acc -= off(c, fid, sgn, nb, d[nb])
        d[c] = acc / diag[c]
    for c in reversed(cells):
        acc = np.zeros(4)
        for fid, sgn, nb in links[c]:
            if nb > c and status[nb] == FIELD:
                acc += off(c, fid, sgn, nb, d[nb])
        d[c] = d[c] - acc / diag[c]
    return d


def face_gamma(setup: Setup, geo: Geometry, W):
    """Gamma_ij from the mean of the two cells' W (boundary faces: the cell)."""
    topo = setup.topo
    L, R = topo.face_L, topo.face_R
    Wf = np.where((R >= 0)[:, None], 0.5 * (W[L] + W[np.maximum(R, 0)]), W[L])
    return spectral_radius(Wf, geo.n[:, 0], geo.n[:, 1], geo.SUn / geo.S, setup.gas)


# -------------------------------------------------------------- the step
@dataclass
class StepInfo:
    dts: np.ndarray
    flux_n: FluxResult
    last_flux: FluxResult
    R: Optional[np.ndarray] = None       # Step-4 macro residual of the last inner iteration
    rhs: Optional[np.ndarray] = None     # Step-5 micro residual of the last inner iteration
    fix: Optional[np.ndarray] = None     # Step-7 moment fix W^{s+1} - W' of the last inner iteration


def step_metrics(geo: Geometry, st: State, info: StepInfo, status):
    """Per-step metrics of the implicit step (Sec. 2.2): squared L2 norms
    over the solved cells of the macro residual R (Step 4), the micro
    residual r (Step 5) and the moment fix W^{s+1} - W' (Step 7) of the last
    inner iteration, and the field totals of Omega^{n+1} W."""
    field = status == FIELD
    return {"res_macro_sq": float((info.R[field] ** 2).sum()),
            "res_micro_sq": float((info.rhs[field] ** 2).sum()),
            "fix_sq": float((info.fix[field] ** 2).sum()),
            "total": (geo.vol_new[field, None] * st.W[field]).sum(axis=0)}


def implicit_step(setup: Setup, geo: Geometry, st: State, dt: float, n_inner: int,
                  status=None, interp: Optional[Callable[[State], None]] = None,
                  fresh: Optional[Callable[[State], None]] = None):
    """One physical step n -> n+1 of the unsteady implicit UGKS
    (Sec. 2.2 Steps 1-8, reading R4 for the moving mesh).  Returns the new
    state and diagnostics.  `interp` overwrites receptor cells from their
    donors (Sec. 3.2) before every flux evaluation; `fresh` initialises cells
    uncovered by the motion once, before Step 1."""
    topo, gas, dvs = setup.topo, setup.gas, setup.dvs
    if status is None:
        status = np.zeros(topo.nc, dtype=np.int64)
    st = st.copy()
    if fresh is not None:
        fresh(st)
    if interp is not None:
        interp(st)
    wS = normal_velocity(setup, geo)
    dts = explicit_dt(setup, geo, wS)
    dtp = setup.cfl_pseudo / setup.cfl_s * dts          # pseudo time step Delta t'
    vol0, vol1 = geo.vol_old, geo.vol_new
    field = status == FIELD

    # Steps 1-2: level-n flux and residual (extensive form)
    fl_n = flux(setup, geo, st, status, dts, wS)
    rho, Vx, Vy, lam = kn.primitive(st.W, gas)
    tau_n = kn.collision_time(rho, lam, gas)
    Qn = (kn.shakhov_equilibrium(st.W, st.q, dvs, gas) - st.f) / tau_n[:, None, None]
    Tf = (vol0 / dt)[:, None, None] * st.f + 0.5 * (vol0[:, None, None] * Qn - fl_n.D)
    TW = (vol0 / dt)[:, None] * st.W - 0.5 * fl_n.F
    fn = st.f.copy()

    # outflow sum per cell for the micro diagonal, Gamma for the macro one
    outsum = np.zeros((topo.nc, dvs.nv))
    for dd in range(4):
        fid = topo.cell_faces[:, dd]
        sgn = topo.cell_face_sign[:, dd]
        outsum += np.maximum(sgn[:, None] * wS[fid], 0.0)

    fl = fl_n
    for s in range(n_inner):
        if s > 0:
            if interp is not None:
                interp(st)
            fl = flux(setup, geo, st, status, dts, wS)     # Step 3
        # Step 4: macro LU-SGS
        R = TW - (vol1 / dt)[:, None] * st.W - 0.5 * fl.F
        Gam = face_gamma(setup, geo, st.W)
        gsum = np.zeros(topo.nc)
        for dd in range(4):
            fid = topo.cell_faces[:, dd]
            gsum += geo.S[fid] * Gam[fid]
        diagW = vol1 * (1.0 / dtp + 1.0 / dt) + 0.25 * gsum
        dW = macro_lusgs(setup, geo, st.W, R, diagW, Gam, status)
        Wp = st.W + dW
        # Step 5: residual with f+ and tau at W'
        rho, Vx, Vy, lam = kn.primitive(Wp, gas)
        taup = kn.collision_time(rho, lam, gas)
        fplus = kn.shakhov_equilibrium(Wp, st.q, dvs, gas)
        rhs = (Tf - (vol1 / dt)[:, None, None] * st.f
               + 0.5 * (vol1[:, None, None] * (fplus - st.f) / taup[:, None, None] - fl.D))
        # Step 6: micro LU-SGS
        diag = vol1[:, None] * (1.0 / dtp + 1.0 / dt + 1.0 / (2.0 * taup))[:, None] + 0.5 * outsum
        df = micro_lusgs(setup, wS, rhs, diag, status)
        fnew = np.where(field[:, None, None], st.f + df, st.f)
        # Step 7: fix W with the moments of f - g(W')
        g = kn.maxwellian(rho, Vx, Vy, lam, dvs, gas)
        Wnew = Wp + kn.moments(fnew - g, dvs)
        qnew = kn.heat_flux(fnew, Vx, Vy, dvs)
        st.f = fnew
        st.W = np.where(field[:, None], Wnew, st.W)
        st.q = np.where(field[:, None], qnew, st.q)
    return st, StepInfo(dts, fl_n, fl, R, rhs, Wnew - Wp)
