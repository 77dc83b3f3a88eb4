"""Seeded synthetic workloads for the implicit moving-mesh UGKS.

This module only *describes inputs*: structured-block node coordinates,
boundary tags, the prescribed rigid/affine motion of each block (the host
evaluates the kinematics, Sec. 3 Step 1 "given motion function"), initial
primitive fields with seeded noise, and the gas / velocity-space / time-step
constants.  It holds none of the scheme's arithmetic, and it is the only code
shared by the CUDA path and the FP64 test oracle.

Configurations (nondimensional, rho0 = T0 = R = L = 1):
  channel   2D channel, top wall oscillating normal to itself, mesh deformed
            linearly in y (the thermal MEMS micro-beam setting of Sec. 4.1,
            reduced to a single block).
  mems      Cartesian background + body-fitted O-grid around a heated thin
            plate translating sinusoidally (overset MEMS, Sec. 4.1/4.2).
  tsto      Ma 8 background + two O-grids (wedge and cylinder) with prescribed
            separation and pitch (2D stand-in for the TSTO case of Sec. 4.3).
  mems_batch  many independent `mems` instances of uneven sizes, velocity
            grids, Knudsen numbers and wall temperatures (batched serving).
  particle  a free rigid cylinder released in a closed box of gas at rest,
            moved by the gas force and torque (Newton-Euler coupling).
The paper's own geometries exist only as missing figures; these synthetic
cases carry their sizes, regimes and motion types.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List

import numpy as np

# boundary kinds of a block side
BC_NONE = 0       # interior / periodic (handled by the periodic_i flag)
BC_WALL = 1       # diffuse isothermal wall (Sec. 2.1, Eq. maxWalldes)
BC_FARFIELD = 2   # ghost cell at the free-stream state (Sec. 2.1)
BC_OUTFLOW = 3    # ghost cell copying the interior state
BC_OVERSET = 4    # outer edge of a component grid: fringe cells are receptors
SIDES = ("ilo", "ihi", "jlo", "jhi")


@dataclass
class BlockSpec:
    ni: int
    nj: int
    periodic_i: bool
    bc: tuple                     # kind per side (ilo, ihi, jlo, jhi)
    wall_T: tuple                 # wall temperature per side (walls only)
    x_ref: np.ndarray             # (ni+1, nj+1, 2) reference node coordinates
    priority: int = 0             # overset: higher wins ties (body grids)
    n_fringe: int = 2             # receptor layers along BC_OVERSET sides
    n_gap: int = 2                # layers beyond the fringe not used to cut holes

    @property
    def ncells(self) -> int:
        return self.ni * self.nj


@dataclass
class Case:
    name: str
    K: int
    Pr: float
    omega: float
    mu_ref: float
    nvx: int
    nvy: int
    vbox: tuple                   # (vx_min, vx_max, vy_min, vy_max)
    blocks: List[BlockSpec]
    farfield: tuple               # (rho, ux, uy, T)
    dt: float
    n_inner: int
    n_steps: int
    motion: Callable[[float], np.ndarray]   # t -> (nblocks, 6) affine maps
    init_prim: np.ndarray         # (ncells_total, 4): rho, ux, uy, T
    cfl_s: float = 0.5            # explicit step for the flux time average
    cfl_pseudo: float = 100.0     # pseudo time step Delta t'
    meta: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return sum(b.ncells for b in self.blocks)

    @property
    def nv(self) -> int:
        return self.nvx * self.nvy

    def nodes_at(self, t: float) -> List[np.ndarray]:
        """Node coordinates of every block at time t: x = M x_ref + b with the
        block's affine map (m00, m01, m10, m11, b0, b1), evaluated as
        (m00*x + m01*y) + b0 in FP64 without contraction."""
        A = self.motion(t)
        out = []
        for b, a in zip(self.blocks, A):
            x = b.x_ref[..., 0]
            y = b.x_ref[..., 1]
            X = np.empty_like(b.x_ref)
            X[..., 0] = (a[0] * x + a[1] * y) + a[4]
            X[..., 1] = (a[2] * x + a[3] * y) + a[5]
            out.append(X)
        return out


def mu_ref_from_knudsen(Kn: float, omega: float, alpha: float = 1.0) -> float:
    """Bird's VHS/VSS relation mu_ref = 5(a+1)(a+2) sqrt(pi) Kn sqrt(2RT) L rho
    / (4 a (5-2w)(7-2w)) at rho = T = R = L = 1 (the paper quotes Kn only)."""
    return (5.0 * (alpha + 1.0) * (alpha + 2.0) * math.sqrt(math.pi)
            / (4.0 * alpha * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega))
            * Kn * math.sqrt(2.0))


# ------------------------------------------------------------------ meshes
def cartesian_nodes(ni, nj, x0, x1, y0, y1):
    X = np.empty((ni + 1, nj + 1, 2))
    xs = np.array([x0 + (x1 - x0) * i / ni for i in range(ni + 1)])
    ys = np.array([y0 + (y1 - y0) * j / nj for j in range(nj + 1)])
    X[..., 0] = xs[:, None]
    X[..., 1] = ys[None, :]
    return X


def ogrid_nodes(ni, nj, contour, center, r_out, stretch):
    """O-grid nodes: i runs clockwise around the body (right-handed cells with
    j pointing outward), j from the body contour (j = 0) to a circle of radius
    r_out with geometric radial stretching.  Column i = ni repeats column 0."""
    X = np.empty((ni + 1, nj + 1, 2))
    s = np.array([(stretch ** j - 1.0) / (stretch ** nj - 1.0) for j in range(nj + 1)])
    for i in range(ni + 1):
        th = -2.0 * math.pi * (i % ni) / ni
        bx, by = contour(th)
        ox = center[0] + r_out * math.cos(th)
        oy = center[1] + r_out * math.sin(th)
        X[i, :, 0] = bx + s * (ox - bx)
        X[i, :, 1] = by + s * (oy - by)
    return X


def ellipse_contour(center, a, b):
    return lambda th: (center[0] + a * math.cos(th), center[1] + b * math.sin(th))


def polygon_contour(center, verts):
    """Closed polygon (vertices relative to `center`, clockwise) traversed by
    arc length: th in (-2 pi, 0] maps to the fraction -th / (2 pi) of the
    perimeter, measured clockwise from the point where the ray at angle 0
    from `center` leaves the polygon, so that an O-grid's contour and outer
    circle start at the same angle and turn the same way."""
    P = [np.asarray(v, dtype=float) for v in verts]
    seg = [(P[i], P[(i + 1) % len(P)]) for i in range(len(P))]
    lens = [float(np.hypot(*(b - a))) for a, b in seg]
    tot = sum(lens)
    s0, acc = 0.0, 0.0
    for (a, b), L in zip(seg, lens):    # the ray (1, 0) from the centre
        ey = b[1] - a[1]
        if ey != 0.0:
            u = -a[1] / ey                  # edge parameter where y = 0
            x = a[0] + u * (b[0] - a[0])
            if 0.0 <= u < 1.0 and x > 0.0:
                s0 = acc + u * L
        acc += L

    def c(th):
        s = (s0 + (-th / (2.0 * math.pi)) * tot) % tot
        for (a, b), L in zip(seg, lens):
            if s <= L:
                q = a + (b - a) * (s / L)
                return center[0] + float(q[0]), center[1] + float(q[1])
            s -= L
        return center[0] + float(P[0][0]), center[1] + float(P[0][1])
    return c


def smallest_cell_width(blocks) -> float:
    """min over the cells of all blocks of 4 * area / perimeter (the width
    of a square cell), from the reference nodes."""
    w = math.inf
    for b in blocks:
        X = b.x_ref
        P = [X[:-1, :-1], X[1:, :-1], X[1:, 1:], X[:-1, 1:]]
        area = 0.5 * sum(P[m][..., 0] * P[(m + 1) % 4][..., 1] - P[m][..., 1] * P[(m + 1) % 4][..., 0]
                         for m in range(4))
        per = sum(np.hypot(*(P[(m + 1) % 4] - P[m]).transpose(2, 0, 1)) for m in range(4))
        w = min(w, float((4.0 * np.abs(area) / per).min()))
    return w


def _affine_identity(n):
    A = np.zeros((n, 6))
    A[:, 0] = 1.0
    A[:, 3] = 1.0
    return A


def _init_noise(ncells, seed, amp, rho=1.0, ux=0.0, uy=0.0, T=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    prim = np.empty((ncells, 4))
    prim[:, 0] = rho * (1.0 + rng.uniform(-amp, amp, ncells))
    prim[:, 1] = ux
    prim[:, 2] = uy
    prim[:, 3] = T
    return prim


# ----------------------------------------------------------- configurations
def channel(ni=64, nj=32, nv=24, vmax=5.0, Kn=0.05, n_steps=20, n_inner=10,
            cfl=10.0, amp_frac=0.05, wall_mach=0.1, noise=1e-3, seed=0,
            omega=0.81, Pr=2.0 / 3.0, K=0) -> Case:
    """Plain FP64 channel: [0,2]x[0,1], periodic in x, bottom wall fixed, top
    wall y = 1 + A sin(2 pi f t) with A = amp_frac, mesh y <- y (1 + A sin/H),
    peak wall speed 2 pi f A = wall_mach * sqrt(gamma).  Walls at T0 = 1."""
    gamma = (K + 5.0) / (K + 3.0)
    H = 1.0
    A = amp_frac * H
    freq = wall_mach * math.sqrt(gamma) / (2.0 * math.pi * A)
    x_ref = cartesian_nodes(ni, nj, 0.0, 2.0, 0.0, H)
    blk = BlockSpec(ni, nj, True, (BC_NONE, BC_NONE, BC_WALL, BC_WALL),
                    (0.0, 0.0, 1.0, 1.0), x_ref)

    def motion(t):
        M = _affine_identity(1)
        M[0, 3] = 1.0 + A * math.sin(2.0 * math.pi * freq * t) / H
        return M

    h = min(2.0 / ni, H / nj)
    dt = cfl * h / (2.0 * vmax)
    return Case("channel", K, Pr, omega, mu_ref_from_knudsen(Kn, omega), nv, nv,
                (-vmax, vmax, -vmax, vmax), [blk], (1.0, 0.0, 0.0, 1.0), dt,
                n_inner, n_steps, motion, _init_noise(ni * nj, seed, noise),
                meta=dict(Kn=Kn, freq=freq, amp=A))


def mems(nbi=256, nbj=128, noi=128, noj=32, nv=32, vmax=6.0, Kn=0.1,
         n_steps=200, n_inner=10, cfl=10.0, Tw=1.5, mach=0.05, amp=0.1,
         plate=(0.1, 0.01), r_out=0.25, stretch=1.1, noise=0.0, seed=0,
         omega=0.81, Pr=2.0 / 3.0, K=0, n_gap=2) -> Case:
    """Thermal rarefied MEMS with overset grids: closed diffuse box [0,2]x[0,1]
    at T0 = 1, body-fitted O-grid around an elliptic plate (semi-axes
    `plate`, wall temperature Tw) translating y_c = 0.5 + amp sin(2 pi f t)
    with peak speed mach * sqrt(gamma)."""
    gamma = (K + 5.0) / (K + 3.0)
    freq = mach * math.sqrt(gamma) / (2.0 * math.pi * amp)
    c = (1.0, 0.5)
    bg = BlockSpec(nbi, nbj, False, (BC_WALL,) * 4, (1.0,) * 4,
                   cartesian_nodes(nbi, nbj, 0.0, 2.0, 0.0, 1.0), priority=0)
    og = BlockSpec(noi, noj, True, (BC_NONE, BC_NONE, BC_WALL, BC_OVERSET),
                   (0.0, 0.0, Tw, 0.0),
                   ogrid_nodes(noi, noj, ellipse_contour(c, *plate), c, r_out, stretch),
                   priority=1, n_gap=n_gap)

    def motion(t):
        M = _affine_identity(2)
        M[1, 5] = amp * math.sin(2.0 * math.pi * freq * t)
        return M

    h = min(2.0 / nbi, 1.0 / nbj)
    dt = cfl * h / (2.0 * vmax)
    n = bg.ncells + og.ncells
    return Case("mems", K, Pr, omega, mu_ref_from_knudsen(Kn, omega), nv, nv,
                (-vmax, vmax, -vmax, vmax), [bg, og], (1.0, 0.0, 0.0, 1.0), dt,
                n_inner, n_steps, motion, _init_noise(n, seed, noise),
                meta=dict(Kn=Kn, freq=freq, amp=amp, Tw=Tw))


def tsto(nbi=512, nbj=256, noi=192, noj=48, nv=64, vmax=15.0, Kn=0.01,
         mach=8.0, n_steps=500, n_inner=15, cfl=10.0, seed=0,
         omega=0.74, Pr=0.72, K=2, pitch_rate=0.5, separation=0.02) -> Case:
    """2D hypersonic two-body separation: free stream Ma 8 from the left,
    far field left/top/bottom, outflow right; a 10-degree half-angle wedge of
    chord 0.3 pitching at `pitch_rate` (0.5 rad per unit time) about its
    centroid, and a cylinder of radius 0.1 separating in +y at `separation`
    (0.02) times u_inf.  Walls at T_inf.
    Gas initially at rest; time step from the smallest cell of all blocks."""
    gamma = (K + 5.0) / (K + 3.0)
    uinf = mach * math.sqrt(gamma)
    bg = BlockSpec(nbi, nbj, False, (BC_FARFIELD, BC_OUTFLOW, BC_FARFIELD, BC_FARFIELD),
                   (0.0,) * 4, cartesian_nodes(nbi, nbj, 0.0, 2.0, 0.0, 1.0))
    cw = (0.7, 0.42)
    half = math.radians(10.0)
    chord = 0.3
    # clockwise vertices relative to the wedge centroid
    verts = [(-2 * chord / 3, 0.0), (chord / 3, chord * math.tan(half)),
             (chord / 3, -chord * math.tan(half))]
    wedge = BlockSpec(noi, noj, True, (BC_NONE, BC_NONE, BC_WALL, BC_OVERSET),
                      (0.0, 0.0, 1.0, 0.0),
                      ogrid_nodes(noi, noj, polygon_contour(cw, verts), cw, 0.28, 1.08),
                      priority=1)
    cc = (1.15, 0.58)
    cyl = BlockSpec(noi, noj, True, (BC_NONE, BC_NONE, BC_WALL, BC_OVERSET),
                    (0.0, 0.0, 1.0, 0.0),
                    ogrid_nodes(noi, noj, ellipse_contour(cc, 0.1, 0.1), cc, 0.22, 1.06),
                    priority=2)

    def motion(t):
        M = _affine_identity(3)
        a = pitch_rate * t
        ca, sa = math.cos(a), math.sin(a)
        M[1, 0], M[1, 1], M[1, 2], M[1, 3] = ca, -sa, sa, ca
        M[1, 4] = cw[0] - (ca * cw[0] - sa * cw[1])
        M[1, 5] = cw[1] - (sa * cw[0] + ca * cw[1])
        M[2, 5] = separation * uinf * t
        return M

    # time step from the smallest cell of all blocks (the body grids' wall
    # cells): CFL relative to the fastest discrete velocity there
    dt = cfl * smallest_cell_width([bg, wedge, cyl]) / (2.0 * vmax)
    n = bg.ncells + wedge.ncells + cyl.ncells
    # start-up from rest: the free stream enters through the far field (an
    # impulsive start with the stream everywhere and the walls at rest
    # empties the cells behind the bodies within a step at CFL 10)
    prim = _init_noise(n, seed, 0.0)
    return Case("tsto", K, Pr, omega, mu_ref_from_knudsen(Kn, omega), nv, nv,
                (-vmax, vmax, -vmax, vmax), [bg, wedge, cyl], (1.0, uinf, 0.0, 1.0),
                dt, n_inner, n_steps, motion, prim, meta=dict(Kn=Kn, uinf=uinf))


def particle(nbi=128, nbj=64, noi=64, noj=16, nv=24, vmax=5.0, Kn=0.1, radius=0.1, r_out=0.3,
             stretch=1.08, u0=(0.3, 0.0), omega0=0.0, density_ratio=10.0, n_steps=100, n_inner=10,
             cfl=10.0, seed=0, omega=0.81, Pr=2.0 / 3.0, K=0) -> Case:
    """Free particle: a rigid cylinder (radius `radius`, density
    `density_ratio` times the gas density) in a closed diffuse box
    [0,2]x[0,1] of gas at rest at T0 = 1, released from the box centre with
    velocity u0 and spin omega0; its motion follows the gas force and torque
    (Newton-Euler, Sec. 3 Step 1), so `motion` is the identity and the
    caller supplies the body's map.  meta: mass and moment of inertia per
    unit depth, reference centre, initial velocity and spin."""
    c = (1.0, 0.5)
    bg = BlockSpec(nbi, nbj, False, (BC_WALL,) * 4, (1.0,) * 4,
                   cartesian_nodes(nbi, nbj, 0.0, 2.0, 0.0, 1.0), priority=0)
    og = BlockSpec(noi, noj, True, (BC_NONE, BC_NONE, BC_WALL, BC_OVERSET), (0.0, 0.0, 1.0, 0.0),
                   ogrid_nodes(noi, noj, ellipse_contour(c, radius, radius), c, r_out, stretch),
                   priority=1)

    def motion(t):
        return _affine_identity(2)

    h = min(2.0 / nbi, 1.0 / nbj)
    dt = cfl * h / (2.0 * vmax)
    n = bg.ncells + og.ncells
    mass = density_ratio * math.pi * radius * radius
    return Case("particle", K, Pr, omega, mu_ref_from_knudsen(Kn, omega), nv, nv,
                (-vmax, vmax, -vmax, vmax), [bg, og], (1.0, 0.0, 0.0, 1.0), dt, n_inner, n_steps,
                motion, _init_noise(n, seed, 0.0),
                meta=dict(Kn=Kn, mass=mass, inertia=0.5 * mass * radius * radius, center=c,
                          u0=tuple(u0), omega0=omega0, body_block=1))


def overlap_gap_layers(nbi, noj, stretch, r_out, r_body, n_fringe=2, cells=3.0, n_min=2):
    """Gap layers of an O-grid (radial geometric stretching) such that the
    rings that do not cut holes span at least `cells` background cells of
    width 2/nbi between the body (radius r_body at its widest) and r_out, so
    that the background's buffer receptors around the hole lie inside the
    body grid.  Pure mesh bookkeeping on the node radii."""
    h = 2.0 / nbi
    frac = lambda j: (stretch ** j - 1.0) / (stretch ** noj - 1.0)
    for g in range(n_min, noj - n_fringe):
        k = noj - n_fringe - g                 # rings below k cut holes
        if (1.0 - frac(k)) * (r_out - r_body) >= cells * h:
            return g
    return noj - n_fringe - 1


def mems_batch(n=64, seed=0, n_steps=200, n_inner=10, ni_range=(48, 192), ntheta_range=(64, 128),
               nv_range=(20, 40), Kn_range=(0.01, 2.0), Tw_range=(1.0, 2.0)) -> List[Case]:
    """Serving-style sweep of independent oscillating-plate instances
    (uneven sizes): background n_i in {48, 56, ..., 192} with n_j = n_i / 2,
    O-grid n_theta in {64, 72, ..., 128} with n_r = n_theta / 4, N_vx = N_vy
    in {20, ..., 40}, Kn log-uniform, wall temperature uniform; everything
    else as `mems`, except that coarse backgrounds get more O-grid gap layers
    (overlap_gap_layers) so that no receptor is left without a donor.
    Seeded (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        nbi = int(rng.integers(ni_range[0] // 8, ni_range[1] // 8 + 1)) * 8
        nth = int(rng.integers(ntheta_range[0] // 8, ntheta_range[1] // 8 + 1)) * 8
        nv = int(rng.integers(nv_range[0], nv_range[1] + 1))
        Kn = float(10.0 ** rng.uniform(math.log10(Kn_range[0]), math.log10(Kn_range[1])))
        Tw = float(rng.uniform(*Tw_range))
        gap = overlap_gap_layers(nbi, nth // 4, 1.1, 0.25, 0.1)
        out.append(mems(nbi=nbi, nbj=nbi // 2, noi=nth, noj=nth // 4, nv=nv, Kn=Kn, Tw=Tw,
                        n_steps=n_steps, n_inner=n_inner, n_gap=gap))
    return out


def random_prim(case: Case, seed: int, amp_rho=0.2, amp_u=0.3, amp_T=0.2):
    """Smooth-plus-noise primitive field (tests): every cell gets its own
    density, velocity and temperature around the case's initial state."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = case.init_prim.copy()
    n = p.shape[0]
    p[:, 0] *= 1.0 + rng.uniform(-amp_rho, amp_rho, n)
    p[:, 1] += rng.uniform(-amp_u, amp_u, n)
    p[:, 2] += rng.uniform(-amp_u, amp_u, n)
    p[:, 3] *= 1.0 + rng.uniform(-amp_T, amp_T, n)
    return p
