"""Newton-Euler coupling of rigid-body blocks for the oracle (test
infrastructure; only tests/ may use it).

Sec. 3 Step 1 lets the motion of a moving domain follow the Newton-Euler
equations instead of a given function.  In 2D a rigid body carried by one
block has three degrees of freedom: the displacement d of a reference point
c, the rotation angle a about it, and their rates V and w.  Per unit depth,

    m dV/dt = F,    I dw/dt = M,    dd/dt = V,    da/dt = w,

with F and M the force and torque (about the current reference point) that
the gas exerts on the body's wall.  Readings (the paper gives no time
discretisation of the coupling):

  C1 loose coupling: the body advances from t^n to t^{n+1} with the wall
     force and torque of the last flux evaluation of the previous physical
     step (zero before the first step), rates first, then positions
     (semi-implicit Euler);
  C2 the wall force is the sum over the block's wall faces of S times the
     momentum components of the wall macro flux (outward from the gas), the
     torque the sum of (x_f - c) x (S F_f) with the mid-time face centres x_f
     and c the reference point at t^n;
  C3 the block's map at t is x = R(a) (x_ref - c_ref) + c_ref + d.
"""
from __future__ import annotations

import math

import numpy as np

from . import mesh, overset, ugks
from .run import Run


class Body:
    def __init__(self, block, mass, inertia, center, velocity=(0.0, 0.0), omega=0.0):
        self.block = block
        self.m = mass
        self.inertia = inertia
        self.c = np.array(center, dtype=np.float64)
        self.d = np.zeros(2)
        self.a = 0.0
        self.V = np.array(velocity, dtype=np.float64)
        self.w = float(omega)

    def point(self):
        return self.c + self.d

    def advance(self, dt, F, M):
        """Reading C1."""
        self.V = self.V + dt * (np.asarray(F) / self.m)
        self.w = self.w + dt * (M / self.inertia)
        self.d = self.d + dt * self.V
        self.a = self.a + dt * self.w

    def affine_map(self):
        """Reading C3 as (m00, m01, m10, m11, b0, b1)."""
        ca, sa = math.cos(self.a), math.sin(self.a)
        b0 = self.c[0] + self.d[0] - (ca * self.c[0] - sa * self.c[1])
        b1 = self.c[1] + self.d[1] - (sa * self.c[0] + ca * self.c[1])
        return np.array([ca, -sa, sa, ca, b0, b1])


def wall_force_torque(run: Run, block: int, point) -> tuple:
    """Reading C2 from the last step of `run`."""
    fl = run.info.last_flux
    topo = run.setup.topo
    F = np.zeros(2)
    M = 0.0
    for n, f in enumerate(fl.wall_face):
        if topo.face_block[f] != block:
            continue
        fx = run.geo.S[f] * fl.wall_F[n, 1]
        fy = run.geo.S[f] * fl.wall_F[n, 2]
        F += (fx, fy)
        M += (run.geo.xf[f, 0] - point[0]) * fy - (run.geo.xf[f, 1] - point[1]) * fx
    return F, M


def nodes(case, maps):
    """Node coordinates of every block under the affine maps (m00, m01, m10,
    m11, b0, b1): x = (m00 x_ref + m01 y_ref) + b0, FP64 without contraction."""
    out = []
    for blk, A in zip(case.blocks, maps):
        x = blk.x_ref[..., 0]
        y = blk.x_ref[..., 1]
        X = np.empty_like(blk.x_ref)
        X[..., 0] = (A[0] * x + A[1] * y) + A[4]
        X[..., 1] = (A[2] * x + A[3] * y) + A[5]
        out.append(X)
    return out


class CoupledRun(Run):
    """Oracle outer loop (Sec. 3) with the bodies of some blocks moved by the
    gas; the other blocks keep the case's prescribed motion."""

    def __init__(self, case, bodies, prim=None):
        super().__init__(case, prim)
        self.bodies = bodies
        self.maps = np.array(case.motion(0.0), dtype=np.float64)

    def step_coupled(self, n_inner=None, dt=None):
        case = self.case
        dt = case.dt if dt is None else dt
        n_inner = case.n_inner if n_inner is None else n_inner
        for b in self.bodies:
            if self.info is None:
                b.advance(dt, np.zeros(2), 0.0)
            else:
                F, M = wall_force_torque(self, b.block, b.point())
                b.advance(dt, F, M)
        new_maps = np.array(case.motion(self.t + dt), dtype=np.float64)
        for b in self.bodies:
            new_maps[b.block] = b.affine_map()
        X0, X1 = nodes(case, self.maps), nodes(case, new_maps)
        geo = mesh.geometry(self.topo, X0, X1, dt)
        conn = overset.connect(self.topo, X1, self.status)
        self.conn = conn
        self.status = conn.status
        interp = lambda st: overset.interpolate(st, conn.receptors, conn.donors, conn.weights)
        fresh = lambda st: overset.interpolate(st, conn.fresh, conn.fresh_donors, conn.fresh_weights)
        self.state, self.info = ugks.implicit_step(self.setup, geo, self.state, dt, n_inner,
                                                   self.status, interp, fresh)
        self.geo = geo
        self.maps = new_maps
        self.t += dt
        return self.state
