"""Time-marching loop of the oracle (test infrastructure).

Sec. 3, the outer loop per physical step: (1) prescribed motion of every
block (the case's affine maps), (2) overset assembly at t^{n+1} when there
is more than one block, (3) one implicit unsteady UGKS step (Sec. 2.2)."""
from __future__ import annotations

import numpy as np

from . import kinetic as kn
from . import mesh, overset, ugks


class Run:
    def __init__(self, case, prim=None, status=None):
        self.case = case
        self.gas = kn.Gas(case.K, case.Pr, case.omega, case.mu_ref)
        self.dvs = kn.make_dvs(case.nvx, case.nvy, *case.vbox)
        self.topo = mesh.Topology(case.blocks)
        r, ux, uy, T = case.farfield
        Winf = kn.conservative(r, ux, uy, 1.0 / (2.0 * T), self.gas)
        self.setup = ugks.Setup(self.topo, self.gas, self.dvs, Winf,
                                case.cfl_s, case.cfl_pseudo)
        self.state = ugks.initial_state(self.setup, case.init_prim if prim is None else prim)
        self.t = 0.0
        self.multi = len(case.blocks) > 1
        self.conn = None
        if self.multi:
            self.conn = overset.connect(self.topo, case.nodes_at(0.0))
            self.status = self.conn.status
        else:
            self.status = np.zeros(self.topo.nc, dtype=np.int64)
        if status is not None:
            self.status = status
        self.info = None
        self.geo = None

    def geometry(self, t=None, dt=None):
        t = self.t if t is None else t
        dt = self.case.dt if dt is None else dt
        return mesh.geometry(self.topo, self.case.nodes_at(t), self.case.nodes_at(t + dt), dt)

    def step(self, n_inner=None, dt=None):
        case = self.case
        dt = case.dt if dt is None else dt
        n_inner = case.n_inner if n_inner is None else n_inner
        geo = self.geometry(self.t, dt)
        interp = fresh = None
        if self.multi:
            conn = overset.connect(self.topo, case.nodes_at(self.t + dt), self.status)
            self.conn = conn
            self.status = conn.status
            interp = lambda st: overset.interpolate(st, conn.receptors, conn.donors, conn.weights)
            fresh = lambda st: overset.interpolate(st, conn.fresh, conn.fresh_donors,
                                                   conn.fresh_weights)
        self.state, self.info = ugks.implicit_step(self.setup, geo, self.state, dt, n_inner,
                                                   self.status, interp, fresh)
        self.geo = geo
        self.t += dt
        return self.state
