"""ctypes binding of libugks (C ABI in include/ugks.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  The library must be built (``__graft_entry__.build()`` or
``python -m paper_2604_09984_gb300.build_lib``); loading fails loudly when it
is missing -- there is no fallback path.  PyTorch provides the device
workspace and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int64, c_size_t, c_void_p

import numpy as np

from . import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libugks.so")

OK = 0
ERR = {-1: "UGKS_ERR_ARG", -2: "UGKS_ERR_CUDA", -3: "UGKS_ERR_GEOMETRY", -4: "UGKS_ERR_ORPHAN",
       -5: "UGKS_ERR_NONPHYSICAL", -6: "UGKS_ERR_WORKSPACE", -7: "UGKS_ERR_ORDER",
       -8: "UGKS_ERR_TIMEOUT"}
FP64, FP32, BF16F = 0, 1, 2      # BF16F: FP32 arithmetic, f stored as bf16 pairs (experiment)
STATIC_SCRATCH_DOUBLES = 1 << 19     # UGKS_STATIC_SCRATCH_DOUBLES
FIELD, RECEPTOR, HOLE = 0, 1, 2


class Params(ctypes.Structure):
    _fields_ = [("precision", c_int), ("nvx", c_int), ("nvy", c_int),
                ("vx_min", c_double), ("vx_max", c_double), ("vy_min", c_double), ("vy_max", c_double),
                ("K", c_int), ("Pr", c_double), ("omega", c_double), ("mu_ref", c_double),
                ("cfl_s", c_double), ("cfl_pseudo", c_double), ("farfield", c_double * 4),
                ("shard_iy0", c_int), ("shard_iy1", c_int)]


class BlockDesc(ctypes.Structure):
    _fields_ = [("ni", c_int), ("nj", c_int), ("periodic_i", c_int), ("bc", c_int * 4),
                ("wall_T", c_double * 4), ("priority", c_int), ("n_fringe", c_int),
                ("n_gap", c_int), ("x_ref", POINTER(c_double))]


class ConnectStats(ctypes.Structure):
    _fields_ = [("n_field", c_int), ("n_receptor", c_int), ("n_hole", c_int),
                ("n_fresh", c_int), ("n_orphan", c_int)]


class StepMetrics(ctypes.Structure):
    _fields_ = [("res_macro_sq", c_double), ("res_micro_sq", c_double), ("fix_sq", c_double),
                ("total", c_double * 4)]


# exchange of a velocity-sharded context: fn(which, stream, user) -> 0
EXCHANGE_FN = ctypes.CFUNCTYPE(c_int, c_int, c_void_p, c_void_p)

SYMBOLS = {
    "ugks_workspace_query": (c_int, [POINTER(Params), c_int, POINTER(BlockDesc), POINTER(c_size_t)]),
    "ugks_create": (c_int, [POINTER(Params), c_void_p, c_size_t, c_void_p, POINTER(c_void_p)]),
    "ugks_destroy": (c_int, [c_void_p]),
    "ugks_last_error": (ctypes.c_char_p, [c_void_p]),
    "ugks_init_mesh": (c_int, [c_void_p, c_int, POINTER(BlockDesc), POINTER(c_double)]),
    "ugks_move_mesh": (c_int, [c_void_p, c_double, POINTER(c_double)]),
    "ugks_overset_connect": (c_int, [c_void_p, POINTER(ConnectStats)]),
    "ugks_step": (c_int, [c_void_p, c_double, c_int]),
    "ugks_set_graphs": (c_int, [c_void_p, c_int]),
    "ugks_set_metrics": (c_int, [c_void_p, c_int]),
    "ugks_get_metrics": (c_int, [c_void_p, POINTER(StepMetrics)]),
    "ugks_graph_stats": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_int64)]),
    "ugks_advance_batch": (c_int, [POINTER(c_void_p), c_int, POINTER(c_double), POINTER(POINTER(c_double)),
                                   c_int, POINTER(c_int)]),
    "ugks_moments": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ugks_wall_torque": (c_int, [c_void_p, POINTER(c_double), c_void_p]),
    "ugks_autotune": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int),
                              POINTER(c_int), POINTER(c_int)]),
    "ugks_sizes": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "ugks_get_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ugks_set_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ugks_get_checkpoint": (c_int, [c_void_p, POINTER(c_double), c_void_p, c_void_p]),
    "ugks_set_checkpoint": (c_int, [c_void_p, c_double, c_void_p, c_void_p]),
    "ugks_eval_flux": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ugks_get_connectivity": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ugks_get_geometry": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ugks_launch_count": (c_int64, [c_void_p]),
    "ugks_set_wait_limit": (c_int, [c_void_p, c_int]),
    "ugks_shard_set_exchange": (c_int, [c_void_p, EXCHANGE_FN, c_void_p]),
    "ugks_shard_buffers": (c_int, [c_void_p, POINTER(c_size_t), POINTER(c_size_t), POINTER(c_size_t),
                                   POINTER(c_size_t)]),
    "ugks_probe_fp64": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p]),
    "ugks_profile_enable": (c_int, [c_void_p, c_int]),
    "ugks_profile_read": (c_int, [c_void_p, POINTER(c_double), POINTER(c_int64), c_int]),
    "ugks_idw_interpolate_static": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p,
                                            c_int, c_void_p, c_void_p, c_void_p]),
}
PROF_GROUPS = ["geometry", "connect", "interp", "cell", "face_reduce", "face_coef",
               "macro_sweep", "micro_fwd", "micro_bwd", "moments", "flux", "residual"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libugks.so and declare its symbols; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libugks.so not built (%s): run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SYMBOLS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class UgksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERR.get(code, "?"), code, msg))
        self.code = code


def make_params(case: wl.Case, precision: int, shard=None) -> Params:
    p = Params()
    if shard is not None:
        p.shard_iy0, p.shard_iy1 = int(shard[0]), int(shard[1])
    p.precision = precision
    p.nvx, p.nvy = case.nvx, case.nvy
    p.vx_min, p.vx_max, p.vy_min, p.vy_max = case.vbox
    p.K, p.Pr, p.omega, p.mu_ref = case.K, case.Pr, case.omega, case.mu_ref
    p.cfl_s, p.cfl_pseudo = case.cfl_s, case.cfl_pseudo
    for i in range(4):
        p.farfield[i] = case.farfield[i]
    return p


def make_blocks(case: wl.Case):
    """Block descriptors plus the node arrays they point to (keep both)."""
    arrs = []
    descs = (BlockDesc * len(case.blocks))()
    for i, b in enumerate(case.blocks):
        xr = np.ascontiguousarray(b.x_ref.transpose(1, 0, 2), dtype=np.float64)
        arrs.append(xr)
        d = descs[i]
        d.ni, d.nj, d.periodic_i = b.ni, b.nj, int(b.periodic_i)
        for s in range(4):
            d.bc[s] = int(b.bc[s])
            d.wall_T[s] = float(b.wall_T[s])
        d.priority, d.n_fringe, d.n_gap = b.priority, b.n_fringe, b.n_gap
        d.x_ref = xr.ctypes.data_as(POINTER(c_double))
    return descs, arrs


def workspace_bytes(case: wl.Case, precision: int) -> int:
    lib = load()
    p = make_params(case, precision)
    descs, _keep = make_blocks(case)
    n = c_size_t(0)
    r = lib.ugks_workspace_query(ctypes.byref(p), len(case.blocks), descs, ctypes.byref(n))
    if r != OK:
        raise UgksError(r, "workspace query")
    return int(n.value)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return c_void_p(t.ctypes.data)
    return c_void_p(t.data_ptr())


class Solver:
    """One libugks context for a workload: owns the device workspace (a torch
    uint8 tensor) and runs on the current torch CUDA stream."""

    def __init__(self, case: wl.Case, precision: int = FP64, device="cuda", stream=None, prim=None, shard=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.case = case
        self.precision = precision
        self.shard = shard
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._p = make_params(case, precision, shard)
        self._descs, self._keep = make_blocks(case)
        nbytes = c_size_t(0)
        self._check(self.lib.ugks_workspace_query(ctypes.byref(self._p), len(case.blocks),
                                                  self._descs, ctypes.byref(nbytes)), None)
        self.ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        ctx = c_void_p()
        self._check(self.lib.ugks_create(ctypes.byref(self._p), c_void_p(self.ws.data_ptr()),
                                         nbytes.value, c_void_p(self.stream.cuda_stream),
                                         ctypes.byref(ctx)), None)
        self.ctx = ctx
        prim = np.ascontiguousarray(case.init_prim if prim is None else prim, dtype=np.float64)
        self._check(self.lib.ugks_init_mesh(self.ctx, len(case.blocks), self._descs,
                                            prim.ctypes.data_as(POINTER(c_double))))
        nc, nf, nv, nvp = c_int(), c_int(), c_int(), c_int()
        self._check(self.lib.ugks_sizes(self.ctx, ctypes.byref(nc), ctypes.byref(nf),
                                        ctypes.byref(nv), ctypes.byref(nvp)))
        self.nc, self.nf, self.nv, self.nvp = nc.value, nf.value, nv.value, nvp.value
        self.t = 0.0
        self.last_stats = None
        self.stepped = False

    # -------------------------------------------------------------- errors
    def _check(self, r, ctx="self"):
        if r != OK:
            c = self.ctx if ctx == "self" else None
            msg = self.lib.ugks_last_error(c).decode() if c is not None else ""
            xerr = getattr(self, "_xerr", None)
            if xerr:
                msg += " (exchange: %s)" % xerr
                self._xerr = None
            raise UgksError(r, msg)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.ugks_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------- the ABI
    def move_mesh(self, t_new, affine=None):
        a = np.ascontiguousarray(self.case.motion(t_new) if affine is None else affine, dtype=np.float64)
        self._check(self.lib.ugks_move_mesh(self.ctx, float(t_new), a.ctypes.data_as(POINTER(c_double))))
        self._t_new = t_new

    def overset_connect(self):
        st = ConnectStats()
        self._check(self.lib.ugks_overset_connect(self.ctx, ctypes.byref(st)))
        self.last_stats = dict(n_field=st.n_field, n_receptor=st.n_receptor, n_hole=st.n_hole,
                               n_fresh=st.n_fresh, n_orphan=st.n_orphan)
        return self.last_stats

    def step(self, dt=None, n_inner=None):
        dt = self._t_new - self.t if dt is None else dt
        n_inner = self.case.n_inner if n_inner is None else n_inner
        self._check(self.lib.ugks_step(self.ctx, float(dt), int(n_inner)))
        self.t = self._t_new
        self.stepped = True

    def advance(self, n_inner=None, dt=None):
        """One physical step of the outer loop (Sec. 3): motion, assembly, evolve."""
        dt = self.case.dt if dt is None else dt
        self.move_mesh(self.t + dt)
        self.overset_connect()
        self.step(dt, n_inner)

    def wall_torque(self, centers):
        """Torque of each block's wall force about centers[b] (ugks_wall_torque)."""
        c = np.ascontiguousarray(centers, dtype=np.float64).reshape(len(self.case.blocks), 2)
        out = np.empty(len(self.case.blocks))
        self._check(self.lib.ugks_wall_torque(self.ctx, c.ctypes.data_as(POINTER(c_double)), _ptr(out)))
        return out

    def advance_coupled(self, bodies, n_inner=None, dt=None):
        """One physical step with rigid bodies moved by the gas (Sec. 3 Step 1,
        Newton-Euler): each body is updated from the wall force and torque of
        the previous step's last flux evaluation (none before the first step),
        then motion, assembly and the implicit step follow as in advance()."""
        dt = self.case.dt if dt is None else dt
        nb = len(self.case.blocks)
        if self.stepped:
            _, _, _, wall = self.moments()
            ctr = np.zeros((nb, 2))
            for b in bodies:
                ctr[b.block] = b.center()
            tq = self.wall_torque(ctr)
            for b in bodies:
                b.update(dt, wall[b.block, 1:3], tq[b.block])
        else:
            for b in bodies:
                b.update(dt, np.zeros(2), 0.0)
        A = np.array(self.case.motion(self.t + dt), dtype=np.float64)
        for b in bodies:
            A[b.block] = b.affine()
        self.move_mesh(self.t + dt, A)
        self.overset_connect()
        self.step(dt, n_inner)

    def autotune(self, reps=3):
        """Pick the fastest tiles on this context's own state (ugks_autotune);
        returns (sweep items per warp step, sweep velocities per lane, forward
        ring depth, backward ring depth, face-kernel velocities per chunk,
        face-kernel threads per face slot)."""
        v = [c_int() for _ in range(6)]
        self._check(self.lib.ugks_autotune(self.ctx, int(reps), *[ctypes.byref(x) for x in v]))
        self.tiles = tuple(x.value for x in v)
        return self.tiles

    def moments(self, W=None, q=None, status=None, wall=None):
        """Copy W, q, status and wall loads into the given buffers (numpy or
        torch, host or device); allocates host numpy arrays when omitted."""
        if W is None:
            W = np.empty((self.nc, 4))
        if q is None:
            q = np.empty((self.nc, 2))
        if status is None:
            status = np.empty(self.nc, dtype=np.int32)
        if wall is None:
            wall = np.empty((len(self.case.blocks), 4))
        self._check(self.lib.ugks_moments(self.ctx, _ptr(W), _ptr(q), _ptr(status), _ptr(wall)))
        return W, q, status, wall

    def get_state(self):
        torch = self.torch
        f = torch.empty((self.nc, self.nv, 2), dtype=torch.float64, device=self.device)
        W = np.empty((self.nc, 4))
        q = np.empty((self.nc, 2))
        self._check(self.lib.ugks_get_state(self.ctx, _ptr(f), _ptr(W), _ptr(q)))
        return f, W, q

    def set_state(self, f=None, W=None, q=None):
        torch = self.torch
        ft = None
        if f is not None:
            ft = torch.as_tensor(np.asarray(f, dtype=np.float64) if not isinstance(f, torch.Tensor) else f,
                                 dtype=torch.float64).to(self.device).contiguous()
        Wn = None if W is None else np.ascontiguousarray(W, dtype=np.float64)
        qn = None if q is None else np.ascontiguousarray(q, dtype=np.float64)
        self._check(self.lib.ugks_set_state(self.ctx, _ptr(ft), _ptr(Wn), _ptr(qn)))

    def checkpoint(self):
        """Everything needed to continue bit for bit from between two steps:
        f (device, FP64), W, q, t, the node coordinates at t and the cell
        status (ugks_get_state, ugks_get_checkpoint)."""
        f, W, q = self.get_state()
        nn = sum((b.ni + 1) * (b.nj + 1) for b in self.case.blocks)
        nodes = np.empty((nn, 2))
        status = np.empty(self.nc, dtype=np.int32)
        t = c_double()
        self._check(self.lib.ugks_get_checkpoint(self.ctx, ctypes.byref(t), _ptr(nodes), _ptr(status)))
        return {"f": f, "W": W, "q": q, "t": float(t.value), "nodes": nodes, "status": status}

    def restore(self, ck):
        """Continue from a checkpoint() of a context of the same case."""
        nodes = np.ascontiguousarray(ck["nodes"], dtype=np.float64)
        status = np.ascontiguousarray(ck["status"], dtype=np.int32)
        self._check(self.lib.ugks_set_checkpoint(self.ctx, float(ck["t"]), _ptr(nodes), _ptr(status)))
        self.set_state(ck["f"], ck["W"], ck["q"])
        self.t = float(ck["t"])

    def eval_flux(self):
        torch = self.torch
        D = torch.empty((self.nc, self.nv, 2), dtype=torch.float64, device=self.device)
        F = np.empty((self.nc, 4))
        self._check(self.lib.ugks_eval_flux(self.ctx, _ptr(D), _ptr(F)))
        return D, F

    def connectivity(self):
        st = np.empty(self.nc, dtype=np.int32)
        dn = np.empty((self.nc, 5), dtype=np.int32)
        w = np.empty((self.nc, 5))
        self._check(self.lib.ugks_get_connectivity(self.ctx, _ptr(st), _ptr(dn), _ptr(w)))
        return st, dn, w

    def geometry(self):
        out = dict(vol_old=np.empty(self.nc), vol_new=np.empty(self.nc), xc=np.empty((self.nc, 2)),
                   dts=np.empty(self.nc), Sn=np.empty((self.nf, 2)), SUn=np.empty(self.nf))
        self._check(self.lib.ugks_get_geometry(self.ctx, *(_ptr(out[k]) for k in
                                                          ("vol_old", "vol_new", "xc", "dts", "Sn", "SUn"))))
        return out

    def launch_count(self):
        return int(self.lib.ugks_launch_count(self.ctx))

    def set_graphs(self, on: bool):
        """CUDA-graph path of ugks_step on or off (ugks_set_graphs)."""
        self._check(self.lib.ugks_set_graphs(self.ctx, int(bool(on))))

    def set_metrics(self, on: bool):
        """Record step metrics in the following steps (ugks_set_metrics)."""
        self._check(self.lib.ugks_set_metrics(self.ctx, int(bool(on))))

    def metrics(self):
        """Metrics of the last step (ugks_get_metrics): the L2 norms of the
        macro residual R, the micro residual r and the Step-7 moment fix of
        the last inner iteration, and the totals of Omega W over the field."""
        m = StepMetrics()
        self._check(self.lib.ugks_get_metrics(self.ctx, ctypes.byref(m)))
        return {"res_macro": m.res_macro_sq ** 0.5, "res_micro": m.res_micro_sq ** 0.5,
                "fix": m.fix_sq ** 0.5, "total": [float(x) for x in m.total],
                "res_macro_sq": m.res_macro_sq, "res_micro_sq": m.res_micro_sq, "fix_sq": m.fix_sq}

    def graph_stats(self):
        """(captures, replays) of the step's CUDA graphs (ugks_graph_stats)."""
        c, r = c_int64(), c_int64()
        self._check(self.lib.ugks_graph_stats(self.ctx, ctypes.byref(c), ctypes.byref(r)))
        return int(c.value), int(r.value)

    def set_exchange(self, fn):
        """Exchange of a velocity-sharded context (ugks_shard_set_exchange):
        fn(which) -> None turns this shard's partial sums in
        shard_views()[which] into the sums over all shards."""
        import weakref
        me = weakref.ref(self)           # no reference cycle through the callback

        def cb(which, stream, user):
            try:
                fn(int(which))
                return 0
            except Exception as e:  # reported as UGKS_ERR_ARG by the library
                s = me()
                if s is not None:
                    s._xerr = repr(e)
                return 1
        self._xfn = EXCHANGE_FN(cb)      # keep a reference while the context lives
        self._check(self.lib.ugks_shard_set_exchange(self.ctx, self._xfn, None))

    def shard_views(self):
        """The two exchange buffers (face sums, cell moment sums) as FP64
        views of this context's workspace."""
        fo, fc, co, cc = c_size_t(), c_size_t(), c_size_t(), c_size_t()
        self._check(self.lib.ugks_shard_buffers(self.ctx, ctypes.byref(fo), ctypes.byref(fc),
                                                ctypes.byref(co), ctypes.byref(cc)))
        f = self.ws[fo.value:fo.value + 8 * fc.value].view(self.torch.float64)
        c = self.ws[co.value:co.value + 8 * cc.value].view(self.torch.float64)
        return f, c

    def set_wait_limit(self, polls):
        """Polls of the sweeps' bounded waits (ugks_set_wait_limit; 0 = default)."""
        self._check(self.lib.ugks_set_wait_limit(self.ctx, int(polls)))

    def profile(self, on: bool):
        self._check(self.lib.ugks_profile_enable(self.ctx, int(bool(on))))

    def profile_read(self, reset=True):
        ms = (c_double * len(PROF_GROUPS))()
        n = (c_int64 * len(PROF_GROUPS))()
        self._check(self.lib.ugks_profile_read(self.ctx, ms, n, int(bool(reset))))
        return {g: (float(ms[i]), int(n[i])) for i, g in enumerate(PROF_GROUPS)}


class StepLog:
    """Per-step metrics as JSON lines, one object per physical step: step
    index, t, the L2 norms of R, r and the moment fix of the last inner
    iteration, the field totals of Omega W, the relative change of the field
    mass since the previous logged step (the conservation defect; null on the
    first line), the last assembly's counters and the step's wall time in ms
    (host clock around the step and the metrics read, which synchronises).
    The solver records metrics from the first advance() on."""

    def __init__(self, out):
        self._own = isinstance(out, (str, os.PathLike))
        self.fh = open(out, "w") if self._own else out
        self.n = 0
        self._mass = None

    def record(self, solver, ms=None, m=None):
        import json
        m = solver.metrics() if m is None else m
        mass = m["total"][0]
        line = {"step": self.n, "t": solver.t, "res_macro": m["res_macro"], "res_micro": m["res_micro"],
                "fix": m["fix"], "total": m["total"],
                "mass_defect": None if self._mass is None else (mass - self._mass) / self._mass,
                "ms": ms}
        line.update(getattr(solver, "last_stats", None) or {})
        self.fh.write(json.dumps(line) + "\n")
        self.fh.flush()
        self._mass = mass
        self.n += 1
        return line

    def advance(self, solver, **kw):
        import time
        solver.set_metrics(True)
        t0 = time.perf_counter()
        solver.advance(**kw)
        m = solver.metrics()            # synchronises: the step is done
        return self.record(solver, 1e3 * (time.perf_counter() - t0), m)

    def close(self):
        if self._own:
            self.fh.close()


def advance_batch(solvers, n_inner=None):
    """One physical step of every solver (instance) through
    ugks_advance_batch: motion from each case's own map at t + dt, overset
    assembly and the implicit step, issued without waiting on the device.
    Solvers created on distinct streams run concurrently."""
    lib = load()
    n = len(solvers)
    if n == 0:
        return
    inner = {s.case.n_inner if n_inner is None else n_inner for s in solvers}
    if len(inner) != 1:
        raise ValueError("one n_inner for the whole batch")
    ctxs = (c_void_p * n)(*[s.ctx.value for s in solvers])
    t_new = (c_double * n)(*[s.t + s.case.dt for s in solvers])
    maps = [np.ascontiguousarray(s.case.motion(t_new[i]), dtype=np.float64) for i, s in enumerate(solvers)]
    aff = (POINTER(c_double) * n)(*[m.ctypes.data_as(POINTER(c_double)) for m in maps])
    failed = c_int(-1)
    r = lib.ugks_advance_batch(ctxs, n, t_new, aff, int(inner.pop()), ctypes.byref(failed))
    if r != OK:
        s = solvers[failed.value] if failed.value >= 0 else None
        msg = lib.ugks_last_error(s.ctx).decode() if s is not None else ""
        raise UgksError(r, "instance %d: %s" % (failed.value, msg))
    for i, s in enumerate(solvers):
        s._t_new = t_new[i]
        s.t = t_new[i]


class RigidBody:
    """Rigid body carried by one block (3 degrees of freedom in 2D): the
    displacement of its reference centre, its rotation angle and their
    rates.  update() applies the gas force and torque per unit depth over one
    step, rates first, then positions (semi-implicit Euler); affine() is the
    block's map x = R (x_ref - c) + c + displacement."""

    def __init__(self, block, mass, inertia, center, velocity=(0.0, 0.0), omega=0.0):
        self.block = int(block)
        self.mass = float(mass)
        self.inertia = float(inertia)
        self.c_ref = np.asarray(center, dtype=np.float64)
        self.disp = np.zeros(2)
        self.angle = 0.0
        self.vel = np.asarray(velocity, dtype=np.float64).copy()
        self.omega = float(omega)

    def center(self):
        return self.c_ref + self.disp

    def update(self, dt, force, torque):
        self.vel = self.vel + dt * np.asarray(force, dtype=np.float64) / self.mass
        self.omega = self.omega + dt * float(torque) / self.inertia
        self.disp = self.disp + dt * self.vel
        self.angle = self.angle + dt * self.omega

    def affine(self):
        co, si = np.cos(self.angle), np.sin(self.angle)
        cx, cy = self.c_ref
        b0 = cx + self.disp[0] - (co * cx - si * cy)
        b1 = cy + self.disp[1] - (si * cx + co * cy)
        return np.array([co, -si, si, co, b0, b1])


# ------------------------------------------------------ velocity sharding
def shard_rows(nvy, n):
    """Contiguous, balanced row ranges [iy0, iy1) of the velocity grid for n
    shards (the first nvy % n shards take one row more)."""
    if not 1 <= n <= nvy:
        raise ValueError("1 <= shards <= velocity rows")
    q, r = divmod(nvy, n)
    out, iy = [], 0
    for i in range(n):
        m = q + (1 if i < r else 0)
        out.append((iy, iy + m))
        iy += m
    return out


def fixed_order_allreduce(t, group=None):
    """Sum of tensor t over the ranks of a torch.distributed group, summed in
    rank order (so every rank gets the same bits), written back into t."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t.contiguous(), group=group)
    acc = parts[0].clone()
    for p in parts[1:]:
        acc += p
    t.copy_(acc)
    return t


def distributed_exchange(solver, group=None):
    """Exchange of a shard held by this rank: fixed-order all-reduce of its
    buffers over the ranks of `group` (one shard per rank, NCCL on GPUs)."""
    views = solver.shard_views()

    def fn(which):
        solver.stream.synchronize()
        fixed_order_allreduce(views[which], group)
        solver.torch.cuda.current_stream(solver.device).synchronize()
    solver.set_exchange(fn)


class ShardSet:
    """Velocity shards of one case on one GPU, stepped together: every shard
    context runs its ugks_* call in its own host thread, and the exchange sums
    the shards' buffers in shard order (the same bits on every shard).  This
    is the sharded data path of several GPUs with the collective replaced by
    an in-process sum."""

    def __init__(self, case, precision, nshards, device="cuda", prim=None):
        import threading
        import torch
        self.case = case
        self.rows = shard_rows(case.nvy, nshards)
        self.solvers = [Solver(case, precision, device=device, prim=prim, shard=r,
                               stream=torch.cuda.Stream(device=device)) for r in self.rows]
        self.views = [s.shard_views() for s in self.solvers]
        self._bar = threading.Barrier(nshards)
        self._torch = torch
        for i, s in enumerate(self.solvers):
            s.set_exchange(self._make_fn(i))

    def _make_fn(self, i):
        # the closure holds the buffers, the barrier and the shard's stream,
        # not the set itself (no cycle set -> solver -> callback -> set)
        torch, views, bar, stream = self._torch, self.views, self._bar, self.solvers[i].stream

        def fn(which):
            stream.synchronize()
            bar.wait()
            if i == 0:
                acc = views[0][which].clone()
                for v in views[1:]:
                    acc += v[which]
                for v in views:
                    v[which].copy_(acc)
                torch.cuda.synchronize()
            bar.wait()
        return fn

    def close(self):
        for s in self.solvers:
            s.close()

    def _parallel(self, name, *args):
        import threading
        errs = [None] * len(self.solvers)

        def run(i):
            try:
                getattr(self.solvers[i], name)(*args)
            except BaseException as e:       # noqa: BLE001 (re-raised below)
                errs[i] = e
                self._bar.abort()
        ts = [threading.Thread(target=run, args=(i,)) for i in range(len(self.solvers))]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        for e in errs:
            if e is not None:
                raise e

    def advance(self, n_inner=None):
        """One physical step of every shard (motion and assembly per shard,
        then the sharded implicit step)."""
        dt = self.case.dt
        for s in self.solvers:
            s.move_mesh(s.t + dt)
            s.overset_connect()
        self._parallel("step", dt, n_inner)

    def moments(self):
        return self.solvers[0].moments()

    def get_f(self):
        """f of the whole velocity grid (the shards' rows side by side)."""
        return self._torch.cat([s.get_state()[0] for s in self.solvers], dim=1)
