"""Precision statement of the mixed path: FP32-mixed (and FP64) GPU density,
velocity, temperature, wall force and wall heat against the FP64 oracle after
several implicit steps, per workload, with the bound 1e-5 relative on the
macroscopic fields; the bf16 storage of f (experiment) is reported beside
them with a loose bound.  Run with -s to print the error table."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle.run import Run  # noqa: E402
from paper_2604_09984_gb300 import ugks as U  # noqa: E402
from paper_2604_09984_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(U.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    U.load()


def cases():
    c = {
        "channel": (wl.channel(ni=12, nj=7, nv=10, n_inner=3), 3),
        "mems": (wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=2), 3),
        "two_bodies": (wl.tsto(nbi=80, nbj=40, noi=24, noj=10, nv=22, n_inner=2), 1),
    }
    # the MEMS Knudsen numbers of the paper-shaped sweep (0.1, 0.5, 1.0), the
    # ends of the batched range (0.01, 2) and a near-continuum case (0.001,
    # dt_s / tau ~ 2 on the background cells, below 1 on the O-grid), so both
    # branches of the time integrals q1..q5 run
    for kn in (0.001, 0.01, 0.5, 1.0, 2.0):
        c["mems_kn%g" % kn] = (wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=16, stretch=1.15, n_inner=2, Kn=kn), 2)
    return c


def primitives(W, K):
    """rho, velocity, temperature (R = 1, D = 2, K internal degrees)."""
    rho = W[:, 0]
    V = W[:, 1:3] / rho[:, None]
    e = W[:, 3] / rho - 0.5 * (V * V).sum(1)
    return rho, V, 2.0 * e / (2.0 + 1.0 + K)


def wall_loads(r):
    """Per block: sum over its wall faces of S times the wall macro flux of the
    last flux evaluation (the oracle's counterpart of ugks_moments)."""
    fl = r.info.last_flux
    topo = r.setup.topo
    out = np.zeros((len(r.case.blocks), 4))
    for n, f in enumerate(fl.wall_face):
        out[topo.face_block[f]] += r.geo.S[f] * fl.wall_F[n]
    return out


def errors(W, wall, r):
    field = r.status == 0
    K = r.case.K
    rho, V, T = primitives(W[field], K)
    rr, Vr, Tr = primitives(r.state.W[field], K)
    wr = wall_loads(r)
    e = {
        "rho": np.abs(rho - rr).max() / np.abs(rr).max(),
        "V": np.abs(V - Vr).max() / max(np.abs(Vr).max(), 1e-3),
        "T": np.abs(T - Tr).max() / np.abs(Tr).max(),
        "W": np.abs(W[field] - r.state.W[field]).max() / np.abs(r.state.W[field]).max(),
    }
    # wall force components relative to the largest force magnitude (a
    # component can be near zero, e.g. the shear on the channel walls), heat
    # relative to the largest heat
    fscale = np.hypot(wr[:, 1], wr[:, 2]).max()
    for m, name in ((1, "Fx"), (2, "Fy")):
        e[name] = np.abs(wall[:, m] - wr[:, m]).max() / fscale if fscale > 0 else 0.0
    hscale = np.abs(wr[:, 3]).max()
    e["heat"] = np.abs(wall[:, 3] - wr[:, 3]).max() / hscale if hscale > 0 else 0.0
    return e


@pytest.mark.parametrize("which", ["channel", "mems", "two_bodies", "mems_kn0.001", "mems_kn0.01", "mems_kn0.5",
                                   "mems_kn1", "mems_kn2"])
def test_errors_against_oracle(which):
    case, nsteps = cases()[which]
    r = Run(case)
    solvers = {"FP32": U.Solver(case, U.FP32), "FP64": U.Solver(case, U.FP64),
               "BF16f": U.Solver(case, U.BF16F)}
    for _ in range(nsteps):
        r.step()
        for s in solvers.values():
            s.advance()
    res = {}
    for name, s in solvers.items():
        W, q, st, wall = s.moments()
        assert np.array_equal(st, r.status)
        res[name] = errors(W, wall, r)
    print("\n%-10s %-4s " % (which, "") + " ".join("%9s" % k for k in res["FP32"]))
    for name, e in res.items():
        print("%-10s %-4s " % ("", name) + " ".join("%9.2e" % v for v in e.values()))
    for k in ("rho", "V", "T", "W"):
        assert res["FP32"][k] < 1e-5, (k, res["FP32"][k])
        assert res["FP64"][k] < 1e-12, (k, res["FP64"][k])
    for k in ("Fx", "Fy", "heat"):
        assert res["FP32"][k] < 1e-4, (k, res["FP32"][k])
        assert res["FP64"][k] < 1e-10, (k, res["FP64"][k])
    # bf16 storage of f (experiment): 8-bit significands, every store rounds
    for k in ("rho", "T", "W"):
        assert res["BF16f"][k] < 2e-2, (k, res["BF16f"][k])
