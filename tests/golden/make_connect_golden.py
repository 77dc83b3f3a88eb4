"""Writes the oracle's overset connectivity (Sec. 3.1 assembly, Sec. 3.2
stencils and inverse-distance weights) of the full-size MEMS and two-body
meshes to ``connect_<name>.npz`` beside this script: at t = 0 and after one
move to t1 (with the t = 0 status as the previous one).  Calls only the
oracle and the seeded input module; the GPU tests compare the library's
assembly against these files bit for bit.  Run from the repository root:

    python tests/golden/make_connect_golden.py [mems|tsto ...]
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))

from oracle import mesh, overset  # noqa: E402
from paper_2604_09984_gb300 import workloads as wl  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def move_time(name, case):
    """t1: 30 steps of the plate (MEMS: 342 cells change status); 200 steps
    of the two-body separation.  Both moves leave no orphan receptor."""
    if name == "mems":
        return 30 * case.dt
    return 200 * case.dt


CASES = {"mems": lambda: wl.mems(), "tsto": lambda: wl.tsto()}


def write(name):
    case = CASES[name]()
    topo = mesh.Topology(case.blocks)
    t1 = move_time(name, case)
    c0 = overset.connect(topo, case.nodes_at(0.0))
    c1 = overset.connect(topo, case.nodes_at(t1), c0.status)
    out = {"t1": np.float64(t1)}
    for tag, c in (("t0", c0), ("t1", c1)):
        out[tag + "_status"] = c.status.astype(np.int8)
        out[tag + "_receptors"] = c.receptors.astype(np.int32)
        out[tag + "_donors"] = c.donors.astype(np.int32)
        out[tag + "_weight_bits"] = c.weights.view(np.int64)
        out[tag + "_fresh"] = c.fresh.astype(np.int32)
        out[tag + "_n_orphan"] = np.int64(c.n_orphan)
    np.savez_compressed(os.path.join(HERE, "connect_%s.npz" % name), **out)
    print(name, "receptors", c0.receptors.size, c1.receptors.size, "fresh", c1.fresh.size,
          "orphans", c0.n_orphan, c1.n_orphan, flush=True)


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(CASES)):
        write(n)
