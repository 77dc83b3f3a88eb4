"""Pins of the oracle's Newton-Euler coupling (Sec. 3 Step 1): the time
update against its closed form under a constant load, the block map against
a rotation about the moving reference point, and the gas loads of a particle
released along the symmetry line of a box (no lift, no torque, drag against
the motion)."""
import math

import numpy as np
import pytest

from oracle import coupling
from paper_2604_09984_gb300 import workloads as wl


def test_update_matches_closed_form_under_constant_load():
    m, inertia, dt, n = 2.0, 0.5, 0.1, 7
    F, M = np.array([0.3, -0.2]), 0.05
    b = coupling.Body(1, m, inertia, (1.0, 0.5), velocity=(0.4, 0.1), omega=0.2)
    for _ in range(n):
        b.advance(dt, F, M)
    # rates first: V_k = V0 + k dt F/m, positions sum dt V_k for k = 1..n
    V0, w0 = np.array([0.4, 0.1]), 0.2
    assert np.allclose(b.V, V0 + n * dt * F / m, rtol=0, atol=1e-15)
    assert np.allclose(b.d, n * dt * V0 + dt * dt * F / m * n * (n + 1) / 2, rtol=0, atol=1e-14)
    assert b.w == pytest.approx(w0 + n * dt * M / inertia, abs=1e-15)
    assert b.a == pytest.approx(n * dt * w0 + dt * dt * M / inertia * n * (n + 1) / 2, abs=1e-14)


def test_block_map_rotates_about_the_moving_point():
    b = coupling.Body(1, 1.0, 1.0, (1.0, 0.5))
    b.d = np.array([0.2, -0.1])
    b.a = 0.7
    A = b.affine_map()
    def apply(p):
        return np.array([A[0] * p[0] + A[1] * p[1] + A[4], A[2] * p[0] + A[3] * p[1] + A[5]])
    assert np.allclose(apply((1.0, 0.5)), (1.2, 0.4), atol=1e-15)
    r = 0.3
    q = apply((1.0 + r, 0.5))
    assert np.allclose(q, (1.2 + r * math.cos(0.7), 0.4 + r * math.sin(0.7)), atol=1e-15)
    assert np.isclose(np.linalg.det([[A[0], A[1]], [A[2], A[3]]]), 1.0)


def particle_run(**kw):
    case = wl.particle(nbi=48, nbj=24, noi=32, noj=10, nv=8, r_out=0.3, n_inner=2, **kw)
    meta = case.meta
    body = coupling.Body(meta["body_block"], meta["mass"], meta["inertia"], meta["center"],
                         velocity=meta["u0"], omega=meta["omega0"])
    return case, body, coupling.CoupledRun(case, [body])


def test_particle_on_the_symmetry_line_feels_drag_only():
    """Released along the box's mirror line: drag against the motion, lift
    and torque only at the level of the discretisation's asymmetries
    (lexicographic sweeps, donor tie-breaks: ~5e-5 of the drag)."""
    case, body, run = particle_run(u0=(0.3, 0.0))
    run.step_coupled()
    F, M = coupling.wall_force_torque(run, body.block, body.point())
    assert F[0] < 0.0
    assert abs(F[1]) < 1e-4 * abs(F[0])
    assert abs(M) < 1e-4 * abs(F[0]) * 0.1
    run.step_coupled()
    assert 0.0 < body.V[0] < 0.3 and body.d[0] > 0.0
    assert abs(body.V[1]) < 1e-4 * body.V[0]


def test_spinning_particle_feels_braking_torque():
    """Spinning at rest in the box centre: the wall shear brakes the spin
    (torque against the rotation), the net force nearly cancels."""
    case, body, run = particle_run(u0=(0.0, 0.0), omega0=2.0)
    run.step_coupled()
    F, M = coupling.wall_force_torque(run, body.block, body.point())
    assert M < 0.0
    assert np.hypot(*F) < 1e-2 * abs(M) / 0.1
    run.step_coupled()
    assert 0.0 < body.w < 2.0 and body.a > 0.0


def test_node_placement_matches_prescribed_motion():
    """The coupled run places nodes with the same affine formula as a
    prescribed motion: identical coordinates for the same maps."""
    case = wl.mems(nbi=16, nbj=8, noi=16, noj=6)
    t = 0.37 / case.meta["freq"]
    got = coupling.nodes(case, case.motion(t))
    for a, b in zip(got, case.nodes_at(t)):
        assert np.array_equal(a, b)
