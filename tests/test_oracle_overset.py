"""Pins of the oracle's overset assembly and interpolation (Sec. 3.1, 3.2),
CPU only: predicates against independent formulations, brute-force donor
search, and the invariants an assembly must satisfy."""
import math

import numpy as np
import pytest

from oracle import mesh, overset
from oracle.run import Run
from oracle.ugks import FIELD, HOLE, RECEPTOR
from paper_2604_09984_gb300 import workloads as wl


def small_mems(**kw):
    args = dict(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15)
    args.update(kw)
    return wl.mems(**args)


def tri_area(a, b, c):
    return 0.5 * abs((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))


def test_inside_quads_matches_area_decomposition():
    rng = np.random.default_rng(0)
    for _ in range(30):
        base = rng.uniform(-1, 1, 2)
        # convex counter-clockwise quad: perturbed square
        q = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float) * rng.uniform(0.5, 2) + base
        q += rng.uniform(-0.15, 0.15, q.shape)
        pts = base + rng.uniform(-0.5, 2.5, (200, 2))
        got = overset.inside_quads(pts, q[None])[:, 0]
        area = tri_area(q[0], q[1], q[2]) + tri_area(q[0], q[2], q[3])
        for p, g in zip(pts, got):
            s = sum(tri_area(p, q[e], q[(e + 1) % 4]) for e in range(4))
            if abs(s - area) < 1e-9 * area and min(
                    tri_area(p, q[e], q[(e + 1) % 4]) for e in range(4)) < 1e-9:
                continue          # on an edge: inclusive test may go either way here
            assert g == (abs(s - area) < 1e-12 * max(1.0, area))


def test_inside_polygon_matches_winding_number():
    c = wl.ellipse_contour((0.2, -0.1), 0.5, 0.2)
    poly = np.array([c(-2 * math.pi * i / 40) for i in range(40)])
    rng = np.random.default_rng(1)
    pts = rng.uniform(-0.6, 0.8, (400, 2))
    got = overset.inside_polygon(pts, poly)
    for p, g in zip(pts, got):
        ang = 0.0
        for i in range(40):
            a = poly[i] - p
            b = poly[(i + 1) % 40] - p
            ang += math.atan2(a[0] * b[1] - a[1] * b[0], a[0] * b[0] + a[1] * b[1])
        assert g == (abs(ang) > math.pi)


def test_wall_distance_matches_projection_formula():
    rng = np.random.default_rng(2)
    segs = rng.uniform(-1, 1, (15, 2, 2))
    pts = rng.uniform(-1.5, 1.5, (300, 2))
    got = overset.wall_dist2(pts, segs)
    for p, g in zip(pts, got):
        best = np.inf
        for a, b in segs:
            d = b - a
            L = math.hypot(*d)
            u = d / L
            s = (p - a) @ u
            if s <= 0:
                dist = math.hypot(*(p - a))
            elif s >= L:
                dist = math.hypot(*(p - b))
            else:
                dist = abs((p - a)[0] * u[1] - (p - a)[1] * u[0])
            best = min(best, dist)
        assert g == pytest.approx(best * best, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("frac", [0.0, 0.25, 0.6])
def test_assembly_invariants(frac):
    case = small_mems()
    topo = mesh.Topology(case.blocks)
    t = frac / case.meta["freq"]
    X = case.nodes_at(t)
    conn = overset.connect(topo, X)
    st = conn.status
    # field cells touch only field or receptor cells
    for c in np.nonzero(st == FIELD)[0]:
        for d in range(4):
            if topo.nb_kind[c, d] == mesh.NB_CELL:
                assert st[topo.nb_id[c, d]] != HOLE
    assert conn.n_orphan == 0
    np.testing.assert_allclose(conn.weights.sum(1), 1.0, rtol=0, atol=1e-15)
    assert (conn.weights >= 0).all()
    Xn = topo.concat_nodes(X)
    xc = 0.25 * ((Xn[topo.cell_nodes[:, 0]] + Xn[topo.cell_nodes[:, 1]])
                 + (Xn[topo.cell_nodes[:, 2]] + Xn[topo.cell_nodes[:, 3]]))
    for r, c in enumerate(conn.receptors):
        dn = conn.donors[r]
        dn = dn[dn >= 0]
        assert dn.size >= 1
        assert (st[dn] != HOLE).all()
        assert (topo.cell_block[dn] != topo.cell_block[c]).all()
        q = Xn[topo.cell_nodes[dn[0]]]
        assert overset.inside_quads(xc[c][None], q[None])[0, 0]
    # both zones keep field cells; the background gets a hole around the plate
    assert (st[:topo.cell_off[1]] == HOLE).any()
    assert (st[topo.cell_off[1]:] == FIELD).any()


def test_donor_search_brute_force():
    """The donor of every receptor equals a plain loop over all cells in the
    stated order (FIELD before RECEPTOR, priority, block, index)."""
    case = small_mems(nbi=32, nbj=16, noi=24, noj=10)
    topo = mesh.Topology(case.blocks)
    X = case.nodes_at(0.3)
    conn = overset.connect(topo, X)
    Xn = topo.concat_nodes(X)
    xc = 0.25 * ((Xn[topo.cell_nodes[:, 0]] + Xn[topo.cell_nodes[:, 1]])
                 + (Xn[topo.cell_nodes[:, 2]] + Xn[topo.cell_nodes[:, 3]]))
    order = sorted(range(len(case.blocks)), key=lambda b: (-case.blocks[b].priority, b))
    for r, c in enumerate(conn.receptors):
        found = -1
        for cls in (FIELD, RECEPTOR):
            for b in order:
                if b == topo.cell_block[c] or found >= 0:
                    continue
                for cell in range(topo.cell_off[b], topo.cell_off[b + 1]):
                    if conn.status[cell] != cls:
                        continue
                    quad = Xn[topo.cell_nodes[cell]]
                    ok = True
                    for e in range(4):
                        a, bb = quad[e], quad[(e + 1) % 4]
                        cr = (bb[0] - a[0]) * (xc[c, 1] - a[1]) - (bb[1] - a[1]) * (xc[c, 0] - a[0])
                        ok &= cr >= 0.0
                    if ok:
                        found = cell
                        break
            if found >= 0:
                break
        assert found == conn.donors[r, 0]


def test_idw_reproduces_constants_and_is_convex():
    case = small_mems()
    run = Run(case)
    conn = run.conn
    st = run.state
    st.f[:] = 0.37
    st.W[:] = 1.25
    st.q[:] = -0.5
    overset.interpolate(st, conn.receptors, conn.donors, conn.weights)
    np.testing.assert_allclose(st.f[conn.receptors], 0.37, rtol=1e-15)
    np.testing.assert_allclose(st.W[conn.receptors], 1.25, rtol=1e-15)
    # a linear field is reproduced to first order (weights sum to one)
    topo = run.topo
    Xn = topo.concat_nodes(case.nodes_at(0.0))
    xc = 0.25 * ((Xn[topo.cell_nodes[:, 0]] + Xn[topo.cell_nodes[:, 1]])
                 + (Xn[topo.cell_nodes[:, 2]] + Xn[topo.cell_nodes[:, 3]]))
    lin = 2.0 + xc[:, 0] - 0.5 * xc[:, 1]
    st.W[:, 0] = lin
    overset.interpolate(st, conn.receptors, conn.donors, conn.weights)
    err = np.abs(st.W[conn.receptors, 0] - lin[conn.receptors]).max()
    assert err < 0.05


def test_overset_run_finite():
    case = small_mems(n_inner=2)
    run = Run(case)
    for _ in range(2):
        run.step()
    f = run.state.f[run.status == FIELD]
    assert np.isfinite(f).all()
    W = run.state.W[run.status == FIELD]
    assert (W[:, 0] > 0).all()


def test_idw_weights_follow_inverse_square_law():
    """Sec. 3.2: the weight of stencil cell j of a receptor is
    d_j^-2 / sum_l d_l^-2, d the Euclidean distance between the receptor's
    and the stencil cell's centres at t^{n+1} (vertex centres, computed here
    with hypot).  A d^-1 law, or equal weights, fail on most rows."""
    case = small_mems()
    run = Run(case)
    conn = run.conn
    topo = run.topo
    Xn = topo.concat_nodes(case.nodes_at(0.0))
    xc = Xn[topo.cell_nodes].mean(axis=1)
    n_multi = 0
    n_discriminating = 0
    for r, cell in enumerate(conn.receptors):
        row = conn.donors[r]
        valid = row >= 0
        assert valid[0]
        d = np.hypot(xc[row[valid], 0] - xc[cell, 0], xc[row[valid], 1] - xc[cell, 1])
        want = d ** -2 / (d ** -2).sum()
        np.testing.assert_allclose(conn.weights[r, valid], want, rtol=1e-12, atol=0)
        assert np.all(conn.weights[r, ~valid] == 0.0)
        if valid.sum() > 1:
            n_multi += 1
            inv1 = d ** -1 / (d ** -1).sum()
            if np.abs(inv1 - want).max() > 1e-3:
                n_discriminating += 1
    assert n_multi > 0.9 * conn.receptors.size
    assert n_discriminating > 0.5 * n_multi


def test_idw_exact_on_constructed_stencil():
    """Sec. 3.2 on a hand-placed receptor: a Cartesian donor grid of spacing
    h, receptor point at (x_d + 0.3 h, y_d - 0.1 h) of donor cell d; the five
    stencil distances are sqrt(0.3^2+0.1^2) h, and those to the four face
    neighbours, and the weights are their inverse squares normalised."""
    h = 0.1
    ni, nj = 6, 5
    X = wl.cartesian_nodes(ni, nj, 0.0, ni * h, 0.0, nj * h)
    bg = wl.BlockSpec(ni, nj, False, (wl.BC_WALL,) * 4, (1.0,) * 4, X)
    # a one-cell component grid whose only cell is a receptor placed by hand
    ci, cj = 2, 2
    xd = np.array([(ci + 0.5) * h, (cj + 0.5) * h])
    p = xd + np.array([0.3 * h, -0.1 * h])
    s = 0.02
    Y = wl.cartesian_nodes(1, 1, p[0] - s, p[0] + s, p[1] - s, p[1] + s)
    comp = wl.BlockSpec(1, 1, False, (wl.BC_OVERSET,) * 4, (0.0,) * 4, Y, priority=1, n_fringe=1)
    topo = mesh.Topology([bg, comp])
    Xn = topo.concat_nodes([X, Y])
    xc_new = Xn[topo.cell_nodes].mean(axis=1)
    status = np.zeros(topo.nc, dtype=np.int64)
    cells = np.array([topo.cell_off[1]])
    donors, weights, orphan = overset._donors(topo, Xn, xc_new, status, cells)
    assert orphan == 0
    d0 = cj * ni + ci
    assert list(donors[0]) == [d0, d0 - 1, d0 + 1, d0 - ni, d0 + ni]
    off = [(0.3, -0.1), (1.3, -0.1), (-0.7, -0.1), (0.3, 0.9), (0.3, -1.1)]
    inv = np.array([1.0 / ((a * a + b * b) * h * h) for a, b in off])
    np.testing.assert_allclose(weights[0], inv / inv.sum(), rtol=1e-13)
