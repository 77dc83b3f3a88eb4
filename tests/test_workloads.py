"""Host checks of the seeded synthetic workloads: meshes are valid (every
cell right-handed, O-grid contours aligned with their outer circle), the
batched sweep spans the stated ranges deterministically, and the overlap
rule leaves enough non-cutting rings for coarse backgrounds."""
import math

import numpy as np
import pytest

from paper_2604_09984_gb300 import workloads as wl


def signed_areas(X):
    a, b, c, d = X[:-1, :-1], X[1:, :-1], X[1:, 1:], X[:-1, 1:]

    def cr(p, q):
        return p[..., 0] * q[..., 1] - p[..., 1] * q[..., 0]
    return 0.5 * (cr(a, b) + cr(b, c) + cr(c, d) + cr(d, a))


@pytest.mark.parametrize("sizes", [(512, 256, 192, 48), (80, 40, 24, 10), (160, 80, 96, 24)])
def test_two_body_cells_right_handed(sizes):
    nbi, nbj, noi, noj = sizes
    case = wl.tsto(nbi=nbi, nbj=nbj, noi=noi, noj=noj, nv=8)
    for b in case.blocks:
        assert (signed_areas(b.x_ref) > 0).all()
    assert case.dt > 0 and case.dt == pytest.approx(
        10.0 * wl.smallest_cell_width(case.blocks) / 30.0)
    # gas at rest; the stream enters through the far field
    assert np.all(case.init_prim[:, 1:3] == 0.0) and case.farfield[1] > 9.0


def test_polygon_contour_starts_at_angle_zero_and_turns_clockwise():
    verts = [(-0.2, 0.0), (0.1, 0.05), (0.1, -0.05)]
    c = wl.polygon_contour((0.5, 0.5), verts)
    x0, y0 = c(0.0)
    assert y0 == pytest.approx(0.5) and x0 == pytest.approx(0.6)
    ths = -2.0 * math.pi * np.arange(64) / 64
    ang = np.unwrap([math.atan2(c(t)[1] - 0.5, c(t)[0] - 0.5) for t in ths])
    assert np.all(np.diff(ang) < 0)          # clockwise, like the outer circle


def test_smallest_cell_width_of_squares():
    b = wl.BlockSpec(8, 4, False, (1,) * 4, (1.0,) * 4, wl.cartesian_nodes(8, 4, 0.0, 2.0, 0.0, 1.0))
    assert wl.smallest_cell_width([b]) == pytest.approx(0.25)


def test_mems_batch_ranges_and_determinism():
    a = wl.mems_batch(n=64, seed=0)
    b = wl.mems_batch(n=64, seed=0)
    assert [c.ncells for c in a] == [c.ncells for c in b]
    assert [c.meta["Kn"] for c in a] == [c.meta["Kn"] for c in b]
    for c in a:
        bg, og = c.blocks
        assert 48 <= bg.ni <= 192 and bg.ni % 8 == 0 and bg.nj == bg.ni // 2
        assert 64 <= og.ni <= 128 and og.ni % 8 == 0 and og.nj == og.ni // 4
        assert 20 <= c.nvx <= 40 and c.nvx == c.nvy
        assert 0.01 <= c.meta["Kn"] <= 2.0 and 1.0 <= c.meta["Tw"] <= 2.0
        assert og.n_gap >= 2 and og.n_fringe + og.n_gap < og.nj
    assert len({c.nv for c in a}) > 5 and len({c.ncells for c in a}) > 20
    total = sum(c.ncells * c.nv for c in a)
    assert 4e8 < total < 9e8


def test_overlap_rule_gives_three_background_cells():
    for nbi in (48, 96, 192):
        for noj in (16, 24, 32):
            g = wl.overlap_gap_layers(nbi, noj, 1.1, 0.25, 0.1)
            k = noj - 2 - g
            frac = (1.1 ** k - 1.0) / (1.1 ** noj - 1.0)
            assert (1.0 - frac) * 0.15 >= 3.0 * 2.0 / nbi or g == noj - 3
            if g > 2:    # one fewer gap layer would not do
                k1 = k + 1
                frac1 = (1.1 ** k1 - 1.0) / (1.1 ** noj - 1.0)
                assert (1.0 - frac1) * 0.15 < 3.0 * 2.0 / nbi
