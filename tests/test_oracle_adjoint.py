"""Pins of the oracle's transposed operators (CPU only): each transpose A^T
returned by ``oracle.adjoint`` satisfies <A x, y> = <x, A^T y> for random x,
y against the forward operator of the oracle, and on a tiny mesh equals the
transpose of the dense matrix assembled column by column from the forward
operator (a transposed coupling, a wrong sweep order or a dropped diagonal
scaling fails these)."""
import numpy as np

from oracle import adjoint, kinetic as kn, mesh, overset, ugks
from oracle.ugks import FIELD, HOLE, RECEPTOR
from paper_2604_09984_gb300 import workloads as wl


def block(ni, nj, periodic):
    return wl.BlockSpec(ni, nj, periodic, (0, 0, wl.BC_WALL, wl.BC_WALL), (0, 0, 1.0, 1.0),
                        wl.cartesian_nodes(ni, nj, 0.0, 2.0, 0.0, 1.0))


def setup_for(blocks, nv=4):
    gas = kn.Gas(0, 2.0 / 3.0, 0.81, 0.05)
    dvs = kn.make_dvs(nv, nv, -3.0, 3.0, -3.0, 3.0)
    topo = mesh.Topology(blocks)
    return ugks.Setup(topo, gas, dvs, kn.conservative(1.0, 0.0, 0.0, 0.5, gas))


def moving_geo(setup, blocks, rng, dt=0.05):
    X0 = [b.x_ref for b in blocks]
    X1 = []
    for b in blocks:
        X = b.x_ref.copy()
        X[..., 1] += 0.02 * np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1])
        X1.append(X)
    return mesh.geometry(setup.topo, X0, X1, dt)


def micro_case(ni, nj, periodic, seed, holes=()):
    rng = np.random.default_rng(seed)
    blocks = [block(ni, nj, periodic)]
    setup = setup_for(blocks)
    geo = moving_geo(setup, blocks, rng)
    wS = ugks.normal_velocity(setup, geo)
    nc, nv = setup.topo.nc, setup.dvs.nv
    status = np.full(nc, FIELD)
    for c in holes:
        status[c] = HOLE
    outsum = np.zeros((nc, nv))
    for d in range(4):
        fid = setup.topo.cell_faces[:, d]
        sgn = setup.topo.cell_face_sign[:, d]
        outsum += np.maximum(sgn[:, None] * wS[fid], 0.0)
    diag = geo.vol_new[:, None] * rng.uniform(5.0, 20.0, (nc, 1)) + 0.5 * outsum
    return setup, wS, diag, status


def field_random(rng, shape, status):
    x = rng.standard_normal(shape)
    x[status != FIELD] = 0.0
    return x


def test_micro_lusgs_transpose_dot_product():
    for ni, nj, per, holes in ((5, 4, False, (7,)), (6, 3, True, (2, 9)), (2, 3, True, ())):
        setup, wS, diag, status = micro_case(ni, nj, per, 3, holes)
        rng = np.random.default_rng(11)
        shape = (setup.topo.nc, setup.dvs.nv, 2)
        x, y = field_random(rng, shape, status), field_random(rng, shape, status)
        Mx = ugks.micro_lusgs(setup, wS, x, diag, status)
        MTy = adjoint.micro_lusgs_transpose(setup, wS, y, diag, status)
        lhs, rhs = (Mx * y).sum(), (x * MTy).sum()
        assert abs(lhs - rhs) <= 1e-12 * (np.abs(Mx * y).sum() + np.abs(x * MTy).sum())
        assert np.all(MTy[status != FIELD] == 0.0)


def test_micro_lusgs_transpose_equals_dense_transpose():
    # a periodic row of two cells: the two cells share two faces
    for ni, nj, per in ((3, 2, False), (2, 2, True)):
        setup, wS, diag, status = micro_case(ni, nj, per, 5)
        nc, nv = setup.topo.nc, setup.dvs.nv
        n = nc * nv * 2
        A = np.zeros((n, n))
        for col in range(n):
            e = np.zeros(n)
            e[col] = 1.0
            A[:, col] = ugks.micro_lusgs(setup, wS, e.reshape(nc, nv, 2), diag, status).ravel()
        y = np.random.default_rng(2).standard_normal(n)
        got = adjoint.micro_lusgs_transpose(setup, wS, y.reshape(nc, nv, 2), diag, status).ravel()
        np.testing.assert_allclose(got, A.T @ y, rtol=1e-12, atol=1e-14 * np.abs(A.T @ y).max())


def test_interpolate_transpose_dot_product_and_dense():
    rng = np.random.default_rng(4)
    nc, nv = 12, 3
    cells = np.array([1, 4, 7, 10])
    donors = np.array([[0, 2, 5, -1, -1], [3, 5, 6, 8, -1], [-1, -1, -1, -1, -1], [9, 11, 1, 4, 0]])
    weights = np.where(donors >= 0, rng.uniform(0.1, 1.0, donors.shape), 0.0)
    weights /= np.maximum(weights.sum(1, keepdims=True), 1e-300)

    def forward(f):
        st = ugks.State(f.copy(), np.zeros((nc, 4)), np.zeros((nc, 2)))
        overset.interpolate(st, cells, donors, weights)
        return st.f

    n = nc * nv * 2
    A = np.zeros((n, n))
    for col in range(n):
        e = np.zeros(n)
        e[col] = 1.0
        A[:, col] = forward(e.reshape(nc, nv, 2)).ravel()
    y = rng.standard_normal((nc, nv, 2))
    got = adjoint.interpolate_transpose(y, cells, donors, weights)
    np.testing.assert_allclose(got.ravel(), A.T @ y.ravel(), rtol=1e-13, atol=1e-15)
    x = rng.standard_normal((nc, nv, 2))
    assert abs((forward(x) * y).sum() - (x * got).sum()) < 1e-12 * np.abs(x * got).sum()
    # the orphan row (third receptor) keeps its value and its cotangent
    assert np.array_equal(got[7], y[7] + sum(weights[r, k] * y[cells[r]] for r in range(4)
                                             for k in range(5) if donors[r, k] == 7))


def test_moments_transpose_dot_product():
    dvs = kn.make_dvs(5, 4, -3.0, 3.0, -2.0, 2.0)
    rng = np.random.default_rng(6)
    f = rng.standard_normal((7, dvs.nv, 2))
    Wbar = rng.standard_normal((7, 4))
    lhs = (kn.moments(f, dvs) * Wbar).sum()
    rhs = (f * adjoint.moments_transpose(Wbar, dvs)).sum()
    assert abs(lhs - rhs) < 1e-12 * (np.abs(f).sum() * np.abs(Wbar).sum())


def macro_case(ni, nj, per, seed, holes=()):
    rng = np.random.default_rng(seed)
    blocks = [block(ni, nj, per)]
    setup = setup_for(blocks)
    geo = moving_geo(setup, blocks, rng)
    nc = setup.topo.nc
    prim = np.empty((nc, 4))
    prim[:, 0] = 1.0 + rng.uniform(-0.2, 0.2, nc)
    prim[:, 1] = rng.uniform(-0.3, 0.3, nc)
    prim[:, 2] = rng.uniform(-0.3, 0.3, nc)
    prim[:, 3] = 1.0 + rng.uniform(-0.2, 0.2, nc)
    W = kn.conservative(prim[:, 0], prim[:, 1], prim[:, 2], 1.0 / (2.0 * prim[:, 3]), setup.gas)
    Gam = ugks.face_gamma(setup, geo, W)
    status = np.full(nc, FIELD)
    for c in holes:
        status[c] = HOLE
    gsum = np.zeros(nc)
    for d in range(4):
        gsum += geo.S[setup.topo.cell_faces[:, d]] * Gam[setup.topo.cell_faces[:, d]]
    diag = geo.vol_new * rng.uniform(2.0, 6.0, nc) + 0.25 * gsum
    # a right-hand side large enough that F_E(W + dW) is far from linear
    R = rng.standard_normal((nc, 4)) * 0.2 * diag[:, None] * np.array([1.0, 0.5, 0.5, 1.5])
    R[status != FIELD] = 0.0
    return setup, geo, W, R, diag, Gam, status


def test_euler_flux_jacobian_matches_central_differences():
    gas = kn.Gas(0, 2.0 / 3.0, 0.81, 0.05)
    rng = np.random.default_rng(8)
    for _ in range(5):
        W = kn.conservative(1.0 + rng.uniform(-0.3, 0.3), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5),
                            1.0 / (2.0 * (1.0 + rng.uniform(-0.3, 0.3))), gas)
        th = rng.uniform(0, 2 * np.pi)
        nx, ny, un = np.cos(th), np.sin(th), rng.uniform(-0.4, 0.4)
        A = adjoint.euler_flux_jacobian(W, nx, ny, un, gas)
        h = 1e-6
        for j in range(4):
            e = np.zeros(4)
            e[j] = h * max(1.0, abs(W[j]))
            fd = (ugks.euler_flux(W + e, nx, ny, un, gas) - ugks.euler_flux(W - e, nx, ny, un, gas)) / (2 * e[j])
            np.testing.assert_allclose(A[:, j], fd, rtol=1e-7, atol=1e-8)


def test_macro_lusgs_tangent_matches_central_differences():
    for ni, nj, per, holes in ((5, 4, False, (6,)), (4, 3, True, ())):
        setup, geo, W, R, diag, Gam, status = macro_case(ni, nj, per, 9, holes)
        rng = np.random.default_rng(1)
        dR = rng.standard_normal(R.shape) * np.abs(R).max()
        dR[status != FIELD] = 0.0
        t = adjoint.macro_lusgs_tangent(setup, geo, W, R, diag, Gam, status, dR)
        h = 1e-5
        fd = (ugks.macro_lusgs(setup, geo, W, R + h * dR, diag, Gam, status)
              - ugks.macro_lusgs(setup, geo, W, R - h * dR, diag, Gam, status)) / (2 * h)
        np.testing.assert_allclose(t, fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max())
        # the map is nonlinear here: the tangent at R differs from the one at 0
        t0 = adjoint.macro_lusgs_tangent(setup, geo, W, 0.0 * R, diag, Gam, status, dR)
        assert np.abs(t - t0).max() > 1e-4 * np.abs(t).max()


def test_macro_lusgs_adjoint_dot_product():
    for ni, nj, per, holes in ((5, 4, False, (6, 13)), (4, 3, True, ()), (2, 3, True, ())):
        setup, geo, W, R, diag, Gam, status = macro_case(ni, nj, per, 10, holes)
        rng = np.random.default_rng(3)
        x, y = rng.standard_normal(R.shape), rng.standard_normal(R.shape)
        x[status != FIELD] = 0.0
        y[status != FIELD] = 0.0
        Tx = adjoint.macro_lusgs_tangent(setup, geo, W, R, diag, Gam, status, x)
        ATy = adjoint.macro_lusgs_adjoint(setup, geo, W, R, diag, Gam, status, y)
        lhs, rhs = (Tx * y).sum(), (x * ATy).sum()
        assert abs(lhs - rhs) <= 1e-12 * (np.abs(Tx * y).sum() + np.abs(x * ATy).sum()), (lhs, rhs)
        assert np.all(ATy[status != FIELD] == 0.0)


def fix_case(seed):
    setup = setup_for([block(4, 3, False)], nv=14)
    rng = np.random.default_rng(seed)
    nc = setup.topo.nc
    prim = np.empty((nc, 4))
    prim[:, 0] = 1.0 + rng.uniform(-0.2, 0.2, nc)
    prim[:, 1] = rng.uniform(-0.3, 0.3, nc)
    prim[:, 2] = rng.uniform(-0.3, 0.3, nc)
    prim[:, 3] = 1.0 + rng.uniform(-0.2, 0.2, nc)
    st = ugks.initial_state(setup, prim)
    f = st.f * (1.0 + rng.uniform(-0.05, 0.05, st.f.shape))
    Wp = st.W * (1.0 + rng.uniform(-0.02, 0.02, st.W.shape))
    return setup, Wp, f


def test_moment_fix_is_the_steps_fix():
    """moment_fix restates Step 7 of the oracle's step: applied to the step's
    predictor W' (= W^{s+1} - fix) and f^{s+1} it returns the step's W."""
    b = block(5, 4, True)
    setup = setup_for([b], nv=12)
    prim = np.empty((setup.topo.nc, 4))
    rng = np.random.default_rng(12)
    prim[:] = (1.0, 0.1, -0.05, 1.0)
    prim[:, 0] *= 1.0 + rng.uniform(-0.1, 0.1, setup.topo.nc)
    st = ugks.initial_state(setup, prim)
    geo = moving_geo(setup, [b], rng)
    st2, info = ugks.implicit_step(setup, geo, st, 0.05, 2)
    Wp = st2.W - info.fix
    np.testing.assert_allclose(adjoint.moment_fix(setup, Wp, st2.f), st2.W, rtol=1e-13, atol=1e-15)


def test_moment_fix_tangent_matches_central_differences():
    setup, Wp, f = fix_case(14)
    rng = np.random.default_rng(15)
    dWp = rng.standard_normal(Wp.shape) * np.abs(Wp).mean(0)
    df = rng.standard_normal(f.shape) * np.abs(f).mean()
    t = adjoint.moment_fix_tangent(setup, Wp, dWp, df)
    h = 1e-6
    fd = (adjoint.moment_fix(setup, Wp + h * dWp, f + h * df)
          - adjoint.moment_fix(setup, Wp - h * dWp, f - h * df)) / (2 * h)
    np.testing.assert_allclose(t, fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max())


def test_moment_fix_adjoint_dot_product():
    setup, Wp, f = fix_case(16)
    rng = np.random.default_rng(17)
    dWp, df = rng.standard_normal(Wp.shape), rng.standard_normal(f.shape)
    Wbar = rng.standard_normal(Wp.shape)
    t = adjoint.moment_fix_tangent(setup, Wp, dWp, df)
    Wpbar, fbar = adjoint.moment_fix_adjoint(setup, Wp, Wbar)
    lhs = (t * Wbar).sum()
    rhs = (dWp * Wpbar).sum() + (df * fbar).sum()
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(t * Wbar).sum() + np.abs(dWp * Wpbar).sum() + np.abs(df * fbar).sum())
