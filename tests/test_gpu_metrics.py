"""Step metrics (GPU): the squared norms of the macro residual R (Step 4),
the micro residual r (Step 5) and the Step-7 moment fix of the last inner
iteration, and the field totals of Omega^{n+1} W, computed by the reduction
kernels behind ugks_get_metrics, agree with the oracle's on a deforming
channel and an overset MEMS case.  Each norm is compared with a bound on its
error from the path's own error on the terms it sums: the FP64 path agrees
with the oracle to ~1e-11 of f, W and the fluxes, the FP32 path to ~2e-5 of
f and the fluxes and 1e-5 of W, so |Delta |X|| <= tol * S_X with S_X the norm
of the largest term of X (Omega W / dt for R, Omega f / dt for r, W for the
fix), tol 1e-9 / 1e-4 for the residuals and 1e-9 / 5e-5 for the fix (FP64 /
FP32); every oracle norm is more than twice its bound, so a missing or zero
value fails.  Recording metrics changes no result, and the JSON-lines log
writes one line per step."""
import io
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import ugks as ou  # noqa: E402
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


def make_case(which):
    if which == "channel":
        return wl.channel(ni=12, nj=7, nv=10, n_inner=3, n_steps=3), 5
    return wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=2), 9


@pytest.mark.parametrize("prec,tol,tol_w", [(U.FP64, 1e-9, 1e-9), (U.FP32, 1e-4, 5e-5)])
@pytest.mark.parametrize("which", ["channel", "mems"])
def test_metrics_match_oracle(which, prec, tol, tol_w):
    case, seed = make_case(which)
    prim = wl.random_prim(case, seed, amp_rho=0.1, amp_u=0.1, amp_T=0.1)
    s = U.Solver(case, prec, prim=prim)
    s.set_metrics(True)
    r = Run(case, prim)
    for _ in range(2):
        s.advance()
        r.step()
    g = s.metrics()
    o = ou.step_metrics(r.geo, r.state, r.info, r.status)
    field = r.status == 0
    vol = r.geo.vol_new[field]
    SR = np.sqrt(((vol[:, None] / case.dt * r.state.W[field]) ** 2).sum())
    Sr = np.sqrt(((vol[:, None, None] / case.dt * r.state.f[field]) ** 2).sum())
    SW = np.sqrt((r.state.W[field] ** 2).sum())
    rows = []
    for key, bound in (("res_macro_sq", tol * SR), ("res_micro_sq", tol * Sr), ("fix_sq", tol_w * SW)):
        rows.append((key, np.sqrt(g[key]), np.sqrt(o[key]), bound))
    tot = np.abs(o["total"]).max()
    dtot = np.abs(np.array(g["total"]) - o["total"]).max()
    print("\n", which, prec, ["%s gpu %.6e oracle %.6e diff %.2e bound %.2e" % (k, a, b, abs(a - b), e)
                               for k, a, b, e in rows], "totals diff %.2e of %.3e" % (dtot, tot))
    for key, a, b, bound in rows:
        assert b > 2 * bound, key
        assert abs(a - b) <= bound, (key, a, b, bound)
    assert dtot <= tol_w * tot


def test_metrics_change_no_result_and_log_lines():
    case, seed = make_case("mems")
    prim = wl.random_prim(case, seed, amp_rho=0.1, amp_u=0.1, amp_T=0.1)
    a = U.Solver(case, U.FP32, prim=prim)
    b = U.Solver(case, U.FP32, prim=prim)
    with pytest.raises(U.UgksError):
        a.metrics()                             # no metered step yet
    buf = io.StringIO()
    log = U.StepLog(buf)
    for _ in range(3):
        log.advance(a)
        b.advance()
    for x, y in zip(a.moments(), b.moments()):
        assert np.array_equal(x, y)
    assert torch.equal(a.get_state()[0], b.get_state()[0])
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert [x["step"] for x in lines] == [0, 1, 2]
    assert lines[0]["mass_defect"] is None and all(np.isfinite(x["mass_defect"]) for x in lines[1:])
    for x in lines:
        assert x["res_macro"] > 0 and x["res_micro"] > 0 and x["n_orphan"] == 0 and x["ms"] > 0
    a.set_metrics(False)
    a.advance()
    with pytest.raises(U.UgksError):
        a.metrics()                             # the last step ran without metrics
