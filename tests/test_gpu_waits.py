"""Bounded device-side waits (GPU): with the poll limit of the sweeps cut to a
single poll, the waits of the macro LU-SGS (bulk copies of the next
diagonal's records) and of the micro-sweep bands (the band before them) run
out; the step reports UGKS_ERR_TIMEOUT at the next synchronising call, no CTA
is left waiting, and the context stays usable: with the default limit back
and the earlier state restored, the next step equals that of a context that
never timed out.  No wait is made to hang: every wait is bounded and the
one that runs out here simply gives up after its single poll."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

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


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_wait_limit_times_out_and_context_recovers(prec):
    # background 48x24: three 8-row bands per micro-sweep CTA, so bands wait
    # on bands; two blocks: the FP32 macro sweep fetches records by bulk copy
    case = wl.mems(nbi=48, nbj=24, noi=32, noj=12, nv=8, stretch=1.15, n_inner=2)
    s = U.Solver(case, prec)
    c = U.Solver(case, prec)
    for x in (s, c):
        x.advance()
    f0, W0, q0 = s.get_state()
    s.set_wait_limit(1)
    s.advance()
    with pytest.raises(U.UgksError) as err:
        s.moments()
    assert err.value.code == -8          # UGKS_ERR_TIMEOUT
    s.set_wait_limit(0)
    s.moments()                           # the flag was cleared
    c.advance()                           # the same physical step, no timeout
    s.set_state(f0, W0, q0)
    c.set_state(f0, W0, q0)
    s.advance()
    c.advance()
    Ws, qs, sts, walls = s.moments()
    Wc, qc, stc, wallc = c.moments()
    assert np.array_equal(sts, stc)
    assert np.isfinite(Ws).all()
    assert np.array_equal(Ws, Wc) and np.array_equal(qs, qc) and np.array_equal(walls, wallc)
    with pytest.raises(U.UgksError):
        s.set_wait_limit(-1)
