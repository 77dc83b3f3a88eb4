"""Host side of the JSON-lines step log: one object per recorded step with
the metrics' norms, the relative change of the field mass between logged
steps (null on the first) and the assembly counters (no GPU: a stand-in
solver supplies the metrics)."""
import io
import json

import pytest

from paper_2604_09984_gb300 import ugks as U


class FakeSolver:
    def __init__(self):
        self.t = 0.0
        self.mass = [2.0, 2.002, 1.999]
        self.k = 0
        self.last_stats = dict(n_field=10, n_receptor=3, n_hole=1, n_fresh=0, n_orphan=0)

    def metrics(self):
        m = self.mass[self.k]
        return {"res_macro": 0.5, "res_micro": 0.25, "fix": 0.125, "total": [m, 0.0, 0.0, 3.0]}


def test_step_log_lines():
    buf = io.StringIO()
    log = U.StepLog(buf)
    s = FakeSolver()
    for k in range(3):
        s.k, s.t = k, 0.1 * (k + 1)
        log.record(s, ms=1.5)
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert len(lines) == 3
    assert [x["step"] for x in lines] == [0, 1, 2]
    assert lines[0]["mass_defect"] is None
    assert lines[1]["mass_defect"] == pytest.approx(0.001, rel=1e-12)
    assert lines[2]["mass_defect"] == pytest.approx((1.999 - 2.002) / 2.002, rel=1e-12)
    assert lines[2]["t"] == pytest.approx(0.3) and lines[2]["ms"] == 1.5
    assert lines[1]["res_micro"] == 0.25 and lines[1]["n_receptor"] == 3


def test_step_log_to_file(tmp_path):
    p = tmp_path / "steps.jsonl"
    log = U.StepLog(str(p))
    log.record(FakeSolver())
    log.close()
    assert json.loads(p.read_text())["fix"] == 0.125
