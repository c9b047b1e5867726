"""Host logic of the run metrics (paper_1310_0956_gb300/metrics.py): the
solve record's arithmetic on a hand-worked profile, percentiles against
numpy's, the serving record, and the JSON-lines log."""
import json

import numpy as np
import pytest

pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402
from paper_1310_0956_gb300 import metrics  # noqa: E402


def test_solve_record_arithmetic():
    # 2 problems of a 4 x 4 image, 3 angles x 5 bins (N = 16, M = 15), FP32;
    # 10 projected and 12 backprojected images in 4 + 2 ms, 20 nonzeros each
    prof = {"project_launches": 5, "project_ms": 4.0, "project_images": 10.0, "backproject_launches": 6,
            "backproject_ms": 2.0, "backproject_images": 12.0, "nnz_per_image": 20.0}
    infos = [(5, 0, 1e-5), (5, 1, 2e-3)]
    rec = metrics.solve_metrics(4, 3, 5, wmg.PREC_F32, wmg.SOLVER_GMRES, True, infos, [[1.0, 0.5], [1.0]],
                                prof, 0.01, 0.5)
    assert rec["a_pairs_per_problem"] == 5.0
    assert rec["intersections_per_s"] == pytest.approx(20 * 22 / 0.006)
    # projector (2 N + M) = 47, backprojector (M + N) = 31 elements of 4 bytes per image
    assert rec["operator_gb_per_s"] == pytest.approx((10 * 47 + 12 * 31) * 4 / 0.006 / 1e9)
    assert rec["status"] == ["OK", "NOT_CONVERGED"] and rec["iterations"] == [5, 5]
    assert rec["solver"] == "GMRES" and rec["precision"] == "f32" and rec["problems"] == 2
    assert rec["residual_history"] == [[1.0, 0.5], [1.0]]
    json.dumps(rec)                                      # serialisable as it stands
    # 4 more images projected on the 2h grid in 1 ms: A-pairs count them, the
    # intersections and bytes of W's grid do not change
    rec2 = metrics.solve_metrics(4, 3, 5, wmg.PREC_F32, wmg.SOLVER_GMRES, True, infos, None,
                                 dict(prof, project_2h_launches=2, project_2h_ms=1.0, project_2h_images=4.0),
                                 0.01)
    assert rec2["a_pairs_per_problem"] == 7.0
    assert rec2["intersections_per_s"] == rec["intersections_per_s"]
    assert rec2["project_2h"] == {"launches": 2, "ms": 1.0, "images": 4.0}


def test_percentiles_match_numpy():
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 100):
        v = rng.random(n) * 100
        for q in (0, 50, 90, 99, 100):
            assert metrics.percentile(v, q) == pytest.approx(np.percentile(v, q))
    assert metrics.percentile([], 50) is None


def test_serving_record_and_log(tmp_path):
    counters = {"queued": 3, "running": 5, "completed": 40}
    rec = metrics.serving_metrics(counters, [10.0, 20.0, 30.0, 40.0], 2.0)
    assert rec["recon_per_s"] == 2.0 and rec["p50_ms"] == 25.0 and rec["queue_depth"] == 3
    log = metrics.JsonlLog(str(tmp_path / "run.jsonl"))
    log.write(rec)
    log.write({"event": "solve", "solve_s": 0.1})
    lines = (tmp_path / "run.jsonl").read_text().splitlines()
    assert [json.loads(x)["event"] for x in lines] == ["serve", "solve"]


class _Event:
    t = 0.0

    def __init__(self, enable_timing=False):
        self.at = None

    def record(self, stream=None):
        _Event.t += 0.25
        self.at = _Event.t

    def elapsed_time(self, other):
        return (other.at - self.at) * 1000.0


class _Stats:
    project_launches, project_ms, project_images = 3, 1.0, 6.0
    backproject_launches, backproject_ms, backproject_images = 3, 1.0, 6.0
    nnz_per_image = 10.0
    project_2h_launches, project_2h_ms, project_2h_images = 0, 0.0, 0.0


class _StandInPlan:
    n, m, D = 4, 3, 5
    opts = wmg.wmg_opts(1, 0, 0, 1.0, 0.0, 0, wmg.CYCLE_ADDITIVE, wmg.PREC_F64)
    handle = "plan"
    setup_s = 0.125

    def __init__(self, torch_ns, fail=False):
        self._torch = torch_ns
        self.fail = fail

    def _stream(self):
        return None

    def solve(self, b, solver, pre, max_iter, rtol, restart, history=False, x0=None):
        if self.fail:
            raise wmg.WmgError(wmg.WMG_ERR_NAN, "stand-in failure")
        return "x", [(2, 0, 1e-6)], None, 0


def _patched(monkeypatch, calls):
    import types
    torch_ns = types.SimpleNamespace(cuda=types.SimpleNamespace(
        Event=_Event, current_stream=lambda: None, synchronize=lambda: None))
    monkeypatch.setattr(metrics, "wmg_profile_begin", lambda h: calls.append(("begin", h)))
    monkeypatch.setattr(metrics, "wmg_profile_end", lambda h, s: calls.append(("end", h)) or _Stats())
    return torch_ns


def test_profiled_solve_plumbing(monkeypatch, tmp_path):
    calls = []
    plan = _StandInPlan(_patched(monkeypatch, calls))
    log = metrics.JsonlLog(str(tmp_path / "s.jsonl"))
    x, infos, hists, rc, rec = metrics.profiled_solve(plan, "b", wmg.SOLVER_CGLS, False, 2, 0.0, log=log)
    assert calls == [("begin", "plan"), ("end", "plan")]
    assert (x, rc, rec["iterations"], rec["setup_s"]) == ("x", 0, [2], 0.125)
    assert rec["solve_s"] == pytest.approx(0.25) and rec["a_pairs_per_problem"] == 6.0
    assert json.loads((tmp_path / "s.jsonl").read_text())["solver"] == "CGLS"


def test_profiled_solve_ends_profiling_when_the_solve_fails(monkeypatch):
    calls = []
    plan = _StandInPlan(_patched(monkeypatch, calls), fail=True)
    with pytest.raises(wmg.WmgError):
        metrics.profiled_solve(plan, "b", wmg.SOLVER_GMRES)
    assert calls == [("begin", "plan"), ("end", "plan")]
