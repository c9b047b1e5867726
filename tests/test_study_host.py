"""Host logic of the semi-convergence study (Section 4.2): which iterate
counts continue the previous run (wmg_solve_resume) and which are solved
afresh, and the error measures, with a stand-in plan whose k-th iterate is
known (x_k = k at every pixel)."""
import pytest

torch = pytest.importorskip("torch")
from paper_1310_0956_gb300 import SOLVER_BICGSTAB, SOLVER_GMRES, SOLVER_SIRT, study  # noqa: E402


class StandInPlan:
    def __init__(self):
        self.calls = []

    def _out(self, k):
        return torch.full((4,), float(k)), [(k, 1, 0.0)], None, 1

    def solve(self, b, solver, preconditioned, k, rtol, restart, problem_errors=True):
        assert rtol == 0.0
        self.calls.append(("solve", k))
        return self._out(k)

    def resume(self, b, k, rtol, problem_errors=True):
        assert rtol == 0.0
        self.calls.append(("resume", k))
        return self._out(k)


@pytest.mark.parametrize("solver", [SOLVER_SIRT, SOLVER_BICGSTAB])
def test_one_run_to_the_largest_count(solver):
    p = StandInPlan()
    curve = study.error_curve(p, None, torch.ones(4), solver, True, [1, 2, 5, 10])
    assert p.calls == [("solve", 1), ("resume", 2), ("resume", 5), ("resume", 10)]
    # e_k = (k - 1) at every pixel of x_ex = 1: both relative errors are k - 1
    assert [(k, it, e2, einf) for k, it, e2, einf in curve] == [(1, 1, 0.0, 0.0), (2, 2, 1.0, 1.0),
                                                               (5, 5, 4.0, 4.0), (10, 10, 9.0, 9.0)]


def test_gmres_continues_only_from_a_restart():
    p = StandInPlan()
    study.error_curve(p, None, torch.ones(4), SOLVER_GMRES, True, [1, 4, 6, 8, 12, 13], restart=4)
    assert p.calls == [("solve", 1), ("solve", 4), ("resume", 6), ("solve", 8), ("resume", 12),
                       ("resume", 13)]


def test_decreasing_counts_are_solved_afresh():
    p = StandInPlan()
    study.error_curve(p, None, torch.ones(4), SOLVER_BICGSTAB, False, [5, 3, 3])
    assert p.calls == [("solve", 5), ("solve", 3), ("resume", 3)]


def test_k_opt_and_log_grid():
    curve = [(1, 1, 0.9, 0.9), (2, 2, 0.5, 0.7), (4, 4, 0.6, 0.6)]
    assert study.k_opt(curve) == (2, curve[1])
    ks = study.log_ks(100, 4)
    assert ks[0] == 1 and ks[-1] == 100 and all(a < b for a, b in zip(ks, ks[1:]))
