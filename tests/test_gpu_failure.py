"""Failure detection on the GPU without a GPU fault: a singular leaf reported
by plan creation, and the projector's bounded waits running out.

* One angle and a 4-bin detector leave the leaf Galerkin blocks off the
  detector's band with exactly zero rows (the oracle pins this case), so
  the leaf Cholesky meets a zero pivot and plan creation reports
  WMG_ERR_LEAF_NOT_SPD; with lambda > 0 (eq. sys_reg) every leaf is SPD and
  the plan's leaf inverses invert the oracle's leaf matrices.
* The staged-pixel projector waits, with a bound, for copies its producer
  warp issues. The test hook WMG_TEST_STALL_STAGED_COPIES=1 makes the
  producer issue none, so every wait runs out after a short limit; the
  kernel aborts its CTA and raises the library's error flag, the solve
  returns WMG_ERR_TIMEOUT, and the next solve on the same plan is correct:
  the context stays usable. No wait in that path is unbounded and no copy is
  in flight when the kernel ends."""
import os

import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [wmg.PREC_F64, wmg.PREC_F32])
def test_leaf_not_spd_is_reported_by_plan_creation(precision):
    with pytest.raises(wmg.WmgError) as e:
        wmg.Plan(16, 1, 4, levels=2, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=precision)
    assert e.value.code == wmg.WMG_ERR_LEAF_NOT_SPD
    # the same geometry regularised: every leaf SPD, inverses of the oracle's leaves
    plan = wmg.Plan(16, 1, 4, levels=2, nu1=0, nu2=0, lam=0.1, cycle=wmg.CYCLE_ADDITIVE, precision=precision)
    ref = oracle.Wmg(oracle.Op(16, 1, 4), 2, lam=0.1, factor=False)
    for k in range(plan.K):
        inv = plan.leaf_inverse(k).double().cpu().numpy().reshape(plan.P, plan.P)
        err = np.abs(inv @ ref.leaf(k) - np.eye(plan.P)).max()
        assert err < (1e-10 if precision == wmg.PREC_F64 else 1e-5), (k, err)
    plan.close()


def test_staged_copy_wait_runs_out_and_the_plan_stays_usable(monkeypatch):
    P = S.workload_small().problems[0]
    op = oracle.Op(P.n, P.m, P.D)
    b = op.project(P.image())
    count = 8                                       # one group tile: the staged-pixel kernel runs
    bs = torch.tensor(np.tile(b, count), dtype=torch.float32, device="cuda")
    plan = wmg.Plan(P.n, P.m, P.D, levels=P.levels, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID,
                    precision=wmg.PREC_F32)
    x_ok, info_ok, _, _ = plan.solve(bs, wmg.SOLVER_GMRES, True, max_iter=4, rtol=0.0)
    x_ok = x_ok.cpu().numpy()
    monkeypatch.setenv("WMG_TEST_STALL_STAGED_COPIES", "1")
    with pytest.raises(wmg.WmgError) as e:
        plan.solve(bs, wmg.SOLVER_GMRES, True, max_iter=4, rtol=0.0)
    assert e.value.code == wmg.WMG_ERR_TIMEOUT
    monkeypatch.delenv("WMG_TEST_STALL_STAGED_COPIES")
    x, info, _, _ = plan.solve(bs, wmg.SOLVER_GMRES, True, max_iter=4, rtol=0.0)
    assert info == info_ok
    assert np.array_equal(x.cpu().numpy(), x_ok)
    plan.close()
    assert os.environ.get("WMG_TEST_STALL_STAGED_COPIES") is None
