"""Failure detection on the GPU without a GPU fault: a singular leaf reported
by plan creation, the projector's and the leaf solves' bounded waits running
out, and a Krylov breakdown.

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
  in flight when the kernel ends.
* The tensor-core leaf solves wait, with a bound, for the products one of
  their threads issues. The test hook WMG_TEST_STALL_TENSOR_PRODUCTS=1 makes
  that thread issue none, so the waits run out after a short limit; every
  CTA frees its tensor memory and returns, the solve returns
  WMG_ERR_TIMEOUT, and the next solve on the same plan is correct.
* A Krylov breakdown from host data alone: WMG-BiCGStab in an FP32 plan run
  past convergence until its search vectors underflow the FP32 copies; the
  problem ends with WMG_ERR_BREAKDOWN and its last (converged) iterate."""
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


def test_tensor_product_wait_runs_out_and_the_plan_stays_usable(monkeypatch):
    P = S.workload_small().problems[0]
    op = oracle.Op(P.n, P.m, P.D)
    bs = torch.tensor(np.tile(op.project(P.image()), 3), dtype=torch.float32, device="cuda")
    plan = wmg.Plan(P.n, P.m, P.D, levels=P.levels, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID,
                    precision=wmg.PREC_F32)
    x_ok, info_ok, _, _ = plan.solve(bs, wmg.SOLVER_GMRES, True, max_iter=4, rtol=0.0)
    x_ok = x_ok.cpu().numpy()
    monkeypatch.setenv("WMG_TEST_STALL_TENSOR_PRODUCTS", "1")
    with pytest.raises(wmg.WmgError) as e:
        plan.solve(bs, wmg.SOLVER_GMRES, True, max_iter=4, rtol=0.0)
    assert e.value.code == wmg.WMG_ERR_TIMEOUT
    monkeypatch.delenv("WMG_TEST_STALL_TENSOR_PRODUCTS")
    x, info, _, _ = plan.solve(bs, wmg.SOLVER_GMRES, True, max_iter=4, rtol=0.0)
    assert info == info_ok
    assert np.array_equal(x.cpu().numpy(), x_ok)
    plan.close()


def test_krylov_breakdown_ends_the_problem_with_its_last_iterate():
    # Run past convergence (rtol 0), the recursive residual of WMG-BiCGStab
    # shrinks geometrically; in an FP32 plan the operator's FP32 copies of
    # the search vectors underflow (below 1e-45) before the FP64 residual is
    # exactly zero, so <r^, v> is exactly 0: a breakdown. Geometry and data
    # of the semi-convergence study (160^2, 400 angles x 160 bins, Joseph's
    # kernel, 1 % uniform noise), lambda = 0.1 m / n.
    n, m, D, levels = 160, 400, 160, 5
    x = S.phantom(n, 12, S.seed_for(6, 0))
    xd = torch.tensor(x.reshape(-1), dtype=torch.float32, device="cuda")
    p64 = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F64,
                   kernel=wmg.KERNEL_JOSEPH)
    b = p64.project(xd.double())
    b = b + 0.01 * b.abs().max() * torch.tensor(S.uniform_noise_draws(m * D, S.seed_for(6, 0)),
                                                dtype=torch.float64, device="cuda")
    p64.close()
    lam = 0.1 * m / n
    plans = {prec: wmg.Plan(n, m, D, levels=levels, nu1=0, nu2=0, lam=lam, hybrid_depth=levels - 1,
                            cycle=wmg.CYCLE_HYBRID, precision=prec, kernel=wmg.KERNEL_JOSEPH)
             for prec in (wmg.PREC_F32, wmg.PREC_F64)}
    b32 = b.float().contiguous()
    pl = plans[wmg.PREC_F32]
    with pytest.raises(wmg.WmgError) as e:
        pl.solve(b32, wmg.SOLVER_BICGSTAB, True, 100, 0.0)
    assert e.value.code == wmg.WMG_ERR_BREAKDOWN
    x, info, _, rc = pl.solve(b32, wmg.SOLVER_BICGSTAB, True, 100, 0.0, problem_errors=False)
    assert rc == wmg.WMG_ERR_BREAKDOWN and info[0][1] == wmg.WMG_ERR_BREAKDOWN and info[0][0] < 100
    # the last iterate is the converged regularised solution (FP32 operator)
    x64, info64, _, _ = plans[wmg.PREC_F64].solve(b32.double(), wmg.SOLVER_BICGSTAB, True, 200, 1e-12)
    assert info64[0][1] == 0
    x, x64 = x.double(), x64
    assert float((x - x64).norm() / x64.norm()) < 1e-5
    # a broken-down solve stays a continuation point: the semi-convergence
    # curve runs on through it (Section 4.2), every k past the breakdown
    # reporting the iterate and iteration count the breakdown left
    k_bd = info[0][0]
    state = pl.state_export()
    assert len(state) > 0
    from paper_1310_0956_gb300 import study
    curve = study.error_curve(pl, b32, xd, wmg.SOLVER_BICGSTAB, True, [4, k_bd + 1, 100])
    assert curve[0][1] == 4 and curve[1][1] == k_bd and curve[2][1] == k_bd
    assert curve[1][2] == curve[2][2]
    # and the plan goes on solving
    _, info, _, rc = pl.solve(b32, wmg.SOLVER_BICGSTAB, True, 100, 1e-4)
    assert rc == 0 and info[0][1] == 0
    for p in plans.values():
        p.close()
