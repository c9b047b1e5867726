"""Semi-convergence on noisy data (Section 4.2): the error ||x_k - x_ex|| /
||x_ex|| of the k-th iterate of SIRT, BiCGStab and WMG-BiCGStab on the GPU
against the same curve from the FP64 oracle, Joseph's kernel, 1 % uniform
white noise (eq. noise_term), with and without Tikhonov regularisation
(eq. sys_reg)."""
import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402
from paper_1310_0956_gb300 import study  # noqa: E402

pytestmark = pytest.mark.gpu

n, m, D = 32, 60, 32


def problem():
    op = oracle.Op(n, m, D, kernel=oracle.KERNEL_JOSEPH)
    x = S.phantom(n, 6, S.seed_for(13, 0))
    b = op.project(x)
    b = b + 0.01 * np.abs(b).max() * S.uniform_noise_draws(op.M, S.seed_for(13, 0))
    return op, x, b


def oracle_curve(op, x, b, method, ks, lam, M=None):
    out = []
    for k in ks:
        if method == "sirt":
            xk, _ = oracle.sirt(op, b, k, lam)
        else:
            xk = oracle.bicgstab(op, b, k, 0.0, lam, M)[0]
        e = xk - x
        out.append((np.linalg.norm(e) / np.linalg.norm(x), np.abs(e).max() / np.abs(x).max()))
    return out


@pytest.mark.parametrize("lam", [0.0, 2e-4])
def test_curves_match_oracle(lam):
    op, x, b = problem()
    plan = wmg.Plan(n, m, D, levels=3, nu1=0, nu2=0, lam=lam, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID,
                    precision=wmg.PREC_F64, kernel=wmg.KERNEL_JOSEPH)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    M = oracle.Wmg(op, 3, 0, 0, 1.0, lam, oracle.CYCLE_HYBRID, 1)
    # SIRT is a stable stationary iteration; the Krylov iterates carry the
    # rounding differences of two FP64 evaluations, amplified by the
    # iteration (a few 1e-8 after 8 steps; see the BiCGStab parity tests)
    cases = [("sirt", wmg.SOLVER_SIRT, False, [1, 3, 10, 30, 100], None, 1e-10),
             ("bicg", wmg.SOLVER_BICGSTAB, False, [1, 2, 4, 8], None, 1e-6),
             ("wmg", wmg.SOLVER_BICGSTAB, True, [1, 2, 4, 8], M, 1e-6)]
    for name, solver, pre, ks, prec, tol in cases:
        gpu = study.error_curve(plan, bd, xd, solver, pre, ks)
        ref = oracle_curve(op, x, b, name, ks, lam, prec)
        for (k, done, e2, einf), (r2, rinf) in zip(gpu, ref):
            assert done == k, (name, k, done)
            assert abs(e2 - r2) <= tol * r2, (name, k, e2, r2)
            assert abs(einf - rinf) <= tol * rinf, (name, k, einf, rinf)
    plan.close()


def reach(curve, tol=0.02):
    """First iterate count whose L2 error is within tol of the last one's."""
    fin = curve[-1][2]
    return next(k for k, _, e, _ in curve if e <= (1 + tol) * fin)


def test_semiconvergence_and_regularisation():
    # without regularisation the error of plain BiCGStab passes through a
    # minimum and grows again (the noise is fitted); with lambda small against
    # the spectral radius of W^T W (about m/n here) it settles at its minimum
    # instead, and WMG gets there in fewer iterations than the plain solver
    op, x, b = problem()
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    ks = study.log_ks(300)
    p0 = wmg.Plan(n, m, D, levels=3, nu1=0, nu2=0, lam=0.0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID,
                  precision=wmg.PREC_F64, kernel=wmg.KERNEL_JOSEPH)
    plain0 = study.error_curve(p0, bd, xd, wmg.SOLVER_BICGSTAB, False, ks)
    _, best = study.k_opt(plain0)
    assert plain0[-1][2] > 1.2 * best[2]
    p0.close()
    lam = 1e-3 * m / n
    pl = wmg.Plan(n, m, D, levels=3, nu1=0, nu2=0, lam=lam, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID,
                  precision=wmg.PREC_F64, kernel=wmg.KERNEL_JOSEPH)
    plain = study.error_curve(pl, bd, xd, wmg.SOLVER_BICGSTAB, False, ks)
    pre = study.error_curve(pl, bd, xd, wmg.SOLVER_BICGSTAB, True, ks)
    for curve in (plain, pre):
        i = min(range(len(curve)), key=lambda j: curve[j][2])
        assert max(r[2] for r in curve[i:]) <= 1.01 * curve[-1][2]
    assert reach(pre) < reach(plain)
    pl.close()
