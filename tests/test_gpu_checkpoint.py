"""Initial guesses and checkpoint / resume on the GPU.

Solves from an initial guess x0 (wmg_solve_x0) against the oracle's solvers
from the same x0 (Section 2.3.1 on eq. sys_reg), SIRT's reported relative
residual against the oracle's, and resumed solves (wmg_solve_resume): in
the same plan, or exported to host bytes and imported into a new plan of
the same geometry, the result is bitwise that of one uninterrupted solve
(iterate, iteration counts, status, residual and residual history)."""
import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu

P = S.workload_small().problems[0]


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def prob():
    op = oracle.Op(P.n, P.m, P.D)
    b = op.project(P.image())
    x0 = 0.5 * P.image()
    return op, b, x0


@pytest.mark.parametrize("lam", [0.0, 0.05])
@pytest.mark.parametrize("pre", [False, True])
def test_cgls_from_x0_matches_oracle(prob, lam, pre):
    op, b, x0 = prob
    M = oracle.Wmg(op, 3, 1, 1, 1.0, lam, oracle.CYCLE_ADDITIVE, 0) if pre else None
    x_ref, k, hist_ref = oracle.cgls(op, b, 8, 0.0, lam, M, x0=x0)
    plan = wmg.Plan(P.n, P.m, P.D, levels=3, nu1=1, nu2=1, lam=lam, hybrid_depth=0, cycle=wmg.CYCLE_ADDITIVE)
    x, info, hists, _ = plan.solve(dev(b), wmg.SOLVER_CGLS, pre, 8, 0.0, history=True, x0=dev(x0))
    assert info[0][0] == k == 8
    assert rel(x.cpu().numpy(), x_ref) < 1e-10
    assert np.abs(hists[0] - hist_ref).max() < 1e-9
    plan.close()


@pytest.mark.parametrize("solver", [wmg.SOLVER_GMRES, wmg.SOLVER_BICGSTAB])
def test_krylov_from_x0_matches_oracle(prob, solver):
    op, b, x0 = prob
    lam = 0.05
    M = oracle.Wmg(op, 3, 0, 0, 1.0, lam, oracle.CYCLE_HYBRID, 1)
    iters = 8 if solver == wmg.SOLVER_GMRES else 4
    if solver == wmg.SOLVER_GMRES:
        x_ref, k, hist_ref = oracle.gmres(op, b, iters, 5, 0.0, lam, M, x0=x0)
    else:
        x_ref, k, hist_ref, _ = oracle.bicgstab(op, b, iters, 0.0, lam, M, x0=x0)
    plan = wmg.Plan(P.n, P.m, P.D, levels=3, nu1=0, nu2=0, lam=lam, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID)
    x, info, hists, _ = plan.solve(dev(b), solver, True, iters, 0.0, 5, history=True, x0=dev(x0))
    assert info[0][0] == k == iters
    assert rel(x.cpu().numpy(), x_ref) < 1e-10
    assert np.abs(hists[0] - hist_ref).max() < 1e-9
    plan.close()


def test_sirt_from_x0_and_its_residual(prob):
    op, b, x0 = prob
    lam = 0.05
    plan = wmg.Plan(P.n, P.m, P.D, levels=3, lam=lam)
    # cold: the relative NE residual |W^T (b - W x) - lam x| / |W^T b|
    x, info, _, _ = plan.solve(dev(b), wmg.SOLVER_SIRT, False, 20, 0.0)
    x_ref, _ = oracle.sirt(op, b, 20, lam)
    assert rel(x.cpu().numpy(), x_ref) < 1e-10
    assert abs(info[0][2] - op.ne_residual(b, x_ref, lam)) < 1e-10 * op.ne_residual(b, x_ref, lam)
    # from x0: eq. sirt_it from x0, the residual relative to that of x0
    x, info, _, _ = plan.solve(dev(b), wmg.SOLVER_SIRT, False, 20, 0.0, x0=dev(x0))
    x_ref, _ = oracle.sirt(op, b, 20, lam, x0=x0)
    assert rel(x.cpu().numpy(), x_ref) < 1e-10
    want = op.ne_residual(b, x_ref, lam) / op.ne_residual(b, x0, lam)
    assert abs(info[0][2] - want) < 1e-10 * want
    plan.close()


def test_exact_initial_guess_ends_at_once():
    # b = 0 and x0 = 0 give r0 = 0: the Krylov solvers stop at iteration 0
    # with WMG_OK and write x0 over the (prefilled) output
    plan = wmg.Plan(P.n, P.m, P.D, levels=3, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID)
    b = torch.zeros(plan.M, dtype=torch.float64, device="cuda")
    x0 = torch.zeros(plan.N, dtype=torch.float64, device="cuda")
    for solver in (wmg.SOLVER_GMRES, wmg.SOLVER_BICGSTAB):
        out = torch.full((plan.N,), 7.0, dtype=torch.float64, device="cuda")
        _, info, _, rc = plan.solve(b, solver, True, 10, 1e-6, out=out, x0=x0)
        assert rc == wmg.WMG_OK and info[0][:2] == (0, wmg.WMG_OK)
        assert torch.count_nonzero(out).item() == 0
    plan.close()


def test_x0_aliasing_x(prob):
    op, b, x0 = prob
    plan = wmg.Plan(P.n, P.m, P.D, levels=3, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID)
    xa = dev(x0)
    ref, _, _, _ = plan.solve(dev(b), wmg.SOLVER_GMRES, True, 6, 0.0, 3, x0=dev(x0))
    plan.solve(dev(b), wmg.SOLVER_GMRES, True, 6, 0.0, 3, out=xa, x0=xa)
    assert torch.equal(xa, ref)
    plan.close()


# ---- checkpoint / resume ----------------------------------------------------
CASES = {
    "sirt": (wmg.SOLVER_SIRT, False, 20, dict(levels=3)),
    "cgls": (wmg.SOLVER_CGLS, False, 20, dict(levels=3)),
    # the symmetric cycle with a first smoothing sweep fused into the
    # backprojection: the sweep's result is part of the state
    "wmg-cgls": (wmg.SOLVER_CGLS, True, 20,
                 dict(levels=3, nu1=1, nu2=1, hybrid_depth=1, cycle=wmg.CYCLE_SYMMETRIC)),
    "wmg-gmres": (wmg.SOLVER_GMRES, True, 4, dict(levels=3, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID)),
    "gmres": (wmg.SOLVER_GMRES, False, 4, dict(levels=3)),
    "wmg-bicgstab": (wmg.SOLVER_BICGSTAB, True, 20,
                     dict(levels=3, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID)),
    "bicgstab": (wmg.SOLVER_BICGSTAB, False, 20, dict(levels=3)),
}


def make(prec, kw, lam=0.02):
    return wmg.Plan(P.n, P.m, P.D, lam=lam, precision=prec, **kw)


def batch(prob, prec):
    # two problems: the phantom's sinogram, and a zero sinogram (solved at
    # once by the Krylov solvers, so it stays ended across the checkpoint)
    dt = torch.float64 if prec == wmg.PREC_F64 else torch.float32
    _, b, _ = prob
    return torch.cat([dev(b, dt), torch.zeros(len(b), dtype=dt, device="cuda")])


def same(a, b):
    xa, ia, ha, rca = a
    xb, ib, hb, rcb = b
    assert torch.equal(xa, xb)
    assert ia == ib and rca == rcb
    assert len(ha) == len(hb) and all(np.array_equal(u, v) for u, v in zip(ha, hb))


@pytest.mark.parametrize("prec", [wmg.PREC_F64, wmg.PREC_F32])
@pytest.mark.parametrize("case", list(CASES))
def test_resume_in_a_new_plan_is_the_uninterrupted_solve(prob, prec, case):
    solver, pre, restart, kw = CASES[case]
    b2 = batch(prob, prec)
    k1, K = 8, 14                      # 8: a restart of GMRES(4)
    p = make(prec, kw)
    full = p.solve(b2, solver, pre, K, 0.0, restart, history=True)
    p.close()
    p1 = make(prec, kw)
    part = p1.solve(b2, solver, pre, k1, 0.0, restart, history=True)
    assert part[1][0][0] == k1 and part[3] == wmg.WMG_NOT_CONVERGED
    blob = p1.state_export()
    p1.close()
    p2 = make(prec, kw)
    p2.state_import(blob)
    res = p2.resume(b2, K, 0.0, history=True)
    same(res, full)
    p2.close()


@pytest.mark.parametrize("case", ["wmg-cgls", "wmg-gmres", "wmg-bicgstab", "sirt"])
def test_chained_resumes_in_the_same_plan(prob, case):
    solver, pre, restart, kw = CASES[case]
    b2 = batch(prob, wmg.PREC_F32)
    p = make(wmg.PREC_F32, kw)
    full = p.solve(b2, solver, pre, 16, 0.0, restart, history=True)
    p.solve(b2, solver, pre, 4, 0.0, restart)
    p.resume(b2, 8, 0.0)
    p.resume(b2, 8, 0.0)               # nothing left to do: the same state
    res = p.resume(b2, 16, 0.0, history=True)
    same(res, full)
    # an export / import round trip in the same plan changes nothing
    blob = p.state_export()
    p.state_import(blob)
    assert p.state_export() == blob
    p.close()


def test_resume_with_a_tolerance_converges_like_the_uninterrupted_solve(prob):
    solver, pre, restart, kw = CASES["wmg-gmres"]
    b2 = batch(prob, wmg.PREC_F64)
    p = make(wmg.PREC_F64, kw)
    full = p.solve(b2, solver, pre, 300, 1e-6, restart, history=True)
    assert full[3] == wmg.WMG_OK
    p.solve(b2, solver, pre, 8, 1e-6, restart)
    res = p.resume(b2, 300, 1e-6, history=True)
    same(res, full)
    p.close()


def test_state_errors(prob):
    solver, pre, restart, kw = CASES["wmg-gmres"]
    b2 = batch(prob, wmg.PREC_F64)
    p = make(wmg.PREC_F64, kw)
    with pytest.raises(wmg.WmgError):
        p.state_export()                                   # no solve yet
    with pytest.raises(wmg.WmgError):
        p.resume(b2, 10, 0.0)
    p.solve(b2, solver, pre, 8, 0.0, restart)
    blob = p.state_export()
    with pytest.raises(wmg.WmgError):
        p.resume(b2, 4, 0.0)                               # below the iterations done
    with pytest.raises(wmg.WmgError):
        p.state_import(blob[:-8])                          # truncated
    with pytest.raises(wmg.WmgError):
        p.state_import(b"x" * len(blob))                   # not a state
    other = make(wmg.PREC_F64, kw, lam=0.03)               # other options
    with pytest.raises(wmg.WmgError):
        other.state_import(blob)
    other.close()
    q = make(wmg.PREC_F32, kw)                             # other precision
    with pytest.raises(wmg.WmgError):
        q.state_import(blob)
    q.close()
    # a projection reuses the solver pools: the state is gone
    p.state_import(blob)
    p.project(torch.zeros(2 * p.N, dtype=torch.float64, device="cuda"))
    with pytest.raises(wmg.WmgError):
        p.resume(b2, 10, 0.0)
    p.close()
