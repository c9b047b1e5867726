"""Pins for the oracle's solvers (Sections 2.2.1 and 2.3.1): convergence to
dense normal-equation solutions, SIRT's fixed point, the Krylov-subspace
optimality that defines CGLS, PCG and GMRES iterates, and the qualitative
ordering of Section 4 (SIRT slowest, WMG-preconditioned Krylov fastest)."""
import numpy as np
import pytest

import oracle
import synthetic as S

GEOM = (16, 24, 23)


def setup(geom=GEOM, noise=0.01, seed=7):
    op = oracle.Op(*geom)
    rng = np.random.default_rng(seed)
    x = rng.random(op.N)
    b = op.project(x) + noise * rng.standard_normal(op.M)
    return op, b


def ls_solution(op, b, lam):
    W = op.dense()
    return np.linalg.solve(W.T @ W + lam * np.eye(op.N), W.T @ b)


@pytest.mark.parametrize("lam", [0.0, 0.05])
@pytest.mark.parametrize("pc", [None, (oracle.CYCLE_ADDITIVE, 0, 1), (2, 2, 1), (2, 1, 0)])
def test_cgls_converges_to_dense_solution(lam, pc):
    op, b = setup()
    xs = ls_solution(op, b, lam)
    M = None if pc is None else oracle.Wmg(op, 3, pc[2], pc[2], 1.0, lam, pc[0], pc[1])
    x, k, hist = oracle.cgls(op, b, 2000, 1e-13, lam, M)
    assert np.linalg.norm(x - xs) < 1e-10 * np.linalg.norm(xs)
    assert abs(op.ne_residual(b, x, lam) - hist[-1]) < 1e-10


@pytest.mark.parametrize("lam", [0.0, 0.05])
@pytest.mark.parametrize("pc", [None, (oracle.CYCLE_HYBRID, 2, 1), (oracle.CYCLE_HYBRID, 1, 0),
                                (oracle.CYCLE_ADDITIVE, 0, 0)])
def test_gmres_converges_to_dense_solution(lam, pc):
    op, b = setup()
    xs = ls_solution(op, b, lam)
    M = None if pc is None else oracle.Wmg(op, 3, pc[2], pc[2], 1.0, lam, pc[0], pc[1])
    x, k, hist = oracle.gmres(op, b, 3000, 20, 1e-13, lam, M)
    # the error is bounded by cond(A) times the residual (1e-13 here)
    W = op.dense()
    kappa = np.linalg.cond(W.T @ W + lam * np.eye(op.N))
    assert hist[-1] < 1e-13
    assert np.linalg.norm(x - xs) < 2e-13 * kappa * np.linalg.norm(xs)


def test_sirt_fixed_point():
    """SIRT's limit solves W^T R W x = W^T R b (C > 0 everywhere here)."""
    op, b = setup((6, 10, 9))
    W = op.dense()
    R, Cc = op.sirt_scalings()
    assert (Cc > 0).all()
    xs = np.linalg.solve(W.T @ (R[:, None] * W), W.T @ (R * b))
    x, hist = oracle.sirt(op, b, 20000)
    assert np.linalg.norm(x - xs) < 1e-10 * np.linalg.norm(xs)


def test_sirt_scalings():
    op = oracle.Op(8, 6, 14)           # wide detector: some rays miss the image
    W = op.dense()
    R, Cc = op.sirt_scalings()
    rs, cs = W.sum(axis=1), W.sum(axis=0)
    assert (rs == 0).any()
    assert np.allclose(R, np.where(rs > 0, 1 / np.where(rs > 0, rs, 1), 0), rtol=1e-14, atol=0)
    assert np.allclose(Cc, np.where(cs > 0, 1 / np.where(cs > 0, cs, 1), 0), rtol=1e-14, atol=0)


def krylov_basis(Mat, v, k):
    cols = [v]
    for _ in range(k - 1):
        cols.append(Mat @ cols[-1])
    Qb, _ = np.linalg.qr(np.column_stack(cols))
    return Qb


@pytest.mark.parametrize("k", [1, 3, 6])
def test_cgls_iterate_minimises_over_krylov_space(k):
    """x_k = argmin ||W x - b||^2 + lam ||x||^2 over K_k(A, W^T b)."""
    op, b = setup()
    lam = 0.02
    W = op.dense()
    A = W.T @ W + lam * np.eye(op.N)
    V = krylov_basis(A, W.T @ b, k)
    y = np.linalg.solve(V.T @ A @ V, V.T @ (W.T @ b))
    x, it, _ = oracle.cgls(op, b, k, 0.0, lam)
    assert it == k
    assert np.linalg.norm(x - V @ y) < 1e-9 * np.linalg.norm(V @ y)


@pytest.mark.parametrize("k", [2, 4])
def test_pcg_iterate_minimises_energy_over_krylov_space(k):
    """Preconditioned: x_k minimises the A-norm error over K_k(B A, B f)."""
    op, b = setup()
    W = op.dense()
    A = W.T @ W
    M = oracle.Wmg(op, 3, 1, 1, 1.0, 0.0, 2, 2)
    B = np.column_stack([M.apply(e) for e in np.eye(op.N)])
    f = W.T @ b
    V = krylov_basis(B @ A, B @ f, k)
    y = np.linalg.solve(V.T @ A @ V, V.T @ f)
    x, it, _ = oracle.cgls(op, b, k, 0.0, 0.0, M)
    assert np.linalg.norm(x - V @ y) < 1e-8 * np.linalg.norm(V @ y)


@pytest.mark.parametrize("k", [3, 7])
def test_gmres_iterate_minimises_residual(k):
    """Right preconditioning, no restart: x_k = B u_k with u_k minimising
    ||f - A B u|| over K_k(A B, f)."""
    op, b = setup()
    W = op.dense()
    A = W.T @ W
    M = oracle.Wmg(op, 3, 0, 0, 1.0, 0.0, oracle.CYCLE_HYBRID, 2)
    B = np.column_stack([M.apply(e) for e in np.eye(op.N)])
    f = W.T @ b
    V = krylov_basis(A @ B, f, k)
    y, *_ = np.linalg.lstsq(A @ B @ V, f, rcond=None)
    x, it, _ = oracle.gmres(op, b, k, 50, 0.0, 0.0, M)
    want = B @ V @ y
    assert np.linalg.norm(x - want) < 1e-8 * np.linalg.norm(want)


def test_full_gmres_terminates_within_N_steps():
    op, b = setup((8, 16, 12))
    xs = ls_solution(op, b, 0.0)
    x, k, hist = oracle.gmres(op, b, op.N, op.N, 1e-12)
    assert k <= op.N
    assert np.linalg.norm(x - xs) < 1e-8 * np.linalg.norm(xs)


def test_qualitative_ordering_small_workload():
    """Section 4.1's ordering on the 64x64 noiseless workload: SIRT far from
    converged, WMG-preconditioned Krylov needs fewer iterations than plain."""
    P = S.workload_small().problems[0]
    op = oracle.Op(P.n, P.m, P.D)
    b = op.project(P.image())
    _, k_plain, _ = oracle.gmres(op, b, 500, 20, 1e-4)
    M = oracle.Wmg(op, P.levels, 1, 1, 1.0, 0.0, oracle.CYCLE_HYBRID, 2)
    _, k_wmg, _ = oracle.gmres(op, b, 500, 20, 1e-4, 0.0, M)
    Ms = oracle.Wmg(op, P.levels, 1, 1, 1.0, 0.0, 2, 2)
    _, k_cg, _ = oracle.cgls(op, b, 500, 1e-4, 0.0, Ms)
    _, k_cgp, _ = oracle.cgls(op, b, 500, 1e-4)
    _, hs = oracle.sirt(op, b, 50)
    assert k_wmg < k_plain / 2
    assert k_cg < k_cgp / 2
    assert hs[-1] > 1e-3


def test_bicgstab_ordering_small_workload():
    """The ordering of the paper's tables (Section 4.1) for its own solver on
    the 64x64 noiseless workload, with the paper's cycle (hybrid rule at
    every depth, no smoothing): WMG-BiCGStab reaches 1e-4 in clearly fewer
    iterations than BiCGStab, and SIRT has not reached it after 20 times
    BiCGStab's count (all three measured by the same relative NE residual)."""
    P = S.workload_small().problems[0]
    op = oracle.Op(P.n, P.m, P.D)
    b = op.project(P.image())
    _, k_plain, _, st_plain = oracle.bicgstab(op, b, 400, 1e-4)
    M = oracle.Wmg(op, P.levels, 0, 0, 1.0, 0.0, oracle.CYCLE_HYBRID, P.levels - 1)
    _, k_wmg, _, st_wmg = oracle.bicgstab(op, b, 400, 1e-4, 0.0, M)
    _, hs = oracle.sirt(op, b, 20 * k_plain)
    assert st_plain == 0 and st_wmg == 0
    assert k_wmg < 0.75 * k_plain
    assert hs[-1] > 1e-4


@pytest.mark.parametrize("lam", [0.0, 0.05])
@pytest.mark.parametrize("pc", [None, (oracle.CYCLE_HYBRID, 2, 1), (oracle.CYCLE_ADDITIVE, 0, 0)])
def test_bicgstab_converges_to_dense_solution(lam, pc):
    """BiCGStab (the paper's solver) reaches the dense normal-equation
    solution, and its recurrence residual is the true residual of its
    iterate (a mismatch between the x and r updates breaks the second)."""
    op, b = setup()
    xs = ls_solution(op, b, lam)
    M = None if pc is None else oracle.Wmg(op, 3, pc[2], pc[2], 1.0, lam, pc[0], pc[1])
    x, k, hist, st = oracle.bicgstab(op, b, 3000, 1e-12, lam, M)
    assert st == 0
    W = op.dense()
    kappa = np.linalg.cond(W.T @ W + lam * np.eye(op.N))
    assert np.linalg.norm(x - xs) < 1e-11 * kappa * np.linalg.norm(xs)
    assert abs(op.ne_residual(b, x, lam) - hist[-1]) < 1e-10


def test_bicgstab_exact_preconditioner_one_step():
    """With B = A^{-1} (one WMG level: the single leaf is the whole operator)
    BiCGStab's first half-step is the exact solution: alpha = 1, s = 0,
    omega = 0, done in one iteration."""
    op, b = setup((8, 10, 13), noise=0.0)
    lam = 0.01
    M = oracle.Wmg(op, 1, 0, 0, 1.0, lam, oracle.CYCLE_ADDITIVE, 0)
    x, k, hist, st = oracle.bicgstab(op, b, 10, 1e-12, lam, M)
    assert (k, st) == (1, 0)
    np.testing.assert_allclose(x, ls_solution(op, b, lam), rtol=0, atol=1e-12 * np.abs(x).max())


def test_bicgstab_first_step_galerkin_conditions():
    """Unpreconditioned, the first half-step is a CG step (the shadow residual
    is r0): s = r0 - alpha A r0 is orthogonal to r0; omega minimises |r1| over
    s - omega A s, so r1 is orthogonal to A s. Both follow from the
    definitions and fail for a wrong alpha, omega or sign."""
    op, b = setup((10, 12, 15))
    W = op.dense()
    A = W.T @ W
    f = W.T @ b
    x1, k, hist, st = oracle.bicgstab(op, b, 1, 0.0, 0.0, None)
    assert k == 1
    r0 = f
    alpha = (r0 @ r0) / (r0 @ (A @ r0))
    s = r0 - alpha * (A @ r0)
    assert abs(s @ r0) < 1e-12 * (r0 @ r0)
    r1 = f - A @ x1
    # x1 = alpha r0 + omega s and r1 = s - omega A s: r1 orthogonal to A s
    assert abs(r1 @ (A @ s)) < 1e-10 * np.linalg.norm(r1) * np.linalg.norm(A @ s)
    omega = (x1 - alpha * r0) @ s / (s @ s)
    np.testing.assert_allclose(x1, alpha * r0 + omega * s, rtol=0, atol=1e-12 * np.abs(x1).max())


@pytest.mark.parametrize("mode", [oracle.SUMMATION_REVERSED, oracle.SUMMATION_PAIRWISE])
def test_summation_orders_evaluate_the_same_arithmetic(mode):
    # the rounding variants behind the parity floor: the products agree with
    # dense ones to rounding, and the converged solution is the dense one
    op, b = setup()
    W = op.dense()
    rng = np.random.default_rng(3)
    x, y = rng.random(op.N), rng.random(op.M)
    lam = 0.05
    xs = ls_solution(op, b, lam)
    try:
        oracle.set_summation(mode)
        p, q = op.project(x), op.backproject(y)
        assert np.abs(p - W @ x).max() < 1e-14 * np.abs(W @ x).max()
        assert np.abs(q - W.T @ y).max() < 1e-14 * np.abs(W.T @ y).max()
        xc, _, _ = oracle.cgls(op, b, 2000, 1e-13, lam)
        xg, _, _ = oracle.gmres(op, b, 400, 20, 1e-13, lam)
    finally:
        oracle.set_summation(oracle.SUMMATION_NATURAL)
    assert np.linalg.norm(xc - xs) < 1e-10 * np.linalg.norm(xs)
    assert np.linalg.norm(xg - xs) < 1e-10 * np.linalg.norm(xs)
    with pytest.raises(ValueError):
        oracle.set_summation(7)
