"""Pins for the oracle's WMG preconditioner (Section 3.1): leaf Galerkin
matrices against dense products of explicit W and the literal Haar operators,
the l1-Jacobi diagonal, the additive and hybrid WTG recursions against a dense
transcription of the WTG scheme's steps with Galerkin coarse operators
(eq. galerkin), and the special case of a single level (B = A^-1)."""
import numpy as np
import pytest

import oracle
from test_oracle_haar import band_ops, literal_packet_matrix

GEOM = (16, 24, 23)


def dense_A(op, lam):
    W = op.dense()
    return W.T @ W + lam * np.eye(op.N)


@pytest.mark.parametrize("levels,lam", [(2, 0.0), (3, 0.0), (3, 0.7), (4, 0.0)])
def test_leaf_matrices(levels, lam):
    op = oracle.Op(*GEOM)
    L = levels - 1
    wmg = oracle.Wmg(op, levels, lam=lam, factor=False)
    Q = literal_packet_matrix(op.n, L)          # rows: leaf coefficients
    A = dense_A(op, lam)
    P = (op.n >> L) ** 2
    for k in range(4 ** L):
        Qk = Q[k * P:(k + 1) * P]
        Dk = Qk @ A @ Qk.T
        assert np.abs(wmg.leaf(k) - Dk).max() < 1e-13 * np.abs(Dk).max()
        assert np.linalg.eigvalsh(Dk).min() > 0


def test_l1_jacobi_diagonal():
    op = oracle.Op(*GEOM)
    A = dense_A(op, 0.3)
    wmg = oracle.Wmg(op, 2, 1, 1, lam=0.3)
    assert np.allclose(wmg.dinv(), 1.0 / np.abs(A).sum(axis=1), rtol=1e-13, atol=0)


def dense_B(wmg, N):
    return np.column_stack([wmg.apply(e) for e in np.eye(N)])


def test_single_level_is_exact_inverse():
    """l = 1: one leaf holds the whole problem, B = A^-1; PCG needs one step."""
    op = oracle.Op(12, 20, 17)
    A = dense_A(op, 0.0)
    wmg = oracle.Wmg(op, 1)
    assert np.abs(dense_B(wmg, op.N) @ A - np.eye(op.N)).max() < 1e-9
    b = op.project(np.random.default_rng(5).random(op.N))
    x, k, hist = oracle.cgls(op, b, 5, 1e-10, precond=wmg)
    assert k == 1 and hist[-1] < 1e-10


def wtg_dense(A, c, side, depth, L, hybrid_depth, symmetric, multiplicative=False):
    """The WTG correction scheme on A e = c, recursively: LL band first, then
    (hybrid) one residual recomputation, then LH, HL, HH; coarse operators by
    Galerkin products I_id A I_id^T; exact solves at depth L. With `symmetric`
    the LL band is corrected once more from the residual of the whole step;
    with `multiplicative` the residual is recomputed before every band."""
    if depth == L:
        return np.linalg.solve(A, c)
    ops = band_ops(side)
    sub = [B @ A @ B.T for B in ops]
    inner = (lambda Ai, ci: wtg_dense(Ai, ci, side // 2, depth + 1, L, hybrid_depth, symmetric,
                                      multiplicative))
    x = ops[0].T @ inner(sub[0], ops[0] @ c)
    active = depth < hybrid_depth
    r = c - A @ x if active else c
    for i in (1, 2, 3):
        if multiplicative and active and i > 1:
            r = c - A @ x
        x = x + ops[i].T @ inner(sub[i], ops[i] @ r)
    if symmetric and active:
        r = c - A @ x
        x = x + ops[0].T @ inner(sub[0], ops[0] @ r)
    return x


def smoothed_dense(A, s, Dinv, nu1, nu2, omega, corr):
    z = np.zeros_like(s)
    for _ in range(nu1):
        z = z + omega * Dinv * (s - A @ z)
    z = z + corr(s - A @ z)
    for _ in range(nu2):
        z = z + omega * Dinv * (s - A @ z)
    return z


CASES = [  # levels, nu1, nu2, cycle, hybrid_depth, lam
    (3, 0, 0, oracle.CYCLE_ADDITIVE, 0, 0.0),
    (3, 1, 1, oracle.CYCLE_ADDITIVE, 0, 0.0),
    (3, 0, 0, oracle.CYCLE_HYBRID, 2, 0.0),
    (3, 1, 1, oracle.CYCLE_HYBRID, 2, 0.5),
    (4, 0, 0, oracle.CYCLE_HYBRID, 1, 0.0),
    (4, 0, 0, oracle.CYCLE_HYBRID, 3, 0.0),
    (3, 0, 0, 2, 2, 0.0),
    (4, 1, 1, 2, 2, 0.2),
    (3, 2, 1, oracle.CYCLE_HYBRID, 1, 0.0),
    (3, 0, 0, oracle.CYCLE_MULTIPLICATIVE, 2, 0.0),
    (4, 0, 0, oracle.CYCLE_MULTIPLICATIVE, 1, 0.0),
    (4, 1, 1, oracle.CYCLE_MULTIPLICATIVE, 3, 0.3),
]


@pytest.mark.parametrize("levels,nu1,nu2,cycle,hd,lam", CASES)
def test_wmg_apply_matches_dense_wtg(levels, nu1, nu2, cycle, hd, lam):
    op = oracle.Op(*GEOM)
    A = dense_A(op, lam)
    Dinv = 1.0 / np.abs(A).sum(axis=1)
    wmg = oracle.Wmg(op, levels, nu1, nu2, 1.0, lam, cycle, hd)
    L = levels - 1
    hyb_depth = 0 if cycle == oracle.CYCLE_ADDITIVE else hd
    rng = np.random.default_rng(6)
    for _ in range(3):
        s = rng.standard_normal(op.N)
        want = smoothed_dense(A, s, Dinv, nu1, nu2, 1.0,
                              lambda r: wtg_dense(A, r, op.n, 0, L, hyb_depth, cycle == 2,
                                                  cycle == oracle.CYCLE_MULTIPLICATIVE))
        got = wmg.apply(s)
        assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()


def test_additive_is_block_jacobi_in_packet_basis():
    op = oracle.Op(*GEOM)
    A = dense_A(op, 0.0)
    L = 2
    Q = literal_packet_matrix(op.n, L)
    P = (op.n >> L) ** 2
    Bd = np.zeros((op.N, op.N))
    for k in range(4 ** L):
        Qk = Q[k * P:(k + 1) * P]
        Bd += Qk.T @ np.linalg.inv(Qk @ A @ Qk.T) @ Qk
    B = dense_B(oracle.Wmg(op, L + 1), op.N)
    assert np.abs(B - Bd).max() < 1e-9 * np.abs(Bd).max()


@pytest.mark.parametrize("nu,cycle,hd", [(1, oracle.CYCLE_ADDITIVE, 0), (0, 2, 2), (1, 2, 2), (1, 2, 1)])
def test_symmetric_cycles_are_spd(nu, cycle, hd):
    op = oracle.Op(*GEOM)
    B = dense_B(oracle.Wmg(op, 3, nu, nu, 1.0, 0.0, cycle, hd), op.N)
    assert np.abs(B - B.T).max() < 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_hybrid_cycle_is_not_symmetric():
    op = oracle.Op(*GEOM)
    B = dense_B(oracle.Wmg(op, 3, 0, 0, 1.0, 0.0, oracle.CYCLE_HYBRID, 2), op.N)
    assert np.abs(B - B.T).max() > 1e-6 * np.abs(B).max()


def test_leaf_without_rays_is_not_spd_unless_regularised():
    # one angle (vertical rays) and a 4-bin detector: the rays cover the
    # central 4 pixel columns only, so the leaf Galerkin matrices
    # Q_k^T W^T W Q_k have exactly zero rows for the 2x2 blocks off that band
    # and Cholesky meets a zero pivot; lambda I (eq. sys_reg) makes every
    # leaf SPD
    op = oracle.Op(16, 1, 4)
    assert oracle.Wmg(op, 2).status == -4
    assert oracle.Wmg(op, 2, lam=0.1).status == 0
    bare = oracle.Wmg(op, 2, factor=False)
    assert any((np.abs(bare.leaf(k)).sum(axis=1) == 0).any() for k in range(bare.K))
    reg = oracle.Wmg(op, 2, lam=0.1, factor=False)
    for k in range(reg.K):
        assert np.linalg.eigvalsh(reg.leaf(k)).min() >= 0.1 * (1 - 1e-12)


def test_two_level_multiplicative_cycle_is_the_wtg_propagator():
    # two levels, the multiplicative rule at the root, exact band solves: the
    # error propagator I - B A is eq. wmg's product of the four band
    # corrections, built densely from the Haar band restrictions
    op = oracle.Op(16, 20, 23)
    for lam in (0.0, 0.4):
        A = dense_A(op, lam)
        B = dense_B(oracle.Wmg(op, 2, 0, 0, 1.0, lam, oracle.CYCLE_MULTIPLICATIVE, 1), op.N)
        E = oracle.wtg_propagator(op, lam)
        assert np.abs((np.eye(op.N) - B @ A) - E).max() < 1e-9
