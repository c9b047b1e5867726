"""Pins for the oracle's solvers started from an initial guess x0 (Section
2.3.1 on the normal equations, eq. sys_reg): the first iterate of CGLS,
GMRES and BiCGStab from x0 against the closed form of that step written
with the dense matrix, CGLS from x0 against CGLS on the shifted system, and
the restart identity of GMRES(m): a run restarted by hand from the iterate
of a restart boundary is the uninterrupted run."""
import numpy as np
import pytest

import oracle

GEOM = (12, 18, 17)


def setup(lam=0.0, seed=3):
    op = oracle.Op(*GEOM)
    rng = np.random.default_rng(seed)
    x = rng.random(op.N)
    b = op.project(x) + 0.01 * rng.standard_normal(op.M)
    x0 = rng.random(op.N) - 0.5
    W = op.dense()
    A = W.T @ W + lam * np.eye(op.N)
    return op, b, x0, W, A


@pytest.mark.parametrize("lam", [0.0, 0.3])
def test_cgls_first_step_from_x0(lam):
    # CGLS's first step is steepest descent with an exact line search on
    # |W x - b|^2 + lam |x|^2 from x0: p = s0 = W^T (b - W x0) - lam x0,
    # alpha = |s0|^2 / (|W p|^2 + lam |p|^2)
    op, b, x0, W, A = setup(lam)
    s0 = W.T @ (b - W @ x0) - lam * x0
    alpha = (s0 @ s0) / ((W @ s0) @ (W @ s0) + lam * (s0 @ s0))
    x1 = x0 + alpha * s0
    x, k, hist = oracle.cgls(op, b, 1, 0.0, lam, None, x0=x0)
    assert k == 1
    assert np.linalg.norm(x - x1) < 1e-12 * np.linalg.norm(x1)
    s1 = W.T @ (b - W @ x1) - lam * x1
    assert abs(hist[1] - np.linalg.norm(s1) / np.linalg.norm(s0)) < 1e-12


def test_cgls_from_x0_is_cgls_on_the_shifted_system():
    # without regularisation, x0 + (CGLS on W e = b - W x0 from e = 0) is
    # CGLS on W x = b from x0, iterate by iterate
    op, b, x0, W, _ = setup()
    for k in (1, 5, 17):
        x, kk, hist = oracle.cgls(op, b, k, 0.0, 0.0, None, x0=x0)
        e, ke, hist_e = oracle.cgls(op, b - op.project(x0), k, 0.0, 0.0, None)
        assert kk == ke == k
        assert np.linalg.norm(x - (x0 + e)) < 1e-11 * np.linalg.norm(x)
        assert np.abs(hist - hist_e).max() < 1e-11


@pytest.mark.parametrize("lam", [0.0, 0.3])
def test_gmres_first_step_from_x0(lam):
    # one Arnoldi step: x1 = x0 + y v, v = r0 / |r0|, y minimising
    # |r0 - y A v|; r0 = W^T b - A x0
    op, b, x0, W, A = setup(lam)
    r0 = W.T @ b - A @ x0
    v = r0 / np.linalg.norm(r0)
    Av = A @ v
    y = (Av @ r0) / (Av @ Av)
    x1 = x0 + y * v
    x, k, hist = oracle.gmres(op, b, 1, 20, 0.0, lam, None, x0=x0)
    assert k == 1
    assert np.linalg.norm(x - x1) < 1e-12 * np.linalg.norm(x1)
    # at the cycle end the history holds the true residual relative to |r0|
    r1 = W.T @ b - A @ x1
    assert abs(hist[1] - np.linalg.norm(r1) / np.linalg.norm(r0)) < 1e-12


@pytest.mark.parametrize("lam", [0.0, 0.3])
def test_bicgstab_first_step_from_x0(lam):
    # van der Vorst's first step from x0 with rh = r0: p = r0, v = A p,
    # alpha = |r0|^2 / <r0, v>, s = r0 - alpha v, t = A s,
    # omega = <t, s> / <t, t>, x1 = x0 + alpha p + omega s
    op, b, x0, W, A = setup(lam)
    r0 = W.T @ b - A @ x0
    v = A @ r0
    alpha = (r0 @ r0) / (r0 @ v)
    s = r0 - alpha * v
    t = A @ s
    omega = (t @ s) / (t @ t)
    x1 = x0 + alpha * r0 + omega * s
    x, k, hist, st = oracle.bicgstab(op, b, 1, 0.0, lam, None, x0=x0)
    assert k == 1 and st == 1
    assert np.linalg.norm(x - x1) < 1e-12 * np.linalg.norm(x1)
    assert abs(hist[1] - np.linalg.norm(s - omega * t) / np.linalg.norm(r0)) < 1e-12


@pytest.mark.parametrize("pre", [False, True])
def test_gmres_restart_identity(pre):
    # GMRES(m) restarts from the current iterate with the true residual
    # f - A x: stopping at a restart boundary and starting again from that
    # iterate continues the same run, to the last bit
    op, b, _, _, _ = setup(0.1)
    M = oracle.Wmg(op, 3, 0, 0, 1.0, 0.1, oracle.CYCLE_HYBRID, 1) if pre else None
    m, k1, K = 5, 10, 17
    x_full, k, hist = oracle.gmres(op, b, K, m, 0.0, 0.1, M)
    x_half, k_a, hist_a = oracle.gmres(op, b, k1, m, 0.0, 0.1, M)
    x_rest, k_b, hist_b = oracle.gmres(op, b, K - k1, m, 0.0, 0.1, M, x0=x_half)
    assert (k, k_a, k_b) == (K, k1, K - k1)
    assert np.array_equal(x_rest, x_full)
    # the continued history is relative to the residual at the restart
    scale = hist[k1]
    assert np.abs(hist_b * scale - hist[k1:]).max() < 1e-12


def test_sirt_continuation_identity():
    # eq. sirt_it is stationary: k1 steps, then k2 from that iterate, are
    # k1 + k2 steps
    op, b, _, _, _ = setup()
    x_full, _ = oracle.sirt(op, b, 30, 0.2)
    x_a, _ = oracle.sirt(op, b, 12, 0.2)
    x_b, _ = oracle.sirt(op, b, 18, 0.2, x0=x_a)
    assert np.array_equal(x_b, x_full)


def test_zero_initial_guess_is_the_cold_start():
    op, b, _, _, _ = setup(0.1)
    z = np.zeros(op.N)
    for f in (lambda **k: oracle.cgls(op, b, 7, 0.0, 0.1, None, **k),
              lambda **k: oracle.gmres(op, b, 7, 3, 0.0, 0.1, None, **k),
              lambda **k: oracle.bicgstab(op, b, 7, 0.0, 0.1, None, **k)):
        assert np.array_equal(f()[0], f(x0=z)[0])
