"""Spectral check of Section 3.2 on the oracle: the condition numbers the
paper prints for N = 40 x 40, 100 angles of 40 rays (Figure 4: kappa =
8.68e4 for W^T W, 4.52e4 with the classical TG(1,1)-SIRT preconditioner,
3.42e2 with the wavelet two-grid WTG of eq. wmg), from dense error
propagators built from the Haar band restrictions and Galerkin products.
The paper gives neither the detector width nor its kernel's normalisation,
and its W is Joseph's kernel, so the printed values are not reproducible
here (parity unpinned for the exact values). What the test holds is what the
paper's text states and what does not depend on those choices: the order of
magnitude of each condition number (O(10^4) unpreconditioned and with the
classical two-grid scheme, O(10^2) with WTG) and their ordering. A 40-bin
detector spanning the image diagonal with exact intersection lengths is the
geometry; Joseph's kernel on the same detectors gives the same ordering at
larger condition numbers."""
import math

import numpy as np
import pytest

import oracle

n, m, D = 40, 100, 40


@pytest.fixture(scope="module")
def strip_op():
    return oracle.Op(n, m, D, math.sqrt(2.0), 0.0)


def test_band_restrictions_are_orthonormal_and_eq_intops():
    R = oracle.haar_band_restrictions(8)
    Q = np.vstack(R)
    assert np.abs(Q @ Q.T - np.eye(64)).max() < 1e-14
    # LL band = eq. intops: (1/sqrt 2)[1 1] in each direction (Kronecker product)
    r1 = np.zeros((4, 8))
    for i in range(4):
        r1[i, 2 * i:2 * i + 2] = 1 / math.sqrt(2)
    assert np.abs(R[0] - np.kron(r1, r1)).max() < 1e-14


def test_paper_condition_numbers(strip_op):
    W = strip_op.dense()
    k_plain = oracle.condition_number(W.T @ W, symmetric=True)
    k_tg = oracle.preconditioned_condition_number(oracle.tg_sirt_propagator(strip_op, 1, 1))
    k_wtg = oracle.preconditioned_condition_number(oracle.wtg_propagator(strip_op))
    # orders of magnitude of Figure 4's values (8.68e4, 4.52e4, 3.42e2)
    assert 1e4 <= k_plain < 1e5
    assert 1e4 <= k_tg < 1e5
    assert 1e2 <= k_wtg < 1e3
    # ordering: the classical two-grid scheme helps little, WTG by orders of magnitude
    assert k_wtg < k_tg < k_plain
    assert k_wtg < 1e-2 * k_plain


def test_exact_coarse_solves_annihilate_their_band(strip_op):
    # after a band's exact correction the residual has no component in that
    # band: R_id A E_id = 0
    W = strip_op.dense()
    A = W.T @ W
    R = oracle.haar_band_restrictions(n)
    E = oracle.wtg_propagator(strip_op)
    # the last correction is HH: its residual component vanishes exactly
    assert np.abs(R[3] @ A @ E).max() < 1e-9 * np.abs(A).max()


def test_joseph_ordering():
    op = oracle.Op(n, m, D, 1.0, 0.0, kernel=oracle.KERNEL_JOSEPH)
    W = op.dense()
    k_plain = oracle.condition_number(W.T @ W, symmetric=True)
    k_tg = oracle.preconditioned_condition_number(oracle.tg_sirt_propagator(op, 1, 1))
    k_wtg = oracle.preconditioned_condition_number(oracle.wtg_propagator(op))
    assert k_wtg < 1e-2 * k_plain and k_wtg < 1e-2 * k_tg and k_tg < k_plain
