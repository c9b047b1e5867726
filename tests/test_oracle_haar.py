"""Pins for the oracle's Haar wavelet-packet transform: the literal
Kronecker-product operators of eq. intops, eq. intops_wav and eq. 1of4-4of4,
their recursive composition (Section 3.1.3), orthonormality and the closed
form of the depth-L basis as blockwise 2D Walsh functions."""
import numpy as np
import pytest

import oracle


def I1(n):
    """Restriction I_{h,1D}^{2h} of eq. intops: rows [1 1]/sqrt2 on pairs."""
    M = np.zeros((n // 2, n))
    for i in range(n // 2):
        M[i, 2 * i] = M[i, 2 * i + 1] = 1 / np.sqrt(2)
    return M


def J1(n):
    """Wavelet operator J_{h,1D}^{2h} of eq. intops_wav: rows [1 -1]/sqrt2."""
    M = np.zeros((n // 2, n))
    for i in range(n // 2):
        M[i, 2 * i], M[i, 2 * i + 1] = 1 / np.sqrt(2), -1 / np.sqrt(2)
    return M


def band_ops(n):
    """eq. 1of4 .. 4of4 in the order LL, LH, HL, HH (row-major vec: the left
    Kronecker factor acts on the row index iy)."""
    return [np.kron(I1(n), I1(n)), np.kron(I1(n), J1(n)),
            np.kron(J1(n), I1(n)), np.kron(J1(n), J1(n))]


def literal_packet_matrix(n, L):
    """Rows = leaf coefficients in the leaf layout (leaf k = sum id_d 4^(L-d),
    id_1 = the first split), built by composing the literal operators."""
    rows = []

    def rec(side, depth, op):
        if depth == L:
            rows.append(op)
            return
        for B in band_ops(side):
            rec(side // 2, depth + 1, B @ op)

    rec(n, 0, np.eye(n * n))
    return np.vstack(rows)


@pytest.mark.parametrize("n,L", [(2, 1), (4, 1), (4, 2), (8, 1), (8, 2), (8, 3), (16, 2), (12, 2)])
def test_matches_literal_kronecker(n, L):
    Q = literal_packet_matrix(n, L)
    Qo = np.column_stack([oracle.packet_analysis(e, n, L) for e in np.eye(n * n)])
    assert np.abs(Q - Qo).max() < 1e-15
    So = np.column_stack([oracle.packet_synthesis(e, n, L) for e in np.eye(n * n)])
    assert np.abs(Q.T - So).max() < 1e-15


@pytest.mark.parametrize("n,L", [(4, 2), (8, 3), (16, 2), (32, 4)])
def test_orthonormal_and_perfect_reconstruction(n, L):
    rng = np.random.default_rng(4)
    x = rng.standard_normal(n * n)
    c = oracle.packet_analysis(x, n, L)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-13 * np.linalg.norm(x)
    assert np.abs(oracle.packet_synthesis(c, n, L) - x).max() < 1e-14 * np.abs(x).max() * L


@pytest.mark.parametrize("n,L", [(8, 2), (16, 3), (16, 4), (24, 3)])
def test_walsh_closed_form(n, L):
    """Leaf k's basis function on block (cy, cx) is
    2^-L (-1)^(popcount(HY & ly) + popcount(HX & lx)), HY/HX collecting the
    y/x high-pass bits of the path (bit d-1 for the d-th split)."""
    B, nc = 1 << L, n >> L
    Q = np.column_stack([oracle.packet_analysis(e, n, L) for e in np.eye(n * n)])
    for k in range(4 ** L):
        ids = [(k >> (2 * (L - d))) & 3 for d in range(1, L + 1)]
        HY = sum(((i >> 1) & 1) << d for d, i in enumerate(ids))
        HX = sum((i & 1) << d for d, i in enumerate(ids))
        for cy in range(nc):
            for cx in range(nc):
                row = Q[k * nc * nc + cy * nc + cx].reshape(n, n)
                want = np.zeros((n, n))
                for ly in range(B):
                    for lx in range(B):
                        sgn = (bin(HY & ly).count("1") + bin(HX & lx).count("1")) & 1
                        want[cy * B + ly, cx * B + lx] = (-1.0) ** sgn / B
                assert np.abs(row - want).max() < 1e-15
