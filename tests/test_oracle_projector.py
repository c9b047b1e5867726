"""Pins for the oracle's projection matrix W (Section 2.1, eq. sys): three
independent constructions, hand-computed chords, closed-form row and column
sums, the symmetries of the parallel-beam geometry, and the trigonometric
table's exact special angles."""
import json
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def trapezoid_dense(n, m, D, dt=1.0, t0=0.0):
    """W from the trapezoid law, one (ray, pixel) pair at a time."""
    op = oracle.Op(n, m, D, dt, t0)
    c, s = op.trig()
    W = np.zeros((m * D, n * n))
    for a in range(m):
        for k in range(D):
            T = (k - (D - 1) / 2) * dt + t0
            for iy in range(n):
                for ix in range(n):
                    tau = (ix + 0.5 - n / 2) * c[a] + (iy + 0.5 - n / 2) * s[a]
                    W[a * D + k, iy * n + ix] = oracle.weight_trapezoid(c[a], s[a], T - tau) / n
    return W


GEOMS = [(4, 8, 7, 1.0, 0.0), (6, 12, 9, 1.0, 0.0), (8, 24, 12, 1.0, 0.0), (5, 7, 8, 1.0, 0.0),
         (4, 4, 6, 1.0, 0.0), (6, 10, 11, 0.75, 0.3), (8, 16, 11, 1.0, 0.5), (3, 2, 3, 1.0, 0.0)]


@pytest.mark.parametrize("n,m,D,dt,t0", GEOMS)
def test_three_constructions_agree(n, m, D, dt, t0):
    walk = oracle.Op(n, m, D, dt, t0).dense()
    clip = oracle.Op(n, m, D, dt, t0, method=1).dense()
    trap = trapezoid_dense(n, m, D, dt, t0)
    assert np.abs(walk - clip).max() < 1e-13
    assert np.abs(walk - trap).max() < 1e-13


def test_golden_chords():
    d = json.load(open(os.path.join(HERE, "golden", "chords.json")))
    for case in d["cases"]:
        n, m, D, a, k = case["n"], case["m"], case["D"], case["a"], case["k"]
        W = oracle.Op(n, m, D).dense()
        row = W[a * D + k].reshape(n, n)
        want = np.zeros((n, n))
        for ix, iy, w in case["weights"]:
            want[iy, ix] = w
        assert np.abs(row - want).max() < 1e-14, case["why"]


def square_chord(c, s, t, side):
    """Length of the line p.(c,s) = t inside a square of the given side
    centred at the origin, with the half-split rule on its border."""
    al, be, d = max(abs(c), abs(s)), min(abs(c), abs(s)), abs(t)
    if be == 0.0:
        return side if d < side / 2 else (side / 2 if d == side / 2 else 0.0)
    return min(max((side * (al + be) / 2 - d) / (al * be), 0.0), side / al)


@pytest.mark.parametrize("n,m,D", [(64, 90, 91), (16, 24, 23), (12, 30, 18)])
def test_row_sums_are_chords(n, m, D):
    op = oracle.Op(n, m, D)
    rowptr, col, val = op.csr()
    c, s = op.trig()
    rs = np.array([val[rowptr[i]:rowptr[i + 1]].sum() for i in range(op.M)])
    want = np.array([square_chord(c[a], s[a], (k - (D - 1) / 2) / n, 1.0)
                     for a in range(m) for k in range(D)])
    assert np.abs(rs - want).max() < 1e-13


@pytest.mark.parametrize("n,D", [(16, 23), (16, 24), (15, 22), (8, 12)])
def test_column_sums_axis_angles(n, D):
    """At theta = 0 (and pi/2 for even m), with detectors covering the image,
    every pixel collects exactly one pixel height h in total."""
    m = 4
    W = oracle.Op(n, m, D).dense()
    for a in (0, m // 2):
        col = W[a * D:(a + 1) * D].sum(axis=0)
        assert np.abs(col - 1.0 / n).max() < 1e-15


def test_adjoint():
    op = oracle.Op(24, 30, 35)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(op.N), rng.standard_normal(op.M)
    lhs, rhs = op.project(x) @ y, x @ op.backproject(y)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert np.allclose(op.project(x), op.dense() @ x, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,m,D", [(16, 20, 23), (16, 20, 24), (12, 8, 17)])
def test_rotation_by_90_degrees(n, m, D):
    """x'(p) = x(R^-1 p), R = +90 deg: (W x')[a,k] = (W x)[a-m/2, k] for a >= m/2,
    (W x)[a+m/2, D-1-k] otherwise (centred detector, t_{D-1-k} = -t_k)."""
    op = oracle.Op(n, m, D)
    x = np.random.default_rng(2).random((n, n))
    xr = np.empty_like(x)
    for iy in range(n):
        for ix in range(n):
            xr[iy, ix] = x[n - 1 - ix, iy]
    p = op.project(x.reshape(-1)).reshape(m, D)
    pr = op.project(xr.reshape(-1)).reshape(m, D)
    h = m // 2
    assert np.abs(pr[h:] - p[:h]).max() < 1e-12
    assert np.abs(pr[:h] - p[h:, ::-1]).max() < 1e-12


@pytest.mark.parametrize("n,m,D", [(16, 20, 23), (10, 9, 15)])
def test_mirror_symmetry(n, m, D):
    """Mirror in x: (W x'')[a,k] = (W x)[m-a, k] for a >= 1, (W x)[0, D-1-k] for a = 0."""
    op = oracle.Op(n, m, D)
    x = np.random.default_rng(3).random((n, n))
    xm = x[:, ::-1].copy()
    p = op.project(x.reshape(-1)).reshape(m, D)
    pm = op.project(xm.reshape(-1)).reshape(m, D)
    assert np.abs(pm[1:] - p[:0:-1]).max() < 1e-12
    assert np.abs(pm[0] - p[0, ::-1]).max() < 1e-12


def test_single_pixel_images():
    """Projection of a unit pixel = that pixel's column of W = its clipped chords."""
    n, m, D = 6, 9, 10
    op = oracle.Op(n, m, D)
    Wc = oracle.Op(n, m, D, method=1).dense()
    for j in (0, 7, 14, 35):
        e = np.zeros(op.N)
        e[j] = 1.0
        assert np.abs(op.project(e) - Wc[:, j]).max() < 1e-13


@pytest.mark.parametrize("m", [2, 4, 8, 12, 90, 180, 1024, 7])
def test_trig_table(m):
    c, s = oracle.Op(4, m, 3).trig()
    theta = np.pi * np.arange(m) / m
    assert np.abs(c - np.cos(theta)).max() < 1e-15
    assert np.abs(s - np.sin(theta)).max() < 1e-15
    assert c[0] == 1.0 and s[0] == 0.0
    if m % 2 == 0:
        h = m // 2
        assert c[h] == 0.0 and s[h] == 1.0
        assert np.array_equal(c[h:], -s[:h]) and np.array_equal(s[h:], c[:h])
    if m % 4 == 0:
        assert c[m // 4] == s[m // 4] == math.sqrt(0.5)
    assert np.array_equal(c[1:], -c[:0:-1]) and np.array_equal(s[1:], s[:0:-1])


def test_nnz_scale():
    """nnz(W) is close to (4/pi) m N for detectors covering the image."""
    op = oracle.Op(64, 90, 91)
    ratio = op.nnz / ((4 / math.pi) * 90 * 64 * 64)
    assert 0.95 < ratio < 1.1


def test_ray_row_matches_assembled_rows():
    """The single-row builder gives exactly the rows of the assembled W."""
    for (n, m, D, dt, t0) in [(16, 12, 23, 1.0, 0.0), (20, 9, 31, 1.25, 0.5), (24, 17, 35, 1.0, 0.0)]:
        op = oracle.Op(n, m, D, dt, t0)
        rp, col, val = op.csr()
        for r in range(0, m * D, 7):
            c, v = oracle.ray_row(n, m, D, r // D, r % D, dt, t0)
            np.testing.assert_array_equal(c, col[rp[r]:rp[r + 1]])
            np.testing.assert_array_equal(v, val[rp[r]:rp[r + 1]])
