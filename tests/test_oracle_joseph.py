"""Pins of the oracle's Joseph kernel (the paper's W, Section 2.1; Joseph's
interpolation along the dominant axis): closed forms at the axis angles, a
hand-worked 3 x 3 example, exactness on affine images (linear interpolation
reproduces them, so a ray sum is a plain sum of the affine function at the
crossings), the perpendicular-distance form of the weights, the 45-degree tie
(rows and columns give the same weights there), the 90-degree rotation and
mirror symmetries, and agreement of the single-row builder with the assembled
matrix."""
import math

import numpy as np
import pytest

import oracle

J = oracle.KERNEL_JOSEPH


def hat(u):
    return max(0.0, 1.0 - abs(u))


@pytest.mark.parametrize("n,m,D,dt,t0", [(8, 6, 12, 1.0, 0.0), (7, 4, 15, 0.6, 0.3)])
def test_axis_angles(n, m, D, dt, t0):
    """theta = 0: the line x = t meets every row at x = t, interpolated between
    the two nearest pixel centres; theta = pi/2: y = t, every column."""
    W = oracle.Op(n, m, D, dt, t0, kernel=J).dense() * n        # pixel widths
    half = 0.5 * n
    for k in range(D):
        t = (k - 0.5 * (D - 1)) * dt + t0
        r0 = W[k].reshape(n, n)                                   # a = 0
        r90 = W[(m // 2) * D + k].reshape(n, n)                   # a = m/2: c = 0, s = 1
        for iy in range(n):
            for ix in range(n):
                assert r0[iy, ix] == pytest.approx(hat(t - (ix + 0.5 - half)), abs=1e-14)
                assert r90[iy, ix] == pytest.approx(hat(t - (iy + 0.5 - half)), abs=1e-14)


def test_hand_worked_example():
    """n = 3, one line at 30 degrees (c = sqrt(3)/2, s = 1/2), t = 1/4, worked
    by hand: rows y = -1, 0, 1 are crossed at x = (1/4 - y/2) / c, i.e. at
    x = sqrt(3)/2, 1/(2 sqrt 3), -1/(2 sqrt 3); each crossing is shared
    between the two nearest pixel centres (x = -1, 0, 1) in proportion to
    closeness, times the step 1/c = 2/sqrt(3)."""
    ang = np.array([np.pi / 6])
    op = oracle.Op(3, 1, 1, 1.0, 0.25, angles=ang, kernel=J)
    w = op.dense()[0].reshape(3, 3) * 3
    step = 2.0 / math.sqrt(3.0)
    a, b = math.sqrt(3.0) / 2.0, 1.0 / (2.0 * math.sqrt(3.0))
    want = np.zeros((3, 3))
    want[0, 1], want[0, 2] = (1 - a) * step, a * step              # row y = -1: x = a between 0 and 1
    want[1, 1], want[1, 2] = (1 - b) * step, b * step              # row y = 0: x = b between 0 and 1
    want[2, 0], want[2, 1] = b * step, (1 - b) * step              # row y = 1: x = -b between -1 and 0
    assert np.abs(w - want).max() < 1e-14


@pytest.mark.parametrize("theta", [0.3, 1.0, 2.2, 2.9])
def test_affine_images_are_exact(theta):
    """f = alpha + beta x + gamma y at the pixel centres: on every line whose
    crossings all lie between the first and last pixel centres of their rows
    (columns), W f = step * sum over rows (columns) of f at the crossing."""
    n, D = 20, 41
    ang = np.array([theta])
    op = oracle.Op(n, 1, D, 0.5, 0.0, angles=ang, kernel=J)
    half = 0.5 * n
    xs = np.arange(n) + 0.5 - half
    X, Y = np.meshgrid(xs, xs)
    al, be, ga = 0.7, -0.3, 0.45
    f = (al + be * X + ga * Y).reshape(-1)
    p = op.project(f) * n
    c, s = math.cos(theta), math.sin(theta)
    rows = abs(c) >= abs(s)
    step = 1.0 / max(abs(c), abs(s))
    checked = 0
    for k in range(D):
        t = (k - 0.5 * (D - 1)) * 0.5
        cross = [((t - u * s) / c, u) if rows else (u, (t - u * c) / s) for u in xs]
        inside = all(xs[0] <= (x if rows else y) <= xs[-1] for x, y in cross)
        if not inside:
            continue
        want = step * sum(al + be * x + ga * y for x, y in cross)
        assert p[k] == pytest.approx(want, rel=1e-12, abs=1e-12)
        checked += 1
    assert checked >= 5


@pytest.mark.parametrize("m", [7, 12])
def test_distance_form(m):
    """Every weight equals (1 - |d| / a) / a, a = max(|c|, |s|), d = t minus
    the pixel centre's projection on (c, s): the interpolation distance along
    the sampled axis is |d| / a."""
    n, D = 9, 15
    op = oracle.Op(n, m, D, 0.8, 0.1, kernel=J)
    W = op.dense() * n
    c, s = op.trig()
    half = 0.5 * n
    xs = np.arange(n) + 0.5 - half
    X, Y = np.meshgrid(xs, xs)
    for a in range(m):
        al = max(abs(c[a]), abs(s[a]))
        tau = (X * c[a] + Y * s[a]).reshape(-1)
        for k in range(D):
            t = (k - 0.5 * (D - 1)) * 0.8 + 0.1
            want = np.maximum(0.0, 1.0 - np.abs(t - tau) / al) / al
            assert np.abs(W[a * D + k] - want).max() < 1e-13


def test_45_degree_tie():
    """At |c| = |s| the oracle samples rows; sampling columns instead gives the
    same weights (both interpolation distances are |d| sqrt 2)."""
    n, m, D = 10, 4, 17                       # angle 1 is pi/4, angle 3 is 3 pi/4
    op = oracle.Op(n, m, D, kernel=J)
    W = op.dense() * n
    c, s = op.trig()
    half = 0.5 * n
    for a in (1, 3):
        step = 1.0 / abs(s[a])
        for k in range(D):
            t = k - 0.5 * (D - 1)
            alt = np.zeros((n, n))
            for ix in range(n):                # columns: crossing y of the column centre line
                x = ix + 0.5 - half
                q = (t - x * c[a]) / s[a] + half - 0.5
                i0 = math.floor(q)
                for i, w in ((i0, 1 - (q - i0)), (i0 + 1, q - i0)):
                    if 0 <= i < n and w > 0:
                        alt[i, ix] += w * step
            assert np.abs(W[a * D + k] - alt.reshape(-1)).max() < 1e-13


@pytest.mark.parametrize("n,m,D", [(12, 16, 19), (9, 10, 14)])
def test_rotation_and_mirror(n, m, D):
    """x'(p) = x(R^-1 p), R = +90 deg: (W x')[a, k] = (W x)[a - m/2, k] for
    a >= m/2, (W x)[a + m/2, D-1-k] otherwise; mirror in x: (W x'')[a, k] =
    (W x)[m - a, k] for a >= 1, (W x)[0, D-1-k] for a = 0."""
    op = oracle.Op(n, m, D, kernel=J)
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
    pm = op.project(x[:, ::-1].copy().reshape(-1)).reshape(m, D)
    assert np.abs(pm[1:] - p[:0:-1]).max() < 1e-12
    assert np.abs(pm[0] - p[0, ::-1]).max() < 1e-12


def test_ray_row_matches_assembled_rows():
    n, m, D = 13, 11, 20
    op = oracle.Op(n, m, D, 0.9, -0.2, kernel=J)
    rowptr, col, val = op.csr()
    for a, k in [(0, 3), (3, 10), (5, 19), (10, 0), (7, 7)]:
        i = a * D + k
        c, v = oracle.ray_row(n, m, D, a, k, 0.9, -0.2, kernel=J)
        assert np.array_equal(c, col[rowptr[i]:rowptr[i + 1]])
        assert np.array_equal(v, val[rowptr[i]:rowptr[i + 1]])


def test_wmg_on_joseph_operator_is_exact_with_one_level():
    """One WMG level is the exact normal-equation solve for any W, so
    preconditioned GMRES converges in one step on the Joseph operator too."""
    n, m, D = 8, 12, 13
    op = oracle.Op(n, m, D, kernel=J)
    b = op.project(np.random.default_rng(4).random(n * n))
    M = oracle.Wmg(op, 1, 0, 0, 1.0, 1e-3, oracle.CYCLE_ADDITIVE, 0)
    x, k, hist = oracle.gmres(op, b, 3, 3, 1e-12, 1e-3, M)
    assert k == 1 and hist[-1] < 1e-12
