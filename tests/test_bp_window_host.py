"""The sinogram window the FP32 backprojector's group tiles stage per angle
(paper_1310_0956_gb300/csrc/projector_f32.cu, bpg_window) holds every
candidate bin of every pixel of the tile, with a margin, on whole geometries
(every 32 x 32 tile, every equiangular angle), so the kernel's clamp of the
window index never binds. Pure arithmetic on the CPU:

* the window starts at floor(tau_min) + kofs - 2, tau_min the smallest of
  tau = x c + y s over the tile's corner pixel centres, evaluated in FP32 with
  c, s the sums of the split trigonometry (c_hi + c_lo, rounded), and the
  kernel reads window indices up to kBgW - 1 = 55;
* a pixel's candidates are the bins k0 = m0 + kofs and k0 + 1 with m0 the
  integer nearest tau - 1/2 (odd D) or tau (even D), kofs = (D - 1) / 2 or
  D / 2 - 1 (bins at t_k = k - (D - 1) / 2), computed from tau with FP32
  rounding: m0 lies within one of floor(tau) for any tau within 1e-3 of the
  exact value.
The exact tau of a tile's pixels spans [tau_min, tau_max] at its corners (tau
is linear); the check takes the extremes of m0 over tau +- 1e-3. On these
geometries the candidates' window indices span 1 .. 48 of 0 .. 55."""
import numpy as np
import pytest

KBGW = 56


def split_trig(m):
    """(c_hi + c_lo, s_hi + s_lo) in FP32, as the angle table builds them:
    c_hi = c rounded to a multiple of 2^-12, c_lo = c - c_hi rounded to FP32."""
    th = np.pi * np.arange(m) / m
    c, s = np.cos(th), np.sin(th)
    # exact values at the multiples of pi/4 (the table's octant reduction)
    for a in range(m):
        if (4 * a) % m == 0:
            q = (4 * a) // m
            c[a], s[a] = [(1.0, 0.0), (np.sqrt(0.5), np.sqrt(0.5)), (0.0, 1.0), (-np.sqrt(0.5), np.sqrt(0.5))][q]
    chi, shi = np.round(c * 4096.0) / 4096.0, np.round(s * 4096.0) / 4096.0
    cf = (np.float32(chi) + np.float32(c - chi)).astype(np.float32)
    sf = (np.float32(shi) + np.float32(s - shi)).astype(np.float32)
    return c, s, cf, sf


def fma32(a, b, c):
    """FP32 fused multiply-add, through FP64 (products of two FP32 values are
    exact in FP64)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


@pytest.mark.parametrize("n,m,D", [(256, 180, 363), (64, 36, 92), (32, 24, 48), (512, 360, 725),
                                   (1024, 1024, 1449), (160, 400, 227)])
def test_window_holds_every_candidate(n, m, D):
    c, s, cf, sf = split_trig(m)
    half = 0.5 * n
    odd = D % 2 == 1
    kofs = (D - 1) // 2 if odd else D // 2 - 1
    t0 = np.arange(0, n, 32, dtype=np.float64)
    xa, ya = np.meshgrid(t0 + 0.5 - half, t0 + 0.5 - half, indexing="ij")
    xa, ya = xa.reshape(-1, 1), ya.reshape(-1, 1)                 # tiles x 1
    # the kernel's window start, in FP32
    x32, y32 = xa.astype(np.float32), ya.astype(np.float32)
    cs = cf.reshape(1, -1)
    ss = sf.reshape(1, -1)
    corners = []
    for dx in (0.0, 31.0):
        for dy in (0.0, 31.0):
            ys = ((y32 + np.float32(dy)) * ss).astype(np.float32)
            corners.append(fma32(x32 + np.float32(dx), cs, ys))
    tmin32 = np.minimum.reduce(corners)
    kwin = np.floor(tmin32).astype(np.int64) + kofs - 2
    # exact tau range of the tile's pixels, then the candidates' extremes
    ce, se = c.reshape(1, -1), s.reshape(1, -1)
    ex = [(xa + dx) * ce + (ya + dy) * se for dx in (0.0, 31.0) for dy in (0.0, 31.0)]
    tmin, tmax = np.minimum.reduce(ex) - 1e-3, np.maximum.reduce(ex) + 1e-3
    off = 0.5 if odd else 0.0
    m0_lo = np.rint(tmin - off).astype(np.int64)
    m0_hi = np.rint(tmax - off).astype(np.int64)
    lo = m0_lo + kofs - kwin                                     # first candidate's window index
    hi = m0_hi + kofs + 1 - kwin                                 # second candidate's
    assert lo.min() >= 1, lo.min()
    assert hi.max() <= KBGW - 3, hi.max()
