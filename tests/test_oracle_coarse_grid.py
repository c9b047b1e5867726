"""The coarse (2h) grid form of a projection whose input lies in the LL band
of the first split (Section 2.3: the coarse grid of 2 x 2 pixel blocks, the
Haar intergrid operators of eq. intops; Section 3.1.3: the packet tree).

An image x = Q_LL e synthesised from the leaves of the first split's LL
subtree alone (the first K/4 leaves of the packet layout) is the
prolongation I_{2h}^h c of the n/2 x n/2 image c that the same leaf values
give through an (L-1)-level synthesis: x = c / 2 on every 2 x 2 block. With
exact intersection lengths, chords add over the four pixels of a block, so
W x = W^{2h} c / 2, W^{2h} the projection of the same scan on pixels of width
2h (detector offset and spacing halved in those units). The hybrid cycle's
band updates project such images on the 2h grid; these tests pin the
identity with the oracle's own operators only. Joseph's interpolation
weights do not add over blocks, so that kernel keeps the fine grid."""
import numpy as np
import pytest

import oracle


def prolong(c, nh):
    """x = c / 2 on every 2 x 2 block (I_{2h}^h of eq. intops in 2D)."""
    return 0.5 * np.kron(c.reshape(nh, nh), np.ones((2, 2))).reshape(-1)


@pytest.mark.parametrize("n,L", [(16, 1), (16, 2), (32, 3), (64, 4), (48, 2)])
def test_ll_leaves_synthesise_to_a_prolonged_coarse_image(n, L):
    rng = np.random.default_rng(n + L)
    N = n * n
    e = np.zeros(N)
    e[:N // 4] = rng.standard_normal(N // 4)
    x = oracle.packet_synthesis(e, n, L)
    c = oracle.packet_synthesis(e[:N // 4], n // 2, L - 1)
    assert np.abs(x - prolong(c, n // 2)).max() < 1e-14 * np.abs(x).max()
    # and a leaf outside the LL subtree changes x where no coarse image can
    e2 = e.copy()
    e2[N // 4] = 1.0
    x2 = oracle.packet_synthesis(e2, n, L)
    d = (x2 - x).reshape(n // 2, 2, n // 2, 2)
    assert np.abs(d - d.mean(axis=(1, 3), keepdims=True)).max() > 1e-3


@pytest.mark.parametrize("n,m,D,dt,t0", [
    (32, 24, 46, 1.0, 0.0),      # every multiple of pi/4 among the angles
    (32, 30, 47, 0.8, 0.3),      # spacing below a pixel, offset detector, odd D
    (64, 36, 92, 1.0, 0.0),
    (48, 20, 70, 1.0, -0.5),     # rays along pixel edges at the axis angles
])
def test_projection_of_a_prolonged_image_on_the_coarse_grid(n, m, D, dt, t0):
    rng = np.random.default_rng(n * m + D)
    nh = n // 2
    c = rng.standard_normal(nh * nh)
    fine = oracle.Op(n, m, D, dt=dt, t0=t0)
    coarse = oracle.Op(nh, m, D, dt=dt / 2, t0=t0 / 2)
    y = fine.project(prolong(c, nh))
    yc = 0.5 * coarse.project(c)
    assert np.abs(y - yc).max() < 1e-12 * np.abs(y).max()


def test_joseph_weights_do_not_add_over_blocks():
    n, m, D = 32, 24, 46
    rng = np.random.default_rng(5)
    c = rng.standard_normal((n // 2) ** 2)
    fine = oracle.Op(n, m, D, kernel=oracle.KERNEL_JOSEPH)
    coarse = oracle.Op(n // 2, m, D, dt=0.5, kernel=oracle.KERNEL_JOSEPH)
    y = fine.project(prolong(c, n // 2))
    yc = 0.5 * coarse.project(c)
    assert np.abs(y - yc).max() > 1e-3 * np.abs(y).max()


@pytest.mark.parametrize("n,m,D,L,lam", [(32, 24, 46, 2, 0.0), (32, 30, 47, 3, 0.7), (64, 36, 92, 4, 0.05)])
def test_band_update_in_its_2h_form(n, m, D, L, lam):
    """The hybrid step's band update at the root (Section 3.1.2): the
    residual of the three children after the LL correction loses
    Q_rest^T (W^T W + lambda) Q_LL E_LL. Its 2h form: synthesise c from the
    LL leaves through L - 1 levels, project on the 2h grid and halve,
    backproject on W's grid, analyse into the other leaves; no lambda term
    (Q_rest^T Q_LL = 0)."""
    rng = np.random.default_rng(n + L)
    N = n * n
    E = np.zeros(N)
    E[:N // 4] = rng.standard_normal(N // 4)
    fine = oracle.Op(n, m, D)
    coarse = oracle.Op(n // 2, m, D, dt=0.5)
    x = oracle.packet_synthesis(E, n, L)
    ref = oracle.packet_analysis(fine.backproject(fine.project(x)) + lam * x, n, L)[N // 4:]
    c = oracle.packet_synthesis(E[:N // 4], n // 2, L - 1)
    got = oracle.packet_analysis(fine.backproject(0.5 * coarse.project(c)), n, L)[N // 4:]
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
