"""Host logic of the WMG cycle's band-local residual updates
(paper_1310_0956_gb300/csrc/band_grid.h), built with g++ into a small driver
and checked for every update a cycle can issue (every node q at every depth
d < L, every mode) against the oracle's own packet transforms:

* the leaf ranges: mode 0 reads the node's LL child and writes its three
  other children, mode 1 reads the whole node and writes its LL child, modes
  2 and 3 read child 1 or 2 and write the children after it (Section 3.1.2);
  the node's leaves are those the oracle's depth-d analysis of an image made
  from them alone puts in band q;
* the 2h grid is taken exactly when the input leaves synthesise (oracle, L
  levels) to an image constant on every 2 x 2 block (I_{2h}^h c, Section 2.3)
  and the oracle's analysis of that image has nothing on the output leaves
  (the lambda term Q_out^T Q_in E is zero); never for a geometry without a
  2h grid."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1310_0956_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "band_grid.h"
int main() {
    int L, d, q, mode, has;
    while (std::scanf("%d %d %d %d %d", &L, &d, &q, &mode, &has) == 5) {
        int a, b, c, e;
        wmg::band_leaf_ranges(L, d, q, mode, a, b, c, e);
        std::printf("%d %d %d %d %d %d %d\n", a, b, c, e, (int)wmg::band_on_2h(has != 0, 1 << (2 * L), a, b, c, e),
                    wmg::node_lo(L, d, q), wmg::node_hi(L, d, q));
    }
    return 0;
}
"""

CASES = [(8, 2), (16, 3)]      # n, L (leaf side 2)


@pytest.fixture(scope="module")
def updates(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    dd = tmp_path_factory.mktemp("band_grid")
    src, exe = dd / "drv.cpp", dd / "drv"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", HDR, str(src), "-o", str(exe)], check=True)
    keys = [(n, L, d, q, mode, has) for n, L in CASES for d in range(L) for q in range(4 ** d)
            for mode in range(4) for has in (1, 0)]
    inp = "".join(f"{L} {d} {q} {mode} {has}\n" for _, L, d, q, mode, has in keys)
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    return {k: tuple(int(v) for v in line.split()) for k, line in zip(keys, out)}


def image_from(k0, k1, n, L, rng):
    """Synthesis (L levels) of random values on leaves k0 .. k1 - 1 (leaf k:
    coefficients k P .. (k + 1) P - 1, P = (n / 2^L)^2)."""
    P = (n >> L) ** 2
    c = np.zeros(n * n)
    c[k0 * P:k1 * P] = rng.standard_normal((k1 - k0) * P)
    return oracle.packet_synthesis(c, n, L)


def test_node_leaves_are_the_oracle_band(updates):
    rng = np.random.default_rng(1)
    for (n, L, d, q, mode, has), (_, _, _, _, _, lo, hi) in updates.items():
        if mode or not has:
            continue
        x = image_from(lo, hi, n, L, rng)
        bands = oracle.packet_analysis(x, n, d).reshape(4 ** d, -1)    # depth-d bands, band order = path
        norms = np.linalg.norm(bands, axis=1)
        assert norms[q] > 0 and np.all(np.delete(norms, q) < 1e-12 * norms[q]), (n, L, d, q)


def test_modes_read_and_write_the_children_they_name(updates):
    for (n, L, d, q, mode, has), (a, b, c, e, _, lo, hi) in updates.items():
        step = (hi - lo) // 4                                   # leaves of one child
        kids = [(lo + i * step, lo + (i + 1) * step) for i in range(4)]
        if mode == 0:
            assert (a, b) == kids[0] and (c, e) == (kids[1][0], hi)
        elif mode == 1:
            assert (a, b) == (lo, hi) and (c, e) == kids[0]
        else:
            assert (a, b) == kids[mode - 1] and (c, e) == (kids[mode][0], hi)


def test_2h_grid_exactly_when_the_input_is_block_constant_and_the_lambda_term_vanishes(updates):
    rng = np.random.default_rng(2)
    taken = 0
    for (n, L, d, q, mode, has), (a, b, c, e, on2h, _, _) in updates.items():
        if not has:
            assert on2h == 0
            continue
        x = image_from(a, b, n, L, rng)
        blocks = x.reshape(n // 2, 2, n // 2, 2)
        constant = np.abs(blocks - blocks.mean(axis=(1, 3), keepdims=True)).max() < 1e-12 * np.abs(x).max()
        P = (n >> L) ** 2
        out = oracle.packet_analysis(x, n, L)[c * P:e * P]
        lam_zero = np.abs(out).max() < 1e-12 * np.abs(x).max()
        assert on2h == int(constant and lam_zero), (n, L, d, q, mode)
        taken += on2h
    assert taken > 0
