"""Host logic of the request server: the first-fit range allocator that
places every admitted request's image and sinogram state in the pools
(paper_1310_0956_gb300/csrc/range_alloc.h), built with g++ into a small
driver and checked, operation by operation, against an independent model
(a list of free intervals) on seeded random admission / retirement
sequences."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1310_0956_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "range_alloc.h"
int main() {
    wmg::RangeAlloc a;
    char op;
    long long x, y;
    while (std::scanf(" %c", &op) == 1) {
        if (op == 'i') { std::scanf("%lld", &x); a.init(x); std::printf("%lld\n", (long long)a.cap); }
        else if (op == 'a') {
            std::scanf("%lld", &x);
            const long long off = a.alloc(x);
            std::printf("%lld %lld\n", off, (long long)a.used);
        }
        else if (op == 'r') { std::scanf("%lld %lld", &x, &y); a.release(x, y); std::printf("%lld %zu\n", (long long)a.used, a.free_.size()); }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("range_alloc")
    src, exe = d / "drv.cpp", d / "drv"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", HDR, str(src), "-o", str(exe)], check=True)
    return str(exe)


class Model:
    """Free intervals of 64-element units, lowest first; first fit."""

    def __init__(self, cap):
        self.cap = cap // 64 * 64
        self.free = [(0, self.cap)] if self.cap > 0 else []
        self.used = 0

    @staticmethod
    def round(n):
        return (n + 63) // 64 * 64

    def alloc(self, n):
        n = self.round(n)
        for i, (o, ln) in enumerate(self.free):
            if ln >= n:
                self.free[i:i + 1] = [(o + n, ln - n)] if ln > n else []
                self.used += n
                return o
        return -1

    def release(self, o, n):
        n = self.round(n)
        self.used -= n
        self.free.append((o, n))
        self.free.sort()
        merged = []
        for a, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((a, ln))
        self.free = merged


@pytest.mark.parametrize("seed", range(4))
def test_first_fit_against_model(driver, seed):
    rng = np.random.default_rng(1000 + seed)
    cap = int(rng.integers(4000, 40000))
    ops, model, live = [f"i {cap}"], Model(cap), []
    want = [str(model.cap)]
    for _ in range(400):
        if live and rng.random() < 0.45:
            o, n = live.pop(int(rng.integers(len(live))))
            model.release(o, n)
            ops.append(f"r {o} {n}")
            want.append(f"{model.used} {len(model.free)}")
        else:
            n = int(rng.integers(1, 3000))
            o = model.alloc(n)
            ops.append(f"a {n}")
            want.append(f"{o} {model.used}")
            if o >= 0:
                live.append((o, n))
    out = subprocess.run([driver], input="\n".join(ops) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    assert out[:len(want)] == want


def test_release_merges_neighbours_and_refuses_when_full(driver):
    ops = "i 1000\na 64\na 100\na 200\na 600\nr 64 100\nr 0 64\na 150\nr 192 200\na 400\n"
    out = subprocess.run([driver], input=ops, capture_output=True, text=True, check=True).stdout.split("\n")
    # cap 960; 64 -> 0, 100 -> 64 (128), 200 -> 192 (256), 600 -> -1 (512 left < 640)
    assert out[:5] == ["960", "0 64", "64 192", "192 448", "-1 448"]
    # releasing 64..192 then 0..64 leaves one free range [0, 192) and [448, 960)
    assert out[5:7] == ["320 2", "256 2"]
    # 150 -> 192 elements at offset 0 (first fit); releasing 192..448 merges with [448, 960)
    assert out[7:9] == ["0 448", "192 1"]
    assert out[9] == "192 640"
