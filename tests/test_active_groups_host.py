"""Host logic of the work lists a batched solve restricts itself to once few
problems are left (paper_1310_0956_gb300/csrc/active_groups.h), built with
g++ into a small driver and checked on seeded random plans (runs of
same-geometry slots, empty slots, problems still going or stopped) against an
independent model of the rule and of the FP32 projector's grouping: every
going problem keeps its tiles; a projector group of the plan's own lists
stays whole exactly when at least `keep` of its members are going; the
restricted lists, cut into runs and groups the way the work-list builder
does, form exactly the kept groups and single problems otherwise (so a
problem's group tiles, where it has any, are those of the full lists)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1310_0956_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "active_groups.h"
int main() {
    int np, groups, group, keep;
    while (std::scanf("%d %d %d %d", &np, &groups, &group, &keep) == 4) {
        std::vector<int> geom(np);
        std::vector<char> go(np);
        for (int q = 0; q < np; ++q) std::scanf("%d", &geom[q]);
        for (int q = 0; q < np; ++q) { int v; std::scanf("%d", &v); go[q] = (char)v; }
        std::vector<char> present, brk;
        wmg::active_groups(geom, go, groups != 0, group, keep, present, brk);
        for (int q = 0; q < np; ++q) std::printf("%d%c", (int)present[q], q + 1 < np ? ' ' : '\n');
        for (int q = 0; q < np; ++q) std::printf("%d%c", (int)brk[q], q + 1 < np ? ' ' : '\n');
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("active_groups")
    src, exe = d / "drv.cpp", d / "drv"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", HDR, str(src), "-o", str(exe)], check=True)
    return str(exe)


def groups_of(geom, present, brk, group):
    """The work-list builder's grouping: runs of consecutive present slots of
    one geometry (a run also starts where brk is set), cut into groups of
    `group` from the run's start; returns (groups as first slots, singles)."""
    n = len(geom)
    firsts, singles = [], []
    q = 0
    while q < n:
        if not present[q]:
            q += 1
            continue
        e = q + 1
        while e < n and present[e] and geom[e] == geom[q] and not brk[e]:
            e += 1
        f = q
        while f + group <= e:
            firsts.append(f)
            f += group
        singles.extend(range(f, e))
        q = e
    return firsts, singles


def case(rng):
    n = int(rng.integers(1, 80))
    geom, g = [], 0
    while len(geom) < n:                        # runs of one geometry, a few empty slots
        run = int(rng.integers(1, 30))
        gid = -1 if rng.random() < 0.1 else g
        geom += [gid] * run
        g += 1
    geom = geom[:n]
    p_go = rng.random()
    go = [int(geom[q] >= 0 and rng.random() < p_go) for q in range(n)]
    return geom, go


def run_driver(driver, cases, groups, group, keep):
    lines = []
    for geom, go in cases:
        lines.append(f"{len(geom)} {int(groups)} {group} {keep}")
        lines.append(" ".join(map(str, geom)))
        lines.append(" ".join(map(str, go)))
    out = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    res = []
    for i in range(len(cases)):
        res.append(([int(v) for v in out[2 * i].split()], [int(v) for v in out[2 * i + 1].split()]))
    return res


@pytest.mark.parametrize("group,keep", [(8, 3), (4, 2), (8, 1)])
def test_restricted_lists_keep_the_own_groups(driver, group, keep):
    rng = np.random.default_rng(1000 + 10 * group + keep)
    cases = [case(rng) for _ in range(300)]
    for (geom, go), (present, brk) in zip(cases, run_driver(driver, cases, True, group, keep)):
        own_groups, _ = groups_of(geom, [int(g >= 0) for g in geom], [0] * len(geom), group)
        kept = [f for f in own_groups if sum(go[f:f + group]) >= keep]
        in_kept = set(q for f in kept for q in range(f, f + group))
        for q in range(len(geom)):
            assert present[q] == int(go[q] == 1 or q in in_kept), (geom, go, q)
        firsts, singles = groups_of(geom, present, brk, group)
        assert firsts == kept
        assert sorted(singles) == [q for q in range(len(geom)) if present[q] and q not in in_kept]


def test_without_groups_exactly_the_going_problems(driver):
    rng = np.random.default_rng(7)
    cases = [case(rng) for _ in range(200)]
    for (geom, go), (present, brk) in zip(cases, run_driver(driver, cases, False, 8, 3)):
        assert present == go
        firsts, singles = groups_of(geom, present, brk, 8)
        assert firsts == [] and singles == [q for q in range(len(geom)) if go[q]]
