// active_groups.h -- the problems a batched solve's restricted work lists
// keep once few problems are left, and where their same-geometry runs
// start. Plain C++ (no CUDA), so that it also builds into host-only tests.
#pragma once

#include <vector>

namespace wmg {

// geom[q]: geometry of slot q in the plan's own work lists (< 0: no problem);
// go[q] != 0: the problem is still iterating. `groups`: the plan's FP32
// projector cuts every run of consecutive same-geometry problems into groups
// of `group` from the run's start (the rest run alone). A group stays whole
// (all its members present; the stopped ones are masked in the kernels, as in
// the full lists) while at least `keep` of its members are going; otherwise
// only its going members are present, each as a run of its own. Without
// groups exactly the going problems are present.
// Out: present[q] != 0 for the slots that keep their tiles; brk[q] != 0
// where a run starts although q - 1 is present with the same geometry (every
// kept group and every single problem is a run of its own, so the restricted
// lists form the same groups as the plan's own ones).
inline void active_groups(const std::vector<int> &geom, const std::vector<char> &go, bool groups, int group,
                          int keep, std::vector<char> &present, std::vector<char> &brk)
{
    const int np = (int)geom.size();
    present.assign(np, 0);
    brk.assign(np, 0);
    for (int q = 0; q < np;) {
        if (geom[q] < 0) { ++q; continue; }
        int e = q + 1;
        while (e < np && geom[e] == geom[q]) ++e;
        int f = q;
        for (; groups && f + group <= e; f += group) {
            int k = 0;
            for (int b = 0; b < group; ++b) k += go[f + b] ? 1 : 0;
            if (k >= keep) {
                for (int b = 0; b < group; ++b) present[f + b] = 1;
                brk[f] = 1;
            } else {
                for (int b = 0; b < group; ++b)
                    if (go[f + b]) present[f + b] = brk[f + b] = 1;
            }
        }
        for (; f < e; ++f)
            if (go[f]) present[f] = brk[f] = 1;
        q = e;
    }
}

}  // namespace wmg
