// band_grid.h -- the leaf ranges of a band-local residual update of the WMG
// cycle (Section 3.1.2) and whether its product runs on the 2h grid. Plain
// C++ (no CUDA), so that it also builds into host-only tests.
#pragma once

namespace wmg {

// A tree node at depth d is named by its path prefix q in [0, 4^d); with L
// levels it owns the leaves [q 4^(L-d), (q+1) 4^(L-d)). The LL child of q is
// 4q, the other children 4q+1 .. 4q+3.
inline int node_lo(int L, int d, int q) { return q << (2 * (L - d)); }
inline int node_hi(int L, int d, int q) { return (q + 1) << (2 * (L - d)); }

// Leaves read ([kin0, kin1): the correction) and written ([kout0, kout1):
// the residual) by the band update of node q at depth d. mode 0: the LL
// child in, the three other children out (the hybrid step, and the
// multiplicative cycle's first); 1: the whole node in, its LL child out (the
// symmetric closing step); 2, 3: child 1 (LH) or 2 (HL) in, the children
// after it out (the multiplicative cycle's later steps).
inline void band_leaf_ranges(int L, int d, int q, int mode, int &kin0, int &kin1, int &kout0, int &kout1)
{
    const int lo = node_lo(L, d, q), hi = node_hi(L, d, q);
    const int ll_hi = node_hi(L, d + 1, 4 * q);
    if (mode == 1) {
        kin0 = lo; kin1 = hi; kout0 = lo; kout1 = ll_hi;
    } else if (mode == 0) {
        kin0 = lo; kin1 = ll_hi; kout0 = ll_hi; kout1 = hi;
    } else {
        kin0 = node_lo(L, d + 1, 4 * q + mode - 1); kin1 = node_hi(L, d + 1, 4 * q + mode - 1);
        kout0 = kin1; kout1 = hi;
    }
}

// The update's synthesis and projection run on the 2h grid when its input
// leaves lie in the LL band of the first split (below K/4 of the K = 4^L
// leaves: the synthesised image is I_{2h}^h c, constant on 2 x 2 blocks) of
// a geometry that has a 2h grid, and its output leaves are disjoint from
// them (so that its lambda term, lambda Q_out^T Q_in E, is zero).
inline bool band_on_2h(bool has_2h, int K, int kin0, int kin1, int kout0, int kout1)
{
    return has_2h && kin1 <= K / 4 && (kout0 >= kin1 || kout1 <= kin0);
}

}  // namespace wmg
