// bp_epilogue.cuh -- fused epilogues of the backprojection kernels: what a
// pixel's value y = (W^T r)_j turns into (Krylov vector updates, residuals,
// smoothing sweeps), with the operator-precision copies the next projection
// reads. Returns the pixel's contribution to the tile's partial dot product.
#pragma once

#include "kern_common.cuh"

namespace wmg {

// T: the plan's operator type (tables); TS: the storage of the operator
// copies and outputs written here and of v_op (T, or bfloat16 for plans with
// BF16 operator storage).
template <class T, int EPI, class TS = T>
__device__ __forceinline__ double bp_epilogue(const GeomDev &g, const ProbDev &pd,
                                              const BpArgs &a, int ix, int iy, double y)
{
    const int n = g.n;
    const int64_t j = pd.img + (int64_t)iy * n + ix;
    const int64_t jt = pd.img + (int64_t)ix * n + iy;
    const double lam = g.lambda;
    const double *S = a.S + (int64_t)pd.slot * NSCAL;
    const T *dinv = static_cast<const T *>(g.dinv) + (j - pd.img);
    double contrib = 0.0;
    if (EPI == BP_STORE) {
        st_op(static_cast<TS *>(a.out_op) + j, y);
    } else if (EPI == BP_CGLS_S) {
        const double xv = a.x[j] + S[SC_ALPHA] * a.p[j];
        a.x[j] = xv;
        const double sv = y - lam * xv;
        a.s[j] = sv;
        contrib = sv * sv;
        if (a.z) {                        // first pre-smoothing sweep from z = 0
            const double zv = g.omega * (double)dinv[0] * sv;
            a.z[j] = zv;
            st_op(static_cast<TS *>(a.copy_op) + j, zv);
            st_op(static_cast<TS *>(a.copyT_op) + jt, zv);
        }
    } else if (EPI == BP_RESID) {
        a.out64[j] = a.s[j] - y - lam * a.z[j];
    } else if (EPI == BP_POST) {
        const double zv = a.z[j] + g.omega * (double)dinv[0] * (a.s[j] - y - lam * a.z[j]);
        a.z[j] = zv;
        contrib = a.s[j] * zv;
        if (a.copy_op) {
            st_op(static_cast<TS *>(a.copy_op) + j, zv);
            st_op(static_cast<TS *>(a.copyT_op) + jt, zv);
        }
    } else if (EPI == BP_APPLY_A) {
        const double v = (double)ld_op(static_cast<const TS *>(a.v_op) + j);
        if (a.out64) a.out64[j] = y + lam * v;
        else st_op(static_cast<TS *>(a.out_op) + j, y + lam * v);
    } else if (EPI == BP_SIRT) {
        const T *C = static_cast<const T *>(g.sirtC) + (j - pd.img);
        const double xv = a.x[j] + (double)C[0] * (y - lam * a.x[j]);
        a.x[j] = xv;
        st_op(static_cast<TS *>(a.copy_op) + j, xv);
        st_op(static_cast<TS *>(a.copyT_op) + jt, xv);
    } else if (EPI == BP_GMRES_W) {
        const double wv = y + lam * a.z[j];
        a.out64[j] = wv;
    } else if (EPI == BP_ATB) {
        a.out64[j] = y;
        contrib = y * y;
    }
    return contrib;
}

}  // namespace wmg
