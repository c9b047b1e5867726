// bp_epilogue.cuh -- fused epilogues of the backprojection kernels: what a
// pixel's value y = (W^T r)_j turns into (Krylov vector updates, residuals,
// smoothing sweeps), with the operator-precision copies the next projection
// reads. Returns the pixel's contribution to the tile's partial dot product.
#pragma once

#include "kern_common.cuh"

namespace wmg {

template <class T, int EPI>
__device__ __forceinline__ double bp_epilogue(const GeomDev &g, const ProbDev &pd,
                                              const BpArgs &a, int ix, int iy, double y)
{
    const int n = g.n;
    const int64_t j = pd.img + (int64_t)iy * n + ix;
    const int64_t jt = pd.img + (int64_t)ix * n + iy;
    const T yT = (T)y;
    const double lam = g.lambda;
    const double *S = a.S + (int64_t)pd.slot * NSCAL;
    const T *dinv = static_cast<const T *>(g.dinv) + (j - pd.img);
    double contrib = 0.0;
    if (EPI == BP_STORE) {
        static_cast<T *>(a.out_op)[j] = yT;
    } else if (EPI == BP_CGLS_S) {
        const double xv = a.x[j] + S[SC_ALPHA] * a.p[j];
        a.x[j] = xv;
        const double sv = y - lam * xv;
        a.s[j] = sv;
        contrib = sv * sv;
        if (a.z) {                        // first pre-smoothing sweep from z = 0
            const double zv = g.omega * (double)dinv[0] * sv;
            a.z[j] = zv;
            static_cast<T *>(a.copy_op)[j] = (T)zv;
            static_cast<T *>(a.copyT_op)[jt] = (T)zv;
        }
    } else if (EPI == BP_RESID) {
        a.out64[j] = a.s[j] - y - lam * a.z[j];
    } else if (EPI == BP_POST) {
        const double zv = a.z[j] + g.omega * (double)dinv[0] * (a.s[j] - y - lam * a.z[j]);
        a.z[j] = zv;
        contrib = a.s[j] * zv;
        if (a.copy_op) {
            static_cast<T *>(a.copy_op)[j] = (T)zv;
            static_cast<T *>(a.copyT_op)[jt] = (T)zv;
        }
    } else if (EPI == BP_APPLY_A) {
        const double v = (double)static_cast<const T *>(a.v_op)[j];
        if (a.out64) a.out64[j] = y + lam * v;
        else static_cast<T *>(a.out_op)[j] = (T)(y + lam * v);
    } else if (EPI == BP_SIRT) {
        const T *C = static_cast<const T *>(g.sirtC) + (j - pd.img);
        const double xv = a.x[j] + (double)C[0] * (y - lam * a.x[j]);
        a.x[j] = xv;
        static_cast<T *>(a.copy_op)[j] = (T)xv;
        static_cast<T *>(a.copyT_op)[jt] = (T)xv;
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
