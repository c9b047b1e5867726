// krylov.cu -- vector updates and deterministic reductions of the Krylov
// solvers on the normal equations (Section 2.3.1): CGLS / PCG, restarted
// GMRES with right preconditioning, and the SIRT iteration (eq. sirt_it).
//
// Krylov vectors and scalars are FP64. Each vector kernel writes one partial
// sum per tile; a finalize kernel (one CTA per problem) adds a problem's
// partials in tile order and updates that problem's scalars, so every
// reduction has the same fixed summation order on every run and whatever the
// batch it runs in.
#include "kern_common.cuh"
#include "krylov.cuh"

namespace wmg {

// ---------------------------------------------------------------------------
// Image kernels over 32 x 32 tiles (backprojection tile list)
// ---------------------------------------------------------------------------
template <class T, int OP>
__global__ void __launch_bounds__(256)
k_img(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P, const int4 *__restrict__ tiles,
      int ntiles, ImgArgs a)
{
    __shared__ T tr[32][33];
    __shared__ double red[8];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(a.S, pd.slot)) continue;
        const GeomDev &g = G[pd.geom];
        const int n = g.n;
        const double *S = a.S ? a.S + (int64_t)pd.slot * NSCAL : nullptr;
        double part = 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int iy = tl.y + ty + 8 * r, ix = tl.z + tx;
            T cp = T(0);
            if (iy < n && ix < n) {
                const int64_t j = pd.img + (int64_t)iy * n + ix;
                double v = 0.0;
                if (OP == IMG_PUPDATE) {            // p = z + beta p
                    v = a.z[j] + S[SC_BETA] * a.p[j];
                    a.p[j] = v;
                    part += v * v;
                } else if (OP == IMG_PINIT) {       // p = z
                    v = a.z[j];
                    a.p[j] = v;
                    part += v * v;
                } else if (OP == IMG_FIRST_SWEEP) { // z = omega D~^-1 s
                    v = g.omega * (double)static_cast<const T *>(g.dinv)[j - pd.img] * a.s[j];
                    a.z[j] = v;
                } else if (OP == IMG_ZERO_RESID) {  // z = 0, r1 = s (operator copy)
                    a.z[j] = 0.0;
                    static_cast<double *>(a.r1)[j] = a.s[j];
                } else if (OP == IMG_LOAD) {        // v64 = (double) in_op ; copies
                    v = (double)static_cast<const T *>(a.in_op)[j];
                    a.z[j] = v;
                } else if (OP == IMG_COPY64) {      // copies of z
                    v = a.z[j];
                } else if (OP == IMG_STORE_OUT) {   // out_op = (T) z
                    static_cast<T *>(a.out_op)[j] = (T)a.z[j];
                } else if (OP == IMG_DOT_SZ) {      // part = s.z
                    part += a.s[j] * a.z[j];
                }
                // bfloat16 copies: one rounding from FP64; the tile keeps
                // the rounded value exactly for the transposed copy
                cp = a.bf16 ? (T)__bfloat162float(__double2bfloat16(v)) : (T)v;
                if (a.copy_op) {
                    if (a.bf16) static_cast<__nv_bfloat16 *>(a.copy_op)[j] = __float2bfloat16_rn((float)cp);
                    else static_cast<T *>(a.copy_op)[j] = cp;
                }
            }
            tr[ty + 8 * r][tx] = cp;
        }
        if (a.copyT_op) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int ox = tl.z + ty + 8 * r, oy = tl.y + tx;
                if (ox < n && oy < n) {
                    const int64_t o = pd.img + (int64_t)ox * n + oy;
                    if (a.bf16) static_cast<__nv_bfloat16 *>(a.copyT_op)[o] = __float2bfloat16_rn((float)tr[tx][ty + 8 * r]);
                    else static_cast<T *>(a.copyT_op)[o] = tr[tx][ty + 8 * r];
                }
            }
        }
        if (a.part) {
            const double tot = block_sum_fixed(part, red);
            if (threadIdx.x == 0) a.part[t] = tot;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 1D chunk kernels: tile = {prob, first element, count, kind} over image
// (kind 0) or sinogram (kind 1) vectors.
// ---------------------------------------------------------------------------
template <class T, int OP>
__global__ void __launch_bounds__(256)
k_vec(const ProbDev *__restrict__ P, const int4 *__restrict__ tiles, int ntiles, VecArgs a)
{
    __shared__ double red[8];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(a.S, pd.slot)) continue;
        const double *S = a.S ? a.S + (int64_t)pd.slot * NSCAL : nullptr;
        const int64_t base = (OP == VEC_R_UPDATE || OP == VEC_R_INIT || OP == VEC_SIRT_R ||
                              OP == VEC_SINO_DIFF) ? pd.sino : pd.img;
        double part = 0.0;
        for (int e = threadIdx.x; e < tl.z; e += blockDim.x) {
            const int64_t j = base + tl.y + e;
            if (OP == VEC_R_UPDATE) {           // r -= alpha q ; operator copy
                const double v = a.r[j] - S[SC_ALPHA] * (double)static_cast<const T *>(a.q)[j];
                a.r[j] = v;
                static_cast<T *>(a.r_op)[j] = (T)v;
            } else if (OP == VEC_R_INIT) {      // r = b ; operator copy
                const T bv = static_cast<const T *>(a.b_op)[j];
                a.r[j] = (double)bv;
                static_cast<T *>(a.r_op)[j] = bv;
            } else if (OP == VEC_SIRT_R) {      // r_op = R (b - q)
                const GeomDev *gg = a.G + pd.geom;
                const T *R = static_cast<const T *>(gg->sirtR) + (j - pd.sino);
                const double v = (double)R[0] * ((double)static_cast<const T *>(a.b_op)[j] -
                                                 (double)static_cast<const T *>(a.q)[j]);
                static_cast<T *>(a.r_op)[j] = (T)v;
            } else if (OP == VEC_NRM2) {        // part = sum w^2
                part += a.w[j] * a.w[j];
            } else if (OP == VEC_SCALE_V) {     // v = w * S[SC_HNORM]^-1 -> Vnext
                a.v[j] = a.w[j] / S[SC_HNORM];
            } else if (OP == VEC_X_ADD) {       // x += z
                a.x[j] += a.w[j];
            } else if (OP == VEC_RESID64) {     // v = f - w (true residual), part = |v|^2
                const double v = a.f[j] - a.w[j];
                a.v[j] = v;
                part += v * v;
            } else if (OP == VEC_TO_OP) {       // out_op = (T) w
                static_cast<T *>(a.r_op)[j] = (T)a.w[j];
            } else if (OP == VEC_SINO_DIFF) {   // r_op = b - q
                static_cast<T *>(a.r_op)[j] = (T)((double)static_cast<const T *>(a.b_op)[j] -
                                                  (double)static_cast<const T *>(a.q)[j]);
            } else if (OP == VEC_NE_RES) {      // part = |w - lambda x|^2
                const double v = a.w[j] - a.G[pd.geom].lambda * a.x[j];
                part += v * v;
            }
        }
        if (a.part) {
            const double tot = block_sum_fixed(part, red);
            if (threadIdx.x == 0) a.part[t] = tot;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// BiCGStab vector steps (right preconditioning; van der Vorst 1992), one
// image chunk per tile, FP64, per-tile partial dot products.
// ---------------------------------------------------------------------------
template <int OP>
__global__ void __launch_bounds__(256)
k_bicg(const ProbDev *__restrict__ P, const int4 *__restrict__ tiles, int ntiles, BicgArgs a)
{
    __shared__ double red[8];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(a.S, pd.slot)) continue;
        const double *S = a.S + (int64_t)pd.slot * NSCAL;
        const double alpha = S[SC_ALPHA], omega = S[SC_DELTA], beta = S[SC_BETA];
        double pa = 0.0, pb = 0.0;
        for (int e = threadIdx.x; e < tl.z; e += blockDim.x) {
            const int64_t j = pd.img + tl.y + e;
            if (OP == BI_INIT) {
                a.rh[j] = a.r[j];
                a.p[j] = 0.0;
                a.v[j] = 0.0;
            } else if (OP == BI_P) {
                a.p[j] = a.r[j] + beta * (a.p[j] - omega * a.v[j]);
            } else if (OP == BI_RV) {
                pa += a.rh[j] * a.v[j];
            } else if (OP == BI_S) {
                a.s[j] = a.r[j] - alpha * a.v[j];
            } else if (OP == BI_TS) {
                pa += a.t[j] * a.s[j];
                pb += a.t[j] * a.t[j];
            } else if (OP == BI_XR) {
                a.x[j] += alpha * a.ph[j] + omega * a.sh[j];
                const double rv = a.s[j] - omega * a.t[j];
                a.r[j] = rv;
                pa += rv * rv;
                pb += a.rh[j] * rv;
            }
        }
        if (OP == BI_RV || OP == BI_TS || OP == BI_XR) {
            const double ta = block_sum_fixed(pa, red);
            if (threadIdx.x == 0) a.part_a[t] = ta;
            __syncthreads();
            if (OP != BI_RV) {
                const double tb = block_sum_fixed(pb, red);
                if (threadIdx.x == 0) a.part_b[t] = tb;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// GMRES: classical Gram-Schmidt passes over the basis V (restart+1 vectors of
// N per problem, stride `vstride` elements between basis vectors). The column
// index j is one for all problems, or, when `jv` is given, jv[slot] per
// problem (problems at different Arnoldi steps in one launch).
// ---------------------------------------------------------------------------
// Partial dots part[t * ldp + i] = <V_i, w> over the tile, i <= j; with
// `wnorm`, also part[t * ldp + j + 1] = <w, w>. Slots with skip[slot] set
// (the second pass skipped) get zero partials and read nothing.
__global__ void __launch_bounds__(256)
k_gm_dots(const ProbDev *__restrict__ P, const int4 *__restrict__ tiles, int ntiles,
          const double *__restrict__ V, int64_t vstride, const double *__restrict__ w, int j0,
          const int *__restrict__ jv, int ldp, double *__restrict__ part, const double *__restrict__ S,
          int wnorm, const int *__restrict__ skip)
{
    __shared__ double red[8];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(S, pd.slot)) continue;
        const int j = jv ? jv[pd.slot] : j0;
        if (skip && skip[pd.slot]) {                                  // CTA-uniform
            for (int i = threadIdx.x; i <= j; i += blockDim.x) part[(int64_t)t * ldp + i] = 0.0;
            continue;
        }
        if (wnorm) {
            double acc = 0.0;
            for (int e = threadIdx.x; e < tl.z; e += blockDim.x) {
                const double v = w[pd.img + tl.y + e];
                acc += v * v;
            }
            const double tot = block_sum_fixed(acc, red);
            if (threadIdx.x == 0) part[(int64_t)t * ldp + j + 1] = tot;
            __syncthreads();
        }
        for (int i = 0; i <= j; ++i) {
            const double *Vi = V + (int64_t)i * vstride + pd.img;
            double acc = 0.0;
            for (int e = threadIdx.x; e < tl.z; e += blockDim.x) {
                const int64_t o = tl.y + e;
                acc += Vi[o] * w[pd.img + o];
            }
            const double tot = block_sum_fixed(acc, red);
            if (threadIdx.x == 0) part[(int64_t)t * ldp + i] = tot;
            __syncthreads();
        }
    }
}

// w -= sum_i h_i V_i (h from Hc[slot*ldp + i]); part = |w|^2 after the update.
// Slots with skip[slot] set are left alone (w and their partials).
__global__ void __launch_bounds__(256)
k_gm_axpy(const ProbDev *__restrict__ P, const int4 *__restrict__ tiles, int ntiles,
          const double *__restrict__ V, int64_t vstride, double *__restrict__ w, int j0,
          const int *__restrict__ jv, int ldp, const double *__restrict__ Hc, double *__restrict__ part,
          const double *__restrict__ S, const int *__restrict__ skip)
{
    __shared__ double red[8];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(S, pd.slot)) continue;
        if (skip && skip[pd.slot]) continue;                          // CTA-uniform
        const int j = jv ? jv[pd.slot] : j0;
        const double *h = Hc + (int64_t)pd.slot * ldp;
        const double *Vb = V + pd.img;
        double acc = 0.0;
        for (int e = threadIdx.x; e < tl.z; e += blockDim.x) {
            const int64_t o = tl.y + e;
            double v = w[pd.img + o];
            for (int i = 0; i <= j; ++i) v -= h[i] * Vb[(int64_t)i * vstride + o];
            w[pd.img + o] = v;
            acc += v * v;
        }
        if (part) {
            const double tot = block_sum_fixed(acc, red);
            if (threadIdx.x == 0) part[t] = tot;
        }
        __syncthreads();
    }
}

// out = sum_i y_i V_i (cycle end); y from Yv[slot*ldp + i], i < jn[slot].
__global__ void __launch_bounds__(256)
k_gm_combine(const ProbDev *__restrict__ P, const int4 *__restrict__ tiles, int ntiles,
             const double *__restrict__ V, int64_t vstride, int ldp, const double *__restrict__ Yv,
             const int *__restrict__ jn, double *__restrict__ out, const double *__restrict__ S)
{
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(S, pd.slot)) continue;
        const double *y = Yv + (int64_t)pd.slot * ldp;
        const double *Vb = V + pd.img;
        const int jj = jn[pd.slot];
        for (int e = threadIdx.x; e < tl.z; e += blockDim.x) {
            const int64_t o = tl.y + e;
            double v = 0.0;
            for (int i = 0; i < jj; ++i) v += y[i] * Vb[(int64_t)i * vstride + o];
            out[pd.img + o] = v;
        }
    }
}

// v_j = w / S[HNORM], written into basis slot j (jv[slot] when given).
__global__ void __launch_bounds__(256)
k_gm_setv(const ProbDev *__restrict__ P, const int4 *__restrict__ tiles, int ntiles,
          double *__restrict__ V, int64_t vstride, int ldp, int j0, const int *__restrict__ jv,
          const double *__restrict__ w, const double *__restrict__ S)
{
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(S, pd.slot)) continue;
        const int j = jv ? jv[pd.slot] : j0;
        const double hn = S[(int64_t)pd.slot * NSCAL + SC_HNORM];
        const double inv = hn != 0.0 ? 1.0 / hn : 0.0;
        double *Vj = V + (int64_t)j * vstride + pd.img;
        for (int e = threadIdx.x; e < tl.z; e += blockDim.x) {
            const int64_t o = tl.y + e;
            Vj[o] = w[pd.img + o] * inv;
        }
    }
}

// out = v_j with j = jv[slot] (the Arnoldi step's preconditioner input).
__global__ void __launch_bounds__(256)
k_gm_getv(const ProbDev *__restrict__ P, const int4 *__restrict__ tiles, int ntiles,
          const double *__restrict__ V, int64_t vstride, const int *__restrict__ jv, double *__restrict__ out,
          const double *__restrict__ S)
{
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(S, pd.slot)) continue;
        const double *Vj = V + (int64_t)jv[pd.slot] * vstride + pd.img;
        for (int e = threadIdx.x; e < tl.z; e += blockDim.x) {
            const int64_t o = tl.y + e;
            out[pd.img + o] = Vj[o];
        }
    }
}

// ---------------------------------------------------------------------------
// Finalize: one CTA per problem.
// ---------------------------------------------------------------------------
__device__ double sum_parts(const double *part, int b, int e, int ld, int i, double *red)
{
    double acc = 0.0;
    // fixed assignment of partials to threads, then a fixed-order block sum
    for (int q = b + threadIdx.x; q < e; q += blockDim.x) acc += part[(int64_t)q * ld + i];
    return block_sum_fixed(acc, red);   // valid in thread 0
}

__global__ void __launch_bounds__(256)
k_finalize(FinArgs f)
{
    __shared__ double red[8];
    __shared__ double sh[72];
    const int p = blockIdx.x;
    if (p >= f.nprob) return;
    double *S = f.S + (int64_t)p * NSCAL;
    const bool active = S[SC_ACTIVE] != 0.0;
    const int nsum = f.nsum_a;
    for (int i = 0; i < nsum; ++i) {
        const double v = sum_parts(f.part_a, f.tb_a[p], f.te_a[p], f.ld_a, i, red);
        if (threadIdx.x == 0) sh[i] = v;
        __syncthreads();
    }
    double sb = 0.0;
    if (f.part_b) {
        sb = sum_parts(f.part_b, f.tb_b[p], f.te_b[p], 1, 0, red);
    }
    if (threadIdx.x != 0 || !active) return;
    const double sa = sh[0];
    auto stop = [&](int status) {
        S[SC_ACTIVE] = 0.0;
        S[SC_STATUS] = status;
    };
    switch (f.op) {
        case FIN_CGLS_INIT: {            // sa = |s0|^2, sb = s.z (or |s|^2 unpreconditioned)
            S[SC_S0] = sqrt(sa);
            S[SC_GAMMA] = f.precond ? sb : sa;
            S[SC_RES] = sa == 0.0 ? 0.0 : 1.0;       // W^T b = 0: x = 0 is exact
            S[SC_ITERS] = 0.0;
            if (f.hist) f.hist[(int64_t)p * f.hist_ld] = 1.0;
            if (!(sa > 0.0)) stop(sa == 0.0 ? WMG_OK : WMG_ERR_NAN);
            break;
        }
        case FIN_PNORM:
            S[SC_PP] = sa;
            break;
        case FIN_CGLS_ALPHA: {           // sa = |q|^2 partials; + lambda |p|^2
            const double delta = sa + f.lambda[p] * S[SC_PP];
            S[SC_DELTA] = delta;
            if (!(delta > 0.0) || !isfinite(delta)) {
                S[SC_ALPHA] = 0.0;
                stop(isfinite(delta) ? WMG_ERR_BREAKDOWN : WMG_ERR_NAN);
            } else {
                S[SC_ALPHA] = S[SC_GAMMA] / delta;
            }
            break;
        }
        case FIN_CGLS_RES: {             // sa = |s|^2 after the x, s update
            const int it = (int)S[SC_ITERS] + 1;
            S[SC_ITERS] = it;
            const double rel = sqrt(sa) / S[SC_S0];
            S[SC_RES] = rel;
            if (f.hist && it < f.hist_ld) f.hist[(int64_t)p * f.hist_ld + it] = rel;
            if (!isfinite(rel)) stop(WMG_ERR_NAN);
            else if (rel < S[SC_RTOL]) stop(WMG_OK);
            else if (it >= (int)S[SC_MAXIT]) stop(WMG_NOT_CONVERGED);
            if (!f.precond) S[SC_GNEW] = sa;      // gamma' = |s|^2 when z = s
            break;
        }
        case FIN_CGLS_BETA: {            // sa = s.z (preconditioned) ; else stored |s|^2
            const double gnew = f.precond ? sa : S[SC_GNEW];
            S[SC_BETA] = gnew / S[SC_GAMMA];
            S[SC_GAMMA] = gnew;
            if (!isfinite(gnew)) stop(WMG_ERR_NAN);
            break;
        }
        case FIN_BI_INIT: {              // sa = |r0|^2 (r0 = f, the shadow residual)
            S[SC_S0] = sqrt(sa);
            S[SC_GAMMA] = sa;                   // rho = <rh, r0> = |r0|^2
            S[SC_ALPHA] = 1.0;
            S[SC_DELTA] = 1.0;                  // omega
            S[SC_BETA] = sa;                    // (rho / 1)(1 / 1); p = r as p = v = 0
            S[SC_RES] = sa == 0.0 ? 0.0 : 1.0;  // b = 0: x = 0 is exact
            S[SC_ITERS] = 0.0;
            if (f.hist) f.hist[(int64_t)p * f.hist_ld] = 1.0;
            if (!(sa > 0.0)) stop(sa == 0.0 ? WMG_OK : WMG_ERR_NAN);
            break;
        }
        case FIN_BI_ALPHA: {             // sa = <rh, v>
            if (!(sa != 0.0) || !isfinite(sa)) stop(isfinite(sa) ? WMG_ERR_BREAKDOWN : WMG_ERR_NAN);
            else S[SC_ALPHA] = S[SC_GAMMA] / sa;
            break;
        }
        case FIN_BI_OMEGA: {             // sa = <t, s>, sb = <t, t>
            S[SC_DELTA] = sb > 0.0 ? sa / sb : 0.0;
            break;
        }
        case FIN_BI_RES: {               // sa = |r|^2, sb = <rh, r>
            const int it = (int)S[SC_ITERS] + 1;
            S[SC_ITERS] = it;
            const double rel = sqrt(sa) / S[SC_S0];
            S[SC_RES] = rel;
            if (f.hist && it < f.hist_ld) f.hist[(int64_t)p * f.hist_ld + it] = rel;
            const double omega = S[SC_DELTA];
            if (!isfinite(rel)) stop(WMG_ERR_NAN);
            else if (rel < S[SC_RTOL] || rel == 0.0) stop(WMG_OK);
            else if (it >= (int)S[SC_MAXIT]) {
                stop(WMG_NOT_CONVERGED);
                // what a resumed solve needs for its next step: beta and rho,
                // or the mark that this step broke down (SC_GNEW = 1)
                const bool broke = omega == 0.0 || sb == 0.0;
                S[SC_GNEW] = broke ? 1.0 : 0.0;
                if (!broke) {
                    S[SC_BETA] = (sb / S[SC_GAMMA]) * (S[SC_ALPHA] / omega);
                    S[SC_GAMMA] = sb;
                }
            }
            else if (omega == 0.0 || sb == 0.0) stop(WMG_ERR_BREAKDOWN);
            else {
                S[SC_BETA] = (sb / S[SC_GAMMA]) * (S[SC_ALPHA] / omega);
                S[SC_GAMMA] = sb;
            }
            break;
        }
        case FIN_SET_RES: {              // sa = |NE residual|^2 of the final iterate
            const double s0 = sqrt(S[SC_S0]);        // FIN_STORE left the squared norm there
            // W^T b = 0 (e.g. b = 0): x = 0 is exact when the residual is 0
            const double rel = s0 > 0.0 ? sqrt(sa) / s0 : (sa == 0.0 ? 0.0 : INFINITY);
            S[SC_RES] = rel;
            if (!isfinite(sa) || !isfinite(s0)) stop(WMG_ERR_NAN);
            else stop(rel < S[SC_RTOL] || rel == 0.0 ? WMG_OK : WMG_NOT_CONVERGED);
            break;
        }
        case FIN_STORE: {
            if (f.store_vec)
                for (int i = 0; i < nsum; ++i) f.store_vec[(int64_t)p * f.store_ld + i] = sh[i];
            else
                S[f.store_slot] = sa;
            break;
        }
        default:
            break;
    }
}

// GMRES scalar work (one thread per problem, after the second CGS pass):
// H column j from the two passes, Givens rotations, residual estimate.
__global__ void k_gm_arnoldi(GmArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.nprob) return;
    double *S = a.S + (int64_t)p * NSCAL;
    if (S[SC_ACTIVE] == 0.0 || a.done[p]) return;
    const int ld = a.ldp, j = a.jslot ? a.jn[p] : a.j, r = a.restart;
    double *H = a.H + (int64_t)p * (r + 1) * r;     // H[i*r + jj]
    double *cs = a.cs + (int64_t)p * r, *sn = a.sn + (int64_t)p * r, *g = a.g + (int64_t)p * (r + 1);
    const double *h1 = a.h1 + (int64_t)p * ld, *h2 = a.h2 + (int64_t)p * ld;
    for (int i = 0; i <= j; ++i) H[i * r + j] = h1[i] + h2[i];
    const double hn = sqrt(S[SC_WNORM2]);           // |w|^2 from the last CGS pass
    S[SC_HNORM] = hn;
    H[(j + 1) * r + j] = hn;
    for (int i = 0; i < j; ++i) {
        const double x0 = H[i * r + j], x1 = H[(i + 1) * r + j];
        H[i * r + j] = cs[i] * x0 + sn[i] * x1;
        H[(i + 1) * r + j] = -sn[i] * x0 + cs[i] * x1;
    }
    const double x0 = H[j * r + j], x1 = H[(j + 1) * r + j];
    const double rr = hypot(x0, x1);
    if (!(rr > 0.0) || !isfinite(rr)) {
        S[SC_ACTIVE] = 0.0;
        S[SC_STATUS] = isfinite(rr) ? WMG_ERR_BREAKDOWN : WMG_ERR_NAN;
        a.jn[p] = j;
        return;
    }
    cs[j] = x0 / rr;
    sn[j] = x1 / rr;
    H[j * r + j] = rr;
    H[(j + 1) * r + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const int it = (int)S[SC_ITERS] + 1;
    S[SC_ITERS] = it;
    const double rel = fabs(g[j + 1]) / S[SC_S0];
    S[SC_RES] = rel;
    if (a.hist && it < a.hist_ld) a.hist[(int64_t)p * a.hist_ld + it] = rel;
    a.jn[p] = j + 1;
    // the cycle ends for this problem when converged, at the iteration cap or
    // on a happy breakdown; the caller finishes the cycle (x update)
    if (rel < S[SC_RTOL] || it >= (int)S[SC_MAXIT] || hn == 0.0) a.done[p] = 1;
}

// Selective reorthogonalisation ("twice is enough", decided per problem):
// after the first classical Gram-Schmidt pass, |w'|^2 = |w|^2 - |h|^2 in
// exact arithmetic; the second pass runs only when the first removed more
// than 1 - kReorthEta^2 of |w|^2, i.e. |w'| < kReorthEta |w| (cancellation,
// where one pass leaves w' measurably non-orthogonal to the basis). With
// |w'| >= kReorthEta |w| one pass keeps the loss of orthogonality below
// about 1 / kReorthEta units in the last place. skip[p] = 1: no second pass.
constexpr double kReorthEta2 = 1.0 / 64.0;                             // kReorthEta = 1/8

__global__ void k_gm_reorth(GmArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.nprob) return;
    const double *S = a.S + (int64_t)p * NSCAL;
    if (S[SC_ACTIVE] == 0.0 || a.done[p]) { a.skip[p] = 1; return; }
    const int j = a.jslot ? a.jn[p] : a.j;
    const double *h1 = a.h1 + (int64_t)p * a.ldp;
    const double wn2 = h1[j + 1];
    double hh = 0.0;
    for (int i = 0; i <= j; ++i) hh += h1[i] * h1[i];
    a.skip[p] = (wn2 > 0.0 && isfinite(wn2) && wn2 - hh >= kReorthEta2 * wn2) ? 1 : 0;
}

// End of cycle: y = H^-1 g (upper triangular jn x jn).
__global__ void k_gm_solve_y(GmArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.nprob) return;
    const double *S = a.S + (int64_t)p * NSCAL;
    if (S[SC_ACTIVE] == 0.0 && a.jn[p] == 0) return;
    const int r = a.restart, ld = a.ldp, jj = a.jn[p];
    const double *H = a.H + (int64_t)p * (r + 1) * r, *g = a.g + (int64_t)p * (r + 1);
    double *y = a.y + (int64_t)p * ld;
    for (int i = jj - 1; i >= 0; --i) {
        double v = g[i];
        for (int q = i + 1; q < jj; ++q) v -= H[i * r + q] * y[q];
        y[i] = v / H[i * r + i];
    }
}

// Restart: beta = |r| from partials; g = [beta, 0...]; status on convergence.
__global__ void k_gm_restart(GmArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.nprob) return;
    double *S = a.S + (int64_t)p * NSCAL;
    if (S[SC_ACTIVE] == 0.0) return;
    const double beta = sqrt(S[SC_WNORM2]);
    S[SC_HNORM] = beta;
    double *g = a.g + (int64_t)p * (a.restart + 1);
    for (int i = 0; i <= a.restart; ++i) g[i] = 0.0;
    g[0] = beta;
    a.jn[p] = 0;
    a.done[p] = 0;
    if (a.init) {
        S[SC_S0] = beta;
        S[SC_RES] = beta == 0.0 ? 0.0 : 1.0;           // b = 0: x = 0 is exact
        S[SC_ITERS] = 0.0;
        if (a.hist) a.hist[(int64_t)p * a.hist_ld] = 1.0;
        if (!(beta > 0.0)) { S[SC_ACTIVE] = 0.0; S[SC_STATUS] = beta == 0.0 ? WMG_OK : WMG_ERR_NAN; }
        return;
    }
    const double rel = beta / S[SC_S0];
    S[SC_RES] = rel;
    const int it = (int)S[SC_ITERS];
    if (a.hist && it < a.hist_ld) a.hist[(int64_t)p * a.hist_ld + it] = rel;
    if (!isfinite(rel)) { S[SC_ACTIVE] = 0.0; S[SC_STATUS] = WMG_ERR_NAN; }
    else if (rel < S[SC_RTOL]) { S[SC_ACTIVE] = 0.0; S[SC_STATUS] = WMG_OK; }
    else if (it >= (int)S[SC_MAXIT]) { S[SC_ACTIVE] = 0.0; S[SC_STATUS] = WMG_NOT_CONVERGED; }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int grid_for(int ntiles) { return ntiles < num_sms() * 8 ? ntiles : num_sms() * 8; }

template <class T>
void launch_img(int op, const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                const ImgArgs &a, cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    const int grid = grid_for(ntiles);
#define WMG_IMG_CASE(O) case O: k_img<T, O><<<grid, 256, 0, st>>>(G, P, tiles, ntiles, a); break;
    switch (op) {
        WMG_IMG_CASE(IMG_PUPDATE)
        WMG_IMG_CASE(IMG_PINIT)
        WMG_IMG_CASE(IMG_FIRST_SWEEP)
        WMG_IMG_CASE(IMG_ZERO_RESID)
        WMG_IMG_CASE(IMG_LOAD)
        WMG_IMG_CASE(IMG_COPY64)
        WMG_IMG_CASE(IMG_STORE_OUT)
        WMG_IMG_CASE(IMG_DOT_SZ)
        default: break;
    }
#undef WMG_IMG_CASE
}

template <class T>
void launch_vec(int op, const ProbDev *P, const int4 *tiles, int ntiles, const VecArgs &a,
                cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    const int grid = grid_for(ntiles);
#define WMG_VEC_CASE(O) case O: k_vec<T, O><<<grid, 256, 0, st>>>(P, tiles, ntiles, a); break;
    switch (op) {
        WMG_VEC_CASE(VEC_R_UPDATE)
        WMG_VEC_CASE(VEC_R_INIT)
        WMG_VEC_CASE(VEC_SIRT_R)
        WMG_VEC_CASE(VEC_NRM2)
        WMG_VEC_CASE(VEC_SCALE_V)
        WMG_VEC_CASE(VEC_X_ADD)
        WMG_VEC_CASE(VEC_RESID64)
        WMG_VEC_CASE(VEC_TO_OP)
        WMG_VEC_CASE(VEC_SINO_DIFF)
        WMG_VEC_CASE(VEC_NE_RES)
        default: break;
    }
#undef WMG_VEC_CASE
}

void launch_finalize(const FinArgs &f, cudaStream_t st)
{
    if (f.nprob <= 0) return;
    count_launches(1);
    k_finalize<<<f.nprob, 256, 0, st>>>(f);
}

void launch_gm_dots(const ProbDev *P, const int4 *tiles, int ntiles, const double *V, int64_t vstride,
                    const double *w, int j, int ldp, double *part, const double *S, cudaStream_t st,
                    const int *jv, bool wnorm, const int *skip)
{
    if (ntiles <= 0) return;
    count_launches(1);
    k_gm_dots<<<grid_for(ntiles), 256, 0, st>>>(P, tiles, ntiles, V, vstride, w, j, jv, ldp, part, S,
                                                wnorm ? 1 : 0, skip);
}
void launch_gm_axpy(const ProbDev *P, const int4 *tiles, int ntiles, const double *V, int64_t vstride,
                    double *w, int j, int ldp, const double *Hc, double *part, const double *S,
                    cudaStream_t st, const int *jv, const int *skip)
{
    if (ntiles <= 0) return;
    count_launches(1);
    k_gm_axpy<<<grid_for(ntiles), 256, 0, st>>>(P, tiles, ntiles, V, vstride, w, j, jv, ldp, Hc, part, S, skip);
}
void launch_gm_combine(const ProbDev *P, const int4 *tiles, int ntiles, const double *V,
                       int64_t vstride, int ldp, const double *Yv, const int *jn, double *out,
                       const double *S, cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    k_gm_combine<<<grid_for(ntiles), 256, 0, st>>>(P, tiles, ntiles, V, vstride, ldp, Yv, jn, out, S);
}
void launch_gm_setv(const ProbDev *P, const int4 *tiles, int ntiles, double *V, int64_t vstride,
                    int ldp, int j, const double *w, const double *S, cudaStream_t st, const int *jv)
{
    if (ntiles <= 0) return;
    count_launches(1);
    k_gm_setv<<<grid_for(ntiles), 256, 0, st>>>(P, tiles, ntiles, V, vstride, ldp, j, jv, w, S);
}
void launch_gm_getv(const ProbDev *P, const int4 *tiles, int ntiles, const double *V, int64_t vstride,
                    const int *jv, double *out, const double *S, cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    k_gm_getv<<<grid_for(ntiles), 256, 0, st>>>(P, tiles, ntiles, V, vstride, jv, out, S);
}
void launch_bicg(int op, const ProbDev *P, const int4 *tiles, int ntiles, const BicgArgs &a, cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    const int grid = grid_for(ntiles);
    switch (op) {
        case BI_INIT: k_bicg<BI_INIT><<<grid, 256, 0, st>>>(P, tiles, ntiles, a); break;
        case BI_P: k_bicg<BI_P><<<grid, 256, 0, st>>>(P, tiles, ntiles, a); break;
        case BI_RV: k_bicg<BI_RV><<<grid, 256, 0, st>>>(P, tiles, ntiles, a); break;
        case BI_S: k_bicg<BI_S><<<grid, 256, 0, st>>>(P, tiles, ntiles, a); break;
        case BI_TS: k_bicg<BI_TS><<<grid, 256, 0, st>>>(P, tiles, ntiles, a); break;
        case BI_XR: k_bicg<BI_XR><<<grid, 256, 0, st>>>(P, tiles, ntiles, a); break;
        default: break;
    }
}

void launch_gm_scalar(int which, const GmArgs &a, cudaStream_t st)
{
    const int blocks = (a.nprob + 127) / 128;
    count_launches(1);
    if (which == 0) k_gm_arnoldi<<<blocks, 128, 0, st>>>(a);
    else if (which == 1) k_gm_solve_y<<<blocks, 128, 0, st>>>(a);
    else if (which == 3) k_gm_reorth<<<blocks, 128, 0, st>>>(a);
    else k_gm_restart<<<blocks, 128, 0, st>>>(a);
}

template void launch_img<float>(int, const GeomDev *, const ProbDev *, const int4 *, int,
                                const ImgArgs &, cudaStream_t);
template void launch_img<double>(int, const GeomDev *, const ProbDev *, const int4 *, int,
                                 const ImgArgs &, cudaStream_t);
template void launch_vec<float>(int, const ProbDev *, const int4 *, int, const VecArgs &, cudaStream_t);
template void launch_vec<double>(int, const ProbDev *, const int4 *, int, const VecArgs &, cudaStream_t);

}  // namespace wmg
