// kern_common.cuh -- device helpers shared by the kernels of this library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "wmg_internal.cuh"

namespace wmg {

int num_sms();

__device__ __forceinline__ bool slot_active(const double *S, int slot)
{
    return S == nullptr || S[(int64_t)slot * NSCAL + SC_ACTIVE] != 0.0;
}

__device__ __forceinline__ void load_cs(const GeomDev &g, int a, float &c, float &s)
{
    const float2 v = g.cs32[a];
    c = v.x;
    s = v.y;
}
__device__ __forceinline__ void load_cs(const GeomDev &g, int a, double &c, double &s)
{
    const double2 v = g.cs64[a];
    c = v.x;
    s = v.y;
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ float ldg_t(const float *p) { return __ldg(p); }

// Operator-storage loads and stores of the FP32 kernels: float, or bfloat16
// (plans with BF16 operator storage) widened to / rounded from float.
__device__ __forceinline__ float ld_op(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_op(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ double ld_op(const double *p) { return __ldg(p); }
__device__ __forceinline__ void st_op(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_op(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st_op(float *p, double v) { *p = (float)v; }
__device__ __forceinline__ void st_op(__nv_bfloat16 *p, double v) { *p = __double2bfloat16(v); }
__device__ __forceinline__ void st_op(double *p, double v) { *p = v; }
__device__ __forceinline__ double ldg_t(const double *p) { return __ldg(p); }

// Distance t - tau between a line p.(c, s) = t and a pixel centre (x, y),
// tau = x c + y s (pixel widths; x, y are half-integers, |x|, |y| <= n/2).
//
// FP64: tau as two rounded products and one sum (no fused multiply-add), so
// the value does not depend on which of the two terms a kernel puts first.
// FP32: with c = c_hi + c_lo, c_hi a multiple of 2^-12 (12 significant bits),
// the products x c_hi, y s_hi and the differences with t are multiples of
// 2^-13 below 2048 in magnitude, hence exact in FP32; only the small
// correction x c_lo + y s_lo (|.| < 1/4) is rounded. The FP32 distance is
// therefore within a few 1e-8 pixel widths of the exact one, however far the
// pixel is from the centre, and both directions of the projector evaluate the
// same expression.
struct LineF {
    float t, chi, clo, shi, slo;
};
struct LineD {
    double t, c, s;
};
__device__ __forceinline__ float line_dist(const LineF &l, float x, float y)
{
    const float ex = __fmaf_rn(-x, l.chi, __fmaf_rn(-y, l.shi, l.t));          // exact
    const float corr = __fadd_rn(__fmul_rn(x, l.clo), __fmul_rn(y, l.slo));
    return __fsub_rn(ex, corr);
}
__device__ __forceinline__ double line_dist(const LineD &l, double x, double y)
{
    return __dsub_rn(l.t, __dadd_rn(__dmul_rn(x, l.c), __dmul_rn(y, l.s)));
}

// Per-angle line description for a kernel's frame; `swap` exchanges the roles
// of x and y (transposed-image frame).
template <class T> struct LineOf;
template <> struct LineOf<float> { typedef LineF type; };
template <> struct LineOf<double> { typedef LineD type; };

__device__ __forceinline__ void make_line(const GeomDev &g, int a, bool swap, float t, LineF &l)
{
    const float4 v = g.csx[a];
    l.t = t;
    if (swap) { l.chi = v.z; l.clo = v.w; l.shi = v.x; l.slo = v.y; }
    else { l.chi = v.x; l.clo = v.y; l.shi = v.z; l.slo = v.w; }
}
__device__ __forceinline__ void make_line(const GeomDev &g, int a, bool swap, double t, LineD &l)
{
    const double2 v = g.cs64[a];
    l.t = t;
    l.c = swap ? v.y : v.x;
    l.s = swap ? v.x : v.y;
}

// Detector offset t_k of bin k in pixel widths: (k - (D-1)/2) * dt + t0.
template <class T>
__device__ __forceinline__ T ray_offset(const GeomDev &g, int k)
{
    return fma_t(T(k) - T(0.5) * T(g.D - 1), T(g.dt), T(g.t0));
}

// Weight of a unit pixel as a function of the distance d >= 0 between the
// pixel centre and the line (per-angle constants):
//  strip:  the trapezoid-law chord, min(max((hw - d) / (alpha beta), 0), 1/alpha)
//          with hw = (alpha + beta) / 2 (a step at 1/2 when beta = 0);
//  Joseph: (1 - d / alpha) / alpha for d < alpha, the same formula with
//          hw = alpha, 1 / alpha^2 in place of 1 / (alpha beta): the line meets
//          the dominant axis' row (column) centre line d / alpha away from the
//          pixel centre, and each row (column) is 1 / alpha of line.
template <class T>
struct Chord {
    T hw;        // half-width of the support
    T inv_ab;    // slope: 1 / (alpha beta) (strip), 1 / alpha^2 (Joseph)
    T lmax;      // 1 / alpha: plateau
    bool axis;   // strip with beta == 0
    __device__ __forceinline__ T operator()(T d) const
    {
        if (axis) return d < T(0.5) ? T(1) : (d == T(0.5) ? T(0.5) : T(0));
        return fmin(fmax((hw - d) * inv_ab, T(0)), lmax);
    }
};

template <class T>
__device__ __forceinline__ Chord<T> make_chord(T c, T s, int kernel)
{
    const T ac = fabs(c), as = fabs(s);
    const T al = fmax(ac, as), be = fmin(ac, as);
    Chord<T> ch;
    ch.lmax = T(1) / al;
    if (kernel == WMG_KERNEL_JOSEPH) {
        ch.hw = al;
        ch.axis = false;
        ch.inv_ab = ch.lmax * ch.lmax;
        return ch;
    }
    ch.hw = T(0.5) * (al + be);
    ch.axis = (be == T(0));
    ch.inv_ab = ch.axis ? T(0) : T(1) / (al * be);
    return ch;
}

// Running sum. FP32: compensated (Kahan) summation, so the error of a long
// sum stays at a few units of FP32 rounding of its terms instead of growing
// with the number of terms; value() returns sum + compensation in FP64.
// FP64: plain summation.
template <class T> struct Accum;
template <> struct Accum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = __fsub_rn(v, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct Accum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ int warp_min(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_min_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ int warp_max(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// Butterfly sum: the same fixed order on every run, every lane gets the result.
__device__ __forceinline__ double warp_sum_fixed(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of one double per thread over a block of `nthreads` (multiple of 32),
// fixed order; result valid in thread 0. `red` holds nthreads/32 doubles.
__device__ __forceinline__ double block_sum_fixed(double v, double *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_fixed(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) t += red[i];
    return t;
}

}  // namespace wmg
