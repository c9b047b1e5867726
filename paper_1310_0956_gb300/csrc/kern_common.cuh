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
__device__ __forceinline__ double ldg_t(const double *p) { return __ldg(p); }

// Signed distance reference tau = x c + y s of a pixel centre, rounded as two
// products and one sum (no fused multiply-add), so the value is the same
// whichever of the two orders of the terms a kernel evaluates.
template <class T> __device__ __forceinline__ T tau_of(T x, T c, T y, T s);
template <> __device__ __forceinline__ float tau_of<float>(float x, float c, float y, float s)
{
    return __fadd_rn(__fmul_rn(x, c), __fmul_rn(y, s));
}
template <> __device__ __forceinline__ double tau_of<double>(double x, double c, double y, double s)
{
    return __dadd_rn(__dmul_rn(x, c), __dmul_rn(y, s));
}

// Detector offset t_k of bin k in pixel widths: (k - (D-1)/2) * dt + t0.
template <class T>
__device__ __forceinline__ T ray_offset(const GeomDev &g, int k)
{
    return fma_t(T(k) - T(0.5) * T(g.D - 1), T(g.dt), T(g.t0));
}

// Trapezoid-law chord of a unit pixel, as a function of the distance d >= 0
// between the pixel centre and the line (per-angle constants).
template <class T>
struct Chord {
    T hw;        // (alpha + beta) / 2: half-width of the support
    T inv_ab;    // 1 / (alpha beta)
    T lmax;      // 1 / alpha: plateau
    bool axis;   // beta == 0
    __device__ __forceinline__ T operator()(T d) const
    {
        if (axis) return d < T(0.5) ? T(1) : (d == T(0.5) ? T(0.5) : T(0));
        return fmin(fmax((hw - d) * inv_ab, T(0)), lmax);
    }
};

template <class T>
__device__ __forceinline__ Chord<T> make_chord(T c, T s)
{
    const T ac = fabs(c), as = fabs(s);
    const T al = fmax(ac, as), be = fmin(ac, as);
    Chord<T> ch;
    ch.hw = T(0.5) * (al + be);
    ch.axis = (be == T(0));
    ch.inv_ab = ch.axis ? T(0) : T(1) / (al * be);
    ch.lmax = T(1) / al;
    return ch;
}

__device__ __forceinline__ int warp_min(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
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
