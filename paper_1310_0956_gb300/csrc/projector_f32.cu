// projector_f32.cu -- FP32 forward projection and backprojection (Section 2.1,
// eq. sys: w_ij = length of ray i in pixel j), the operator of the mixed
// precision path. Same weights as projector.cu (trapezoid law of the chord
// of a unit pixel), organised for the FP32 pipes:
//  - per-angle constants (split trigonometry, chord constants, frame slope)
//    come from a table built once per plan in FP64, so no division, square
//    root or FP64 instruction runs per tile;
//  - the distance t - tau is exact up to a small rounded correction (split
//    trigonometry: products with the 12-bit heads are exact in FP32), so the
//    weights do not lose accuracy far from the image centre;
//  - rows are walked incrementally (exact head terms, rounded tails), two
//    candidate pixels per row in the forward direction, two candidate bins
//    per pixel and angle in the backward direction (unit bin spacing; a
//    general loop otherwise);
//  - sums are compensated (Kahan) so a ray or pixel sum of a few hundred
//    terms keeps FP32 rounding of its terms, not of its length.
// Deterministic: no atomics, fixed combination orders.
#include <cmath>
#include <cstring>

#include "bp_epilogue.cuh"
#include "kern_common.cuh"

namespace wmg {

__device__ __forceinline__ float chord_f(const AngleF &A, bool axis, float d)
{
    if (axis) return d < 0.5f ? 1.f : (d == 0.5f ? 0.5f : 0.f);
    return fminf(fmaxf(__fmaf_rn(-d, A.inv_ab, A.hw_inv), 0.f), A.lmax);
}

// Chord divided by lmax = 1/alpha, in [0, 1]: one saturating FMA.
__device__ __forceinline__ float chord_n(float wa, float wb, float d)
{
    return __saturatef(__fmaf_rn(-d, wa, wb));
}

// ---------------------------------------------------------------------------
// Forward: tile = {prob, angle, first ray, 0}; lane = ray, warps take every
// NW-th row of the rays' common row range.
// ---------------------------------------------------------------------------
template <int NW>
__global__ void __launch_bounds__(32 * NW, 4)
k_project_f32(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
              const int4 *__restrict__ tiles, int ntiles, PjArgs a)
{
    __shared__ float red_s[NW][32], red_c[NW][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(a.S, pd.slot)) continue;
        const GeomDev &g = G[pd.geom];
        const int n = g.n, D = g.D, ang = tl.y, k = tl.z + lane;
        const bool valid = k < D;
        const AngleF A = g.angf[ang];
        const int flags = __float_as_int(A.flags);
        const bool steep = flags & 1, axis = flags & 2;
        const float cc_hi = steep ? A.chi : A.shi, cc_lo = steep ? A.clo : A.slo;
        const float ss_hi = steep ? A.shi : A.chi, ss_lo = steep ? A.slo : A.clo;
        const float *__restrict__ src = static_cast<const float *>(steep ? a.img : a.imgT) + pd.img;
        const float half_n = 0.5f * (float)n;
        const float tk = __fmaf_rn((float)k - g.hDf, g.dtf, g.t0f);
        // rows the lane's ray can touch (image x-range widened by one pixel)
        int lo = n, hi = -1;
        if (valid) {
            const float xs0 = tk * A.inv_cc;           // crossing of y = 0
            if (ss_hi == 0.f && ss_lo == 0.f) {
                if (fabsf(xs0) < half_n + 1.f) { lo = 0; hi = n - 1; }
            } else {
                const float ya = (xs0 - (half_n + 1.f)) * A.inv_slope, yb = (xs0 + (half_n + 1.f)) * A.inv_slope;
                lo = max(0, __float2int_ru(fminf(ya, yb) + half_n - 0.5f));
                hi = min(n - 1, __float2int_rd(fmaxf(ya, yb) + half_n - 0.5f));
            }
        }
        lo = warp_min(lo);
        hi = warp_max(hi);
        float s = 0.f, c = 0.f;                        // compensated sum
        const int nrows = hi - lo + 1;
        if (nrows > 0) {
            // warp w takes rows lo + w + NW*j; R consecutive ones per step,
            // their 2R loads issued before any is used
            constexpr int R = 4;
            const int iy0 = lo + w;
            const float dy = (float)NW;
            float yc = (float)iy0 + 0.5f - half_n;
            float brow = __fmaf_rn(-yc, ss_hi, tk);            // t - yc ss_hi: exact
            float cy = yc * ss_lo;
            float xs = __fmaf_rn(-yc, A.slope, tk * A.inv_cc); // crossing of the row centre line
            const float dbrow = -dy * ss_hi, dcy = dy * ss_lo, dxs = -dy * A.slope;
            // candidates: the two pixel centres nearest the crossing. The
            // support half-width hwx is at most 1, so every pixel with a
            // nonzero weight is one of them whatever the rounding of xs.
            const float off = half_n - 0.5f;
            const int nmine = (nrows - w + NW - 1) / NW;       // rows of this warp
            const float *__restrict__ row = src + (int64_t)iy0 * n;
            const int64_t drow = (int64_t)NW * n;
            const float wa = A.wa, wb = A.wb, ccf = A.cc;
            for (int j = 0; j < nmine; j += R) {
                float v0[R], v1[R], w0[R], w1[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const bool live = valid && (j + r < nmine);
                    const int ix0 = __float2int_rd(xs + off);
                    const float *rp = row + ix0;
                    v0[r] = (live && (unsigned)ix0 < (unsigned)n) ? __ldg(rp) : 0.f;
                    v1[r] = (live && (unsigned)(ix0 + 1) < (unsigned)n) ? __ldg(rp + 1) : 0.f;
                    const float xc = (float)ix0 + 0.5f - half_n;
                    const float dl0 = __fmaf_rn(-xc, cc_hi, brow) - __fmaf_rn(xc, cc_lo, cy);
                    w0[r] = chord_n(wa, wb, fabsf(dl0));
                    w1[r] = chord_n(wa, wb, fabsf(dl0 - ccf));
                    brow += dbrow;
                    cy += dcy;
                    xs += dxs;
                    row += drow;
                }
#pragma unroll
                for (int r = 0; r < R; r += 2) {
                    const float rs = __fmaf_rn(w0[r], v0[r], __fmaf_rn(w1[r], v1[r],
                                     __fmaf_rn(w0[r + 1], v0[r + 1], w1[r + 1] * v1[r + 1])));
                    const float y = rs - c;                    // Kahan step
                    const float tt = s + y;
                    c = (tt - s) - y;
                    s = tt;
                }
            }
        }
        red_s[w][lane] = s;
        red_c[w][lane] = c;
        __syncthreads();
        if (w == 0) {
            float S = 0.f, Cc = 0.f;
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                const float y = (red_s[i][lane] - red_c[i][lane]) - Cc;
                const float tt = S + y;
                Cc = (tt - S) - y;
                S = tt;
            }
            const float v = (S - Cc) * (A.lmax * g.hf);
            if (valid) static_cast<float *>(a.sino)[pd.sino + (int64_t)ang * D + k] = v;
            if (a.part) {
                double q2 = valid ? (double)v * (double)v : 0.0;
                q2 = warp_sum_fixed(q2);
                if (lane == 0) a.part[t] = q2;
            }
        }
        __syncthreads();
    }
}

void launch_project_f32(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                        const PjArgs &a, cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    constexpr int NW = 8;
    const int grid = min(ntiles, num_sms() * (a.ctas_per_sm > 0 ? a.ctas_per_sm : 8));
    k_project_f32<NW><<<grid, 32 * NW, 0, st>>>(G, P, tiles, ntiles, a);
}

// ---------------------------------------------------------------------------
// Backward: tile = {prob, iy0, ix0, 0} of 32 x 32 pixels, thread = one column
// and 4 rows 8 apart. Geometries with unit bins (g.unit) take the two-bin
// path, the others the general one; ALL_UNIT (every geometry of the launch
// has unit bins) compiles the general path out. The choice depends on the
// tile's own geometry only, so a problem gets the same bits in any batch.
// ---------------------------------------------------------------------------
template <int EPI, bool ALL_UNIT>
__global__ void __launch_bounds__(256)
k_backproject_f32(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
                  const int4 *__restrict__ tiles, int ntiles, BpArgs a)
{
    __shared__ double red[8];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(a.S, pd.slot)) continue;
        const GeomDev &g = G[pd.geom];
        const int n = g.n, m = g.m, D = g.D;
        const int ix = tl.z + tx;
        const float half_n = 0.5f * (float)n;
        const float xo = (float)ix + 0.5f - half_n;
        const float yo0 = (float)(tl.y + ty) + 0.5f - half_n;
        const float *__restrict__ sg = static_cast<const float *>(a.sino) + pd.sino;
        const float hD = g.hDf, dt = g.dtf, t0 = g.t0f, inv_dt = 1.f / g.dtf;
        const bool unit = ALL_UNIT || g.unit;
        float s[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
        for (int ang = 0; ang < m; ++ang) {
            const AngleF A = g.angf[ang];
            const bool axis = __float_as_int(A.flags) & 2;
            const float *__restrict__ row = sg + (int64_t)ang * D;
            float ph = __fmaf_rn(xo, A.chi, yo0 * A.shi);        // exact head of tau
            float pc = __fmaf_rn(xo, A.clo, yo0 * A.slo);        // rounded tail
            const float dph = 8.f * A.shi, dpc = 8.f * A.slo;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float rs;
                if (unit) {
                    // the two bins nearest tau (support half-width <= sqrt(1/2))
                    const int k0 = __float2int_rd((ph + pc) - t0 + hD);
                    const float tk = (float)k0 - hD + t0;
                    const float d0 = (tk - ph) - pc;
                    const float w0 = chord_n(A.wa, A.wb, fabsf(d0)), w1 = chord_n(A.wa, A.wb, fabsf(d0 + 1.f));
                    const float v0 = (unsigned)k0 < (unsigned)D ? __ldg(row + k0) : 0.f;
                    const float v1 = (unsigned)(k0 + 1) < (unsigned)D ? __ldg(row + k0 + 1) : 0.f;
                    // explicit rounding: no contraction into the Kahan step
                    // below, whichever paths the instantiation holds
                    rs = __fmul_rn(__fmaf_rn(w0, v0, w1 * v1), A.lmax);
                } else {
                    const float hwb = A.hw * inv_dt;
                    const int k0 = __float2int_ru(((ph + pc) - t0) * inv_dt + hD - hwb);
                    const int nc = __float2int_rd(2.f * hwb) + 1;
                    rs = 0.f;
                    for (int q = 0; q < nc; ++q) {
                        const int kk = k0 + q;
                        if ((unsigned)kk < (unsigned)D) {
                            const float tk = __fmaf_rn((float)kk - hD, dt, t0);
                            rs = __fmaf_rn(chord_f(A, axis, fabsf((tk - ph) - pc)), __ldg(row + kk), rs);
                        }
                    }
                }
                const float y = rs - cmp[r];
                const float tt = s[r] + y;
                cmp[r] = (tt - s[r]) - y;
                s[r] = tt;
                ph += dph;
                pc += dpc;
            }
        }
        double part = 0.0;
        if (ix < n) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int iy = tl.y + ty + 8 * r;
                if (iy < n)
                    part += bp_epilogue<float, EPI>(g, pd, a, ix, iy, ((double)s[r] - (double)cmp[r]) * g.h);
            }
        }
        if (a.part) {
            part = warp_sum_fixed(part);
            if (tx == 0) red[ty] = part;
            __syncthreads();
            if (threadIdx.x == 0) {
                double v = 0.0;
                for (int i = 0; i < 8; ++i) v += red[i];
                a.part[t] = v;
            }
            __syncthreads();
        }
    }
}

void launch_backproject_f32(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                            const BpArgs &a, bool unit, cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    const int grid = min(ntiles, num_sms() * (a.ctas_per_sm > 0 ? a.ctas_per_sm : 8));
#define WMG_BPF(E)                                                                                  \
    case E:                                                                                         \
        if (unit) k_backproject_f32<E, true><<<grid, 256, 0, st>>>(G, P, tiles, ntiles, a);         \
        else k_backproject_f32<E, false><<<grid, 256, 0, st>>>(G, P, tiles, ntiles, a);             \
        break;
    switch (a.epi) {
        WMG_BPF(BP_STORE) WMG_BPF(BP_CGLS_S) WMG_BPF(BP_RESID) WMG_BPF(BP_POST)
        WMG_BPF(BP_APPLY_A) WMG_BPF(BP_SIRT) WMG_BPF(BP_GMRES_W) WMG_BPF(BP_ATB)
        default: break;
    }
#undef WMG_BPF
}

void fill_angle_table(const double2 *cs, int m, AngleF *out)
{
    for (int a = 0; a < m; ++a) {
        const double c = cs[a].x, s = cs[a].y;
        AngleF A{};
        const double ch = std::nearbyint(c * 4096.0) / 4096.0, sh = std::nearbyint(s * 4096.0) / 4096.0;
        A.chi = (float)ch; A.clo = (float)(c - ch); A.shi = (float)sh; A.slo = (float)(s - sh);
        const double al = std::fmax(std::fabs(c), std::fabs(s)), be = std::fmin(std::fabs(c), std::fabs(s));
        const bool steep = std::fabs(c) >= std::fabs(s), axis = be == 0.0;
        const double cc = steep ? c : s, ss = steep ? s : c;
        const double hw = 0.5 * (al + be);
        A.hw = (float)hw;
        A.inv_ab = axis ? 0.f : (float)(1.0 / (al * be));
        A.hw_inv = axis ? 0.f : (float)(hw / (al * be));
        A.lmax = (float)(1.0 / al);
        A.hwx = (float)(hw / std::fabs(cc));
        A.inv_cc = (float)(1.0 / cc);
        A.slope = (float)(ss / cc);
        A.inv_slope = ss != 0.0 ? (float)(cc / ss) : 0.f;
        const int flags = (steep ? 1 : 0) | (axis ? 2 : 0);
        std::memcpy(&A.flags, &flags, sizeof(int));
        A.wa = axis ? 4194304.f : (float)(1.0 / be);
        A.wb = axis ? 2097152.5f : (float)(hw / be);
        A.cc = (float)cc;
        out[a] = A;
    }
}

}  // namespace wmg
