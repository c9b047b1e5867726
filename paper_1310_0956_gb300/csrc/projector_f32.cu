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
// Forward: tile = {first problem, angle, first ray, images}: `images`
// consecutive problems of one geometry (0 or 1: one problem). Lane = ray,
// warps take every NW-th row of the rays' common row range. The candidate
// pixels and their weights are computed once per row and applied to every
// image of the tile; each image keeps its own compensated sums in the same
// order whatever the tile holds, so a problem gets the same bits alone and
// grouped with others.
// ---------------------------------------------------------------------------
template <int NW, int IB, class TS>
__global__ void __launch_bounds__(32 * NW, 2)
k_project_f32(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
              const int4 *__restrict__ tiles, int ntiles, PjArgs a)
{
    __shared__ float red_s[NW][IB][32], red_c[NW][IB][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const int nimg = min(IB, max(1, tl.w));
        const ProbDev p0 = P[tl.x];
        const GeomDev &g = G[p0.geom];
        const int n = g.n, D = g.D, ang = tl.y, k = tl.z + lane;
        const AngleF A = g.angf[ang];
        const int flags = __float_as_int(A.flags);
        const bool steep = flags & 1;
        const TS *__restrict__ base = static_cast<const TS *>(steep ? a.img : a.imgT);
        const TS *src[IB];
        bool act[IB];
        bool any = false;
#pragma unroll
        for (int b = 0; b < IB; ++b) {
            act[b] = false;
            src[b] = base;
            if (b < nimg) {
                const ProbDev pb = P[tl.x + b];
                act[b] = slot_active(a.S, pb.slot);
                src[b] = base + pb.img;
            }
            any |= act[b];
        }
        if (!any) continue;                                        // CTA-uniform
        const bool valid = k < D;
        const float cc_hi = steep ? A.chi : A.shi, cc_lo = steep ? A.clo : A.slo;
        const float ss_hi = steep ? A.shi : A.chi, ss_lo = steep ? A.slo : A.clo;
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
        float s[IB], c[IB];                            // compensated sums per image
#pragma unroll
        for (int b = 0; b < IB; ++b) { s[b] = 0.f; c[b] = 0.f; }
        const int nrows = hi - lo + 1;
        if (nrows > 0) {
            // warp w takes rows lo + w + NW*j, R consecutive ones per step
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
            int roff = iy0 * n;
            const int drow = NW * n;
            const float wa = A.wa, wb = A.wb, ccf = A.cc;
            for (int j = 0; j < nmine; j += R) {
                int idx[R];
                bool ok0[R], ok1[R];
                float w0[R], w1[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const bool live = valid && (j + r < nmine);
                    const int ix0 = __float2int_rd(xs + off);
                    idx[r] = roff + ix0;
                    ok0[r] = live && (unsigned)ix0 < (unsigned)n;
                    ok1[r] = live && (unsigned)(ix0 + 1) < (unsigned)n;
                    const float xc = (float)ix0 + 0.5f - half_n;
                    const float dl0 = __fmaf_rn(-xc, cc_hi, brow) - __fmaf_rn(xc, cc_lo, cy);
                    w0[r] = chord_n(wa, wb, fabsf(dl0));
                    w1[r] = chord_n(wa, wb, fabsf(dl0 - ccf));
                    brow += dbrow;
                    cy += dcy;
                    xs += dxs;
                    roff += drow;
                }
#pragma unroll
                for (int b = 0; b < IB; ++b) {
                    if (!act[b]) continue;                      // uniform across the CTA
                    float v0[R], v1[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        v0[r] = ok0[r] ? ld_op(src[b] + idx[r]) : 0.f;
                        v1[r] = ok1[r] ? ld_op(src[b] + idx[r] + 1) : 0.f;
                    }
                    // one product chain over the step's rows in row order,
                    // then one compensated (Kahan) step
                    float rs = w0[0] * v0[0];
                    rs = __fmaf_rn(w1[0], v1[0], rs);
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        rs = __fmaf_rn(w0[r], v0[r], rs);
                        rs = __fmaf_rn(w1[r], v1[r], rs);
                    }
                    const float y = rs - c[b];
                    const float tt = s[b] + y;
                    c[b] = (tt - s[b]) - y;
                    s[b] = tt;
                }
            }
        }
#pragma unroll
        for (int b = 0; b < IB; ++b) {
            red_s[w][b][lane] = s[b];
            red_c[w][b][lane] = c[b];
        }
        __syncthreads();
        if (w < IB && act[w]) {                                  // warp w finishes image w
            const int b = w;
            float S = 0.f, Cc = 0.f;
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                const float y = (red_s[i][b][lane] - red_c[i][b][lane]) - Cc;
                const float tt = S + y;
                Cc = (tt - S) - y;
                S = tt;
            }
            const ProbDev pb = P[tl.x + b];
            const float v = (S - Cc) * (A.lmax * g.hf);
            if (valid) st_op(static_cast<TS *>(a.sino) + pb.sino + (int64_t)ang * D + k, v);
            if (a.part) {
                double q2 = valid ? (double)v * (double)v : 0.0;
                q2 = warp_sum_fixed(q2);
                // the problem's partial of this (angle, ray block), at the
                // index its one-image tile list gives it
                if (lane == 0) a.part[a.part_base[tl.x + b] + ang * ((D + 31) / 32) + tl.z / 32] = q2;
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
    if (a.bf16) {
        if (a.group == kProjGroup)
            k_project_f32<NW, kProjGroup, __nv_bfloat16><<<grid, 32 * NW, 0, st>>>(G, P, tiles, ntiles, a);
        else k_project_f32<NW, 1, __nv_bfloat16><<<grid, 32 * NW, 0, st>>>(G, P, tiles, ntiles, a);
    } else if (a.group == kProjGroup) {
        k_project_f32<NW, kProjGroup, float><<<grid, 32 * NW, 0, st>>>(G, P, tiles, ntiles, a);
    } else {
        k_project_f32<NW, 1, float><<<grid, 32 * NW, 0, st>>>(G, P, tiles, ntiles, a);
    }
}

// ---------------------------------------------------------------------------
// Backward: tile = {problem, iy0, ix0, -} of 32 x 32 pixels, 128 threads;
// thread = one column and kBpRows rows 4 apart. Geometries with unit bins
// (g.unit) take the two-bin path, the others the general one; ALL_UNIT
// (every geometry of the launch has unit bins) compiles the general path
// out. Per-thread partials of the epilogue are summed over its rows in row
// order, then over the lanes (fixed tree) and the 4 warps in order.
// ---------------------------------------------------------------------------
constexpr int kBpRows = 8;
constexpr int kBpWarps = 32 / kBpRows;

// Unit-bin sums of one thread's kBpRows pixels (column xo, rows yo0 + 4r),
// two angles per compensated step (their contributions are added, rounded
// explicitly, before the step). QPAIR (an even number of equiangular angles:
// angle a + m/2 is angle a turned by a quarter, (c, s) -> (-s, c) exactly in
// the table) pairs a with a + m/2: the pair shares its chord constants and
// the second angle's split trigonometry follows from the first's; otherwise
// a pairs with a + 1.
// At each angle the candidates are the two bins nearest tau: t = m0, m0 + 1
// with m0 = rint(tau - 1/2) (odd D: bins at integers) or t = m0 -+ 1/2 with
// m0 = rint(tau) (even D). The support half-width is at most sqrt(1/2), so
// every bin with a nonzero weight is one of them whatever the rounding of
// tau. Adding 1.5 * 2^23 rounds to an integer without the conversion pipe:
// the sum's low mantissa bits hold m0 and subtracting the constant again
// gives it as an exact float. The half is taken off the exact head ph (odd D)
// before the sum, so both parities cost the same; t - tau is exact up to the
// one rounding of the tail pc (split trigonometry).
// COVERED: both candidates always lie on the detector (GeomDev::unit == 2).
template <bool COVERED, bool QPAIR, class TS>
__device__ __forceinline__ void bp_unit_sums(const GeomDev &g, const TS *__restrict__ sg, float xo, float yo0,
                                             float (&s)[kBpRows], float (&cmp)[kBpRows])
{
    constexpr float kRound = 12582912.f;   // 1.5 * 2^23
    constexpr int kRoundBits = 0x4B400000;
    const int m = g.m, D = g.D;
    const bool odd = D & 1;
    const float e = odd ? 0.5f : 0.f;
    // bin of t = m0 (odd D) or m0 - 1/2 (even D), m0 in the mantissa bits
    const int kofs = odd ? (D - 1) / 2 : D / 2 - 1;
    const int npair = QPAIR ? m / 2 : (m + 1) / 2;
    const float dy = (float)kBpWarps;
    for (int pr = 0; pr < npair; ++pr) {
        const int a0 = QPAIR ? pr : 2 * pr;
        const bool two = QPAIR || a0 + 1 < m;
        const int a1 = QPAIR ? pr + m / 2 : (two ? a0 + 1 : a0);
        // (chi, clo, shi, slo) and (wa, wb, lmax, flags) of both angles
        const float4 *q0 = reinterpret_cast<const float4 *>(g.angf + a0);
        const float4 t0 = __ldg(q0), c0 = __ldg(q0 + 1);
        float4 t1, c1;
        if (QPAIR) {
            t1 = make_float4(-t0.z, -t0.w, t0.x, t0.y);
            c1 = c0;
        } else {
            const float4 *q1 = reinterpret_cast<const float4 *>(g.angf + a1);
            t1 = __ldg(q1);
            c1 = __ldg(q1 + 1);
        }
        const float l0 = c0.z, l1 = two ? c1.z : 0.f;   // a missing second angle weighs 0
        // the second angle's row: its own, or (no second angle) the first's
        const TS *row0 = sg + ((int64_t)a0 * D + kofs - kRoundBits);
        const TS *row1 = sg + ((int64_t)a1 * D + kofs - kRoundBits);
        float ph0 = __fmaf_rn(xo, t0.x, yo0 * t0.z) - e, pc0 = __fmaf_rn(xo, t0.y, yo0 * t0.w);
        float ph1 = __fmaf_rn(xo, t1.x, yo0 * t1.z) - e, pc1 = __fmaf_rn(xo, t1.y, yo0 * t1.w);
        const float dph0 = dy * t0.z, dpc0 = dy * t0.w, dph1 = dy * t1.z, dpc1 = dy * t1.w;
#pragma unroll
        for (int r = 0; r < kBpRows; ++r) {
            const float y0 = __fadd_rn(ph0, pc0) + kRound;
            const float y1 = __fadd_rn(ph1, pc1) + kRound;
            const int b0 = __float_as_int(y0), b1 = __float_as_int(y1);   // m0 + kRoundBits
            const float d0 = (((__fadd_rn(y0, -kRound) - ph0) - 0.5f) - pc0);
            const float d1 = (((__fadd_rn(y1, -kRound) - ph1) - 0.5f) - pc1);
            const float wa0 = chord_n(c0.x, c0.y, fabsf(d0)), wb0 = chord_n(c0.x, c0.y, fabsf(d0 + 1.f));
            const float wa1 = chord_n(c1.x, c1.y, fabsf(d1)), wb1 = chord_n(c1.x, c1.y, fabsf(d1 + 1.f));
            bool o00 = true, o01 = true, o10 = true, o11 = true;
            if (!COVERED) {
                const int k0 = b0 - kRoundBits + kofs, k1 = b1 - kRoundBits + kofs;
                o00 = (unsigned)k0 < (unsigned)D; o01 = (unsigned)(k0 + 1) < (unsigned)D;
                o10 = (unsigned)k1 < (unsigned)D; o11 = (unsigned)(k1 + 1) < (unsigned)D;
            }
            const float u0 = o00 ? ld_op(row0 + b0) : 0.f, u1 = o01 ? ld_op(row0 + b0 + 1) : 0.f;
            const float v0 = o10 ? ld_op(row1 + b1) : 0.f, v1 = o11 ? ld_op(row1 + b1 + 1) : 0.f;
            // explicit rounding: no contraction into the Kahan step
            float rs;
            if (QPAIR) {
                const float x0 = __fmaf_rn(wa0, u0, __fmul_rn(wb0, u1));
                rs = __fmul_rn(__fmaf_rn(wa1, v0, __fmaf_rn(wb1, v1, x0)), l0);
            } else {
                const float x0 = __fmaf_rn(wa0, u0, __fmul_rn(wb0, u1));
                const float x1 = __fmaf_rn(wa1, v0, __fmul_rn(wb1, v1));
                rs = __fmaf_rn(x0, l0, __fmul_rn(x1, l1));
            }
            const float yk = rs - cmp[r];
            const float tt = s[r] + yk;
            cmp[r] = (tt - s[r]) - yk;
            s[r] = tt;
            ph0 += dph0; pc0 += dpc0; ph1 += dph1; pc1 += dpc1;
        }
    }
}

// The quarter-turn pairs of bp_unit_sums with the two angles' candidate and
// distance arithmetic, and the compensated steps of rows r, r + 1, in paired
// FP32 instructions (two IEEE single-precision operations, each rounded to
// nearest, per instruction): every value is the one bp_unit_sums<COVERED,
// true> computes, in fewer instructions.
template <bool COVERED, class TS>
__device__ __forceinline__ void bp_unit_sums_qpair(const GeomDev &g, const TS *__restrict__ sg, float xo,
                                                   float yo0, float (&s)[kBpRows], float (&cmp)[kBpRows])
{
    constexpr float kRound = 12582912.f;   // 1.5 * 2^23
    constexpr int kRoundBits = 0x4B400000;
    const int m = g.m, D = g.D;
    const bool odd = D & 1;
    const float e = odd ? 0.5f : 0.f;
    const int kofs = odd ? (D - 1) / 2 : D / 2 - 1;
    const float dy = (float)kBpWarps;
    const float2 kr2 = make_float2(kRound, kRound), nkr2 = make_float2(-kRound, -kRound);
    const float2 m1 = make_float2(-1.f, -1.f), mh = make_float2(-0.5f, -0.5f), one = make_float2(1.f, 1.f);
    float2 s2[kBpRows / 2], c2[kBpRows / 2];
#pragma unroll
    for (int r = 0; r < kBpRows / 2; ++r) {
        s2[r] = make_float2(s[2 * r], s[2 * r + 1]);
        c2[r] = make_float2(cmp[2 * r], cmp[2 * r + 1]);
    }
    for (int pr = 0; pr < m / 2; ++pr) {
        const int a0 = pr, a1 = pr + m / 2;
        const float4 *q0 = reinterpret_cast<const float4 *>(g.angf + a0);
        const float4 t0 = __ldg(q0), c0 = __ldg(q0 + 1);
        const float4 t1 = make_float4(-t0.z, -t0.w, t0.x, t0.y);
        const float l0 = c0.z;
        const TS *row0 = sg + ((int64_t)a0 * D + kofs - kRoundBits);
        const TS *row1 = sg + ((int64_t)a1 * D + kofs - kRoundBits);
        float2 ph = make_float2(__fmaf_rn(xo, t0.x, yo0 * t0.z) - e, __fmaf_rn(xo, t1.x, yo0 * t1.z) - e);
        float2 pc = make_float2(__fmaf_rn(xo, t0.y, yo0 * t0.w), __fmaf_rn(xo, t1.y, yo0 * t1.w));
        const float2 dph = make_float2(dy * t0.z, dy * t1.z), dpc = make_float2(dy * t0.w, dy * t1.w);
#pragma unroll
        for (int r2 = 0; r2 < kBpRows / 2; ++r2) {
            float rs[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 y = __fadd2_rn(__fadd2_rn(ph, pc), kr2);
                const int b0 = __float_as_int(y.x), b1 = __float_as_int(y.y);    // m0 + kRoundBits
                // ((y - kRound) - ph - 1/2) - pc, each step rounded as in the scalar form
                float2 d = __ffma2_rn(ph, m1, __fadd2_rn(y, nkr2));
                d = __ffma2_rn(pc, m1, __fadd2_rn(d, mh));
                const float2 d1 = __fadd2_rn(d, one);
                const float wa0 = chord_n(c0.x, c0.y, fabsf(d.x)), wb0 = chord_n(c0.x, c0.y, fabsf(d1.x));
                const float wa1 = chord_n(c0.x, c0.y, fabsf(d.y)), wb1 = chord_n(c0.x, c0.y, fabsf(d1.y));
                bool o00 = true, o01 = true, o10 = true, o11 = true;
                if (!COVERED) {
                    const int k0 = b0 - kRoundBits + kofs, k1 = b1 - kRoundBits + kofs;
                    o00 = (unsigned)k0 < (unsigned)D; o01 = (unsigned)(k0 + 1) < (unsigned)D;
                    o10 = (unsigned)k1 < (unsigned)D; o11 = (unsigned)(k1 + 1) < (unsigned)D;
                }
                const float u0 = o00 ? ld_op(row0 + b0) : 0.f, u1 = o01 ? ld_op(row0 + b0 + 1) : 0.f;
                const float v0 = o10 ? ld_op(row1 + b1) : 0.f, v1 = o11 ? ld_op(row1 + b1 + 1) : 0.f;
                const float x0 = __fmaf_rn(wa0, u0, __fmul_rn(wb0, u1));
                rs[h] = __fmul_rn(__fmaf_rn(wa1, v0, __fmaf_rn(wb1, v1, x0)), l0);
                ph = __fadd2_rn(ph, dph);
                pc = __fadd2_rn(pc, dpc);
            }
            // compensated steps of rows 2 r2 and 2 r2 + 1 together
            const float2 yk = __ffma2_rn(c2[r2], m1, make_float2(rs[0], rs[1]));
            const float2 tt = __fadd2_rn(s2[r2], yk);
            c2[r2] = __ffma2_rn(yk, m1, __ffma2_rn(s2[r2], m1, tt));
            s2[r2] = tt;
        }
    }
#pragma unroll
    for (int r = 0; r < kBpRows / 2; ++r) {
        s[2 * r] = s2[r].x; s[2 * r + 1] = s2[r].y;
        cmp[2 * r] = c2[r].x; cmp[2 * r + 1] = c2[r].y;
    }
}

template <int EPI, bool ALL_UNIT, class TS>
__global__ void __launch_bounds__(32 * kBpWarps, 4)
k_backproject_f32(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
                  const int4 *__restrict__ tiles, int ntiles, BpArgs a)
{
    __shared__ double red[kBpWarps];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pb = P[tl.x];
        if (!slot_active(a.S, pb.slot)) continue;                  // CTA-uniform
        const TS *sg = static_cast<const TS *>(a.sino) + pb.sino;
        const GeomDev &g = G[pb.geom];
        const int n = g.n, m = g.m, D = g.D;
        const int ix = tl.z + tx;
        const float half_n = 0.5f * (float)n;
        const float xo = (float)ix + 0.5f - half_n;
        const float yo0 = (float)(tl.y + ty) + 0.5f - half_n;
        const bool unit = ALL_UNIT || g.unit;
        float s[kBpRows], cmp[kBpRows];
#pragma unroll
        for (int r = 0; r < kBpRows; ++r) { s[r] = 0.f; cmp[r] = 0.f; }
        if (unit) {
            const bool qp = g.qpair;
            if (g.unit == 2) {
                if (qp) bp_unit_sums_qpair<true, TS>(g, sg, xo, yo0, s, cmp);
                else bp_unit_sums<true, false, TS>(g, sg, xo, yo0, s, cmp);
            } else {
                if (qp) bp_unit_sums_qpair<false, TS>(g, sg, xo, yo0, s, cmp);
                else bp_unit_sums<false, false, TS>(g, sg, xo, yo0, s, cmp);
            }
        } else {
            const float hD = g.hDf, dt = g.dtf, t0 = g.t0f, inv_dt = 1.f / g.dtf;
            const float dy = (float)kBpWarps;
            for (int ang = 0; ang < m; ++ang) {
                const AngleF A = g.angf[ang];
                const bool axis = __float_as_int(A.flags) & 2;
                const int64_t roff = (int64_t)ang * D;
                float ph = __fmaf_rn(xo, A.chi, yo0 * A.shi);        // exact head of tau
                float pc = __fmaf_rn(xo, A.clo, yo0 * A.slo);        // rounded tail
                const float dph = dy * A.shi, dpc = dy * A.slo;
#pragma unroll
                for (int r = 0; r < kBpRows; ++r) {
                    const float hwb = A.hw * inv_dt;
                    const int k0 = __float2int_ru(((ph + pc) - t0) * inv_dt + hD - hwb);
                    const int nc = __float2int_rd(2.f * hwb) + 1;
                    float rs = 0.f;
                    for (int q = 0; q < nc; ++q) {
                        const int kk = k0 + q;
                        if ((unsigned)kk < (unsigned)D) {
                            const float tkk = __fmaf_rn((float)kk - hD, dt, t0);
                            const float wq = chord_f(A, axis, fabsf((tkk - ph) - pc));
                            rs = __fmaf_rn(wq, ld_op(sg + roff + kk), rs);
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
        }
        double part = 0.0;
        if (ix < n) {
#pragma unroll
            for (int r = 0; r < kBpRows; ++r) {
                const int iy = tl.y + ty + kBpWarps * r;
                if (iy < n)
                    part += bp_epilogue<float, EPI, TS>(g, pb, a, ix, iy, ((double)s[r] - (double)cmp[r]) * g.h);
            }
        }
        if (a.part) {
            part = warp_sum_fixed(part);
            if (tx == 0) red[ty] = part;
            __syncthreads();
            if (threadIdx.x == 0) {
                double v = 0.0;
                for (int i = 0; i < kBpWarps; ++i) v += red[i];
                // the problem's partial of this pixel tile
                const int ntx = (n + 31) / 32;
                a.part[a.part_base[tl.x] + (tl.y / 32) * ntx + tl.z / 32] = v;
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Backward, group tiles: tile = {first problem, iy0, ix0, kBpGroup} of the
// same 32 x 32 pixels of kBpGroup consecutive problems of one geometry with
// unit bins covering every tile (GeomDev::unit == 2) and quarter-turn angle
// pairs (GeomDev::qpair). Thread = one column and kBpRows rows 4 apart, as in
// the one-image tile; every image gets exactly the arithmetic of
// bp_unit_sums_qpair<true> (same candidates, weights, products, compensated
// steps and epilogue order), so a problem's bits do not depend on its tile.
// What the group shares is each pixel's candidate bins and weights, computed
// once for the group's images, and the sinogram values come from shared
// memory: per stage, kBgPairs angle pairs, the window of kBgW bins of each
// angle that the tile's pixels can reach (from the tile's corners), for
// every image, copied in by cp.async (zero fill off the detector), the
// values of an image pair interleaved so that one 64-bit read gives both;
// two stages, the copies of the next in flight while the current is summed.
// Within a warp the 32 columns' bins at one angle span fewer than 32 bins,
// so the reads are free of bank conflicts.
// ---------------------------------------------------------------------------
constexpr int kBgPairs = 8;                       // angle pairs per stage
constexpr int kBgW = 56;                          // window width (bins); the tile's reach is < 51
constexpr int kBgStageFloats = kBgPairs * 2 * kBpGroup * kBgW;
constexpr size_t kBgSmem = 2 * (size_t)kBgStageFloats * sizeof(float);

// 0 = fine; 1 = a candidate bin fell outside its staged window (a bound of
// the window width did not hold; the read was clamped into the window)
__device__ int g_bpg_error;

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// First bin of the window of angle a for the tile whose pixel centres span
// x in [xa, xa + 31], y in [ya, ya + 31] (pixel widths from the image centre):
// every candidate bin k = m0 + kofs, k + 1 of those pixels (m0 within one of
// floor(tau)) lies in [floor(tau_min) + kofs - 2, floor(tau_max) + kofs + 3].
__device__ __forceinline__ int bpg_window(const AngleF &A, float xa, float ya, int kofs)
{
    const float c = A.chi + A.clo, s = A.shi + A.slo;
    const float t00 = __fmaf_rn(xa, c, ya * s), t10 = __fmaf_rn(xa + 31.f, c, ya * s);
    const float t01 = __fmaf_rn(xa, c, (ya + 31.f) * s), t11 = __fmaf_rn(xa + 31.f, c, (ya + 31.f) * s);
    const float tmin = fminf(fminf(t00, t10), fminf(t01, t11));
    return (int)floorf(tmin) + kofs - 2;
}

template <int EPI>
__global__ void __launch_bounds__(32 * kBpWarps, kBpGroup == 8 ? 2 : 3)
k_backproject_f32_group(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
                        const int4 *__restrict__ tiles, int ntiles, BpArgs a)
{
    constexpr int NI = kBpGroup;
    constexpr float kRound = 12582912.f;   // 1.5 * 2^23
    constexpr int kRoundBits = 0x4B400000;
    extern __shared__ __align__(16) float win[];           // [stage][pair][angle][image pair][bin][2]
    __shared__ int kwin[2][2 * kBgPairs];
    __shared__ double red[NI][kBpWarps];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    bool bad = false;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        unsigned actm = 0;                                      // active images (bit b)
#pragma unroll
        for (int b = 0; b < NI; ++b) actm |= slot_active(a.S, P[tl.x + b].slot) ? 1u << b : 0u;
        if (!actm) continue;                                    // CTA-uniform
        const GeomDev &g = G[P[tl.x].geom];
        const int n = g.n, m = g.m, D = g.D;
        const int ix = tl.z + tx;
        const float half_n = 0.5f * (float)n;
        const float xo = (float)ix + 0.5f - half_n;
        const float yo0 = (float)(tl.y + ty) + 0.5f - half_n;
        const float xa = (float)tl.z + 0.5f - half_n, ya = (float)tl.y + 0.5f - half_n;
        const bool odd = D & 1;
        const float e = odd ? 0.5f : 0.f;
        const int kofs = odd ? (D - 1) / 2 : D / 2 - 1;
        const int npair = m / 2;
        const int nstage = (npair + kBgPairs - 1) / kBgPairs;
        // stage copies: warp ty takes the angles ty, ty + 4, ... of the stage
        // (one window each), all images, lanes the bins (coalesced); inactive
        // images are zero-filled
        int64_t sino_of[NI];
#pragma unroll
        for (int b = 0; b < NI; ++b) sino_of[b] = P[tl.x + b].sino;
        auto stage_copy = [&](int sidx, int buf) {
            float *dst = win + (size_t)buf * kBgStageFloats;
            const int pr0 = sidx * kBgPairs;
            for (int slot = ty; slot < 2 * kBgPairs; slot += kBpWarps) {     // slot = 2 * pair + angle of pair
                const int pr = pr0 + (slot >> 1);
                const bool have = pr < npair;
                const int ang = have ? ((slot & 1) ? pr + m / 2 : pr) : 0;
                const int k0 = have ? bpg_window(g.angf[ang], xa, ya, kofs) : 0;
                if (tx == 0) kwin[buf][slot] = k0;
#pragma unroll
                for (int b = 0; b < NI; ++b) {
                    const float *src = static_cast<const float *>(a.sino) + sino_of[b] + (int64_t)ang * D;
                    const bool on = have && ((actm >> b) & 1u);
                    // image b's values of this angle: bins at stride 2 in its pair's row
                    float *drow = dst + ((size_t)slot * (NI / 2) + (b >> 1)) * (2 * kBgW) + (b & 1);
                    for (int q = tx; q < kBgW; q += 32) {
                        const int k = k0 + q;
                        const bool valid = on && (unsigned)k < (unsigned)D;
                        cp_async4(drow + 2 * q, valid ? src + k : src, valid);
                    }
                }
            }
            cp_async_commit();
        };
        // sums and compensations of images 2 pr, 2 pr + 1 (x, y) and row r
        float2 s2[NI / 2][kBpRows], c2[NI / 2][kBpRows];
#pragma unroll
        for (int pr = 0; pr < NI / 2; ++pr)
#pragma unroll
            for (int r = 0; r < kBpRows; ++r) { s2[pr][r] = make_float2(0.f, 0.f); c2[pr][r] = s2[pr][r]; }
        const float dy = (float)kBpWarps;
        const float2 kr2 = make_float2(kRound, kRound), nkr2 = make_float2(-kRound, -kRound);
        const float2 m1 = make_float2(-1.f, -1.f), mh = make_float2(-0.5f, -0.5f), one = make_float2(1.f, 1.f);
        stage_copy(0, 0);
        for (int si = 0; si < nstage; ++si) {
            const int buf = si & 1;
            cp_async_wait_all();
            __syncthreads();                                    // stage si in place; stage si - 1 read by all
            if (si + 1 < nstage) stage_copy(si + 1, buf ^ 1);
            const float *wst = win + (size_t)buf * kBgStageFloats;
            const int np = min(kBgPairs, npair - si * kBgPairs);
            for (int pl = 0; pl < np; ++pl) {
                const int a0 = si * kBgPairs + pl;
                const float4 *q0 = reinterpret_cast<const float4 *>(g.angf + a0);
                const float4 t0 = __ldg(q0), c0 = __ldg(q0 + 1);
                const float4 t1 = make_float4(-t0.z, -t0.w, t0.x, t0.y);
                const float l0 = c0.z;
                const int kb0 = kofs - kRoundBits - kwin[buf][2 * pl];
                const int kb1 = kofs - kRoundBits - kwin[buf][2 * pl + 1];
                // the pair's two angles: rows of image pairs, (value of image 2 q, of 2 q + 1) per bin
                const float2 *w0p = reinterpret_cast<const float2 *>(wst + (size_t)(2 * pl) * NI * kBgW);
                const float2 *w1p = w0p + (NI / 2) * kBgW;
                float2 ph = make_float2(__fmaf_rn(xo, t0.x, yo0 * t0.z) - e, __fmaf_rn(xo, t1.x, yo0 * t1.z) - e);
                float2 pc = make_float2(__fmaf_rn(xo, t0.y, yo0 * t0.w), __fmaf_rn(xo, t1.y, yo0 * t1.w));
                const float2 dph = make_float2(dy * t0.z, dy * t1.z), dpc = make_float2(dy * t0.w, dy * t1.w);
#pragma unroll
                for (int r2 = 0; r2 < kBpRows / 2; ++r2) {
                    int i0[2], i1[2];
                    float wa0[2], wb0[2], wa1[2], wb1[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 y = __fadd2_rn(__fadd2_rn(ph, pc), kr2);
                        int l = __float_as_int(y.x) + kb0, l1 = __float_as_int(y.y) + kb1;
                        bad |= (unsigned)l > (unsigned)(kBgW - 2) || (unsigned)l1 > (unsigned)(kBgW - 2);
                        i0[h] = min(max(l, 0), kBgW - 2);
                        i1[h] = min(max(l1, 0), kBgW - 2);
                        float2 d = __ffma2_rn(ph, m1, __fadd2_rn(y, nkr2));
                        d = __ffma2_rn(pc, m1, __fadd2_rn(d, mh));
                        const float2 d1 = __fadd2_rn(d, one);
                        wa0[h] = chord_n(c0.x, c0.y, fabsf(d.x));
                        wb0[h] = chord_n(c0.x, c0.y, fabsf(d1.x));
                        wa1[h] = chord_n(c0.x, c0.y, fabsf(d.y));
                        wb1[h] = chord_n(c0.x, c0.y, fabsf(d1.y));
                        ph = __fadd2_rn(ph, dph);
                        pc = __fadd2_rn(pc, dpc);
                    }
                    // each image's products and compensated step are those of
                    // the one-image tile (rows paired there, images here: the
                    // same IEEE operations, each rounded to nearest)
                    const float2 l02 = make_float2(l0, l0);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 a0 = make_float2(wa0[h], wa0[h]), b0 = make_float2(wb0[h], wb0[h]);
                        const float2 a1 = make_float2(wa1[h], wa1[h]), b1 = make_float2(wb1[h], wb1[h]);
                        const int r = 2 * r2 + h;
#pragma unroll
                        for (int q = 0; q < NI / 2; ++q) {
                            const float2 *u = w0p + q * kBgW, *v = w1p + q * kBgW;
                            const float2 x0 = __ffma2_rn(a0, u[i0[h]], __fmul2_rn(b0, u[i0[h] + 1]));
                            const float2 rs = __fmul2_rn(__ffma2_rn(a1, v[i1[h]], __ffma2_rn(b1, v[i1[h] + 1], x0)), l02);
                            const float2 yk = __ffma2_rn(c2[q][r], m1, rs);
                            const float2 tt = __fadd2_rn(s2[q][r], yk);
                            c2[q][r] = __ffma2_rn(yk, m1, __ffma2_rn(s2[q][r], m1, tt));
                            s2[q][r] = tt;
                        }
                    }
                }
            }
        }
        // epilogues, image by image, in the one-image tile's order
#pragma unroll
        for (int b = 0; b < NI; ++b) {
            const ProbDev pb = P[tl.x + b];
            double part = 0.0;
            if (((actm >> b) & 1u) && ix < n) {
#pragma unroll
                for (int r = 0; r < kBpRows; ++r) {
                    const int iy = tl.y + ty + kBpWarps * r;
                    const float sv = (b & 1) ? s2[b >> 1][r].y : s2[b >> 1][r].x;
                    const float cv = (b & 1) ? c2[b >> 1][r].y : c2[b >> 1][r].x;
                    if (iy < n) part += bp_epilogue<float, EPI, float>(g, pb, a, ix, iy, ((double)sv - (double)cv) * g.h);
                }
            }
            if (a.part) {
                part = warp_sum_fixed(part);
                if (tx == 0) red[b][ty] = part;
            }
        }
        if (a.part) {
            __syncthreads();
            if (threadIdx.x < NI && ((actm >> threadIdx.x) & 1u)) {
                const int b = threadIdx.x;
                double v = 0.0;
                for (int i = 0; i < kBpWarps; ++i) v += red[b][i];
                const int ntx = (n + 31) / 32;
                a.part[a.part_base[tl.x + b] + (tl.y / 32) * ntx + tl.z / 32] = v;
            }
        }
        __syncthreads();                                        // window and red reused by the next tile
    }
    if (__any_sync(0xffffffffu, bad) && tx == 0) atomicExch(&g_bpg_error, 1);
}

bool launch_backproject_f32_group(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                                  const BpArgs &a, cudaStream_t st)
{
    if (ntiles <= 0) return true;
    if (a.bf16) return false;
    count_launches(1);
    const int grid = min(ntiles, num_sms() * 2);
#define WMG_BPG(E)                                                                                          \
    case E:                                                                                                 \
        ensure_dyn_smem((const void *)k_backproject_f32_group<E>, (int)kBgSmem);                            \
        k_backproject_f32_group<E><<<grid, 32 * kBpWarps, kBgSmem, st>>>(G, P, tiles, ntiles, a);           \
        break;
    switch (a.epi) {
        WMG_BPG(BP_STORE) WMG_BPG(BP_CGLS_S) WMG_BPG(BP_RESID) WMG_BPG(BP_POST)
        WMG_BPG(BP_APPLY_A) WMG_BPG(BP_SIRT) WMG_BPG(BP_GMRES_W) WMG_BPG(BP_ATB)
        default: break;
    }
#undef WMG_BPG
    return true;
}

int bpg_error_take()
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_bpg_error, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_bpg_error, &z, sizeof(int));
    }
    return v;
}

void launch_backproject_f32(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                            const BpArgs &a, bool unit, cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    const int grid = min(ntiles, num_sms() * 2 * (a.ctas_per_sm > 0 ? a.ctas_per_sm : 8));
#define WMG_BPF(E)                                                                                        \
    case E:                                                                                               \
        if (a.bf16) {                                                                                     \
            if (unit) k_backproject_f32<E, true, __nv_bfloat16><<<grid, 32 * kBpWarps, 0, st>>>(G, P, tiles, ntiles, a); \
            else k_backproject_f32<E, false, __nv_bfloat16><<<grid, 32 * kBpWarps, 0, st>>>(G, P, tiles, ntiles, a);    \
        } else if (unit) {                                                                                \
            k_backproject_f32<E, true, float><<<grid, 32 * kBpWarps, 0, st>>>(G, P, tiles, ntiles, a);   \
        } else {                                                                                          \
            k_backproject_f32<E, false, float><<<grid, 32 * kBpWarps, 0, st>>>(G, P, tiles, ntiles, a);  \
        }                                                                                                 \
        break;
    switch (a.epi) {
        WMG_BPF(BP_STORE) WMG_BPF(BP_CGLS_S) WMG_BPF(BP_RESID) WMG_BPF(BP_POST)
        WMG_BPF(BP_APPLY_A) WMG_BPF(BP_SIRT) WMG_BPF(BP_GMRES_W) WMG_BPF(BP_ATB)
        default: break;
    }
#undef WMG_BPF
}

void fill_angle_table(const double2 *cs, int m, int kernel, AngleF *out)
{
    for (int a = 0; a < m; ++a) {
        const double c = cs[a].x, s = cs[a].y;
        AngleF A{};
        const double ch = std::nearbyint(c * 4096.0) / 4096.0, sh = std::nearbyint(s * 4096.0) / 4096.0;
        A.chi = (float)ch; A.clo = (float)(c - ch); A.shi = (float)sh; A.slo = (float)(s - sh);
        const double al = std::fmax(std::fabs(c), std::fabs(s)), be = std::fmin(std::fabs(c), std::fabs(s));
        const bool steep = std::fabs(c) >= std::fabs(s), axis = be == 0.0;
        const double cc = steep ? c : s, ss = steep ? s : c;
        if (kernel == WMG_KERNEL_JOSEPH) {
            // weight (1 - d/al)/al = lmax sat(1 - d lmax): no step at the axes
            const double lm = 1.0 / al;
            A.hw = (float)al;
            A.inv_ab = (float)(lm * lm);
            A.hw_inv = (float)lm;
            A.lmax = (float)lm;
            A.hwx = 1.f;
            A.inv_cc = (float)(1.0 / cc);
            A.slope = (float)(ss / cc);
            A.inv_slope = ss != 0.0 ? (float)(cc / ss) : 0.f;
            const int flags = steep ? 1 : 0;
            std::memcpy(&A.flags, &flags, sizeof(int));
            A.wa = (float)lm;
            A.wb = 1.f;
            A.cc = (float)cc;
            out[a] = A;
            continue;
        }
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
