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
