// projector.cu -- matrix-free forward projection q = W p and backprojection
// y = W^T r for 2D parallel-beam geometry (Section 2.1, eq. sys: w_ij is the
// length of ray i inside pixel j; the normal-equation operator W^T W of
// eq. sys_ne is applied as these two products, never formed).
//
// Weights are recomputed on the fly from the trapezoid law: for a line with
// unit normal (c, s), alpha = max(|c|,|s|), beta = min(|c|,|s|), the chord of
// a unit pixel whose centre is at distance d from the line is
//     L(d) = clamp((hw - d) / (alpha beta), 0, 1/alpha),  hw = (alpha+beta)/2
// and, for axis-aligned lines (beta = 0), 1 if d < 1/2, 1/2 if d = 1/2 (a line
// on a pixel edge shares the edge between the two pixels), 0 otherwise.
// All lengths are in pixel widths; the factor h = 1/n is applied once per
// output value.
//
// Forward: one CTA = 32 consecutive rays (one per lane) of one angle; the
// warps split the rows. Rays with |cos| >= |sin| walk the rows of the
// row-major image; the others walk the rows of the transposed copy, so both
// cases read consecutive pixels across a warp. Every row holds at most two
// pixels with a nonzero weight. The per-warp partial sums are combined in a
// fixed order: deterministic, no atomics.
//
// Backward: pixel driven, one CTA = 32 x 32 pixels (four per thread), loop
// over angles, at most floor((alpha+beta)/spacing)+1 bins per pixel and angle.
// The distance t - tau uses the same rounded products in both directions, so
// the two directions use bitwise identical weights.
#include <type_traits>

#include "kern_common.cuh"
#include "bp_epilogue.cuh"

namespace wmg {

// ---------------------------------------------------------------------------
// Forward projection
// ---------------------------------------------------------------------------
template <class T, int NW>
__global__ void __launch_bounds__(32 * NW)
k_project(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
          const int4 *__restrict__ tiles, int ntiles, PjArgs a)
{
    __shared__ double red[NW][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(a.S, pd.slot)) continue;
        const GeomDev &g = G[pd.geom];
        const int n = g.n, D = g.D, ang = tl.y, k = tl.z + lane;
        const bool valid = k < D;
        T c, s;
        load_cs(g, ang, c, s);
        const bool steep = fabs(c) >= fabs(s);
        const T cc = steep ? c : s, ss = steep ? s : c;
        const T *__restrict__ src = static_cast<const T *>(steep ? a.img : a.imgT) + pd.img;
        const Chord<T> ch = make_chord<T>(cc, ss, g.kernel);
        const T inv_cc = T(1) / cc;
        const T hwx = ch.hw / fabs(cc);
        const T half_n = T(0.5) * T(n);
        const T tk = ray_offset<T>(g, k);
        typename LineOf<T>::type line;
        make_line(g, ang, !steep, tk, line);
        // rows this lane's ray can touch (image x-range widened by one pixel)
        int lo = n, hi = -1;
        if (valid) {
            if (ss == T(0)) {
                if (fabs(tk * inv_cc) < half_n + T(1)) { lo = 0; hi = n - 1; }
            } else {
                const T xb = half_n + T(1);
                const T ya = (tk + xb * cc) / ss, yb = (tk - xb * cc) / ss;
                const T ymin = fmin(ya, yb), ymax = fmax(ya, yb);
                lo = max(0, (int)ceil(ymin + half_n - T(0.5)));
                hi = min(n - 1, (int)floor(ymax + half_n - T(0.5)));
            }
        }
        lo = warp_min(lo);
        hi = warp_max(hi);
        Accum<T> acc;
        if (lo <= hi) {
            const int rows = hi - lo + 1, per = (rows + NW - 1) / NW;
            const int r0 = lo + w * per, r1 = min(hi + 1, r0 + per);
            for (int iy = r0; iy < r1; ++iy) {
                const T yc = T(iy) + T(0.5) - half_n;
                const T xs = (tk - yc * ss) * inv_cc;          // crossing of the row centre line
                const int ix0 = (int)ceil(xs + half_n - T(0.5) - hwx);
                const T *__restrict__ row = src + (int64_t)iy * n;
                T rs = T(0);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int ix = ix0 + q;
                    if (valid && ix >= 0 && ix < n) {
                        const T xc = T(ix) + T(0.5) - half_n;
                        const T wgt = ch(fabs(line_dist(line, xc, yc)));
                        rs = fma_t(wgt, ldg_t(row + ix), rs);
                    }
                }
                acc.add(rs);
            }
        }
        red[w][lane] = acc.value();
        __syncthreads();
        if (w == 0) {
            double vd = 0.0;
#pragma unroll
            for (int i = 0; i < NW; ++i) vd += red[i][lane];
            const T v = (T)(vd * g.h);
            if (valid) static_cast<T *>(a.sino)[pd.sino + (int64_t)ang * D + k] = v;
            if (a.part) {
                double q2 = valid ? (double)v * (double)v : 0.0;
                q2 = warp_sum_fixed(q2);
                if (lane == 0) a.part[t] = q2;
            }
        }
        __syncthreads();
    }
}

template <class T>
void launch_project(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                    const PjArgs &a, cudaStream_t st)
{
    if (std::is_same<T, float>::value) {
        launch_project_f32(G, P, tiles, ntiles, a, st);
        return;
    }
    if (ntiles <= 0) return;
    count_launches(1);
    constexpr int NW = 8;
    const int grid = min(ntiles, num_sms() * (a.ctas_per_sm > 0 ? a.ctas_per_sm : 8));
    k_project<T, NW><<<grid, 32 * NW, 0, st>>>(G, P, tiles, ntiles, a);
}

// ---------------------------------------------------------------------------
// Backprojection with fused epilogues
// ---------------------------------------------------------------------------
template <class T, int EPI>
__global__ void __launch_bounds__(256)
k_backproject(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
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
        const T half_n = T(0.5) * T(n);
        const T xo = T(ix) + T(0.5) - half_n;
        T yo[4];
        Accum<T> acc[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) yo[r] = T(tl.y + ty + 8 * r) + T(0.5) - half_n;
        const T *__restrict__ sg = static_cast<const T *>(a.sino) + pd.sino;
        const T dt = T(g.dt), inv_dt = T(1) / T(g.dt), t0 = T(g.t0);
        const T hD = T(0.5) * T(D - 1);
        for (int ang = 0; ang < m; ++ang) {
            T c, s;
            load_cs(g, ang, c, s);
            const Chord<T> ch = make_chord<T>(c, s, g.kernel);
            const T hwb = ch.hw * inv_dt;
            const int ncand = (int)floor(T(2) * hwb) + 1;
            typename LineOf<T>::type line0, line;
            make_line(g, ang, false, T(0), line0);
            line = line0;
            const T *__restrict__ row = sg + (int64_t)ang * D;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const T tau = -line_dist(line0, xo, yo[r]);     // approximate, for the bin range
                const int k0 = (int)ceil((tau - t0) * inv_dt + hD - hwb);
                T rs = T(0);
                for (int q = 0; q < ncand; ++q) {
                    const int k = k0 + q;
                    if (k >= 0 && k < D) {
                        line.t = fma_t(T(k) - hD, dt, t0);
                        const T wgt = ch(fabs(line_dist(line, xo, yo[r])));
                        rs = fma_t(wgt, ldg_t(row + k), rs);
                    }
                }
                acc[r].add(rs);
            }
        }
        double part = 0.0;
        if (ix < n) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int iy = tl.y + ty + 8 * r;
                if (iy < n) part += bp_epilogue<T, EPI>(g, pd, a, ix, iy, acc[r].value() * g.h);
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

template <class T>
void launch_backproject(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                        const BpArgs &a, cudaStream_t st)
{
    if (std::is_same<T, float>::value) {
        launch_backproject_f32(G, P, tiles, ntiles, a, a.unit != 0, st);
        return;
    }
    if (ntiles <= 0) return;
    count_launches(1);
    const int grid = min(ntiles, num_sms() * (a.ctas_per_sm > 0 ? a.ctas_per_sm : 8));
#define WMG_BP_CASE(E) \
    case E: k_backproject<T, E><<<grid, 256, 0, st>>>(G, P, tiles, ntiles, a); break;
    switch (a.epi) {
        WMG_BP_CASE(BP_STORE)
        WMG_BP_CASE(BP_CGLS_S)
        WMG_BP_CASE(BP_RESID)
        WMG_BP_CASE(BP_POST)
        WMG_BP_CASE(BP_APPLY_A)
        WMG_BP_CASE(BP_SIRT)
        WMG_BP_CASE(BP_GMRES_W)
        WMG_BP_CASE(BP_ATB)
        default: break;
    }
#undef WMG_BP_CASE
}

// Count of nonzero weights (FP64 geometry), same walk as the forward kernel.
__global__ void __launch_bounds__(256)
k_count_nnz(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
            const int4 *__restrict__ tiles, int ntiles, unsigned long long *count)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const GeomDev &g = G[P[tl.x].geom];
        const int n = g.n, D = g.D, ang = tl.y, k = tl.z + lane;
        if (k >= D) continue;
        double c, s;
        load_cs(g, ang, c, s);
        const bool steep = fabs(c) >= fabs(s);
        const double cc = steep ? c : s, ss = steep ? s : c;
        const Chord<double> ch = make_chord<double>(cc, ss, g.kernel);
        const double hwx = ch.hw / fabs(cc), half_n = 0.5 * n;
        const double tk = ray_offset<double>(g, k);
        LineD line;
        make_line(g, ang, !steep, tk, line);
        unsigned long long cnt = 0;
        for (int iy = w; iy < n; iy += 8) {
            const double yc = iy + 0.5 - half_n;
            const int ix0 = (int)ceil((tk - yc * ss) / cc + half_n - 0.5 - hwx);
            for (int q = 0; q < 2; ++q) {
                const int ix = ix0 + q;
                if (ix >= 0 && ix < n && ch(fabs(line_dist(line, ix + 0.5 - half_n, yc))) > kNnzEps) ++cnt;
            }
        }
        atomicAdd(count, cnt);
    }
}

void launch_count_nnz(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                      unsigned long long *count, cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    k_count_nnz<<<min(ntiles, num_sms() * 8), 256, 0, st>>>(G, P, tiles, ntiles, count);
}

// ---------------------------------------------------------------------------
// 32 x 32 tiled transpose of the images of a tile list (backprojection tiles).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256)
k_transpose(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
            const int4 *__restrict__ tiles, int ntiles, const T *__restrict__ src,
            T *__restrict__ dst)
{
    __shared__ T tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        const int n = G[pd.geom].n;
        for (int r = 0; r < 4; ++r) {
            const int iy = tl.y + ty + 8 * r, ix = tl.z + tx;
            if (iy < n && ix < n) tile[ty + 8 * r][tx] = src[pd.img + (int64_t)iy * n + ix];
        }
        __syncthreads();
        for (int r = 0; r < 4; ++r) {
            const int ox = tl.z + ty + 8 * r, oy = tl.y + tx;   // dst[ox][oy] = src[oy][ox]
            if (ox < n && oy < n) dst[pd.img + (int64_t)ox * n + oy] = tile[tx][ty + 8 * r];
        }
        __syncthreads();
    }
}

template <class T>
void launch_transpose(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                      const void *src, void *dst, cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    const int grid = min(ntiles, num_sms() * 8);
    k_transpose<T><<<grid, 256, 0, st>>>(G, P, tiles, ntiles, static_cast<const T *>(src),
                                         static_cast<T *>(dst));
}

template void launch_project<float>(const GeomDev *, const ProbDev *, const int4 *, int,
                                    const PjArgs &, cudaStream_t);
template void launch_project<double>(const GeomDev *, const ProbDev *, const int4 *, int,
                                     const PjArgs &, cudaStream_t);
template void launch_backproject<float>(const GeomDev *, const ProbDev *, const int4 *, int,
                                        const BpArgs &, cudaStream_t);
template void launch_backproject<double>(const GeomDev *, const ProbDev *, const int4 *, int,
                                         const BpArgs &, cudaStream_t);
template void launch_transpose<float>(const GeomDev *, const ProbDev *, const int4 *, int,
                                      const void *, void *, cudaStream_t);
template void launch_transpose<double>(const GeomDev *, const ProbDev *, const int4 *, int,
                                       const void *, void *, cudaStream_t);

}  // namespace wmg
