// setup.cu -- leaf Galerkin matrices of the WMG hierarchy and their inverses
// (Section 3.1.3: the 4^(l-1) coarsest-level subproblems, solved exactly by
// Cholesky in the paper, Section 4.1).
//
// Leaf k's matrix is D_k = Q_k^T (W^T W + lambda I) Q_k = G_k^T G_k + lambda I
// with G_k = W Q_k (the paper's tall-and-skinny W I_{2h,id}^h, here never
// stored whole). Each column of Q_k is a 2^L x 2^L Walsh pattern
// (+-2^-L) on one pixel block, so G_k[ray, block] -- the ray's "profile"
// coefficient -- is the ray's intersection lengths inside the block weighted
// by the pattern's signs. Leaf k is the pattern pair (HY, HX) (row and column
// Walsh indices) with HY, HX the bit-reversed odd / even bits of k.
//
// The assembly runs over tiles of leaves and chunks of angles, in two passes
// per (tile, chunk):
//   1. profiles: for every (angle, block) and every ray that can cross the
//      block, the tile's coefficients. A ray crosses at most two pixels per
//      frame row (the image rows for |cos| >= |sin|, columns otherwise), so
//      the tile is "S masks along the frame columns x all B masks along the
//      frame rows" (sign of pixel (row, col) under masks (R, C):
//      (-1)^(popc(R & row) + popc(C & col))): h[row][j] = sum over the row's
//      pixels of sign x weight for each of the S column masks, then a fast
//      Walsh-Hadamard transform along the rows gives all B row masks
//      (2 + log2 B operations per coefficient);
//   2. pairs: for every block b1 and every block b2 >= b1 whose ray ranges
//      overlap at an angle, the sum over the shared rays of the products of
//      their coefficients, added to D[b1][b2] (FP64).
// Profiles and pair sums run in the operator precision (FP32 for F32 plans:
// a pair sum has at most ~1.5 B terms), D accumulates over angles in FP64.
// Every D entry is owned by one thread of one launch and the launches run in
// a fixed order, so the result is the same on every run.
// Then D_k += lambda I and every leaf is factorised (Cholesky, FP64, pivot
// test) and inverted (two triangular solves per column).
#include <climits>

#include "kern_common.cuh"

namespace wmg {

// Rays (bin indices) that can touch pixel block b at angle a: |t_k - tau_b|
// <= B (|c| + |s|) / 2, tau_b the block centre's offset.
__device__ __forceinline__ void block_ray_range(const GeomDev &g, int a, int b, int &klo, int &khi)
{
    const double2 cs = g.cs64[a];
    const int cy = b / g.nc, cx = b - cy * g.nc;
    const double half_n = 0.5 * g.n;
    const double bx = (cx + 0.5) * g.B - half_n, by = (cy + 0.5) * g.B - half_n;
    const double tau = bx * cs.x + by * cs.y;
    // the block's pixel centres lie within (B-1)(|c|+|s|)/2 of tau; a pixel's
    // weight reaches (|c|+|s|)/2 (strip) or max(|c|,|s|) (Joseph) further
    const double ac = fabs(cs.x), as = fabs(cs.y);
    const double hw = 0.5 * (g.B - 1) * (ac + as) + (g.kernel == WMG_KERNEL_JOSEPH ? fmax(ac, as) : 0.5 * (ac + as));
    const double u = (tau - g.t0) / g.dt + 0.5 * (g.D - 1);
    klo = max(0, (int)ceil(u - hw / g.dt - 1e-9));
    khi = min(g.D - 1, (int)floor(u + hw / g.dt + 1e-9));
}

__device__ __forceinline__ int spread_bits(int v, int L)
{
    int r = 0;
    for (int i = 0; i < L; ++i) r |= ((v >> i) & 1) << (2 * i);
    return r;
}
__device__ __forceinline__ int unspread_bits(int v, int L)
{
    int r = 0;
    for (int i = 0; i < L; ++i) r |= ((v >> (2 * i)) & 1) << i;
    return r;
}
__device__ __forceinline__ int bitrev_L(int u, int L) { return L ? (int)(__brev((unsigned)u) >> (32 - L)) : 0; }

// Tile-local coefficient index t of (column pattern j, row pattern T) and the
// (HY, HX) index c = HY * B + HX it stands for. Class 0 (|cos| >= |sin|):
// frame rows are image rows, so T = HY and HX = q0 + j, t = T * S + j.
// Class 1: frame rows are image columns, T = HX and HY = q0 + j, t = j * B + T.
__device__ __forceinline__ int tile_t(int cls, int j, int T, int S, int B) { return cls ? j * B + T : T * S + j; }
__device__ __forceinline__ int tile_c(int cls, int t, int q0, int S, int B)
{
    if (cls) { const int j = t / B, T = t - j * B; return (q0 + j) * B + T; }
    const int T = t / S, j = t - T * S;
    return T * B + q0 + j;
}

// Pass 1a. CTA = (angle al of the chunk, block b); thread = (ray, frame row).
// The ray's (at most) two pixels of the frame row inside the block:
// Fw[(((al * P + b) * R + kk) * B + row) * 2 + q] = weight x h / B (0 if none),
// Fc[...] = frame column (-1 if none). rng[al * P + b] = (klo, ray count).
template <class TG>
__global__ void __launch_bounds__(256)
k_leaf_footprint(const GeomDev *__restrict__ Gd, const int *__restrict__ alist, int na, int R,
                 int2 *__restrict__ rng, TG *__restrict__ Fw, signed char *__restrict__ Fc)
{
    const GeomDev &g = *Gd;
    const int P = g.P, B = g.B, n = g.n;
    for (int tile = blockIdx.x; tile < na * P; tile += gridDim.x) {
        const int al = tile / P, b = tile - al * P, a = alist[al];
        int klo, khi;
        block_ray_range(g, a, b, klo, khi);
        const int cnt = max(0, min(khi - klo + 1, R));
        if (threadIdx.x == 0) rng[tile] = make_int2(klo, cnt);
        const double2 cs = g.cs64[a];
        const bool steep = fabs(cs.x) >= fabs(cs.y);
        const double cc = steep ? cs.x : cs.y, ss = steep ? cs.y : cs.x;
        const Chord<double> ch = make_chord<double>(cc, ss, g.kernel);
        const double inv_cc = 1.0 / cc, hwx = ch.hw / fabs(cc), half_n = 0.5 * n;
        const int cy = b / g.nc, cx = b - cy * g.nc;
        const int fr0 = (steep ? cy : cx) * B, fx0 = (steep ? cx : cy) * B;
        const double scale = g.h / (double)B;                        // unit-square length x 2^-L
        for (int e = threadIdx.x; e < cnt * B; e += blockDim.x) {
            const int kk = e / B, row = e - kk * B;
            const double tk = ray_offset<double>(g, klo + kk);
            const int fr = fr0 + row;
            const double yc = fr + 0.5 - half_n;
            const double xs = (tk - yc * ss) * inv_cc;
            const int f0 = (int)ceil(xs + half_n - 0.5 - hwx);
            const int64_t o = (((int64_t)tile * R + kk) * B + row) * 2;
            for (int q = 0; q < 2; ++q) {
                const int fx = f0 + q;
                double w = 0.0;
                int col = -1;
                if (fx >= fx0 && fx < fx0 + B) {
                    const double xc = fx + 0.5 - half_n;
                    const LineD ln{tk, cc, ss};
                    w = ch(fabs(line_dist(ln, xc, yc)));
                    col = fx - fx0;
                }
                Fw[o + q] = (TG)(w * scale);
                Fc[o + q] = (signed char)col;
            }
        }
    }
}

// Pass 1b. One warp per ray: lane holds frame rows lane + 32 i (i < NR) and
// the S column masks q0 + j of the tile; h[i][j] = sum over the row's pixels
// of (-1)^popc(mask & column) w, then a Walsh-Hadamard transform along the
// rows (shuffles below 32 rows, registers above). Output coefficient (j, row
// mask r) goes to Gbuf[((al * P + b) * R + kk) * KT + tile_t(cls, j, r)].
template <class TG, int NR, int S>
__global__ void __launch_bounds__(256)
k_leaf_profiles(const GeomDev *__restrict__ Gd, int na, int cls, int q0, int R, int KT,
                const int2 *__restrict__ rng, const TG *__restrict__ Fw, const signed char *__restrict__ Fc,
                TG *__restrict__ Gbuf)
{
    const GeomDev &g = *Gd;
    const int P = g.P, B = g.B;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)na * P * R;
    for (int64_t wid = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); wid < nwarps;
         wid += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const int tile = (int)(wid / R), kk = (int)(wid - (int64_t)tile * R);
        if (kk >= rng[tile].y) continue;                              // warp-uniform
        const int64_t fo = ((int64_t)tile * R + kk) * B;
        TG h[NR][S];
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int row = lane + 32 * i;
            TG w0 = TG(0), w1 = TG(0);
            int c0 = -1, c1 = -1;
            if (row < B) {
                w0 = Fw[(fo + row) * 2]; w1 = Fw[(fo + row) * 2 + 1];
                c0 = Fc[(fo + row) * 2]; c1 = Fc[(fo + row) * 2 + 1];
            }
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const int mask = q0 + j;
                TG v = TG(0);
                if (c0 >= 0) v += (__popc(mask & c0) & 1) ? -w0 : w0;
                if (c1 >= 0) v += (__popc(mask & c1) & 1) ? -w1 : w1;
                h[i][j] = v;
            }
        }
        // butterflies across lanes (row distance < 32)
        for (int half = 1; half < 32 && half < B; half <<= 1) {
            const bool upper = lane & half;
#pragma unroll
            for (int i = 0; i < NR; ++i)
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    const TG o = __shfl_xor_sync(0xffffffffu, h[i][j], half);
                    h[i][j] = upper ? o - h[i][j] : h[i][j] + o;
                }
        }
        // butterflies within the lane (row distance 32 i)
#pragma unroll
        for (int hs = 1; hs < NR; hs <<= 1)
#pragma unroll
            for (int i = 0; i < NR; ++i)
                if (!(i & hs))
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        const TG u = h[i][j], v = h[i + hs][j];
                        h[i][j] = u + v;
                        h[i + hs][j] = u - v;
                    }
        TG *out = Gbuf + ((int64_t)tile * R + kk) * KT;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int r = lane + 32 * i;
            if (r < B)
#pragma unroll
                for (int j = 0; j < S; ++j) out[tile_t(cls, j, r, S, B)] = h[i][j];
        }
    }
}

template <class TG>
static void launch_profiles(int B, int S, const GeomDev *gd, int na, int cls, int q0, int R, int KT, int P,
                            const int2 *rng, const TG *Fw, const signed char *Fc, TG *Gbuf, cudaStream_t st)
{
    const int64_t warps = (int64_t)na * P * R;
    const int grid = (int)std::min<int64_t>((warps + 7) / 8, (int64_t)num_sms() * 16);
    count_launches(1);
#define WMG_PROF(NR_, S_) k_leaf_profiles<TG, NR_, S_><<<grid, 256, 0, st>>>(gd, na, cls, q0, R, KT, rng, Fw, Fc, Gbuf)
    if (B == 128) WMG_PROF(4, 2);
    else if (B == 64) WMG_PROF(2, 4);
    else if (B == 32) WMG_PROF(1, 8);
    else if (B == 16) WMG_PROF(1, 16);
    else if (B == 8) WMG_PROF(1, 8);
    else if (B == 4) WMG_PROF(1, 4);
    else if (B == 2) WMG_PROF(1, 2);
    else WMG_PROF(1, 1);
#undef WMG_PROF
    (void)S;
}

// Four consecutive coefficients t .. t + 3 of a profile row (t a multiple
// of 4; entries at or past KT read as 0).
__device__ __forceinline__ void load4(const float *__restrict__ p, int t, int KT, float (&v)[4])
{
    if (t + 4 <= KT && !(KT & 3)) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p + t));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = t + j < KT ? __ldg(p + t + j) : 0.f;
    }
}
__device__ __forceinline__ void load4(const double *__restrict__ p, int t, int KT, double (&v)[4])
{
    if (t + 4 <= KT && !(KT & 3)) {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p + t));
        const double2 b = __ldg(reinterpret_cast<const double2 *>(p + t + 2));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = t + j < KT ? __ldg(p + t + j) : 0.0;
    }
}

// Pass 2. Thread = (block pair b1 <= b2, four consecutive coefficients of
// the tile); a warp takes 128 coefficients of one pair, so its loads of a
// ray's coefficients are 512 contiguous bytes per block. For each angle of
// the chunk the thread sums, over the rays the two blocks share (in
// ascending order, FP32 for F32 plans), the products of their coefficients
// and adds each sum to the pair's FP64 total, which is read from Dacc before
// the first angle and written back after the last: no shared memory, no
// barrier, no range test inside the ray loop. Every Dacc entry belongs to one
// thread of a launch; the launches run in a fixed order.
template <class TG>
__global__ void __launch_bounds__(256)
k_leaf_pairs(const GeomDev *__restrict__ Gd, const int2 *__restrict__ rng, int na, int cls, int q0, int S,
             int R, int KT, const TG *__restrict__ Gbuf, double *__restrict__ Dacc)
{
    const GeomDev &g = *Gd;
    const int P = g.P, B = g.B, K = g.K;
    const int lane = threadIdx.x & 31;
    const int halves = (KT + 127) / 128;                          // warps per pair
    const int64_t ntasks = (int64_t)P * P * halves;
    const int wpb = blockDim.x >> 5;
    for (int64_t task = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); task < ntasks;
         task += (int64_t)gridDim.x * wpb) {
        const int h = (int)(task % halves);
        const int64_t pr = task / halves;
        const int b1 = (int)(pr / P), b2 = (int)(pr - (int64_t)b1 * P);
        if (b2 < b1) continue;                                     // each unordered pair once
        const int t = 4 * (h * 32 + lane);
        bool any = false;                                          // the pair shares a ray at some angle
        for (int al = 0; al < na && !any; ++al) {
            const int2 r1 = rng[al * P + b1], r2 = rng[al * P + b2];
            any = max(r1.x, r2.x) < min(r1.x + r1.y, r2.x + r2.y);
        }
        if (!any) continue;                                        // warp-uniform
        int cj[4];
        double d64[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            cj[j] = t + j < KT ? tile_c(cls, t + j, q0, S, B) : -1;
            d64[j] = cj[j] >= 0 ? Dacc[((int64_t)b1 * P + b2) * K + cj[j]] : 0.0;
        }
        for (int al = 0; al < na; ++al) {
            const int2 r1 = rng[al * P + b1], r2 = rng[al * P + b2];
            const int lo = max(r1.x, r2.x), hi = min(r1.x + r1.y, r2.x + r2.y);
            if (lo >= hi) continue;                                // warp-uniform
            const TG *p1 = Gbuf + (((int64_t)al * P + b1) * R + (lo - r1.x)) * KT;
            const TG *p2 = Gbuf + (((int64_t)al * P + b2) * R + (lo - r2.x)) * KT;
            TG acc[4] = {TG(0), TG(0), TG(0), TG(0)};
            const int nk = hi - lo;
            int k = 0;
            for (; k + 2 <= nk; k += 2) {                          // two rays' loads in flight
                TG u0[4], v0[4], u1[4], v1[4];
                load4(p1 + (int64_t)k * KT, t, KT, u0);
                load4(p2 + (int64_t)k * KT, t, KT, v0);
                load4(p1 + (int64_t)(k + 1) * KT, t, KT, u1);
                load4(p2 + (int64_t)(k + 1) * KT, t, KT, v1);
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j] = fma_t(u0[j], v0[j], acc[j]);
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j] = fma_t(u1[j], v1[j], acc[j]);
            }
            if (k < nk) {
                TG u0[4], v0[4];
                load4(p1 + (int64_t)k * KT, t, KT, u0);
                load4(p2 + (int64_t)k * KT, t, KT, v0);
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j] = fma_t(u0[j], v0[j], acc[j]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) d64[j] += (double)acc[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (cj[j] >= 0) Dacc[((int64_t)b1 * P + b2) * K + cj[j]] = d64[j];
    }
}

// D_k + lambda I gathered from Dacc (upper triangle, layout [b1][b2][c]),
// Cholesky D_k = L L^T (left looking, FP64) in a per-CTA work matrix M
// stored by columns of L (M[q * P + i] = L[i][q]: thread i's loads are
// consecutive across threads), pivot test, then the inverse columns by two
// triangular solves (thread c owns column c of Y; the factor entries it
// reads are the same for every thread; only the lower triangle of the
// symmetric inverse is solved, the upper one is its mirror image). One CTA
// per leaf. status[k] = 0 ok,
// -1 if a pivot is not positive.
template <class T>
__global__ void __launch_bounds__(256)
k_leaf_invert(const GeomDev *__restrict__ Gd, const double *__restrict__ Dacc, double *__restrict__ Mwork,
              double *__restrict__ Ywork, T *__restrict__ inv, int *__restrict__ status)
{
    __shared__ double colbuf[256];
    __shared__ int bad;
    const GeomDev &g = *Gd;
    const int P = g.P, K = g.K, L = g.L, B = g.B;
    for (int k = blockIdx.x; k < K; k += gridDim.x) {
        double *M = Mwork + (int64_t)blockIdx.x * P * P;
        double *Y = Ywork + (int64_t)blockIdx.x * P * P;
        const int HY = bitrev_L(unspread_bits(k >> 1, L), L), HX = bitrev_L(unspread_bits(k, L), L);
        const int c = HY * B + HX;
        if (threadIdx.x == 0) bad = 0;
        for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
            const int q = e / P, i = e - q * P;
            const int lo = min(i, q), hi = max(i, q);
            M[e] = Dacc[((int64_t)lo * P + hi) * K + c] + (i == q ? g.lambda : 0.0);
        }
        __syncthreads();
        // column j: L[i][j] = (A[i][j] - sum_q L[i][q] L[j][q]) / sqrt(pivot), i >= j
        for (int j = 0; j < P; ++j) {
            for (int i = j + threadIdx.x; i < P; i += blockDim.x) {
                double v = M[(int64_t)j * P + i];
                for (int q = 0; q < j; ++q) v -= M[(int64_t)q * P + i] * M[(int64_t)q * P + j];
                colbuf[i] = v;
            }
            __syncthreads();
            const double piv = colbuf[j];
            if (!(piv > 0.0)) {
                if (threadIdx.x == 0) bad = 1;
            }
            const double d = piv > 0.0 ? sqrt(piv) : 1.0;
            for (int i = j + threadIdx.x; i < P; i += blockDim.x)
                M[(int64_t)j * P + i] = (i == j) ? d : colbuf[i] / d;
            __syncthreads();
        }
        if (threadIdx.x == 0) status[k] = bad ? -1 : 0;
        const int col = threadIdx.x;
        if (col < P) {
            // L y = e_col: y is 0 above row col, so the sums start there
            for (int i = col; i < P; ++i) {
                double y = (i == col) ? 1.0 : 0.0;
                for (int q = col; q < i; ++q) y -= M[(int64_t)q * P + i] * Y[(int64_t)q * P + col];
                Y[(int64_t)i * P + col] = y / M[(int64_t)i * P + i];
            }
            // L^T x = y for the rows i >= col only: the inverse is symmetric,
            // its lower triangle is solved and the upper one mirrors it
            for (int i = P - 1; i >= col; --i) {
                double x = Y[(int64_t)i * P + col];
                for (int q = i + 1; q < P; ++q) x -= M[(int64_t)i * P + q] * Y[(int64_t)q * P + col];
                x /= M[(int64_t)i * P + i];
                Y[(int64_t)i * P + col] = x;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
            const int i = e / P, j = e - i * P;
            inv[(int64_t)k * P * P + e] = (T)Y[(int64_t)max(i, j) * P + min(i, j)];
        }
        __syncthreads();
    }
}

// Host driver: assembles, factorises and inverts every leaf of one geometry.
// `fp32` (F32 plans): profiles and pair sums in FP32 and the inverses stored
// as K*P*P floats in `leafinv_out`; else FP64 throughout and K*P*P doubles.
// The Cholesky factorisation and the triangular solves are FP64 in both.
template <class TG>
static int32_t assemble(const GeomDev &gh, const GeomDev *gd, double *Dacc, cudaStream_t st)
{
    const int P = gh.P, K = gh.K, B = gh.B;
    // rays per block: at most ((B-1) sqrt 2 + 2) / dt + 1 (Joseph), B sqrt 2 / dt + 1 (strip)
    const int R = (int)floor(gh.B * 1.4142135623730951 / gh.dt) + 4;
    const int KT = std::min(K, 256), S = KT / B;
    // angle classes from the FP64 table (|cos| >= |sin|: class 0)
    std::vector<double2> cs(gh.m);
    WMG_CUDA(cudaMemcpyAsync(cs.data(), gh.cs64, gh.m * sizeof(double2), cudaMemcpyDeviceToHost, st));
    WMG_CUDA(cudaStreamSynchronize(st));
    std::vector<int> lists[2];
    for (int a = 0; a < gh.m; ++a) lists[std::fabs(cs[a].x) >= std::fabs(cs[a].y) ? 0 : 1].push_back(a);
    // angle chunk: about 96 MB of profiles (L2-sized); the chunk's
    // footprints are computed once and serve every leaf tile
    const double per_angle = (double)P * R * KT * sizeof(TG);
    const int chunk = (int)std::max(1.0, std::min((double)gh.m, 96.0 * 1024 * 1024 / per_angle));
    TG *Gbuf = nullptr, *Fw = nullptr;
    signed char *Fc = nullptr;
    int2 *rng = nullptr;
    int *dlist = nullptr;
    // stream-ordered scratch: no device-wide synchronisation on free, so
    // setups on other streams and the solves keep running
    auto cleanup = [&]() {
        cudaFreeAsync(Gbuf, st); cudaFreeAsync(Fw, st); cudaFreeAsync(Fc, st); cudaFreeAsync(rng, st);
        cudaFreeAsync(dlist, st);
    };
    const size_t nfoot = (size_t)chunk * P * R * B * 2;
    if (cudaMallocAsync(&Gbuf, (size_t)chunk * P * R * KT * sizeof(TG), st) != cudaSuccess ||
        cudaMallocAsync(&Fw, nfoot * sizeof(TG), st) != cudaSuccess || cudaMallocAsync(&Fc, nfoot, st) != cudaSuccess ||
        cudaMallocAsync(&rng, (size_t)chunk * P * sizeof(int2), st) != cudaSuccess ||
        cudaMallocAsync(&dlist, (size_t)gh.m * sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(WMG_ERR_OOM, "leaf setup: device allocation failed");
    }
    const int64_t pair_warps = (int64_t)P * P * ((KT + 127) / 128);
    const int pair_grid = (int)std::min<int64_t>((pair_warps + 7) / 8, (int64_t)num_sms() * 64);
    int off = 0;
    for (int cls = 0; cls < 2; ++cls) {
        const std::vector<int> &lst = lists[cls];
        if (lst.empty()) continue;
        WMG_CUDA(cudaMemcpyAsync(dlist + off, lst.data(), lst.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        for (int c0 = 0; c0 < (int)lst.size(); c0 += chunk) {
            const int na = std::min(chunk, (int)lst.size() - c0);
            count_launches(1);
            k_leaf_footprint<TG><<<std::min(na * P, num_sms() * 16), 256, 0, st>>>(gd, dlist + off + c0, na, R,
                                                                                   rng, Fw, Fc);
            for (int q0 = 0; q0 < B; q0 += S) {
                launch_profiles<TG>(B, S, gd, na, cls, q0, R, KT, P, rng, Fw, Fc, Gbuf, st);
                count_launches(1);
                k_leaf_pairs<TG><<<pair_grid, 256, 0, st>>>(gd, rng, na, cls, q0, S, R, KT, Gbuf, Dacc);
            }
        }
        off += (int)lst.size();
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();              // a launch that did not start
    cleanup();
    if (e != cudaSuccess) return fail(WMG_ERR_CUDA, std::string("leaf setup: ") + cudaGetErrorString(e));
    return WMG_OK;
}

int32_t build_leaf_inverses(const GeomDev &gh, const GeomDev *gd, void *leafinv_out, bool fp32,
                            cudaStream_t st)
{
    const int P = gh.P, K = gh.K;
    const int inv_ctas = std::min(K, num_sms() * 4);
    double *Dacc = nullptr, *A = nullptr, *Y = nullptr;
    int *status = nullptr;
    auto cleanup = [&]() {
        cudaFreeAsync(Dacc, st); cudaFreeAsync(A, st); cudaFreeAsync(Y, st); cudaFreeAsync(status, st);
    };
    if (cudaMallocAsync(&Dacc, (size_t)K * P * P * sizeof(double), st) != cudaSuccess ||
        cudaMallocAsync(&A, (size_t)inv_ctas * P * P * sizeof(double), st) != cudaSuccess ||
        cudaMallocAsync(&Y, (size_t)inv_ctas * P * P * sizeof(double), st) != cudaSuccess ||
        cudaMallocAsync(&status, (size_t)K * sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(WMG_ERR_OOM, "leaf setup: device allocation failed");
    }
    cudaMemsetAsync(Dacc, 0, (size_t)K * P * P * sizeof(double), st);
    int32_t rc = fp32 ? assemble<float>(gh, gd, Dacc, st) : assemble<double>(gh, gd, Dacc, st);
    if (rc) { cleanup(); return rc; }
    count_launches(1);
    if (fp32) k_leaf_invert<float><<<inv_ctas, 256, 0, st>>>(gd, Dacc, A, Y, static_cast<float *>(leafinv_out), status);
    else k_leaf_invert<double><<<inv_ctas, 256, 0, st>>>(gd, Dacc, A, Y, static_cast<double *>(leafinv_out), status);
    std::vector<int> hs(K);
    cudaError_t e = cudaGetLastError();                         // a launch that did not start
    cudaMemcpyAsync(hs.data(), status, (size_t)K * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        rc = fail(WMG_ERR_CUDA, std::string("leaf setup: ") + cudaGetErrorString(e));
    } else {
        for (int k = 0; k < K; ++k)
            if (hs[k] != 0) {
                rc = fail(WMG_ERR_LEAF_NOT_SPD, "leaf " + std::to_string(k) +
                                                    " matrix is not positive definite");
                break;
            }
    }
    cleanup();
    return rc;
}


}  // namespace wmg
