// setup.cu -- leaf Galerkin matrices of the WMG hierarchy and their inverses
// (Section 3.1.3: the 4^(l-1) coarsest-level subproblems, solved exactly by
// Cholesky in the paper, Section 4.1).
//
// Leaf k's matrix is D_k = Q_k^T (W^T W + lambda I) Q_k = G_k^T G_k + lambda I
// with G_k = W Q_k (the paper's tall-and-skinny W I_{2h,id}^h, here never
// stored whole). Each column of Q_k is a 2^L x 2^L Walsh pattern
// (+-2^-L) on one pixel block, so G_k[ray, block] is the ray's intersection
// lengths inside the block weighted by the pattern's signs. The assembly runs
// per chunk of angles in two deterministic passes:
//   1. for every (angle, block) and every ray that can cross the block, the
//      K leaf coefficients of the ray's weights inside the block;
//   2. for every pair of blocks (b1 <= b2) and every leaf, the sum over the
//      chunk's rays that cross both blocks, added to D_k[b1][b2] in FP64.
// Then D_k += lambda I and every leaf is factorised (Cholesky, FP64, pivot
// test) and inverted (two triangular solves per column), the inverse
// rounded to the operator precision.
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
    const double hw = 0.5 * g.B * (fabs(cs.x) + fabs(cs.y));
    const double u = (tau - g.t0) / g.dt + 0.5 * (g.D - 1);
    klo = max(0, (int)ceil(u - hw / g.dt - 1e-9));
    khi = min(g.D - 1, (int)floor(u + hw / g.dt + 1e-9));
}

__device__ __forceinline__ int unspread_bits(int v, int L)
{
    int r = 0;
    for (int i = 0; i < L; ++i) r |= ((v >> (2 * i)) & 1) << i;
    return r;
}
__device__ __forceinline__ int bitrev_L(int u, int L) { return L ? (int)(__brev((unsigned)u) >> (32 - L)) : 0; }

// Pass 1. tile = {angle a (absolute), block b, 0, 0}; writes
// Gbuf[((a - a0) * P + b) * R + (k - klo)) * K + leaf].
__global__ void __launch_bounds__(256)
k_leaf_coeffs(const GeomDev *__restrict__ Gd, int a0, int na, int R, double *__restrict__ Gbuf)
{
    __shared__ double wv[2 * 128];
    __shared__ int wl[2 * 128];
    const GeomDev &g = *Gd;
    const int P = g.P, K = g.K, B = g.B, L = g.L, n = g.n;
    const int ntiles = na * P;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int al = t / P, b = t - al * P, a = a0 + al;
        int klo, khi;
        block_ray_range(g, a, b, klo, khi);
        const double2 cs = g.cs64[a];
        const bool steep = fabs(cs.x) >= fabs(cs.y);
        const double cc = steep ? cs.x : cs.y, ss = steep ? cs.y : cs.x;
        const Chord<double> ch = make_chord<double>(cc, ss);
        const double hwx = ch.hw / fabs(cc), half_n = 0.5 * n;
        const int cy = b / g.nc, cx = b - cy * g.nc;
        const int fr0 = (steep ? cy : cx) * B, fx0 = (steep ? cx : cy) * B;
        for (int k = klo; k <= khi && k - klo < R; ++k) {
            const double tk = ray_offset<double>(g, k);
            if (threadIdx.x < B) {                       // one frame row per thread
                const int fr = fr0 + threadIdx.x;
                const double yc = fr + 0.5 - half_n;
                const double xs = (tk - yc * ss) / cc;
                const int f0 = (int)ceil(xs + half_n - 0.5 - hwx);
                for (int q = 0; q < 2; ++q) {
                    const int fx = f0 + q;
                    double w = 0.0;
                    int loc = 0;
                    if (fx >= fx0 && fx < fx0 + B) {
                        const double xc = fx + 0.5 - half_n;
                        const LineD ln{tk, cc, ss};
                        w = ch(fabs(line_dist(ln, xc, yc)));
                        const int ly = steep ? fr - fr0 : fx - fx0;
                        const int lx = steep ? fx - fx0 : fr - fr0;
                        loc = (ly << 8) | lx;
                    }
                    wv[2 * threadIdx.x + q] = w;
                    wl[2 * threadIdx.x + q] = loc;
                }
            }
            __syncthreads();
            const double scale = g.h / (double)B;        // unit-square length x 2^-L
            for (int leaf = threadIdx.x; leaf < K; leaf += blockDim.x) {
                const int HY = bitrev_L(unspread_bits(leaf >> 1, L), L);
                const int HX = bitrev_L(unspread_bits(leaf, L), L);
                double acc = 0.0;
                for (int e = 0; e < 2 * B; ++e) {
                    const double w = wv[e];
                    if (w != 0.0) {
                        const int loc = wl[e];
                        const int par = (__popc(HY & (loc >> 8)) + __popc(HX & (loc & 255))) & 1;
                        acc += par ? -w : w;
                    }
                }
                Gbuf[(((int64_t)al * P + b) * R + (k - klo)) * K + leaf] = acc * scale;
            }
            __syncthreads();
        }
    }
}

// Pass 2. tile = pair index over b1 <= b2 (row-major upper triangle).
__global__ void k_leaf_gram(const GeomDev *__restrict__ Gd, int a0, int na, int R,
                            const double *__restrict__ Gbuf, const int2 *__restrict__ pairs,
                            int npairs, double *__restrict__ Dm)
{
    const GeomDev &g = *Gd;
    const int P = g.P, K = g.K;
    for (int t = blockIdx.x; t < npairs; t += gridDim.x) {
        const int2 pr = pairs[t];
        const int b1 = pr.x, b2 = pr.y;
        for (int leaf0 = 0; leaf0 < K; leaf0 += blockDim.x) {
            const int leaf = leaf0 + threadIdx.x;
            double acc = 0.0;
            for (int al = 0; al < na; ++al) {
                int l1, h1, l2, h2;
                block_ray_range(g, a0 + al, b1, l1, h1);
                block_ray_range(g, a0 + al, b2, l2, h2);
                h1 = min(h1, l1 + R - 1);
                h2 = min(h2, l2 + R - 1);
                const int lo = max(l1, l2), hi = min(h1, h2);
                if (leaf < K)
                    for (int k = lo; k <= hi; ++k) {
                        const double g1 = Gbuf[(((int64_t)al * P + b1) * R + (k - l1)) * K + leaf];
                        const double g2 = Gbuf[(((int64_t)al * P + b2) * R + (k - l2)) * K + leaf];
                        acc = __fma_rn(g1, g2, acc);
                    }
            }
            if (leaf < K) {
                double *Dk = Dm + (int64_t)leaf * P * P;
                Dk[(int64_t)b1 * P + b2] += acc;
                if (b1 != b2) Dk[(int64_t)b2 * P + b1] += acc;
            }
        }
    }
}

// D_k += lambda I, Cholesky D_k = L L^T in place (lower triangle, left
// looking, FP64), pivot test, then inverse columns by two triangular solves.
// One CTA per leaf. status[k] = 0 ok, -1 if a pivot is not positive.
template <class T>
__global__ void __launch_bounds__(256)
k_leaf_invert(const GeomDev *__restrict__ Gd, double *__restrict__ Dm, double *__restrict__ Ywork,
              T *__restrict__ inv, int *__restrict__ status)
{
    __shared__ double colbuf[256];
    __shared__ int bad;
    const GeomDev &g = *Gd;
    const int P = g.P;
    for (int k = blockIdx.x; k < g.K; k += gridDim.x) {
        double *A = Dm + (int64_t)k * P * P;
        double *Y = Ywork + (int64_t)blockIdx.x * P * P;
        if (threadIdx.x == 0) bad = 0;
        for (int i = threadIdx.x; i < P; i += blockDim.x) A[(int64_t)i * P + i] += g.lambda;
        __syncthreads();
        // left-looking Cholesky: column j = (A[j:, j] - L[j:, :j] L[j, :j]^T) / sqrt(pivot)
        for (int j = 0; j < P; ++j) {
            for (int i = j + threadIdx.x; i < P; i += blockDim.x) {
                double v = A[(int64_t)i * P + j];
                for (int q = 0; q < j; ++q) v -= A[(int64_t)i * P + q] * A[(int64_t)j * P + q];
                colbuf[i] = v;
            }
            __syncthreads();
            const double piv = colbuf[j];
            if (!(piv > 0.0)) {
                if (threadIdx.x == 0) bad = 1;
            }
            const double d = piv > 0.0 ? sqrt(piv) : 1.0;
            for (int i = j + threadIdx.x; i < P; i += blockDim.x)
                A[(int64_t)i * P + j] = (i == j) ? d : colbuf[i] / d;
            __syncthreads();
        }
        if (threadIdx.x == 0) status[k] = bad ? -1 : 0;
        // inverse: column c solves L y = e_c, then L^T x = y. Thread c owns
        // column c of the work matrix (coalesced across threads); the factor
        // entries are the same address for every thread (broadcast).
        const int c = threadIdx.x;
        if (c < P) {
            for (int i = 0; i < P; ++i) {
                double y = (i == c) ? 1.0 : 0.0;
                for (int q = 0; q < i; ++q) y -= A[(int64_t)i * P + q] * Y[(int64_t)q * P + c];
                Y[(int64_t)i * P + c] = y / A[(int64_t)i * P + i];
            }
            for (int i = P - 1; i >= 0; --i) {
                double x = Y[(int64_t)i * P + c];
                for (int q = i + 1; q < P; ++q) x -= A[(int64_t)q * P + i] * Y[(int64_t)q * P + c];
                x /= A[(int64_t)i * P + i];
                Y[(int64_t)i * P + c] = x;
            }
            for (int i = 0; i < P; ++i) inv[(int64_t)k * P * P + (int64_t)i * P + c] = (T)Y[(int64_t)i * P + c];
        }
        __syncthreads();
    }
}

// Host driver: assembles, factorises and inverts every leaf of one geometry.
// `leafinv_out` receives K*P*P values of type T. Returns WMG_OK or an error.
int32_t build_leaf_inverses(const GeomDev &gh, const GeomDev *gd, double *leafinv_out, cudaStream_t st)
{
    const int P = gh.P, K = gh.K;
    const int R = (int)floor(gh.B * 1.4142135623730951 / gh.dt) + 3;
    // angle chunk sized for a ~256 MB coefficient buffer
    const double per_angle = (double)P * R * K * sizeof(double);
    int chunk = (int)fmax(1.0, fmin((double)gh.m, 256.0 * 1024 * 1024 / per_angle));
    double *Gbuf = nullptr, *Dm = nullptr, *Y = nullptr;
    int *status = nullptr;
    int2 *pairs = nullptr;
    const int npairs = P * (P + 1) / 2;
    std::vector<int2> hp;
    hp.reserve(npairs);
    for (int b1 = 0; b1 < P; ++b1)
        for (int b2 = b1; b2 < P; ++b2) hp.push_back(make_int2(b1, b2));
    const int inv_ctas = std::min(K, num_sms() * 2);
    int32_t rc = WMG_OK;
    auto cleanup = [&]() {
        cudaFree(Gbuf); cudaFree(Dm); cudaFree(Y); cudaFree(status); cudaFree(pairs);
    };
    if (cudaMalloc(&Gbuf, (size_t)chunk * P * R * K * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&Dm, (size_t)K * P * P * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&Y, (size_t)inv_ctas * P * P * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&status, (size_t)K * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&pairs, (size_t)npairs * sizeof(int2)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(WMG_ERR_OOM, "leaf setup: device allocation failed");
    }
    cudaMemcpyAsync(pairs, hp.data(), (size_t)npairs * sizeof(int2), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(Dm, 0, (size_t)K * P * P * sizeof(double), st);
    const int gram_threads = std::min(256, std::max(32, ((K + 31) / 32) * 32));
    for (int a0 = 0; a0 < gh.m; a0 += chunk) {
        const int na = std::min(chunk, gh.m - a0);
        count_launches(2);
        k_leaf_coeffs<<<std::min(na * P, num_sms() * 8), 256, 0, st>>>(gd, a0, na, R, Gbuf);
        k_leaf_gram<<<std::min(npairs, num_sms() * 16), gram_threads, 0, st>>>(gd, a0, na, R, Gbuf,
                                                                               pairs, npairs, Dm);
    }
    count_launches(1);
    k_leaf_invert<double><<<inv_ctas, 256, 0, st>>>(gd, Dm, Y, leafinv_out, status);
    std::vector<int> hs(K);
    cudaMemcpyAsync(hs.data(), status, (size_t)K * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
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
