// csr.cu -- stored-matrix comparator for the matrix-free operators (Section
// 2.1: W holds the pixel-ray intersection lengths). W or W^T of a plan's
// geometry is assembled once on the device as CSR -- exact chords evaluated in
// FP64 by the same trapezoid law as the projectors, stored in the plan
// precision -- and applied by a sparse matrix-vector product that streams the
// matrix. It is a measurement reference: its time and its HBM bandwidth
// against the measured peak show what storing W would cost next to
// recomputing the weights.
#include <numeric>

#include "engine.cuh"

struct wmg_csr {
    int prec = WMG_PREC_F64;
    int64_t rows = 0, cols = 0, nnz = 0;
    wmg::DevBuf rowptr, col, val;
};

namespace wmg {

// Rows of W (one warp per ray (a, k), lanes over frame rows): the at most two
// pixels of each frame row with a chord above kNnzEps, in frame-row order.
// FILL = 0 writes the row lengths, FILL = 1 the entries at rowptr[ray].
template <class T, int FILL>
__global__ void __launch_bounds__(256)
k_csr_rays(const GeomDev *__restrict__ Gd, int64_t *__restrict__ rp, int *__restrict__ col, T *__restrict__ val)
{
    const GeomDev &g = *Gd;
    const int n = g.n, D = g.D;
    const int64_t M = (int64_t)g.m * D;
    const int lane = threadIdx.x & 31;
    for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < M;
         r += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const int a = (int)(r / D), k = (int)(r - (int64_t)a * D);
        double c, s;
        load_cs(g, a, c, s);
        const bool steep = fabs(c) >= fabs(s);
        const double cc = steep ? c : s, ss = steep ? s : c;
        const Chord<double> ch = make_chord<double>(cc, ss, g.kernel);
        const double hwx = ch.hw / fabs(cc), half_n = 0.5 * n;
        const double tk = ray_offset<double>(g, k);
        LineD line;
        make_line(g, a, !steep, tk, line);
        int64_t pos = FILL ? rp[r] : 0;
        int total = 0;
        for (int base = 0; base < n; base += 32) {
            const int fr = base + lane;
            double w[2] = {0.0, 0.0};
            int fx0 = 0, cnt = 0;
            if (fr < n) {
                const double yc = fr + 0.5 - half_n;
                fx0 = (int)ceil((tk - yc * ss) / cc + half_n - 0.5 - hwx);
                for (int q = 0; q < 2; ++q) {
                    const int fx = fx0 + q;
                    if (fx >= 0 && fx < n) w[q] = ch(fabs(line_dist(line, fx + 0.5 - half_n, yc)));
                    if (!(w[q] > kNnzEps)) w[q] = 0.0;
                    cnt += w[q] > 0.0;
                }
            }
            // exclusive prefix of the lanes' counts keeps the frame-row order
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (FILL && cnt) {
                int64_t p = pos + incl - cnt;
                for (int q = 0; q < 2; ++q)
                    if (w[q] > 0.0) {
                        const int fx = fx0 + q;
                        col[p] = steep ? fr * n + fx : fx * n + fr;
                        val[p] = (T)(w[q] * g.h);
                        ++p;
                    }
            }
            const int sum = __shfl_sync(0xffffffffu, incl, 31);
            pos += sum;
            total += sum;
        }
        if (!FILL && lane == 0) rp[r] = total;
    }
}

// Rows of W^T (one thread per pixel): for every angle, the bins whose chord
// through the pixel is above kNnzEps, in (angle, bin) order.
template <class T, int FILL>
__global__ void __launch_bounds__(256)
k_csr_pixels(const GeomDev *__restrict__ Gd, int64_t *__restrict__ rp, int *__restrict__ col, T *__restrict__ val)
{
    const GeomDev &g = *Gd;
    const int n = g.n, m = g.m, D = g.D;
    const int64_t N = (int64_t)n * n;
    const double dt = g.dt, inv_dt = 1.0 / g.dt, t0 = g.t0, hD = 0.5 * (D - 1), half_n = 0.5 * n;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const int iy = (int)(j / n), ix = (int)(j - (int64_t)iy * n);
        const double xo = ix + 0.5 - half_n, yo = iy + 0.5 - half_n;
        int64_t pos = FILL ? rp[j] : 0;
        int64_t cnt = 0;
        for (int a = 0; a < m; ++a) {
            double c, s;
            load_cs(g, a, c, s);
            const Chord<double> ch = make_chord<double>(c, s, g.kernel);
            const double hwb = ch.hw * inv_dt;
            const int ncand = (int)floor(2.0 * hwb) + 1;
            LineD line;
            make_line(g, a, false, 0.0, line);
            const double tau = -line_dist(line, xo, yo);
            const int k0 = (int)ceil((tau - t0) * inv_dt + hD - hwb);
            for (int q = 0; q < ncand; ++q) {
                const int k = k0 + q;
                if (k < 0 || k >= D) continue;
                line.t = fma((double)k - hD, dt, t0);
                const double w = ch(fabs(line_dist(line, xo, yo)));
                if (w > kNnzEps) {
                    if (FILL) {
                        col[pos] = a * D + k;
                        val[pos] = (T)(w * g.h);
                        ++pos;
                    }
                    ++cnt;
                }
            }
        }
        if (!FILL) rp[j] = cnt;
    }
}

// y_v = A x_v for `count` vectors (x_v at x + v * cols, y_v at y + v * rows):
// one half-warp per row (two rows per warp in flight), four entries per lane
// per step; the row's entries are re-read from L1 for each vector.
template <class T>
__global__ void __launch_bounds__(256)
k_csr_spmv(int64_t rows, int64_t cols, const int64_t *__restrict__ rp, const int *__restrict__ col,
           const T *__restrict__ val, int count, const T *__restrict__ x, T *__restrict__ y)
{
    const int lane = threadIdx.x & 15;
    const int64_t hw0 = blockIdx.x * (int64_t)(blockDim.x >> 4) + (threadIdx.x >> 4);
    const int64_t nhw = (int64_t)gridDim.x * (blockDim.x >> 4);
    // every half-warp runs the same number of iterations (shuffles stay converged)
    const int64_t iters = (rows + nhw - 1) / nhw;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t r = hw0 + it * nhw;
        const bool live = r < rows;
        const int64_t b = live ? rp[r] : 0, e = live ? rp[r + 1] : 0;
        for (int v = 0; v < count; ++v) {
            const T *xv = x + (int64_t)v * cols;
            T acc[4] = {T(0), T(0), T(0), T(0)};
            int64_t p = b + lane;
            for (; p + 48 < e; p += 64) {
                int cl[4];
                T vl[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) { cl[u] = __ldg(col + p + 16 * u); vl[u] = __ldg(val + p + 16 * u); }
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = fma_t(vl[u], __ldg(xv + cl[u]), acc[u]);
            }
            for (; p < e; p += 16) acc[0] = fma_t(__ldg(val + p), __ldg(xv + __ldg(col + p)), acc[0]);
            T sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
            for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (live && lane == 0) y[(int64_t)v * rows + r] = sum;
        }
    }
}

template <class T>
static int32_t build_csr(const GeomDev *gd, const GeomDev &gh, bool transposed, wmg_csr *c, cudaStream_t st)
{
    const int64_t N = (int64_t)gh.n * gh.n, M = (int64_t)gh.m * gh.D;
    c->rows = transposed ? N : M;
    c->cols = transposed ? M : N;
    if (!c->rowptr.ensure((size_t)(c->rows + 1) * sizeof(int64_t)))
        return fail(WMG_ERR_OOM, "wmg_csr_create: row pointers");
    int64_t *rp = c->rowptr.as<int64_t>();
    const int grid = num_sms() * 8;
    count_launches(1);
    if (transposed) k_csr_pixels<T, 0><<<grid, 256, 0, st>>>(gd, rp, nullptr, nullptr);
    else k_csr_rays<T, 0><<<grid, 256, 0, st>>>(gd, rp, nullptr, nullptr);
    std::vector<int64_t> h((size_t)c->rows + 1, 0);
    WMG_CUDA(cudaMemcpyAsync(h.data() + 1, rp, (size_t)c->rows * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    WMG_CUDA(cudaStreamSynchronize(st));
    std::partial_sum(h.begin(), h.end(), h.begin());      // row lengths -> row pointers
    c->nnz = h.back();
    WMG_CUDA(cudaMemcpyAsync(rp, h.data(), h.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (!c->col.ensure((size_t)std::max<int64_t>(c->nnz, 1) * sizeof(int)) ||
        !c->val.ensure((size_t)std::max<int64_t>(c->nnz, 1) * sizeof(T)))
        return fail(WMG_ERR_OOM, "wmg_csr_create: entries");
    count_launches(1);
    if (transposed) k_csr_pixels<T, 1><<<grid, 256, 0, st>>>(gd, rp, c->col.as<int>(), c->val.as<T>());
    else k_csr_rays<T, 1><<<grid, 256, 0, st>>>(gd, rp, c->col.as<int>(), c->val.as<T>());
    WMG_CUDA(cudaStreamSynchronize(st));
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

}  // namespace wmg

using namespace wmg;

extern "C" int32_t wmg_csr_create(wmg_plan *pl, int32_t transposed, void *stream, wmg_csr **out)
{
    if (!pl || !out) return fail(WMG_ERR_INVALID_ARG, "wmg_csr_create: bad arguments");
    *out = nullptr;
    if (pl->batch || pl->geos.empty() || !pl->geos[0])
        return fail(WMG_ERR_INVALID_ARG, "wmg_csr_create: needs a single-geometry plan");
    const GeomDev &gh = pl->geos[0]->g;
    if ((int64_t)gh.n * gh.n > INT32_MAX || (int64_t)gh.m * gh.D > INT32_MAX)
        return fail(WMG_ERR_INVALID_ARG, "wmg_csr_create: too many columns for 32-bit indices");
    auto c = std::make_unique<wmg_csr>();
    c->prec = pl->prec;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const GeomDev *gd = pl->d_geom.as<GeomDev>();
    int32_t rc = pl->prec == WMG_PREC_F64 ? build_csr<double>(gd, gh, transposed != 0, c.get(), st)
                                          : build_csr<float>(gd, gh, transposed != 0, c.get(), st);
    if (rc) return rc;
    *out = c.release();
    return WMG_OK;
}

extern "C" int32_t wmg_csr_destroy(wmg_csr *csr)
{
    if (!csr) return WMG_OK;
    cudaDeviceSynchronize();
    delete csr;
    return WMG_OK;
}

extern "C" int32_t wmg_csr_info(const wmg_csr *csr, int64_t *rows, int64_t *cols, int64_t *nnz)
{
    if (!csr) return fail(WMG_ERR_INVALID_ARG, "wmg_csr_info: csr is NULL");
    if (rows) *rows = csr->rows;
    if (cols) *cols = csr->cols;
    if (nnz) *nnz = csr->nnz;
    return WMG_OK;
}

extern "C" int32_t wmg_csr_apply(const wmg_csr *csr, int32_t count, const void *x, void *y, void *stream)
{
    if (!csr || !x || !y || count < 1) return fail(WMG_ERR_INVALID_ARG, "wmg_csr_apply: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = num_sms() * 16;
    count_launches(1);
    if (csr->prec == WMG_PREC_F64)
        k_csr_spmv<double><<<grid, 256, 0, st>>>(csr->rows, csr->cols, csr->rowptr.as<int64_t>(), csr->col.as<int>(),
                                                 csr->val.as<double>(), count, static_cast<const double *>(x),
                                                 static_cast<double *>(y));
    else
        k_csr_spmv<float><<<grid, 256, 0, st>>>(csr->rows, csr->cols, csr->rowptr.as<int64_t>(), csr->col.as<int>(),
                                                csr->val.as<float>(), count, static_cast<const float *>(x),
                                                static_cast<float *>(y));
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}
