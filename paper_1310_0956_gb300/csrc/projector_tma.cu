// projector_tma.cu -- FP32 forward projection q = W p (Section 2.1, eq. sys:
// w_ij = length of ray i in pixel j) of groups of kProjGroup same-geometry
// images, with the image rows a tile reads staged in shared memory by the
// tensor memory accelerator (TMA).
//
// Same tiles, weights and summation order as k_project_f32's group tiles in
// projector_f32.cu (so a problem gets the same bits from either kernel, alone
// or grouped): a tile is one angle, 32 rays (lane = ray) and 8 images; the
// consumer warp w takes rows lo + w + 8i, four of them per step, with a
// compensated sum per image and the warps' sums combined in warp order.
// What differs is where the pixel values come from. A producer warp walks
// the same tiles and, for every 16 rows, loads the band of pixels the 32
// rays cross -- two boxes of 64 columns x 8 rows x the 8 images (the frame's
// rows: the images for steep angles, their transposes otherwise), each box
// starting on a 16-byte boundary a few pixels left of the band -- into a
// ring of shared-memory stages; the consumers read their two candidate
// pixels per row from there.
// Columns outside the image arrive as zeros (TMA out-of-bounds fill), which
// are exactly the values the one-image kernel substitutes for them.
//
// Synchronisation: per stage a `full` mbarrier (the producer's arrival with
// the expected byte count, completed by the copies) and an `empty` one (one
// arrival per consumer warp). Every wait is bounded: on timeout the CTA
// raises an abort flag that ends all its further waits and the copies it
// would issue, and sets the module's error flag, which the host reads at its
// next synchronising call (tma_error_take). Deterministic: no atomics in
// the arithmetic.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "kern_common.cuh"

namespace wmg {

namespace {
constexpr int kNW = 8;                                  // consumer warps
constexpr int kIB = kProjGroup;                         // images per tile
constexpr int kBoxW = 64;                               // box width (pixels)
constexpr int kBoxH = 8;                                // box height: one row per consumer warp
constexpr int kSub = 2;                                 // boxes per stage: 16 rows
constexpr int kStages = 3;
constexpr int kBoxFloats = kBoxW * kBoxH * kIB;         // one box: 8 rows of all 8 images (16 KB)
constexpr int kStageFloats = kSub * kBoxFloats;         // 32 KB
constexpr uint32_t kStageBytes = kStageFloats * 4;
constexpr long long kWaitCycles = 1LL << 31;            // about a second
constexpr long long kStallWaitCycles = 1LL << 22;       // about 2 ms: the test hook's limit
constexpr size_t kSmemBytes = (size_t)kStages * kStageFloats * sizeof(float);
}  // namespace

// 0 = fine; 1 = a stage wait timed out; 2 = a candidate pixel fell outside its
// staged box (a bound of the band width did not hold)
__device__ int g_tma_error;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of parity `parity` of the barrier; false if the CTA
// has aborted or the wait timed out (then it aborts the CTA).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          long long limit)
{
    if (mbar_try(bar, parity)) return true;                 // the phase has completed: data in place
    if (*abort_flag) return false;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            atomicExch(&g_tma_error, 1);
            return false;
        }
    }
    return true;
}
// The same wait without the abort check (draining the producer's copies).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity, long long limit)
{
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > limit) return;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Per-tile quantities both roles derive identically (lane = ray).
struct TileRays {
    int nimg;
    bool act[kIB];
    bool any, steep, valid;
    float tk, half_n;
    int lo, hi;
};

__device__ __forceinline__ void tile_rays(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
                                          const int4 &tl, const PjArgs &a, int lane, TileRays &r)
{
    r.nimg = min(kIB, max(1, tl.w));
    r.any = false;
#pragma unroll
    for (int b = 0; b < kIB; ++b) {
        r.act[b] = b < r.nimg && slot_active(a.S, P[tl.x + b].slot);
        r.any |= r.act[b];
    }
    const GeomDev &g = G[P[tl.x].geom];
    const int n = g.n, D = g.D, k = tl.z + lane;
    const AngleF &A = g.angf[tl.y];
    r.steep = __float_as_int(A.flags) & 1;
    r.valid = k < D;
    const float ss_hi = r.steep ? A.shi : A.chi, ss_lo = r.steep ? A.slo : A.clo;
    r.half_n = 0.5f * (float)n;
    r.tk = __fmaf_rn((float)k - g.hDf, g.dtf, g.t0f);
    // rows the lane's ray can touch (image x-range widened by one pixel)
    int lo = n, hi = -1;
    if (r.valid) {
        const float xs0 = r.tk * A.inv_cc;
        if (ss_hi == 0.f && ss_lo == 0.f) {
            if (fabsf(xs0) < r.half_n + 1.f) { lo = 0; hi = n - 1; }
        } else {
            const float ya = (xs0 - (r.half_n + 1.f)) * A.inv_slope, yb = (xs0 + (r.half_n + 1.f)) * A.inv_slope;
            lo = max(0, __float2int_ru(fminf(ya, yb) + r.half_n - 0.5f));
            hi = min(n - 1, __float2int_rd(fmaxf(ya, yb) + r.half_n - 0.5f));
        }
    }
    r.lo = warp_min(lo);
    r.hi = warp_max(hi);
}

__global__ void __launch_bounds__(32 * (kNW + 1), 2)
k_project_f32_tma(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P, const int4 *__restrict__ tiles,
                  int ntiles, PjArgs a, const __grid_constant__ CUtensorMap map_img,
                  const __grid_constant__ CUtensorMap map_imgT, int stall, long long wait_limit)
{
    // stage s, box q: [image][row][column] (the TMA box order)
    extern __shared__ __align__(1024) float ring[];
    __shared__ float red[kNW][kIB][32];            // per warp, image and lane: s - c
    __shared__ __align__(8) unsigned long long full[kStages], empty[kStages];
    __shared__ int xoff[kStages][kSub];
    __shared__ int abort_flag;
    volatile int *abort_v = &abort_flag;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), kNW);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    if (w == kNW) {
        // ---------------- producer warp ----------------
        if (stall) return;          // test hook: no copies, so the consumers' waits run out
        int seq = 0, st = 0;
        uint32_t ph = 0;
        for (int t = blockIdx.x; t < ntiles && !*abort_v; t += gridDim.x) {
            const int4 tl = tiles[t];
            TileRays tr;
            tile_rays(G, P, tl, a, lane, tr);
            const int nrows = tr.hi - tr.lo + 1;
            if (!tr.any || nrows <= 0) continue;
            const GeomDev &g = G[P[tl.x].geom];
            const int n = g.n;
            const AngleF &A = g.angf[tl.y];
            const CUtensorMap *map = tr.steep ? &map_img : &map_imgT;
            const float off = tr.half_n - 0.5f;
            // leftmost crossing of the row y = 0 over the tile's rays; a
            // box's first column follows from it without a warp reduction
            const float xs_min = warp_min_f(tr.valid ? tr.tk * A.inv_cc : INFINITY);
            const int z0 = (int)(P[tl.x].img / ((int64_t)n * n));
            // two stages of 16 rows per step of 4 rows of each consumer warp
            const int nst = 2 * ((nrows + 31) / 32);
            for (int c = 0; c < nst; ++c, ++seq) {
                const int s = st;
                if (seq >= kStages && !mbar_wait(smem_u32(&empty[s]), ph ^ 1, abort_v, wait_limit)) break;
                // box q holds rows ya .. ya + 7; its first column: two pixels
                // left of the leftmost crossing of its rows (the row centre
                // line's crossing is linear in the row), rounded down to a
                // multiple of 4. Consumers check that every candidate they
                // read lies in the box.
                if (lane < kSub) {
                    const int ya = tr.lo + 16 * c + 8 * lane;
                    const float y0 = (float)ya + 0.5f - tr.half_n, y1 = y0 + 7.f;
                    const float f0 = __fmaf_rn(-y0, A.slope, xs_min), f1 = __fmaf_rn(-y1, A.slope, xs_min);
                    const int xl = (int)floorf(fminf(f0, f1) + off);
                    xoff[s][lane] = ((xl - 2) >> 2) << 2;                 // floor to a multiple of 4
                }
                __syncwarp();
                if (lane == 0) {
                    const uint32_t fb = smem_u32(&full[s]);
                    mbar_expect_tx(fb, kStageBytes);
                    float *stage = ring + (size_t)s * kStageFloats;
#pragma unroll
                    for (int q = 0; q < kSub; ++q)
                        tma_load_3d(smem_u32(stage + q * kBoxFloats), map, xoff[s][q], tr.lo + 16 * c + 8 * q, z0,
                                    fb);
                }
                __syncwarp();
                if (++st == kStages) { st = 0; ph ^= 1; }
            }
        }
        if (*abort_v) {
            // wait (bounded) for the copies of the stages still in flight
            for (int d = max(0, seq - kStages); d < seq; ++d)
                mbar_drain(smem_u32(&full[d % kStages]), (uint32_t)(d / kStages) & 1, wait_limit);
        }
        return;
    }

    // ---------------- consumer warps ----------------
    // Pairs of images go through the paired FP32 instructions (two IEEE
    // single-precision operations, each rounded to nearest, per
    // instruction): the per-image arithmetic is exactly the one-image
    // kernel's, in half the arithmetic instructions.
    constexpr int kP = kIB / 2;
    const float2 neg1 = make_float2(-1.f, -1.f);
    int st = 0;                                                      // ring stage and its phase parity
    uint32_t ph = 0;
    bool bad = false;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        TileRays tr;
        tile_rays(G, P, tl, a, lane, tr);
        if (!tr.any) continue;                                       // CTA-uniform
        const GeomDev &g = G[P[tl.x].geom];
        const int D = g.D, ang = tl.y;
        const AngleF A = g.angf[ang];
        const float cc_hi = tr.steep ? A.chi : A.shi, cc_lo = tr.steep ? A.clo : A.slo;
        const float ss_hi = tr.steep ? A.shi : A.chi, ss_lo = tr.steep ? A.slo : A.clo;
        const float half_n = tr.half_n, tk = tr.tk;
        float2 s2[kP], c2[kP], acc[kP];
#pragma unroll
        for (int q = 0; q < kP; ++q) { s2[q] = make_float2(0.f, 0.f); c2[q] = s2[q]; acc[q] = s2[q]; }
        const int nrows = tr.hi - tr.lo + 1;
        if (nrows > 0) {
            const int iy0 = tr.lo + w;
            const float dy = (float)kNW;
            const float yc = (float)iy0 + 0.5f - half_n;
            float brow = __fmaf_rn(-yc, ss_hi, tk);                  // t - yc ss_hi: exact
            float cy = yc * ss_lo;
            float xs = __fmaf_rn(-yc, A.slope, tk * A.inv_cc);       // crossing of the row centre line
            const float dbrow = -dy * ss_hi, dcy = dy * ss_lo, dxs = -dy * A.slope;
            const float off = half_n - 0.5f;
            const int nmine = (nrows - w + kNW - 1) / kNW;           // rows of this warp
            const float wa = A.wa, wb = A.wb, ccf = A.cc;
            const int nsteps = (nrows + 31) / 32;                    // two stages of 16 rows per step
            for (int c = 0; c < nsteps; ++c) {
                // the warp's step of 4 rows j .. j + 3: rows 0, 1 in the
                // first stage, 2, 3 in the second, one product chain per
                // image over the 4 rows and one compensated step. A warp
                // whose rows have all been summed takes no further step (as
                // in the one-image kernel: a step of zeros still moves a sum)
                const int j = 4 * c;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    mbar_wait(smem_u32(&full[st]), ph, abort_v, wait_limit);
                    if (j < nmine) {
                        const float *stage = ring + (size_t)st * kStageFloats + w * kBoxW;
                        int li[2];
                        float2 w0[2], w1[2];
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const bool live = tr.valid && (j + 2 * h + r < nmine);
                            const int ix0 = __float2int_rd(xs + off);
                            const int l = ix0 - xoff[st][r];
                            bad |= live && (unsigned)l > (unsigned)(kBoxW - 2);
                            li[r] = min(max(l, 0), kBoxW - 2);
                            const float xc = (float)ix0 + 0.5f - half_n;
                            const float dl0 = __fmaf_rn(-xc, cc_hi, brow) - __fmaf_rn(xc, cc_lo, cy);
                            // rows past the warp's last one weigh 0 (the one-
                            // image kernel reads 0 there instead: the same sums)
                            const float u0 = live ? __saturatef(__fmaf_rn(-fabsf(dl0), wa, wb)) : 0.f;
                            const float u1 = live ? __saturatef(__fmaf_rn(-fabsf(dl0 - ccf), wa, wb)) : 0.f;
                            w0[r] = make_float2(u0, u0);
                            w1[r] = make_float2(u1, u1);
                            brow += dbrow;
                            cy += dcy;
                            xs += dxs;
                        }
#pragma unroll
                        for (int q = 0; q < kP; ++q) {
                            // images 2q, 2q + 1 (inactive ones are computed
                            // and not written: the pair stays uniform)
                            const float *pa = stage + (2 * q) * (kBoxW * kBoxH);
                            const float *pb = pa + kBoxW * kBoxH;
                            const float2 v00 = make_float2(pa[li[0]], pb[li[0]]);
                            const float2 v01 = make_float2(pa[li[0] + 1], pb[li[0] + 1]);
                            const float2 v10 = make_float2(pa[kBoxFloats + li[1]], pb[kBoxFloats + li[1]]);
                            const float2 v11 = make_float2(pa[kBoxFloats + li[1] + 1], pb[kBoxFloats + li[1] + 1]);
                            float2 x = h == 0 ? __fmul2_rn(w0[0], v00) : __ffma2_rn(w0[0], v00, acc[q]);
                            x = __ffma2_rn(w1[0], v01, x);
                            x = __ffma2_rn(w0[1], v10, x);
                            acc[q] = __ffma2_rn(w1[1], v11, x);
                        }
                        if (h == 1) {
#pragma unroll
                            for (int q = 0; q < kP; ++q) {                 // Kahan step
                                const float2 y = __ffma2_rn(c2[q], neg1, acc[q]);
                                const float2 tt = __fadd2_rn(s2[q], y);
                                c2[q] = __ffma2_rn(y, neg1, __ffma2_rn(s2[q], neg1, tt));
                                s2[q] = tt;
                            }
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&empty[st]));
                    if (++st == kStages) { st = 0; ph ^= 1; }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kP; ++q) {
            red[w][2 * q][lane] = s2[q].x - c2[q].x;
            red[w][2 * q + 1][lane] = s2[q].y - c2[q].y;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kNW) : "memory");
        bool mine = false;
#pragma unroll
        for (int b = 0; b < kIB; ++b) mine |= b == w && tr.act[b];
        if (mine) {                                                  // warp w finishes image w
            const int b = w;
            float S = 0.f, Cc = 0.f;
#pragma unroll
            for (int i = 0; i < kNW; ++i) {
                const float y = red[i][b][lane] - Cc;
                const float tt = S + y;
                Cc = (tt - S) - y;
                S = tt;
            }
            const ProbDev pb = P[tl.x + b];
            const int k = tl.z + lane;
            const float v = (S - Cc) * (A.lmax * g.hf);
            if (tr.valid) static_cast<float *>(a.sino)[pb.sino + (int64_t)ang * D + k] = v;
            if (a.part) {
                double q2 = tr.valid ? (double)v * (double)v : 0.0;
                q2 = warp_sum_fixed(q2);
                if (lane == 0) a.part[a.part_base[tl.x + b] + ang * ((D + 31) / 32) + tl.z / 32] = q2;
            }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kNW) : "memory");
    }
    // an aborted CTA read stages that never arrived: its box checks mean nothing
    const bool aborted = *abort_v;
    if (__any_sync(0xffffffffu, bad) && lane == 0 && !aborted) atomicExch(&g_tma_error, 2);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Pool of `count` row-major n x n FP32 images starting at base (image z at
// z n^2), read in boxes of 64 columns x 8 rows x 8 images, zeros outside.
static bool encode_pool_map(CUtensorMap *m, const void *base, int n, int64_t count)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)count};
    const cuuint64_t strides[2] = {(cuuint64_t)n * sizeof(float), (cuuint64_t)n * n * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)kBoxW, (cuuint32_t)kBoxH, (cuuint32_t)kIB};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool project_tma_available() { return tensor_map_encoder() != nullptr; }

// Test hook for the bounded waits: with WMG_TEST_STALL_STAGED_COPIES=1 in the
// environment at launch time, the producer warp issues no copies and the
// consumers' waits run out after kStallWaitCycles, so the timeout path
// (abort, error flag, WMG_ERR_TIMEOUT at the next synchronising call) runs
// without any fault: every wait is bounded and no copy is in flight.
static bool stall_requested()
{
    const char *v = std::getenv("WMG_TEST_STALL_STAGED_COPIES");
    return v && v[0] == '1';
}

bool launch_project_f32_tma(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles, const PjArgs &a,
                            int n, int64_t count, cudaStream_t st)
{
    if (ntiles <= 0) return true;
    if (n % 4 != 0 || !a.img || !a.imgT || (reinterpret_cast<uintptr_t>(a.img) & 15) ||
        (reinterpret_cast<uintptr_t>(a.imgT) & 15))
        return false;
    CUtensorMap mi, mt;
    if (!encode_pool_map(&mi, a.img, n, count) || !encode_pool_map(&mt, a.imgT, n, count)) return false;
    ensure_dyn_smem((const void *)k_project_f32_tma, (int)kSmemBytes);
    count_launches(1);
    const int grid = min(ntiles, 2 * num_sms());               // two CTAs per SM
    const bool stall = stall_requested();
    k_project_f32_tma<<<grid, 32 * (kNW + 1), kSmemBytes, st>>>(G, P, tiles, ntiles, a, mi, mt, stall ? 1 : 0,
                                                                stall ? kStallWaitCycles : kWaitCycles);
    return true;
}

int tma_error_take()
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tma_error, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tma_error, &z, sizeof(int));
    }
    return v;
}

}  // namespace wmg
