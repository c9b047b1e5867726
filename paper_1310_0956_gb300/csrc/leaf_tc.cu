// leaf_tc.cu -- FP32 leaf solves e_k = D_k^{-1} c_k on the tensor cores
// (Section 3.1.2: the exact solves of the coarsest-level subproblems; Section
// 3.1.3: applied to many right-hand sides at once they are dense matrix
// products). F32 plans only; FP64 plans keep k_leaf_apply (haar.cu).
//
// A work item (built by the host) is {first problem p0, leaf k, count np <=
// 64 consecutive problems of one geometry, row block of 128 rows of D_k^{-1}}:
//     E[rows, group] = Dinv_k[rows, :] * C_k[:, group]      (128 x P x 64)
// with P = n_c^2 <= 256. The product runs as tcgen05.mma (M = 128, N = 64,
// K = 8 per instruction, kind::tf32) with the accumulators in tensor memory.
//
// Precision. Both operands are FP32 values (the inverse is stored in FP32,
// the FP64 coefficients are rounded to FP32 exactly as the CUDA-core form
// does) split as x = hi + lo, hi = x rounded to the nearest TF32 value (10
// explicit mantissa bits), lo = x - hi (exact in FP32) rounded to TF32. Three
// TF32 products per k-step, hi*hi into one accumulator and hi*lo + lo*hi into
// a second, summed in the epilogue: the split-operand method of Ootomo and
// Yokota ("Recovering single precision accuracy from Tensor Cores while
// surpassing the FP32 theoretical peak performance", IJHPCA 36(4), 2022),
// which keeps the small terms from being rounded against the large running
// sum. The dropped lo*lo term and the TF32 rounding of lo leave about 2^-21
// relative per product; the sums of 256 products then sit at the FP32
// rounding level of the CUDA-core form (tests compare both with the FP64
// oracle).
//
// Shared memory: per stage, K-chunks of 32 values (128 bytes) per row of
// A_hi, A_lo (128 rows) and B_hi, B_lo (64 rows), each in the K-major
// 128-byte-swizzle layout the tensor core reads (8-row atoms of 1024 bytes,
// the 16-byte chunk c of row r stored at chunk c ^ (r mod 8)), written by the
// threads after the split; two stages, and the global loads of chunk c + 1
// are issued before the products of chunk c, so they overlap. One thread issues the products and commits them to
// the stage's mbarrier; every wait is bounded (about a second), after which
// the CTA records the module's error flag, drains its products in flight
// (bounded again), frees its tensor memory and returns.
//
// Deterministic: a problem's column of the product depends only on its own
// coefficients and the leaf inverse, whatever the other columns hold, so a
// problem gets the same bits alone and in any batch.
#include <cstdint>
#include <cstdlib>

#include "kern_common.cuh"

namespace wmg {

namespace {
constexpr int kTM = kLeafTcRows;             // rows per work item (MMA M) = 128
constexpr int kTN = kLeafTcProblems;         // problems per work item (MMA N) = 64
constexpr int kTK = 32;                      // K values per stage (128 bytes of FP32)
constexpr int kThreads = 256;                // 8 warps: warp w reads TMEM lanes 32 (w mod 4) ..
constexpr uint32_t kATile = kTM * kTK * 4;   // 16 KB
constexpr uint32_t kBTile = kTN * kTK * 4;   // 8 KB
constexpr uint32_t kStage = 2 * kATile + 2 * kBTile;
constexpr uint32_t kSmem = 2 * kStage + 1024;   // two stages + room to align to 1024 bytes
constexpr uint32_t kTmemCols = 2 * kTN;      // hi*hi accumulator | hi*lo + lo*hi accumulator
constexpr long long kWaitCycles = 1LL << 31; // about a second
constexpr long long kStallWaitCycles = 1LL << 22;   // about 2 ms: the test hook's limit
static_assert(kStage % 1024 == 0, "stages must keep the 1024-byte alignment of the swizzle atoms");

// Instruction descriptor of kind::tf32: D = F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);
}  // namespace

// 0 = fine; 1 = a wait for the tensor-core products timed out
__device__ int g_tc_error;

__device__ __forceinline__ uint32_t tc_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset 0 (unused for swizzled K-major tiles), stride byte offset 1024
// >> 4 (bits 32-45: from one 8-row atom to the next), descriptor version 1
// (bit 46), 128-byte swizzle (bits 61-63 = 2).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Byte offset of element (row r, k) of a K-chunk tile in the 128-byte-swizzle layout.
__device__ __forceinline__ uint32_t tc_swz(int r, int k)
{
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + (k & 3) * 4);
}

// x rounded to the nearest TF32 value (ties away from zero; finite inputs):
// the low 13 mantissa bits cleared after adding half of their range.
__device__ __forceinline__ float tf32_round(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void tc_mbar_init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool tc_mbar_try(uint32_t bar, uint32_t parity)
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
// Bounded wait for the phase of parity `parity`; false on timeout (the
// module's error flag is then set).
__device__ __forceinline__ bool tc_mbar_wait(uint32_t bar, uint32_t parity, long long limit)
{
    if (tc_mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!tc_mbar_try(bar, parity)) {
        if (clock64() - t0 > limit) {
            atomicExch(&g_tc_error, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[adesc] * B[bdesc]^T, M = 128, N = 64, K = 8 (TF32), one thread.
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
// Arrival on `bar` once every product this thread issued has completed.
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// 16 consecutive accumulator columns of TMEM lane (taddr >> 16) + lane id.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// One work item's operands as this thread loads them: rows warp + 8 i of the
// inverse's row block, problems warp + 8 i of the item (coefficient offsets of
// leaf k, -1 for none or an inactive problem).
struct TcItem {
    const float *arow;       // row warp of the block, column lane
    int Pn, arows, nk, row0;
    int64_t boff[kTN * kTK / kThreads];
};

// Lane 0 of each warp also records its problems' offsets (without the lane)
// in coef[], which the item's epilogue reads.
__device__ __forceinline__ void tc_item(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
                                        const double *__restrict__ S, const int4 &tl, int warp, int lane, TcItem &q,
                                        int64_t *coef)
{
    const GeomDev &g = G[P[tl.x].geom];
    const int Pn = g.P, k = tl.y;
    q.Pn = Pn;
    q.row0 = tl.w * kTM;
    q.nk = (Pn + kTK - 1) / kTK;
    q.arows = Pn - q.row0 - warp;
    q.arow = static_cast<const float *>(g.leafinv) + (int64_t)k * Pn * Pn + (int64_t)(q.row0 + warp) * Pn + lane;
#pragma unroll
    for (int i = 0; i < kTN * kTK / kThreads; ++i) {
        const int p = warp + 8 * i;
        int64_t off = -1;
        if (p < tl.z) {
            const ProbDev pd = P[tl.x + p];
            if (slot_active(S, pd.slot)) off = pd.coef + (int64_t)k * Pn;
        }
        if (lane == 0) coef[p] = off;
        q.boff[i] = off < 0 ? off : off + lane;
    }
}

__global__ void __launch_bounds__(kThreads, 2)
k_leaf_apply_tc(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P, const int4 *__restrict__ items,
                int nitems, const double *__restrict__ C, double *__restrict__ E, int accumulate,
                const double *__restrict__ S, int stall, long long limit)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int64_t coef[2][kTN];         // per item (alternating): offsets of leaf k, -1: none
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *base = smem_raw + ((1024u - (tc_smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = tc_smem_u32(base);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        tc_mbar_init(tc_smem_u32(&mbar[0]));
        tc_mbar_init(tc_smem_u32(&mbar[1]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t bar0 = tc_smem_u32(&mbar[0]), bar1 = tc_smem_u32(&mbar[1]);

    float a[kTM * kTK / kThreads], b[kTN * kTK / kThreads];
    auto load = [&](const TcItem &q, int col0) {
        const bool cok = col0 + lane < q.Pn;
#pragma unroll
        for (int i = 0; i < kTM * kTK / kThreads; ++i)
            a[i] = (cok && 8 * i < q.arows) ? __ldg(q.arow + (int64_t)8 * i * q.Pn + col0) : 0.f;
#pragma unroll
        for (int i = 0; i < kTN * kTK / kThreads; ++i)
            b[i] = (cok && q.boff[i] >= 0) ? (float)__ldg(C + q.boff[i] + col0) : 0.f;
    };

    uint32_t chunk = 0;                      // stages used so far by this CTA (phase tracking)
    int it = blockIdx.x, ib = 0;
    TcItem cur, nxt;
    if (it < nitems) {
        tc_item(G, P, S, items[it], warp, lane, cur, coef[0]);
        load(cur, 0);
    }
    while (it < nitems) {
        const int nit = it + gridDim.x;
        for (int kc = 0; kc < cur.nk; ++kc, ++chunk) {
            const uint32_t buf = chunk & 1, bar = buf ? bar1 : bar0;
            // the stage's previous products (chunk - 2) must have read it
            if (chunk >= 2 && !tc_mbar_wait(bar, ((chunk - 2) >> 1) & 1, limit)) abort_flag = 1;
            uint8_t *st = base + buf * kStage;
            uint8_t *ahi = st, *alo = st + kATile, *bhi = st + 2 * kATile, *blo = st + 2 * kATile + kBTile;
#pragma unroll
            for (int i = 0; i < kTM * kTK / kThreads; ++i) {
                const float h = tf32_round(a[i]);
                const uint32_t o = tc_swz(warp + 8 * i, lane);
                *reinterpret_cast<float *>(ahi + o) = h;
                *reinterpret_cast<float *>(alo + o) = tf32_round(a[i] - h);
            }
#pragma unroll
            for (int i = 0; i < kTN * kTK / kThreads; ++i) {
                const float h = tf32_round(b[i]);
                const uint32_t o = tc_swz(warp + 8 * i, lane);
                *reinterpret_cast<float *>(bhi + o) = h;
                *reinterpret_cast<float *>(blo + o) = tf32_round(b[i] - h);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (abort_flag) break;                              // CTA-uniform after the barrier
            // the next chunk's loads (of this item or the next) fly during the products
            if (kc + 1 < cur.nk) {
                load(cur, (kc + 1) * kTK);
            } else if (nit < nitems) {
                tc_item(G, P, S, items[nit], warp, lane, nxt, coef[ib ^ 1]);
                load(nxt, 0);
            }
            if (tid == 0 && !stall) {
                tc_fence_after();
                const uint32_t s_ahi = sbase + buf * kStage, s_alo = s_ahi + kATile;
                const uint32_t s_bhi = s_ahi + 2 * kATile, s_blo = s_bhi + kBTile;
#pragma unroll
                for (int s = 0; s < kTK / 8; ++s) {             // 8 TF32 values = 32 bytes per k-step
                    const uint32_t first = (kc == 0 && s == 0) ? 0u : 1u;
                    tc_mma(tmem, tc_desc(s_ahi + 32 * s), tc_desc(s_bhi + 32 * s), first);
                    tc_mma(tmem + kTN, tc_desc(s_ahi + 32 * s), tc_desc(s_blo + 32 * s), first);
                    tc_mma(tmem + kTN, tc_desc(s_alo + 32 * s), tc_desc(s_bhi + 32 * s), 1u);
                }
                tc_commit(bar);
            }
        }
        if (abort_flag) break;
        // the last stage's commit covers every product of this item
        {
            const uint32_t last = chunk - 1;
            if (!tc_mbar_wait((last & 1) ? bar1 : bar0, (last >> 1) & 1, limit)) abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) break;
        tc_fence_after();
        // warp w reads TMEM lanes 32 (w mod 4) .. +31 (its rows), columns of half w / 4
        {
            const int quad = warp & 3, half = warp >> 2;
            const int row = cur.row0 + 32 * quad + lane;
            const uint32_t tl_addr = tmem + ((uint32_t)(32 * quad) << 16);
#pragma unroll
            for (int cc = 0; cc < kTN / 2; cc += 16) {
                const int c0 = half * (kTN / 2) + cc;
                float hh[16], hl[16];
                tc_ld16(tl_addr + c0, hh);
                tc_ld16(tl_addr + kTN + c0, hl);
                tc_wait_ld();
                if (row < cur.Pn) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int64_t off = coef[ib][c0 + j];
                        if (off < 0) continue;
                        const double v = (double)(hh[j] + hl[j]);
                        double *e = E + off + row;
                        *e = accumulate ? *e + v : v;
                    }
                }
            }
        }
        // tensor-memory reads done before the next item's products overwrite it
        tc_fence_before();
        __syncthreads();
        it = nit;
        cur = nxt;
        ib ^= 1;
    }
    // drain: wait (bounded) for any commit still outstanding, then free TMEM
    if (abort_flag && chunk > 0 && tid == 0) {
        const uint32_t last = chunk - 1;
        const long long t0 = clock64();
        const uint32_t bar = (last & 1) ? bar1 : bar0;
        while (!tc_mbar_try(bar, (last >> 1) & 1))
            if (clock64() - t0 > limit) break;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
}

// Test hook for the bounded waits: with WMG_TEST_STALL_TENSOR_PRODUCTS=1 in
// the environment at launch time, the issuing thread issues no products and
// no commits, so the waits run out after kStallWaitCycles and the timeout
// path (error flag, TMEM freed, WMG_ERR_TIMEOUT at the next synchronising
// call) runs without any fault: nothing is in flight.
static bool tc_stall_requested()
{
    const char *v = std::getenv("WMG_TEST_STALL_TENSOR_PRODUCTS");
    return v && v[0] == '1';
}

void launch_leaf_apply_tc(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles, const double *C,
                          double *E, int accumulate, const double *S, cudaStream_t st)
{
    if (ntiles <= 0) return;
    ensure_dyn_smem((const void *)k_leaf_apply_tc, (int)kSmem);
    count_launches(1);
    const int grid = min(ntiles, 2 * num_sms());                 // two CTAs per SM (shared memory)
    const bool stall = tc_stall_requested();
    k_leaf_apply_tc<<<grid, kThreads, kSmem, st>>>(G, P, tiles, ntiles, C, E, accumulate, S, stall ? 1 : 0,
                                                   stall ? kStallWaitCycles : kWaitCycles);
}

int tc_error_take()
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
    }
    return v;
}

}  // namespace wmg
