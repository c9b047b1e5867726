// haar.cu -- Haar wavelet-packet restriction/prolongation and the leaf
// (coarsest-level) exact solves of the WMG cycle.
//
// Restriction by the four 2D Haar operators (eq. intops, eq. intops_wav,
// eq. 1of4-4of4), applied recursively to depth L (Section 3.1.3), acts
// independently on every 2^L x 2^L pixel block: the result is the block's 2D
// Walsh-Hadamard transform scaled by 2^-L, with the packet path read from the
// bit-reversed Walsh indices. The kernels below stage a strip of blocks in
// shared memory, run L butterfly stages along x and L along y, and scatter to
// the leaf layout C[k][cy][cx] (k = sum_d id_d 4^(L-d), id = 2*hy + hx, the
// d-th split's high-pass bits in y and x). Prolongation (synthesis) is the
// same transform run backwards. Fused epilogues update the preconditioner's
// FP64 iterate and write the operator-precision copies (row-major and
// transposed) that the next projection reads.
//
// Leaf solves: e_k = D_k^-1 c_k with the stored symmetric inverse. FP64 plans
// here: one CTA per leaf streams D_k^-1 once for every problem of a
// same-geometry group, thread i forming e_i = sum_j D^-1[j][i] c_j (rows read
// coalesced, symmetry). FP32 plans: a tensor-core matrix product per leaf
// and group of problems (leaf_tc.cu).
#include "kern_common.cuh"

namespace wmg {

__device__ __forceinline__ int bitrev_bits(int u, int L) { return L ? (int)(__brev((unsigned)u) >> (32 - L)) : 0; }

// Bits 0..7 of v moved to the even positions 0, 2, .., 14.
__device__ __forceinline__ int spread_bits(int v)
{
    v = (v | (v << 4)) & 0x0F0F;
    v = (v | (v << 2)) & 0x3333;
    v = (v | (v << 1)) & 0x5555;
    return v;
}

// Leaf index of Walsh position (uy, ux) inside a block (L <= 8).
__device__ __forceinline__ int leaf_of(int uy, int ux, int L)
{
    return (spread_bits(bitrev_bits(uy, L)) << 1) | spread_bits(bitrev_bits(ux, L));
}

// Shared-memory column of strip column x: one pad slot after every B-wide
// segment, so that the block columns a warp touches at one Walsh position
// (stride B + 1 doubles) fall in different banks.
__device__ __forceinline__ int padx(int x, int L) { return x + (x >> L); }

// Thread layout over a 2D loop of `width` columns: tx runs along the
// columns, ty along the rows (threads with ty >= ny idle). One division per
// tile instead of one per element.
struct Lay {
    int tx, ty, nx, ny;
};
__device__ __forceinline__ Lay lay(int width)
{
    const int nx = min(width, (int)blockDim.x);
    return Lay{(int)threadIdx.x % nx, (int)threadIdx.x / nx, nx, (int)blockDim.x / nx};
}

// In-place Walsh-Hadamard butterflies over a B x W strip in shared memory
// (pitch pw, columns padded by padx), along x (within every B-wide segment)
// then along y, in the compute type TC.
template <class TC>
__device__ __forceinline__ void strip_wht(TC *sm, int B, int W, int L, int pw)
{
    const Lay lx = lay(W >> 1);
    for (int st = 0; st < L; ++st) {
        const int hbit = 1 << st;
        if (lx.ty < lx.ny)
            for (int r = lx.ty; r < B; r += lx.ny) {
                TC *row = sm + r * pw;
                for (int pi = lx.tx; pi < (W >> 1); pi += lx.nx) {
                    const int i = ((pi >> st) << (st + 1)) | (pi & (hbit - 1));
                    const int i0 = padx(i, L), i1 = padx(i + hbit, L);
                    const TC a = row[i0], b = row[i1];
                    row[i0] = a + b;
                    row[i1] = a - b;
                }
            }
        __syncthreads();
    }
    const Lay ly = lay(W);
    for (int st = 0; st < L; ++st) {
        const int hbit = 1 << st;
        if (ly.ty < ly.ny)
            for (int pi = ly.ty; pi < (B >> 1); pi += ly.ny) {
                const int i = ((pi >> st) << (st + 1)) | (pi & (hbit - 1));
                TC *r0 = sm + i * pw, *r1 = sm + (i + hbit) * pw;
                for (int x = ly.tx; x < W; x += ly.nx) {
                    const int col = padx(x, L);
                    const TC a = r0[col], b = r1[col];
                    r0[col] = a + b;
                    r1[col] = a - b;
                }
            }
        __syncthreads();
    }
}

// Analysis: tile = {prob, y0, x0, W}; strip of B rows x W columns. The
// butterflies run in TC (FP64, or FP32 in the WMG cycle of FP32 plans:
// GB300 issues FP64 arithmetic at a small fraction of the FP32 rate)
// whatever the storage types.
template <class TIn, class TOut, int MODE, class TC>
__global__ void __launch_bounds__(256)
k_haar_analysis(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
                const int4 *__restrict__ tiles, int ntiles, HaarArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    TC *sm = reinterpret_cast<TC *>(smraw);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(a.S, pd.slot)) continue;
        const GeomDev &g = G[pd.geom];
        const int n = g.n, B = g.B, L = g.L, W = tl.w, pw = W + (W >> L) + 1;
        const TIn *in = static_cast<const TIn *>(a.in) + pd.img + (int64_t)tl.y * n + tl.z;
        {
            const Lay l = lay(W);
            if (l.ty < l.ny)
                for (int r = l.ty; r < B; r += l.ny)
                    for (int x = l.tx; x < W; x += l.nx) sm[r * pw + padx(x, L)] = (TC)in[(int64_t)r * n + x];
        }
        __syncthreads();
        strip_wht(sm, B, W, L, pw);
        const TC scale = TC(1) / (TC)B;                              // a power of two: exact
        const int nb = W >> L, cy = tl.y >> L, cx0 = tl.z >> L;
        TOut *C = static_cast<TOut *>(a.out) + pd.coef + (int64_t)cy * g.nc + cx0;
        {
            // consecutive threads: consecutive blocks of one Walsh position,
            // i.e. consecutive entries of one leaf's coefficient vector
            const Lay l = lay(nb);
            if (l.ty < l.ny)
                for (int u = l.ty; u < B * B; u += l.ny) {
                    const int uy = u >> L, ux = u & (B - 1);
                    const int k = leaf_of(uy, ux, L);
                    if (MODE != HA_STORE && (k < pd.kout0 || k >= pd.kout1)) continue;
                    TOut *Ck = C + (int64_t)k * g.P;
                    const TC *src = sm + uy * pw + ux;
                    for (int bc = l.tx; bc < nb; bc += l.nx) {
                        const TOut v = (TOut)(src[bc * (B + 1)] * scale);
                        if (MODE == HA_SUB_MASKED) Ck[bc] -= v;
                        else Ck[bc] = v;
                    }
                }
        }
        __syncthreads();
    }
}

// Synthesis: the transpose of the analysis (butterflies in TC).
template <class TIn, class TOut, int MODE, class TC>
__global__ void __launch_bounds__(256)
k_haar_synthesis(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
                 const int4 *__restrict__ tiles, int ntiles, HaarArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    TC *sm = reinterpret_cast<TC *>(smraw);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const ProbDev pd = P[tl.x];
        if (!slot_active(a.S, pd.slot)) continue;
        const GeomDev &g = G[pd.geom];
        const int n = g.n, B = g.B, L = g.L, W = tl.w, pw = W + (W >> L) + 1;
        const int nb = W >> L, cy = tl.y >> L, cx0 = tl.z >> L;
        const TIn *E = static_cast<const TIn *>(a.in) + pd.coef + (int64_t)cy * g.nc + cx0;
        {
            const Lay l = lay(nb);
            if (l.ty < l.ny)
                for (int u = l.ty; u < B * B; u += l.ny) {
                    const int uy = u >> L, ux = u & (B - 1);
                    const int k = leaf_of(uy, ux, L);
                    const bool in = MODE != HS_STORE_MASKED || (k >= pd.kin0 && k < pd.kin1);
                    const TIn *Ek = E + (int64_t)k * g.P;
                    TC *dst = sm + uy * pw + ux;
                    for (int bc = l.tx; bc < nb; bc += l.nx) dst[bc * (B + 1)] = in ? (TC)Ek[bc] : TC(0);
                }
        }
        __syncthreads();
        strip_wht(sm, B, W, L, pw);
        const TC scale = TC(1) / (TC)B;
        TOut *out = static_cast<TOut *>(a.out);
        {
            const Lay l = lay(W);
            if (l.ty < l.ny)
                for (int r = l.ty; r < B; r += l.ny)
                    for (int x = l.tx; x < W; x += l.nx) {
                        const int64_t j = pd.img + (int64_t)(tl.y + r) * n + tl.z + x;
                        TC *cell = sm + r * pw + padx(x, L);
                        const TC v = *cell * scale;
                        if (MODE == HS_CORRECT) {
                            const double zv = a.z[j] + (double)v;
                            a.z[j] = zv;
                            const TOut zt = (TOut)zv;
                            *cell = (TC)zt;
                            if (out) out[j] = zt;
                        } else {
                            const TOut vt = (TOut)v;
                            *cell = (TC)vt;
                            out[j] = vt;
                        }
                    }
        }
        if (a.outT) {
            __syncthreads();
            TOut *outT = static_cast<TOut *>(a.outT) + pd.img + tl.y;
            const Lay l = lay(B);
            if (l.ty < l.ny)
                for (int x = l.ty; x < W; x += l.ny) {
                    const int col = padx(x, L);
                    for (int r = l.tx; r < B; r += l.nx)
                        outT[(int64_t)(tl.z + x) * n + r] = (TOut)sm[r * pw + col];
                }
        }
        __syncthreads();
    }
}

static void set_smem(const void *fn, int bytes)
{
    if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <class TIn, class TOut>
void launch_haar_analysis(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                          int smem_elems, const HaarArgs &a, cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    const int grid = min(ntiles, num_sms() * 8);
#define WMG_HA(M)                                                                                  \
    case M:                                                                                        \
        if (a.fp32) {                                                                              \
            const int bytes = smem_elems * (int)sizeof(float);                                     \
            set_smem((const void *)k_haar_analysis<TIn, TOut, M, float>, bytes);                   \
            k_haar_analysis<TIn, TOut, M, float><<<grid, 256, bytes, st>>>(G, P, tiles, ntiles, a); \
        } else {                                                                                   \
            const int bytes = smem_elems * (int)sizeof(double);                                    \
            set_smem((const void *)k_haar_analysis<TIn, TOut, M, double>, bytes);                  \
            k_haar_analysis<TIn, TOut, M, double><<<grid, 256, bytes, st>>>(G, P, tiles, ntiles, a); \
        }                                                                                          \
        break;
    switch (a.mode) { WMG_HA(HA_STORE) WMG_HA(HA_SUB_MASKED) WMG_HA(HA_STORE_MASKED) default: break; }
#undef WMG_HA
}

template <class TIn, class TOut>
void launch_haar_synthesis(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                           int smem_elems, const HaarArgs &a, cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    const int grid = min(ntiles, num_sms() * 8);
#define WMG_HS(M)                                                                                  \
    case M:                                                                                        \
        if (a.fp32) {                                                                              \
            const int bytes = smem_elems * (int)sizeof(float);                                     \
            set_smem((const void *)k_haar_synthesis<TIn, TOut, M, float>, bytes);                  \
            k_haar_synthesis<TIn, TOut, M, float><<<grid, 256, bytes, st>>>(G, P, tiles, ntiles, a); \
        } else {                                                                                   \
            const int bytes = smem_elems * (int)sizeof(double);                                    \
            set_smem((const void *)k_haar_synthesis<TIn, TOut, M, double>, bytes);                 \
            k_haar_synthesis<TIn, TOut, M, double><<<grid, 256, bytes, st>>>(G, P, tiles, ntiles, a); \
        }                                                                                          \
        break;
    switch (a.mode) { WMG_HS(HS_STORE) WMG_HS(HS_STORE_MASKED) WMG_HS(HS_CORRECT) default: break; }
#undef WMG_HS
}

// ---------------------------------------------------------------------------
// Leaf solves. tile = {first problem p0, leaf k, problem count np, 0}; the
// problems p0 .. p0+np-1 share one geometry. NPB problems per pass.
// ---------------------------------------------------------------------------
template <int NPB>
__global__ void __launch_bounds__(256)
k_leaf_apply(const GeomDev *__restrict__ G, const ProbDev *__restrict__ P,
             const int4 *__restrict__ tiles, int ntiles, const double *__restrict__ C,
             double *__restrict__ E, int accumulate, const double *__restrict__ S)
{
    typedef double T;
    __shared__ T cb[NPB][256];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const GeomDev &g = G[P[tl.x].geom];
        const int Pn = g.P, k = tl.y;
        const T *__restrict__ Dk = static_cast<const T *>(g.leafinv) + (int64_t)k * Pn * Pn;
        for (int pb = 0; pb < tl.z; pb += NPB) {
            const int np = min(NPB, tl.z - pb);
            for (int q = threadIdx.x; q < NPB * Pn; q += blockDim.x) {
                const int pi = q / Pn, j = q - pi * Pn;
                T v = T(0);
                if (pi < np) {
                    const ProbDev pd = P[tl.x + pb + pi];
                    if (slot_active(S, pd.slot)) v = C[pd.coef + (int64_t)k * Pn + j];
                }
                cb[pi][j] = v;
            }
            __syncthreads();
            const int i = threadIdx.x;
            if (i < Pn) {
                T acc[NPB];
#pragma unroll
                for (int u = 0; u < NPB; ++u) acc[u] = T(0);
#pragma unroll 8
                for (int j = 0; j < Pn; ++j) {
                    const T d = ldg_t(Dk + (int64_t)j * Pn + i);
#pragma unroll
                    for (int u = 0; u < NPB; ++u) acc[u] = fma_t(d, cb[u][j], acc[u]);
                }
#pragma unroll
                for (int u = 0; u < NPB; ++u) {
                    if (u < np) {
                        const ProbDev pd = P[tl.x + pb + u];
                        if (!slot_active(S, pd.slot)) continue;
                        T *e = E + pd.coef + (int64_t)k * Pn + i;
                        *e = accumulate ? *e + acc[u] : acc[u];
                    }
                }
            }
            __syncthreads();
        }
    }
}

void launch_leaf_apply(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                       const double *C, double *E, int accumulate, const double *S, bool fp32,
                       cudaStream_t st)
{
    if (ntiles <= 0) return;
    count_launches(1);
    if (fp32) {                       // F32 plans: tensor cores (leaf_tc.cu)
        launch_leaf_apply_tc(G, P, tiles, ntiles, C, E, accumulate, S, st);
        return;
    }
    const int grid = min(ntiles, num_sms() * 8);
    k_leaf_apply<4><<<grid, 256, 0, st>>>(G, P, tiles, ntiles, C, E, accumulate, S);
}

#define WMG_INST(TI, TO)                                                                         \
    template void launch_haar_analysis<TI, TO>(const GeomDev *, const ProbDev *, const int4 *,  \
                                               int, int, const HaarArgs &, cudaStream_t);        \
    template void launch_haar_synthesis<TI, TO>(const GeomDev *, const ProbDev *, const int4 *, \
                                                int, int, const HaarArgs &, cudaStream_t);
WMG_INST(float, float)
WMG_INST(double, double)
WMG_INST(float, double)
WMG_INST(double, float)
#undef WMG_INST
// synthesis into bfloat16 operator copies (plans with BF16 operator storage)
template void launch_haar_synthesis<double, __nv_bfloat16>(const GeomDev *, const ProbDev *, const int4 *, int, int,
                                                           const HaarArgs &, cudaStream_t);

}  // namespace wmg
