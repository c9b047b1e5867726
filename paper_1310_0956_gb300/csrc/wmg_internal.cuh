// wmg_internal.cuh -- shared declarations of the GB300 kernels and the host
// engine behind include/wmgct.h. Device code targets sm_103a only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "wmgct.h"

namespace wmg {

// ---------------------------------------------------------------------------
// Device-side tables. Every kernel is table driven: a launch covers a list of
// tiles, each tile belongs to one problem, each problem points at one
// geometry. A single reconstruction, a same-geometry batch and the
// band-local multi-image products of the hybrid cycle are all just tables.
// ---------------------------------------------------------------------------

// Per-angle constants of the FP32 kernels (built in FP64 on the host).
// Split trigonometry: c = chi + clo with chi a multiple of 2^-12; chord of a
// unit pixel at distance d: clamp(hw_inv - d * inv_ab, 0, lmax); frame =
// rows of the image (steep, |c| >= |s|) or of its transpose (cc, ss = the
// frame's cos / sin): inv_cc = 1/cc, slope = ss/cc, inv_slope = cc/ss,
// hwx = hw/|cc|.
// Normalised chord: L(d) = lmax * sat(wb - d * wa) with wa = 1/beta,
// wb = hw/beta (sat = clamp to [0, 1], one saturating FMA); axis-aligned
// angles use wa = 2^22, wb = 2^21 + 1/2, which is the step 1 / 1/2 / 0 at the
// half-integer distances those rays have to pixel centres.
// The fields the unit-bin backprojector reads are the first 28 bytes.
struct __align__(16) AngleF {
    float chi, clo, shi, slo;
    float wa, wb, lmax;       // normalised chord
    float flags;              // int bits: 1 = steep, 2 = axis-aligned
    float hw_inv, inv_ab, hwx, hw;
    float inv_cc, slope, inv_slope, cc;   // cc: frame cos
};

// Immutable per-geometry data (lengths in pixel widths, h = 1/n applied to
// the weights at the end).
struct GeomDev {
    int n, m, D, L;          // image side, angles, bins per angle, Haar levels
    int nc, P, K, B;         // leaf side n/2^L, P = nc^2, K = 4^L leaves, B = 2^L block side
    double h;                // pixel width on the unit square
    double t0, dt;           // detector offset and spacing (pixel widths)
    double lambda, omega;    // Tikhonov parameter, smoother damping
    const double2 *cs64;     // (cos, sin) per angle, FP64
    const float2 *cs32;      // round-to-nearest FP32 copy
    const float4 *csx;       // (c_hi, c_lo, s_hi, s_lo): c_hi = c rounded to a
                             // multiple of 2^-12, c_lo = c - c_hi in FP32
    const void *dinv;        // N: 1/D~ (0 where D~ = 0), operator precision
    const void *leafinv;     // K*P*P: leaf inverses (FP64 for F64 plans, FP32 for F32 plans)
    const void *sirtR;       // M: 1/row sums (0 if empty)
    const void *sirtC;       // N: 1/column sums (0 if empty)
    const AngleF *angf;      // m per-angle constants (FP32 kernels)
    float hf, dtf, t0f, hDf; // FP32 copies of h, dt, t0 and (D-1)/2
    int unit;                // bins of one pixel width, no offset: the FP32
                             // backprojector takes its two-bin path (1); 2: in
                             // addition both candidate bins of every pixel of
                             // every 32 x 32 tile lie on the detector at every
                             // angle, so that path needs no bounds checks
    int kernel;              // WMG_KERNEL_STRIP or WMG_KERNEL_JOSEPH
    int qpair;               // even m, angle a + m/2 = angle a turned by pi/2 in
                             // the FP32 table (the unit-bin backprojector pairs them)
};

// A weight counts as a nonzero of W when its chord exceeds this many pixel
// widths: lines through a pixel corner give chords of rounding size (~1e-16)
// that are zero in exact arithmetic.
constexpr double kNnzEps = 1e-12;

// Fills the FP32 per-angle table from FP64 (cos, sin) pairs.
void fill_angle_table(const double2 *cs, int m, int kernel, AngleF *out);

// Host tables of one geometry (engine.cu): angles == NULL means equiangular
// in [0, pi); every array holds m entries and is the caller's. Allocates
// nothing, so the allocation-free entry point builds its tables with it too.
void geometry_tables(int m, const double *angles, int kernel, double2 *cs, float2 *cs32, float4 *csx,
                     AngleF *angf);
// Fields of a geometry derived from n, m, D, h, dt, t0 and its FP32 angle
// table: FP32 copies of the scalars, the unit-bin flag and quarter-turn pairs.
void geometry_scalars(GeomDev &gd, const AngleF *angf);

// One problem slot (or one virtual image of a multi-image product).
struct ProbDev {
    int geom;                // index into the GeomDev table
    int slot;                // owning real problem (scalar / flag index)
    int64_t img;             // element offset of its image-sized vectors
    int64_t sino;            // element offset of its sinogram-sized vectors
    int64_t coef;            // element offset of its packet-coefficient vectors
    int kin0, kin1;          // leaf range read by masked synthesis
    int kout0, kout1;        // leaf range written by masked analysis
};

// Per-problem scalar slots (FP64), S[slot * NSCAL + i].
enum Scal : int {
    SC_GAMMA = 0, SC_DELTA, SC_ALPHA, SC_BETA, SC_S0, SC_RES, SC_PP, SC_ITERS, SC_ACTIVE,
    SC_STATUS, SC_RTOL, SC_MAXIT, SC_HNORM, SC_WNORM2, SC_GNEW,
    SC_HELD,                 // server: SC_ACTIVE of a slot held out of a phase group
    NSCAL = 16
};

// Work lists: int4 tiles, problem index in .x.
//  project:     {prob, angle a, first ray k0, 0}   -- 32 rays of one angle
//  backproject: {prob, iy0, ix0, 0}                -- 32 x 32 pixel tile
//  haar:        {prob, first pixel row y0, first column x0, width}
//  vec (image): {prob, first element, count, 0}
//  vec (sino):  {prob, first element, count, 0}
//  leaf:        {geom, leaf k, first problem in group, problem count}

// ---------------------------------------------------------------------------
// Host-side error state
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
int32_t fail(int32_t code, const std::string &msg);
// library-wide kernel launch counter (every launcher adds its launches)
void count_launches(int n);

#define WMG_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return ::wmg::fail(WMG_ERR_CUDA, std::string(#call) + ": " +            \
                                                 cudaGetErrorString(e_));           \
    } while (0)

// ---------------------------------------------------------------------------
// Kernel launchers (projector.cu, haar.cu, setup.cu, krylov.cu).
// `T` = operator element type (float or double).
// ---------------------------------------------------------------------------

// Epilogue selectors of the backprojector (see projector.cu for the exact
// formulas; y = h * sum of weighted bins at a pixel).
enum BpEpi : int {
    BP_STORE = 0,      // out_op = y                                      (T)
    BP_CGLS_S,         // x += alpha p; s = y - lambda x; z1 = w D~^-1 s;  (FP64) + z1 copies
    BP_RESID,          // r1 = s - y - lambda z                            (T)
    BP_POST,           // z += w D~^-1 (s - y - lambda z); dot s.z         (FP64)
    BP_APPLY_A,        // out = y + lambda v                               (T or FP64)
    BP_SIRT,           // x += C (y - lambda x)                            (FP64) + copies
    BP_GMRES_W,        // w = y + lambda u                                 (FP64)
    BP_ATB,            // f = y (FP64), dot f.f
};

struct BpArgs {
    int epi;
    int ctas_per_sm;         // grid = min(tiles, SMs x this) (0: 8); any value gives the same bits
    int unit;                // FP32 kernels: every geometry of the launch has unit bins
    const void *sino;        // T, sinogram input pool
    void *out_op;            // T image output (BP_STORE, BP_RESID, BP_APPLY_A)
    double *x, *s, *z, *p;   // FP64 Krylov vectors (pools)
    const void *v_op;        // T image (BP_APPLY_A, BP_RESID uses z FP64)
    void *copy_op;           // T copy of the updated FP64 vector (row-major)
    void *copyT_op;          // T transposed copy
    double *part;            // per-tile partial dot (or NULL)
    const double *S;         // per-problem scalars
    double *out64;           // FP64 output (BP_GMRES_W, BP_ATB, BP_APPLY_A in FP64 mode)
    const int *part_base;    // FP32 kernels: problem p's first partial index (its one-image tile list)
    int bf16;                // FP32 kernels: sinogram input and T image copies / outputs stored as bfloat16
};

struct PjArgs {
    int ctas_per_sm;         // grid = min(tiles, SMs x this) (0: 8); any value gives the same bits
    const void *img;         // T image pool (row-major)
    const void *imgT;        // T transposed image pool (for |sin| > |cos| angles)
    void *sino;              // T sinogram output pool
    double *part;            // per-tile partial ||q||^2 (or NULL)
    const double *S;         // scalars (active flags), or NULL = all active
    const int *part_base;    // FP32 kernel: problem p's first partial index (its one-image tile list)
    int group;               // FP32 kernel: images per tile of the tile list (1 or kProjGroup)
    int bf16;                // FP32 kernels: image input and sinogram output stored as bfloat16
};

// Images per group tile of the FP32 projector (consecutive problems of one
// geometry share the weight computation). The backprojector keeps one image
// per tile: grouping cost it more occupancy than it saved (measured).
constexpr int kProjGroup = 8;
// Images per group tile of the FP32 backprojector (a divisor of kProjGroup:
// each projector group's problems form kProjGroup / kBpGroup such tiles;
// 4 measured 14 % slower than 8 on the 256-image batch).
constexpr int kBpGroup = 8;

template <class T>
void launch_project(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                    const PjArgs &a, cudaStream_t st);
template <class T>
void launch_backproject(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                        const BpArgs &a, cudaStream_t st);
// nnz of W: rays x pixels with a nonzero weight, added into *count (one problem)
void launch_count_nnz(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                      unsigned long long *count, cudaStream_t st);
void launch_project_f32(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                        const PjArgs &a, cudaStream_t st);
void launch_backproject_f32(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                            const BpArgs &a, bool unit, cudaStream_t st);
// Group tiles (kProjGroup images) with the pixels staged by TMA
// (projector_tma.cu): pools a.img / a.imgT of `count` images of side n (a
// multiple of 4), problem p's image number img / n^2 there, the images of a
// group consecutive. false: not launched (no tensor-map encoder, or
// unaligned pools): use launch_project_f32.
bool launch_project_f32_tma(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                            const PjArgs &a, int n, int64_t count, cudaStream_t st);
// Error flag of the TMA projector since the last call (0: none; 1: a staged
// copy wait timed out; 2: a candidate pixel outside its box), cleared.
// Synchronising.
int tma_error_take();
// Group tiles {first problem, iy0, ix0, kBpGroup} of the FP32 backprojector
// (projector_f32.cu): geometries with unit == 2 and quarter-turn pairs, FP32
// storage; false: not launched (bfloat16 storage): use the one-image tiles.
bool launch_backproject_f32_group(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                                  const BpArgs &a, cudaStream_t st);
// Error flag of the group backprojector since the last call (0: none; 1: a
// candidate bin outside its staged window), cleared. Synchronising.
int bpg_error_take();
template <class T>
void launch_transpose(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                      const void *src, void *dst, cudaStream_t st);

// Haar packet transforms (haar.cu).
enum HaarMode : int {
    HA_STORE = 0,      // C = Q^T img
    HA_SUB_MASKED,     // C[k] -= (Q^T img)[k] for k in [kout0, kout1)
    HA_STORE_MASKED,   // C[k]  = (Q^T img)[k] for k in [kout0, kout1)
};
enum HaarSynMode : int {
    HS_STORE = 0,      // img_op = Q E (T)                       + optional transposed copy
    HS_STORE_MASKED,   // img_op = Q (E masked to [kin0, kin1))  + optional transposed copy
    HS_CORRECT,        // z += Q E (FP64) ; copies of z in T     (row-major + transposed)
};
struct HaarArgs {
    int mode;
    const void *in;          // analysis: T image; synthesis: T coefficients
    void *out;               // analysis: T coefficients; synthesis: T image
    void *outT;              // synthesis: transposed T copy (or NULL)
    double *z;               // HS_CORRECT: FP64 vector updated in place
    const double *S;         // scalars (active flags) or NULL
    int fp32;                // butterflies in FP32 (the WMG cycle of FP32 plans), else FP64
};
template <class TIn, class TOut>
void launch_haar_analysis(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                          int smem_elems, const HaarArgs &a, cudaStream_t st);
template <class TIn, class TOut>
void launch_haar_synthesis(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                           int smem_elems, const HaarArgs &a, cudaStream_t st);

// Lets kernel `fn` take `bytes` of dynamic shared memory on the current
// device (once per device and kernel; thread-safe).
void ensure_dyn_smem(const void *fn, int bytes);

// Leaf solves E[k] = Dinv_k C[k] for the problems of a group (haar.cu):
// FP64 inverses and arithmetic (fp32 = false) or FP32 inverses on the tensor
// cores (F32 plans, launch_leaf_apply_tc); C and E are FP64 in both.
// accumulate = 1 adds into E.
void launch_leaf_apply(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                       const double *C, double *E, int accumulate, const double *S, bool fp32,
                       cudaStream_t st);

// The FP32 form on the tensor cores (leaf_tc.cu): tcgen05 TF32 products of
// split operands, FP32 accumulation in tensor memory, leaves of P <= 256.
// Its tiles are work items {first problem, leaf k, count <= kLeafTcProblems
// (consecutive same-geometry problems), row block of kLeafTcRows rows}.
constexpr int kLeafTcProblems = 64;
constexpr int kLeafTcRows = 128;
void launch_leaf_apply_tc(const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles, const double *C,
                          double *E, int accumulate, const double *S, cudaStream_t st);
// Error flag of the tensor-core leaf solves since the last call (0: none; 1:
// a wait for the products timed out), cleared. Synchronising.
int tc_error_take();

// Setup (setup.cu).
// fp32: profiles and pair sums in FP32 (FP64 accumulation over angles).
int32_t build_leaf_inverses(const GeomDev &g_host, const GeomDev *g_dev, void *leafinv_out, bool fp32,
                            cudaStream_t st);

// Elementwise / reduction kernels (krylov.cu), all FP64 Krylov state.
void launch_vec_kernel(int op, const ProbDev *P, const int4 *tiles, int ntiles,
                       const GeomDev *G, void *const *ptrs, const double *S, double *part,
                       int is_f32, cudaStream_t st);
void launch_finalize(int op, int nprob, const int *tile_begin, const int *tile_end,
                     const double *partA, const double *partB, double *S, int iter_idx,
                     double *hist, int hist_stride, cudaStream_t st);

}  // namespace wmg
