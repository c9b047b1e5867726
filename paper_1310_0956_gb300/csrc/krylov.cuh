// krylov.cuh -- argument blocks and launchers of the Krylov vector kernels.
#pragma once

#include "wmg_internal.cuh"

namespace wmg {

enum ImgOp : int {
    IMG_PUPDATE = 0,   // p = z + beta p (FP64), copies of p, part = |p|^2
    IMG_PINIT,         // p = z, copies, part = |p|^2
    IMG_FIRST_SWEEP,   // z = omega D~^-1 s, copies of z
    IMG_ZERO_RESID,    // z = 0, r1_op = s
    IMG_LOAD,          // z = (double) in_op, copies of z
    IMG_COPY64,        // copies of z
    IMG_STORE_OUT,     // out_op = (T) z
    IMG_DOT_SZ,        // part = s.z
};

struct ImgArgs {
    double *z, *p;
    const double *s;
    const void *in_op;
    void *out_op;
    void *r1;
    void *copy_op, *copyT_op;
    double *part;
    const double *S;
    int bf16;                // copy_op / copyT_op stored as bfloat16 (FP32 plans with BF16 storage)
};

enum VecOp : int {
    VEC_R_UPDATE = 0,  // r -= alpha q, r_op = r            (sinogram)
    VEC_R_INIT,        // r = b_op, r_op = b_op              (sinogram)
    VEC_SIRT_R,        // r_op = R (b_op - q)                (sinogram)
    VEC_NRM2,          // part = |w|^2                       (image)
    VEC_SCALE_V,       // v = w / S[HNORM]                   (image)
    VEC_X_ADD,         // x += w                             (image)
    VEC_RESID64,       // v = f - w, part = |v|^2            (image)
    VEC_TO_OP,         // r_op = (T) w                       (image)
    VEC_SINO_DIFF,     // r_op = b_op - q                    (sinogram)
    VEC_NE_RES,        // part = |w - lambda x|^2            (image)
};

struct VecArgs {
    const GeomDev *G;
    double *r, *x, *v;
    const double *w, *f;
    const void *q, *b_op;
    void *r_op;
    double *part;
    const double *S;
};

enum FinOp : int {
    FIN_CGLS_INIT = 0,
    FIN_PNORM,
    FIN_CGLS_ALPHA,
    FIN_CGLS_RES,
    FIN_CGLS_BETA,
    FIN_SIRT_RES,
    FIN_STORE,         // S[store_slot] = sum of part_a
    FIN_SET_RES,       // S[RES] = sqrt(sum) / S[S0], end of a fixed-count solve
    FIN_BI_INIT,       // BiCGStab: |r0|^2 -> S0, rho = |r0|^2, alpha = omega = 1, beta = rho
    FIN_BI_ALPHA,      // <rh, v> -> alpha = rho / <rh, v>
    FIN_BI_OMEGA,      // <t, s>, <t, t> -> omega
    FIN_BI_RES,        // |r|^2, <rh, r> -> residual, stop tests, beta, rho
};

struct FinArgs {
    int op;
    int nprob;
    int precond;
    const double *part_a;
    const int *tb_a, *te_a;
    int ld_a, nsum_a;
    const double *part_b;
    const int *tb_b, *te_b;
    double *S;
    const double *lambda;    // per problem
    double *hist;
    int hist_ld;
    int store_slot;
    double *store_vec;       // FIN_STORE with nsum_a > 1: out[p*ld + i]
    int store_ld;
};

// BiCGStab vector steps over image chunks (scalars rho = S[GAMMA],
// alpha = S[ALPHA], omega = S[DELTA], beta = S[BETA]).
enum BicgOp : int {
    BI_INIT = 0,       // rh = r, p = 0, v = 0
    BI_P,              // p = r + beta (p - omega v)
    BI_RV,             // part_a = <rh, v>
    BI_S,              // s = r - alpha v
    BI_TS,             // part_a = <t, s>, part_b = <t, t>
    BI_XR,             // x += alpha ph + omega sh, r = s - omega t; part_a = |r|^2, part_b = <rh, r>
};

struct BicgArgs {
    double *x, *r, *rh, *p, *v, *s, *t, *ph, *sh;
    double *part_a, *part_b;
    const double *S;
};

struct GmArgs {
    int nprob, restart, ldp, j, init;
    int jslot;               // Arnoldi step: column jn[p] per problem instead of j
    double *S, *H, *cs, *sn, *g, *y;
    const double *h1, *h2;
    int *jn, *done;
    int *skip;               // per problem: 1 = no second Gram-Schmidt pass (which = 3 writes it)
    double *hist;
    int hist_ld;
};

template <class T>
void launch_img(int op, const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles,
                const ImgArgs &a, cudaStream_t st);
template <class T>
void launch_vec(int op, const ProbDev *P, const int4 *tiles, int ntiles, const VecArgs &a,
                cudaStream_t st);
void launch_finalize(const FinArgs &f, cudaStream_t st);
// jv (optional): per-slot column index replacing j; wnorm: also <w, w> into
// column j + 1 of the partials; skip (optional): per-slot flag of problems
// whose second Gram-Schmidt pass is skipped (zero dots, w untouched)
void launch_gm_dots(const ProbDev *P, const int4 *tiles, int ntiles, const double *V, int64_t vstride,
                    const double *w, int j, int ldp, double *part, const double *S, cudaStream_t st,
                    const int *jv = nullptr, bool wnorm = false, const int *skip = nullptr);
void launch_gm_axpy(const ProbDev *P, const int4 *tiles, int ntiles, const double *V, int64_t vstride,
                    double *w, int j, int ldp, const double *Hc, double *part, const double *S,
                    cudaStream_t st, const int *jv = nullptr, const int *skip = nullptr);
void launch_gm_combine(const ProbDev *P, const int4 *tiles, int ntiles, const double *V,
                       int64_t vstride, int ldp, const double *Yv, const int *jn, double *out,
                       const double *S, cudaStream_t st);
void launch_gm_setv(const ProbDev *P, const int4 *tiles, int ntiles, double *V, int64_t vstride,
                    int ldp, int j, const double *w, const double *S, cudaStream_t st,
                    const int *jv = nullptr);
// out = v_{jv[slot]} for every active problem
void launch_gm_getv(const ProbDev *P, const int4 *tiles, int ntiles, const double *V, int64_t vstride,
                    const int *jv, double *out, const double *S, cudaStream_t st);
void launch_bicg(int op, const ProbDev *P, const int4 *tiles, int ntiles, const BicgArgs &a, cudaStream_t st);
// which: 0 = Arnoldi scalar step, 1 = solve H y = g, 2 = restart,
// 3 = selective reorthogonalisation test (skip[] from the first pass)
void launch_gm_scalar(int which, const GmArgs &a, cudaStream_t st);

}  // namespace wmg
