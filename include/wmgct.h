/*
 * wmgct.h -- C ABI of the GB300 library for wavelet-multigrid (WMG)
 * preconditioned Krylov reconstruction in 2D parallel-beam algebraic
 * tomography (Cools, Ghysels, van Aarle, Sijbers, Vanroose, arXiv 1310.0956).
 *
 * The calls follow the paper's statement of the problem (Section 2.1,
 * eq. sys / sys_ne / sys_reg): an n x n image x on the unit square, m
 * projection angles, D detector bins per angle, a sinogram b of M = m*D
 * values; W holds the exact pixel-ray intersection lengths; the solvers
 * work on the normal equations (W^T W + lambda I) x = W^T b, optionally
 * preconditioned by one WMG cycle (Section 3.1).
 *
 * Conventions shared by every call
 *  - Image layout: row-major x[iy*n + ix], iy = 0 at y = -1/2, pixel width
 *    h = 1/n. Sinogram layout: angle-major b[a*D + k]. Ray (a, k) is the line
 *    p . (cos t_a, sin t_a) = t_k with t_k = ((k - (D-1)/2)*det_spacing +
 *    det_offset) * h. A line that runs exactly along a pixel edge gives half
 *    of the edge to each of the two pixels sharing it.
 *  - Batches: calls that take `count` operate on `count` problems of the same
 *    geometry stored back to back (problem q's image at x + q*N, its sinogram
 *    at b + q*M).
 *  - Element type of every image/sinogram buffer passed in or out: double
 *    for WMG_PREC_F64 plans, float for WMG_PREC_F32 plans.
 *  - Memory: every buffer argument is caller-owned DEVICE memory unless the
 *    argument says "host". The library keeps no pointer to caller buffers
 *    after a call returns. Plans own their workspace (device memory taken at
 *    creation and, for larger batches, at the first solve that needs it).
 *  - Streams: work is enqueued on the caller's cudaStream_t (passed as
 *    void*; NULL = the legacy default stream). Calls documented as
 *    "synchronising" wait for the stream before returning.
 *  - Errors: every call returns an int32 status (WMG_OK = 0, WMG_NOT_CONVERGED
 *    = 1, negative = error); no exception crosses the ABI. wmg_last_error()
 *    returns a message for the last failing call of the calling thread.
 *  - Threads: a plan, batch or server is not thread-safe; use one per stream.
 */
#ifndef WMGCT_H
#define WMGCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define WMG_OK                 0
#define WMG_NOT_CONVERGED      1   /* iteration cap reached; x is still valid */
#define WMG_ERR_INVALID_ARG   -1
#define WMG_ERR_OOM           -2
#define WMG_ERR_CUDA          -3
#define WMG_ERR_LEAF_NOT_SPD  -4   /* a leaf matrix failed its Cholesky pivot test */
#define WMG_ERR_BREAKDOWN     -5   /* Krylov breakdown: zero curvature / Hessenberg */
#define WMG_ERR_TIMEOUT       -6   /* a kernel's bounded wait for staged data ran out
                                      (TMA projector); the results computed since are
                                      invalid, the CUDA context stays usable. Reported
                                      when the next wmg_solve (any plan of the process)
                                      completes */
#define WMG_ERR_NAN           -7   /* non-finite value in a reduction */
#define WMG_ERR_REJECTED      -8   /* server: request larger than the memory budget */

/* ---- enumerations --------------------------------------------------------- */
#define WMG_PREC_F64   0   /* operator, vectors and reductions in FP64 */
#define WMG_PREC_F32   1   /* operator (W, W^T, Haar, leaf solves) in FP32,
                              Krylov vectors, scalars and reductions in FP64 */
#define WMG_PREC_F32_BF16STORE 2  /* as WMG_PREC_F32, and inside the Arnoldi
                              steps of preconditioned GMRES the operator's
                              stored inputs -- the preconditioned image and
                              the sinogram W applies to it, with the band
                              images of the hybrid update -- are bfloat16,
                              widened to FP32 for the arithmetic (FP32
                              accumulation). Each restart recomputes the true
                              residual with the FP32 operator (residual
                              replacement), which wins back the accuracy the
                              rounded inputs cost. Other solvers, unpreconditioned
                              GMRES and the operator calls run as WMG_PREC_F32.
                              Buffers passed in and out are FP32. Plans only
                              (not batches or the server). */

#define WMG_CYCLE_ADDITIVE   0  /* all leaf corrections from one residual */
#define WMG_CYCLE_HYBRID     1  /* Section 3.1.2: residual recomputed after the
                                   LL band at every node above hybrid_depth.
                                   A residual update whose correction lies in
                                   the LL band of the first split projects it
                                   on the 2h grid (Section 2.3: pixels of 2 x 2
                                   blocks): with exact intersection lengths
                                   the same product up to rounding, at half
                                   the cost; Joseph's kernel and levels < 3
                                   keep the full grid (all cycles) */
#define WMG_CYCLE_SYMMETRIC  2  /* hybrid followed by a second LL correction
                                   (LL, rest, LL): symmetric, for CGLS */
#define WMG_CYCLE_MULTIPLICATIVE 3  /* Section 3.1.2, eq. wmg: the fully
                                   multiplicative WTG at every node above
                                   hybrid_depth: LL, LH, HL, HH corrected in
                                   turn, each from the residual the corrections
                                   before it leave (three band-local residual
                                   updates per node); not symmetric: for GMRES
                                   and BiCGStab */

#define WMG_KERNEL_STRIP   0  /* w_ij = length of line i inside pixel j (exact) */
#define WMG_KERNEL_JOSEPH  1  /* Joseph's kernel (Section 2.1): the line sampled
                                 at every row (column) centre of the dominant
                                 axis, linear interpolation between the two
                                 nearest pixel centres, weight = step length */

#define WMG_SOLVER_SIRT   0   /* eq. sirt_it */
#define WMG_SOLVER_CGLS   1   /* CGLS / PCG on the normal equations */
#define WMG_SOLVER_GMRES  2   /* restarted GMRES, right preconditioning */
#define WMG_SOLVER_BICGSTAB 3 /* BiCGStab, right preconditioning: the solver of
                                 the paper's experiments (Section 4) */

/* ---- workspace allocator ---------------------------------------------------
 * By default plans, batches and servers take their device workspace with
 * cudaMalloc (a server's geometry setups with stream-ordered
 * cudaMallocAsync on their own stream). wmg_set_allocator sends every later
 * workspace allocation of the process to the caller's functions instead,
 * e.g. a framework's caching allocator, so that the library's memory is
 * counted and reused there:
 *   alloc(bytes, stream, ctx) returns device memory of at least `bytes`
 *     bytes on the current device, aligned to 256 bytes, or NULL (the call
 *     that needed it fails with WMG_ERR_OOM);
 *   free(ptr, bytes, stream, ctx) takes it back.
 * stream: the stream the memory is allocated for; NULL when that is the
 * stream of the library call in progress (which the allocator is not told:
 * a binding that passes its framework's current stream to every call can
 * take that one), a server's setup stream otherwise. Each buffer goes back to the functions that allocated
 * it, so the allocator may change while plans exist; ctx must stay valid
 * until all of its buffers are freed. Plans free their buffers in
 * wmg_plan_destroy (and batches, servers and stored matrices in their
 * destroy calls) or when a pool grows. Both functions may be called from a
 * server's setup thread. Short-lived setup temporaries (the leaf Galerkin
 * assembly's chunk buffers, one counter) still use cudaMallocAsync.
 * alloc = NULL restores cudaMalloc. */
typedef void *(*wmg_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*wmg_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int32_t wmg_set_allocator(wmg_alloc_fn alloc, wmg_free_fn free, void *ctx);

/* ---- parameter blocks ----------------------------------------------------- */
typedef struct wmg_geom {
    int32_t n;              /* image side in pixels, >= 1 */
    int32_t m;              /* number of projection angles, >= 1 */
    const double *angles;   /* HOST array of m angles in radians, or NULL for
                               theta_a = a*pi/m (equiangular over [0, pi)) */
    int32_t D;              /* detector bins per angle, >= 1 */
    double det_spacing;     /* bin spacing in pixel widths; <= 0 means 1 */
    double det_offset;      /* detector centre offset in pixel widths */
    int32_t kernel;         /* WMG_KERNEL_STRIP (0) or WMG_KERNEL_JOSEPH (1) */
} wmg_geom;

typedef struct wmg_opts {
    int32_t levels;         /* WMG levels l >= 1; L = l-1 Haar levels, n must be
                               divisible by 2^L; leaves are (n/2^L)^2 unknowns
                               (at most 256) and there are 4^L of them.
                               0 = no preconditioner: operator, Haar (identity)
                               and unpreconditioned solver calls only */
    int32_t nu1, nu2;       /* l1-Jacobi pre/post smoothing sweeps (>= 0) */
    double omega;           /* smoother damping; <= 0 means 1 */
    double lambda;          /* Tikhonov parameter >= 0 (eq. sys_reg) */
    int32_t hybrid_depth;   /* nodes at depth < hybrid_depth use the hybrid
                               residual update (HYBRID/SYMMETRIC cycles) */
    int32_t cycle;          /* WMG_CYCLE_* */
    int32_t precision;      /* WMG_PREC_* */
} wmg_opts;

/* Per-problem outcome of a solve (host memory, one entry per problem). */
typedef struct wmg_solve_info {
    int32_t iters;          /* iterations done (A-pairs of the outer solver) */
    int32_t status;         /* WMG_OK, WMG_NOT_CONVERGED or a negative error */
    double rel_res;         /* last relative NE residual ||W^T(b-Wx)-lambda x|| / ||W^T b||
                               as tracked by the solver's recurrence (GMRES, BiCGStab: the
                               residual of their own system); 0 with status WMG_OK and x = 0
                               when the initial residual is exactly 0 (e.g. b = 0) */
} wmg_solve_info;

typedef struct wmg_plan wmg_plan;

/* Returns the message of the calling thread's last failing call (empty if
 * none); copies at most len-1 characters into buf and NUL-terminates. */
int32_t wmg_last_error(char *buf, size_t len);

/* Library version as major*10000 + minor*100 + patch. */
int32_t wmg_version(void);

/* Plan creation: validates g and o, builds the angle table (equiangular
 * angles are reduced to the first octant so that multiples of pi/2 and
 * pi/4 are exact), allocates the plan's device workspace, and runs the setup
 * on `stream`: the l1-Jacobi diagonal D~ = W^T(W 1) + lambda, the SIRT
 * scalings R = 1/(W 1), C = 1/(W^T 1) (0 where a sum is 0), and the leaf
 * Galerkin matrices D_k = Q_k^T (W^T W + lambda I) Q_k (Section 3.1.3: the
 * coarsest-level subproblems), factorised by Cholesky and inverted in FP64.
 * Synchronising (the leaf pivots are checked on the host).
 * Errors: INVALID_ARG (bad sizes, n not divisible by 2^L, leaf larger than
 * 256 unknowns), OOM, CUDA, LEAF_NOT_SPD (a leaf matrix is singular: use
 * lambda > 0 or fewer levels). On error *out is NULL. */
int32_t wmg_plan_create(const wmg_geom *g, const wmg_opts *o, void *stream, wmg_plan **out);

/* Releases the plan and its device memory (after synchronising its stream).
 * NULL is ignored. */
int32_t wmg_plan_destroy(wmg_plan *plan);

/* Sizes of the plan's problem: *N = n*n, *M = m*D (either pointer may be NULL). */
int32_t wmg_plan_sizes(const wmg_plan *plan, int64_t *N, int64_t *M);

/* Forward projection b = W x (Section 2.1, eq. sys), matrix-free: the
 * intersection lengths are recomputed per ray. x: count images, b: count
 * sinograms (outputs overwritten). Asynchronous. */
int32_t wmg_project(wmg_plan *plan, int32_t count, const void *x, void *b, void *stream);

/* Backprojection x = W^T b (the transpose of wmg_project, same weights).
 * Asynchronous. */
int32_t wmg_backproject(wmg_plan *plan, int32_t count, const void *b, void *x, void *stream);

/* Preconditioner z = B s: one WMG cycle (Section 3.1) of the plan's options
 * applied to the normal-equation residual s (count images). Asynchronous. */
int32_t wmg_precond_apply(wmg_plan *plan, int32_t count, const void *s, void *z, void *stream);

/* Haar wavelet-packet analysis to depth L (eq. 1of4-4of4 applied
 * recursively): c (count x N) in leaf layout, leaf k = sum_d id_d 4^(L-d)
 * (id_1 = first split, LL=0, LH=1, HL=2, HH=3) holding an (n/2^L)^2
 * row-major grid. wmg_haar_synthesis is its transpose (= inverse).
 * Asynchronous. */
int32_t wmg_haar_analysis(wmg_plan *plan, int32_t count, const void *x, void *c, void *stream);
int32_t wmg_haar_synthesis(wmg_plan *plan, int32_t count, const void *c, void *x, void *stream);

/* Copies leaf k's inverse Galerkin matrix D_k^-1 ((n/2^L)^2 squared, plan
 * precision, row-major) into the device buffer out. Asynchronous. */
int32_t wmg_leaf_inverse(wmg_plan *plan, int64_t k, void *out, void *stream);

/* Solve `count` problems of the plan's geometry: b (count sinograms) ->
 * x (count images). x0 = 0 (x is output only; wmg_solve_x0 takes an
 * initial guess). solver = WMG_SOLVER_*;
 * preconditioned = 1 uses one WMG cycle per iteration (two for BiCGStab;
 * CGLS needs the SYMMETRIC or ADDITIVE cycle; GMRES and BiCGStab any; SIRT
 * ignores it). A BiCGStab iteration counts as one (two A-pairs); its
 * breakdowns (rho, <rh, v> or omega zero before convergence) end the problem
 * with WMG_ERR_BREAKDOWN and the last iterate in x. Stops a problem
 * when its relative NE residual drops below rtol or after max_iter
 * iterations; restart is the GMRES cycle length (<= 64). info: HOST array
 * of count entries, or NULL. res_hist: optional HOST array of
 * count*(max_iter+1) doubles receiving each problem's residual history
 * (entry 0 = 1), or NULL. Synchronising: convergence is checked on the host
 * every few iterations. Returns WMG_OK if every problem converged,
 * WMG_NOT_CONVERGED if any hit max_iter, or the first negative status. */
int32_t wmg_solve(wmg_plan *plan, int32_t solver, int32_t preconditioned, int32_t count,
                  const void *b, void *x, int32_t max_iter, double rtol, int32_t restart,
                  wmg_solve_info *info, double *res_hist, void *stream);

/* As wmg_solve, from the initial guess x0 (count images, device, plan
 * precision; NULL means x0 = 0, which is wmg_solve; x0 may be x itself).
 * Each solver starts from the NE residual of x0, r0 = W^T (b - W x0) -
 * lambda x0 (Section 2.1, eq. sys_reg): CGLS with r = b - W x0 and s = r0,
 * GMRES and BiCGStab with r0 (BiCGStab's shadow residual is r0), SIRT
 * iterates eq. sirt_it from x0. rel_res, rtol and res_hist are relative to
 * |r0| (to |W^T b| when x0 = 0); a Krylov solve with r0 = 0 ends at once
 * with WMG_OK and x = x0. Synchronising. */
int32_t wmg_solve_x0(wmg_plan *plan, int32_t solver, int32_t preconditioned, int32_t count,
                     const void *b, const void *x0, void *x, int32_t max_iter, double rtol, int32_t restart,
                     wmg_solve_info *info, double *res_hist, void *stream);

/* ---- checkpoint / resume ----------------------------------------------------
 * A plan (wmg_plan_create) keeps the state of its last wmg_solve or
 * wmg_solve_x0 that ran to its end: returned WMG_OK or WMG_NOT_CONVERGED, or
 * the status of a problem that stopped on its own (WMG_ERR_BREAKDOWN,
 * WMG_ERR_NAN; such a problem keeps its result when resumed): the FP64 iterate,
 * the solver's other vectors (CGLS: r, p, s; GMRES at its last restart:
 * W^T b, the true residual, rotation data; BiCGStab: r, the shadow
 * residual, p, v; operator-precision copies included) and per-problem
 * scalars, iteration counts, status and residual histories.
 * wmg_solve_resume continues that solve; wmg_state_export copies the state
 * to a host buffer and wmg_state_import copies it back, into the same plan
 * or into another plan made with the same geometry and options (as in a
 * restarted process). Any wmg_project, wmg_precond_apply or solve call on
 * the plan, or a call with another problem count, discards the state.
 * Batches and the server keep none. The contents of the buffer are native
 * binary (same machine architecture and library version). */

/* Bytes wmg_state_export writes. WMG_ERR_INVALID_ARG if the plan holds no
 * state. */
int32_t wmg_state_bytes(wmg_plan *plan, int64_t *bytes);

/* Copies the state into host (HOST, at least wmg_state_bytes bytes).
 * Synchronising. */
int32_t wmg_state_export(wmg_plan *plan, void *host, int64_t bytes, void *stream);

/* Makes host (HOST, bytes long; written by wmg_state_export) the plan's
 * state. WMG_ERR_INVALID_ARG when it is not a state, or the state of a
 * plan with another geometry, options, precision or problem sizes; the
 * plan then holds no state. Synchronising. */
int32_t wmg_state_import(wmg_plan *plan, const void *host, int64_t bytes, void *stream);

/* Continues the plan's state to max_iter iterations IN TOTAL (the state's
 * iterations included; max_iter below them is WMG_ERR_INVALID_ARG), with
 * the same solver, preconditioning, restart length and problem count, and
 * a new rtol. count: the state's problem count (checked: b and x are read
 * and written for that many problems). b: the same right-hand side (count
 * sinograms, device). x receives the iterates (count images). Problems that stopped at the old
 * iteration cap run on; converged or failed ones keep their result (SIRT
 * runs every problem to max_iter, as its fixed count). info, res_hist and
 * the return value as wmg_solve over all max_iter iterations. The kernels'
 * summation orders are fixed, so the results are bitwise those of one
 * uninterrupted solve with this max_iter; for GMRES when the checkpoint is
 * at a restart of that solve (its iteration count a multiple of restart),
 * else the continuation restarts at the checkpoint. Synchronising. */
int32_t wmg_solve_resume(wmg_plan *plan, int32_t count, const void *b, void *x, int32_t max_iter, double rtol,
                         wmg_solve_info *info, double *res_hist, void *stream);

/* ---- batches of problems of different geometries ------------------------- */
/* A batch solves `count` independent reconstructions, each with its own
 * geometry (image side, angles, bins) and WMG levels, together: every
 * operator application is one launch over all of them (the problems are
 * independent: no data moves between them). Identical geometries are set up
 * once and share their leaf inverses.
 * wmg_batch_create: gs, os are HOST arrays of count entries; all problems
 * must share precision, nu1, nu2, omega, cycle and hybrid depth (levels and
 * lambda may differ). Runs every distinct geometry's setup (as
 * wmg_plan_create). Synchronising. */
typedef struct wmg_batch wmg_batch;
int32_t wmg_batch_create(const wmg_geom *gs, const wmg_opts *os, int32_t count, void *stream, wmg_batch **out);
int32_t wmg_batch_destroy(wmg_batch *batch);

/* N = n*n and M = m*D of problem i. */
int32_t wmg_batch_sizes(const wmg_batch *batch, int32_t i, int64_t *N, int64_t *M);

/* Solve every problem of the batch: b[i] (device sinogram of problem i),
 * x[i] (device image of problem i) are HOST arrays of device pointers; the
 * element type is the batch precision's. Other arguments as wmg_solve; info
 * and res_hist are in the caller's problem order. A problem alone and the
 * same problem inside a batch give bitwise identical results (fixed
 * per-problem summation orders). Synchronising. */
int32_t wmg_batch_solve(wmg_batch *batch, int32_t solver, int32_t preconditioned, const void *const *b,
                        void *const *x, int32_t max_iter, double rtol, int32_t restart,
                        wmg_solve_info *info, double *res_hist, void *stream);

/* ---- continuous-batching server -------------------------------------------
 * A request loop for reconstructions that arrive over time. Each request is
 * an independent problem of its own geometry (image side, angle set,
 * detector grid) solved by restarted GMRES(restart) on the normal equations
 * (Section 2.3) with right preconditioning by one WMG cycle (Section 3.1), as
 * wmg_solve with WMG_SOLVER_GMRES does.
 *
 * Requests wait in a FIFO queue; the head is admitted when a slot is free and
 * its footprint fits the free memory. An admitted request keeps all of its
 * solver state (x, W^T b, the Arnoldi basis, Hessenberg and Givens data,
 * residual history) resident in the server's device pools until it ends.
 * Every wmg_server_step admits what fits, then runs one GMRES step for all
 * admitted requests together, each at its own position in its own cycle: one
 * preconditioner application and one A-pair launched over all of them, then
 * the per-request Gram-Schmidt / restart steps. Requests that converged (or
 * hit max_iter, or broke down) retire at the end of the step: x is written
 * to the caller's buffer and their memory and slot go to waiting requests.
 * A request's arithmetic does not depend on the other requests: its x is
 * bitwise the same alone, in any mix, and as from wmg_solve on that problem.
 *
 * Memory. hbm_budget bytes in total: state_bytes (0: half) are taken at
 * creation as the state pools, sized for sino_ratio (0: 4) sinogram elements
 * per image element; the rest holds geometry setups (trig tables, D~^-1,
 * SIRT scalings, leaf inverses K * P^2 values of the plan precision), cached by geometry and
 * evicted least-recently-used when no admitted or queued request uses them.
 * Footprint of a request: (restart + 11) * 8 + 2 s bytes per pixel and 2 s
 * bytes per ray (s = 8 for F64, 4 for F32), more with hybrid depth h >= 1
 * (band images, 3^(h-1) (2 s + 8) per pixel and 3^(h-1) s per ray) and the
 * symmetric cycle (24 h per pixel); plus, when its geometry is not cached,
 * the geometry's setup and, while that setup runs, its scratch
 * (wmg_server_footprint gives all three).
 *
 * Geometry setups run on three worker threads, each with a stream of its
 * own, so that they overlap one another and the steps of the requests
 * already admitted; a request waits in the queue until its geometry is ready
 * (requests behind it whose geometries are ready may pass it); at most four
 * setups are started or queued at a time.
 *
 * Streams: all request work is on the stream given at creation;
 * wmg_server_step synchronises it. Not thread-safe. */
#define WMG_REQ_QUEUED   0
#define WMG_REQ_RUNNING  1
#define WMG_REQ_DONE     2

typedef struct wmg_server_config {
    int64_t hbm_budget;      /* bytes: state pools + geometry setups */
    int64_t state_bytes;     /* bytes of hbm_budget for the state pools (0: half) */
    double sino_ratio;       /* sinogram elements per image element in the pools (0: 4) */
    int32_t max_slots;       /* requests in flight at most */
    int32_t preconditioned;  /* 1: WMG-GMRES (levels >= 1 per request), 0: GMRES */
    int32_t max_iter;        /* iteration cap per request */
    double rtol;             /* stop when |W^T b - (W^T W + lambda) x| / |W^T b| < rtol */
    int32_t restart;         /* GMRES restart length, 1..64 */
    wmg_opts opts;           /* precision, cycle, nu1, nu2, omega and hybrid_depth shared by
                                every request; levels and lambda are the defaults of
                                requests submitted with opts = NULL */
} wmg_server_config;

typedef struct wmg_server_counters {
    int64_t submitted, admitted, completed, rejected, ticks;
    int64_t geometry_setups, geometries_evicted;
    int32_t running, queued, geometries_cached;
    int64_t state_bytes_capacity, state_bytes_used;
    int64_t geometry_bytes_capacity, geometry_bytes_used;
} wmg_server_counters;

typedef struct wmg_server wmg_server;

/* Create a server: takes the state pools (device) and pinned host staging.
 * WMG_ERR_INVALID_ARG for an invalid configuration or a state budget below
 * one 64-pixel image, WMG_ERR_OOM when the pools do not fit. Synchronising. */
int32_t wmg_server_create(const wmg_server_config *cfg, void *stream, wmg_server **out);
/* Destroy a server (waits for its stream); outstanding requests are dropped. */
int32_t wmg_server_destroy(wmg_server *srv);

/* Queue a request: geometry g (angles, if given, are copied), options o
 * (NULL: the server's; precision, cycle, nu1, nu2, omega and hybrid_depth
 * must equal the server's), sinogram b (device, m*D elements of the server
 * precision's type) and the output image x (device, n*n elements). b and x
 * must stay valid and unchanged (x unread) until wmg_server_poll reports
 * WMG_REQ_DONE. Does not block and launches nothing. Returns
 * WMG_ERR_REJECTED (no ticket) when the footprint can never fit the budget,
 * WMG_ERR_INVALID_ARG for an invalid geometry or options. */
int32_t wmg_server_submit(wmg_server *srv, const wmg_geom *g, const wmg_opts *o, const void *b, void *x,
                          uint64_t *ticket);

/* One tick: install finished geometry setups, admit, run one GMRES step for
 * every admitted request, retire the finished ones. *pending (may be NULL) =
 * requests running + queued after the tick. When nothing is admitted and
 * setups run, waits about 0.2 ms. Synchronising. */
int32_t wmg_server_step(wmg_server *srv, int32_t *pending);

/* State of a request (WMG_REQ_QUEUED / RUNNING / DONE). When DONE: *info
 * (iterations, status, final relative residual), *latency_ms (host time from
 * submit to retirement) and res_hist (max_iter + 1 doubles, as wmg_solve's)
 * are filled where not NULL, x holds the result, and the ticket is released
 * (polling it again is WMG_ERR_INVALID_ARG). Host-only, never blocks. */
int32_t wmg_server_poll(wmg_server *srv, uint64_t ticket, int32_t *state, wmg_solve_info *info,
                        double *latency_ms, double *res_hist);

/* Counters and memory use. Host-only. */
int32_t wmg_server_stats(const wmg_server *srv, wmg_server_counters *out);

/* The footprint the server charges a request of geometry g, options o (NULL:
 * the server's): *state = bytes of its state in the pools, *geometry = its
 * geometry's setup kept while cached, *setup = bytes the setup holds only
 * while it runs (any pointer may be NULL). Host-only. */
int32_t wmg_server_footprint(const wmg_server *srv, const wmg_geom *g, const wmg_opts *o, int64_t *state,
                             int64_t *geometry, int64_t *setup);

/* ---- stored-matrix comparator -------------------------------------------
 * W (transposed = 0: M rows, one per ray) or W^T (transposed = 1: N rows, one
 * per pixel) of a single-geometry plan assembled on the device as CSR: int64
 * row pointers, int32 column indices, values = the exact intersection lengths
 * (evaluated in FP64 by the same trapezoid law as the matrix-free kernels,
 * stored as double for F64 plans and float for F32 plans). Not part of the
 * method: a reference for what storing W instead of recomputing it costs.
 * Device memory 12 or 16 bytes per nonzero; synchronising. */
typedef struct wmg_csr wmg_csr;
int32_t wmg_csr_create(wmg_plan *plan, int32_t transposed, void *stream, wmg_csr **out);
int32_t wmg_csr_destroy(wmg_csr *csr);
int32_t wmg_csr_info(const wmg_csr *csr, int64_t *rows, int64_t *cols, int64_t *nnz);
/* y_v = A x_v for v < count (x_v at x + v * cols, y_v at y + v * rows, device
 * memory of the plan precision's type); one launch, asynchronous on stream. */
int32_t wmg_csr_apply(const wmg_csr *csr, int32_t count, const void *x, void *y, void *stream);

/* Number of nonzero intersection lengths of the plan's W (rays x pixels with
 * a nonzero weight), counted on the device at the first call (on the legacy
 * default stream, synchronising) and cached. */
int32_t wmg_plan_nnz(const wmg_plan *plan, int64_t *nnz);

/* Launch shapes of the plan's projector and backprojector: CTAs per SM of
 * their grid-stride launches (grid = min(tiles, SMs x value)). The library
 * times 1, 2, 4, 8 and 16 (F32 plans) whenever a plan's problem table changes
 * (wmg_plan_create, a new count in a call, wmg_batch_create) and keeps the
 * fastest; WMG_AUTOTUNE=0 in the environment keeps 8. Every shape gives
 * bitwise the same results (each tile's arithmetic does not depend on the
 * CTA that runs it). set: values in [1, 64]; kept until the table changes. */
int32_t wmg_plan_get_tuning(const wmg_plan *plan, int32_t *project_ctas, int32_t *backproject_ctas);
int32_t wmg_plan_set_tuning(wmg_plan *plan, int32_t project_ctas, int32_t backproject_ctas);

/* Library-wide count of kernel launches since the last reset (all plans of
 * the process); reset != 0 zeroes the counter after reading it. */
int64_t wmg_launch_count(int32_t reset);

/* Per-kernel timing of the projector and backprojector launches of one plan:
 * between wmg_profile_begin and wmg_profile_end every such launch is
 * bracketed by CUDA events recorded on its stream (adds a few microseconds
 * per launch; for measurement runs only). wmg_profile_end synchronises the
 * stream and fills *out. Projections on the 2h grid (the hybrid cycle's band
 * updates whose input lies in the first split's LL band: n/2 x n/2 images,
 * about half the nonzeros of W) are counted apart from those of W. */
typedef struct wmg_profile_stats {
    int32_t project_launches;
    double project_ms;            /* summed device time */
    double project_images;        /* summed images processed */
    int32_t backproject_launches;
    double backproject_ms;
    double backproject_images;
    double nnz_per_image;         /* nonzeros of W */
    int32_t project_2h_launches;  /* projections on the 2h grid */
    double project_2h_ms;
    double project_2h_images;
} wmg_profile_stats;
int32_t wmg_profile_begin(wmg_plan *plan);
int32_t wmg_profile_end(wmg_plan *plan, wmg_profile_stats *out, void *stream);

/* Measured arithmetic peak of the current GPU, for the roofline of the
 * library's ALU-bound kernels (the matrix-free projector and backprojector
 * recompute their weights and are bound by FP32 arithmetic and issue, not by
 * memory). The paper has no counterpart: this is measurement support.
 * kind: WMG_PEAK_FP32_FMA (one FP32 multiply-add per instruction),
 * WMG_PEAK_FP32_FMA2 (the paired FP32 multiply-add, two per instruction) or
 * WMG_PEAK_FP64_FMA. *tflops receives 2 x multiply-adds per second / 1e12,
 * the best of five timed launches of independent multiply-add chains (8
 * CTAs of 256 threads per SM, no memory traffic). Synchronising on
 * `stream`; allocates 16 bytes of device memory for the duration of the call.
 * WMG_ERR_INVALID_ARG for an unknown kind or a NULL result pointer. */
enum { WMG_PEAK_FP32_FMA = 0, WMG_PEAK_FP32_FMA2 = 1, WMG_PEAK_FP64_FMA = 2 };
int32_t wmg_measure_peak(int32_t kind, double *tflops, void *stream);

/* Forward projection b = W x that allocates no device memory, for callers
 * that cannot call cudaMalloc once they are running: an acquisition loop that
 * reserves all its device memory at start-up so that nothing can fail or
 * stall mid-scan, or a program whose framework allocator already holds all
 * free device memory. The paper has no counterpart: this is an interface
 * variant of wmg_project, not part of the method.
 * Geometry: n x n image, m equiangular angles over [0, pi), D bins of one
 * pixel width, centred, W = exact intersection lengths (WMG_KERNEL_STRIP);
 * FP32 image x (n*n) and sinogram b (m*D), device memory, one image per call.
 * Results equal wmg_project's for that geometry bit for bit (the same
 * angle tables and the same projector kernel).
 * Limits: n <= 1024, m <= 4096, D <= 2048; larger sizes return
 * WMG_ERR_INVALID_ARG. The scratch (transposed image, work lists, angle
 * tables: 8,830,976 bytes, about 8.4 MiB) lives in fixed __device__ arrays
 * that every GPU on which the library's device code is loaded keeps until
 * the process exits. With lazy module loading (the CUDA default) that
 * memory is taken by the first call on each device, when the call looks up
 * the arrays' device addresses: make that first call at start-up, before
 * the caller's allocator takes the free memory, and before any stream
 * capture. Later calls take no device memory. The host side is locked, so
 * calls from several host threads and on several devices are safe to issue;
 * every call on one device shares the same arrays, so calls whose work
 * overlaps on that GPU (other streams, other host threads) race: serialise
 * them. Asynchronous on `stream`. */
int32_t wmg_project_noalloc(int32_t n, int32_t m, int32_t D, const float *x, float *b, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* WMGCT_H */
