// engine.cuh -- host-side structures of the engine (device buffers, work
// lists, geometries, the plan) and the engine steps shared by the plan and
// batch drivers in engine.cu and the request server in server.cu.
#pragma once

#include <algorithm>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "kern_common.cuh"
#include "krylov.cuh"

namespace wmg {

int num_sms();

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
// Stream for the allocations of this host thread's non-persistent buffers
// (set by threads that build geometries concurrently with running solves):
// when set, DevBuf allocates and frees stream-ordered on it, so that freeing
// a temporary does not synchronise the device.
extern thread_local cudaStream_t g_alloc_stream;

// The caller's workspace allocator (wmg_set_allocator), or none (cudaMalloc).
struct Allocator {
    wmg_alloc_fn alloc = nullptr;
    wmg_free_fn free = nullptr;
    void *ctx = nullptr;
};
Allocator current_allocator();

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    bool persistent = false;       // outlives the thread's allocation stream
    cudaStream_t ast = nullptr;    // stream of a stream-ordered allocation
    Allocator owner;               // the caller's allocator that made p, if any
    void *owner_stream = nullptr;
    DevBuf() = default;
    explicit DevBuf(bool persist) : persistent(persist) {}
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) {
            if (owner.free) owner.free(p, bytes, owner_stream, owner.ctx);
            else if (ast) cudaFreeAsync(p, ast);
            else cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
        ast = nullptr;
        owner = Allocator{};
        owner_stream = nullptr;
    }
    // grow-only; contents are not preserved
    bool ensure(size_t b)
    {
        if (b <= bytes && p) return true;
        release();
        if (b == 0) b = 16;
        const Allocator a = current_allocator();
        if (a.alloc) {
            // the caller's allocator: returned to the same functions; the
            // kernels and tensor maps want 256-byte aligned bases
            void *st = !persistent && g_alloc_stream ? static_cast<void *>(g_alloc_stream) : nullptr;
            void *q = a.alloc(b, st, a.ctx);
            if (!q) return false;
            if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
                a.free(q, b, st, a.ctx);
                return false;
            }
            p = q;
            bytes = b;
            owner = a;
            owner_stream = st;
            return true;
        }
        cudaError_t e;
        if (!persistent && g_alloc_stream) {
            e = cudaMallocAsync(&p, b, g_alloc_stream);
            if (e == cudaSuccess) ast = g_alloc_stream;
        } else {
            e = cudaMalloc(&p, b);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        bytes = b;
        return true;
    }
    template <class U> U *as() const { return static_cast<U *>(p); }
};

// ---------------------------------------------------------------------------
// work lists and geometries
// ---------------------------------------------------------------------------
struct TileList {
    DevBuf tiles, tb, te;
    int n = 0;
    std::vector<int4> h;
    bool upload(int nprob, cudaStream_t st)
    {
        n = (int)h.size();
        std::vector<int> b(nprob, 0), e(nprob, 0);
        for (int i = 0; i < n; ++i) {
            const int p = h[i].x;
            if (i == 0 || h[i - 1].x != p) b[p] = i;
            e[p] = i + 1;
        }
        if (!tiles.ensure(std::max<size_t>(1, h.size()) * sizeof(int4)) ||
            !tb.ensure(nprob * sizeof(int)) || !te.ensure(nprob * sizeof(int)))
            return false;
        if (n) cudaMemcpyAsync(tiles.p, h.data(), h.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(tb.p, b.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(te.p, e.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, st);
        // host vectors must outlive the async copies: keep them (b, e are
        // copied synchronously with respect to pageable memory)
        return true;
    }
};

// A set of (real or virtual) problems with their tiles (problems may have
// different geometries; each tile belongs to one problem).
struct ProbSet {
    int nprob = 0;
    std::vector<ProbDev> h;
    DevBuf d;
    TileList proj, bp, haar, vimg, vsino;
    // FP32 projector tiles ({first problem, angle, first ray, images}): full
    // groups of kProjGroup consecutive same-geometry problems, and one-image
    // tiles for the problems left over
    TileList projg, proj1;
    // FP32 backprojector tiles: group tiles ({first problem, iy0, ix0,
    // kBpGroup}) of the projector's groups whose geometry has unit bins
    // covering every tile and quarter-turn pairs, and one-image tiles of the
    // other problems
    TileList bpg, bp1;
    // the group tiles read their pixels through TMA boxes (projector_tma.cu)
    // when every problem has image side tma_n (> 0; a multiple of 4) and bins
    // no wider than a pixel, its image is image number img / n^2 of a pool of
    // tma_count images, and each group's images are consecutive there
    int tma_n = 0;
    int64_t tma_count = 0;
    // brk[q] != 0: a run of same-geometry problems (for the projector's
    // groups) starts at q even if q - 1 has the same geometry (empty: none)
    std::vector<char> brk;
    int haar_smem = 0;
    // launch shapes of the projector / backprojector over this set's tiles
    // (CTAs per SM; 0 = 8), chosen by autotune(); they do not change results
    int pj_ctas = 0, bp_ctas = 0;
    // on_2h: the set's tiles and launches use its geometries' 2h grids
    // (Geo::gc, the plan's d_geom_2h table) and its images are n/2 x n/2
    bool on_2h = false;
    // Band sets, split by entry (an entry's path never depends on the other
    // entries): grid2h = the entries whose input lies in the first split's LL
    // band, on the 2h grid, for their synthesis and projection; bp2h = the
    // same entries on W's grid, for their backprojection (null: all entries);
    // rest = the other entries (null: none)
    std::unique_ptr<ProbSet> grid2h, bp2h, rest;
};

// One geometry of a plan with its device tables.
struct Geo {
    GeomDev g{};
    int64_t N = 0, M = 0, nnz = -1;     // nnz: counted on first request
    bool has_wmg = true, unit_bins = true;
    int hd = 0;                 // hybrid depth in use: min(hybrid_depth, L), 0 for additive
    int haar_W = 1;             // Haar strip width (pixels)
    // The same scan on the 2h grid of 2 x 2 pixel blocks (Section 2.3),
    // exact-length kernel and L >= 2 only: side n/2, L - 1 levels, the same
    // leaves (nc, P), detector offset and spacing in 2h pixel widths, and h
    // kept at the fine pixel width, so that projecting an n/2 x n/2 image c
    // gives W^{2h} c / 2 = W I_{2h}^h c (eq. intops; chords add over the
    // four pixels of a block). Tables shared with g; no smoother or leaf data.
    bool has_2h = false;
    GeomDev gc{};
    int64_t Nc = 0;             // (n/2)^2
    int haar_Wc = 1;            // Haar strip width of the 2h grid
    DevBuf cs64{true}, cs32{true}, csx{true}, angf{true}, dinv{true}, leafinv{true}, sirtR{true}, sirtC{true};
};

// CUDA graphs for the solver iterations unless WMG_GRAPHS=0 in the environment.
bool graphs_default();

// What the last solve on a single-geometry plan left in the plan's pools:
// enough to continue it (wmg_solve_resume) or to copy it out and back
// (wmg_state_export / wmg_state_import). Any call that reuses those pools
// (a solve, a projection, a preconditioner application, a change of the
// problem count) clears `valid`.
struct SolveState {
    bool valid = false;
    int solver = 0, pre = 0, restart = 0, count = 0;
    int steps = 0;        // iterations the solve's loop ran (the same for every problem)
    int hist_ld = 1;      // row length of the residual histories in the hist pool
};

}  // namespace wmg

// ---------------------------------------------------------------------------
// The plan: one or more geometries and a table of problem slots. A plan made
// by wmg_plan_create has one geometry and any number of same-geometry
// problems per call; a batch (wmg_batch_create) has a fixed list of problems
// of several geometries, stored grouped by geometry.
// ---------------------------------------------------------------------------
struct wmg_plan {
    int prec = WMG_PREC_F64;      // arithmetic of the operator: F64 or F32 (also for BF16 storage)
    bool bf16 = false;            // WMG_PREC_F32_BF16STORE: bfloat16 operator inputs in the Arnoldi steps
    bool bf16_now = false;        // the operator calls being issued use bfloat16 storage
    size_t esz = 8;
    wmg_opts opts{};
    std::vector<std::unique_ptr<wmg::Geo>> geos;
    wmg::DevBuf d_geom;         // GeomDev array, one per geometry
    wmg::DevBuf d_geom_2h;      // their 2h grids (Geo::gc; zeros where there is none)
    bool unit_bins = true;      // every geometry has unit bins, zero offset
    bool batch = false;         // fixed problem list
    int cap = 0;                // problem slots
    std::vector<int> pgeo;      // geometry of each slot
    std::vector<int64_t> img_off, sino_off;
    int64_t Ntot = 0, Mtot = 0;
    std::vector<int> order;     // batch: slot of the caller's problem i
    std::vector<int> live;      // slots that hold a problem, ascending (all slots but in a server)
    wmg::ProbSet real;
    std::map<std::vector<int>, std::unique_ptr<wmg::ProbSet>> bands;   // band-update groups
    std::map<std::vector<int>, std::unique_ptr<wmg::TileList>> leafsets;
    std::map<std::vector<int>, std::unique_ptr<wmg::DevBuf>> segsets;
    // FP64 pools (all slots back to back)
    wmg::DevBuf x, s, z, p, f, w, t, u, r;
    // operator-precision pools
    wmg::DevBuf p_op, pT_op, z_op, zT_op, r1, C, E, q, r_op, sinoS, b_op, x_io;
    std::vector<std::unique_ptr<wmg::DevBuf>> csave, c2, e2;   // per hybrid depth
    wmg::DevBuf band_img, band_imgT, band_img2, band_sino;
    // scalars and partials
    wmg::DevBuf S, part_a, part_b, part_c, lam, hist;
    // GMRES
    wmg::DevBuf V, H, gcs, gsn, gg, gy, h1, h2, jn, done, reo;
    // BiCGStab (t and the preconditioned s)
    wmg::DevBuf bi_t, bi_sh;
    // profiling: (kind 0 = project / 1 = backproject, images, start, stop)
    // CUDA graphs of the solver iterations are captured on this private
    // stream (capture cannot use the legacy default stream) and launched on
    // the caller's stream. use_graphs: WMG_GRAPHS=0 in the environment at
    // plan creation keeps every launch eager.
    cudaStream_t cap_stream = nullptr;
    bool use_graphs = wmg::graphs_default();
    int tuned_pj = 8, tuned_bp = 8;     // last autotune result (CTAs per SM)
    wmg::SolveState state;              // continuation point of the last solve
    uint64_t fingerprint = 0;           // geometry and options (single-geometry plans)
    ~wmg_plan()
    {
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
    bool profiling = false;
    struct ProfRec { int kind; int images; cudaEvent_t e0, e1; };
    std::vector<ProfRec> prof;
    const wmg::Geo &geo(int slot) const { return *geos[pgeo[slot]]; }
    bool has_wmg() const
    {
        for (auto &g : geos)
            if (g && !g->has_wmg) return false;
        return true;
    }
};

namespace wmg {

// One captured sequence of launches (a solver iteration), replayed with
// cudaGraphLaunch; `launches` = kernels per replay (for the launch counter).
struct Graph {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    Graph() = default;
    Graph(const Graph &) = delete;
    Graph &operator=(const Graph &) = delete;
    ~Graph() { reset(); }
    void reset()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        launches = 0;
    }
};

// ---- engine steps (engine.cu) ----------------------------------------------
// Time the projector and backprojector over ps's tiles at 1, 2, 4, 8 and 16
// CTAs per SM and keep the fastest (F32 plans; skipped when WMG_AUTOTUNE=0 in
// the environment or when the set has fewer tiles than SMs).
template <class T>
int32_t autotune(wmg_plan *pl, ProbSet &ps, cudaStream_t st);
void build_tiles(const wmg_plan *pl, ProbSet &ps);
bool upload_set(ProbSet &ps, cudaStream_t st);
bool ensure_pool(DevBuf &b, int64_t elems, size_t esz);
bool ensure_partials(wmg_plan *pl, size_t per_tile_max);
template <class T>
void project(wmg_plan *pl, const ProbSet &ps, const void *img, const void *imgT, void *sino, double *part,
             const double *S, cudaStream_t st);
template <class T>
void backproject(wmg_plan *pl, const ProbSet &ps, BpArgs a, cudaStream_t st);
BpArgs bp_args(int epi, const void *sino, const double *S);
template <class T>
void img_op(wmg_plan *pl, int op, ImgArgs a, cudaStream_t st);
template <class T>
void vec_op(wmg_plan *pl, int op, bool sino, VecArgs a, cudaStream_t st);
void finalize(wmg_plan *pl, int op, const TileList &ta, const double *pa, int nsum, const TileList *tb,
              const double *pb, int precond, double *hist, int hist_ld, cudaStream_t st, int store_slot = 0,
              double *store_vec = nullptr, int store_ld = 0, int part_ld = 1);
template <class T>
int32_t wmg_apply(wmg_plan *pl, double *s, double *z, bool first_done, bool copies, bool sz_part,
                  bool *have_sz, cudaStream_t st);
int32_t ensure_wmg_pools(wmg_plan *pl);
int32_t validate(const wmg_geom *g, const wmg_opts *o);
int32_t make_geo(const wmg_geom *g, const wmg_opts *o, Geo &G, cudaStream_t st);
int32_t upload_geoms(wmg_plan *pl, cudaStream_t st);
template <class T>
int32_t setup_geometry(wmg_plan *pl, int gi, cudaStream_t st);

}  // namespace wmg
