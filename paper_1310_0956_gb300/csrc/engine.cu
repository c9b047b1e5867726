// engine.cu -- host engine behind the C ABI of include/wmgct.h: plan
// creation and setup, work lists, the WMG cycle schedules and the Krylov
// drivers. Every arithmetic step runs in the kernels of projector.cu,
// haar.cu, setup.cu and krylov.cu; this file only orders launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "active_groups.h"
#include "band_grid.h"
#include "engine.cuh"

namespace wmg {

// ---------------------------------------------------------------------------
// errors, device properties
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }
int32_t fail(int32_t code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

thread_local cudaStream_t g_alloc_stream = nullptr;

static std::mutex g_allocator_mu;
static Allocator g_allocator;

Allocator current_allocator()
{
    std::lock_guard<std::mutex> lk(g_allocator_mu);
    return g_allocator;
}

bool graphs_default()
{
    static const bool on = [] {
        const char *v = std::getenv("WMG_GRAPHS");
        return !(v && v[0] == '0');
    }();
    return on;
}

// TMA-staged group tiles of the FP32 projector unless WMG_PROJ_TMA=0 in the
// environment (both kernels give the same bits).
static bool proj_tma_default()
{
    static const bool on = [] {
        const char *v = std::getenv("WMG_PROJ_TMA");
        return !(v && v[0] == '0');
    }();
    return on;
}

static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void ensure_dyn_smem(const void *fn, int bytes)
{
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int d = 0;
    cudaGetDevice(&d);
    std::lock_guard<std::mutex> lk(mu);
    if (done.insert({d, fn}).second) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int num_sms()
{
    static int v = [] {
        int d = 0, n = 0;
        cudaGetDevice(&d);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
        return n > 0 ? n : 148;
    }();
    return v;
}

// Angle tables of a geometry, into caller-provided arrays of m entries.
// Equiangular angles (angles == NULL): theta_a = pi*a/m reduced to the first
// octant so that multiples of pi/2 are exactly 0 / +-1, odd multiples of pi/4
// give cos = sin = sqrt(1/2), and theta + pi/2 gets exactly (-sin, cos).
// cs32 is the round-to-nearest FP32 copy; csx the split (12-significant-bit
// head, a multiple of 2^-12, and FP32 tail); angf the FP32 kernels' table.
void geometry_tables(int m, const double *angles, int kernel, double2 *cs, float2 *cs32, float4 *csx,
                     AngleF *angf)
{
    for (int a = 0; a < m; ++a) {
        double c, s;
        if (angles) {
            c = std::cos(angles[a]);
            s = std::sin(angles[a]);
        } else {
            const long twice = 2L * a, quad = twice / m, rem = twice - quad * m;
            if (rem == 0) { c = 1.0; s = 0.0; }
            else if (2 * rem == m) { c = std::sqrt(0.5); s = c; }
            else if (2 * rem < m) {
                const double phi = (M_PI / 2.0) * ((double)rem / (double)m);
                c = std::cos(phi); s = std::sin(phi);
            } else {
                const double phi = (M_PI / 2.0) * ((double)(m - rem) / (double)m);
                c = std::sin(phi); s = std::cos(phi);
            }
            if (quad & 1) { const double t = c; c = -s; s = t; }
        }
        cs[a] = make_double2(c, s);
        cs32[a] = make_float2((float)c, (float)s);
        const double ch = std::nearbyint(c * 4096.0) / 4096.0;
        const double sh = std::nearbyint(s * 4096.0) / 4096.0;
        csx[a] = make_float4((float)ch, (float)(c - ch), (float)sh, (float)(s - sh));
    }
    fill_angle_table(cs, m, kernel, angf);
}

// FP32 scalars and the backprojector's path flags of a geometry whose n, m,
// D, h, dt and t0 are set, from its FP32 angle table (host copy).
void geometry_scalars(GeomDev &gd, const AngleF *angf)
{
    // quarter-turn pairs: angle a + m/2 is angle a turned by pi/2 in the
    // FP32 table, (c, s) -> (-s, c) with the same chord constants
    gd.qpair = gd.m % 2 == 0 && gd.m >= 2;
    for (int a = 0; gd.qpair && a < gd.m / 2; ++a) {
        const AngleF &u = angf[a], &v = angf[a + gd.m / 2];
        gd.qpair = v.chi == -u.shi && v.clo == -u.slo && v.shi == u.chi && v.slo == u.clo && v.wa == u.wa &&
                   v.wb == u.wb && v.lmax == u.lmax;
    }
    gd.hf = (float)gd.h;
    gd.dtf = (float)gd.dt;
    gd.t0f = (float)gd.t0;
    gd.hDf = 0.5f * (float)(gd.D - 1);
    gd.unit = gd.dt == 1.0 && gd.t0 == 0.0 ? 1 : 0;
    if (gd.unit) {
        // Pixel centres of the 32 x 32 backprojection tiles (the last tile
        // row and column may reach past the image) lie within rmax of the
        // centre, so |tau| <= rmax at every angle. The unit-bin path takes
        // bins k0 = rint(tau + hD - 1/2) and k0 + 1 (up to FP32 rounding of
        // tau, far below the 0.01 margin): both lie in [0, D) when
        // rmax < hD.
        const double half = 0.5 * gd.n;
        const double xmax = std::max(half - 0.5, 32.0 * ((gd.n + 31) / 32) - half - 0.5);
        const double rmax = std::sqrt(2.0) * xmax;
        if (rmax + 0.01 < 0.5 * (gd.D - 1)) gd.unit = 2;
    }
}

// ---- tile lists ------------------------------------------------------------
// Haar strip width of a geometry: a whole number of 2^L blocks that divides
// the image side, at most max(B, 4096 / B) pixels wide.
static int haar_width(const GeomDev &g)
{
    const int nb = g.n / g.B, wmax = std::max(1, std::max(g.B, 4096 / g.B) / g.B);
    int wb = 1;
    for (int d = 1; d <= std::min(nb, wmax); ++d)
        if (nb % d == 0) wb = d;
    return wb * g.B;
}

// The geometry a set's tiles and launches use for geometry gi: its own, or
// its 2h grid (sets on the 2h grid).
static const GeomDev &set_geom(const wmg_plan *pl, const ProbSet &ps, int gi)
{
    const Geo &G = *pl->geos[gi];
    return ps.on_2h ? G.gc : G.g;
}

void build_tiles(const wmg_plan *pl, ProbSet &ps)
{
    ps.proj.h.clear(); ps.bp.h.clear(); ps.haar.h.clear(); ps.vimg.h.clear(); ps.vsino.h.clear();
    ps.projg.h.clear(); ps.proj1.h.clear(); ps.bpg.h.clear(); ps.bp1.h.clear();
    std::vector<char> in_bpg(ps.nprob, 0);
    ps.haar_smem = 0;
    // FP32 projector tiles: runs of consecutive problems of one geometry cut
    // into full groups of kProjGroup images (one tile per group, angle and
    // ray block); the problems left over get one-image tiles
    for (int q = 0; q < ps.nprob;) {
        if (ps.h[q].geom < 0) { ++q; continue; }
        int e = q + 1;
        while (e < ps.nprob && ps.h[e].geom == ps.h[q].geom && !(e < (int)ps.brk.size() && ps.brk[e])) ++e;
        const GeomDev &g = set_geom(pl, ps, ps.h[q].geom);
        int f = q;
        const bool bpg = pl->prec != WMG_PREC_F64 && g.unit == 2 && g.qpair;
        for (; f + kProjGroup <= e; f += kProjGroup) {
            for (int a = 0; a < g.m; ++a)
                for (int k0 = 0; k0 < g.D; k0 += 32) ps.projg.h.push_back(make_int4(f, a, k0, kProjGroup));
            if (!bpg) continue;
            for (int iy = 0; iy < g.n; iy += 32)
                for (int ix = 0; ix < g.n; ix += 32)
                    for (int b = 0; b < kProjGroup; b += kBpGroup) ps.bpg.h.push_back(make_int4(f + b, iy, ix, kBpGroup));
            for (int b = 0; b < kProjGroup; ++b) in_bpg[f + b] = 1;
        }
        for (; f < e; ++f)
            for (int a = 0; a < g.m; ++a)
                for (int k0 = 0; k0 < g.D; k0 += 32) ps.proj1.h.push_back(make_int4(f, a, k0, 1));
        q = e;
    }
    ps.tma_n = 0;
    ps.tma_count = 0;
    if (pl->prec == WMG_PREC_F32 && !ps.projg.h.empty() && proj_tma_default()) {
        int n0 = -1;
        bool ok = true;
        int64_t count = 0;
        for (int q = 0; q < ps.nprob && ok; ++q) {
            if (ps.h[q].geom < 0) continue;
            const GeomDev &g = set_geom(pl, ps, ps.h[q].geom);
            if (n0 < 0) n0 = g.n;
            const int64_t N = (int64_t)g.n * g.n;
            ok = g.n == n0 && g.n % 4 == 0 && g.dt <= 1.0 && ps.h[q].img % N == 0;
            count = std::max<int64_t>(count, ps.h[q].img / N + 1);
        }
        for (size_t i = 0; i < ps.projg.h.size() && ok; ++i) {
            const int f = ps.projg.h[i].x;
            if (i > 0 && ps.projg.h[i - 1].x == f) continue;
            for (int b = 1; b < kProjGroup && ok; ++b)
                ok = ps.h[f + b].img == ps.h[f].img + (int64_t)b * n0 * n0;
        }
        if (ok && n0 > 0) {
            ps.tma_n = n0;
            ps.tma_count = count;
        }
    }
    for (int q = 0; q < ps.nprob; ++q) {
        if (ps.h[q].geom < 0) continue;          // an empty server slot: no tiles
        const Geo &G = *pl->geos[ps.h[q].geom];
        const GeomDev &g = set_geom(pl, ps, ps.h[q].geom);
        const int W = ps.on_2h ? G.haar_Wc : G.haar_W;
        const int64_t Nq = ps.on_2h ? G.Nc : G.N;
        ps.haar_smem = std::max(ps.haar_smem, g.B * (W + W / g.B + 1));
        for (int a = 0; a < g.m; ++a)
            for (int k0 = 0; k0 < g.D; k0 += 32) ps.proj.h.push_back(make_int4(q, a, k0, 0));
        for (int iy = 0; iy < g.n; iy += 32)
            for (int ix = 0; ix < g.n; ix += 32) {
                ps.bp.h.push_back(make_int4(q, iy, ix, 0));
                if (!in_bpg[q]) ps.bp1.h.push_back(make_int4(q, iy, ix, 0));
            }
        for (int cy = 0; cy < g.nc; ++cy)
            for (int x0 = 0; x0 < g.n; x0 += W) ps.haar.h.push_back(make_int4(q, cy * g.B, x0, W));
        for (int64_t s0 = 0; s0 < Nq; s0 += 8192)
            ps.vimg.h.push_back(make_int4(q, (int)s0, (int)std::min<int64_t>(8192, Nq - s0), 0));
        for (int64_t s0 = 0; s0 < G.M; s0 += 8192)
            ps.vsino.h.push_back(make_int4(q, (int)s0, (int)std::min<int64_t>(8192, G.M - s0), 0));
    }
}

bool upload_set(ProbSet &ps, cudaStream_t st)
{
    if (!ps.d.ensure(std::max<size_t>(1, ps.h.size()) * sizeof(ProbDev))) return false;
    cudaMemcpyAsync(ps.d.p, ps.h.data(), ps.h.size() * sizeof(ProbDev), cudaMemcpyHostToDevice, st);
    return ps.proj.upload(ps.nprob, st) && ps.bp.upload(ps.nprob, st) && ps.haar.upload(ps.nprob, st) &&
           ps.projg.upload(ps.nprob, st) && ps.proj1.upload(ps.nprob, st) &&
           ps.bpg.upload(ps.nprob, st) && ps.bp1.upload(ps.nprob, st) &&
           ps.vimg.upload(ps.nprob, st) && ps.vsino.upload(ps.nprob, st);
}

// (Re)build the slot tables from pgeo (offsets in slot order).
static int32_t set_slots(wmg_plan *pl, cudaStream_t st)
{
    const int count = (int)pl->pgeo.size();
    pl->img_off.assign(count, 0);
    pl->sino_off.assign(count, 0);
    int64_t ni = 0, ns = 0;
    for (int q = 0; q < count; ++q) {
        pl->img_off[q] = ni;
        pl->sino_off[q] = ns;
        ni += pl->geo(q).N;
        ns += pl->geo(q).M;
    }
    pl->Ntot = ni;
    pl->Mtot = ns;
    ProbSet &ps = pl->real;
    ps.nprob = count;
    ps.h.assign(count, ProbDev{});
    for (int q = 0; q < count; ++q) {
        ProbDev &d = ps.h[q];
        d.geom = pl->pgeo[q]; d.slot = q;
        d.img = pl->img_off[q]; d.sino = pl->sino_off[q]; d.coef = pl->img_off[q];
        d.kin0 = 0; d.kin1 = pl->geo(q).g.K; d.kout0 = 0; d.kout1 = pl->geo(q).g.K;
    }
    pl->state.valid = false;
    build_tiles(pl, ps);
    if (!upload_set(ps, st)) return fail(WMG_ERR_OOM, "work-list allocation failed");
    pl->bands.clear();
    pl->leafsets.clear();
    pl->segsets.clear();
    pl->cap = count;
    pl->live.resize(count);
    for (int q = 0; q < count; ++q) pl->live[q] = q;
    if (!pl->S.ensure((size_t)count * NSCAL * sizeof(double)) ||
        !pl->lam.ensure((size_t)count * sizeof(double)))
        return fail(WMG_ERR_OOM, "scalar allocation failed");
    std::vector<double> lam(count);
    for (int q = 0; q < count; ++q) lam[q] = pl->geo(q).g.lambda;
    cudaMemcpyAsync(pl->lam.p, lam.data(), count * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
    return WMG_OK;
}

// Single-geometry plans: `count` problems of geometry 0 back to back.
static int32_t ensure_count(wmg_plan *pl, int count, cudaStream_t st)
{
    if (pl->batch) {
        if (count != pl->cap) return fail(WMG_ERR_INVALID_ARG, "a batch has a fixed problem count");
        return WMG_OK;
    }
    if (count == pl->cap) return WMG_OK;
    pl->pgeo.assign(count, 0);
    int32_t rc = set_slots(pl, st);
    if (rc) return rc;
    return pl->prec == WMG_PREC_F64 ? autotune<double>(pl, pl->real, st) : autotune<float>(pl, pl->real, st);
}

bool ensure_pool(DevBuf &b, int64_t elems, size_t esz) { return b.ensure((size_t)elems * esz); }

bool ensure_partials(wmg_plan *pl, size_t per_tile_max)
{
    const ProbSet &ps = pl->real;
    size_t n = std::max({(size_t)ps.proj.h.size(), (size_t)ps.bp.h.size(), (size_t)ps.vimg.h.size(),
                         (size_t)ps.vsino.h.size(), (size_t)1});
    return pl->part_a.ensure(n * per_tile_max * sizeof(double)) &&
           pl->part_b.ensure(n * sizeof(double)) && pl->part_c.ensure(n * sizeof(double));
}

// ---------------------------------------------------------------------------
// Operator steps
// ---------------------------------------------------------------------------
static void prof_begin(wmg_plan *pl, int kind, int images, cudaStream_t st)
{
    wmg_plan::ProfRec r{kind, images, nullptr, nullptr};
    cudaEventCreate(&r.e0);
    cudaEventCreate(&r.e1);
    cudaEventRecord(r.e0, st);
    pl->prof.push_back(r);
}
static void prof_end(wmg_plan *pl, cudaStream_t st) { cudaEventRecord(pl->prof.back().e1, st); }

template <class T>
void project(wmg_plan *pl, const ProbSet &ps, const void *img, const void *imgT, void *sino,
                    double *part, const double *S, cudaStream_t st)
{
    PjArgs a{ps.pj_ctas, img, imgT, sino, part, S, ps.proj.tb.as<int>(), 1};
    a.bf16 = pl->bf16_now ? 1 : 0;
    const GeomDev *G = (ps.on_2h ? pl->d_geom_2h : pl->d_geom).as<GeomDev>();
    if (pl->profiling) prof_begin(pl, ps.on_2h ? 2 : 0, ps.nprob, st);
    if (sizeof(T) == 4) {
        // FP32: groups of kProjGroup images share the weights; the rest run
        // one image per tile (the same per-image arithmetic in both). The
        // staged-pixel kernel reads FP32 pools only.
        a.group = kProjGroup;
        if (!(ps.tma_n > 0 && !a.bf16 && launch_project_f32_tma(G, ps.d.as<ProbDev>(), ps.projg.tiles.as<int4>(),
                                                                ps.projg.n, a, ps.tma_n, ps.tma_count, st)))
            launch_project<T>(G, ps.d.as<ProbDev>(), ps.projg.tiles.as<int4>(), ps.projg.n, a, st);
        a.group = 1;
        launch_project<T>(G, ps.d.as<ProbDev>(), ps.proj1.tiles.as<int4>(), ps.proj1.n, a, st);
    } else {
        launch_project<T>(G, ps.d.as<ProbDev>(), ps.proj.tiles.as<int4>(), ps.proj.n, a, st);
    }
    if (pl->profiling) prof_end(pl, st);
}

template <class T>
void backproject(wmg_plan *pl, const ProbSet &ps, BpArgs a, cudaStream_t st)
{
    a.unit = pl->unit_bins ? 1 : 0;
    a.bf16 = pl->bf16_now ? 1 : 0;
    a.ctas_per_sm = ps.bp_ctas;
    a.part_base = ps.bp.tb.as<int>();
    if (pl->profiling) prof_begin(pl, 1, ps.nprob, st);
    // FP32 storage: the group tiles (shared bins and weights, staged
    // sinograms) and the other problems' one-image tiles; the same bits
    if (sizeof(T) == 4 && ps.bpg.n > 0 &&
        launch_backproject_f32_group(pl->d_geom.as<GeomDev>(), ps.d.as<ProbDev>(), ps.bpg.tiles.as<int4>(),
                                     ps.bpg.n, a, st))
        launch_backproject<T>(pl->d_geom.as<GeomDev>(), ps.d.as<ProbDev>(), ps.bp1.tiles.as<int4>(), ps.bp1.n, a,
                              st);
    else
        launch_backproject<T>(pl->d_geom.as<GeomDev>(), ps.d.as<ProbDev>(), ps.bp.tiles.as<int4>(), ps.bp.n, a, st);
    if (pl->profiling) prof_end(pl, st);
}

static bool autotune_enabled()
{
    static const bool on = [] {
        const char *v = std::getenv("WMG_AUTOTUNE");
        return !(v && v[0] == '0');
    }();
    return on;
}

template <class T>
int32_t autotune(wmg_plan *pl, ProbSet &ps, cudaStream_t st)
{
    ps.pj_ctas = ps.bp_ctas = 0;
    // FP32 plans only: the FP64 operators are the parity path, and timing
    // them would cost more than it can save
    if (!autotune_enabled() || sizeof(T) != 4 || ps.proj.n < num_sms() || pl->profiling) return WMG_OK;
    int64_t VN = 0, VM = 0;
    for (const ProbDev &pd : ps.h) {
        if (pd.geom < 0) continue;
        VN = std::max<int64_t>(VN, pd.img + pl->geos[pd.geom]->N);
        VM = std::max<int64_t>(VM, pd.sino + pl->geos[pd.geom]->M);
    }
    DevBuf img, imgT, sino;
    if (!img.ensure(VN * sizeof(T)) || !imgT.ensure(VN * sizeof(T)) || !sino.ensure(VM * sizeof(T)))
        return WMG_OK;                                   // no room to tune: keep the default shapes
    cudaMemsetAsync(img.p, 0, VN * sizeof(T), st);
    cudaMemsetAsync(imgT.p, 0, VN * sizeof(T), st);
    cudaMemsetAsync(sino.p, 0, VM * sizeof(T), st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int opts[] = {1, 2, 4, 8, 16};
    float best_p = 1e30f, best_b = 1e30f;
    for (int c : opts) {
        ps.pj_ctas = ps.bp_ctas = c;
        for (int kind = 0; kind < 2; ++kind) {
            float total = 0.f;
            for (int rep = 0; rep < 4; ++rep) {
                cudaEventRecord(e0, st);
                if (kind == 0) {
                    project<T>(pl, ps, img.p, imgT.p, sino.p, nullptr, nullptr, st);
                } else {
                    BpArgs a = bp_args(BP_STORE, sino.p, nullptr);
                    a.out_op = img.p;
                    backproject<T>(pl, ps, a, st);
                }
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) total += ms;                // the first launch is a warm-up
            }
            if (kind == 0 && total < best_p) { best_p = total; pl->tuned_pj = c; }
            if (kind == 1 && total < best_b) { best_b = total; pl->tuned_bp = c; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ps.pj_ctas = pl->tuned_pj;
    ps.bp_ctas = pl->tuned_bp;
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

BpArgs bp_args(int epi, const void *sino, const double *S)
{
    BpArgs a{};
    a.unit = 0;
    a.epi = epi;
    a.sino = sino;
    a.S = S;
    return a;
}

template <class T>
void img_op(wmg_plan *pl, int op, ImgArgs a, cudaStream_t st)
{
    const ProbSet &ps = pl->real;
    a.bf16 = pl->bf16_now ? 1 : 0;
    launch_img<T>(op, pl->d_geom.as<GeomDev>(), ps.d.as<ProbDev>(), ps.bp.tiles.as<int4>(), ps.bp.n, a, st);
}

template <class T>
void vec_op(wmg_plan *pl, int op, bool sino, VecArgs a, cudaStream_t st)
{
    const ProbSet &ps = pl->real;
    const TileList &tl = sino ? ps.vsino : ps.vimg;
    a.G = pl->d_geom.as<GeomDev>();
    launch_vec<T>(op, ps.d.as<ProbDev>(), tl.tiles.as<int4>(), tl.n, a, st);
}

void finalize(wmg_plan *pl, int op, const TileList &ta, const double *pa, int nsum, const TileList *tb,
              const double *pb, int precond, double *hist, int hist_ld, cudaStream_t st, int store_slot,
              double *store_vec, int store_ld, int part_ld)
{
    FinArgs f{};
    f.op = op;
    f.nprob = pl->cap;
    f.precond = precond;
    f.part_a = pa;
    f.tb_a = ta.tb.as<int>();
    f.te_a = ta.te.as<int>();
    f.ld_a = std::max(part_ld, std::max(1, nsum));
    f.nsum_a = std::max(1, nsum);
    f.part_b = pb;
    f.tb_b = tb ? tb->tb.as<int>() : nullptr;
    f.te_b = tb ? tb->te.as<int>() : nullptr;
    f.S = pl->S.as<double>();
    f.lambda = pl->lam.as<double>();
    f.hist = hist;
    f.hist_ld = hist_ld;
    f.store_slot = store_slot;
    f.store_vec = store_vec;
    f.store_ld = store_ld;
    launch_finalize(f, st);
}

// ---------------------------------------------------------------------------
// WMG coarse correction (Section 3.1.2 recursion) on the packet coefficients.
// Tree nodes, their leaf ranges and the band updates' ranges: band_grid.h.
// ---------------------------------------------------------------------------

static std::vector<int> make_key(int tag, int d, const std::vector<int> &nodes, const std::vector<int> &slots)
{
    std::vector<int> key{tag, d, (int)nodes.size()};
    key.insert(key.end(), nodes.begin(), nodes.end());
    key.insert(key.end(), slots.begin(), slots.end());
    return key;
}

// Band-update group tables: one virtual image per (slot, node); it reads the
// slot's correction coefficients and writes the slot's residual coefficients.
// Band-local products of a group of nodes. mode 0: the LL child in, the
// three other children out (the hybrid step, and the multiplicative cycle's
// first); 1: the whole node in, its LL child out (the symmetric closing
// step); 2, 3: child 1 (LH) or 2 (HL) in, the children after it out (the
// multiplicative cycle's later steps).
static ProbSet *band_set(wmg_plan *pl, int d, const std::vector<int> &nodes, const std::vector<int> &slots,
                         int mode, cudaStream_t st)
{
    const std::vector<int> key = make_key(mode, d, nodes, slots);
    auto it = pl->bands.find(key);
    if (it != pl->bands.end()) return it->second.get();
    auto ps = std::make_unique<ProbSet>();
    ps->nprob = (int)(slots.size() * nodes.size());
    ps->h.resize(ps->nprob);
    int64_t oi = 0, os = 0;
    int v = 0;
    for (int slot : slots)
        for (int q : nodes) {
            const Geo &G = pl->geo(slot);
            const int L = G.g.L;
            ProbDev &pd = ps->h[v++];
            pd.geom = pl->pgeo[slot]; pd.slot = slot;
            pd.img = oi; pd.sino = os; pd.coef = pl->img_off[slot];
            oi += G.N; os += G.M;
            band_leaf_ranges(L, d, q, mode, pd.kin0, pd.kin1, pd.kout0, pd.kout1);
        }
    build_tiles(pl, *ps);
    if (!upload_set(*ps, st)) return nullptr;
    ps->pj_ctas = pl->real.pj_ctas;
    ps->bp_ctas = pl->real.bp_ctas;
    // Entries whose input lies inside the first split's LL band (leaves
    // below K/4) of a geometry with a 2h grid, and whose outputs lie on other
    // leaves: their synthesis and projection run on the 2h grid, on n/2 x n/2
    // images (the same leaf values, one level fewer), and their lambda term,
    // Q_out^T Q_in = 0, drops. Decided per entry, so that a problem takes the
    // same path alone and in any batch.
    std::vector<char> e2h(ps->nprob, 0);
    int n2h = 0;
    for (int q = 0; q < ps->nprob; ++q) {
        const ProbDev &pd = ps->h[q];
        const Geo &G = *pl->geos[pd.geom];
        e2h[q] = band_on_2h(G.has_2h, G.g.K, pd.kin0, pd.kin1, pd.kout0, pd.kout1);
        n2h += e2h[q];
    }
    auto subset = [&](bool want, bool grid) -> std::unique_ptr<ProbSet> {
        auto cs = std::make_unique<ProbSet>();
        cs->on_2h = grid;
        int64_t oc = 0;
        for (int q = 0; q < ps->nprob; ++q) {
            if ((e2h[q] != 0) != want) continue;
            ProbDev pd = ps->h[q];
            if (grid) {                      // n/2 x n/2 images, back to back
                pd.img = oc;
                oc += pl->geos[pd.geom]->Nc;
            }
            cs->h.push_back(pd);
        }
        cs->nprob = (int)cs->h.size();
        build_tiles(pl, *cs);
        if (!upload_set(*cs, st)) return nullptr;
        cs->pj_ctas = pl->real.pj_ctas;
        cs->bp_ctas = pl->real.bp_ctas;
        return cs;
    };
    if (n2h > 0) {
        if (!(ps->grid2h = subset(true, true))) return nullptr;
        if (n2h < ps->nprob && (!(ps->bp2h = subset(true, false)) || !(ps->rest = subset(false, false))))
            return nullptr;
    }
    ProbSet *raw = ps.get();
    pl->bands[key] = std::move(ps);
    return raw;
}

// Leaf-solve tiles: {first slot of a run of same-geometry slots, leaf, run
// length, 0}. FP32 plans (tensor-core leaf solves): one work item per leaf,
// chunk of at most kLeafTcProblems slots of a run and block of kLeafTcRows
// rows of the inverse, {first slot, leaf, chunk length, row block}.
static TileList *leaf_tiles(wmg_plan *pl, int d, const std::vector<int> &nodes, const std::vector<int> &slots,
                            cudaStream_t st)
{
    const std::vector<int> key = make_key(2, d, nodes, slots);
    auto it = pl->leafsets.find(key);
    if (it != pl->leafsets.end()) return it->second.get();
    auto tl = std::make_unique<TileList>();
    const bool tc = pl->prec != WMG_PREC_F64;
    size_t i = 0;
    while (i < slots.size()) {
        size_t j = i + 1;
        while (j < slots.size() && slots[j] == slots[j - 1] + 1 && pl->pgeo[slots[j]] == pl->pgeo[slots[i]]) ++j;
        const GeomDev &g = pl->geo(slots[i]).g;
        const int run = (int)(j - i);
        for (int q : nodes)
            for (int k = node_lo(g.L, d, q); k < node_hi(g.L, d, q); ++k) {
                if (!tc) {
                    tl->h.push_back(make_int4(slots[i], k, run, 0));
                    continue;
                }
                for (int c0 = 0; c0 < run; c0 += kLeafTcProblems)
                    for (int mb = 0; mb * kLeafTcRows < g.P; ++mb)
                        tl->h.push_back(make_int4(slots[i] + c0, k, std::min(kLeafTcProblems, run - c0), mb));
            }
        i = j;
    }
    if (!tl->upload(pl->cap, st)) return nullptr;
    TileList *raw = tl.get();
    pl->leafsets[key] = std::move(tl);
    return raw;
}

// E[seg] += E2[seg] over absolute element segments of the coefficient pool.
__global__ void k_coef_add(double *E, const double *E2, const longlong2 *segs, int nseg)
{
    for (int sgi = 0; sgi < nseg; ++sgi) {
        const longlong2 sg = segs[sgi];
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < sg.y;
             i += (long long)gridDim.x * blockDim.x)
            E[sg.x + i] += E2[sg.x + i];
    }
}

// Haar synthesis whose outputs are operator copies: bfloat16 when the
// operator calls being issued use bfloat16 storage, else the plan's type.
template <class T>
static void syn_op(wmg_plan *pl, const GeomDev *G, const ProbDev *P, const int4 *tiles, int ntiles, int smem,
                   const HaarArgs &a, cudaStream_t st)
{
    if (sizeof(T) == 4 && pl->bf16_now) launch_haar_synthesis<double, __nv_bfloat16>(G, P, tiles, ntiles, smem, a, st);
    else launch_haar_synthesis<double, T>(G, P, tiles, ntiles, smem, a, st);
}

// One band-local residual update for a group of nodes (hybrid cycle): for
// every slot and node, C[out range] -= Q_out^T (W^T W + lambda) Q_in E[in range].
template <class T>
static int32_t band_update(wmg_plan *pl, int d, const std::vector<int> &nodes, const std::vector<int> &slots,
                           int mode, DevBuf &Cb, DevBuf &Eb, cudaStream_t st)
{
    ProbSet *bs = band_set(pl, d, nodes, slots, mode, st);
    if (!bs) return fail(WMG_ERR_OOM, "band tables");
    int64_t VN = 0, VM = 0;
    for (const ProbDev &pd : bs->h) { VN += pl->geos[pd.geom]->N; VM += pl->geos[pd.geom]->M; }
    if (!ensure_pool(pl->band_img, VN, pl->esz) || !ensure_pool(pl->band_imgT, VN, pl->esz) ||
        !ensure_pool(pl->band_img2, VN, 8) || !ensure_pool(pl->band_sino, VM, pl->esz))
        return fail(WMG_ERR_OOM, "band pools");
    const GeomDev *G = pl->d_geom.as<GeomDev>();
    const double *S = pl->S.as<double>();
    HaarArgs hs{};
    hs.mode = HS_STORE_MASKED;
    hs.in = Eb.p;
    hs.out = pl->band_img.p;
    hs.outT = pl->band_imgT.p;
    hs.S = S;
    hs.fp32 = pl->prec == WMG_PREC_F32;
    if (const ProbSet *cs = bs->grid2h.get()) {
        // inputs in the LL band of the first split: Q_in E = I_{2h}^h c with
        // c the n/2 x n/2 synthesis of the same leaves, and W I_{2h}^h c the
        // 2h grid's projection (half the rows); lambda Q_out^T Q_in E = 0 (the
        // leaf ranges are disjoint), so the backprojection is W^T u alone
        syn_op<T>(pl, pl->d_geom_2h.as<GeomDev>(), cs->d.as<ProbDev>(), cs->haar.tiles.as<int4>(), cs->haar.n,
                  cs->haar_smem, hs, st);
        project<T>(pl, *cs, pl->band_img.p, pl->band_imgT.p, pl->band_sino.p, nullptr, S, st);
        BpArgs a = bp_args(BP_ATB, pl->band_sino.p, S);
        a.out64 = pl->band_img2.as<double>();
        backproject<T>(pl, bs->bp2h ? *bs->bp2h : *bs, a, st);
        if (const ProbSet *rs = bs->rest.get()) {
            // the other entries on W's grid (their images overwrite the 2h
            // ones in the pool only after the 2h projection, in stream order)
            syn_op<T>(pl, G, rs->d.as<ProbDev>(), rs->haar.tiles.as<int4>(), rs->haar.n, rs->haar_smem, hs, st);
            project<T>(pl, *rs, pl->band_img.p, pl->band_imgT.p, pl->band_sino.p, nullptr, S, st);
            BpArgs r = bp_args(BP_APPLY_A, pl->band_sino.p, S);
            r.v_op = pl->band_img.p;
            r.out64 = pl->band_img2.as<double>();
            backproject<T>(pl, *rs, r, st);
        }
    } else {
        syn_op<T>(pl, G, bs->d.as<ProbDev>(), bs->haar.tiles.as<int4>(), bs->haar.n, bs->haar_smem, hs, st);
        project<T>(pl, *bs, pl->band_img.p, pl->band_imgT.p, pl->band_sino.p, nullptr, S, st);
        BpArgs a = bp_args(BP_APPLY_A, pl->band_sino.p, S);
        a.v_op = pl->band_img.p;
        a.out64 = pl->band_img2.as<double>();
        backproject<T>(pl, *bs, a, st);
    }
    HaarArgs ha{};
    ha.mode = HA_SUB_MASKED;
    ha.in = pl->band_img2.p;
    ha.out = Cb.p;
    ha.S = S;
    ha.fp32 = pl->prec == WMG_PREC_F32;
    launch_haar_analysis<double, double>(G, bs->d.as<ProbDev>(), bs->haar.tiles.as<int4>(), bs->haar.n,
                                         bs->haar_smem, ha, st);
    return WMG_OK;
}

// Coarse correction for the nodes `nodes` at depth d of the slots `slots`
// (Section 3.1.2, siblings processed together): slots whose hybrid depth is
// reached solve their leaves exactly; the others correct the LL child first,
// update the residual of the other three children once, correct them, and
// (symmetric cycle) correct the LL child again from the residual of the
// whole node correction.
template <class T>
static int32_t coarse(wmg_plan *pl, int d, const std::vector<int> &nodes, const std::vector<int> &slots,
                      DevBuf &Cb, DevBuf &Eb, cudaStream_t st)
{
    std::vector<int> done, deeper;
    for (int s : slots) (d >= pl->geo(s).hd ? done : deeper).push_back(s);
    if (!done.empty()) {
        TileList *lt = leaf_tiles(pl, d, nodes, done, st);
        if (!lt) return fail(WMG_ERR_OOM, "leaf tables");
        launch_leaf_apply(pl->d_geom.as<GeomDev>(), pl->real.d.as<ProbDev>(), lt->tiles.as<int4>(),
                          lt->n, Cb.as<double>(), Eb.as<double>(), 0, pl->S.as<double>(), pl->prec == WMG_PREC_F32,
                          st);
    }
    if (deeper.empty()) return WMG_OK;
    std::vector<int> lls, rests;
    for (int q : nodes) {
        lls.push_back(4 * q);
        for (int c = 1; c < 4; ++c) rests.push_back(4 * q + c);
    }
    if (pl->opts.cycle == WMG_CYCLE_MULTIPLICATIVE) {
        // eq. wmg: LL, LH, HL, HH in turn; before each of the last three, the
        // residual of the children still to come loses A_p times the
        // correction just made
        int32_t rc = coarse<T>(pl, d + 1, lls, deeper, Cb, Eb, st);
        for (int c = 1; c < 4 && !rc; ++c) {
            std::vector<int> kids;
            for (int q : nodes) kids.push_back(4 * q + c);
            if ((rc = band_update<T>(pl, d, nodes, deeper, c == 1 ? 0 : c, Cb, Eb, st))) break;
            rc = coarse<T>(pl, d + 1, kids, deeper, Cb, Eb, st);
        }
        return rc;
    }
    const bool sym = pl->opts.cycle == WMG_CYCLE_SYMMETRIC;
    const size_t cbytes = (size_t)pl->Ntot * sizeof(double);
    if (sym) cudaMemcpyAsync(pl->csave[d]->p, Cb.p, cbytes, cudaMemcpyDeviceToDevice, st);
    int32_t rc = coarse<T>(pl, d + 1, lls, deeper, Cb, Eb, st);
    if (rc) return rc;
    if ((rc = band_update<T>(pl, d, nodes, deeper, 0, Cb, Eb, st))) return rc;
    if ((rc = coarse<T>(pl, d + 1, rests, deeper, Cb, Eb, st))) return rc;
    if (sym) {
        DevBuf &C2 = *pl->c2[d], &E2 = *pl->e2[d];
        cudaMemcpyAsync(C2.p, pl->csave[d]->p, cbytes, cudaMemcpyDeviceToDevice, st);
        if ((rc = band_update<T>(pl, d, nodes, deeper, 1, C2, Eb, st))) return rc;
        if ((rc = coarse<T>(pl, d + 1, lls, deeper, C2, E2, st))) return rc;
        const std::vector<int> key = make_key(3, d, nodes, deeper);
        auto it = pl->segsets.find(key);
        if (it == pl->segsets.end()) {
            std::vector<longlong2> segs;
            for (int s : deeper) {
                const Geo &G = pl->geo(s);
                for (int q : lls) {
                    const long long lo = node_lo(G.g.L, d + 1, q), hi = node_hi(G.g.L, d + 1, q);
                    longlong2 sg;
                    sg.x = pl->img_off[s] + lo * G.g.P;
                    sg.y = (hi - lo) * G.g.P;
                    segs.push_back(sg);
                }
            }
            auto db = std::make_unique<DevBuf>();
            if (!db->ensure(segs.size() * sizeof(longlong2))) return fail(WMG_ERR_OOM, "segments");
            cudaMemcpy(db->p, segs.data(), segs.size() * sizeof(longlong2), cudaMemcpyHostToDevice);
            db->bytes = segs.size() * sizeof(longlong2);
            it = pl->segsets.emplace(key, std::move(db)).first;
        }
        count_launches(1);
        k_coef_add<<<num_sms() * 4, 256, 0, st>>>(Eb.as<double>(), E2.as<double>(),
                                                   it->second->as<longlong2>(),
                                                   (int)(it->second->bytes / sizeof(longlong2)));
    }
    return WMG_OK;
}

static int max_levels(const wmg_plan *pl)
{
    int L = 0;
    for (auto &g : pl->geos)
        if (g) L = std::max(L, g->g.L);
    return L;
}

int32_t ensure_wmg_pools(wmg_plan *pl)
{
    const int64_t nN = pl->Ntot, nM = pl->Mtot;
    const size_t e = pl->esz;
    if (!ensure_pool(pl->z, nN, 8) || !ensure_pool(pl->s, nN, 8) || !ensure_pool(pl->z_op, nN, e) ||
        !ensure_pool(pl->zT_op, nN, e) || !ensure_pool(pl->r1, nN, 8) || !ensure_pool(pl->C, nN, 8) ||
        !ensure_pool(pl->E, nN, 8) || !ensure_pool(pl->sinoS, nM, e))
        return fail(WMG_ERR_OOM, "preconditioner pools");
    const int L = max_levels(pl);
    while ((int)pl->csave.size() < L) {
        pl->csave.push_back(std::make_unique<DevBuf>());
        pl->c2.push_back(std::make_unique<DevBuf>());
        pl->e2.push_back(std::make_unique<DevBuf>());
    }
    if (pl->opts.cycle == WMG_CYCLE_SYMMETRIC)
        for (int d = 0; d < std::min(pl->opts.hybrid_depth, L); ++d)
            if (!ensure_pool(*pl->csave[d], nN, 8) || !ensure_pool(*pl->c2[d], nN, 8) ||
                !ensure_pool(*pl->e2[d], nN, 8))
                return fail(WMG_ERR_OOM, "symmetric-cycle pools");
    return WMG_OK;
}

// z = B s (FP64 pools s, z). If `first_done`, z already holds omega D~^-1 s
// and z_op / zT_op its copies. If `copies`, z_op / zT_op hold z at the end.
// If `sz_part`, the tile partials of s.z over the backprojection tiles are
// left in part_b (returns true in *have_sz).
template <class T>
int32_t wmg_apply(wmg_plan *pl, double *s, double *z, bool first_done, bool copies, bool sz_part,
                         bool *have_sz, cudaStream_t st)
{
    const wmg_opts &o = pl->opts;
    const ProbSet &ps = pl->real;
    const double *S = pl->S.as<double>();
    *have_sz = false;
    if (o.nu1 >= 1) {
        if (!first_done) {
            ImgArgs ia{};
            ia.z = z; ia.s = s; ia.copy_op = pl->z_op.p; ia.copyT_op = pl->zT_op.p; ia.S = S;
            img_op<T>(pl, IMG_FIRST_SWEEP, ia, st);
        }
        for (int it = 1; it < o.nu1; ++it) {
            project<T>(pl, ps, pl->z_op.p, pl->zT_op.p, pl->sinoS.p, nullptr, S, st);
            BpArgs a = bp_args(BP_POST, pl->sinoS.p, S);
            a.s = s; a.z = z; a.copy_op = pl->z_op.p; a.copyT_op = pl->zT_op.p;
            backproject<T>(pl, ps, a, st);
        }
        project<T>(pl, ps, pl->z_op.p, pl->zT_op.p, pl->sinoS.p, nullptr, S, st);
        BpArgs a = bp_args(BP_RESID, pl->sinoS.p, S);
        a.s = s; a.z = z; a.out64 = pl->r1.as<double>();
        backproject<T>(pl, ps, a, st);
    } else {
        ImgArgs ia{};
        ia.z = z; ia.s = s; ia.r1 = pl->r1.p; ia.S = S;
        img_op<T>(pl, IMG_ZERO_RESID, ia, st);
    }
    const GeomDev *G = pl->d_geom.as<GeomDev>();
    HaarArgs ha{};
    ha.mode = HA_STORE; ha.in = pl->r1.p; ha.out = pl->C.p; ha.S = S; ha.fp32 = pl->prec == WMG_PREC_F32;
    launch_haar_analysis<double, double>(G, ps.d.as<ProbDev>(), ps.haar.tiles.as<int4>(), ps.haar.n,
                                         ps.haar_smem, ha, st);
    int32_t rc = coarse<T>(pl, 0, std::vector<int>{0}, pl->live, pl->C, pl->E, st);
    if (rc) return rc;
    const bool need_copies_after_syn = copies || o.nu2 > 0;
    HaarArgs hs{};
    hs.mode = HS_CORRECT; hs.in = pl->E.p; hs.z = z; hs.S = S; hs.fp32 = pl->prec == WMG_PREC_F32;
    hs.out = need_copies_after_syn ? pl->z_op.p : nullptr;
    hs.outT = need_copies_after_syn ? pl->zT_op.p : nullptr;
    syn_op<T>(pl, G, ps.d.as<ProbDev>(), ps.haar.tiles.as<int4>(), ps.haar.n, ps.haar_smem, hs, st);
    for (int it = 0; it < o.nu2; ++it) {
        const bool last = it == o.nu2 - 1;
        project<T>(pl, ps, pl->z_op.p, pl->zT_op.p, pl->sinoS.p, nullptr, S, st);
        BpArgs a = bp_args(BP_POST, pl->sinoS.p, S);
        a.s = s; a.z = z;
        if (!last || copies) { a.copy_op = pl->z_op.p; a.copyT_op = pl->zT_op.p; }
        if (last && sz_part) { a.part = pl->part_b.as<double>(); *have_sz = true; }
        backproject<T>(pl, ps, a, st);
    }
    return WMG_OK;
}

// ---------------------------------------------------------------------------
// geometry creation and setup
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_fill(T *p, int64_t n, T v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void k_to_f32(const double *in, float *out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
// out = 1 / (in + add) where positive, else 0
template <class T>
__global__ void k_recip(const T *in, T *out, int64_t n, double add)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)in[i] + add;
        out[i] = v > 0.0 ? (T)(1.0 / v) : T(0);
    }
}

int32_t validate(const wmg_geom *g, const wmg_opts *o)
{
    if (!g || !o) return fail(WMG_ERR_INVALID_ARG, "geometry or options NULL");
    if (g->n < 1 || g->m < 1 || g->D < 1) return fail(WMG_ERR_INVALID_ARG, "n, m and D must be >= 1");
    if (g->kernel != WMG_KERNEL_STRIP && g->kernel != WMG_KERNEL_JOSEPH)
        return fail(WMG_ERR_INVALID_ARG, "kernel must be WMG_KERNEL_STRIP or WMG_KERNEL_JOSEPH");
    if (o->levels < 0 || o->levels > 12) return fail(WMG_ERR_INVALID_ARG, "levels must be in [0, 12]");
    const int L = o->levels >= 1 ? o->levels - 1 : 0;
    if (g->n % (1 << L) != 0) return fail(WMG_ERR_INVALID_ARG, "n must be divisible by 2^(levels-1)");
    const int nc = g->n >> L;
    if (o->levels >= 1 && nc * nc > 256) return fail(WMG_ERR_INVALID_ARG, "leaf side n/2^(levels-1) must be <= 16");
    if ((1 << L) > 128) return fail(WMG_ERR_INVALID_ARG, "block side 2^(levels-1) must be <= 128");
    if (o->nu1 < 0 || o->nu2 < 0 || o->lambda < 0 || o->hybrid_depth < 0 ||
        o->cycle < WMG_CYCLE_ADDITIVE || o->cycle > WMG_CYCLE_MULTIPLICATIVE ||
        (o->precision != WMG_PREC_F64 && o->precision != WMG_PREC_F32 && o->precision != WMG_PREC_F32_BF16STORE))
        return fail(WMG_ERR_INVALID_ARG, "invalid options");
    if ((int64_t)g->n * g->n > (int64_t)1 << 30 || (int64_t)g->m * g->D > (int64_t)1 << 31)
        return fail(WMG_ERR_INVALID_ARG, "problem too large");
    return WMG_OK;
}

// Host part of a geometry: angle tables and scalar fields.
int32_t make_geo(const wmg_geom *g, const wmg_opts *o, Geo &G, cudaStream_t st)
{
    G.has_wmg = o->levels >= 1;
    const int L = G.has_wmg ? o->levels - 1 : 0;
    const int nc = g->n >> L;
    G.N = (int64_t)g->n * g->n;
    G.M = (int64_t)g->m * g->D;
    GeomDev &gd = G.g;
    gd.n = g->n; gd.m = g->m; gd.D = g->D; gd.L = L;
    gd.nc = nc; gd.P = nc * nc; gd.K = 1 << (2 * L); gd.B = 1 << L;
    gd.h = 1.0 / g->n;
    gd.dt = g->det_spacing > 0 ? g->det_spacing : 1.0;
    gd.t0 = g->det_offset;
    gd.kernel = g->kernel;
    gd.lambda = o->lambda;
    gd.omega = o->omega > 0 ? o->omega : 1.0;
    G.hd = (o->cycle == WMG_CYCLE_ADDITIVE || !G.has_wmg) ? 0 : std::min(o->hybrid_depth, L);
    G.haar_W = haar_width(gd);
    std::vector<double2> cs(g->m);
    std::vector<float2> cs32(g->m);
    std::vector<float4> csx(g->m);
    std::vector<AngleF> angf(g->m);
    geometry_tables(g->m, g->angles, gd.kernel, cs.data(), cs32.data(), csx.data(), angf.data());
    if (!G.cs64.ensure(g->m * sizeof(double2)) || !G.cs32.ensure(g->m * sizeof(float2)) ||
        !G.csx.ensure(g->m * sizeof(float4)) || !G.angf.ensure(g->m * sizeof(AngleF)))
        return fail(WMG_ERR_OOM, "plan allocation failed");
    WMG_CUDA(cudaMemcpyAsync(G.angf.p, angf.data(), g->m * sizeof(AngleF), cudaMemcpyHostToDevice, st));
    WMG_CUDA(cudaMemcpyAsync(G.csx.p, csx.data(), g->m * sizeof(float4), cudaMemcpyHostToDevice, st));
    WMG_CUDA(cudaMemcpyAsync(G.cs64.p, cs.data(), g->m * sizeof(double2), cudaMemcpyHostToDevice, st));
    WMG_CUDA(cudaMemcpyAsync(G.cs32.p, cs32.data(), g->m * sizeof(float2), cudaMemcpyHostToDevice, st));
    WMG_CUDA(cudaStreamSynchronize(st));
    gd.cs64 = G.cs64.as<double2>();
    gd.cs32 = G.cs32.as<float2>();
    gd.csx = G.csx.as<float4>();
    gd.angf = G.angf.as<AngleF>();
    geometry_scalars(gd, angf.data());
    G.unit_bins = gd.unit != 0;
    // The 2h grid (Section 2.3): pixels of 2 x 2 blocks, L - 1 levels over
    // the same leaves, detector in 2h pixel widths; h stays the fine pixel
    // width (the halving of W^{2h} c / 2 = W I_{2h}^h c)
    G.has_2h = G.has_wmg && L >= 2 && gd.kernel == WMG_KERNEL_STRIP;
    if (G.has_2h) {
        GeomDev &gc = G.gc;
        gc = gd;
        gc.n = gd.n / 2; gc.L = L - 1; gc.K = gd.K / 4; gc.B = gd.B / 2;
        gc.t0 = 0.5 * gd.t0;
        gc.dt = 0.5 * gd.dt;
        gc.dinv = gc.leafinv = gc.sirtR = gc.sirtC = nullptr;
        geometry_scalars(gc, angf.data());
        G.Nc = (int64_t)gc.n * gc.n;
        G.haar_Wc = haar_width(gc);
    }
    return WMG_OK;
}

int32_t upload_geoms(wmg_plan *pl, cudaStream_t st)
{
    std::vector<GeomDev> h, h2;
    bool unit = true;
    for (auto &g : pl->geos) {
        if (!g) { h.push_back(GeomDev{}); h2.push_back(GeomDev{}); continue; }   // an evicted server geometry
        h.push_back(g->g);
        h2.push_back(g->has_2h ? g->gc : GeomDev{});
        unit = unit && g->unit_bins;
    }
    pl->unit_bins = unit;
    if (!pl->d_geom.ensure(h.size() * sizeof(GeomDev)) || !pl->d_geom_2h.ensure(h2.size() * sizeof(GeomDev)))
        return fail(WMG_ERR_OOM, "geometry table");
    WMG_CUDA(cudaMemcpyAsync(pl->d_geom.p, h.data(), h.size() * sizeof(GeomDev), cudaMemcpyHostToDevice, st));
    WMG_CUDA(cudaMemcpyAsync(pl->d_geom_2h.p, h2.data(), h2.size() * sizeof(GeomDev), cudaMemcpyHostToDevice, st));
    WMG_CUDA(cudaStreamSynchronize(st));
    return WMG_OK;
}

// nnz(W) of geometry gi, counted on the device on first use (a measurement
// aid: the solvers do not need it). Synchronising.
static int32_t count_nnz(wmg_plan *pl, int gi, cudaStream_t st, int64_t *out)
{
    Geo &G = *pl->geos[gi];
    if (G.nnz < 0) {
        ProbSet one;
        one.nprob = 1;
        one.h.assign(1, ProbDev{});
        one.h[0].geom = gi;
        one.h[0].kin1 = one.h[0].kout1 = G.g.K;
        build_tiles(pl, one);
        if (!upload_set(one, st)) return fail(WMG_ERR_OOM, "nnz tables");
        unsigned long long *dcount = nullptr;
        WMG_CUDA(cudaMallocAsync(&dcount, sizeof(unsigned long long), st));
        cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), st);
        launch_count_nnz(pl->d_geom.as<GeomDev>(), one.d.as<ProbDev>(), one.proj.tiles.as<int4>(), one.proj.n,
                         dcount, st);
        unsigned long long hcount = 0;
        cudaMemcpyAsync(&hcount, dcount, sizeof(hcount), cudaMemcpyDeviceToHost, st);
        WMG_CUDA(cudaStreamSynchronize(st));
        cudaFreeAsync(dcount, st);
        WMG_CUDA(cudaGetLastError());
        G.nnz = (int64_t)hcount;
    }
    *out = G.nnz;
    return WMG_OK;
}

// Device setup of geometry gi: D~ = W^T (W 1) + lambda, SIRT R and C and the
// leaf inverses. Runs on a one-slot table of that geometry.
template <class T>
int32_t setup_geometry(wmg_plan *pl, int gi, cudaStream_t st)
{
    Geo &G = *pl->geos[gi];
    const int64_t N = G.N, M = G.M;
    ProbSet one;
    one.nprob = 1;
    one.h.assign(1, ProbDev{});
    one.h[0].geom = gi;
    one.h[0].slot = 0;
    one.h[0].kin1 = one.h[0].kout1 = G.g.K;
    build_tiles(pl, one);
    if (!upload_set(one, st)) return fail(WMG_ERR_OOM, "setup tables");
    DevBuf ones_img, ones_sino, tmp_img, tmp_sino;
    if (!ones_img.ensure(N * sizeof(T)) || !ones_sino.ensure(M * sizeof(T)) ||
        !tmp_img.ensure(N * sizeof(T)) || !tmp_sino.ensure(M * sizeof(T)) ||
        !G.dinv.ensure(N * sizeof(T)) || !G.sirtR.ensure(M * sizeof(T)) || !G.sirtC.ensure(N * sizeof(T)))
        return fail(WMG_ERR_OOM, "setup allocation failed");
    count_launches(5);
    k_fill<T><<<num_sms() * 4, 256, 0, st>>>(ones_img.as<T>(), N, T(1));
    k_fill<T><<<num_sms() * 4, 256, 0, st>>>(ones_sino.as<T>(), M, T(1));
    // W 1 (row sums) -> R; W^T (W 1) -> D~; W^T 1 (column sums) -> C
    project<T>(pl, one, ones_img.p, ones_img.p, tmp_sino.p, nullptr, nullptr, st);
    k_recip<T><<<num_sms() * 4, 256, 0, st>>>(tmp_sino.as<T>(), G.sirtR.as<T>(), M, 0.0);
    BpArgs a = bp_args(BP_STORE, tmp_sino.p, nullptr);
    a.out_op = tmp_img.p;
    backproject<T>(pl, one, a, st);
    k_recip<T><<<num_sms() * 4, 256, 0, st>>>(tmp_img.as<T>(), G.dinv.as<T>(), N, G.g.lambda);
    a = bp_args(BP_STORE, ones_sino.p, nullptr);
    a.out_op = tmp_img.p;
    backproject<T>(pl, one, a, st);
    k_recip<T><<<num_sms() * 4, 256, 0, st>>>(tmp_img.as<T>(), G.sirtC.as<T>(), N, 0.0);
    G.nnz = -1;                                      // counted on first request (count_nnz)
    WMG_CUDA(cudaGetLastError());
    G.g.dinv = G.dinv.p;
    G.g.sirtR = G.sirtR.p;
    G.g.sirtC = G.sirtC.p;
    int32_t rc = upload_geoms(pl, st);
    if (rc) return rc;
    if (!G.has_wmg) return WMG_OK;
    if (!G.leafinv.ensure((size_t)G.g.K * G.g.P * G.g.P * sizeof(T)))
        return fail(WMG_ERR_OOM, "leaf inverse allocation failed");
    G.g.leafinv = G.leafinv.p;
    if ((rc = upload_geoms(pl, st))) return rc;
    rc = build_leaf_inverses(G.g, pl->d_geom.as<GeomDev>() + gi, G.leafinv.p, sizeof(T) == 4, st);
    if (rc) return rc;
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

template void project<float>(wmg_plan *, const ProbSet &, const void *, const void *, void *, double *,
                             const double *, cudaStream_t);
template void project<double>(wmg_plan *, const ProbSet &, const void *, const void *, void *, double *,
                              const double *, cudaStream_t);
template void backproject<float>(wmg_plan *, const ProbSet &, BpArgs, cudaStream_t);
template void backproject<double>(wmg_plan *, const ProbSet &, BpArgs, cudaStream_t);
template void img_op<float>(wmg_plan *, int, ImgArgs, cudaStream_t);
template void img_op<double>(wmg_plan *, int, ImgArgs, cudaStream_t);
template void vec_op<float>(wmg_plan *, int, bool, VecArgs, cudaStream_t);
template void vec_op<double>(wmg_plan *, int, bool, VecArgs, cudaStream_t);
template int32_t wmg_apply<float>(wmg_plan *, double *, double *, bool, bool, bool, bool *, cudaStream_t);
template int32_t wmg_apply<double>(wmg_plan *, double *, double *, bool, bool, bool, bool *, cudaStream_t);
template int32_t setup_geometry<float>(wmg_plan *, int, cudaStream_t);
template int32_t setup_geometry<double>(wmg_plan *, int, cudaStream_t);

}  // namespace wmg

using namespace wmg;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int32_t wmg_last_error(char *buf, size_t len)
{
    if (!buf || len == 0) return WMG_ERR_INVALID_ARG;
    const size_t n = std::min(len - 1, g_last_error.size());
    std::memcpy(buf, g_last_error.data(), n);
    buf[n] = 0;
    return WMG_OK;
}

extern "C" int32_t wmg_version(void) { return 100; }

extern "C" int32_t wmg_set_allocator(wmg_alloc_fn alloc, wmg_free_fn free, void *ctx)
{
    if (alloc && !free) return fail(WMG_ERR_INVALID_ARG, "wmg_set_allocator: an allocator needs its free function");
    std::lock_guard<std::mutex> lk(g_allocator_mu);
    g_allocator = alloc ? Allocator{alloc, free, ctx} : Allocator{};
    return WMG_OK;
}

// FNV-1a over everything that shapes a plan's arithmetic: the geometry
// (with every angle) and the WMG and solver options. A solver state is
// accepted only by a plan with the same fingerprint.
static uint64_t plan_fingerprint(const wmg_geom &g, const wmg_opts &o)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    };
    const double ds = g.det_spacing > 0 ? g.det_spacing : 1.0;
    const int32_t ints[] = {g.n, g.m, g.D, g.kernel, o.levels, o.nu1, o.nu2, o.hybrid_depth, o.cycle, o.precision};
    const double dbls[] = {ds, g.det_offset, o.omega, o.lambda};
    mix(ints, sizeof ints);
    mix(dbls, sizeof dbls);
    for (int a = 0; a < g.m; ++a) {
        const double t = g.angles ? g.angles[a] : a * (M_PI / g.m);
        mix(&t, sizeof t);
    }
    return h;
}

extern "C" int32_t wmg_plan_create(const wmg_geom *g, const wmg_opts *o, void *stream, wmg_plan **out)
{
    if (!out) return fail(WMG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int32_t rc = validate(g, o);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto pl = std::make_unique<wmg_plan>();
    pl->bf16 = o->precision == WMG_PREC_F32_BF16STORE;
    pl->prec = pl->bf16 ? WMG_PREC_F32 : o->precision;
    pl->esz = o->precision == WMG_PREC_F64 ? 8 : 4;
    pl->opts = *o;
    if (pl->opts.omega <= 0) pl->opts.omega = 1.0;
    pl->fingerprint = plan_fingerprint(*g, pl->opts);
    pl->geos.push_back(std::make_unique<Geo>());
    if ((rc = make_geo(g, o, *pl->geos[0], st))) return rc;
    if ((rc = upload_geoms(pl.get(), st))) return rc;
    if ((rc = ensure_count(pl.get(), 1, st))) return rc;
    rc = pl->prec == WMG_PREC_F64 ? setup_geometry<double>(pl.get(), 0, st) : setup_geometry<float>(pl.get(), 0, st);
    if (rc) return rc;
    WMG_CUDA(cudaStreamSynchronize(st));
    *out = pl.release();
    return WMG_OK;
}

extern "C" int32_t wmg_plan_destroy(wmg_plan *plan)
{
    if (!plan) return WMG_OK;
    cudaDeviceSynchronize();
    delete plan;
    return WMG_OK;
}

extern "C" int32_t wmg_plan_nnz(const wmg_plan *plan, int64_t *nnz)
{
    if (!plan || !nnz) return fail(WMG_ERR_INVALID_ARG, "wmg_plan_nnz: bad arguments");
    return count_nnz(const_cast<wmg_plan *>(plan), 0, nullptr, nnz);
    return WMG_OK;
}

extern "C" int32_t wmg_plan_get_tuning(const wmg_plan *plan, int32_t *project_ctas, int32_t *backproject_ctas)
{
    if (!plan) return fail(WMG_ERR_INVALID_ARG, "wmg_plan_get_tuning: plan is NULL");
    if (project_ctas) *project_ctas = plan->real.pj_ctas > 0 ? plan->real.pj_ctas : 8;
    if (backproject_ctas) *backproject_ctas = plan->real.bp_ctas > 0 ? plan->real.bp_ctas : 8;
    return WMG_OK;
}

extern "C" int32_t wmg_plan_set_tuning(wmg_plan *plan, int32_t project_ctas, int32_t backproject_ctas)
{
    if (!plan || project_ctas < 1 || project_ctas > 64 || backproject_ctas < 1 || backproject_ctas > 64)
        return fail(WMG_ERR_INVALID_ARG, "wmg_plan_set_tuning: bad arguments");
    plan->real.pj_ctas = project_ctas;
    plan->real.bp_ctas = backproject_ctas;
    for (auto &kv : plan->bands) {
        kv.second->pj_ctas = project_ctas;
        kv.second->bp_ctas = backproject_ctas;
    }
    return WMG_OK;
}

extern "C" int64_t wmg_launch_count(int32_t reset)
{
    return reset ? g_launches.exchange(0) : g_launches.load();
}

extern "C" int32_t wmg_profile_begin(wmg_plan *plan)
{
    if (!plan) return fail(WMG_ERR_INVALID_ARG, "wmg_profile_begin: plan is NULL");
    for (auto &r : plan->prof) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
    plan->prof.clear();
    plan->profiling = true;
    return WMG_OK;
}

extern "C" int32_t wmg_profile_end(wmg_plan *plan, wmg_profile_stats *out, void *stream)
{
    if (!plan || !out) return fail(WMG_ERR_INVALID_ARG, "wmg_profile_end: bad arguments");
    plan->profiling = false;
    WMG_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    std::memset(out, 0, sizeof(*out));
    for (auto &r : plan->prof) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        if (r.kind == 0) { out->project_launches++; out->project_ms += ms; out->project_images += r.images; }
        else if (r.kind == 2) {
            out->project_2h_launches++;
            out->project_2h_ms += ms;
            out->project_2h_images += r.images;
        } else { out->backproject_launches++; out->backproject_ms += ms; out->backproject_images += r.images; }
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    plan->prof.clear();
    int64_t nnz = 0;
    int32_t rc = count_nnz(plan, 0, static_cast<cudaStream_t>(stream), &nnz);
    if (rc) return rc;
    out->nnz_per_image = (double)nnz;
    return WMG_OK;
}

extern "C" int32_t wmg_plan_sizes(const wmg_plan *plan, int64_t *N, int64_t *M)
{
    if (!plan) return fail(WMG_ERR_INVALID_ARG, "plan is NULL");
    if (N) *N = plan->geos[0]->N;
    if (M) *M = plan->geos[0]->M;
    return WMG_OK;
}

#define WMG_DISPATCH(pl, fn, ...) \
    ((pl)->prec == WMG_PREC_F64 ? fn<double>(__VA_ARGS__) : fn<float>(__VA_ARGS__))

static int32_t single_geometry(wmg_plan *pl, const char *what)
{
    if (pl->batch) return fail(WMG_ERR_INVALID_ARG, std::string(what) + ": not available on a batch");
    return WMG_OK;
}

template <class T>
static int32_t do_project(wmg_plan *pl, const void *x, void *b, cudaStream_t st)
{
    if (!ensure_pool(pl->pT_op, pl->Ntot, pl->esz)) return fail(WMG_ERR_OOM, "workspace");
    const ProbSet &ps = pl->real;
    launch_transpose<T>(pl->d_geom.as<GeomDev>(), ps.d.as<ProbDev>(), ps.bp.tiles.as<int4>(), ps.bp.n, x,
                        pl->pT_op.p, st);
    project<T>(pl, ps, x, pl->pT_op.p, b, nullptr, nullptr, st);
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

extern "C" int32_t wmg_project(wmg_plan *pl, int32_t count, const void *x, void *b, void *stream)
{
    if (!pl || !x || !b || count < 1) return fail(WMG_ERR_INVALID_ARG, "wmg_project: bad arguments");
    int32_t rc = single_geometry(pl, "wmg_project");
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_count(pl, count, st))) return rc;
    pl->state.valid = false;                 // the transposed copy lives in a solver pool
    return WMG_DISPATCH(pl, do_project, pl, x, b, st);
}

template <class T>
static int32_t do_backproject(wmg_plan *pl, const void *b, void *x, cudaStream_t st)
{
    BpArgs a = bp_args(BP_STORE, b, nullptr);
    a.out_op = x;
    backproject<T>(pl, pl->real, a, st);
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

extern "C" int32_t wmg_backproject(wmg_plan *pl, int32_t count, const void *b, void *x, void *stream)
{
    if (!pl || !x || !b || count < 1) return fail(WMG_ERR_INVALID_ARG, "wmg_backproject: bad arguments");
    int32_t rc = single_geometry(pl, "wmg_backproject");
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_count(pl, count, st))) return rc;
    return WMG_DISPATCH(pl, do_backproject, pl, b, x, st);
}

template <class T>
static int32_t do_haar(wmg_plan *pl, bool analysis, const void *in, void *out, cudaStream_t st)
{
    const ProbSet &ps = pl->real;
    const GeomDev *G = pl->d_geom.as<GeomDev>();
    HaarArgs a{};
    a.in = in;
    a.out = out;
    if (analysis) {
        a.mode = HA_STORE;
        launch_haar_analysis<T, T>(G, ps.d.as<ProbDev>(), ps.haar.tiles.as<int4>(), ps.haar.n, ps.haar_smem, a, st);
    } else {
        a.mode = HS_STORE;
        launch_haar_synthesis<T, T>(G, ps.d.as<ProbDev>(), ps.haar.tiles.as<int4>(), ps.haar.n, ps.haar_smem, a, st);
    }
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

extern "C" int32_t wmg_haar_analysis(wmg_plan *pl, int32_t count, const void *x, void *c, void *stream)
{
    if (!pl || !x || !c || count < 1) return fail(WMG_ERR_INVALID_ARG, "wmg_haar_analysis: bad arguments");
    int32_t rc = single_geometry(pl, "wmg_haar_analysis");
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_count(pl, count, st))) return rc;
    return WMG_DISPATCH(pl, do_haar, pl, true, x, c, st);
}

extern "C" int32_t wmg_haar_synthesis(wmg_plan *pl, int32_t count, const void *c, void *x, void *stream)
{
    if (!pl || !x || !c || count < 1) return fail(WMG_ERR_INVALID_ARG, "wmg_haar_synthesis: bad arguments");
    int32_t rc = single_geometry(pl, "wmg_haar_synthesis");
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_count(pl, count, st))) return rc;
    return WMG_DISPATCH(pl, do_haar, pl, false, c, x, st);
}

extern "C" int32_t wmg_leaf_inverse(wmg_plan *pl, int64_t k, void *out, void *stream)
{
    if (!pl || !out || pl->batch || !pl->geos[0]->has_wmg || k < 0 || k >= pl->geos[0]->g.K)
        return fail(WMG_ERR_INVALID_ARG, "wmg_leaf_inverse: bad arguments (or a plan without WMG levels)");
    const Geo &G = *pl->geos[0];
    const int64_t PP = (int64_t)G.g.P * G.g.P;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WMG_CUDA(cudaMemcpyAsync(out, static_cast<const char *>(G.leafinv.p) + k * PP * pl->esz, PP * pl->esz,
                             cudaMemcpyDeviceToDevice, st));
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

// Fresh per-problem scalars. `warm`: CGLS from a given x0 takes its first
// residual as r = b - 1 * W x0 through the alpha-scaled residual update.
static void init_scalars(wmg_plan *pl, double rtol, int max_iter, cudaStream_t st, bool warm = false)
{
    const int count = pl->cap;
    std::vector<double> S((size_t)count * NSCAL, 0.0);
    for (int q = 0; q < count; ++q) {
        double *s = &S[(size_t)q * NSCAL];
        s[SC_ACTIVE] = 1.0;
        s[SC_STATUS] = WMG_NOT_CONVERGED;
        s[SC_RTOL] = rtol;
        s[SC_MAXIT] = max_iter;
        if (warm) s[SC_ALPHA] = 1.0;
    }
    cudaMemcpyAsync(pl->S.p, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
}

template <class T>
static int32_t do_precond(wmg_plan *pl, const void *s_in, void *z_out, cudaStream_t st)
{
    int32_t rc = ensure_wmg_pools(pl);
    if (rc) return rc;
    if (!ensure_partials(pl, 1)) return fail(WMG_ERR_OOM, "partials");
    init_scalars(pl, 0.0, 1, st);
    ImgArgs ia{};
    ia.in_op = s_in;
    ia.z = pl->s.as<double>();
    img_op<T>(pl, IMG_LOAD, ia, st);
    bool have = false;
    rc = wmg_apply<T>(pl, pl->s.as<double>(), pl->z.as<double>(), false, false, false, &have, st);
    if (rc) return rc;
    ImgArgs io{};
    io.z = pl->z.as<double>();
    io.out_op = z_out;
    img_op<T>(pl, IMG_STORE_OUT, io, st);
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

extern "C" int32_t wmg_precond_apply(wmg_plan *pl, int32_t count, const void *s, void *z, void *stream)
{
    if (!pl || !s || !z || count < 1) return fail(WMG_ERR_INVALID_ARG, "wmg_precond_apply: bad arguments");
    int32_t rc = single_geometry(pl, "wmg_precond_apply");
    if (rc) return rc;
    if (!pl->has_wmg()) return fail(WMG_ERR_INVALID_ARG, "wmg_precond_apply: the plan has no WMG levels");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_count(pl, count, st))) return rc;
    pl->state.valid = false;                 // runs in the solver pools
    return WMG_DISPATCH(pl, do_precond, pl, s, z, st);
}

// ---------------------------------------------------------------------------
// Solvers (every slot of the plan's table; b and x in slot layout)
// ---------------------------------------------------------------------------

// Capture `body(stream)` (a fixed sequence of launches) into g on the plan's
// private stream. Returns false (and leaves g empty) when graphs are off or
// the capture fails; the caller then runs the body eagerly.
template <class F>
static bool capture(wmg_plan *pl, Graph &g, F body)
{
    if (!pl->use_graphs || pl->profiling) return false;
    if (!pl->cap_stream && cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        pl->use_graphs = false;
        return false;
    }
    const long long before = g_launches.load();
    if (cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int32_t rc = body(pl->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &graph);
    const long long n = g_launches.load() - before;
    g_launches.fetch_sub(n);                 // nothing ran during the capture
    if (rc != WMG_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return false;
    }
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        g.exec = nullptr;
        return false;
    }
    g.launches = n;
    return true;
}

static int32_t replay(const Graph &g, cudaStream_t st)
{
    count_launches((int)g.launches);
    WMG_CUDA(cudaGraphLaunch(g.exec, st));
    return WMG_OK;
}

// ---------------------------------------------------------------------------
// Work lists of the problems still iterating. A batched solve runs until its
// slowest problem has converged; the problems that have stopped are skipped
// by every kernel (inactive flag), but their tiles are still scheduled, and
// the FP32 projector's group tiles, the leaf solves' work items and the
// band-update sets keep costing for every problem they cover. Once few
// problems are left, the solver swaps in a set whose stopped slots have no
// tiles at all -- the form a server's empty slots take -- and the slot list
// the WMG cycle walks is cut to the same problems. Every problem keeps its
// slot, offsets and arithmetic, and tiles never mix problems' sums, so the
// bits of each problem are those of the full set.
// ---------------------------------------------------------------------------
static void swap_buf(DevBuf &a, DevBuf &b)
{
    std::swap(a.p, b.p);
    std::swap(a.bytes, b.bytes);
    std::swap(a.persistent, b.persistent);
    std::swap(a.ast, b.ast);
    std::swap(a.owner, b.owner);
    std::swap(a.owner_stream, b.owner_stream);
}
static void swap_list(TileList &a, TileList &b)
{
    swap_buf(a.tiles, b.tiles);
    swap_buf(a.tb, b.tb);
    swap_buf(a.te, b.te);
    std::swap(a.n, b.n);
    std::swap(a.h, b.h);
}
static void swap_set(ProbSet &a, ProbSet &b)
{
    std::swap(a.nprob, b.nprob);
    std::swap(a.h, b.h);
    swap_buf(a.d, b.d);
    swap_list(a.proj, b.proj); swap_list(a.bp, b.bp); swap_list(a.haar, b.haar);
    swap_list(a.vimg, b.vimg); swap_list(a.vsino, b.vsino);
    swap_list(a.projg, b.projg); swap_list(a.proj1, b.proj1);
    swap_list(a.bpg, b.bpg); swap_list(a.bp1, b.bp1);
    std::swap(a.tma_n, b.tma_n);
    std::swap(a.tma_count, b.tma_count);
    std::swap(a.brk, b.brk);
    std::swap(a.haar_smem, b.haar_smem);
    std::swap(a.pj_ctas, b.pj_ctas);
    std::swap(a.bp_ctas, b.bp_ctas);
    std::swap(a.on_2h, b.on_2h);
    std::swap(a.grid2h, b.grid2h);
    std::swap(a.bp2h, b.bp2h);
    std::swap(a.rest, b.rest);
}

// A restriction pays once the live slots have fallen to this fraction; a
// projector group stays whole while this many of its problems are going.
constexpr double kRestrictFraction = 0.75;
constexpr int kGroupKeep = 3;

// Restriction of a plan's work lists to the slots still iterating, for the
// duration of one solve: restrict_to() swaps the restricted set into
// pl->real and pl->live; the destructor swaps the plan's own set back and
// drops the work-list caches built for restricted slot lists.
class ActiveSet {
  public:
    explicit ActiveSet(wmg_plan *p) : pl_(p) {}
    ActiveSet(const ActiveSet &) = delete;
    ActiveSet &operator=(const ActiveSet &) = delete;
    ~ActiveSet() { restore(); }
    int size() const { return (int)pl_->live.size(); }
    // The plan's own live slots whose active flag is set in the scalar table.
    std::vector<int> active(const std::vector<double> &S) const
    {
        std::vector<int> a;
        for (int q : on_ ? full_live_ : pl_->live)
            if (S[(size_t)q * NSCAL + SC_ACTIVE] != 0.0) a.push_back(q);
        return a;
    }
    bool on() const { return on_; }
    const std::vector<int> &live() const { return pl_->live; }
    // Restricts to the problems `going` (ascending, of the plan's own live
    // slots). FP32 plans keep a projector group of the plan's own set whole
    // while at least kGroupKeep of its problems are going (its other members
    // are masked in the kernels, as in the full set); a sparser group is
    // dropped and its going problems run one-image tiles. The slot list the
    // WMG cycle walks is every present problem whose active flag is set.
    // *changed: whether the work lists changed (they stay when the same
    // problems would be present with the same active ones).
    int32_t restrict_to(const std::vector<int> &going, const std::vector<double> &S, cudaStream_t st,
                        bool *changed)
    {
        *changed = false;
        if (!on_) {
            for (auto &kv : pl_->bands) kb_.push_back(kv.first);
            for (auto &kv : pl_->leafsets) kl_.push_back(kv.first);
            for (auto &kv : pl_->segsets) ks_.push_back(kv.first);
            full_live_ = pl_->live;
        }
        ProbSet &cur = pl_->real;
        const ProbSet &own = on_ ? *full_ : cur;
        const int np = own.nprob;
        std::vector<int> geom(np);
        std::vector<char> go(np, 0), present, brk;
        for (int q = 0; q < np; ++q) geom[q] = own.h[q].geom;
        for (int q : going) go[q] = 1;
        active_groups(geom, go, pl_->prec != WMG_PREC_F64, kProjGroup, kGroupKeep, present, brk);
        std::vector<int> live;
        for (int q = 0; q < np; ++q)
            if (present[q] && S[(size_t)q * NSCAL + SC_ACTIVE] != 0.0) live.push_back(q);
        if (on_ && live == pl_->live) {
            bool same = true;
            for (int q = 0; q < np && same; ++q) same = (cur.h[q].geom >= 0) == (present[q] != 0);
            if (same) return WMG_OK;
        }
        auto rs = std::make_unique<ProbSet>();
        rs->nprob = np;
        rs->h = own.h;
        rs->brk = brk;
        for (int q = 0; q < np; ++q)
            if (!present[q]) rs->h[q].geom = -1;
        build_tiles(pl_, *rs);
        if (!upload_set(*rs, st)) return fail(WMG_ERR_OOM, "work-list allocation failed");
        rs->pj_ctas = cur.pj_ctas;
        rs->bp_ctas = cur.bp_ctas;
        // the plan's own set is kept aside (first restriction) or the previous
        // restricted set is held (later ones)
        if (!on_) {
            full_ = std::make_unique<ProbSet>();
            swap_set(*full_, cur);
        }
        swap_set(cur, *rs);                  // rs now holds the previous restricted set (or nothing)
        held_.push_back(std::move(rs));      // freed at restore (graphs may still name it)
        pl_->live = live;
        on_ = true;
        *changed = true;
        return WMG_OK;
    }

    // The plan's own set and slot list back (before the results are stored).
    void restore()
    {
        if (!on_) return;
        swap_set(pl_->real, *full_);
        pl_->live = full_live_;
        drop_new(pl_->bands, kb_);
        drop_new(pl_->leafsets, kl_);
        drop_new(pl_->segsets, ks_);
        on_ = false;
    }

  private:
    template <class M>
    static void drop_new(M &m, const std::vector<std::vector<int>> &keep)
    {
        for (auto it = m.begin(); it != m.end();) {
            if (std::find(keep.begin(), keep.end(), it->first) == keep.end()) it = m.erase(it);
            else ++it;
        }
    }
    wmg_plan *pl_;
    bool on_ = false;
    std::unique_ptr<ProbSet> full_;
    std::vector<std::unique_ptr<ProbSet>> held_;
    std::vector<int> full_live_;
    std::vector<std::vector<int>> kb_, kl_, ks_;
};

// Per-slot results; `order` (optional) maps the caller's problem i to its slot.
static int32_t collect(wmg_plan *pl, int max_iter, wmg_solve_info *info, double *res_hist, cudaStream_t st)
{
    const int count = pl->cap;
    std::vector<double> S((size_t)count * NSCAL);
    std::vector<double> H;
    WMG_CUDA(cudaMemcpyAsync(S.data(), pl->S.p, S.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (res_hist) {
        H.resize((size_t)count * (max_iter + 1));
        WMG_CUDA(cudaMemcpyAsync(H.data(), pl->hist.p, H.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    WMG_CUDA(cudaStreamSynchronize(st));
    WMG_CUDA(cudaGetLastError());
    if (const int e = tma_error_take())
        return e == 1 ? fail(WMG_ERR_TIMEOUT, "projector: a wait for staged pixels timed out")
                      : fail(WMG_ERR_CUDA, "projector: a candidate pixel fell outside its staged box");
    if (tc_error_take()) return fail(WMG_ERR_TIMEOUT, "leaf solves: a wait for the tensor-core products timed out");
    if (bpg_error_take()) return fail(WMG_ERR_CUDA, "backprojector: a candidate bin fell outside its staged window");
    int32_t rc = WMG_OK;
    for (int i = 0; i < count; ++i) {
        const int q = pl->batch ? pl->order[i] : i;
        const double *s = &S[(size_t)q * NSCAL];
        int status = (int)s[SC_STATUS];
        if (s[SC_ACTIVE] != 0.0) status = WMG_NOT_CONVERGED;
        if (info) {
            info[i].iters = (int)s[SC_ITERS];
            info[i].status = status;
            info[i].rel_res = s[SC_RES];
        }
        if (res_hist)
            std::memcpy(res_hist + (size_t)i * (max_iter + 1), H.data() + (size_t)q * (max_iter + 1),
                        (max_iter + 1) * sizeof(double));
        if (status < 0 && rc >= 0) rc = status;
        else if (status == WMG_NOT_CONVERGED && rc == WMG_OK) rc = WMG_NOT_CONVERGED;
    }
    return rc;
}

// The pools each solver keeps its vectors in (all slots back to back). A
// resumed solve and a state import ask for the same sizes, so neither moves
// (and so empties) a pool the other filled.
static int32_t solver_pools(wmg_plan *pl, int solver, bool pre, int restart)
{
    const int count = pl->cap;
    const int64_t nN = pl->Ntot, nM = pl->Mtot;
    const size_t e = pl->esz;
    bool ok;
    const char *what;
    if (solver == WMG_SOLVER_CGLS) {
        what = "CGLS pools";
        ok = ensure_pool(pl->x, nN, 8) && ensure_pool(pl->s, nN, 8) && ensure_pool(pl->z, nN, 8) &&
             ensure_pool(pl->p, nN, 8) && ensure_pool(pl->r, nM, 8) && ensure_pool(pl->p_op, nN, e) &&
             ensure_pool(pl->pT_op, nN, e) && ensure_pool(pl->q, nM, e) && ensure_pool(pl->r_op, nM, e) &&
             ensure_partials(pl, 1);
    } else if (solver == WMG_SOLVER_SIRT) {
        what = "SIRT pools";
        ok = ensure_pool(pl->x, nN, 8) && ensure_pool(pl->p_op, nN, e) && ensure_pool(pl->pT_op, nN, e) &&
             ensure_pool(pl->q, nM, e) && ensure_pool(pl->r_op, nM, e) && ensure_pool(pl->s, nN, 8) &&
             ensure_partials(pl, 1);
    } else if (solver == WMG_SOLVER_GMRES) {
        what = "GMRES pools";
        const int ldp = restart + 1;
        ok = ensure_pool(pl->x, nN, 8) && ensure_pool(pl->f, nN, 8) && ensure_pool(pl->w, nN, 8) &&
             ensure_pool(pl->t, nN, 8) && ensure_pool(pl->u, nN, 8) && ensure_pool(pl->V, nN * ldp, 8) &&
             ensure_pool(pl->z_op, nN, e) && ensure_pool(pl->zT_op, nN, e) && ensure_pool(pl->sinoS, nM, e) &&
             ensure_partials(pl, ldp) && pl->H.ensure((size_t)count * ldp * restart * 8) &&
             pl->gcs.ensure((size_t)count * restart * 8) && pl->gsn.ensure((size_t)count * restart * 8) &&
             pl->gg.ensure((size_t)count * ldp * 8) && pl->gy.ensure((size_t)count * ldp * 8) &&
             pl->h1.ensure((size_t)count * ldp * 8) && pl->h2.ensure((size_t)count * ldp * 8) &&
             pl->jn.ensure((size_t)count * 4) && pl->done.ensure((size_t)count * 4) &&
             pl->reo.ensure((size_t)count * 4);
    } else {
        what = "BiCGStab pools";
        ok = ensure_pool(pl->x, nN, 8) && ensure_pool(pl->f, nN, 8) && ensure_pool(pl->w, nN, 8) &&
             ensure_pool(pl->p, nN, 8) && ensure_pool(pl->t, nN, 8) && ensure_pool(pl->u, nN, 8) &&
             ensure_pool(pl->z, nN, 8) && ensure_pool(pl->bi_t, nN, 8) && ensure_pool(pl->bi_sh, nN, 8) &&
             ensure_pool(pl->z_op, nN, e) && ensure_pool(pl->zT_op, nN, e) && ensure_pool(pl->sinoS, nM, e) &&
             ensure_partials(pl, 1);
    }
    if (!ok) return fail(WMG_ERR_OOM, what);
    if (pre && solver != WMG_SOLVER_SIRT) return ensure_wmg_pools(pl);
    return WMG_OK;
}

// The device ranges that hold the state of the plan's last solve: the
// per-problem scalars and residual histories, and every vector a later
// iteration reads (operator-precision copies included, so that nothing is
// rounded again on the way back).
struct Region {
    void *p;
    size_t bytes;
};

static std::vector<Region> state_regions(wmg_plan *pl)
{
    const SolveState &st = pl->state;
    const size_t count = (size_t)pl->cap, nN8 = (size_t)pl->Ntot * 8, nM8 = (size_t)pl->Mtot * 8;
    const size_t nNe = (size_t)pl->Ntot * pl->esz, ldp = (size_t)st.restart + 1;
    std::vector<Region> r{{pl->S.p, count * NSCAL * 8}, {pl->hist.p, count * st.hist_ld * 8}, {pl->x.p, nN8}};
    if (st.solver == WMG_SOLVER_SIRT) {
        // x and its operator copies (the next projection's input)
        r.insert(r.end(), {{pl->p_op.p, nNe}, {pl->pT_op.p, nNe}});
    } else if (st.solver == WMG_SOLVER_CGLS) {
        // r, p and their copies; s (and with a preconditioner z and its
        // copies, the fused first smoothing sweep) for the end of the step
        r.insert(r.end(), {{pl->r.p, nM8}, {pl->p.p, nN8}, {pl->s.p, nN8}, {pl->z.p, nN8},
                           {pl->p_op.p, nNe}, {pl->pT_op.p, nNe}});
        if (st.pre) r.insert(r.end(), {{pl->z_op.p, nNe}, {pl->zT_op.p, nNe}});
    } else if (st.solver == WMG_SOLVER_GMRES) {
        // at a restart: W^T b, the true residual in basis slot 0, the
        // least-squares and rotation data
        r.insert(r.end(), {{pl->f.p, nN8}, {pl->V.p, nN8}, {pl->H.p, count * ldp * st.restart * 8},
                           {pl->gcs.p, count * st.restart * 8}, {pl->gsn.p, count * st.restart * 8},
                           {pl->gg.p, count * ldp * 8}, {pl->jn.p, count * 4}, {pl->done.p, count * 4}});
    } else {
        // r, the shadow residual, p and v
        r.insert(r.end(), {{pl->f.p, nN8}, {pl->w.p, nN8}, {pl->p.p, nN8}, {pl->t.p, nN8}});
    }
    return r;
}

// CGLS from x0 (NULL: 0), or, with start > 0, the continuation of the solve
// whose state the plan holds after `start` iterations.
template <class T>
static int32_t solve_cgls(wmg_plan *pl, bool pre, const void *b, const void *x0, void *xout, int max_iter,
                          int start, cudaStream_t st)
{
    const int64_t nN = pl->Ntot;
    int32_t rc0 = solver_pools(pl, WMG_SOLVER_CGLS, pre, 0);
    if (rc0) return rc0;
    const ProbSet &ps = pl->real;
    const double *S = pl->S.as<double>();
    double *hist = pl->hist.as<double>();
    const int hld = max_iter + 1;
    double *pa = pl->part_a.as<double>(), *pb = pl->part_b.as<double>(), *pc = pl->part_c.as<double>();
    const bool smooth_fused = pre && pl->opts.nu1 >= 1;
    double *zvec = pre ? pl->z.as<double>() : pl->s.as<double>();
    bool have_sz = false;
    auto bp_s = [&](cudaStream_t s) {
        BpArgs a = bp_args(BP_CGLS_S, pl->r_op.p, S);
        a.x = pl->x.as<double>(); a.p = pl->p.as<double>(); a.s = pl->s.as<double>();
        a.part = pa;
        if (smooth_fused) { a.z = pl->z.as<double>(); a.copy_op = pl->z_op.p; a.copyT_op = pl->zT_op.p; }
        backproject<T>(pl, ps, a, s);
    };
    // z = B s, beta, p = z + beta p: the end of an iteration, after the
    // residual test
    auto step_end = [&](cudaStream_t s) -> int32_t {
        if (pre) {
            int32_t rc = wmg_apply<T>(pl, pl->s.as<double>(), pl->z.as<double>(), smooth_fused, false, true,
                                      &have_sz, s);
            if (rc) return rc;
            if (!have_sz) {
                ImgArgs ia{};
                ia.s = pl->s.as<double>(); ia.z = pl->z.as<double>(); ia.part = pb; ia.S = S;
                img_op<T>(pl, IMG_DOT_SZ, ia, s);
            }
        }
        finalize(pl, FIN_CGLS_BETA, ps.bp, pb, 1, nullptr, nullptr, pre, hist, hld, s);
        ImgArgs pu{};
        pu.z = zvec; pu.p = pl->p.as<double>(); pu.copy_op = pl->p_op.p; pu.copyT_op = pl->pT_op.p; pu.part = pc;
        pu.S = S;
        img_op<T>(pl, IMG_PUPDATE, pu, s);
        finalize(pl, FIN_PNORM, ps.bp, pc, 1, nullptr, nullptr, pre, hist, hld, s);
        return WMG_OK;
    };
    if (start == 0) {
        cudaMemsetAsync(pl->p.p, 0, nN * 8, st);
        VecArgs va{};
        va.r = pl->r.as<double>(); va.b_op = b; va.r_op = pl->r_op.p; va.S = S;
        if (x0) {
            // x = x0; r = b - alpha W x0 with alpha = 1 (init_scalars), so that
            // the x update of the backprojection below (x += alpha p, p = 0)
            // leaves x0 as it is
            ImgArgs il{};
            il.in_op = x0; il.z = pl->x.as<double>(); il.copy_op = pl->p_op.p; il.copyT_op = pl->pT_op.p; il.S = S;
            img_op<T>(pl, IMG_LOAD, il, st);
            project<T>(pl, ps, pl->p_op.p, pl->pT_op.p, pl->q.p, nullptr, S, st);
            vec_op<T>(pl, VEC_R_INIT, true, va, st);
            VecArgs vr{};
            vr.r = pl->r.as<double>(); vr.q = pl->q.p; vr.r_op = pl->r_op.p; vr.S = S;
            vec_op<T>(pl, VEC_R_UPDATE, true, vr, st);
        } else {
            // r = b, s = W^T r (x = 0, alpha = 0)
            cudaMemsetAsync(pl->x.p, 0, nN * 8, st);
            vec_op<T>(pl, VEC_R_INIT, true, va, st);
        }
        bp_s(st);
        if (pre) {
            int32_t rc = wmg_apply<T>(pl, pl->s.as<double>(), pl->z.as<double>(), smooth_fused, false, true,
                                      &have_sz, st);
            if (rc) return rc;
            if (!have_sz) {
                ImgArgs ia{};
                ia.s = pl->s.as<double>(); ia.z = pl->z.as<double>(); ia.part = pb; ia.S = S;
                img_op<T>(pl, IMG_DOT_SZ, ia, st);
            }
        }
        finalize(pl, FIN_CGLS_INIT, ps.bp, pa, 1, pre ? &ps.bp : nullptr, pre ? pb : nullptr, pre, hist, hld, st);
        ImgArgs pi{};
        pi.z = zvec; pi.p = pl->p.as<double>(); pi.copy_op = pl->p_op.p; pi.copyT_op = pl->pT_op.p; pi.part = pc;
        pi.S = S;
        img_op<T>(pl, IMG_PINIT, pi, st);
        finalize(pl, FIN_PNORM, ps.bp, pc, 1, nullptr, nullptr, pre, hist, hld, st);
    } else {
        // the problems resumed stopped at the residual test of their last
        // iteration: finish that iteration
        int32_t rc = step_end(st);
        if (rc) return rc;
    }
    // one iteration (a fixed launch sequence: every per-iteration decision is
    // taken on the device from the scalars)
    auto iteration = [&](cudaStream_t s) -> int32_t {
        project<T>(pl, ps, pl->p_op.p, pl->pT_op.p, pl->q.p, pa, S, s);
        finalize(pl, FIN_CGLS_ALPHA, ps.proj, pa, 1, nullptr, nullptr, pre, hist, hld, s);
        VecArgs vr{};
        vr.r = pl->r.as<double>(); vr.q = pl->q.p; vr.r_op = pl->r_op.p; vr.S = S;
        vec_op<T>(pl, VEC_R_UPDATE, true, vr, s);
        bp_s(s);
        finalize(pl, FIN_CGLS_RES, ps.bp, pa, 1, nullptr, nullptr, pre, hist, hld, s);
        return step_end(s);
    };
    const int chunk = 4;
    // once few problems are left, the iterations run on their work lists only
    // (ActiveSet), eagerly, with the flags tested after every iteration
    ActiveSet act(pl);
    Graph graph;
    bool graphed = false;
    std::vector<double> Sh((size_t)pl->cap * NSCAL);
    for (int it = start; it < max_iter; ++it) {
        // the first iteration runs eagerly (it fills the work-list caches),
        // the others replay its captured graph
        if (it == start + 1 && !act.on()) graphed = capture(pl, graph, iteration);
        int32_t rc = graphed ? replay(graph, st) : iteration(st);
        if (rc) return rc;
        if ((it + 1) % (act.on() ? 1 : chunk) == 0 || it + 1 == max_iter) {
            WMG_CUDA(cudaMemcpyAsync(Sh.data(), pl->S.p, Sh.size() * 8, cudaMemcpyDeviceToHost, st));
            WMG_CUDA(cudaStreamSynchronize(st));
            const std::vector<int> left = act.active(Sh);
            if (left.empty()) break;
            if (left.size() <= kRestrictFraction * act.size() && it + 1 < max_iter) {
                bool changed = false;
                if ((rc = act.restrict_to(left, Sh, st, &changed))) return rc;
                if (changed) {
                    graph.reset();
                    graphed = false;
                }
            }
        }
    }
    act.restore();
    ImgArgs io{};
    io.z = pl->x.as<double>(); io.out_op = xout;
    img_op<T>(pl, IMG_STORE_OUT, io, st);
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

// SIRT from x0 (NULL: 0), or its continuation after `start` iterations.
template <class T>
static int32_t solve_sirt(wmg_plan *pl, const void *b, const void *x0, void *xout, int max_iter, int start,
                          cudaStream_t st)
{
    const int count = pl->cap;
    const int64_t nN = pl->Ntot;
    const size_t e = pl->esz;
    int32_t rc0 = solver_pools(pl, WMG_SOLVER_SIRT, false, 0);
    if (rc0) return rc0;
    const ProbSet &ps = pl->real;
    const double *S = pl->S.as<double>();
    double *pb = pl->part_b.as<double>();
    // |W^T (b - W x) - lambda x|^2 of the current x, finished by `fin`
    auto ne_residual = [&](int fin, int slot) {
        project<T>(pl, ps, pl->p_op.p, pl->pT_op.p, pl->q.p, nullptr, S, st);
        VecArgs vd{};
        vd.b_op = b; vd.q = pl->q.p; vd.r_op = pl->r_op.p; vd.S = S;
        vec_op<T>(pl, VEC_SINO_DIFF, true, vd, st);
        BpArgs ra = bp_args(BP_ATB, pl->r_op.p, S);
        ra.out64 = pl->s.as<double>();
        backproject<T>(pl, ps, ra, st);
        VecArgs vn{};
        vn.w = pl->s.as<double>(); vn.x = pl->x.as<double>(); vn.part = pb; vn.S = S;
        vec_op<T>(pl, VEC_NE_RES, false, vn, st);
        finalize(pl, fin, ps.vimg, pb, 1, nullptr, nullptr, 0, nullptr, 0, st, slot);
    };
    if (start == 0) {
        // the reference of the relative residual: |W^T b|, or from x0 the
        // NE residual of x0
        if (x0) {
            ImgArgs il{};
            il.in_op = x0; il.z = pl->x.as<double>(); il.copy_op = pl->p_op.p; il.copyT_op = pl->pT_op.p; il.S = S;
            img_op<T>(pl, IMG_LOAD, il, st);
            ne_residual(FIN_STORE, SC_S0);
        } else {
            cudaMemsetAsync(pl->x.p, 0, nN * 8, st);
            cudaMemsetAsync(pl->p_op.p, 0, nN * e, st);
            cudaMemsetAsync(pl->pT_op.p, 0, nN * e, st);
            BpArgs fa = bp_args(BP_ATB, b, S);
            fa.out64 = pl->s.as<double>(); fa.part = pb;
            backproject<T>(pl, ps, fa, st);
            finalize(pl, FIN_STORE, ps.bp, pb, 1, nullptr, nullptr, 0, nullptr, 0, st, SC_S0);
        }
    }
    for (int it = start; it < max_iter; ++it) {
        project<T>(pl, ps, pl->p_op.p, pl->pT_op.p, pl->q.p, nullptr, S, st);
        VecArgs va{};
        va.b_op = b; va.q = pl->q.p; va.r_op = pl->r_op.p; va.S = S;
        vec_op<T>(pl, VEC_SIRT_R, true, va, st);
        BpArgs a = bp_args(BP_SIRT, pl->r_op.p, S);
        a.x = pl->x.as<double>(); a.copy_op = pl->p_op.p; a.copyT_op = pl->pT_op.p;
        backproject<T>(pl, ps, a, st);
    }
    // relative NE residual of the final iterate: |W^T (b - W x) - lambda x| / S0
    ne_residual(FIN_SET_RES, 0);
    std::vector<double> Sh((size_t)count * NSCAL);
    WMG_CUDA(cudaMemcpyAsync(Sh.data(), pl->S.p, Sh.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    WMG_CUDA(cudaStreamSynchronize(st));
    for (int q = 0; q < count; ++q) Sh[(size_t)q * NSCAL + SC_ITERS] = std::max(max_iter, start);
    WMG_CUDA(cudaMemcpyAsync(pl->S.p, Sh.data(), Sh.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    ImgArgs io{};
    io.z = pl->x.as<double>(); io.out_op = xout;
    img_op<T>(pl, IMG_STORE_OUT, io, st);
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

// Restarted GMRES from x0 (NULL: 0), or, with start > 0, the continuation of
// the solve whose state (at a restart) the plan holds after `start` steps.
template <class T>
static int32_t solve_gmres(wmg_plan *pl, bool pre, const void *b, const void *x0, void *xout, int max_iter,
                           int restart, int start, cudaStream_t st)
{
    const int count = pl->cap;
    const int64_t nN = pl->Ntot;
    const int ldp = restart + 1;
    int32_t rc0 = solver_pools(pl, WMG_SOLVER_GMRES, pre, restart);
    if (rc0) return rc0;
    const ProbSet &ps = pl->real;
    const double *S = pl->S.as<double>();
    double *hist = pl->hist.as<double>();
    const int hld = max_iter + 1;
    double *pa = pl->part_a.as<double>(), *pb = pl->part_b.as<double>();
    double *V = pl->V.as<double>();
    const int64_t vstride = nN;
    GmArgs ga{};
    ga.nprob = count; ga.restart = restart; ga.ldp = ldp;
    ga.S = pl->S.as<double>(); ga.H = pl->H.as<double>(); ga.cs = pl->gcs.as<double>();
    ga.sn = pl->gsn.as<double>(); ga.g = pl->gg.as<double>(); ga.y = pl->gy.as<double>();
    ga.h1 = pl->h1.as<double>(); ga.h2 = pl->h2.as<double>(); ga.jn = pl->jn.as<int>();
    ga.done = pl->done.as<int>(); ga.skip = pl->reo.as<int>(); ga.hist = hist; ga.hist_ld = hld;
    // the work lists in use (the plan's own, or those of the problems left)
    const ProbDev *P = ps.d.as<ProbDev>();
    const int4 *vt = ps.vimg.tiles.as<int4>();
    int nv = ps.vimg.n;
    if (start == 0) {
        cudaMemsetAsync(pl->H.p, 0, (size_t)count * ldp * restart * 8, st);
        // f = W^T b ; r0 = f - A x0 ; V_0 = r0 / |r0|
        BpArgs fa = bp_args(BP_ATB, b, S);
        fa.out64 = pl->f.as<double>(); fa.part = pb;
        backproject<T>(pl, ps, fa, st);
        if (x0) {
            ImgArgs il{};
            il.in_op = x0; il.z = pl->x.as<double>(); il.copy_op = pl->z_op.p; il.copyT_op = pl->zT_op.p; il.S = S;
            img_op<T>(pl, IMG_LOAD, il, st);
            project<T>(pl, ps, pl->z_op.p, pl->zT_op.p, pl->sinoS.p, nullptr, S, st);
            BpArgs wa = bp_args(BP_GMRES_W, pl->sinoS.p, S);
            wa.z = pl->x.as<double>(); wa.out64 = pl->w.as<double>();
            backproject<T>(pl, ps, wa, st);
            VecArgs rv{};
            rv.f = pl->f.as<double>(); rv.w = pl->w.as<double>(); rv.v = V; rv.part = pb; rv.S = S;
            vec_op<T>(pl, VEC_RESID64, false, rv, st);
            finalize(pl, FIN_STORE, ps.vimg, pb, 1, nullptr, nullptr, 0, nullptr, 0, st, SC_WNORM2);
        } else {
            cudaMemsetAsync(pl->x.p, 0, nN * 8, st);
            finalize(pl, FIN_STORE, ps.bp, pb, 1, nullptr, nullptr, 0, nullptr, 0, st, SC_WNORM2);
        }
        ga.init = 1;
        launch_gm_scalar(2, ga, st);
        ga.init = 0;
        launch_gm_setv(P, vt, nv, V, vstride, ldp, 0, x0 ? V : pl->f.as<double>(), S, st);
    } else {
        // the problems resumed stopped at the restart test, before their
        // true residual was scaled into v_0
        launch_gm_setv(P, vt, nv, V, vstride, ldp, 0, V, S, st);
    }
    const int *jv = pl->jn.as<int>();
    ga.jslot = 1;
    // One Arnoldi step for every problem at its own column j = jn[slot]
    // (the same for all problems of a solve): u = B v_j, w = A u, two
    // classical Gram-Schmidt passes, Hessenberg column, Givens, v_{j+1}.
    // Every index lives on the device, so the step is one fixed launch
    // sequence (a graph after its first run).
    auto arnoldi = [&](cudaStream_t s) -> int32_t {
        // BF16 operator storage (WMG_PREC_F32_BF16STORE): the operator inputs
        // of the step; the restarts' true residuals stay FP32
        struct Bf16Scope {
            wmg_plan *p;
            Bf16Scope(wmg_plan *q, bool on) : p(q) { p->bf16_now = on; }
            ~Bf16Scope() { p->bf16_now = false; }
        } bf16_scope(pl, pl->bf16 && pre);
        launch_gm_getv(P, vt, nv, V, vstride, jv, pl->t.as<double>(), S, s);
        if (pre) {
            bool have = false;
            int32_t rc = wmg_apply<T>(pl, pl->t.as<double>(), pl->u.as<double>(), false, true, false, &have, s);
            if (rc) return rc;
        } else {
            WMG_CUDA(cudaMemcpyAsync(pl->u.p, pl->t.p, nN * 8, cudaMemcpyDeviceToDevice, s));
            ImgArgs ic{};
            ic.z = pl->u.as<double>(); ic.copy_op = pl->z_op.p; ic.copyT_op = pl->zT_op.p; ic.S = S;
            img_op<T>(pl, IMG_COPY64, ic, s);
        }
        project<T>(pl, ps, pl->z_op.p, pl->zT_op.p, pl->sinoS.p, nullptr, S, s);
        BpArgs wa = bp_args(BP_GMRES_W, pl->sinoS.p, S);
        wa.z = pl->u.as<double>(); wa.out64 = pl->w.as<double>();
        backproject<T>(pl, ps, wa, s);
        // classical Gram-Schmidt, the second pass only where the first one
        // cancelled (k_gm_reorth); |w|^2 partials from the last pass run
        int *skip = pl->reo.as<int>();
        for (int pass = 0; pass < 2; ++pass) {
            launch_gm_dots(P, vt, nv, V, vstride, pl->w.as<double>(), 0, ldp, pa, S, s, jv, pass == 0,
                           pass == 1 ? skip : nullptr);
            double *hv = pass == 0 ? pl->h1.as<double>() : pl->h2.as<double>();
            // all ldp columns are summed; the Arnoldi step reads those <= j
            // (and the reorthogonalisation test column j + 1 of the first)
            finalize(pl, FIN_STORE, ps.vimg, pa, ldp, nullptr, nullptr, 0, nullptr, 0, s, 0, hv, ldp, ldp);
            launch_gm_axpy(P, vt, nv, V, vstride, pl->w.as<double>(), 0, ldp, hv, pb, S, s, jv,
                           pass == 1 ? skip : nullptr);
            if (pass == 0) launch_gm_scalar(3, ga, s);
        }
        finalize(pl, FIN_STORE, ps.vimg, pb, 1, nullptr, nullptr, 0, nullptr, 0, s, SC_WNORM2);
        launch_gm_scalar(0, ga, s);
        launch_gm_setv(P, vt, nv, V, vstride, ldp, 0, pl->w.as<double>(), S, s, jv);
        return WMG_OK;
    };
    // End of a cycle: y = H^-1 g, t = V y, x += B t, true residual r = f - A x
    // into v_0, restart (or stop) on |r|.
    auto cycle_end = [&](cudaStream_t s) -> int32_t {
        launch_gm_scalar(1, ga, s);
        launch_gm_combine(P, vt, nv, V, vstride, ldp, pl->gy.as<double>(), pl->jn.as<int>(), pl->t.as<double>(), S,
                          s);
        if (pre) {
            bool have = false;
            int32_t rc = wmg_apply<T>(pl, pl->t.as<double>(), pl->u.as<double>(), false, false, false, &have, s);
            if (rc) return rc;
        } else {
            WMG_CUDA(cudaMemcpyAsync(pl->u.p, pl->t.p, nN * 8, cudaMemcpyDeviceToDevice, s));
        }
        VecArgs xa{};
        xa.x = pl->x.as<double>(); xa.w = pl->u.as<double>(); xa.S = S;
        vec_op<T>(pl, VEC_X_ADD, false, xa, s);
        ImgArgs ic{};
        ic.z = pl->x.as<double>(); ic.copy_op = pl->z_op.p; ic.copyT_op = pl->zT_op.p; ic.S = S;
        img_op<T>(pl, IMG_COPY64, ic, s);
        project<T>(pl, ps, pl->z_op.p, pl->zT_op.p, pl->sinoS.p, nullptr, S, s);
        BpArgs wa = bp_args(BP_GMRES_W, pl->sinoS.p, S);
        wa.z = pl->x.as<double>(); wa.out64 = pl->w.as<double>();
        backproject<T>(pl, ps, wa, s);
        VecArgs rv{};
        rv.f = pl->f.as<double>(); rv.w = pl->w.as<double>(); rv.v = V; rv.part = pb; rv.S = S;
        vec_op<T>(pl, VEC_RESID64, false, rv, s);
        finalize(pl, FIN_STORE, ps.vimg, pb, 1, nullptr, nullptr, 0, nullptr, 0, s, SC_WNORM2);
        launch_gm_scalar(2, ga, s);
        launch_gm_setv(P, vt, nv, V, vstride, ldp, 0, V, S, s);
        return WMG_OK;
    };
    ActiveSet act(pl);                        // declared before the graphs that may name its lists
    Graph g_step, g_end;
    bool step_graphed = false, end_graphed = false, step_tried = false, end_tried = false;
    int done_iters = start, eager_steps = 0;
    // Restriction to the problems left (ActiveSet): the Arnoldi steps run on
    // the problems still iterating in the cycle (active, not done), the cycle
    // end on every active problem (those done in the cycle update x and
    // restart or stop there). Once restricted, the loop tests the flags after
    // every step, and the launches stay eager (the lists change too often for
    // graphs to pay).
    std::vector<double> Sh((size_t)count * NSCAL);
    std::vector<int> dn(count);
    auto use = [&](const std::vector<int> &slots) -> int32_t {
        bool changed = false;
        int32_t rc = act.restrict_to(slots, Sh, st, &changed);
        if (rc || !changed) return rc;
        P = ps.d.as<ProbDev>();
        vt = ps.vimg.tiles.as<int4>();
        nv = ps.vimg.n;
        g_step.reset(); g_end.reset();
        step_graphed = end_graphed = false;
        step_tried = end_tried = true;                 // no further captures
        return WMG_OK;
    };
    auto read_flags = [&]() -> int32_t {
        WMG_CUDA(cudaMemcpyAsync(dn.data(), pl->done.p, count * 4, cudaMemcpyDeviceToHost, st));
        WMG_CUDA(cudaMemcpyAsync(Sh.data(), pl->S.p, Sh.size() * 8, cudaMemcpyDeviceToHost, st));
        WMG_CUDA(cudaStreamSynchronize(st));
        return WMG_OK;
    };
    while (true) {
        cudaMemsetAsync(pl->done.p, 0, (size_t)count * 4, st);
        int j = 0;
        for (; j < restart && done_iters < max_iter; ++j, ++done_iters) {
            // first step on a work list eager (fills the work-list caches), then the graph
            if (!step_tried && eager_steps >= 1) {
                step_tried = true;
                step_graphed = capture(pl, g_step, arnoldi);
            }
            if (!step_tried) ++eager_steps;
            int32_t rc = step_graphed ? replay(g_step, st) : arnoldi(st);
            if (rc) return rc;
            if ((j + 1) % (act.on() ? 1 : 4) == 0) {
                if ((rc = read_flags())) return rc;
                std::vector<int> going;
                for (int q : act.live())
                    if (Sh[(size_t)q * NSCAL + SC_ACTIVE] != 0.0 && !dn[q]) going.push_back(q);
                if (going.empty()) { ++j; ++done_iters; break; }
                if (going.size() <= kRestrictFraction * act.size() && j + 1 < restart && done_iters + 1 < max_iter)
                    if ((rc = use(going))) return rc;
            }
        }
        if (act.on()) {
            // the cycle end takes every active problem, done ones included
            int32_t rc = read_flags();
            if (rc) return rc;
            const std::vector<int> ending = act.active(Sh);
            if (ending != act.live() && (rc = use(ending))) return rc;
        }
        if (end_tried && !end_graphed) {
            int32_t rc = cycle_end(st);
            if (rc) return rc;
        } else if (end_tried) {
            int32_t rc = replay(g_end, st);
            if (rc) return rc;
        } else {
            int32_t rc = cycle_end(st);                       // first one eager
            if (rc) return rc;
            end_tried = true;
            end_graphed = capture(pl, g_end, cycle_end);
        }
        int32_t rc = read_flags();
        if (rc) return rc;
        const std::vector<int> left = act.active(Sh);
        if (left.empty() || done_iters >= max_iter) break;
        if (left.size() <= kRestrictFraction * act.size() && (rc = use(left))) return rc;
    }
    act.restore();
    ImgArgs io{};
    io.z = pl->x.as<double>(); io.out_op = xout;
    img_op<T>(pl, IMG_STORE_OUT, io, st);
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

// Right-preconditioned BiCGStab (van der Vorst 1992), the solver of the
// paper's experiments (Section 2.3.1, Section 4): two preconditioner
// applications and two A-pairs per iteration; every scalar lives on the
// device, so one iteration is a fixed launch sequence (a graph after its first
// run). Vectors: r = f, rh = w, p = p, v = t, s = u, t = bi_t, ph = z, sh = bi_sh.
template <class T>
static int32_t solve_bicgstab(wmg_plan *pl, bool pre, const void *b, const void *x0, void *xout, int max_iter,
                              int start, cudaStream_t st)
{
    const int64_t nN = pl->Ntot;
    int32_t rc0 = solver_pools(pl, WMG_SOLVER_BICGSTAB, pre, 0);
    if (rc0) return rc0;
    const ProbSet &ps = pl->real;
    // the work lists in use (the plan's own, or those of the problems left)
    const ProbDev *P = ps.d.as<ProbDev>();
    const int4 *vt = ps.vimg.tiles.as<int4>();
    int nv = ps.vimg.n;
    const double *S = pl->S.as<double>();
    double *hist = pl->hist.as<double>();
    const int hld = max_iter + 1;
    double *pa = pl->part_a.as<double>(), *pb = pl->part_b.as<double>();
    BicgArgs ba{};
    ba.x = pl->x.as<double>(); ba.r = pl->f.as<double>(); ba.rh = pl->w.as<double>(); ba.p = pl->p.as<double>();
    ba.v = pl->t.as<double>(); ba.s = pl->u.as<double>(); ba.t = pl->bi_t.as<double>();
    ba.ph = pl->z.as<double>(); ba.sh = pl->bi_sh.as<double>();
    ba.part_a = pa; ba.part_b = pb; ba.S = S;
    if (start == 0) {
        // r0 = W^T b - A x0, rh = r0, p = v = 0
        BpArgs fa = bp_args(BP_ATB, b, S);
        fa.out64 = ba.r; fa.part = pb;
        backproject<T>(pl, ps, fa, st);
        if (x0) {
            ImgArgs il{};
            il.in_op = x0; il.z = ba.x; il.copy_op = pl->z_op.p; il.copyT_op = pl->zT_op.p; il.S = S;
            img_op<T>(pl, IMG_LOAD, il, st);
            project<T>(pl, ps, pl->z_op.p, pl->zT_op.p, pl->sinoS.p, nullptr, S, st);
            BpArgs wa = bp_args(BP_GMRES_W, pl->sinoS.p, S);
            wa.z = ba.x; wa.out64 = ba.s;
            backproject<T>(pl, ps, wa, st);
            VecArgs rv{};
            rv.f = ba.r; rv.w = ba.s; rv.v = ba.sh; rv.part = pb; rv.S = S;
            vec_op<T>(pl, VEC_RESID64, false, rv, st);
            WMG_CUDA(cudaMemcpyAsync(ba.r, ba.sh, nN * 8, cudaMemcpyDeviceToDevice, st));
            finalize(pl, FIN_BI_INIT, ps.vimg, pb, 1, nullptr, nullptr, 0, hist, hld, st);
        } else {
            cudaMemsetAsync(pl->x.p, 0, nN * 8, st);
            finalize(pl, FIN_BI_INIT, ps.bp, pb, 1, nullptr, nullptr, 0, hist, hld, st);
        }
        launch_bicg(BI_INIT, P, vt, nv, ba, st);
    }
    // z_out = B z_in (FP64) with the operator copies of z_out; then w_out = A z_out
    auto precond_then_A = [&](double *z_in, double *z_out, double *w_out, cudaStream_t s) -> int32_t {
        if (pre) {
            bool have = false;
            int32_t rc = wmg_apply<T>(pl, z_in, z_out, false, true, false, &have, s);
            if (rc) return rc;
        } else {
            WMG_CUDA(cudaMemcpyAsync(z_out, z_in, nN * 8, cudaMemcpyDeviceToDevice, s));
            ImgArgs ic{};
            ic.z = z_out; ic.copy_op = pl->z_op.p; ic.copyT_op = pl->zT_op.p; ic.S = S;
            img_op<T>(pl, IMG_COPY64, ic, s);
        }
        project<T>(pl, ps, pl->z_op.p, pl->zT_op.p, pl->sinoS.p, nullptr, S, s);
        BpArgs wa = bp_args(BP_GMRES_W, pl->sinoS.p, S);
        wa.z = z_out; wa.out64 = w_out;
        backproject<T>(pl, ps, wa, s);
        return WMG_OK;
    };
    auto iteration = [&](cudaStream_t s) -> int32_t {
        launch_bicg(BI_P, P, vt, nv, ba, s);                           // p = r + beta (p - omega v)
        int32_t rc = precond_then_A(ba.p, ba.ph, ba.v, s);              // ph = B p, v = A ph
        if (rc) return rc;
        launch_bicg(BI_RV, P, vt, nv, ba, s);
        finalize(pl, FIN_BI_ALPHA, ps.vimg, pa, 1, nullptr, nullptr, 0, hist, hld, s);
        launch_bicg(BI_S, P, vt, nv, ba, s);                           // s = r - alpha v
        if ((rc = precond_then_A(ba.s, ba.sh, ba.t, s))) return rc;     // sh = B s, t = A sh
        launch_bicg(BI_TS, P, vt, nv, ba, s);
        finalize(pl, FIN_BI_OMEGA, ps.vimg, pa, 1, &ps.vimg, pb, 0, hist, hld, s);
        launch_bicg(BI_XR, P, vt, nv, ba, s);                          // x, r updates
        finalize(pl, FIN_BI_RES, ps.vimg, pa, 1, &ps.vimg, pb, 0, hist, hld, s);
        return WMG_OK;
    };
    // once few problems are left, the iterations run on their work lists only
    // (ActiveSet), eagerly, with the flags tested after every iteration
    ActiveSet act(pl);
    Graph graph;
    bool graphed = false;
    std::vector<double> Sh((size_t)pl->cap * NSCAL);
    for (int it = start; it < max_iter; ++it) {
        if (it == start + 1 && !act.on()) graphed = capture(pl, graph, iteration);
        int32_t rc = graphed ? replay(graph, st) : iteration(st);
        if (rc) return rc;
        if ((it + 1) % (act.on() ? 1 : 4) == 0 || it + 1 == max_iter) {
            WMG_CUDA(cudaMemcpyAsync(Sh.data(), pl->S.p, Sh.size() * 8, cudaMemcpyDeviceToHost, st));
            WMG_CUDA(cudaStreamSynchronize(st));
            const std::vector<int> left = act.active(Sh);
            if (left.empty()) break;
            if (left.size() <= kRestrictFraction * act.size() && it + 1 < max_iter) {
                bool changed = false;
                if ((rc = act.restrict_to(left, Sh, st, &changed))) return rc;
                if (changed) {
                    P = ps.d.as<ProbDev>();
                    vt = ps.vimg.tiles.as<int4>();
                    nv = ps.vimg.n;
                    graph.reset();
                    graphed = false;
                }
            }
        }
    }
    act.restore();
    ImgArgs io{};
    io.z = pl->x.as<double>(); io.out_op = xout;
    img_op<T>(pl, IMG_STORE_OUT, io, st);
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

template <class T>
static int32_t do_solve(wmg_plan *pl, int solver, bool pre, const void *b, const void *x0, void *x, int max_iter,
                        int restart, int start, cudaStream_t st)
{
    if (solver == WMG_SOLVER_CGLS) return solve_cgls<T>(pl, pre, b, x0, x, max_iter, start, st);
    if (solver == WMG_SOLVER_GMRES) return solve_gmres<T>(pl, pre, b, x0, x, max_iter, restart, start, st);
    if (solver == WMG_SOLVER_BICGSTAB) return solve_bicgstab<T>(pl, pre, b, x0, x, max_iter, start, st);
    return solve_sirt<T>(pl, b, x0, x, max_iter, start, st);
}

static int32_t check_solve_args(wmg_plan *pl, int32_t solver, int32_t preconditioned, int32_t max_iter,
                                int32_t restart)
{
    if (max_iter < 0 || solver < WMG_SOLVER_SIRT || solver > WMG_SOLVER_BICGSTAB)
        return fail(WMG_ERR_INVALID_ARG, "wmg_solve: bad arguments");
    if (solver == WMG_SOLVER_GMRES && (restart < 1 || restart > 64))
        return fail(WMG_ERR_INVALID_ARG, "wmg_solve: restart must be in [1, 64]");
    if (preconditioned && !pl->has_wmg() && solver != WMG_SOLVER_SIRT)
        return fail(WMG_ERR_INVALID_ARG, "wmg_solve: the plan has no WMG levels to precondition with");
    if (solver == WMG_SOLVER_CGLS && preconditioned &&
        (pl->opts.cycle == WMG_CYCLE_HYBRID || pl->opts.cycle == WMG_CYCLE_MULTIPLICATIVE))
        return fail(WMG_ERR_INVALID_ARG, "CGLS needs a symmetric preconditioner (ADDITIVE or SYMMETRIC cycle)");
    return WMG_OK;
}

// Statuses a solve reports for single problems (the others ran on): the
// solve's state stays a valid continuation point.
static bool problem_status(int32_t rc) { return rc == WMG_ERR_BREAKDOWN || rc == WMG_ERR_NAN; }

static int32_t run_solve(wmg_plan *pl, int32_t solver, int32_t preconditioned, const void *b, const void *x0,
                         void *x, int32_t max_iter, double rtol, int32_t restart, wmg_solve_info *info,
                         double *res_hist, cudaStream_t st)
{
    pl->state.valid = false;
    if (!pl->hist.ensure((size_t)pl->cap * (max_iter + 1) * sizeof(double)))
        return fail(WMG_ERR_OOM, "history");
    cudaMemsetAsync(pl->hist.p, 0, (size_t)pl->cap * (max_iter + 1) * sizeof(double), st);
    init_scalars(pl, rtol, max_iter, st, x0 != nullptr && solver == WMG_SOLVER_CGLS);
    int32_t rc = WMG_DISPATCH(pl, do_solve, pl, solver, preconditioned != 0, b, x0, x, max_iter, restart, 0, st);
    if (rc) return rc;
    rc = collect(pl, max_iter, info, res_hist, st);
    if ((rc >= 0 || problem_status(rc)) && !pl->batch) {
        SolveState &s = pl->state;
        s.valid = true;
        s.solver = solver; s.pre = preconditioned != 0; s.restart = solver == WMG_SOLVER_GMRES ? restart : 0;
        s.count = pl->cap; s.steps = max_iter; s.hist_ld = max_iter + 1;
    }
    return rc;
}

extern "C" int32_t wmg_solve_x0(wmg_plan *pl, int32_t solver, int32_t preconditioned, int32_t count,
                                const void *b, const void *x0, void *x, int32_t max_iter, double rtol,
                                int32_t restart, wmg_solve_info *info, double *res_hist, void *stream)
{
    if (!pl || !b || !x || count < 1) return fail(WMG_ERR_INVALID_ARG, "wmg_solve: bad arguments");
    int32_t rc = single_geometry(pl, "wmg_solve");
    if (rc) return rc;
    if ((rc = check_solve_args(pl, solver, preconditioned, max_iter, restart))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_count(pl, count, st))) return rc;
    return run_solve(pl, solver, preconditioned, b, x0, x, max_iter, rtol, restart, info, res_hist, st);
}

extern "C" int32_t wmg_solve(wmg_plan *pl, int32_t solver, int32_t preconditioned, int32_t count,
                             const void *b, void *x, int32_t max_iter, double rtol, int32_t restart,
                             wmg_solve_info *info, double *res_hist, void *stream)
{
    return wmg_solve_x0(pl, solver, preconditioned, count, b, nullptr, x, max_iter, rtol, restart, info,
                        res_hist, stream);
}

// ---------------------------------------------------------------------------
// Checkpoint / resume: the state of the last solve, copied out and back
// ---------------------------------------------------------------------------
namespace {
constexpr int kMaxRegions = 20;     // device ranges of a state (the GMRES state has 11)
struct StateHeader {
    char magic[8];
    int32_t version, solver, pre, restart, count, prec, steps, hist_ld, nregions, pad;
    uint64_t fingerprint;
    int64_t N, M;
    int64_t bytes[kMaxRegions];
};
constexpr char kStateMagic[8] = {'W', 'M', 'G', 'S', 'T', 'A', 'T', 'E'};
}  // namespace

static int64_t state_total(wmg_plan *pl)
{
    int64_t t = sizeof(StateHeader);
    for (const Region &r : state_regions(pl)) t += (int64_t)r.bytes;
    return t;
}

extern "C" int32_t wmg_state_bytes(wmg_plan *pl, int64_t *bytes)
{
    if (!pl || !bytes) return fail(WMG_ERR_INVALID_ARG, "wmg_state_bytes: bad arguments");
    if (!pl->state.valid) return fail(WMG_ERR_INVALID_ARG, "wmg_state_bytes: the plan holds no solver state");
    *bytes = state_total(pl);
    return WMG_OK;
}

extern "C" int32_t wmg_state_export(wmg_plan *pl, void *host, int64_t bytes, void *stream)
{
    if (!pl || !host) return fail(WMG_ERR_INVALID_ARG, "wmg_state_export: bad arguments");
    if (!pl->state.valid) return fail(WMG_ERR_INVALID_ARG, "wmg_state_export: the plan holds no solver state");
    const std::vector<Region> regs = state_regions(pl);
    if (bytes < state_total(pl) || regs.size() > (size_t)kMaxRegions)
        return fail(WMG_ERR_INVALID_ARG, "wmg_state_export: buffer smaller than wmg_state_bytes");
    const SolveState &s = pl->state;
    StateHeader h{};
    std::memcpy(h.magic, kStateMagic, 8);
    h.version = 1; h.solver = s.solver; h.pre = s.pre; h.restart = s.restart; h.count = s.count;
    h.prec = pl->prec; h.steps = s.steps; h.hist_ld = s.hist_ld; h.nregions = (int)regs.size();
    h.fingerprint = pl->fingerprint; h.N = pl->Ntot; h.M = pl->Mtot;
    for (size_t k = 0; k < regs.size(); ++k) h.bytes[k] = (int64_t)regs[k].bytes;
    char *out = static_cast<char *>(host);
    std::memcpy(out, &h, sizeof h);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    size_t off = sizeof h;
    for (const Region &r : regs) {
        WMG_CUDA(cudaMemcpyAsync(out + off, r.p, r.bytes, cudaMemcpyDeviceToHost, st));
        off += r.bytes;
    }
    WMG_CUDA(cudaStreamSynchronize(st));
    return WMG_OK;
}

extern "C" int32_t wmg_state_import(wmg_plan *pl, const void *host, int64_t bytes, void *stream)
{
    if (!pl || !host || bytes < (int64_t)sizeof(StateHeader))
        return fail(WMG_ERR_INVALID_ARG, "wmg_state_import: bad arguments");
    int32_t rc = single_geometry(pl, "wmg_state_import");
    if (rc) return rc;
    pl->state.valid = false;
    StateHeader h;
    std::memcpy(&h, host, sizeof h);
    if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != 1)
        return fail(WMG_ERR_INVALID_ARG, "wmg_state_import: not a solver state");
    if (h.fingerprint != pl->fingerprint || h.prec != pl->prec)
        return fail(WMG_ERR_INVALID_ARG, "wmg_state_import: the state belongs to another geometry or options");
    if (h.count < 1 || h.steps < 0 || h.hist_ld != h.steps + 1 || h.nregions < 1 || h.nregions > kMaxRegions)
        return fail(WMG_ERR_INVALID_ARG, "wmg_state_import: corrupt header");
    if ((rc = check_solve_args(pl, h.solver, h.pre, h.steps, h.solver == WMG_SOLVER_GMRES ? h.restart : 1)))
        return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_count(pl, h.count, st))) return rc;
    if (h.N != pl->Ntot || h.M != pl->Mtot)
        return fail(WMG_ERR_INVALID_ARG, "wmg_state_import: problem sizes differ");
    if ((rc = solver_pools(pl, h.solver, h.pre != 0, h.restart))) return rc;
    if (!pl->hist.ensure((size_t)h.count * h.hist_ld * sizeof(double))) return fail(WMG_ERR_OOM, "history");
    SolveState s;
    s.solver = h.solver; s.pre = h.pre != 0; s.restart = h.restart; s.count = h.count;
    s.steps = h.steps; s.hist_ld = h.hist_ld;
    pl->state = s;
    const std::vector<Region> regs = state_regions(pl);
    int64_t need = sizeof h;
    bool same = (int)regs.size() == h.nregions;
    for (size_t k = 0; same && k < regs.size(); ++k) {
        same = h.bytes[k] == (int64_t)regs[k].bytes;
        need += h.bytes[k];
    }
    if (!same || bytes < need) {
        pl->state.valid = false;
        return fail(WMG_ERR_INVALID_ARG, "wmg_state_import: sizes do not match the plan");
    }
    const char *in = static_cast<const char *>(host);
    size_t off = sizeof h;
    for (const Region &r : regs) {
        WMG_CUDA(cudaMemcpyAsync(r.p, in + off, r.bytes, cudaMemcpyHostToDevice, st));
        off += r.bytes;
    }
    WMG_CUDA(cudaStreamSynchronize(st));
    pl->state.valid = true;
    return WMG_OK;
}

template <class T>
static int32_t store_x(wmg_plan *pl, void *x, cudaStream_t st)
{
    ImgArgs io{};
    io.z = pl->x.as<double>(); io.out_op = x;
    img_op<T>(pl, IMG_STORE_OUT, io, st);
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}

extern "C" int32_t wmg_solve_resume(wmg_plan *pl, int32_t count, const void *b, void *x, int32_t max_iter,
                                    double rtol, wmg_solve_info *info, double *res_hist, void *stream)
{
    if (!pl || !b || !x || max_iter < 0) return fail(WMG_ERR_INVALID_ARG, "wmg_solve_resume: bad arguments");
    if (!pl->state.valid) return fail(WMG_ERR_INVALID_ARG, "wmg_solve_resume: the plan holds no solver state");
    if (count != pl->state.count || count != pl->cap)
        return fail(WMG_ERR_INVALID_ARG, "wmg_solve_resume: count differs from the state's problem count");
    const SolveState s0 = pl->state;
    if (max_iter < s0.steps)
        return fail(WMG_ERR_INVALID_ARG, "wmg_solve_resume: max_iter is below the iterations already done");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // histories: the entries so far, in rows of the new length
    const int new_ld = max_iter + 1;
    {
        std::vector<double> H0((size_t)count * s0.hist_ld), H1((size_t)count * new_ld, 0.0);
        WMG_CUDA(cudaMemcpyAsync(H0.data(), pl->hist.p, H0.size() * 8, cudaMemcpyDeviceToHost, st));
        WMG_CUDA(cudaStreamSynchronize(st));
        for (int q = 0; q < count; ++q)
            std::memcpy(&H1[(size_t)q * new_ld], &H0[(size_t)q * s0.hist_ld], (size_t)s0.hist_ld * 8);
        if (!pl->hist.ensure(H1.size() * 8)) {
            pl->state.valid = false;
            return fail(WMG_ERR_OOM, "history");
        }
        WMG_CUDA(cudaMemcpyAsync(pl->hist.p, H1.data(), H1.size() * 8, cudaMemcpyHostToDevice, st));
    }
    pl->state.hist_ld = new_ld;
    int32_t rc;
    if (max_iter > s0.steps) {
        // problems that stopped at the old iteration cap run on (SIRT: every
        // problem, it runs a fixed count); converged or failed ones stay
        std::vector<double> S((size_t)count * NSCAL);
        WMG_CUDA(cudaMemcpyAsync(S.data(), pl->S.p, S.size() * 8, cudaMemcpyDeviceToHost, st));
        WMG_CUDA(cudaStreamSynchronize(st));
        for (int q = 0; q < count; ++q) {
            double *v = &S[(size_t)q * NSCAL];
            const int status = (int)v[SC_STATUS];
            bool run = status == WMG_NOT_CONVERGED;
            if (s0.solver == WMG_SOLVER_SIRT) run = status != WMG_ERR_NAN;
            if (run && s0.solver == WMG_SOLVER_BICGSTAB && v[SC_GNEW] != 0.0) {
                v[SC_STATUS] = WMG_ERR_BREAKDOWN;     // the capped step had broken down
                run = false;
            }
            if (run) { v[SC_ACTIVE] = 1.0; v[SC_STATUS] = WMG_NOT_CONVERGED; }
            v[SC_RTOL] = rtol;
            v[SC_MAXIT] = max_iter;
        }
        WMG_CUDA(cudaMemcpyAsync(pl->S.p, S.data(), S.size() * 8, cudaMemcpyHostToDevice, st));
        pl->state.valid = false;
        rc = WMG_DISPATCH(pl, do_solve, pl, s0.solver, s0.pre != 0, b, nullptr, x, max_iter, s0.restart,
                          s0.steps, st);
        if (rc) return rc;
        pl->state = s0;
        pl->state.steps = max_iter;
        pl->state.hist_ld = new_ld;
    } else {
        rc = WMG_DISPATCH(pl, store_x, pl, x, st);
        if (rc) return rc;
    }
    rc = collect(pl, max_iter, info, res_hist, st);
    if (rc < 0 && !problem_status(rc)) pl->state.valid = false;
    return rc;
}

// ---------------------------------------------------------------------------
// Batches of problems with different geometries
// ---------------------------------------------------------------------------
struct wmg_batch {
    wmg_plan *plan = nullptr;
};

static bool same_geometry(const wmg_geom &a, const wmg_geom &b, const wmg_opts &oa, const wmg_opts &ob)
{
    if (a.n != b.n || a.m != b.m || a.D != b.D || a.det_spacing != b.det_spacing || a.det_offset != b.det_offset ||
        a.kernel != b.kernel || oa.levels != ob.levels || oa.lambda != ob.lambda)
        return false;
    if ((a.angles == nullptr) != (b.angles == nullptr)) return false;
    if (a.angles && std::memcmp(a.angles, b.angles, a.m * sizeof(double)) != 0) return false;
    return true;
}

extern "C" int32_t wmg_batch_create(const wmg_geom *gs, const wmg_opts *os, int32_t count, void *stream,
                                    wmg_batch **out)
{
    if (!out) return fail(WMG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!gs || !os || count < 1) return fail(WMG_ERR_INVALID_ARG, "wmg_batch_create: bad arguments");
    if (os[0].precision == WMG_PREC_F32_BF16STORE)
        return fail(WMG_ERR_INVALID_ARG, "wmg_batch_create: BF16 operator storage is for plans only");
    for (int i = 0; i < count; ++i) {
        int32_t rc = validate(&gs[i], &os[i]);
        if (rc) return rc;
        const wmg_opts &a = os[0], &b = os[i];
        if (a.nu1 != b.nu1 || a.nu2 != b.nu2 || a.cycle != b.cycle || a.hybrid_depth != b.hybrid_depth ||
            a.precision != b.precision || a.omega != b.omega || (a.levels >= 1) != (b.levels >= 1))
            return fail(WMG_ERR_INVALID_ARG,
                        "wmg_batch_create: problems must share nu1, nu2, omega, cycle, hybrid depth and precision");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto pl = std::make_unique<wmg_plan>();
    pl->prec = os[0].precision;
    pl->esz = pl->prec == WMG_PREC_F64 ? 8 : 4;
    pl->opts = os[0];
    if (pl->opts.omega <= 0) pl->opts.omega = 1.0;
    pl->batch = true;
    // distinct geometries (first occurrence order), each set up once
    std::vector<int> gid(count, -1), first;
    for (int i = 0; i < count; ++i) {
        for (size_t u = 0; u < first.size(); ++u)
            if (same_geometry(gs[i], gs[first[u]], os[i], os[first[u]])) { gid[i] = (int)u; break; }
        if (gid[i] < 0) { gid[i] = (int)first.size(); first.push_back(i); }
    }
    int32_t rc;
    for (size_t u = 0; u < first.size(); ++u) {
        pl->geos.push_back(std::make_unique<Geo>());
        if ((rc = make_geo(&gs[first[u]], &os[first[u]], *pl->geos.back(), st))) return rc;
    }
    if ((rc = upload_geoms(pl.get(), st))) return rc;
    for (size_t u = 0; u < first.size(); ++u) {
        rc = pl->prec == WMG_PREC_F64 ? setup_geometry<double>(pl.get(), (int)u, st)
                                      : setup_geometry<float>(pl.get(), (int)u, st);
        if (rc) return rc;
    }
    // slots grouped by geometry; order[i] = slot of problem i
    std::vector<int> idx(count);
    for (int i = 0; i < count; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return gid[a] < gid[b]; });
    pl->order.assign(count, 0);
    pl->pgeo.assign(count, 0);
    for (int q = 0; q < count; ++q) {
        pl->order[idx[q]] = q;
        pl->pgeo[q] = gid[idx[q]];
    }
    if ((rc = set_slots(pl.get(), st))) return rc;
    rc = pl->prec == WMG_PREC_F64 ? autotune<double>(pl.get(), pl->real, st) : autotune<float>(pl.get(), pl->real, st);
    if (rc) return rc;
    WMG_CUDA(cudaStreamSynchronize(st));
    auto bt = std::make_unique<wmg_batch>();
    bt->plan = pl.release();
    *out = bt.release();
    return WMG_OK;
}

extern "C" int32_t wmg_batch_destroy(wmg_batch *batch)
{
    if (!batch) return WMG_OK;
    wmg_plan_destroy(batch->plan);
    delete batch;
    return WMG_OK;
}

extern "C" int32_t wmg_batch_sizes(const wmg_batch *batch, int32_t i, int64_t *N, int64_t *M)
{
    if (!batch || i < 0 || i >= batch->plan->cap) return fail(WMG_ERR_INVALID_ARG, "wmg_batch_sizes: bad arguments");
    const Geo &G = batch->plan->geo(batch->plan->order[i]);
    if (N) *N = G.N;
    if (M) *M = G.M;
    return WMG_OK;
}

// copy kernels between the caller's per-problem buffers and the slot pools
template <class T>
static int32_t gather_scatter(wmg_plan *pl, const void *const *src, void *const *dst, bool to_pool, void *pool,
                              bool image, cudaStream_t st)
{
    for (int i = 0; i < pl->cap; ++i) {
        const int q = pl->order[i];
        const Geo &G = pl->geo(q);
        const int64_t off = image ? pl->img_off[q] : pl->sino_off[q];
        const size_t bytes = (size_t)(image ? G.N : G.M) * sizeof(T);
        char *pp = static_cast<char *>(pool) + off * sizeof(T);
        if (to_pool) WMG_CUDA(cudaMemcpyAsync(pp, src[i], bytes, cudaMemcpyDeviceToDevice, st));
        else WMG_CUDA(cudaMemcpyAsync(dst[i], pp, bytes, cudaMemcpyDeviceToDevice, st));
    }
    return WMG_OK;
}

extern "C" int32_t wmg_batch_solve(wmg_batch *batch, int32_t solver, int32_t preconditioned, const void *const *b,
                                   void *const *x, int32_t max_iter, double rtol, int32_t restart,
                                   wmg_solve_info *info, double *res_hist, void *stream)
{
    if (!batch || !b || !x) return fail(WMG_ERR_INVALID_ARG, "wmg_batch_solve: bad arguments");
    wmg_plan *pl = batch->plan;
    for (int i = 0; i < pl->cap; ++i)
        if (!b[i] || !x[i]) return fail(WMG_ERR_INVALID_ARG, "wmg_batch_solve: NULL problem buffer");
    int32_t rc = check_solve_args(pl, solver, preconditioned, max_iter, restart);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!ensure_pool(pl->b_op, pl->Mtot, pl->esz) || !ensure_pool(pl->x_io, pl->Ntot, pl->esz))
        return fail(WMG_ERR_OOM, "batch input pools");
    rc = pl->prec == WMG_PREC_F64 ? gather_scatter<double>(pl, b, nullptr, true, pl->b_op.p, false, st)
                                  : gather_scatter<float>(pl, b, nullptr, true, pl->b_op.p, false, st);
    if (rc) return rc;
    rc = run_solve(pl, solver, preconditioned, pl->b_op.p, nullptr, pl->x_io.p, max_iter, rtol, restart, info, res_hist,
                   st);
    if (rc < 0) return rc;
    const int32_t rc2 = pl->prec == WMG_PREC_F64 ? gather_scatter<double>(pl, nullptr, x, false, pl->x_io.p, true, st)
                                                 : gather_scatter<float>(pl, nullptr, x, false, pl->x_io.p, true, st);
    if (rc2) return rc2;
    WMG_CUDA(cudaStreamSynchronize(st));
    return rc;
}
