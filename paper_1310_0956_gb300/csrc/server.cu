// server.cu -- continuous-batching reconstruction server behind the
// wmg_server_* calls of include/wmgct.h.
//
// Requests (independent problems of any geometry, each solved by restarted
// GMRES with right WMG preconditioning, Section 3.1 with the Krylov solver of
// Section 2.3) wait in a FIFO queue until a slot and device memory free up.
// An admitted request owns a slot: ranges of the image and sinogram pools
// that hold its whole solver state (x, f = W^T b, the Arnoldi basis, the
// Hessenberg/Givens data) for as long as it runs. Every tick runs one GMRES
// step for all slots together, each slot at its own position:
//
//   INIT  f = W^T b, beta = |f|, v_0 = f / beta                  (admitted)
//   ARN   u = B v_j, w = A u, two classical Gram-Schmidt passes, Givens
//   END   y = H^-1 g, u = B (V y), x += u, w = A x, r = f - w, v_0 = r / |r|
//
// All slots share the preconditioner application and the A-pair of a tick
// (one launch each over every slot's tiles); the phase-specific scalar steps
// run with the other slots held inactive. Every reduction is per slot with a
// fixed order, so a request's arithmetic does not depend on what else runs:
// it gives the same x alone, in any mix, and through wmg_solve.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "engine.cuh"
#include "range_alloc.h"

namespace wmg {

enum SrvPhase : int { PH_EMPTY = -1, PH_INIT = 0, PH_ARN = 1, PH_END = 2 };

// Hold (release = 0) or restore (release = 1) SC_ACTIVE of every slot whose
// phase is not `want`, so that the kernels of one phase group see only their
// own slots. Releasing the INIT group moves its slots to ARN.
__global__ void k_srv_hold(double *S, int *phase, int cap, int want, int release)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= cap) return;
    const int ph = phase[p];
    if (ph == want) {
        if (release && want == PH_INIT) phase[p] = PH_ARN;
        return;
    }
    double *s = S + (int64_t)p * NSCAL;
    if (!release) {
        s[SC_HELD] = s[SC_ACTIVE];
        s[SC_ACTIVE] = 0.0;
    } else {
        s[SC_ACTIVE] = s[SC_HELD];
    }
}

// ARN slots: t = v_j with j = jn[slot] (the preconditioner input of the step).
__global__ void __launch_bounds__(256)
k_srv_gather(const ProbDev *__restrict__ P, const int4 *__restrict__ tiles, int ntiles,
             const double *__restrict__ V, int64_t vstride, const int *__restrict__ jn,
             const int *__restrict__ phase, double *__restrict__ t, const double *__restrict__ S)
{
    for (int q = blockIdx.x; q < ntiles; q += gridDim.x) {
        const int4 tl = tiles[q];
        const ProbDev pd = P[tl.x];
        if (phase[pd.slot] != PH_ARN || !slot_active(S, pd.slot)) continue;
        const double *Vj = V + (int64_t)jn[pd.slot] * vstride + pd.img;
        for (int e = threadIdx.x; e < tl.z; e += blockDim.x) {
            const int64_t o = tl.y + e;
            t[pd.img + o] = Vj[o];
        }
    }
}

// END slots: x += u, then u = x (the input of the true-residual product).
__global__ void __launch_bounds__(256)
k_srv_end_update(const ProbDev *__restrict__ P, const int4 *__restrict__ tiles, int ntiles,
                 const int *__restrict__ phase, double *__restrict__ x, double *__restrict__ u,
                 const double *__restrict__ S)
{
    for (int q = blockIdx.x; q < ntiles; q += gridDim.x) {
        const int4 tl = tiles[q];
        const ProbDev pd = P[tl.x];
        if (phase[pd.slot] != PH_END || !slot_active(S, pd.slot)) continue;
        for (int e = threadIdx.x; e < tl.z; e += blockDim.x) {
            const int64_t j = pd.img + tl.y + e;
            const double v = x[j] + u[j];
            x[j] = v;
            u[j] = v;
        }
    }
}

// Scalars of a newly admitted slot.
__global__ void k_srv_admit(double *S, double *lam, int slot, double rtol, int max_iter, double lambda)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double *s = S + (int64_t)slot * NSCAL;
    for (int i = 0; i < NSCAL; ++i) s[i] = 0.0;
    s[SC_ACTIVE] = 1.0;
    s[SC_STATUS] = WMG_NOT_CONVERGED;
    s[SC_RTOL] = rtol;
    s[SC_MAXIT] = max_iter;
    lam[slot] = lambda;
}

// Retirement: the caller's image = (T) x.
template <class T>
__global__ void k_srv_store(const double *__restrict__ x, T *__restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)x[i];
}

}  // namespace wmg

using namespace wmg;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    wmg_geom g{};
    std::vector<double> angles;
    wmg_opts o{};
    std::string key;
    const void *b = nullptr;
    void *x = nullptr;
    int state = WMG_REQ_QUEUED;
    int slot = -1, gi = -1;
    int64_t N = 0, M = 0, ioff = -1, soff = -1;
    wmg_solve_info info{};
    std::vector<double> hist;
    Clock::time_point t_submit, t_admit, t_done;
};

struct GeoEntry {
    std::string key;
    int refs = 0;
    uint64_t last_use = 0;
    int64_t bytes = 0;
};

// A geometry setup run by the worker thread on its own stream.
struct SetupJob {
    std::string key;
    wmg_geom g{};
    std::vector<double> angles;
    wmg_opts o{};
    int64_t bytes = 0, transient = 0;
    std::unique_ptr<Geo> geo;
    int32_t rc = WMG_OK;
};

// Geometry setups (leaf Gram assembly and inverses) run on kSetupThreads
// worker threads, each with a stream of its own, overlapping one another and
// the ticks of the requests already admitted. Each setup builds a
// one-geometry plan on its thread's stream and hands the geometry over.
constexpr int kSetupThreads = 3;

struct SetupWorker {
    std::thread th[kSetupThreads];
    cudaStream_t sts[kSetupThreads] = {};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<SetupJob>> todo;
    std::vector<std::shared_ptr<SetupJob>> done;
    bool stop = false;
    int device = 0;

    void start()
    {
        cudaGetDevice(&device);
        for (int i = 0; i < kSetupThreads; ++i) {
            cudaStreamCreateWithFlags(&sts[i], cudaStreamNonBlocking);
            th[i] = std::thread([this, i] { run(sts[i]); });
        }
    }
    void run(cudaStream_t st)
    {
        cudaSetDevice(device);
        g_alloc_stream = st;           // temporaries of the setups: stream-ordered
        for (;;) {
            std::shared_ptr<SetupJob> job;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || !todo.empty(); });
                if (stop) return;
                job = todo.front();
                todo.pop_front();
            }
            wmg_geom g = job->g;
            g.angles = job->angles.empty() ? nullptr : job->angles.data();
            wmg_plan *tmp = nullptr;
            job->rc = wmg_plan_create(&g, &job->o, st, &tmp);
            if (job->rc == WMG_OK) {
                job->geo = std::move(tmp->geos[0]);
                cudaStreamSynchronize(st);
                delete tmp;
            }
            std::lock_guard<std::mutex> lk(mu);
            done.push_back(job);
        }
    }
    void submit(std::shared_ptr<SetupJob> job)
    {
        std::lock_guard<std::mutex> lk(mu);
        todo.push_back(std::move(job));
        cv.notify_one();
    }
    std::vector<std::shared_ptr<SetupJob>> take_done()
    {
        std::lock_guard<std::mutex> lk(mu);
        std::vector<std::shared_ptr<SetupJob>> out;
        out.swap(done);
        return out;
    }
    void shutdown()
    {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
            cv.notify_all();
        }
        for (int i = 0; i < kSetupThreads; ++i) {
            if (th[i].joinable()) th[i].join();
            if (sts[i]) {
                cudaStreamSynchronize(sts[i]);
                cudaStreamDestroy(sts[i]);
            }
            sts[i] = nullptr;
        }
    }
};

constexpr int kMaxSetupsInFlight = kSetupThreads + 1;

}  // namespace

struct wmg_server {
    wmg_server_config cfg{};
    cudaStream_t st = nullptr;
    std::unique_ptr<wmg_plan> pl;
    int ldp = 0, hld = 0, band_mult = 1;
    int64_t bpi = 0, bps = 0;            // state bytes per pool element (image / sinogram)
    int64_t geo_budget = 0, geo_used = 0;
    RangeAlloc img, sino;
    std::vector<int> phase;              // host copy of every slot's phase
    std::vector<uint64_t> slot_req;
    DevBuf d_phase;
    int *h_phase = nullptr, *h_jn = nullptr, *h_done = nullptr;
    double *h_S = nullptr, *h_hist = nullptr;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Request> reqs;
    uint64_t next_id = 1, use_clock = 0;
    std::vector<GeoEntry> geo_entries;   // by geometry index of the plan
    std::map<std::string, int> geo_by_key;
    std::map<std::string, std::shared_ptr<SetupJob>> in_setup;   // running or waiting setups
    std::map<std::string, int32_t> failed;                       // geometries whose setup failed
    SetupWorker worker;
    bool dirty = false;
    wmg_server_counters stats{};
    ~wmg_server()
    {
        worker.shutdown();
        if (st) cudaStreamSynchronize(st);
        if (h_phase) cudaFreeHost(h_phase);
        if (h_jn) cudaFreeHost(h_jn);
        if (h_done) cudaFreeHost(h_done);
        if (h_S) cudaFreeHost(h_S);
        if (h_hist) cudaFreeHost(h_hist);
    }
};

namespace {

std::string geo_key(const wmg_geom &g, const wmg_opts &o)
{
    std::string k;
    auto put = [&](const void *p, size_t n) { k.append(static_cast<const char *>(p), n); };
    put(&g.n, 4); put(&g.m, 4); put(&g.D, 4); put(&g.det_spacing, 8); put(&g.det_offset, 8); put(&g.kernel, 4);
    put(&o.levels, 4); put(&o.lambda, 8); put(&o.hybrid_depth, 4);
    const char has = g.angles ? 1 : 0;
    put(&has, 1);
    if (g.angles) put(g.angles, (size_t)g.m * sizeof(double));
    return k;
}

// Device bytes of a geometry's setup (trig tables, D~^-1, SIRT scalings,
// leaf inverses), as allocated by make_geo and setup_geometry.
int64_t geo_bytes(const wmg_geom &g, const wmg_opts &o, size_t esz)
{
    const int64_t N = (int64_t)g.n * g.n, M = (int64_t)g.m * g.D;
    int64_t b = (int64_t)g.m * (sizeof(double2) + sizeof(float2) + sizeof(float4) + sizeof(AngleF));
    b += (2 * N + M) * (int64_t)esz;
    if (o.levels >= 1) {
        const int L = o.levels - 1;
        const int64_t nc = g.n >> L, P = nc * nc, K = (int64_t)1 << (2 * L);
        b += K * P * P * (int64_t)esz;                     // leaf inverses in the plan precision
    }
    return b;
}

// Device bytes a geometry setup holds only while it runs, as allocated by
// setup_geometry and build_leaf_inverses: the all-ones and product vectors,
// the pair sums D (K P^2 doubles), the per-CTA Cholesky work matrices, and
// the profile / footprint buffers of one angle chunk.
int64_t setup_transient_bytes(const wmg_geom &g, const wmg_opts &o, size_t esz)
{
    const int64_t N = (int64_t)g.n * g.n, M = (int64_t)g.m * g.D;
    int64_t b = 2 * (N + M) * (int64_t)esz + (64 << 10);
    if (o.levels >= 1) {
        const int L = o.levels - 1;
        const int64_t nc = g.n >> L, P = nc * nc, K = (int64_t)1 << (2 * L), B = (int64_t)1 << L;
        int sms = 148, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const double dt = g.det_spacing > 0 ? g.det_spacing : 1.0;
        const int64_t R = (int64_t)std::floor((double)B * 1.4142135623730951 / dt) + 4;
        const int64_t KT = std::min<int64_t>(K, 256);
        const double per_angle = (double)P * R * KT * esz;
        const int64_t chunk = (int64_t)std::max(1.0, std::min((double)g.m, 96.0 * 1024 * 1024 / per_angle));
        b += K * P * P * 8 + 2 * std::min<int64_t>(K, 4 * sms) * P * P * 8 + K * 4;
        b += chunk * P * R * KT * (int64_t)esz + chunk * P * R * B * 2 * ((int64_t)esz + 1) + chunk * P * 8 +
             (int64_t)g.m * 4;
    }
    return b;
}

int64_t state_bytes(const wmg_server *s, int64_t N, int64_t M)
{
    return RangeAlloc::round(N) * s->bpi + RangeAlloc::round(M) * s->bps;
}

int free_slot(const wmg_server *s)
{
    for (int q = 0; q < (int)s->phase.size(); ++q)
        if (s->phase[q] == PH_EMPTY) return q;
    return -1;
}

// Evict unused geometries (least recently used first; none that a queued
// request waits for) until `need` more bytes fit in the geometry budget.
bool make_room(wmg_server *s, int64_t need, const std::map<std::string, int> &wanted)
{
    while (s->geo_used + need > s->geo_budget) {
        int victim = -1;
        for (int gi = 0; gi < (int)s->geo_entries.size(); ++gi) {
            const GeoEntry &e = s->geo_entries[gi];
            if (!s->pl->geos[gi] || e.refs > 0 || wanted.count(e.key)) continue;
            if (victim < 0 || e.last_use < s->geo_entries[victim].last_use) victim = gi;
        }
        if (victim < 0) return false;
        s->geo_used -= s->geo_entries[victim].bytes;
        s->geo_by_key.erase(s->geo_entries[victim].key);
        s->pl->geos[victim].reset();
        s->geo_entries[victim] = GeoEntry{};
        s->stats.geometries_evicted++;
    }
    return true;
}

// Finished background setups: install their geometries (or record the
// failure for the requests that wait for them).
int32_t collect_setups(wmg_server *s)
{
    wmg_plan *pl = s->pl.get();
    bool installed = false;
    for (auto &job : s->worker.take_done()) {
        s->in_setup.erase(job->key);
        s->geo_used -= job->transient;
        if (job->rc != WMG_OK || !job->geo) {
            s->geo_used -= job->bytes;
            s->failed[job->key] = job->rc != WMG_OK ? job->rc : WMG_ERR_CUDA;
            continue;
        }
        int gi = -1;
        for (int i = 0; i < (int)pl->geos.size(); ++i)
            if (!pl->geos[i]) { gi = i; break; }
        if (gi < 0) {
            gi = (int)pl->geos.size();
            pl->geos.emplace_back();
            s->geo_entries.emplace_back();
        }
        pl->geos[gi] = std::move(job->geo);
        s->geo_entries[gi] = GeoEntry{job->key, 0, ++s->use_clock, job->bytes};
        s->geo_by_key[job->key] = gi;
        s->stats.geometry_setups++;
        installed = true;
    }
    if (installed) return upload_geoms(pl, s->st);
    return WMG_OK;
}

// Start the setup of request r's geometry on the worker if memory allows.
bool start_setup(wmg_server *s, const Request &r, const std::map<std::string, int> &wanted)
{
    if ((int)s->in_setup.size() >= kMaxSetupsInFlight) return false;
    auto job = std::make_shared<SetupJob>();
    job->key = r.key;
    job->g = r.g;
    job->angles = r.angles;
    job->o = r.o;
    job->bytes = geo_bytes(r.g, r.o, s->pl->esz);
    job->transient = setup_transient_bytes(r.g, r.o, s->pl->esz);
    if (!make_room(s, job->bytes + job->transient, wanted)) return false;
    s->geo_used += job->bytes + job->transient;
    s->in_setup[r.key] = job;
    s->worker.submit(job);
    return true;
}

void finish(wmg_server *s, Request &r, int status)
{
    r.state = WMG_REQ_DONE;
    r.info.status = status;
    r.t_done = Clock::now();
    s->stats.completed++;
}

// Admit queued requests in arrival order while slots and memory are free. A
// request whose geometry is not set up yet starts that setup in the
// background (at most kMaxSetupsInFlight at a time) and waits; requests
// behind it whose geometries are ready may pass it.
int32_t admit(wmg_server *s)
{
    wmg_plan *pl = s->pl.get();
    int32_t rc = collect_setups(s);
    if (rc) return rc;
    std::map<std::string, int> wanted;
    for (uint64_t id : s->queue) wanted[s->reqs[id].key]++;
    std::deque<uint64_t> keep;
    while (!s->queue.empty()) {
        const uint64_t id = s->queue.front();
        s->queue.pop_front();
        Request &r = s->reqs[id];
        auto fk = s->failed.find(r.key);
        if (fk != s->failed.end()) {                       // setup failed: the request ends with that status
            finish(s, r, fk->second);
            continue;
        }
        auto gk = s->geo_by_key.find(r.key);
        const int slot = free_slot(s);
        if (gk == s->geo_by_key.end() || slot < 0) {
            if (gk == s->geo_by_key.end() && !s->in_setup.count(r.key)) start_setup(s, r, wanted);
            keep.push_back(id);
            continue;
        }
        const int gi = gk->second;
        const int64_t io = s->img.alloc(r.N);
        const int64_t so = io < 0 ? -1 : s->sino.alloc(r.M);
        if (so < 0) {
            if (io >= 0) s->img.release(io, r.N);
            keep.push_back(id);
            continue;
        }
        GeoEntry &e = s->geo_entries[gi];
        e.refs++;
        e.last_use = ++s->use_clock;
        r.gi = gi; r.slot = slot; r.ioff = io; r.soff = so;
        r.state = WMG_REQ_RUNNING;
        r.t_admit = Clock::now();
        s->slot_req[slot] = r.id;
        s->phase[slot] = PH_INIT;
        pl->pgeo[slot] = gi;
        pl->img_off[slot] = io;
        pl->sino_off[slot] = so;
        s->dirty = true;
        s->stats.admitted++;
        // resident state of the slot: x = 0, H = 0, history = 0, b copied in
        const cudaStream_t st = s->st;
        const Geo &G = *pl->geos[gi];
        WMG_CUDA(cudaMemcpyAsync(static_cast<char *>(pl->b_op.p) + so * pl->esz, r.b, r.M * pl->esz,
                                 cudaMemcpyDeviceToDevice, st));
        WMG_CUDA(cudaMemsetAsync(pl->x.as<double>() + io, 0, r.N * sizeof(double), st));
        WMG_CUDA(cudaMemsetAsync(pl->H.as<double>() + (int64_t)slot * s->ldp * s->cfg.restart, 0,
                                 (size_t)s->ldp * s->cfg.restart * sizeof(double), st));
        WMG_CUDA(cudaMemsetAsync(pl->hist.as<double>() + (int64_t)slot * s->hld, 0, s->hld * sizeof(double), st));
        count_launches(1);
        k_srv_admit<<<1, 32, 0, st>>>(pl->S.as<double>(), pl->lam.as<double>(), slot, s->cfg.rtol,
                                      s->cfg.max_iter, G.g.lambda);
    }
    s->queue.swap(keep);
    return WMG_OK;
}

// Rebuild the slot table and work lists after admissions or retirements.
int32_t relayout(wmg_server *s)
{
    wmg_plan *pl = s->pl.get();
    ProbSet &ps = pl->real;
    pl->live.clear();
    for (int q = 0; q < pl->cap; ++q) {
        ProbDev &d = ps.h[q];
        d = ProbDev{};
        d.slot = q;
        d.geom = -1;
        if (s->phase[q] == PH_EMPTY) continue;
        pl->live.push_back(q);
        const Geo &G = pl->geo(q);
        d.geom = pl->pgeo[q];
        d.img = pl->img_off[q];
        d.sino = pl->sino_off[q];
        d.coef = pl->img_off[q];
        d.kin0 = 0; d.kin1 = G.g.K; d.kout0 = 0; d.kout1 = G.g.K;
    }
    build_tiles(pl, ps);
    if (!upload_set(ps, s->st)) return fail(WMG_ERR_OOM, "server work lists");
    pl->bands.clear();
    pl->leafsets.clear();
    pl->segsets.clear();
    if (!ensure_partials(pl, s->ldp)) return fail(WMG_ERR_OOM, "server partials");
    s->dirty = false;
    return WMG_OK;
}

void hold(wmg_server *s, int want, int release)
{
    count_launches(1);
    k_srv_hold<<<(s->pl->cap + 127) / 128, 128, 0, s->st>>>(s->pl->S.as<double>(), s->d_phase.as<int>(), s->pl->cap,
                                                          want, release);
}

// One GMRES step for every slot (see the top of this file).
template <class T>
int32_t tick(wmg_server *s)
{
    wmg_plan *pl = s->pl.get();
    const cudaStream_t st = s->st;
    const ProbSet &ps = pl->real;
    const ProbDev *P = ps.d.as<ProbDev>();
    const int4 *vt = ps.vimg.tiles.as<int4>();
    const int nv = ps.vimg.n;
    const int ldp = s->ldp;
    const int64_t vstride = pl->Ntot;
    double *S = pl->S.as<double>();
    double *pa = pl->part_a.as<double>(), *pb = pl->part_b.as<double>();
    double *V = pl->V.as<double>();
    bool any_init = false, any_arn = false, any_end = false;
    int jmax = 0;
    for (int q : pl->live) {
        any_init |= s->phase[q] == PH_INIT;
        any_end |= s->phase[q] == PH_END;
        if (s->phase[q] == PH_ARN) { any_arn = true; jmax = std::max(jmax, s->h_jn[q]); }
    }
    std::memcpy(s->h_phase, s->phase.data(), pl->cap * sizeof(int));
    WMG_CUDA(cudaMemcpyAsync(s->d_phase.p, s->h_phase, pl->cap * sizeof(int), cudaMemcpyHostToDevice, st));
    GmArgs ga{};
    ga.nprob = pl->cap; ga.restart = s->cfg.restart; ga.ldp = ldp;
    ga.S = S; ga.H = pl->H.as<double>(); ga.cs = pl->gcs.as<double>(); ga.sn = pl->gsn.as<double>();
    ga.g = pl->gg.as<double>(); ga.y = pl->gy.as<double>(); ga.h1 = pl->h1.as<double>();
    ga.h2 = pl->h2.as<double>(); ga.jn = pl->jn.as<int>(); ga.done = pl->done.as<int>();
    ga.skip = pl->reo.as<int>();
    ga.hist = pl->hist.as<double>(); ga.hist_ld = s->hld;
    // INIT: f = W^T b, beta = |f|, v_0 = f / beta; the slots join ARN at j = 0
    if (any_init) {
        hold(s, PH_INIT, 0);
        BpArgs fa = bp_args(BP_ATB, pl->b_op.p, S);
        fa.out64 = pl->f.as<double>(); fa.part = pb;
        backproject<T>(pl, ps, fa, st);
        finalize(pl, FIN_STORE, ps.bp, pb, 1, nullptr, nullptr, 0, nullptr, 0, st, SC_WNORM2);
        ga.init = 1;
        launch_gm_scalar(2, ga, st);
        ga.init = 0;
        launch_gm_setv(P, vt, nv, V, vstride, ldp, 0, pl->f.as<double>(), S, st);
        hold(s, PH_INIT, 1);
        for (int q : pl->live)
            if (s->phase[q] == PH_INIT) { s->phase[q] = PH_ARN; s->h_jn[q] = 0; any_arn = true; }
    }
    // shared part: t = V y (END) or v_j (ARN); u = B t; END: x += u, u = x; w = A u
    launch_gm_scalar(1, ga, st);
    launch_gm_combine(P, vt, nv, V, vstride, ldp, pl->gy.as<double>(), pl->jn.as<int>(), pl->t.as<double>(), S, st);
    count_launches(1);
    k_srv_gather<<<std::min(nv, num_sms() * 8), 256, 0, st>>>(P, vt, nv, V, vstride, pl->jn.as<int>(),
                                                                s->d_phase.as<int>(), pl->t.as<double>(), S);
    if (s->cfg.preconditioned) {
        bool have = false;
        int32_t rc = wmg_apply<T>(pl, pl->t.as<double>(), pl->u.as<double>(), false, false, false, &have, st);
        if (rc) return rc;
    } else {
        WMG_CUDA(cudaMemcpyAsync(pl->u.p, pl->t.p, pl->Ntot * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    if (any_end) {
        count_launches(1);
        k_srv_end_update<<<std::min(nv, num_sms() * 8), 256, 0, st>>>(P, vt, nv, s->d_phase.as<int>(),
                                                                        pl->x.as<double>(), pl->u.as<double>(), S);
    }
    ImgArgs ic{};
    ic.z = pl->u.as<double>(); ic.copy_op = pl->z_op.p; ic.copyT_op = pl->zT_op.p; ic.S = S;
    img_op<T>(pl, IMG_COPY64, ic, st);
    project<T>(pl, ps, pl->z_op.p, pl->zT_op.p, pl->sinoS.p, nullptr, S, st);
    BpArgs wa = bp_args(BP_GMRES_W, pl->sinoS.p, S);
    wa.z = pl->u.as<double>(); wa.out64 = pl->w.as<double>();
    backproject<T>(pl, ps, wa, st);
    // END: true residual r = f - w into v_0, restart (or stop) on beta = |r|
    if (any_end) {
        hold(s, PH_END, 0);
        VecArgs rv{};
        rv.f = pl->f.as<double>(); rv.w = pl->w.as<double>(); rv.v = V; rv.part = pb; rv.S = S;
        vec_op<T>(pl, VEC_RESID64, false, rv, st);
        finalize(pl, FIN_STORE, ps.vimg, pb, 1, nullptr, nullptr, 0, nullptr, 0, st, SC_WNORM2);
        launch_gm_scalar(2, ga, st);
        launch_gm_setv(P, vt, nv, V, vstride, ldp, 0, V, S, st);
        hold(s, PH_END, 1);
    }
    // ARN: two classical Gram-Schmidt passes against v_0 .. v_j, Hessenberg
    // column j, Givens rotation, v_{j+1} -- each slot at its own j = jn[slot]
    if (any_arn) {
        hold(s, PH_ARN, 0);
        const int *jv = pl->jn.as<int>();
        // classical Gram-Schmidt, the second pass only where the first one
        // cancelled (k_gm_reorth); |w|^2 partials from the last pass run
        int *skip = pl->reo.as<int>();
        for (int pass = 0; pass < 2; ++pass) {
            launch_gm_dots(P, vt, nv, V, vstride, pl->w.as<double>(), 0, ldp, pa, S, st, jv, pass == 0,
                           pass == 1 ? skip : nullptr);
            double *hv = pass == 0 ? pl->h1.as<double>() : pl->h2.as<double>();
            finalize(pl, FIN_STORE, ps.vimg, pa, jmax + 2, nullptr, nullptr, 0, nullptr, 0, st, 0, hv, ldp, ldp);
            launch_gm_axpy(P, vt, nv, V, vstride, pl->w.as<double>(), 0, ldp, hv, pb, S, st, jv,
                           pass == 1 ? skip : nullptr);
            if (pass == 0) {
                ga.jslot = 1;
                launch_gm_scalar(3, ga, st);
            }
        }
        finalize(pl, FIN_STORE, ps.vimg, pb, 1, nullptr, nullptr, 0, nullptr, 0, st, SC_WNORM2);
        ga.jslot = 1;
        launch_gm_scalar(0, ga, st);
        ga.jslot = 0;
        launch_gm_setv(P, vt, nv, V, vstride, ldp, 0, pl->w.as<double>(), S, st, jv);
        hold(s, PH_ARN, 1);
    }
    WMG_CUDA(cudaMemcpyAsync(s->h_S, S, (size_t)pl->cap * NSCAL * sizeof(double), cudaMemcpyDeviceToHost, st));
    WMG_CUDA(cudaMemcpyAsync(s->h_jn, pl->jn.p, pl->cap * sizeof(int), cudaMemcpyDeviceToHost, st));
    WMG_CUDA(cudaMemcpyAsync(s->h_done, pl->done.p, pl->cap * sizeof(int), cudaMemcpyDeviceToHost, st));
    WMG_CUDA(cudaStreamSynchronize(st));
    WMG_CUDA(cudaGetLastError());
    s->stats.ticks++;
    // phase transitions; stopped slots retire (x to the caller's buffer)
    std::vector<int> retiring;
    for (int q : pl->live) {
        const double *sq = s->h_S + (size_t)q * NSCAL;
        if (sq[SC_ACTIVE] == 0.0) { retiring.push_back(q); continue; }
        if (s->phase[q] == PH_END) { s->phase[q] = PH_ARN; continue; }
        if (s->h_done[q] || s->h_jn[q] >= s->cfg.restart) s->phase[q] = PH_END;
    }
    if (retiring.empty()) return WMG_OK;
    for (int q : retiring) {
        Request &r = s->reqs[s->slot_req[q]];
        count_launches(1);
        k_srv_store<T><<<std::max<int64_t>(1, std::min<int64_t>((r.N + 255) / 256, num_sms() * 4)), 256, 0, st>>>(
            pl->x.as<double>() + r.ioff, static_cast<T *>(r.x), r.N);
        WMG_CUDA(cudaMemcpyAsync(s->h_hist + (size_t)q * s->hld, pl->hist.as<double>() + (size_t)q * s->hld,
                                 s->hld * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    WMG_CUDA(cudaStreamSynchronize(st));
    WMG_CUDA(cudaGetLastError());
    for (int q : retiring) {
        Request &r = s->reqs[s->slot_req[q]];
        const double *sq = s->h_S + (size_t)q * NSCAL;
        r.info.iters = (int)sq[SC_ITERS];
        r.info.rel_res = sq[SC_RES];
        r.hist.assign(s->h_hist + (size_t)q * s->hld, s->h_hist + (size_t)(q + 1) * s->hld);
        finish(s, r, (int)sq[SC_STATUS]);
        s->img.release(r.ioff, r.N);
        s->sino.release(r.soff, r.M);
        s->geo_entries[r.gi].refs--;
        s->geo_entries[r.gi].last_use = ++s->use_clock;
        s->phase[q] = PH_EMPTY;
        s->slot_req[q] = 0;
        pl->pgeo[q] = -1;
        s->dirty = true;
    }
    return WMG_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int32_t wmg_server_create(const wmg_server_config *cfg, void *stream, wmg_server **out)
{
    if (!out || !cfg) return fail(WMG_ERR_INVALID_ARG, "wmg_server_create: bad arguments");
    *out = nullptr;
    const wmg_opts &o = cfg->opts;
    if (cfg->max_slots < 1 || cfg->max_iter < 1 || cfg->restart < 1 || cfg->restart > 64 || cfg->hbm_budget <= 0 ||
        cfg->state_bytes < 0 || cfg->state_bytes > cfg->hbm_budget || cfg->sino_ratio < 0 ||
        (o.precision != WMG_PREC_F64 && o.precision != WMG_PREC_F32) || o.cycle < WMG_CYCLE_ADDITIVE ||
        o.cycle > WMG_CYCLE_MULTIPLICATIVE || o.nu1 < 0 || o.nu2 < 0 || o.hybrid_depth < 0)
        return fail(WMG_ERR_INVALID_ARG, "wmg_server_create: invalid configuration");
    auto s = std::make_unique<wmg_server>();
    s->cfg = *cfg;
    if (s->cfg.opts.omega <= 0) s->cfg.opts.omega = 1.0;
    if (s->cfg.state_bytes == 0) s->cfg.state_bytes = cfg->hbm_budget / 2;
    if (s->cfg.sino_ratio == 0) s->cfg.sino_ratio = 4.0;
    s->st = static_cast<cudaStream_t>(stream);
    s->ldp = cfg->restart + 1;
    s->hld = cfg->max_iter + 1;
    s->pl = std::make_unique<wmg_plan>();
    wmg_plan *pl = s->pl.get();
    pl->prec = o.precision;
    pl->esz = o.precision == WMG_PREC_F64 ? 8 : 4;
    pl->opts = s->cfg.opts;
    pl->batch = true;
    const int cap = cfg->max_slots;
    const int hdm = o.cycle == WMG_CYCLE_ADDITIVE ? 0 : std::min(o.hybrid_depth, 11);
    int mult = 1;
    for (int d = 1; d < std::min(hdm, 12); ++d) mult *= 3;   // widest band group: 3^(h-1) nodes
    s->band_mult = mult;
    const int64_t esz = (int64_t)pl->esz;
    // per image element: x f w t u r1 C E + basis (FP64); z_op zT_op (T);
    // band images (2 T + 1 FP64 per node); symmetric-cycle copies
    s->bpi = (8 + s->ldp) * 8 + 2 * esz + (hdm > 0 ? mult * (2 * esz + 8) : 0) +
             (o.cycle == WMG_CYCLE_SYMMETRIC ? 3 * 8 * hdm : 0);
    // per sinogram element: b, A-pair sinogram, band sinograms (T)
    s->bps = 2 * esz + (hdm > 0 ? mult * esz : 0);
    const double ratio = s->cfg.sino_ratio;
    const int64_t Ncap = (int64_t)((double)s->cfg.state_bytes / ((double)s->bpi + ratio * (double)s->bps)) / 64 * 64;
    const int64_t Mcap = (int64_t)(ratio * (double)Ncap) / 64 * 64;
    if (Ncap < 64 || Mcap < 64) return fail(WMG_ERR_INVALID_ARG, "wmg_server_create: state budget too small");
    s->img.init(Ncap);
    s->sino.init(Mcap);
    s->geo_budget = cfg->hbm_budget - s->cfg.state_bytes;
    pl->Ntot = Ncap;
    pl->Mtot = Mcap;
    pl->cap = cap;
    pl->pgeo.assign(cap, -1);
    pl->img_off.assign(cap, 0);
    pl->sino_off.assign(cap, 0);
    pl->real.nprob = cap;
    pl->real.h.assign(cap, ProbDev{});
    s->phase.assign(cap, PH_EMPTY);
    s->slot_req.assign(cap, 0);
    const int64_t band_N = hdm > 0 ? mult * Ncap : 0, band_M = hdm > 0 ? mult * Mcap : 0;
    bool ok = ensure_pool(pl->x, Ncap, 8) && ensure_pool(pl->f, Ncap, 8) && ensure_pool(pl->w, Ncap, 8) &&
              ensure_pool(pl->t, Ncap, 8) && ensure_pool(pl->u, Ncap, 8) && ensure_pool(pl->r1, Ncap, 8) &&
              ensure_pool(pl->C, Ncap, 8) && ensure_pool(pl->E, Ncap, 8) &&
              ensure_pool(pl->V, Ncap * s->ldp, 8) && ensure_pool(pl->z_op, Ncap, esz) &&
              ensure_pool(pl->zT_op, Ncap, esz) && ensure_pool(pl->sinoS, Mcap, esz) &&
              ensure_pool(pl->b_op, Mcap, esz);
    if (ok && hdm > 0)
        ok = ensure_pool(pl->band_img, band_N, esz) && ensure_pool(pl->band_imgT, band_N, esz) &&
             ensure_pool(pl->band_img2, band_N, 8) && ensure_pool(pl->band_sino, band_M, esz);
    for (int d = 0; ok && d < std::max(hdm, 1); ++d) {
        pl->csave.push_back(std::make_unique<DevBuf>());
        pl->c2.push_back(std::make_unique<DevBuf>());
        pl->e2.push_back(std::make_unique<DevBuf>());
        if (o.cycle == WMG_CYCLE_SYMMETRIC && d < hdm)
            ok = ensure_pool(*pl->csave[d], Ncap, 8) && ensure_pool(*pl->c2[d], Ncap, 8) &&
                 ensure_pool(*pl->e2[d], Ncap, 8);
    }
    ok = ok && pl->S.ensure((size_t)cap * NSCAL * 8) && pl->lam.ensure((size_t)cap * 8) &&
         pl->H.ensure((size_t)cap * s->ldp * cfg->restart * 8) && pl->gcs.ensure((size_t)cap * cfg->restart * 8) &&
         pl->gsn.ensure((size_t)cap * cfg->restart * 8) && pl->gg.ensure((size_t)cap * s->ldp * 8) &&
         pl->gy.ensure((size_t)cap * s->ldp * 8) && pl->h1.ensure((size_t)cap * s->ldp * 8) &&
         pl->h2.ensure((size_t)cap * s->ldp * 8) && pl->jn.ensure((size_t)cap * 4) &&
         pl->done.ensure((size_t)cap * 4) && pl->reo.ensure((size_t)cap * 4) &&
         pl->hist.ensure((size_t)cap * s->hld * 8) &&
         s->d_phase.ensure((size_t)cap * 4);
    if (!ok) return fail(WMG_ERR_OOM, "wmg_server_create: state pools do not fit in device memory");
    if (cudaMallocHost(&s->h_phase, cap * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&s->h_jn, cap * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&s->h_done, cap * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&s->h_S, (size_t)cap * NSCAL * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&s->h_hist, (size_t)cap * s->hld * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(WMG_ERR_OOM, "wmg_server_create: pinned host buffers");
    }
    std::memset(s->h_jn, 0, cap * sizeof(int));
    WMG_CUDA(cudaMemsetAsync(pl->S.p, 0, (size_t)cap * NSCAL * 8, s->st));
    WMG_CUDA(cudaMemsetAsync(pl->jn.p, 0, (size_t)cap * 4, s->st));
    WMG_CUDA(cudaMemsetAsync(pl->done.p, 0, (size_t)cap * 4, s->st));
    int32_t rc = relayout(s.get());
    if (rc) return rc;
    WMG_CUDA(cudaStreamSynchronize(s->st));
    s->worker.start();
    s->stats.state_bytes_capacity = Ncap * s->bpi + Mcap * s->bps;
    s->stats.geometry_bytes_capacity = s->geo_budget;
    *out = s.release();
    return WMG_OK;
}

extern "C" int32_t wmg_server_destroy(wmg_server *srv)
{
    delete srv;
    return WMG_OK;
}

extern "C" int32_t wmg_server_submit(wmg_server *srv, const wmg_geom *g, const wmg_opts *o, const void *b,
                                     void *x, uint64_t *ticket)
{
    if (!srv || !g || !b || !x || !ticket) return fail(WMG_ERR_INVALID_ARG, "wmg_server_submit: bad arguments");
    *ticket = 0;
    wmg_opts opt = o ? *o : srv->cfg.opts;
    if (opt.omega <= 0) opt.omega = 1.0;
    int32_t rc = validate(g, &opt);
    if (rc) return rc;
    const wmg_opts &so = srv->cfg.opts;
    if (opt.precision != so.precision || opt.cycle != so.cycle || opt.nu1 != so.nu1 || opt.nu2 != so.nu2 ||
        opt.omega != so.omega || opt.hybrid_depth != so.hybrid_depth)
        return fail(WMG_ERR_INVALID_ARG,
                    "wmg_server_submit: precision, cycle, nu1, nu2, omega and hybrid depth must be the server's");
    if (srv->cfg.preconditioned && opt.levels < 1)
        return fail(WMG_ERR_INVALID_ARG, "wmg_server_submit: a preconditioned server needs levels >= 1");
    Request r;
    r.id = srv->next_id++;
    r.g = *g;
    if (g->angles) r.angles.assign(g->angles, g->angles + g->m);
    r.g.angles = nullptr;
    r.o = opt;
    r.key = geo_key(*g, opt);
    r.b = b;
    r.x = x;
    r.N = (int64_t)g->n * g->n;
    r.M = (int64_t)g->m * g->D;
    const int64_t gb = srv->geo_by_key.count(r.key)
                           ? 0
                           : geo_bytes(*g, opt, srv->pl->esz) + setup_transient_bytes(*g, opt, srv->pl->esz);
    if (RangeAlloc::round(r.N) > srv->img.cap || RangeAlloc::round(r.M) > srv->sino.cap || gb > srv->geo_budget) {
        srv->stats.rejected++;
        return fail(WMG_ERR_REJECTED, "wmg_server_submit: the request's footprint exceeds the server's budget");
    }
    r.t_submit = Clock::now();
    srv->stats.submitted++;
    *ticket = r.id;
    srv->queue.push_back(r.id);
    srv->reqs.emplace(r.id, std::move(r));
    return WMG_OK;
}

extern "C" int32_t wmg_server_step(wmg_server *srv, int32_t *pending)
{
    if (!srv) return fail(WMG_ERR_INVALID_ARG, "wmg_server_step: server is NULL");
    int32_t rc = admit(srv);
    if (!rc && srv->dirty) rc = relayout(srv);
    if (!rc && !srv->pl->live.empty())
        rc = srv->pl->prec == WMG_PREC_F64 ? tick<double>(srv) : tick<float>(srv);
    else if (!rc && !srv->in_setup.empty())
        std::this_thread::sleep_for(std::chrono::microseconds(200));   // nothing to run: let setups progress
    if (rc) return rc;
    int running = 0;
    for (int ph : srv->phase) running += ph != PH_EMPTY;
    srv->stats.running = running;
    srv->stats.queued = (int32_t)srv->queue.size();
    if (pending) *pending = running + (int32_t)srv->queue.size();
    return WMG_OK;
}

extern "C" int32_t wmg_server_poll(wmg_server *srv, uint64_t ticket, int32_t *state, wmg_solve_info *info,
                                   double *latency_ms, double *res_hist)
{
    if (!srv || !state) return fail(WMG_ERR_INVALID_ARG, "wmg_server_poll: bad arguments");
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(WMG_ERR_INVALID_ARG, "wmg_server_poll: unknown ticket");
    Request &r = it->second;
    *state = r.state;
    if (r.state != WMG_REQ_DONE) return WMG_OK;
    if (info) *info = r.info;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
    if (res_hist && !r.hist.empty()) std::memcpy(res_hist, r.hist.data(), r.hist.size() * sizeof(double));
    srv->reqs.erase(it);
    return WMG_OK;
}

extern "C" int32_t wmg_server_footprint(const wmg_server *srv, const wmg_geom *g, const wmg_opts *o,
                                        int64_t *state, int64_t *geometry, int64_t *setup)
{
    if (!srv || !g) return fail(WMG_ERR_INVALID_ARG, "wmg_server_footprint: bad arguments");
    wmg_opts opt = o ? *o : srv->cfg.opts;
    int32_t rc = validate(g, &opt);
    if (rc) return rc;
    const int64_t N = (int64_t)g->n * g->n, M = (int64_t)g->m * g->D;
    if (state) *state = state_bytes(srv, N, M);
    if (geometry) *geometry = geo_bytes(*g, opt, srv->pl->esz);
    if (setup) *setup = setup_transient_bytes(*g, opt, srv->pl->esz);
    return WMG_OK;
}

extern "C" int32_t wmg_server_stats(const wmg_server *srv, wmg_server_counters *out)
{
    if (!srv || !out) return fail(WMG_ERR_INVALID_ARG, "wmg_server_stats: bad arguments");
    *out = srv->stats;
    out->state_bytes_used = srv->img.used * srv->bpi + srv->sino.used * srv->bps;
    out->geometry_bytes_used = srv->geo_used;
    int cached = 0;
    for (auto &g : srv->pl->geos) cached += g != nullptr;
    out->geometries_cached = cached;
    return WMG_OK;
}
