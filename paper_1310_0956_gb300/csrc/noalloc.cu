// noalloc.cu -- forward projection that allocates no device memory.
//
// wmg_project needs workspace for the transposed copy of the image (the
// projector walks the rows of that copy for angles closer to 90 degrees than
// to 0). Plans take that workspace, and their tables, from cudaMalloc. Some
// callers cannot allocate: a scanner's acquisition loop that reserves all the
// device memory it will ever use at start-up, so that no allocation can fail
// or stall in the middle of a scan, or a host program whose framework
// allocator already owns all free device memory. wmg_project_noalloc serves
// them: it keeps its scratch (the transposed image, the work lists and the
// geometry tables) in file-scope __device__ arrays of a fixed maximum size,
// which every GPU that loads the library holds until the process exits, and
// calls neither cudaMalloc nor cudaFree nor any allocating routine.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "kern_common.cuh"

namespace wmg {
namespace {

constexpr int kMaxSide = 1024;                       // n <= 1024: 4 MiB image scratch
constexpr int kMaxAngles = 4096;
constexpr int kMaxBins = 2048;
constexpr int kMaxProjTiles = kMaxAngles * ((kMaxBins + 31) / 32);
constexpr int kMaxImgTiles = (kMaxSide / 32) * (kMaxSide / 32);

// Shared by every call on a device; the last call's contents stay in place.
static __device__ __align__(256) float g_scratch_T[(size_t)kMaxSide * kMaxSide];
static __device__ __align__(256) int4 g_proj_tiles[kMaxProjTiles];
static __device__ __align__(256) int4 g_img_tiles[kMaxImgTiles];
static __device__ __align__(256) double2 g_cs64[kMaxAngles];
static __device__ __align__(256) float2 g_cs32[kMaxAngles];
static __device__ __align__(256) float4 g_csx[kMaxAngles];
static __device__ __align__(256) AngleF g_angf[kMaxAngles];
static __device__ __align__(256) GeomDev g_geom;
static __device__ __align__(256) ProbDev g_prob;

// Device memory the arrays above hold on every GPU that loads them:
// 8,830,976 bytes of arrays (about 8.4 MiB) plus the two small records.
constexpr size_t kArrayBytes = sizeof(float) * (size_t)kMaxSide * kMaxSide +
                               sizeof(int4) * (size_t)(kMaxProjTiles + kMaxImgTiles) +
                               (sizeof(double2) + sizeof(float2) + sizeof(float4) + sizeof(AngleF)) *
                                   (size_t)kMaxAngles;
static_assert(kArrayBytes == 8830976, "the documented scratch size is 8,830,976 bytes of arrays");

struct DeviceSlots {
    bool ready = false;
    float *scratch_T = nullptr;
    int4 *proj_tiles = nullptr, *img_tiles = nullptr;
    double2 *cs64 = nullptr;
    float2 *cs32 = nullptr;
    float4 *csx = nullptr;
    AngleF *angf = nullptr;
    GeomDev *geom = nullptr;
    ProbDev *prob = nullptr;
};
constexpr int kMaxDevices = 64;
static DeviceSlots g_slots[kMaxDevices];

// Host staging of the angle tables (fixed size, no heap use), shared by every
// host thread and device: a call holds g_host_lock from the first write into
// it until its copies have been issued. A copy from pageable host memory
// returns once the source has been read, so the lock need not outlast it.
static double2 h_cs64[kMaxAngles];
static float2 h_cs32[kMaxAngles];
static float4 h_csx[kMaxAngles];
static AngleF h_angf[kMaxAngles];
static std::mutex g_host_lock;

// Device addresses of the arrays above, looked up once per device with that
// device current (host code may not use the symbols' names as addresses).
// The first lookup on a device loads the module there, which is when the
// arrays take their device memory. Called with g_host_lock held.
int32_t device_slots(DeviceSlots **out)
{
    int dev = 0;
    WMG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(WMG_ERR_INVALID_ARG, "device index out of range");
    DeviceSlots &s = g_slots[dev];
    if (!s.ready) {
        WMG_CUDA(cudaGetSymbolAddress((void **)&s.scratch_T, g_scratch_T));
        WMG_CUDA(cudaGetSymbolAddress((void **)&s.proj_tiles, g_proj_tiles));
        WMG_CUDA(cudaGetSymbolAddress((void **)&s.img_tiles, g_img_tiles));
        WMG_CUDA(cudaGetSymbolAddress((void **)&s.cs64, g_cs64));
        WMG_CUDA(cudaGetSymbolAddress((void **)&s.cs32, g_cs32));
        WMG_CUDA(cudaGetSymbolAddress((void **)&s.csx, g_csx));
        WMG_CUDA(cudaGetSymbolAddress((void **)&s.angf, g_angf));
        WMG_CUDA(cudaGetSymbolAddress((void **)&s.geom, g_geom));
        WMG_CUDA(cudaGetSymbolAddress((void **)&s.prob, g_prob));
        s.ready = true;
    }
    *out = &s;
    return WMG_OK;
}

// Work lists of one image: 32-ray tiles per angle, 32 x 32 pixel tiles.
__global__ void k_noalloc_tiles(int n, int m, int D, int4 *proj, int4 *img)
{
    const int nk = (D + 31) / 32, nb = (n + 31) / 32;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m * nk; t += gridDim.x * blockDim.x)
        proj[t] = make_int4(0, t / nk, (t % nk) * 32, 0);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nb * nb; t += gridDim.x * blockDim.x)
        img[t] = make_int4(0, (t / nb) * 32, (t % nb) * 32, 0);
}

}  // namespace
}  // namespace wmg

using namespace wmg;

extern "C" int32_t wmg_project_noalloc(int32_t n, int32_t m, int32_t D, const float *x, float *b,
                                       void *stream)
{
    if (n < 1 || m < 1 || D < 1 || !x || !b)
        return fail(WMG_ERR_INVALID_ARG, "wmg_project_noalloc: bad arguments");
    if (n > kMaxSide || m > kMaxAngles || D > kMaxBins)
        return fail(WMG_ERR_INVALID_ARG, "wmg_project_noalloc: n <= 1024, m <= 4096 and D <= 2048 "
                                         "(fixed scratch size); use wmg_project for larger problems");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> hold(g_host_lock);
    DeviceSlots *s = nullptr;
    int32_t rc = device_slots(&s);
    if (rc) return rc;
    // geometry: the same host routines as a plan's (equiangular angles,
    // exact intersection lengths, unit bins centred on the image)
    geometry_tables(m, nullptr, WMG_KERNEL_STRIP, h_cs64, h_cs32, h_csx, h_angf);
    GeomDev g{};
    g.n = n; g.m = m; g.D = D; g.L = 0; g.nc = n; g.P = n * n; g.K = 1; g.B = 1;
    g.h = 1.0 / n; g.t0 = 0.0; g.dt = 1.0; g.lambda = 0.0; g.omega = 1.0;
    g.kernel = WMG_KERNEL_STRIP;
    g.cs64 = s->cs64; g.cs32 = s->cs32; g.csx = s->csx; g.angf = s->angf;
    geometry_scalars(g, h_angf);
    ProbDev p{};
    p.geom = 0; p.slot = 0; p.img = 0; p.sino = 0; p.coef = 0;
    WMG_CUDA(cudaMemcpyAsync(s->cs64, h_cs64, m * sizeof(double2), cudaMemcpyHostToDevice, st));
    WMG_CUDA(cudaMemcpyAsync(s->cs32, h_cs32, m * sizeof(float2), cudaMemcpyHostToDevice, st));
    WMG_CUDA(cudaMemcpyAsync(s->csx, h_csx, m * sizeof(float4), cudaMemcpyHostToDevice, st));
    WMG_CUDA(cudaMemcpyAsync(s->angf, h_angf, m * sizeof(AngleF), cudaMemcpyHostToDevice, st));
    WMG_CUDA(cudaMemcpyAsync(s->geom, &g, sizeof(g), cudaMemcpyHostToDevice, st));
    WMG_CUDA(cudaMemcpyAsync(s->prob, &p, sizeof(p), cudaMemcpyHostToDevice, st));
    const int nproj = m * ((D + 31) / 32), nimg = ((n + 31) / 32) * ((n + 31) / 32);
    count_launches(1);
    k_noalloc_tiles<<<std::min(1024, (std::max(nproj, nimg) + 255) / 256), 256, 0, st>>>(
        n, m, D, s->proj_tiles, s->img_tiles);
    // the transposed copy overwrites every element the projector reads, so
    // nothing has to be cleared between calls
    launch_transpose<float>(s->geom, s->prob, s->img_tiles, nimg, x, s->scratch_T, st);
    PjArgs a{0, x, s->scratch_T, b, nullptr, nullptr, nullptr, 1};
    launch_project<float>(s->geom, s->prob, s->proj_tiles, nproj, a, st);
    WMG_CUDA(cudaGetLastError());
    return WMG_OK;
}
