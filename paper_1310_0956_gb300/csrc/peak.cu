// peak.cu -- measured arithmetic peaks of the GPU the library runs on: the
// denominators of the roofline of its ALU-bound kernels (the matrix-free
// projector and backprojector are bound by FP32 arithmetic and instruction
// issue, not by memory). A kernel of independent multiply-add chains with no
// memory traffic, timed with CUDA events on the caller's stream.
#include <algorithm>

#include "kern_common.cuh"

namespace wmg {

namespace {
constexpr int kChains = 8;          // independent accumulators per thread
constexpr int kSteps = 4096;        // multiply-adds per chain
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

template <class T>
__global__ void __launch_bounds__(kThreads) k_peak_fma(T a, T c, T *sink)
{
    T acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = (T)(threadIdx.x + i);
    for (int s = 0; s < kSteps; s += 4)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) acc[i] = fma_t(acc[i], a, c);
    T v = T(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) v += acc[i];
    if (v == T(-1)) *sink = v;         // never true: keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_peak_fma2(float a, float c, float *sink)
{
    float2 acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = make_float2((float)threadIdx.x + i, (float)i);
    const float2 a2 = make_float2(a, a), c2 = make_float2(c, c);
    for (int s = 0; s < kSteps; s += 4)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) acc[i] = __ffma2_rn(acc[i], a2, c2);
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) v += acc[i].x + acc[i].y;
    if (v == -1.f) *sink = v;
}
}  // namespace

}  // namespace wmg

using namespace wmg;

extern "C" int32_t wmg_measure_peak(int32_t kind, double *tflops, void *stream)
{
    if (!tflops || kind < WMG_PEAK_FP32_FMA || kind > WMG_PEAK_FP64_FMA)
        return fail(WMG_ERR_INVALID_ARG, "wmg_measure_peak: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = num_sms() * kCtasPerSm;
    // the sink is never written; any valid device address would do, so the
    // kernel takes the address of a small buffer of its own
    void *sink = nullptr;
    WMG_CUDA(cudaMallocAsync(&sink, 16, st));
    cudaEvent_t e0, e1;
    WMG_CUDA(cudaEventCreate(&e0));
    WMG_CUDA(cudaEventCreate(&e1));
    auto launch = [&]() {
        count_launches(1);
        if (kind == WMG_PEAK_FP32_FMA) k_peak_fma<float><<<grid, kThreads, 0, st>>>(0.999999f, 1e-6f, (float *)sink);
        else if (kind == WMG_PEAK_FP32_FMA2) k_peak_fma2<<<grid, kThreads, 0, st>>>(0.999999f, 1e-6f, (float *)sink);
        else k_peak_fma<double><<<grid, kThreads, 0, st>>>(0.999999, 1e-6, (double *)sink);
    };
    launch();                                              // warm-up
    float best = 0.f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == 0 || ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    WMG_CUDA(cudaStreamSynchronize(st));
    WMG_CUDA(cudaGetLastError());
    const double fmas = (double)grid * kThreads * kChains * kSteps * (kind == WMG_PEAK_FP32_FMA2 ? 2.0 : 1.0);
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return WMG_OK;
}
