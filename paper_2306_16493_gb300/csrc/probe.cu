// Throughput probe for the FP32 and FP64 FMA rates of the device: the denominators of the
// roofline fractions of the SIMT kernels (the sum-factorised FP32 interpolation, the FP64
// path).  Each thread runs kChains independent FMA chains of a register-resident recurrence,
// so the probe is limited by the FMA pipe alone (no memory traffic, no dependent latency
// once a scheduler has a few warps); the grid covers every SM several times over.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "epwi.h"
#include "epwi_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int64_t iters, T a, T b, T *sink) {
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) acc[c] = acc[c] * a + b;   // one FMA
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == (T)-12345.678) sink[threadIdx.x] = s;   // never true for these a, b; keeps the chains live
}

template <typename T>
float time_probe(int64_t iters, int blocks, cudaStream_t st, T *sink) {
    cudaEvent_t e0, e1;
    EPWI_CUDA(cudaEventCreate(&e0));
    EPWI_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    // a < 1 and b small: the recurrence converges to b / (1 - a) and never overflows
    k_fma_probe<T><<<blocks, kThreads, 0, st>>>(iters, (T)0.999, (T)1e-4, sink);
    cudaEventRecord(e1, st);
    EPWI_CUDA(cudaGetLastError());
    EPWI_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

template <typename T>
double run_probe(int device, cudaStream_t st, double target_ms, double *ms_out) {
    int sms = 0;
    EPWI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int blocks = sms * kBlocksPerSm;
    T *sink = nullptr;
    EPWI_CUDA(cudaMalloc(&sink, sizeof(T) * kThreads));
    double best = 0, best_ms = 0;
    try {
        // size the launch from a short calibration run, then keep the best of three
        int64_t iters = 64;
        float ms = time_probe<T>(iters, blocks, st, sink);
        while (ms < 2.0f && iters < (int64_t(1) << 30)) {
            iters *= 4;
            ms = time_probe<T>(iters, blocks, st, sink);
        }
        iters = std::max<int64_t>(1, (int64_t)(iters * target_ms / std::max(ms, 1e-3f)));
        for (int r = 0; r < 3; ++r) {
            ms = time_probe<T>(iters, blocks, st, sink);
            const double flop = 2.0 * kChains * kUnroll * (double)iters * blocks * kThreads;
            const double tf = flop / (ms * 1e-3) / 1e12;
            if (tf > best) {
                best = tf;
                best_ms = ms;
            }
        }
    } catch (...) {
        cudaFree(sink);
        throw;
    }
    cudaFree(sink);
    if (ms_out) *ms_out = best_ms;
    return best;
}

}  // namespace

extern "C" epwi_status epwi_fma_peak(int32_t fp64, int32_t device, void *cuda_stream, double target_ms,
                                     double *tflops, double *ms) {
    if (!tflops || !(target_ms > 0) || (fp64 != 0 && fp64 != 1)) return EPWI_EINVAL;
    try {
        EPWI_CUDA(cudaSetDevice(device));
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        *tflops = fp64 ? run_probe<double>(device, st, target_ms, ms) : run_probe<float>(device, st, target_ms, ms);
        return EPWI_OK;
    } catch (const EpwiError &e) {
        return e.status;
    } catch (...) {
        return EPWI_ECUDA;
    }
}
