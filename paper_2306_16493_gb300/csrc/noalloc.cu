// Conductivity from per-state device arrays without any device allocation.
//
// Some callers cannot call cudaMalloc: a host framework that owns all device memory
// through its own pool, or a long-running service that must not allocate after start-up
// (cudaMalloc and cudaFree may synchronise the device and can fail under memory pressure
// in the middle of a run).  epwi_conductivity_noalloc serves them: the caller passes its own
// input and output buffers, and the only scratch (per-block partial sums of the reduction)
// lives in a fixed file-scope device array.
//
// The array is shared by every call in the process and keeps the last call's contents;
// each call overwrites every slot it reads, so nothing needs clearing, but two calls that
// overlap on the GPU (different streams, or different host threads) race on it.
//
// The device address of the array is looked up once per device and cached.  Two host
// threads that make their first call on a device at the same time both store the same
// address, which is harmless.  A cudaDeviceReset (or any teardown of the primary context)
// unloads the module, and the array may come back at another address: the cached one is
// then stale, so this entry point must not be used after a device reset in the same process.
#include <cuda_runtime.h>

#include <cstdint>

#include "epwi.h"

namespace {

constexpr int kThreads = 256;
constexpr int64_t kStatesPerBlock = 4096;          // fixed-order chunk of one block
constexpr int kMaxBlocks = 1024;                   // scratch: kMaxBlocks x 6 doubles (48 KiB)
constexpr int kMaxDevices = 64;

// Partial sums (xx, yy, zz, xy, xz, yz) of each block of the first reduction pass.
static __device__ __align__(256) double g_sigma_scratch[kMaxBlocks * 6];

double *g_scratch_ptr[kMaxDevices] = {nullptr};   // device address of g_sigma_scratch per device

__device__ __forceinline__ double fermi(double e, double mu, double kT) {
    const double x = (e - mu) / kT;
    const double ex = exp(-fabs(x));
    return x > 0 ? ex / (1.0 + ex) : 1.0 / (1.0 + ex);
}

__global__ void __launch_bounds__(kThreads) k_sigma_part_na(int64_t ns, const double *__restrict__ eps,
                                                            const double *__restrict__ vel,
                                                            const double *__restrict__ inv_tau, double mu,
                                                            double kT, double *__restrict__ part) {
    __shared__ double sm[6][kThreads];
    const int64_t b0 = (int64_t)blockIdx.x * kStatesPerBlock;
    const int64_t b1 = b0 + kStatesPerBlock < ns ? b0 + kStatesPerBlock : ns;
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t s = b0 + threadIdx.x; s < b1; s += kThreads) {
        const double r = inv_tau[s];
        if (!(r > 0)) continue;
        const double f = fermi(eps[s], mu, kT);
        const double w = f * (1.0 - f) / r;
        const double vx = vel[3 * s], vy = vel[3 * s + 1], vz = vel[3 * s + 2];
        v[0] += w * vx * vx;
        v[1] += w * vy * vy;
        v[2] += w * vz * vz;
        v[3] += w * vx * vy;
        v[4] += w * vx * vz;
        v[5] += w * vy * vz;
    }
    for (int j = 0; j < 6; ++j) sm[j][threadIdx.x] = v[j];
    __syncthreads();
    for (int st = kThreads / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int j = 0; j < 6; ++j) sm[j][threadIdx.x] += sm[j][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int j = 0; j < 6; ++j) part[blockIdx.x * 6 + j] = sm[j][0];
}

// One block sums the partials in a fixed order and writes the 3x3 tensor.
__global__ void __launch_bounds__(kThreads) k_sigma_final_na(int nb, const double *__restrict__ part,
                                                             double pref, double *__restrict__ sigma) {
    __shared__ double sm[6][kThreads];
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += kThreads)
        for (int j = 0; j < 6; ++j) v[j] += part[b * 6 + j];
    for (int j = 0; j < 6; ++j) sm[j][threadIdx.x] = v[j];
    __syncthreads();
    for (int st = kThreads / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int j = 0; j < 6; ++j) sm[j][threadIdx.x] += sm[j][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double h[6] = {sm[0][0], sm[1][0], sm[2][0], sm[3][0], sm[4][0], sm[5][0]};
        const double t[9] = {h[0], h[3], h[4], h[3], h[1], h[5], h[4], h[5], h[2]};
        for (int i = 0; i < 9; ++i) sigma[i] = pref * t[i];
    }
}

}  // namespace

extern "C" epwi_status epwi_conductivity_noalloc(int64_t n_states, const double *eps_dev,
                                                 const double *vel_dev, const double *inv_tau_dev,
                                                 double mu_eV, double T_K, double volume_A3,
                                                 int64_t nk, void *cuda_stream, double *sigma_dev) {
    if (n_states < 0 || n_states > (int64_t)kMaxBlocks * kStatesPerBlock) return EPWI_EUNSUPPORTED;
    if (!sigma_dev || !(T_K > 0) || !(volume_A3 > 0) || nk < 1) return EPWI_EINVAL;
    if (n_states > 0 && (!eps_dev || !vel_dev || !inv_tau_dev)) return EPWI_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EPWI_ECUDA;
    if (!g_scratch_ptr[dev]) {
        // first call on this device: resolve the device address of the scratch array
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sigma_scratch) != cudaSuccess || !p) return EPWI_ECUDA;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int nb = n_states > 0 ? (int)((n_states + kStatesPerBlock - 1) / kStatesPerBlock) : 1;
    const double kT = 8.617333262e-5 * T_K;                   // k_B in eV/K (CODATA 2018)
    const double e = 1.602176634e-19;
    const double pref = 2.0 * e * e / ((double)nk * volume_A3 * 1e-30 * kT * e);
    k_sigma_part_na<<<nb, kThreads, 0, st>>>(n_states, eps_dev, vel_dev, inv_tau_dev, mu_eV, kT,
                                             g_scratch_ptr[dev]);
    if (cudaGetLastError() != cudaSuccess) return EPWI_ECUDA;
    k_sigma_final_na<<<1, kThreads, 0, st>>>(nb, g_scratch_ptr[dev], pref, sigma_dev);
    if (cudaGetLastError() != cudaSuccess) return EPWI_ECUDA;
    return EPWI_OK;
}
