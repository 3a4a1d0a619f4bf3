// Energy-conservation sieve predicate (internal), shared by the sieve kernels and the
// importance-sampling path (Sec. III A).
#pragma once

#include "epwi_internal.cuh"

// Threads of the sieve kernels.  This fixes the candidate order of every pair list the sieve
// writes: for each k-point, plane blocks pb of kSieveBlock consecutive (q2, q3) combinations,
// then q1, then the combination; the sum-factorised interpolation relies on that order.
constexpr int kSieveBlock = 256;

struct SieveArgs {
    GridInfo g;
    int W, Nm;
    const double *eps;
    const float *eps32;
    const double *hw;
    const float *hw32;       // per mode, -1 for dropped modes
    const float *hwmax32;
    double omega_min, ceta;
    float ceta32, delta32;   // delta32 bounds |x_fp32 - x_fp64| for every candidate
    float lim_extra;         // c eta + delta32
    // pruning table: band energy ranges (min, max; FP32) over aligned segments of kSegLen
    // consecutive points along axis 1 of every (axis 2, axis 3) column of the grid,
    // segr[((col * nseg) + seg) * W + m]; seglim bounds hwmax(q) + the prefilter's pad
    const float2 *segr;
    int nseg;
    float seglim;
};
constexpr int kSegLen = 8;
constexpr int kSegMinGrid = 64;   // grids with fewer axis-1 points skip the table

// Decision for one candidate (k, q).  FP32 evaluates x = (e_n + s w) - e_m for every
// (n, m, nu, s); a value inside c eta - delta (outside c eta + delta) is decided in FP32,
// anything closer to the boundary is re-evaluated in FP64 with the oracle's rounding order,
// so the outcome equals an FP64 evaluation.
__device__ __forceinline__ bool pair_valid(const SieveArgs &a, int nsel, const double *en,
                                           const float *en32, int64_t iq, int64_t ikq) {
    const float hm = a.hwmax32[iq];
    if (hm < 0.f) return false;
    const float lim = hm + a.lim_extra;
    const float inner = a.ceta32 - a.delta32, outer = a.ceta32 + a.delta32;
    bool ambiguous = false;
    for (int m = 0; m < a.W; ++m) {
        const float em32 = a.eps32[ikq * a.W + m];
        for (int n = 0; n < nsel; ++n) {
            const float d = en32[n] - em32;
            if (!(fabsf(d) <= lim)) continue;
            for (int nu = 0; nu < a.Nm; ++nu) {
                const float w = a.hw32[iq * a.Nm + nu];
                if (w < 0.f) continue;
                const float x1 = fabsf(d + w), x2 = fabsf(d - w);
                const float xm = fminf(x1, x2);
                if (xm <= inner) return true;
                if (xm <= outer) ambiguous = true;
            }
        }
    }
    if (!ambiguous) return false;
    for (int m = 0; m < a.W; ++m) {
        const double em = a.eps[ikq * a.W + m];
        for (int nu = 0; nu < a.Nm; ++nu) {
            const double w = a.hw[iq * a.Nm + nu];
            if (!(w >= a.omega_min)) continue;
            for (int n = 0; n < nsel; ++n) {
                const double x1 = (en[n] + w) - em;
                const double x2 = (en[n] - w) - em;
                if (fabs(x1) <= a.ceta || fabs(x2) <= a.ceta) return true;
            }
        }
    }
    return false;
}

// The k+q energies of a candidate (one or two 16-byte loads where WT is a multiple of 4).
template <int WT>
__device__ __forceinline__ void load_kq_energies(const SieveArgs &a, int64_t ikq, float (&em)[WT]) {
    if constexpr (WT % 4 == 0) {
#pragma unroll
        for (int m4 = 0; m4 < WT / 4; ++m4) {
            const float4 e = reinterpret_cast<const float4 *>(a.eps32 + ikq * WT)[m4];
            em[4 * m4] = e.x; em[4 * m4 + 1] = e.y; em[4 * m4 + 2] = e.z; em[4 * m4 + 3] = e.w;
        }
    } else {
#pragma unroll
        for (int m = 0; m < WT; ++m) em[m] = a.eps32[ikq * WT + m];
    }
}

// pair_valid_t after its loads: hm = hwmax32[iq] >= 0 and em = the k+q energies.
template <int WT, int NMT>
__device__ __forceinline__ bool pair_valid_tail(const SieveArgs &a, int nsel, const double *en, const float *en32,
                                                int64_t iq, int64_t ikq, float hm, const float (&em)[WT]) {
    const float lim = hm + a.lim_extra;
    const float inner = a.ceta32 - a.delta32, outer = a.ceta32 + a.delta32;
    bool near = false;
    for (int n = 0; n < nsel; ++n)
#pragma unroll
        for (int m = 0; m < WT; ++m) near |= fabsf(en32[n] - em[m]) <= lim;
    if (!near) return false;
    float w[NMT];
#pragma unroll
    for (int nu = 0; nu < NMT; ++nu) w[nu] = a.hw32[iq * NMT + nu];
    bool ambiguous = false;
#pragma unroll
    for (int m = 0; m < WT; ++m) {
        for (int n = 0; n < nsel; ++n) {
            const float d = en32[n] - em[m];
            if (!(fabsf(d) <= lim)) continue;
#pragma unroll
            for (int nu = 0; nu < NMT; ++nu) {
                if (w[nu] < 0.f) continue;
                const float xm = fminf(fabsf(d + w[nu]), fabsf(d - w[nu]));
                if (xm <= inner) return true;
                if (xm <= outer) ambiguous = true;
            }
        }
    }
    if (!ambiguous) return false;
    for (int m = 0; m < WT; ++m) {
        const double emd = a.eps[ikq * WT + m];
        for (int nu = 0; nu < NMT; ++nu) {
            const double wd = a.hw[iq * NMT + nu];
            if (!(wd >= a.omega_min)) continue;
            for (int n = 0; n < nsel; ++n) {
                const double x1 = (en[n] + wd) - emd;
                const double x2 = (en[n] - wd) - emd;
                if (fabs(x1) <= a.ceta || fabs(x2) <= a.ceta) return true;
            }
        }
    }
    return false;
}

// pair_valid for compile-time W and N_m: the k+q energies in 16-byte loads, the mode energies
// loaded once per candidate, the FP32 tests in pair_valid's arithmetic, and the FP64 re-check
// of pair_valid for candidates near c eta.  Same outcome as pair_valid.
template <int WT, int NMT>
__device__ __forceinline__ bool pair_valid_t(const SieveArgs &a, int nsel, const double *en, const float *en32,
                                             int64_t iq, int64_t ikq) {
    const float hm = a.hwmax32[iq];
    if (hm < 0.f) return false;
    float em[WT];
    load_kq_energies<WT>(a, ikq, em);
    return pair_valid_tail<WT, NMT>(a, nsel, en, en32, iq, ikq, hm, em);
}

__device__ __forceinline__ void load_window(const SieveArgs &a, int ik, int lo, int nsel,
                                            double *en, float *en32) {
    if (threadIdx.x < nsel) {
        en[threadIdx.x] = a.eps[(int64_t)ik * a.W + lo + threadIdx.x];
        en32[threadIdx.x] = a.eps32[(int64_t)ik * a.W + lo + threadIdx.x];
    }
    __syncthreads();
}

SieveArgs make_sieve_args(epwi_ctx *c);
