// Iterative Boltzmann transport equation (Sec. II C, the iteration equation after Eq. 10).
//
// Gamma storage: the sieved pairs of the window in pair order (k-point major, as the sieve
// writes them), and for every pair (k, q) one block Gamma[n][m] over the window bands n of k
// and m of k+q, blocks back to back.  goff[pair] is the first entry of a pair's block.  The
// value stored is sum_nu |g|^2 [(N + f_m) e^{-x+^2/eta^2} + (1 + N - f_m) e^{-x-^2/eta^2}] (eV^2),
// the summand of Eq. 10 without its constant 2 pi / (hbar N_q sqrt(pi) eta), which the step
// applies once per state.
//
// Step: one block per window k-point, four warps splitting its pairs into contiguous ranges.
// A warp takes 32 pairs at a time; a warp scan of the block sizes n_k x n_{k+q} gives each
// lane its block, and the lane accumulates Gamma[n][m] F_{m,k+q} for its pair.  Per-state
// sums are reduced in a fixed order (lanes by a butterfly, then warps in index order), so the
// result does not depend on scheduling.
#include <algorithm>
#include <cstring>

#include "epwi_internal.cuh"
#include "scatter.cuh"

namespace {

constexpr int kIbThreads = 128;
constexpr int kIbWarps = kIbThreads / 32;
constexpr int kIbBands = 8;     // bands of k accumulated in registers at a time

__global__ void k_ib_kpos(int64_t nkp, const int *__restrict__ kpts, int *__restrict__ kpos) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nkp) kpos[kpts[p]] = (int)p;
}

// sizes[pair] = n_window(k) x n_window(k+q); one block per window k-point
__global__ void k_ib_sizes(GridInfo g, const int *__restrict__ kpts, const int *__restrict__ win_n,
                           const int64_t *__restrict__ kp_pairs, const int *__restrict__ pairs,
                           int64_t *__restrict__ sizes) {
    const int kp = blockIdx.x;
    const int ik = kpts[kp];
    const int nsel = win_n[ik];
    for (int64_t p = kp_pairs[kp] + threadIdx.x; p < kp_pairs[kp + 1]; p += blockDim.x)
        sizes[p] = (int64_t)nsel * win_n[kplusq(g, ik, pairs[p])];
}

// F0 = v tau (tau = 1 / (1/tau), 0 where 1/tau = 0); F = F0
__global__ void k_ib_f0(int64_t ns, int W, const int *__restrict__ st_k, const int *__restrict__ st_n,
                        const double *__restrict__ inv_tau, const double *__restrict__ vel,
                        double *__restrict__ F0, double *__restrict__ F) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const double r = inv_tau[s];
    const double tau = r > 0 ? 1.0 / r : 0.0;
    const int64_t idx = (int64_t)st_k[s] * W + st_n[s];
    for (int a = 0; a < 3; ++a) {
        const double f = vel[idx * 3 + a] * tau;
        F0[s * 3 + a] = f;
        F[s * 3 + a] = f;
    }
}

template <typename GT>
struct StepArgs {
    GridInfo g;
    const int *kpts, *win_n, *kpos;
    const int64_t *kp_state, *kp_pairs, *goff;
    const int *pairs;
    const GT *gam;
    const double *inv_tau, *F0, *Fin;
    double *Fout;
    double pref;                          // 2 pi / (hbar N_q sqrt(pi) eta), s^-1 per eV^2
    unsigned long long *red;              // [2] max |dF|, max |F| as bit patterns
};

template <typename GT>
__global__ void __launch_bounds__(kIbThreads) k_ib_step(StepArgs<GT> a) {
    __shared__ double part[kIbWarps][kIbBands][3];
    const int kp = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int ik = a.kpts[kp];
    const int nsel = a.win_n[ik];
    const int64_t s0 = a.kp_state[kp];
    const int64_t p0 = a.kp_pairs[kp], np = a.kp_pairs[kp + 1] - p0;
    const int64_t wb = p0 + np * wid / kIbWarps, we = p0 + np * (wid + 1) / kIbWarps;
    double dmax = 0, fmax_ = 0;
    for (int b0 = 0; b0 < nsel; b0 += kIbBands) {
        const int nb = min(kIbBands, nsel - b0);
        double y[kIbBands][3];
#pragma unroll
        for (int n = 0; n < kIbBands; ++n) y[n][0] = y[n][1] = y[n][2] = 0;
        int64_t off = wb < we ? a.goff[wb] : 0;
        for (int64_t pb = wb; pb < we; pb += 32) {
            const int64_t p = pb + lane;
            int nw = 0;
            int64_t sb = 0;
            if (p < we) {
                const int64_t ikq = kplusq(a.g, ik, a.pairs[p]);
                nw = a.win_n[ikq];
                if (nw > 0) sb = a.kp_state[a.kpos[ikq]];
            }
            const int size = nsel * nw;
            int incl = size;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            const GT *gb = a.gam + off + (incl - size) + (int64_t)b0 * nw;
            for (int j = 0; j < nw; ++j) {
                const double fx = a.Fin[(sb + j) * 3], fy = a.Fin[(sb + j) * 3 + 1],
                             fz = a.Fin[(sb + j) * 3 + 2];
#pragma unroll
                for (int n = 0; n < kIbBands; ++n) {
                    if (n < nb) {
                        const double gv = (double)gb[n * nw + j];
                        y[n][0] = fma(gv, fx, y[n][0]);
                        y[n][1] = fma(gv, fy, y[n][1]);
                        y[n][2] = fma(gv, fz, y[n][2]);
                    }
                }
            }
            off += tot;
        }
#pragma unroll
        for (int n = 0; n < kIbBands; ++n)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double v = y[n][c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) part[wid][n][c] = v;
            }
        __syncthreads();
        if (threadIdx.x < nb * 3) {
            const int n = threadIdx.x / 3, c = threadIdx.x % 3;
            const double sum = (part[0][n][c] + part[1][n][c]) + (part[2][n][c] + part[3][n][c]);
            const int64_t s = s0 + b0 + n;
            const double r = a.inv_tau[s];
            const double tau = r > 0 ? 1.0 / r : 0.0;
            const double f = a.F0[s * 3 + c] + tau * (a.pref * sum);
            a.Fout[s * 3 + c] = f;
            dmax = fmax(dmax, fabs(f - a.Fin[s * 3 + c]));
            fmax_ = fmax(fmax_, fabs(f));
        }
        __syncthreads();
    }
    // max is order independent: the bit patterns of non-negative doubles order like the values
    if (threadIdx.x < 3 * kIbBands && (dmax > 0 || fmax_ > 0)) {
        atomicMax(&a.red[0], (unsigned long long)__double_as_longlong(dmax));
        atomicMax(&a.red[1], (unsigned long long)__double_as_longlong(fmax_));
    }
}

template <typename GT>
void launch_step(epwi_ctx *c, const double *Fin, double *Fout) {
    StepArgs<GT> a;
    a.g = make_grid_info(c);
    a.kpts = c->kpts.as<int>();
    a.win_n = c->win_n.as<int>();
    a.kpos = c->ib_kpos.as<int>();
    a.kp_state = c->kp_state.as<int64_t>();
    a.kp_pairs = c->kp_pairs.as<int64_t>();
    a.goff = c->ib_goff.as<int64_t>();
    a.pairs = c->ib_pairs.as<int>();
    a.gam = c->ib_gam.as<GT>();
    a.inv_tau = c->inv_tau.as<double>();
    a.F0 = c->ib_F0.as<double>();
    a.Fin = Fin;
    a.Fout = Fout;
    a.pref = 2.0 * epc::kPi / epc::kHbarEVs / (double)c->nk / (sqrt(epc::kPi) * c->eta);
    a.red = c->ib_red.as<unsigned long long>();
    k_ib_step<GT><<<(unsigned)c->nkp, kIbThreads, 0, c->stream>>>(a);
    EPWI_CHECK_LAUNCH();
}

}  // namespace

// Pair list, Gamma layout and storage for the window of the current call; the caller then
// runs the interpolation over the returned work set (which also fills inv_tau).
void ibte_prepare(epwi_ctx *c, WorkSet &ws) {
    const int64_t nkp = c->nkp, npairs = c->npairs;
    const bool fp64 = c->opt.precision == EPWI_FP64;
    c->ib_pairs.ensure(sizeof(int) * (npairs + 1));
    sieve_fill_chunk(c, 0, nkp, c->ib_pairs.as<int>());
    c->ib_kpos.ensure(sizeof(int) * c->nk);
    EPWI_CUDA(cudaMemsetAsync(c->ib_kpos.p, 0xff, sizeof(int) * c->nk, c->stream));
    if (nkp > 0) {
        k_ib_kpos<<<(unsigned)((nkp + 255) / 256), 256, 0, c->stream>>>(nkp, c->kpts.as<int>(),
                                                                      c->ib_kpos.as<int>());
        EPWI_CHECK_LAUNCH();
    }
    c->ib_goff.ensure(sizeof(int64_t) * (npairs + 1));
    int64_t nent = 0;
    {
        DevBuf sizes;
        try {
            sizes.ensure(sizeof(int64_t) * (npairs + 1));
            if (nkp > 0) {
                k_ib_sizes<<<(unsigned)nkp, 256, 0, c->stream>>>(
                    make_grid_info(c), c->kpts.as<int>(), c->win_n.as<int>(), c->kp_pairs.as<int64_t>(),
                    c->ib_pairs.as<int>(), sizes.as<int64_t>());
                EPWI_CHECK_LAUNCH();
            }
            scan_exclusive_i64(c, sizes.as<int64_t>(), c->ib_goff.as<int64_t>(), npairs, &nent);
        } catch (...) {
            sizes.release();
            throw;
        }
        sizes.release();
    }
    const size_t eb = fp64 ? sizeof(double) : sizeof(float);
    c->ib_gam.ensure(eb * (size_t)(nent + 1));
    c->ib_stats.n_entries = nent;
    c->ib_stats.entry_bytes = (int32_t)eb;
    ws.pairs_dev = c->ib_pairs.as<int>();
    ws.goff = c->ib_goff.as<int64_t>();
    if (fp64) ws.gam64 = c->ib_gam.as<double>();
    else ws.gam32 = c->ib_gam.as<float>();
}

// Iterates from F0 = v tau; leaves the last iterate in c->ib_F.
void ibte_iterate(epwi_ctx *c, int max_iter, double tol) {
    const int64_t ns = c->nstates;
    const bool fp64 = c->opt.precision == EPWI_FP64;
    c->ib_F0.ensure(sizeof(double) * 3 * (ns + 1));
    c->ib_F.ensure(sizeof(double) * 3 * (ns + 1));
    c->ib_Fn.ensure(sizeof(double) * 3 * (ns + 1));
    c->ib_red.ensure(sizeof(unsigned long long) * 2);
    if (ns > 0) {
        k_ib_f0<<<(unsigned)((ns + 255) / 256), 256, 0, c->stream>>>(
            ns, c->nw, c->st_k.as<int>(), c->st_n.as<int>(), c->inv_tau.as<double>(), c->vel.as<double>(),
            c->ib_F0.as<double>(), c->ib_F.as<double>());
        EPWI_CHECK_LAUNCH();
    }
    cudaEvent_t e0, e1;
    EPWI_CUDA(cudaEventCreate(&e0));
    EPWI_CUDA(cudaEventCreate(&e1));
    unsigned long long *h = nullptr;
    auto cleanup = [&] {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (h) cudaFreeHost(h);
    };
    int it = 0;
    double change = 0, ms_steps = 0;
    try {
        EPWI_CUDA(cudaMallocHost(&h, sizeof(unsigned long long) * 2));
        for (it = 0; it < max_iter && c->nkp > 0;) {
            EPWI_CUDA(cudaMemsetAsync(c->ib_red.p, 0, sizeof(unsigned long long) * 2, c->stream));
            EPWI_CUDA(cudaEventRecord(e0, c->stream));
            if (fp64) launch_step<double>(c, c->ib_F.as<double>(), c->ib_Fn.as<double>());
            else launch_step<float>(c, c->ib_F.as<double>(), c->ib_Fn.as<double>());
            EPWI_CUDA(cudaEventRecord(e1, c->stream));
            EPWI_CUDA(cudaMemcpyAsync(h, c->ib_red.p, sizeof(unsigned long long) * 2, cudaMemcpyDeviceToHost,
                                      c->stream));
            EPWI_CUDA(cudaStreamSynchronize(c->stream));
            float ms = 0;
            EPWI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            ms_steps += ms;
            ++it;
            std::swap(c->ib_F, c->ib_Fn);
            double dmax, fmax_;
            std::memcpy(&dmax, &h[0], sizeof(double));
            std::memcpy(&fmax_, &h[1], sizeof(double));
            EPWI_REQUIRE(std::isfinite(dmax) && std::isfinite(fmax_), EPWI_ENUMERIC,
                         "non-finite mean free path in the iteration");
            change = fmax_ > 0 ? dmax / fmax_ : 0.0;
            if (dmax <= tol * fmax_) break;
        }
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
    c->ib_stats.iters = it;
    c->ib_stats.change = change;
    c->ib_stats.ms_step = it > 0 ? ms_steps / it : 0.0;
    // one step reads the q list and Gamma once, F0, 1/tau and F at the states, writes F
    c->ib_stats.bytes_per_step = 4.0 * (double)c->npairs +
                                 (double)c->ib_stats.entry_bytes * (double)c->ib_stats.n_entries +
                                 8.0 * (double)ns * (3 + 1 + 3 + 3);
}
