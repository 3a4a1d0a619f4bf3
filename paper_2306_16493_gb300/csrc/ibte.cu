// Iterative Boltzmann transport equation (Sec. II C, the iteration equation after Eq. 10).
//
// Gamma storage: the sieved pairs of the window in pair order (k-point major, as the sieve
// writes them), and for every pair (k, q) one block Gamma[n][m] over the window bands n of k
// and m of k+q, blocks back to back.  goff[pair] is the first entry of a pair's block.  The
// value stored is sum_nu |g|^2 [(N + f_m) e^{-x+^2/eta^2} + (1 + N - f_m) e^{-x-^2/eta^2}] (eV^2),
// the summand of Eq. 10 without its constant 2 pi / (hbar N_q sqrt(pi) eta), which the step
// applies once per state.
//
// After the capture every Gamma entry gets a 4-byte column word: the index of its final state
// (k+q, m) in the window's state list and the band n of k, (s << 5) | n.  The step is then a
// sparse product over entries, Gamma_e F_s accumulated into the row of band n of k: it reads one
// column word and one value per entry, gathers F at s, and needs no grid arithmetic or table
// lookups.  The pair list and the per-pair block offsets serve only the capture and are freed
// afterwards, so the resident index is the column word per entry plus 8 bytes per k-point
// (half the bytes of FP64 Gamma, equal to those of FP32 Gamma).
//
// Step: one block per window k-point, its entries split into eight contiguous warp ranges;
// lanes take entries 32 apart, several at a time with their loads issued together (coalesced
// column and value loads, F gathers from a table that stays in L2).  The k-point's bands are
// accumulated in registers in groups of 1, 2, 4 or 8 (the smallest covering the crystal's
// bands) with the band selection specialised to the window's exact band count (none for one
// band).  With FP32 Gamma (split paths) the lanes accumulate and reduce in FP32 from an FP32
// copy of F; the sum over warps, the per-state update and F itself are FP64.  Per-state sums
// are reduced in a fixed order (lanes by a butterfly, then warps in index order), so the result
// does not depend on scheduling.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "epwi_internal.cuh"
#include "scatter.cuh"

namespace {

constexpr int kIbThreads = 256;
constexpr int kIbWarps = kIbThreads / 32;
constexpr int kIbMaxBands = 8;  // bands of k accumulated in registers at a time (at most)
constexpr int kIbUnroll = 4;    // entries per lane whose loads are issued together

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

// Column words of the Gamma entries: entry goff[p] + n nw + j of pair p = (k, q) gets
// ((s + j) << 5) | n, s the first window state of k+q, j its band, n the band of k; and the
// first entry of every window k-point (ent[nkp] = the entry count).  One block per k-point.
__global__ void k_ib_columns(GridInfo g, int64_t nkp, const int *__restrict__ kpts, const int *__restrict__ win_n,
                             const int *__restrict__ kpos, const int64_t *__restrict__ kp_state,
                             const int64_t *__restrict__ kp_pairs, const int *__restrict__ pairs,
                             const int64_t *__restrict__ goff, unsigned *__restrict__ col,
                             int64_t *__restrict__ ent) {
    const int kp = blockIdx.x;
    const int ik = kpts[kp];
    const int nsel = win_n[ik];
    for (int64_t p = kp_pairs[kp] + threadIdx.x; p < kp_pairs[kp + 1]; p += blockDim.x) {
        const int64_t ikq = kplusq(g, ik, pairs[p]);
        const int nw = win_n[ikq];
        if (nw == 0) continue;
        const unsigned sb = (unsigned)kp_state[kpos[ikq]];
        unsigned *c = col + goff[p];
        for (int n = 0; n < nsel; ++n)
            for (int j = 0; j < nw; ++j) c[n * nw + j] = ((sb + (unsigned)j) << 5) | (unsigned)n;
    }
    if (threadIdx.x == 0) {
        ent[kp] = goff[kp_pairs[kp]];
        if (kp == nkp - 1) ent[nkp] = goff[kp_pairs[nkp]];
    }
}

// F0 = v tau (tau = 1 / (1/tau), 0 where 1/tau = 0); F = F0
__global__ void k_ib_f0(int64_t ns, int W, const int *__restrict__ st_k, const int *__restrict__ st_n,
                        const double *__restrict__ inv_tau, const double *__restrict__ vel,
                        double *__restrict__ F0, double *__restrict__ F, float4 *__restrict__ F32) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const double r = inv_tau[s];
    const double tau = r > 0 ? 1.0 / r : 0.0;
    const int64_t idx = (int64_t)st_k[s] * W + st_n[s];
    float4 f32 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int a = 0; a < 3; ++a) {
        const double f = vel[idx * 3 + a] * tau;
        F0[s * 3 + a] = f;
        F[s * 3 + a] = f;
        reinterpret_cast<float *>(&f32)[a] = (float)f;
    }
    if (F32) F32[s] = f32;
}

template <typename GT>
struct StepArgs {
    const int *kpts, *win_n;
    const int64_t *kp_state;
    const int64_t *ent;                   // first Gamma entry of each window k-point
    const unsigned *col;                  // per entry ((final state) << 5) | band of k
    const GT *gam;
    const double *inv_tau, *F0, *Fin;
    double *Fout;
    const float4 *Fin32;                  // FP32 copy of Fin (split paths), w unused
    float4 *Fout32;
    double pref;                          // 2 pi / (hbar N_q sqrt(pi) eta), s^-1 per eV^2
    unsigned long long *red;              // [2] max |dF|, max |F| as bit patterns
};

// Accumulation type of the lane and warp sums: FP64 with FP64 Gamma; FP32 with FP32 Gamma
// (GB300 issues FP64 at 1/64 of the FP32 rate, so FP64 sums would bind the split paths on
// the FP64 pipe).  The sum over warps is FP64.
template <typename GT> struct Acc { using T = double; };
template <> struct Acc<float> { using T = float; };

__device__ __forceinline__ void load_F(const StepArgs<double> &a, int64_t s, double &x, double &y, double &z) {
    const double *f = a.Fin + s * 3;
    x = __ldg(f);
    y = __ldg(f + 1);
    z = __ldg(f + 2);
}
__device__ __forceinline__ void load_F(const StepArgs<float> &a, int64_t s, float &x, float &y, float &z) {
    const float4 f = __ldg(a.Fin32 + s);
    x = f.x;
    y = f.y;
    z = f.z;
}

// The warp's entries [e0, e1) for the bands b0 .. b0+NBX-1 of the k-point: y[n] += Gamma_e F_s
// for every entry e whose column word holds state s and band b0 + n.  Lane l takes entries
// e0 + l, e0 + l + 32, ...; kIbUnroll of them have their column, value and F loads issued
// before their multiplies.  ALL: every entry's band lies in the group (one group covers the
// window); otherwise an entry of another group adds zero products.
template <typename GT, int NB, int NBX, bool ALL>
__device__ __forceinline__ void step_entries(const StepArgs<GT> &a, int b0, int64_t e0, int64_t e1, int lane,
                                             typename Acc<GT>::T (&y)[NB][3]) {
    using AT = typename Acc<GT>::T;
    for (int64_t eb = e0 + lane; eb < e1; eb += 32 * kIbUnroll) {
        unsigned cw[kIbUnroll];
        AT g[kIbUnroll], fx[kIbUnroll], fy[kIbUnroll], fz[kIbUnroll];
#pragma unroll
        for (int u = 0; u < kIbUnroll; ++u) {
            const int64_t e = eb + 32 * u;
            cw[u] = e < e1 ? __ldg(a.col + e) : 0u;
            g[u] = e < e1 ? (AT)__ldg(a.gam + e) : AT(0);
        }
#pragma unroll
        for (int u = 0; u < kIbUnroll; ++u) load_F(a, (int64_t)(cw[u] >> 5), fx[u], fy[u], fz[u]);
#pragma unroll
        for (int u = 0; u < kIbUnroll; ++u) {
            if constexpr (NBX == 1 && ALL) {
                y[0][0] = fma(g[u], fx[u], y[0][0]);
                y[0][1] = fma(g[u], fy[u], y[0][1]);
                y[0][2] = fma(g[u], fz[u], y[0][2]);
            } else {
                const int n = (int)(cw[u] & 31u) - b0;
#pragma unroll
                for (int b = 0; b < NBX; ++b) {
                    const AT gb = n == b ? g[u] : AT(0);
                    y[b][0] = fma(gb, fx[u], y[b][0]);
                    y[b][1] = fma(gb, fy[u], y[b][1]);
                    y[b][2] = fma(gb, fz[u], y[b][2]);
                }
            }
        }
    }
}

template <typename GT, int NB, int NBX>
__device__ __forceinline__ void step_group(const StepArgs<GT> &a, bool all, int b0, int64_t e0, int64_t e1, int lane,
                                           typename Acc<GT>::T (&y)[NB][3]) {
    if (all) step_entries<GT, NB, NBX, true>(a, b0, e0, e1, lane, y);
    else step_entries<GT, NB, NBX, false>(a, b0, e0, e1, lane, y);
}

// One block per window k-point; its entries split into eight contiguous warp ranges.  The
// k-point's bands are taken in groups of NB (the smallest of 1, 2, 4, 8 covering the crystal's
// bands; wider windows loop over groups).  Lanes reduce by a butterfly in the accumulation
// type, warps in index order in FP64, so the result does not depend on scheduling.  Entry 0 of
// an unused column word (col 0, value 0) adds exactly zero.
template <typename GT, int NB>
__global__ void __launch_bounds__(kIbThreads, NB <= 4 ? 4 : 2) k_ib_step(StepArgs<GT> a) {
    using AT = typename Acc<GT>::T;
    __shared__ AT part[kIbWarps][NB][3];
    const int kp = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int ik = a.kpts[kp];
    const int nsel = a.win_n[ik];
    const int64_t s0 = a.kp_state[kp];
    const int64_t q0 = a.ent[kp], ne = a.ent[kp + 1] - q0;
    const int64_t e0 = q0 + ne * wid / kIbWarps, e1 = q0 + ne * (wid + 1) / kIbWarps;
    double dmax = 0, fmax_ = 0;
    for (int b0 = 0; b0 < nsel; b0 += NB) {
        const int nb = min(NB, nsel - b0);
        AT y[NB][3];
#pragma unroll
        for (int n = 0; n < NB; ++n) y[n][0] = y[n][1] = y[n][2] = 0;
        // exact band count of this group (uniform over the block)
        const bool all = nsel <= NB;
        switch (nb) {
        case 1: step_group<GT, NB, 1>(a, all, b0, e0, e1, lane, y); break;
        case 2: if constexpr (NB >= 2) step_group<GT, NB, 2>(a, all, b0, e0, e1, lane, y); break;
        case 3: if constexpr (NB >= 3) step_group<GT, NB, 3>(a, all, b0, e0, e1, lane, y); break;
        case 4: if constexpr (NB >= 4) step_group<GT, NB, 4>(a, all, b0, e0, e1, lane, y); break;
        default: if constexpr (NB > 4) step_group<GT, NB, NB>(a, all, b0, e0, e1, lane, y); break;
        }
#pragma unroll
        for (int n = 0; n < NB; ++n) {
            if (n >= nb) break;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                AT v = y[n][c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) part[wid][n][c] = v;
            }
        }
        __syncthreads();
        if (threadIdx.x < nb * 3) {
            const int n = threadIdx.x / 3, c = threadIdx.x % 3;
            double sum = 0;
#pragma unroll
            for (int w = 0; w < kIbWarps; ++w) sum += (double)part[w][n][c];
            const int64_t s = s0 + b0 + n;
            const double r = a.inv_tau[s];
            const double tau = r > 0 ? 1.0 / r : 0.0;
            const double f = a.F0[s * 3 + c] + tau * (a.pref * sum);
            a.Fout[s * 3 + c] = f;
            if (a.Fout32) reinterpret_cast<float *>(a.Fout32 + s)[c] = (float)f;
            dmax = fmax(dmax, fabs(f - a.Fin[s * 3 + c]));
            fmax_ = fmax(fmax_, fabs(f));
        }
        __syncthreads();
    }
    // max is order independent: the bit patterns of non-negative doubles order like the values
    if (threadIdx.x < 3 * NB && (dmax > 0 || fmax_ > 0)) {
        atomicMax(&a.red[0], (unsigned long long)__double_as_longlong(dmax));
        atomicMax(&a.red[1], (unsigned long long)__double_as_longlong(fmax_));
    }
}

template <typename GT>
void launch_step(epwi_ctx *c, const double *Fin, double *Fout, const float4 *Fin32, float4 *Fout32) {
    StepArgs<GT> a;
    a.kpts = c->kpts.as<int>();
    a.win_n = c->win_n.as<int>();
    a.kp_state = c->kp_state.as<int64_t>();
    a.ent = c->ib_ent.as<int64_t>();
    a.col = c->ib_col.as<unsigned>();
    a.gam = c->ib_gam.as<GT>();
    a.inv_tau = c->inv_tau.as<double>();
    a.F0 = c->ib_F0.as<double>();
    a.Fin = Fin;
    a.Fout = Fout;
    a.Fin32 = Fin32;
    a.Fout32 = Fout32;
    a.pref = 2.0 * epc::kPi / epc::kHbarEVs / (double)c->nk / (sqrt(epc::kPi) * c->eta);
    a.red = c->ib_red.as<unsigned long long>();
    // band group: the smallest of 1, 2, 4, 8 covering the bands (wider windows loop)
    const unsigned grid = (unsigned)c->nkp;
    if (c->nw <= 1) k_ib_step<GT, 1><<<grid, kIbThreads, 0, c->stream>>>(a);
    else if (c->nw <= 2) k_ib_step<GT, 2><<<grid, kIbThreads, 0, c->stream>>>(a);
    else if (c->nw <= 4) k_ib_step<GT, 4><<<grid, kIbThreads, 0, c->stream>>>(a);
    else k_ib_step<GT, kIbMaxBands><<<grid, kIbThreads, 0, c->stream>>>(a);
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
    const size_t gam_bytes = eb * (size_t)(nent + 1);
    c->ib_gam.ensure(gam_bytes);
    // the fp32 mode writes only the bands it does not skip (the others are exactly zero)
    if (c->opt.precision == EPWI_FP32) EPWI_CUDA(cudaMemsetAsync(c->ib_gam.p, 0, gam_bytes, c->stream));
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
    if (!fp64) {
        c->ib_F32.ensure(sizeof(float4) * (ns + 1));
        c->ib_Fn32.ensure(sizeof(float4) * (ns + 1));
    }
    c->ib_red.ensure(sizeof(unsigned long long) * 2);
    // the step's index: one column word per Gamma entry and the first entry of every k-point;
    // the pair list and per-pair offsets are needed only by the capture and are freed here
    EPWI_REQUIRE(ns < (int64_t(1) << 27), EPWI_EUNSUPPORTED, "iterative BTE needs fewer than 2^27 states");
    const int64_t nkp = c->nkp, nent = c->ib_stats.n_entries;
    c->ib_ent.ensure(sizeof(int64_t) * (nkp + 1));
    c->ib_col.ensure(sizeof(unsigned) * (nent + 1));
    if (nkp > 0) {
        k_ib_columns<<<(unsigned)nkp, 256, 0, c->stream>>>(
            make_grid_info(c), nkp, c->kpts.as<int>(), c->win_n.as<int>(), c->ib_kpos.as<int>(),
            c->kp_state.as<int64_t>(), c->kp_pairs.as<int64_t>(), c->ib_pairs.as<int>(), c->ib_goff.as<int64_t>(),
            c->ib_col.as<unsigned>(), c->ib_ent.as<int64_t>());
        EPWI_CHECK_LAUNCH();
    }
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    c->ib_goff.release();
    c->ib_pairs.release();
    if (ns > 0) {
        k_ib_f0<<<(unsigned)((ns + 255) / 256), 256, 0, c->stream>>>(
            ns, c->nw, c->st_k.as<int>(), c->st_n.as<int>(), c->inv_tau.as<double>(), c->vel.as<double>(),
            c->ib_F0.as<double>(), c->ib_F.as<double>(), fp64 ? nullptr : c->ib_F32.as<float4>());
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
            if (fp64) launch_step<double>(c, c->ib_F.as<double>(), c->ib_Fn.as<double>(), nullptr, nullptr);
            else launch_step<float>(c, c->ib_F.as<double>(), c->ib_Fn.as<double>(), c->ib_F32.as<float4>(),
                                    c->ib_Fn32.as<float4>());
            EPWI_CUDA(cudaEventRecord(e1, c->stream));
            EPWI_CUDA(cudaMemcpyAsync(h, c->ib_red.p, sizeof(unsigned long long) * 2, cudaMemcpyDeviceToHost,
                                      c->stream));
            EPWI_CUDA(cudaStreamSynchronize(c->stream));
            float ms = 0;
            EPWI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            ms_steps += ms;
            ++it;
            std::swap(c->ib_F, c->ib_Fn);
            std::swap(c->ib_F32, c->ib_Fn32);
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
    // one step reads the column words and Gamma once, F0, 1/tau and F at the states, writes F
    c->ib_stats.index_bytes = 4 * nent + 8 * (nkp + 1);
    c->ib_stats.bytes_per_step = (double)c->ib_stats.index_bytes +
                                 (double)c->ib_stats.entry_bytes * (double)c->ib_stats.n_entries +
                                 8.0 * (double)ns * (3 + 1 + 3 + 3);
}
