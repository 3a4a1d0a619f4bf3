// Iterative Boltzmann transport equation (Sec. II C, the iteration equation after Eq. 10).
//
// Gamma storage: the sieved pairs of the window in pair order (k-point major, as the sieve
// writes them), and for every pair (k, q) one block Gamma[n][m] over the window bands n of k
// and m of k+q, blocks back to back.  goff[pair] is the first entry of a pair's block.  The
// value stored is sum_nu |g|^2 [(N + f_m) e^{-x+^2/eta^2} + (1 + N - f_m) e^{-x-^2/eta^2}] (eV^2),
// the summand of Eq. 10 without its constant 2 pi / (hbar N_q sqrt(pi) eta), which the step
// applies once per state.
//
// After the capture each pair's q index is replaced in place by a step code: the first state
// of the final k-point's window (sb) and its band count (nw), (sb << 5) | nw.  The step then
// reads one word per pair and needs no grid arithmetic or table lookups.  The per-pair block
// offsets are needed only by the capture: afterwards the step keeps one offset per (k-point,
// warp range) (wbase) and the per-pair array is freed, so the resident index is the step code
// per pair plus 64 bytes per k-point.
//
// Step: one block per window k-point, eight warps splitting its pairs into contiguous ranges,
// the k-point's bands taken in register groups of 1, 2, 4 or 8 (the smallest that covers the
// crystal's bands) with the inner loop specialised to the group's exact band count.  With
// FP32 Gamma (split paths) the lanes accumulate and reduce in FP32 from an FP32 copy of F;
// the sum over warps, the per-state update and F itself are FP64.
// A warp takes 32 pairs at a time (the next 32 codes are loaded ahead); a warp scan of the
// block sizes n_k x n_{k+q} gives each lane its block, and the lane accumulates
// Gamma[n][m] F_{m,k+q} for its pair.  Per-state sums are reduced in a fixed order (lanes by a
// butterfly, then warps in index order), so the result does not depend on scheduling.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "epwi_internal.cuh"
#include "scatter.cuh"

namespace {

constexpr int kIbThreads = 256;
constexpr int kIbWarps = kIbThreads / 32;
constexpr int kIbMaxBands = 8;  // bands of k accumulated in registers at a time (at most)
constexpr int kPpl = 2;         // narrow-window path: pairs per lane whose loads are in flight together

// First Gamma entry of every (k-point, warp range) of k_ib_step (same range formula).
__global__ void k_ib_wbase(int64_t nkp, const int64_t *__restrict__ kp_pairs, const int64_t *__restrict__ goff,
                           int64_t *__restrict__ wbase) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nkp * kIbWarps) return;
    const int64_t kp = t / kIbWarps;
    const int w = (int)(t % kIbWarps);
    const int64_t p0 = kp_pairs[kp], np = kp_pairs[kp + 1] - p0;
    const int64_t wb = p0 + np * w / kIbWarps, we = p0 + np * (w + 1) / kIbWarps;
    wbase[t] = wb < we ? goff[wb] : 0;
}

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

// q index -> step code (sb << 5) | nw of the final k-point, in place; one block per k-point
__global__ void k_ib_encode(GridInfo g, const int *__restrict__ kpts, const int *__restrict__ win_n,
                            const int *__restrict__ kpos, const int64_t *__restrict__ kp_state,
                            const int64_t *__restrict__ kp_pairs, unsigned *__restrict__ code) {
    const int kp = blockIdx.x;
    const int ik = kpts[kp];
    for (int64_t p = kp_pairs[kp] + threadIdx.x; p < kp_pairs[kp + 1]; p += blockDim.x) {
        const int64_t ikq = kplusq(g, ik, (int)code[p]);
        const unsigned nw = (unsigned)win_n[ikq];
        const unsigned sb = nw ? (unsigned)kp_state[kpos[ikq]] : 0u;
        code[p] = (sb << 5) | nw;
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
    const int64_t *kp_state, *kp_pairs;
    const int64_t *wbase;                 // first Gamma entry of each (k-point, warp range)
    const unsigned *code;                 // per pair (sb << 5) | nw
    const GT *gam;
    const double *inv_tau, *F0, *Fin;
    double *Fout;
    const float4 *Fin32;                  // FP32 copy of Fin (split paths), w unused
    float4 *Fout32;
    double pref;                          // 2 pi / (hbar N_q sqrt(pi) eta), s^-1 per eV^2
    unsigned long long *red;              // [2] max |dF|, max |F| as bit patterns
    int narrow;                           // every window has <= 4 bands: narrow-window path
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

// The warp's pairs [wb, we) for the bands b0 .. b0+NBX-1 of the k-point: y[n] += sum over the
// pairs and final bands m of Gamma[b0+n][m] F_m.
template <typename GT, int NB, int NBX>
__device__ __forceinline__ void step_pairs(const StepArgs<GT> &a, int nsel, int b0, int64_t wb, int64_t we,
                                           int64_t off, int lane, typename Acc<GT>::T (&y)[NB][3]) {
    using AT = typename Acc<GT>::T;
    unsigned cnext = wb + lane < we ? __ldg(a.code + wb + lane) : 0u;
    for (int64_t pb = wb; pb < we; pb += 32) {
        const unsigned code = cnext;
        cnext = pb + 32 + lane < we ? __ldg(a.code + pb + 32 + lane) : 0u;
        const int nw = (int)(code & 31u);
        const int64_t sb = (int64_t)(code >> 5);
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
            AT fx, fy, fz;
            load_F(a, sb + j, fx, fy, fz);
#pragma unroll
            for (int n = 0; n < NBX; ++n) {
                const AT gv = (AT)__ldg(gb + n * nw + j);
                y[n][0] = fma(gv, fx, y[n][0]);
                y[n][1] = fma(gv, fy, y[n][1]);
                y[n][2] = fma(gv, fz, y[n][2]);
            }
        }
        off += tot;
    }
}

// Narrow windows (every k+q window <= JMAX bands, this group NBX bands): each lane takes PPL
// pairs per round (pairs pb + i*32 + lane), issues all their F and Gamma loads (predicated on
// the pair's band count) before any multiply, so PPL x JMAX loads are in flight per lane.
template <typename GT, int NB, int NBX, int JMAX, int PPL>
__device__ __forceinline__ void step_pairs_narrow(const StepArgs<GT> &a, int nsel, int b0, int64_t wb,
                                                  int64_t we, int64_t off, int lane,
                                                  typename Acc<GT>::T (&y)[NB][3]) {
    using AT = typename Acc<GT>::T;
    unsigned cnext[PPL];
#pragma unroll
    for (int i = 0; i < PPL; ++i) {
        const int64_t p = wb + i * 32 + lane;
        cnext[i] = p < we ? __ldg(a.code + p) : 0u;
    }
    for (int64_t pb = wb; pb < we; pb += 32 * PPL) {
        unsigned cd[PPL];
        int64_t base[PPL];
#pragma unroll
        for (int i = 0; i < PPL; ++i) {
            cd[i] = cnext[i];
            const int64_t p = pb + 32 * PPL + i * 32 + lane;
            cnext[i] = p < we ? __ldg(a.code + p) : 0u;
        }
#pragma unroll
        for (int i = 0; i < PPL; ++i) {
            const int size = nsel * (int)(cd[i] & 31u);
            int incl = size;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            base[i] = off + (incl - size);
            off += __shfl_sync(0xffffffffu, incl, 31);
        }
        AT f[PPL][JMAX][3], g[PPL][JMAX][NBX];
#pragma unroll
        for (int i = 0; i < PPL; ++i) {
            const int nw = (int)(cd[i] & 31u);
            const int64_t sb = (int64_t)(cd[i] >> 5);
#pragma unroll
            for (int j = 0; j < JMAX; ++j) {
                f[i][j][0] = f[i][j][1] = f[i][j][2] = 0;
#pragma unroll
                for (int n = 0; n < NBX; ++n) g[i][j][n] = 0;
                if (j < nw) {
                    load_F(a, sb + j, f[i][j][0], f[i][j][1], f[i][j][2]);
#pragma unroll
                    for (int n = 0; n < NBX; ++n) g[i][j][n] = (AT)__ldg(a.gam + base[i] + (int64_t)(b0 + n) * nw + j);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < PPL; ++i)
#pragma unroll
            for (int j = 0; j < JMAX; ++j)
#pragma unroll
                for (int n = 0; n < NBX; ++n) {
                    y[n][0] = fma(g[i][j][n], f[i][j][0], y[n][0]);
                    y[n][1] = fma(g[i][j][n], f[i][j][1], y[n][1]);
                    y[n][2] = fma(g[i][j][n], f[i][j][2], y[n][2]);
                }
    }
}

template <typename GT, int kIbBands>
__global__ void __launch_bounds__(kIbThreads, kIbBands <= 2 ? 4 : (kIbBands <= 4 ? 3 : 2)) k_ib_step(StepArgs<GT> a) {
    using AT = typename Acc<GT>::T;
    __shared__ AT part[kIbWarps][kIbBands][3];
    const int kp = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int ik = a.kpts[kp];
    const int nsel = a.win_n[ik];
    const int64_t s0 = a.kp_state[kp];
    const int64_t p0 = a.kp_pairs[kp], np = a.kp_pairs[kp + 1] - p0;
    const int64_t wb = p0 + np * wid / kIbWarps, we = p0 + np * (wid + 1) / kIbWarps;
    const int64_t off = a.wbase[(int64_t)kp * kIbWarps + wid];
    double dmax = 0, fmax_ = 0;
    for (int b0 = 0; b0 < nsel; b0 += kIbBands) {
        const int nb = min(kIbBands, nsel - b0);
        AT y[kIbBands][3];
#pragma unroll
        for (int n = 0; n < kIbBands; ++n) y[n][0] = y[n][1] = y[n][2] = 0;
        // exact band count of this group (uniform over the block)
        // narrow-window path: FP32 Gamma and 4-band groups (the register budget of the other
        // instantiations has no room for its staged loads)
        constexpr bool kNarrow = std::is_same<GT, float>::value && kIbBands == 4;
        if (kNarrow && a.narrow && nb <= 2) {
            if constexpr (kNarrow) {
                if (nb == 1) step_pairs_narrow<GT, kIbBands, 1, 4, kPpl>(a, nsel, b0, wb, we, off, lane, y);
                else step_pairs_narrow<GT, kIbBands, 2, 4, kPpl>(a, nsel, b0, wb, we, off, lane, y);
            }
        } else switch (nb) {
        case 1: step_pairs<GT, kIbBands, 1>(a, nsel, b0, wb, we, off, lane, y); break;
        case 2: if constexpr (kIbBands >= 2) step_pairs<GT, kIbBands, 2>(a, nsel, b0, wb, we, off, lane, y); break;
        case 3: if constexpr (kIbBands >= 3) step_pairs<GT, kIbBands, 3>(a, nsel, b0, wb, we, off, lane, y); break;
        case 4: if constexpr (kIbBands >= 4) step_pairs<GT, kIbBands, 4>(a, nsel, b0, wb, we, off, lane, y); break;
        default:
            if constexpr (kIbBands > 4) step_pairs<GT, kIbBands, kIbBands>(a, nsel, b0, wb, we, off, lane, y);
            break;
        }
        // lanes: butterfly in the accumulation type; warps: FP64 in index order
#pragma unroll
        for (int n = 0; n < kIbBands; ++n) {
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
    if (threadIdx.x < 3 * kIbBands && (dmax > 0 || fmax_ > 0)) {
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
    a.kp_pairs = c->kp_pairs.as<int64_t>();
    a.wbase = c->ib_wbase.as<int64_t>();
    a.code = c->ib_pairs.as<unsigned>();
    a.gam = c->ib_gam.as<GT>();
    a.inv_tau = c->inv_tau.as<double>();
    a.F0 = c->ib_F0.as<double>();
    a.Fin = Fin;
    a.Fout = Fout;
    a.Fin32 = Fin32;
    a.Fout32 = Fout32;
    a.pref = 2.0 * epc::kPi / epc::kHbarEVs / (double)c->nk / (sqrt(epc::kPi) * c->eta);
    a.narrow = c->nw <= 4;
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
    c->ib_gam.ensure(eb * (size_t)(nent + 1));
    // the fp32 mode writes only the bands it does not skip (the others are exactly zero)
    if (c->opt.precision == EPWI_FP32)
        EPWI_CUDA(cudaMemsetAsync(c->ib_gam.p, 0, eb * (size_t)(nent + 1), c->stream));
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
    // the captured pairs' q indices become step codes (the capture is done with them), and the
    // per-pair offsets become one offset per (k-point, warp range)
    EPWI_REQUIRE(ns < (int64_t(1) << 27), EPWI_EUNSUPPORTED, "iterative BTE needs fewer than 2^27 states");
    c->ib_wbase.ensure(sizeof(int64_t) * (c->nkp * kIbWarps + 1));
    if (c->nkp > 0) {
        const int64_t nt = c->nkp * kIbWarps;
        k_ib_wbase<<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(
            c->nkp, c->kp_pairs.as<int64_t>(), c->ib_goff.as<int64_t>(), c->ib_wbase.as<int64_t>());
        EPWI_CHECK_LAUNCH();
    }
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    c->ib_goff.release();
    if (c->nkp > 0) {
        k_ib_encode<<<(unsigned)c->nkp, 256, 0, c->stream>>>(
            make_grid_info(c), c->kpts.as<int>(), c->win_n.as<int>(), c->ib_kpos.as<int>(),
            c->kp_state.as<int64_t>(), c->kp_pairs.as<int64_t>(), c->ib_pairs.as<unsigned>());
        EPWI_CHECK_LAUNCH();
    }
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
    // one step reads the pair codes and Gamma once, F0, 1/tau and F at the states, writes F
    c->ib_stats.bytes_per_step = 4.0 * (double)c->npairs +
                                 (double)c->ib_stats.entry_bytes * (double)c->ib_stats.n_entries +
                                 8.0 * (double)ns * (3 + 1 + 3 + 3);
}
