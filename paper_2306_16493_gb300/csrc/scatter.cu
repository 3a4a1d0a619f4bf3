// On-the-fly EPWI + SERTA scattering rates, q-batched (Sec. III C-D, Eq. 16; Sec. II C,
// Eq. 10), with the FP64 kernels of the reference path and the chunk orchestration shared
// by every precision mode.
//
// Per k-point chunk:
//   1. sieve fill: the kept q of each k (ascending), built per chunk (Sec. III A sieve).
//   2. Re->k stage: ghat(k)[Rp][mu][i][n] = sum_j [sum_Re w e^{ik.Re} g_ij^mu(Re,Rp)] V_jn(k)
//      for the window bands n (the inner bracket (g P^el) U^dag(k) of Eq. 16).
//   3. Rp->q stage fused with the rotations and the delta sum, one thread per (k, q) pair:
//      G = sum_Rp e^{iq.Rp} ghat, g^nu_mn = sum_mu [sum_i conj(V_im(k+q)) G^mu_in] u_mu,nu(q),
//      rate_n += |g|^2 [(N + f) e^{-(x+/eta)^2} + (1 + N - f) e^{-(x-/eta)^2}] on |x| <= c eta.
//   4. fixed-order reduction of the 128-pair tile partials into 1/tau_nk.
#include <algorithm>

#include "epwi_internal.cuh"
#include "scatter.cuh"

namespace {

template <int WT, int KG>
__global__ void __launch_bounds__(128) k_restage_fp64(RestageArgs a) {
    constexpr int WM = WT ? WT : epc::kMaxW;
    const int W = WT ? WT : a.W;
    extern __shared__ double2 P[];   // [KG][nRe]
    const int kg0 = blockIdx.y * KG;
    for (int idx = threadIdx.x; idx < KG * a.nRe; idx += blockDim.x) {
        const int kk = idx / a.nRe, r = idx % a.nRe;
        double2 p = make_double2(0, 0);
        if (kg0 + kk < a.nkp) {
            int i1, i2, i3;
            grid_coords(a.g, a.kpts[kg0 + kk], i1, i2, i3);
            p = a.ph64[phase_index(i1 * a.g.s1 % a.g.L, i2 * a.g.s2 % a.g.L, i3 * a.g.s3 % a.g.L,
                                   a.Re[3 * r], a.Re[3 * r + 1], a.Re[3 * r + 2], a.g.L)];
        }
        P[idx] = p;
    }
    __syncthreads();
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= a.nrow) return;
    double2 acc[KG][WM];
    for (int kk = 0; kk < KG; ++kk)
        for (int j = 0; j < W; ++j) acc[kk][j] = make_double2(0, 0);
    const double2 *gw = a.gw64 + (size_t)row * W;
    for (int r = 0; r < a.nRe; ++r) {
        double2 gv[WM];
        for (int j = 0; j < W; ++j) gv[j] = gw[(size_t)r * a.nrow * W + j];
        for (int kk = 0; kk < KG; ++kk) {
            const double2 p = P[kk * a.nRe + r];
            for (int j = 0; j < W; ++j) acc[kk][j] = cfma(p, gv[j], acc[kk][j]);
        }
    }
    for (int kk = 0; kk < KG; ++kk) {
        if (kg0 + kk >= a.nkp) break;
        const int ik = a.kpts[kg0 + kk];
        const int lo = a.ovr_nsel >= 0 ? a.ovr_lo : a.win_lo[ik];
        const int ns = a.ovr_nsel >= 0 ? a.ovr_nsel : a.win_n[ik];
        const int64_t s0 = a.kp_state[kg0 + kk] - a.s_base;
        const double2 *Vk = a.V64 + (int64_t)ik * W * W;
        for (int np = 0; np < ns; ++np) {
            double2 o = make_double2(0, 0);
            for (int j = 0; j < W; ++j) o = cfma(acc[kk][j], Vk[j * W + lo + np], o);
            a.ghat64[(s0 + np) * a.nrow + row] = o;
        }
    }
}

template <int WT, int NMT, bool TERMS>
__global__ void __launch_bounds__(128) k_scatter_fp64(ScatterArgs a) {
    constexpr int WM = WT ? WT : epc::kMaxW;
    constexpr int NMM = NMT ? NMT : epc::kMaxNm;
    const int W = WT ? WT : a.W;
    const int Nm = NMT ? NMT : a.Nm;
    __shared__ double red[4][epc::kMaxW];
    const int4 t = a.tiles[blockIdx.x];
    const int kpl = t.x;
    const int64_t pair = (int64_t)t.y + threadIdx.x;
    const bool active = pair < t.z;
    const int ik = a.kpts[kpl];
    const int lo = a.ovr_nsel >= 0 ? a.ovr_lo : a.win_lo[ik];
    const int nsel = a.ovr_nsel >= 0 ? a.ovr_nsel : a.win_n[ik];
    const int64_t s0 = a.kp_state[kpl] - a.s_base;
    int iq = 0;
    int64_t ikq = 0;
    int a1 = 0, a2 = 0, a3 = 0;
    if (active) {
        iq = a.pairs[pair];
        ikq = kplusq(a.g, ik, iq);
        int i1, i2, i3;
        grid_coords(a.g, iq, i1, i2, i3);
        a1 = i1 * a.g.s1 % a.g.L;
        a2 = i2 * a.g.s2 % a.g.L;
        a3 = i3 * a.g.s3 % a.g.L;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int np = 0; np < nsel; ++np) {
        double rate = 0;
        double tacc[TERMS ? NMM : 1];
        if (TERMS)
            for (int nu = 0; nu < Nm; ++nu) tacc[nu] = 0;
        if (active) {
            double2 G[NMM][WM];
            for (int mu = 0; mu < Nm; ++mu)
                for (int i = 0; i < W; ++i) G[mu][i] = make_double2(0, 0);
            const double2 *gh = a.ghat64 + (s0 + np) * a.nrow;
            for (int rp = 0; rp < a.nRp; ++rp) {
                const double2 p = a.ph64[phase_index(a1, a2, a3, a.Rp[3 * rp], a.Rp[3 * rp + 1],
                                                     a.Rp[3 * rp + 2], a.g.L)];
                const double2 *gr = gh + (size_t)rp * Nm * W;
                for (int mu = 0; mu < Nm; ++mu)
                    for (int i = 0; i < W; ++i) G[mu][i] = cfma(p, gr[mu * W + i], G[mu][i]);
            }
            const double en = a.eps[(int64_t)ik * W + lo + np];
            const double2 *Vq = a.V64 + ikq * W * W;
            const double2 *uq = a.u64 + (int64_t)iq * Nm * Nm;
            const int lokq = a.gam64 ? a.win_lo[ikq] : 0, nwkq = a.gam64 ? a.win_n[ikq] : 0;
            for (int m = 0; m < W; ++m) {
                double gm = 0;                    // Gamma capture: sum over modes
                double2 h[NMM];
                for (int mu = 0; mu < Nm; ++mu) {
                    h[mu] = make_double2(0, 0);
                    for (int i = 0; i < W; ++i) h[mu] = cfmac(Vq[i * W + m], G[mu][i], h[mu]);
                }
                const double em = a.eps[ikq * W + m];
                const double fm = a.focc ? a.focc[ikq * W + m] : 0.0;
                for (int nu = 0; nu < Nm; ++nu) {
                    const double w = a.hw[(int64_t)iq * Nm + nu];
                    double2 gv = make_double2(0, 0);
                    for (int mu = 0; mu < Nm; ++mu) gv = cfma(h[mu], uq[mu * Nm + nu], gv);
                    const double g2 = gv.x * gv.x + gv.y * gv.y;
                    if (a.g2out) {
                        a.g2out[(((a.g2_base + pair) * nsel + np) * Nm + nu) * W + m] =
                            (w >= a.omega_min) ? g2 : 0.0;
                        continue;
                    }
                    if (!(w >= a.omega_min)) continue;
                    const double x1 = (en + w) - em;
                    const double x2 = (en - w) - em;
                    const double N = a.nocc[(int64_t)iq * Nm + nu];
                    double term = 0;
                    if (fabs(x1) <= a.ceta) {
                        const double y = x1 / a.eta;
                        term += (N + fm) * exp(-y * y);
                    }
                    if (fabs(x2) <= a.ceta) {
                        const double y = x2 / a.eta;
                        term += (1.0 + N - fm) * exp(-y * y);
                    }
                    if (TERMS) tacc[nu] += g2 * term;
                    else rate += g2 * term;
                    gm += g2 * term;
                }
                if (!TERMS && a.gam64 && m >= lokq && m < lokq + nwkq)
                    a.gam64[a.goff[pair] + (int64_t)np * nwkq + (m - lokq)] = gm;
            }
        }
        if (TERMS) {
            // terms mode: sum_m |g|^2 [(N + f) delta(x+) + (1 + N - f) delta(x-)] per mode
            if (active) {
                const double inv_norm = 1.0 / (sqrt(epc::kPi) * a.eta);
                double *o = a.tout + ((a.g2_base + pair) * a.tstride + np) * Nm;
                for (int nu = 0; nu < Nm; ++nu) o[nu] = tacc[nu] * inv_norm;
            }
            continue;
        }
        if (a.pair_w && active) rate *= a.pair_w[pair];
        for (int o = 16; o > 0; o >>= 1) rate += __shfl_down_sync(0xffffffffu, rate, o);
        if (lane == 0) red[wid][np] = rate;
    }
    __syncthreads();
    if (threadIdx.x < nsel)
        a.tile_part[(int64_t)blockIdx.x * epc::kMaxW + threadIdx.x] =
            (red[0][threadIdx.x] + red[1][threadIdx.x]) + (red[2][threadIdx.x] + red[3][threadIdx.x]);
}

__global__ void k_tiles_count(int64_t nkp, const int64_t *__restrict__ kp_pairs, int64_t p_base,
                              int64_t *__restrict__ ntile) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nkp) return;
    const int64_t n = kp_pairs[p + 1] - kp_pairs[p];
    ntile[p] = (n + epc::kTile - 1) / epc::kTile;
    (void)p_base;
}

__global__ void k_tiles_fill(int64_t nkp, const int64_t *__restrict__ kp_pairs, int64_t p_base,
                             const int64_t *__restrict__ kp_tile, int4 *__restrict__ tiles) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nkp) return;
    const int64_t b = kp_pairs[p] - p_base, e = kp_pairs[p + 1] - p_base;
    int64_t t = kp_tile[p];
    for (int64_t s = b; s < e; s += epc::kTile, ++t)
        tiles[t] = make_int4((int)p, (int)s, (int)min(e, s + (int64_t)epc::kTile), 0);
}

// 1/tau_nk = pref * sum over the k-point's tiles (in order) of the tile partials.
__global__ void k_reduce_tiles(int64_t nkp, const int *__restrict__ kpts,
                               const int *__restrict__ win_n, const int64_t *__restrict__ kp_state,
                               const int64_t *__restrict__ kp_tile,
                               const double *__restrict__ part, double pref,
                               double *__restrict__ inv_tau) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nkp) return;
    const int ns = win_n[kpts[p]];
    for (int np = 0; np < ns; ++np) {
        double s = 0;
        for (int64_t t = kp_tile[p]; t < kp_tile[p + 1]; ++t) s += part[t * epc::kMaxW + np];
        inv_tau[kp_state[p] + np] = pref * s;
    }
}

template <int WT, int NMT>
void launch_fp64_pair(const RestageArgs &ra, const ScatterArgs &sa, int64_t ntiles, cudaStream_t st) {
    constexpr int KG = WT ? (WT >= 16 ? 1 : (WT >= 8 ? 4 : 8)) : 1;
    dim3 grid((ra.nrow + 127) / 128, (unsigned)((ra.nkp + KG - 1) / KG));
    const size_t sm = sizeof(double2) * KG * ra.nRe;
    if (sm > 48 * 1024)
        EPWI_CUDA(cudaFuncSetAttribute(k_restage_fp64<WT, KG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_restage_fp64<WT, KG><<<grid, 128, sm, st>>>(ra);
    EPWI_CHECK_LAUNCH();
    (void)sa;
    (void)ntiles;
}

template <int WT, int NMT>
void launch_fp64_scatter(const ScatterArgs &sa, int64_t ntiles, cudaStream_t st) {
    if (ntiles > 0) {
        if (sa.tout) k_scatter_fp64<WT, NMT, true><<<(unsigned)ntiles, 128, 0, st>>>(sa);
        else k_scatter_fp64<WT, NMT, false><<<(unsigned)ntiles, 128, 0, st>>>(sa);
        EPWI_CHECK_LAUNCH();
    }
}

void fp64_restage(const RestageArgs &ra, int W, cudaStream_t st) {
    if (W == 1) launch_fp64_pair<1, 0>(ra, ScatterArgs{}, 0, st);
    else if (W == 4) launch_fp64_pair<4, 0>(ra, ScatterArgs{}, 0, st);
    else if (W == 8) launch_fp64_pair<8, 0>(ra, ScatterArgs{}, 0, st);
    else launch_fp64_pair<0, 0>(ra, ScatterArgs{}, 0, st);
}

void fp64_scatter(const ScatterArgs &sa, int64_t ntiles, cudaStream_t st) {
    if (sa.W == 1 && sa.Nm == 3) launch_fp64_scatter<1, 3>(sa, ntiles, st);
    else if (sa.W == 4 && sa.Nm == 3) launch_fp64_scatter<4, 3>(sa, ntiles, st);
    else if (sa.W == 8 && sa.Nm == 6) launch_fp64_scatter<8, 6>(sa, ntiles, st);
    else launch_fp64_scatter<0, 0>(sa, ntiles, st);
}

struct Ev {
    cudaEvent_t e[2];
    Ev() { cudaEventCreate(&e[0]); cudaEventCreate(&e[1]); }
    ~Ev() { cudaEventDestroy(e[0]); cudaEventDestroy(e[1]); }
    float ms() { float m = 0; cudaEventElapsedTime(&m, e[0], e[1]); return m; }
};

}  // namespace

void sieve_fill_chunk(epwi_ctx *c, int64_t kp0, int64_t kp1, int *pairs);

// Processes the work set ws (k-points with their pair lists) chunk by chunk.  In rates mode
// it writes inv_tau for every state of the work set; in g2 mode (g2out != nullptr) it writes
// |g|^2 per pair instead.
namespace {

// One chunk of k-points kp0 .. kp1-1 of a work set: its pair list (chunk-local, q index per
// pair), the device pair offsets of its k-points (kp_pairs[kp - kp0] - p_off is the first
// local pair of kp), its global pair index base and its states.
struct ChunkView {
    int64_t kp0, kp1;
    const int *pairs;
    const int64_t *kp_pairs;
    int64_t p_off;
    int64_t np;
    int64_t g_base;                       // global index of the chunk's first pair
    int64_t s_base, ns;
};

struct StageTimers {
    Ev fill, re, sc, red;
};

// Tiles, Re->k, Rp->q with rotations and the delta sum, and the reduction of one chunk.
int64_t run_chunk(epwi_ctx *c, const WorkSet &ws, const ChunkView &cv, double *g2out, double *tout,
                  int tstride, StageTimers &tm) {
    const int W = c->nw, Nm = c->nm;
    const bool sf = c->opt.precision == EPWI_FP32;
    const bool tc = !sf && c->opt.precision != EPWI_FP64;
    const int nRp = tc ? tc_rp_count(c) : c->nRp;           // the split modes' view of R_p
    const int64_t nrow = (int64_t)nRp * Nm * W;
    const size_t state_bytes = sf ? sf_state_bytes(c) : tc ? tc_state_bytes(c) : sizeof(double2) * nrow;
    GridInfo g = make_grid_info(c);
    const int64_t nkpc = cv.kp1 - cv.kp0;
    // tiles (the fp32 mode works per (k-point, band) instead)
    int64_t nt = 0;
    if (!sf) {
        c->kp_tile.ensure(sizeof(int64_t) * (nkpc + 1));
        c->scan_tmp.ensure(sizeof(int64_t) * (nkpc + 1));
        k_tiles_count<<<(unsigned)((nkpc + 255) / 256), 256, 0, c->stream>>>(
            nkpc, cv.kp_pairs, cv.p_off, c->scan_tmp.as<int64_t>());
        EPWI_CHECK_LAUNCH();
        scan_exclusive_i64(c, c->scan_tmp.as<int64_t>(), c->kp_tile.as<int64_t>(), nkpc, &nt);
        c->tiles.ensure(sizeof(int4) * (nt + 1));
        c->tile_part.ensure(sizeof(double) * epc::kMaxW * (nt + 1));
        k_tiles_fill<<<(unsigned)((nkpc + 255) / 256), 256, 0, c->stream>>>(
            nkpc, cv.kp_pairs, cv.p_off, c->kp_tile.as<int64_t>(), c->tiles.as<int4>());
        EPWI_CHECK_LAUNCH();
    }
    cudaEventRecord(tm.fill.e[1], c->stream);
    // Re->k
    c->ghat.ensure(state_bytes * (cv.ns + 1));
    RestageArgs ra;
    ra.g = g;
    ra.W = W;
    ra.Nm = Nm;
    ra.nRe = c->nRe;
    ra.nRp = nRp;
    ra.nrow = (int)nrow;
    ra.Re = c->Re.as<int>();
    ra.gw64 = c->gw64.as<double2>();
    ra.gw32 = (tc && c->rp_cube_r < 0) ? c->gcube32.as<float2>() : c->gw32.as<float2>();
    ra.ph64 = c->ph64.as<double2>();
    ra.ph32 = c->ph32.as<float2>();
    ra.V64 = c->V.as<double2>();
    ra.V32 = c->V32.as<float2>();
    ra.nkp = (int)nkpc;
    ra.kpts = ws.kpts + cv.kp0;
    ra.kp_state = ws.kp_state + cv.kp0;
    ra.s_base = cv.s_base;
    ra.win_lo = c->win_lo.as<int>();
    ra.win_n = c->win_n.as<int>();
    ra.ovr_lo = ws.ovr_lo;
    ra.ovr_nsel = ws.ovr_nsel;
    ra.ghat64 = c->ghat.as<double2>();
    ra.ghat_raw = c->ghat.p;
    ra.precision = c->opt.precision;
    ra.nstates_chunk = cv.ns;
    cudaEventRecord(tm.re.e[0], c->stream);
    if (sf) sf_restage(c, ra);
    else if (tc) tc_restage(c, ra);
    else fp64_restage(ra, W, c->stream);
    cudaEventRecord(tm.re.e[1], c->stream);
    // Rp->q + rotations + delta sum
    ScatterArgs sa;
    sa.g = g;
    sa.W = W;
    sa.Nm = Nm;
    sa.nRp = nRp;
    sa.nrow = (int)nrow;
    sa.Rp = c->Rp.as<int>();
    sa.ph64 = c->ph64.as<double2>();
    sa.ph32 = c->ph32.as<float2>();
    sa.tiles = c->tiles.as<int4>();
    sa.kpts = ws.kpts + cv.kp0;
    sa.kp_state = ws.kp_state + cv.kp0;
    sa.s_base = cv.s_base;
    sa.win_lo = c->win_lo.as<int>();
    sa.win_n = c->win_n.as<int>();
    sa.ovr_lo = ws.ovr_lo;
    sa.ovr_nsel = ws.ovr_nsel;
    sa.pairs = cv.pairs;
    sa.ghat64 = c->ghat.as<double2>();
    sa.ghat_raw = c->ghat.p;
    sa.V64 = c->V.as<double2>();
    sa.V32 = c->V32.as<float2>();
    sa.u64 = c->u.as<double2>();
    sa.u32 = c->u32.as<float2>();
    sa.eps = c->eps.as<double>();
    sa.hw = c->hw.as<double>();
    sa.focc = g2out ? nullptr : c->focc.as<double>();
    sa.nocc = g2out ? nullptr : c->nocc.as<double>();
    sa.omega_min = c->opt.omega_min_eV;
    sa.eta = c->eta > 0 ? c->eta : 1.0;
    sa.ceta = c->opt.sieve_c * c->eta;
    sa.tile_part = c->tile_part.as<double>();
    sa.g2out = g2out;
    sa.g2_base = cv.g_base;
    sa.pair_w = ws.pair_w ? ws.pair_w + cv.g_base : nullptr;
    sa.tout = tout;
    sa.tstride = tstride;
    sa.gam32 = ws.gam32;
    sa.gam64 = ws.gam64;
    sa.goff = ws.goff ? ws.goff + cv.g_base : nullptr;
    sa.precision = c->opt.precision;
    sa.nstates_chunk = cv.ns;
    sa.nsel_max = 1;
    if (ws.ovr_nsel >= 0) {
        sa.nsel_max = ws.ovr_nsel;
    } else {
        for (int64_t p = cv.kp0; p < cv.kp1; ++p)
            sa.nsel_max = std::max<int64_t>(sa.nsel_max, ws.h_kp_state[p + 1] - ws.h_kp_state[p]);
    }
    cudaEventRecord(tm.sc.e[0], c->stream);
    if (sf) {
        std::vector<int64_t> hks(ws.h_kp_state.begin() + cv.kp0, ws.h_kp_state.begin() + cv.kp1 + 1);
        sf_scatter(c, sa, nkpc, cv.kp_pairs, cv.p_off, hks);
    } else if (tc) {
        tc_scatter(c, sa, nt);
    } else {
        fp64_scatter(sa, nt, c->stream);
    }
    cudaEventRecord(tm.sc.e[1], c->stream);
    // reduce (the fp32 mode wrote 1/tau already)
    cudaEventRecord(tm.red.e[0], c->stream);
    if (!sf && !g2out && !tout && nkpc > 0) {
        const double pref = 2.0 * epc::kPi / epc::kHbarEVs / (double)c->nk /
                            (sqrt(epc::kPi) * c->eta);
        k_reduce_tiles<<<(unsigned)((nkpc + 127) / 128), 128, 0, c->stream>>>(
            nkpc, ws.kpts + cv.kp0, c->win_n.as<int>(), ws.kp_state + cv.kp0, c->kp_tile.as<int64_t>(),
            c->tile_part.as<double>(), pref, c->inv_tau.as<double>());
        EPWI_CHECK_LAUNCH();
    }
    cudaEventRecord(tm.red.e[1], c->stream);
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    if (tc && nt > 0)
        EPWI_REQUIRE(tc_check_error(c) == 0, EPWI_ETIMEOUT,
                     "tensor-core kernel: a bounded mbarrier wait timed out");
    c->stats.ms_sieve += tm.fill.ms();
    c->stats.ms_restage += tm.re.ms();
    c->stats.ms_scatter += tm.sc.ms();
    c->stats.ms_reduce += tm.red.ms();
    return nt;
}

}  // namespace

// Processes the work set ws (k-points with their pair lists) chunk by chunk.  In rates mode
// it writes inv_tau for every state of the work set; in g2 mode (g2out != nullptr) it writes
// |g|^2 per pair instead.
void process_workset(epwi_ctx *c, const WorkSet &ws, double *g2out, double *tout, int tstride) {
    const int W = c->nw, Nm = c->nm;
    const int64_t nrow = (int64_t)c->nRp * Nm * W;
    const bool sf = c->opt.precision == EPWI_FP32;
    const bool tc = !sf && c->opt.precision != EPWI_FP64;
    EPWI_REQUIRE(!tc || !tout, EPWI_EINVAL, "per-pair terms need the FP64 path");
    EPWI_REQUIRE(!sf || (!g2out && !tout && !ws.pair_w && !ws.gam64 && ws.ovr_nsel < 0),
                 EPWI_EUNSUPPORTED, "the fp32 mode serves the sieved rates (and their Gamma) only");
    if (sf) {
        sf_check(c);
        sf_prepare(c);
    }
    if (tc) tc_prepare(c);
    // chunk limits: pairs and Re->k output size
    // pair lists per chunk: 2^32 q indices (16 GiB) in the fp32 mode, whose launches are one
    // CTA per state and need thousands of states per chunk to fill the GPU on large grids (200^3:
    // ~1.8 M pairs per state); 2^27 otherwise
    const int64_t max_pairs = int64_t(1) << (sf ? 32 : 27);
    const size_t state_bytes = sf ? sf_state_bytes(c) : tc ? tc_state_bytes(c) : sizeof(double2) * nrow;
    const int64_t max_states = std::max<int64_t>(1, (int64_t)((size_t(3) << 30) / state_bytes));
    const int64_t kp_cap = c->opt.kpoint_chunk > 0 ? c->opt.kpoint_chunk : (int64_t)1 << 40;
    StageTimers tm;
    int64_t kp0 = 0, nchunks = 0, ntiles_total = 0;
    while (kp0 < ws.nkp) {
        int64_t kp1 = kp0 + 1;
        while (kp1 < ws.nkp && kp1 - kp0 < kp_cap &&
               ws.h_kp_pairs[kp1 + 1] - ws.h_kp_pairs[kp0] <= max_pairs &&
               ws.h_kp_state[kp1 + 1] - ws.h_kp_state[kp0] <= max_states)
            ++kp1;
        ChunkView cv;
        cv.kp0 = kp0;
        cv.kp1 = kp1;
        cv.p_off = ws.h_kp_pairs[kp0];
        cv.g_base = cv.p_off;
        cv.np = ws.h_kp_pairs[kp1] - cv.p_off;
        cv.s_base = ws.h_kp_state[kp0];
        cv.ns = ws.h_kp_state[kp1] - cv.s_base;
        cv.kp_pairs = ws.kp_pairs + kp0;
        cudaEventRecord(tm.fill.e[0], c->stream);
        cv.pairs = ws.pairs_dev ? ws.pairs_dev + cv.p_off : nullptr;
        if (!cv.pairs) {
            c->pairs.ensure(sizeof(int) * (cv.np + 1));
            sieve_fill_chunk(c, kp0, kp1, c->pairs.as<int>());
            cv.pairs = c->pairs.as<int>();
        }
        ntiles_total += run_chunk(c, ws, cv, g2out, tout, tstride, tm);
        ++nchunks;
        kp0 = kp1;
    }
    c->stats.n_tiles = ntiles_total;
    c->stats.n_chunks = nchunks;
}
