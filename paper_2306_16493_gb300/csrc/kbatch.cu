// k-batch ordering of the interpolation, the alternative the paper measures against its
// q-batch ordering (Sec. III C, Table 3).  FP64, for the ablation.
//
// q-batch (the default path): ghat(k) = [sum_Re e^{ik.Re} g(Re, Rp)] U^dag(k) once per k-point,
// then per pair the Rp sum, n_Rp x N_m x W x n_k complex MACs.
// k-batch (this file): gq(q) = [sum_Rp e^{iq.Rp} g(Re, Rp)] u(q) once per q-point, then per
// pair the Re sum, n_Re x N_m x W x W complex MACs, and both Bloch rotations.
// The ratio of the per-pair volumes is (n_k / W)(n_Rp / n_Re).
//
// Pairs come from the sieve in k-major order.  They are bucketed by q (a histogram, a scan
// and an atomic scatter; the order inside a bucket does not matter because every pair writes
// its own slot), processed in tiles of one q, and each pair writes its per-band terms
// t[pair][n].  1/tau is then the fixed-order sum over each k-point's pairs in sieve order, so
// the result is deterministic.
#include <algorithm>
#include <vector>

#include "epwi_internal.cuh"
#include "scatter.cuh"

namespace {

constexpr int kKbTile = 128;
constexpr int kKbMaxW = 8;
constexpr int kKbMaxNm = 6;

struct KbTile {
    int q;
    int pad;
    int64_t b, e;                           // positions in the q-major pair list
};

struct KbArgs {
    GridInfo g;
    int W, Nm, nRe, nRp;
    const int *Re, *Rp;
    const double2 *gw64;                    // [nRe][nRp][Nm][W][W], weights folded
    const double2 *ph64;
    const double2 *u64;                     // [Nq][Nm][Nm]
    const double2 *V64;                     // [Nk][W][W]
    int q0, nq;                             // q range of the chunk
    double2 *gq;                            // [q - q0][nRe][Nm (nu)][W][W]
    const KbTile *tiles;
    const int64_t *qlist;                   // q-major list of pair indices
    const int *pkp;                         // pair -> window k-point
    const int *kpts, *win_lo, *win_n;
    const double *eps, *hw, *focc, *nocc;
    double omega_min, eta, ceta;
    double *tout;                           // [pair][W] per-band terms
};

__global__ void k_kb_pair_kp(const int64_t *__restrict__ kp_pairs, int *__restrict__ pkp) {
    const int kp = blockIdx.x;
    for (int64_t p = kp_pairs[kp] + threadIdx.x; p < kp_pairs[kp + 1]; p += blockDim.x) pkp[p] = kp;
}

__global__ void k_kb_hist(int64_t np, const int *__restrict__ pairs, unsigned long long *__restrict__ cnt) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) atomicAdd(&cnt[pairs[p]], 1ull);
}

__global__ void k_kb_bucket(int64_t np, const int *__restrict__ pairs, const int64_t *__restrict__ qoff,
                            unsigned long long *__restrict__ fill, int64_t *__restrict__ qlist) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int q = pairs[p];
    qlist[qoff[q] + (int64_t)atomicAdd(&fill[q], 1ull)] = p;
}

// gq[q][re][nu][i][j] = sum_mu u_{mu nu}(q) sum_Rp e^{iq.Rp} g(Re, Rp)[mu][i][j]; one thread per
// (re, i, j), KG q-points per block row.
template <int NMT, int KG>
__global__ void __launch_bounds__(128) k_kb_restage(KbArgs a) {
    constexpr int NMM = NMT ? NMT : kKbMaxNm;
    const int Nm = NMT ? NMT : a.Nm;
    extern __shared__ double2 P[];          // [KG][nRp]
    const int qg = blockIdx.y * KG;
    for (int idx = threadIdx.x; idx < KG * a.nRp; idx += blockDim.x) {
        const int kk = idx / a.nRp, r = idx % a.nRp;
        double2 p = make_double2(0, 0);
        if (qg + kk < a.nq) {
            int i1, i2, i3;
            grid_coords(a.g, a.q0 + qg + kk, i1, i2, i3);
            p = a.ph64[phase_index(i1 * a.g.s1 % a.g.L, i2 * a.g.s2 % a.g.L, i3 * a.g.s3 % a.g.L,
                                   a.Rp[3 * r], a.Rp[3 * r + 1], a.Rp[3 * r + 2], a.g.L)];
        }
        P[idx] = p;
    }
    __syncthreads();
    const int WW = a.W * a.W;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;     // (re, i, j)
    if (row >= a.nRe * WW) return;
    const int re = row / WW, ij = row % WW;
    double2 acc[KG][NMM];
    for (int kk = 0; kk < KG; ++kk)
        for (int mu = 0; mu < Nm; ++mu) acc[kk][mu] = make_double2(0, 0);
    const double2 *gw = a.gw64 + (size_t)re * a.nRp * Nm * WW + ij;
    for (int rp = 0; rp < a.nRp; ++rp) {
        for (int mu = 0; mu < Nm; ++mu) {
            const double2 gv = gw[((size_t)rp * Nm + mu) * WW];
            for (int kk = 0; kk < KG; ++kk) acc[kk][mu] = cfma(P[kk * a.nRp + rp], gv, acc[kk][mu]);
        }
    }
    for (int kk = 0; kk < KG; ++kk) {
        if (qg + kk >= a.nq) break;
        const int q = a.q0 + qg + kk;
        const double2 *u = a.u64 + (int64_t)q * Nm * Nm;
        double2 *o = a.gq + ((size_t)(qg + kk) * a.nRe + re) * Nm * WW + ij;
        for (int nu = 0; nu < Nm; ++nu) {
            double2 s = make_double2(0, 0);
            for (int mu = 0; mu < Nm; ++mu) s = cfma(acc[kk][mu], u[mu * Nm + nu], s);
            o[(size_t)nu * WW] = s;
        }
    }
}

// One thread per pair of a one-q tile: Re sum, U(k+q) [.] U^dag(k), |g|^2 and the delta terms.
template <int WT, int NMT>
__global__ void __launch_bounds__(128) k_kb_scatter(KbArgs a) {
    constexpr int WM = WT ? WT : kKbMaxW;
    const int W = WT ? WT : a.W;
    const int Nm = NMT ? NMT : a.Nm;
    const KbTile t = a.tiles[blockIdx.x];
    const int64_t pos = t.b + threadIdx.x;
    if (pos >= t.e) return;
    const int64_t pair = a.qlist[pos];
    const int q = t.q;
    const int kp = a.pkp[pair];
    const int ik = a.kpts[kp];
    const int lo = a.win_lo[ik], nsel = a.win_n[ik];
    const int64_t ikq = kplusq(a.g, ik, q);
    int i1, i2, i3;
    grid_coords(a.g, ik, i1, i2, i3);
    const int a1 = i1 * a.g.s1 % a.g.L, a2 = i2 * a.g.s2 % a.g.L, a3 = i3 * a.g.s3 % a.g.L;
    const double2 *gqq = a.gq + (size_t)(q - a.q0) * a.nRe * Nm * W * W;
    const double2 *Vk = a.V64 + (int64_t)ik * W * W;
    const double2 *Vq = a.V64 + ikq * W * W;
    double tn[WM];
    for (int n = 0; n < W; ++n) tn[n] = 0;
    for (int nu = 0; nu < Nm; ++nu) {
        const double w = a.hw[(int64_t)q * Nm + nu];
        if (!(w >= a.omega_min)) continue;
        const double N = a.nocc[(int64_t)q * Nm + nu];
        double2 G[WM][WM];
        for (int i = 0; i < W; ++i)
            for (int j = 0; j < W; ++j) G[i][j] = make_double2(0, 0);
        for (int re = 0; re < a.nRe; ++re) {
            const double2 p = a.ph64[phase_index(a1, a2, a3, a.Re[3 * re], a.Re[3 * re + 1],
                                                 a.Re[3 * re + 2], a.g.L)];
            const double2 *gr = gqq + ((size_t)re * Nm + nu) * W * W;
            for (int i = 0; i < W; ++i)
                for (int j = 0; j < W; ++j) G[i][j] = cfma(p, gr[i * W + j], G[i][j]);
        }
        for (int m = 0; m < W; ++m) {
            double2 h[WM];                  // h_j = sum_i conj(V_im(k+q)) G_ij
            for (int j = 0; j < W; ++j) {
                h[j] = make_double2(0, 0);
                for (int i = 0; i < W; ++i) h[j] = cfmac(Vq[i * W + m], G[i][j], h[j]);
            }
            const double em = a.eps[ikq * W + m];
            const double fm = a.focc[ikq * W + m];
            for (int n = 0; n < nsel; ++n) {
                double2 gv = make_double2(0, 0);
                for (int j = 0; j < W; ++j) gv = cfma(h[j], Vk[j * W + lo + n], gv);
                const double g2 = gv.x * gv.x + gv.y * gv.y;
                const double en = a.eps[(int64_t)ik * W + lo + n];
                const double x1 = (en + w) - em;
                const double x2 = (en - w) - em;
                double term = 0;
                if (fabs(x1) <= a.ceta) {
                    const double y = x1 / a.eta;
                    term += (N + fm) * exp(-y * y);
                }
                if (fabs(x2) <= a.ceta) {
                    const double y = x2 / a.eta;
                    term += (1.0 + N - fm) * exp(-y * y);
                }
                tn[n] += g2 * term;
            }
        }
    }
    for (int n = 0; n < nsel; ++n) a.tout[pair * W + n] = tn[n];
}

// 1/tau_nk = pref * sum over the k-point's pairs, in sieve order
__global__ void k_kb_reduce(int64_t nkp, int W, const int *__restrict__ kpts, const int *__restrict__ win_n,
                            const int64_t *__restrict__ kp_state, const int64_t *__restrict__ kp_pairs,
                            const double *__restrict__ tout, double pref, double *__restrict__ inv_tau) {
    const int64_t kp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (kp >= nkp) return;
    const int ns = win_n[kpts[kp]];
    for (int n = 0; n < ns; ++n) {
        double s = 0;
        for (int64_t p = kp_pairs[kp]; p < kp_pairs[kp + 1]; ++p) s += tout[p * W + n];
        inv_tau[kp_state[kp] + n] = pref * s;
    }
}

template <int NMT>
void launch_restage(const KbArgs &a, cudaStream_t st) {
    constexpr int KG = 8;
    const size_t sm = sizeof(double2) * KG * a.nRp;
    if (sm > 48 * 1024)
        EPWI_CUDA(cudaFuncSetAttribute(k_kb_restage<NMT, KG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid((unsigned)((a.nRe * a.W * a.W + 127) / 128), (unsigned)((a.nq + KG - 1) / KG));
    k_kb_restage<NMT, KG><<<grid, 128, sm, st>>>(a);
    EPWI_CHECK_LAUNCH();
}

struct KbEv {
    cudaEvent_t e[2];
    KbEv() { cudaEventCreate(&e[0]); cudaEventCreate(&e[1]); }
    ~KbEv() { cudaEventDestroy(e[0]); cudaEventDestroy(e[1]); }
    float ms() { float m = 0; cudaEventElapsedTime(&m, e[0], e[1]); return m; }
};

}  // namespace

// The rates of the current window by the k-batch ordering (FP64); fills inv_tau.
void process_kbatch(epwi_ctx *c) {
    const int W = c->nw, Nm = c->nm;
    EPWI_REQUIRE(W <= kKbMaxW && Nm <= kKbMaxNm, EPWI_EUNSUPPORTED,
                 "k-batch ordering built for nw <= 8 and <= 6 modes");
    const int64_t nkp = c->nkp, np = c->npairs, nk = c->nk;
    KbEv ev_fill, ev_re, ev_sc, ev_red;
    float ms_re = 0, ms_sc = 0;
    DevBuf pairs, pkp, cnt, qoff, fill, qlist, tiles, gq, tout;
    auto cleanup = [&] {
        for (DevBuf *b : {&pairs, &pkp, &cnt, &qoff, &fill, &qlist, &tiles, &gq, &tout}) b->release();
    };
    try {
        cudaEventRecord(ev_fill.e[0], c->stream);
        pairs.ensure(sizeof(int) * (np + 1));
        sieve_fill_chunk(c, 0, nkp, pairs.as<int>());
        pkp.ensure(sizeof(int) * (np + 1));
        if (nkp > 0) {
            k_kb_pair_kp<<<(unsigned)nkp, 256, 0, c->stream>>>(c->kp_pairs.as<int64_t>(), pkp.as<int>());
            EPWI_CHECK_LAUNCH();
        }
        cnt.ensure(sizeof(int64_t) * (nk + 1));
        fill.ensure(sizeof(int64_t) * (nk + 1));
        qoff.ensure(sizeof(int64_t) * (nk + 1));
        qlist.ensure(sizeof(int64_t) * (np + 1));
        EPWI_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int64_t) * (nk + 1), c->stream));
        EPWI_CUDA(cudaMemsetAsync(fill.p, 0, sizeof(int64_t) * (nk + 1), c->stream));
        const unsigned nb = (unsigned)((np + 255) / 256);
        if (np > 0) {
            k_kb_hist<<<nb, 256, 0, c->stream>>>(np, pairs.as<int>(), cnt.as<unsigned long long>());
            EPWI_CHECK_LAUNCH();
        }
        scan_exclusive_i64(c, cnt.as<int64_t>(), qoff.as<int64_t>(), nk, nullptr);
        if (np > 0) {
            k_kb_bucket<<<nb, 256, 0, c->stream>>>(np, pairs.as<int>(), qoff.as<int64_t>(),
                                                  fill.as<unsigned long long>(), qlist.as<int64_t>());
            EPWI_CHECK_LAUNCH();
        }
        std::vector<int64_t> h_qoff(nk + 1);
        EPWI_CUDA(cudaMemcpyAsync(h_qoff.data(), qoff.p, sizeof(int64_t) * (nk + 1), cudaMemcpyDeviceToHost,
                                  c->stream));
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
        cudaEventRecord(ev_fill.e[1], c->stream);
        std::vector<KbTile> h_tiles;
        std::vector<int64_t> q_tile(nk + 1, 0);     // first tile of each q
        for (int64_t q = 0; q < nk; ++q) {
            q_tile[q] = (int64_t)h_tiles.size();
            for (int64_t b = h_qoff[q]; b < h_qoff[q + 1]; b += kKbTile)
                h_tiles.push_back(KbTile{(int)q, 0, b, std::min(h_qoff[q + 1], b + (int64_t)kKbTile)});
        }
        q_tile[nk] = (int64_t)h_tiles.size();
        tiles.ensure(sizeof(KbTile) * (h_tiles.size() + 1));
        if (!h_tiles.empty())
            EPWI_CUDA(cudaMemcpyAsync(tiles.p, h_tiles.data(), sizeof(KbTile) * h_tiles.size(),
                                      cudaMemcpyHostToDevice, c->stream));
        tout.ensure(sizeof(double) * W * (np + 1));
        const size_t per_q = sizeof(double2) * (size_t)c->nRe * Nm * W * W;
        const int64_t qchunk = std::max<int64_t>(1, (int64_t)((size_t(2) << 30) / per_q));
        gq.ensure(per_q * (size_t)std::min<int64_t>(qchunk, std::max<int64_t>(1, nk)));
        KbArgs a;
        a.g = make_grid_info(c);
        a.W = W;
        a.Nm = Nm;
        a.nRe = c->nRe;
        a.nRp = c->nRp;
        a.Re = c->Re.as<int>();
        a.Rp = c->Rp.as<int>();
        a.gw64 = c->gw64.as<double2>();
        a.ph64 = c->ph64.as<double2>();
        a.u64 = c->u.as<double2>();
        a.V64 = c->V.as<double2>();
        a.gq = gq.as<double2>();
        a.tiles = tiles.as<KbTile>();
        a.qlist = qlist.as<int64_t>();
        a.pkp = pkp.as<int>();
        a.kpts = c->kpts.as<int>();
        a.win_lo = c->win_lo.as<int>();
        a.win_n = c->win_n.as<int>();
        a.eps = c->eps.as<double>();
        a.hw = c->hw.as<double>();
        a.focc = c->focc.as<double>();
        a.nocc = c->nocc.as<double>();
        a.omega_min = c->opt.omega_min_eV;
        a.eta = c->eta;
        a.ceta = c->opt.sieve_c * c->eta;
        a.tout = tout.as<double>();
        for (int64_t q0 = 0; q0 < nk; q0 += qchunk) {
            const int64_t q1 = std::min(nk, q0 + qchunk);
            const int64_t t0 = q_tile[q0], t1 = q_tile[q1];
            if (t1 == t0) continue;
            a.q0 = (int)q0;
            a.nq = (int)(q1 - q0);
            cudaEventRecord(ev_re.e[0], c->stream);
            if (Nm == 3) launch_restage<3>(a, c->stream);
            else if (Nm == 6) launch_restage<6>(a, c->stream);
            else launch_restage<0>(a, c->stream);
            cudaEventRecord(ev_re.e[1], c->stream);
            KbArgs at = a;
            at.tiles = a.tiles + t0;
            cudaEventRecord(ev_sc.e[0], c->stream);
            const unsigned nt = (unsigned)(t1 - t0);
            if (W == 1 && Nm == 3) k_kb_scatter<1, 3><<<nt, kKbTile, 0, c->stream>>>(at);
            else if (W == 4 && Nm == 3) k_kb_scatter<4, 3><<<nt, kKbTile, 0, c->stream>>>(at);
            else if (W == 8 && Nm == 6) k_kb_scatter<8, 6><<<nt, kKbTile, 0, c->stream>>>(at);
            else k_kb_scatter<0, 0><<<nt, kKbTile, 0, c->stream>>>(at);
            EPWI_CHECK_LAUNCH();
            cudaEventRecord(ev_sc.e[1], c->stream);
            EPWI_CUDA(cudaStreamSynchronize(c->stream));
            ms_re += ev_re.ms();
            ms_sc += ev_sc.ms();
        }
        cudaEventRecord(ev_red.e[0], c->stream);
        if (nkp > 0) {
            const double pref = 2.0 * epc::kPi / epc::kHbarEVs / (double)c->nk / (sqrt(epc::kPi) * c->eta);
            k_kb_reduce<<<(unsigned)((nkp + 127) / 128), 128, 0, c->stream>>>(
                nkp, W, c->kpts.as<int>(), c->win_n.as<int>(), c->kp_state.as<int64_t>(),
                c->kp_pairs.as<int64_t>(), tout.as<double>(), pref, c->inv_tau.as<double>());
            EPWI_CHECK_LAUNCH();
        }
        cudaEventRecord(ev_red.e[1], c->stream);
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
        c->stats.ms_sieve += ev_fill.ms();
        c->stats.ms_restage = ms_re;
        c->stats.ms_scatter = ms_sc;
        c->stats.ms_reduce = ev_red.ms();
        c->stats.n_tiles = (int64_t)h_tiles.size();
        c->stats.n_chunks = (nk + qchunk - 1) / qchunk;
    } catch (...) {
        cudaStreamSynchronize(c->stream);
        cleanup();
        throw;
    }
    cleanup();
}
