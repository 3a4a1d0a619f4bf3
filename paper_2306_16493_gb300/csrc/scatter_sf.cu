// Sum-factorised Rp->q stage in FP32 (precision EPWI_FP32), fused with the rotations and the
// delta sum of Eq. 10.
//
// R_p is the full cube [-r, r]^3, so the phase of Eq. 16 factorises per axis:
// e^{iq.Rp} = e1(q1, R1) e2(q2, R2) e3(q3, R3) with e_a(x, R) = e^{2 pi i x R / N_a}.  The sum
// over the cube is then three nested sums of D = 2r + 1 terms, and each is done where its
// result can be shared.  The sieve lists the pairs of a k-point in plane blocks pb of 256
// consecutive (q2, q3) combinations, then by q1, then by combination.
//   Y[R1][R3][j]  = sum_R2 e2(q2_j, R2) ghat[R1, R2, R3]   once per plane block (its q2 values j)
//   U[R3][j]      = sum_R1 e1(q1, R1) Y[R1][R3][j]          once per run (plane block, q1)
//   G             = sum_R3 e3(q3, R3) U[R3][j(q)]           per pair
// with ghat = (g P^el) U^dag(k) from the FP32 Re->k stage, every column (mu, i) at once.  A
// pair costs D N_m W complex MACs instead of D^3 N_m W.  Then, per pair, come the rotations
// U(k+q) [.] u(q), |g|^2 and the two delta terms, in FP32.
//
// One CTA per (window k-point, band), eight warps.  Warps take the runs of a plane block
// two at a time, round-robin by q1, and walk the pairs of both as one list.  With a Gamma capture (iterative BTE) the CTA also writes its band's row
// of every pair's Gamma block; rows of bands skipped as out of range stay at the zero the
// buffer was cleared to.  Lane sums are FP32 within a run; the run sums go into per-warp FP64
// accumulators, which are added in warp order, so the result is deterministic.
#include <algorithm>

#include "epwi_internal.cuh"
#include "scatter.cuh"
#include "sieve.cuh"

namespace {

constexpr int kSfThreads = 256;
constexpr int kSfWarps = kSfThreads / 32;

// Re->k in FP32: ghat32[state][row] = sum_j [sum_Re w e^{ik.Re} g(Re)[row][j]] V_{j, lo+n}(k),
// row = (rp N_m + mu) W + i; one thread per row, KG k-points per block row.
template <int WT, int KG>
__global__ void __launch_bounds__(128) k_restage_f32(RestageArgs a, float2 *__restrict__ out) {
    constexpr int WM = WT ? WT : epc::kMaxW;
    const int W = WT ? WT : a.W;
    extern __shared__ float2 P32[];                 // [KG][nRe]
    const int kg0 = blockIdx.y * KG;
    for (int idx = threadIdx.x; idx < KG * a.nRe; idx += blockDim.x) {
        const int kk = idx / a.nRe, r = idx % a.nRe;
        float2 p = make_float2(0.f, 0.f);
        if (kg0 + kk < a.nkp) {
            int i1, i2, i3;
            grid_coords(a.g, a.kpts[kg0 + kk], i1, i2, i3);
            p = a.ph32[phase_index(i1 * a.g.s1 % a.g.L, i2 * a.g.s2 % a.g.L, i3 * a.g.s3 % a.g.L,
                                   a.Re[3 * r], a.Re[3 * r + 1], a.Re[3 * r + 2], a.g.L)];
        }
        P32[idx] = p;
    }
    __syncthreads();
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= a.nrow) return;
    float2 acc[KG][WM];
    for (int kk = 0; kk < KG; ++kk)
        for (int j = 0; j < W; ++j) acc[kk][j] = make_float2(0.f, 0.f);
    const float2 *gw = a.gw32 + (size_t)row * W;
    for (int r = 0; r < a.nRe; ++r) {
        float2 gv[WM];
        for (int j = 0; j < W; ++j) gv[j] = gw[(size_t)r * a.nrow * W + j];
        for (int kk = 0; kk < KG; ++kk) {
            const float2 p = P32[kk * a.nRe + r];
            for (int j = 0; j < W; ++j) acc[kk][j] = cfmaf(p, gv[j], acc[kk][j]);
        }
    }
    for (int kk = 0; kk < KG; ++kk) {
        if (kg0 + kk >= a.nkp) break;
        const int ik = a.kpts[kg0 + kk];
        const int lo = a.win_lo[ik], ns = a.win_n[ik];
        const int64_t s0 = a.kp_state[kg0 + kk] - a.s_base;
        const float2 *Vk = a.V32 + (int64_t)ik * W * W;
        for (int np = 0; np < ns; ++np) {
            float2 o = make_float2(0.f, 0.f);
            for (int j = 0; j < W; ++j) o = cfmaf(acc[kk][j], Vk[j * W + lo + np], o);
            out[(s0 + np) * a.nrow + row] = o;
        }
    }
}

struct SfArgs {
    GridInfo g;
    int64_t nplane;                 // N2 N3
    int nq2max;                     // largest count of q2 values in one plane block
    const float2 *ph32;             // e^{2 pi i m / L}
    const float2 *ghat;             // [state - s_base][D^3][N_m][W]
    const int *kpts, *win_lo, *win_n;
    const int64_t *kp_state;        // chunk k-points' first states (global)
    int64_t s_base;
    const int64_t *kp_pairs;        // chunk-local pair offsets, minus p_off
    int64_t p_off;
    const int *pairs;               // chunk pair list: q index
    const float2 *V32, *u32;
    const float *erel, *f32, *n32, *hw32;
    float ceta32, inv_eta32;
    double pref;                    // 2 pi / (hbar N_q sqrt(pi) eta)
    double *inv_tau;
    const int2 *items;              // {chunk kp, band}
    float *gam;                     // Gamma capture (iterative BTE) or nullptr: row n of each
    const int64_t *goff;            // pair's block, block start goff[chunk pair]
};

__device__ __forceinline__ float2 axis_phase(const float2 *ph, int x, int s, int R, int L) {
    int t = ((x * s) % L) * R % L;
    if (t < 0) t += L;
    return ph[t];
}

// first position in [lo, hi) whose key is >= key (keys ascending)
template <typename F>
__device__ __forceinline__ int64_t lower_bound(int64_t lo, int64_t hi, int64_t key, F keyof) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keyof(mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <int W, int NM, int RC, bool GAM>
__global__ void __launch_bounds__(kSfThreads, 2) k_scatter_sf(SfArgs a) {
    constexpr int D = 2 * RC + 1;
    constexpr int X = NM * W;                    // columns (mu, i)
    extern __shared__ float2 sm[];
    const int Q = a.nq2max;
    const int N1 = a.g.n1, N2 = a.g.n2, N3 = a.g.n3, L = a.g.L;
    float2 *gk = sm;                             // [D^3][X]
    float2 *Y = gk + D * D * D * X;              // [D (R1)][D (R3)][Q][X]
    float2 *Uall = Y + D * D * Q * X;            // [warp][2 runs][D (R3)][Q][X]
    float2 *E1 = Uall + 2 * kSfWarps * D * Q * X;   // [N1][D] axis phases e^{2 pi i x R / N}
    float2 *E2 = E1 + N1 * D;                    // [N2][D]
    float2 *E3 = E2 + N2 * D;                    // [N3][D]
    int *cq = reinterpret_cast<int *>(E3 + N3 * D);   // [kSieveBlock]: (j << 16) | q3 of combination c_lo + t
    int *rs = cq + kSieveBlock;                  // [N1]: run start (relative to the block), -1 if none
    int *re = rs + N1;                           // [N1]: run end
    __shared__ double wsum[kSfWarps];
    const int2 item = a.items[blockIdx.x];
    const int kp = item.x, n = item.y;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float2 *U = Uall + (size_t)wid * 2 * D * Q * X;
    const int ik = a.kpts[kp];
    const int lo = a.win_lo[ik];
    const int64_t s = a.kp_state[kp] + n;        // global state
    const float2 *gs = a.ghat + (size_t)(s - a.s_base) * D * D * D * X;
    for (int e = threadIdx.x; e < D * D * D * X; e += kSfThreads) gk[e] = gs[e];
    for (int e = threadIdx.x; e < (N1 + N2 + N3) * D; e += kSfThreads) {
        const int R = e % D - RC, x = e / D;
        float2 v;
        if (x < N1) v = axis_phase(a.ph32, x, a.g.s1, R, L);
        else if (x < N1 + N2) v = axis_phase(a.ph32, x - N1, a.g.s2, R, L);
        else v = axis_phase(a.ph32, x - N1 - N2, a.g.s3, R, L);
        E1[e] = v;                               // E1, E2, E3 are consecutive
    }
    const int nplane = (int)a.nplane;
    const int pb_n = (nplane + kSieveBlock - 1) / kSieveBlock;
    const int64_t P0 = a.kp_pairs[kp] - a.p_off, P1 = a.kp_pairs[kp + 1] - a.p_off;
    const int *pl = a.pairs;
    auto pbof = [&](int64_t p) -> int64_t { return (int64_t)((pl[p] % nplane) / kSieveBlock); };
    int k1, k2, k3;
    grid_coords(a.g, ik, k1, k2, k3);
    const float en = a.erel[(int64_t)ik * W + lo + n];
    double wacc = 0;                             // this warp's run sums
    __syncthreads();
    int64_t seg0 = P0;
    for (int pb = 0; pb < pb_n && seg0 < P1; ++pb) {
        // the plane block's pairs [seg0, seg1)
        const int64_t seg1 = lower_bound(seg0, P1, (int64_t)pb + 1, pbof);
        if (seg1 == seg0) continue;
        const int c_lo = pb * kSieveBlock, c_hi = min(nplane, c_lo + kSieveBlock) - 1;
        const int q2lo = c_lo / N3, nq2 = c_hi / N3 - q2lo + 1;
        // per combination of the block: (j, q3); runs: none yet
        for (int t = threadIdx.x; t < kSieveBlock; t += kSfThreads) {
            const int c = c_lo + t, q2 = c / N3;
            cq[t] = ((q2 - q2lo) << 16) | (c - q2 * N3);
        }
        for (int t = threadIdx.x; t < N1; t += kSfThreads) rs[t] = -1;
        // Y over this block's q2 values (all threads)
        for (int e = threadIdx.x; e < D * D * nq2 * X; e += kSfThreads) {
            const int col = e % X, t = e / X;
            const int j = t % nq2, r13 = t / nq2;
            const int R3 = r13 % D, R1 = r13 / D;
            const float2 *e2 = E2 + (q2lo + j) * D;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int R2 = 0; R2 < D; ++R2) acc = cfmaf(e2[R2], gk[((R1 * D + R2) * D + R3) * X + col], acc);
            Y[((R1 * D + R3) * Q + j) * X + col] = acc;
        }
        __syncthreads();
        // run boundaries: the block's pairs are ordered by q1
        const int nseg = (int)(seg1 - seg0);
        for (int t = threadIdx.x; t < nseg; t += kSfThreads) {
            const int q1 = pl[seg0 + t] / nplane;
            if (t == 0 || pl[seg0 + t - 1] / nplane != q1) rs[q1] = t;
            if (t == nseg - 1 || pl[seg0 + t + 1] / nplane != q1) re[q1] = t + 1;
        }
        __syncthreads();
        // runs: warp w takes q1 = w + 16 i and w + 16 i + 8 together (U of both in shared
        // memory) and walks their pairs as one list, so that short runs share lane rounds
        for (int qa = wid; qa < N1; qa += 2 * kSfWarps) {
            const int qb = qa + kSfWarps;
            const int ra0 = rs[qa];
            const int na = ra0 < 0 ? 0 : re[qa] - ra0;
            const int rb0 = qb < N1 ? rs[qb] : -1;
            const int nb = rb0 < 0 ? 0 : re[qb] - rb0;
            if (na + nb == 0) continue;
            for (int h2 = 0; h2 < 2; ++h2) {
                if ((h2 == 0 ? na : nb) == 0) continue;
                const float2 *e1 = E1 + (h2 == 0 ? qa : qb) * D;
                float2 *Uh = U + h2 * D * Q * X;
                for (int e = lane; e < D * nq2 * X; e += 32) {
                    const int col = e % X, t = e / X;
                    const int j = t % nq2, R3 = t / nq2;
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int R1 = 0; R1 < D; ++R1) acc = cfmaf(e1[R1], Y[((R1 * D + R3) * Q + j) * X + col], acc);
                    Uh[(R3 * Q + j) * X + col] = acc;
                }
            }
            __syncwarp();
            float rate = 0.f;
            for (int tt0 = lane; tt0 < na + nb; tt0 += 32) {
                const bool inA = tt0 < na;
                const int q1 = inA ? qa : qb;
                const int t = inA ? ra0 + tt0 : rb0 + (tt0 - na);
                const float2 *Ur = inA ? U : U + D * Q * X;
                int b1 = k1 + q1;
                if (b1 >= N1) b1 -= N1;
                const int qbase = q1 * nplane + c_lo;
                const int q = pl[seg0 + t];
                const int cl = q - qbase;
                if ((unsigned)cl > (unsigned)(c_hi - c_lo)) continue;   // never in sieve order
                const int jq = cq[cl];
                const int j = jq >> 16, q3 = jq & 0xffff;
                const float2 *e3 = E3 + q3 * D;
                float2 G[X];
#pragma unroll
                for (int x = 0; x < X; ++x) G[x] = make_float2(0.f, 0.f);
#pragma unroll
                for (int R3 = 0; R3 < D; ++R3) {
                    const float2 p3 = e3[R3];
                    const float2 *u_ = Ur + (R3 * Q + j) * X;
                    if constexpr (X % 2 == 0) {          // rows of X float2 are 16-byte aligned
                        const float4 *u4 = reinterpret_cast<const float4 *>(u_);
#pragma unroll
                        for (int x = 0; x < X / 2; ++x) {
                            const float4 v = u4[x];
                            G[2 * x] = cfmaf(p3, make_float2(v.x, v.y), G[2 * x]);
                            G[2 * x + 1] = cfmaf(p3, make_float2(v.z, v.w), G[2 * x + 1]);
                        }
                    } else {
#pragma unroll
                        for (int x = 0; x < X; ++x) G[x] = cfmaf(p3, u_[x], G[x]);
                    }
                }
                int b2 = k2 + q2lo + j, b3 = k3 + q3;
                if (b2 >= N2) b2 -= N2;
                if (b3 >= N3) b3 -= N3;
                const int ikq = (b1 * N2 + b2) * N3 + b3;   // nk W^2 < 2^31 (checked on the host)
                int lokq = 0, nwkq = 0;
                int64_t grow = 0;                // this band's row of the pair's Gamma block
                if constexpr (GAM) {
                    lokq = __ldg(a.win_lo + ikq);
                    nwkq = __ldg(a.win_n + ikq);
                    grow = a.goff[seg0 + t] + (int64_t)n * nwkq - lokq;
                }
                const float2 *Vq = a.V32 + ikq * (W * W);
                const float2 *uq = a.u32 + q * (NM * NM);
                float wq[NM], nq[NM];
#pragma unroll
                for (int nu = 0; nu < NM; ++nu) {
                    wq[nu] = __ldg(a.hw32 + q * NM + nu);
                    nq[nu] = __ldg(a.n32 + q * NM + nu);
                }
                float2 ur[NM * NM];
#pragma unroll
                for (int x = 0; x < NM * NM; ++x) ur[x] = __ldg(uq + x);
                // V(k+q), eps - mu and f at k+q: 16-byte loads where W = 4 keeps them aligned
                float2 Vr[W * W];
                float emr[W], fmr[W];
                if constexpr (W == 4) {
                    const float4 *v4 = reinterpret_cast<const float4 *>(Vq);
#pragma unroll
                    for (int x = 0; x < W * W / 2; ++x) {
                        const float4 v = __ldg(v4 + x);
                        Vr[2 * x] = make_float2(v.x, v.y);
                        Vr[2 * x + 1] = make_float2(v.z, v.w);
                    }
                    const float4 e4 = __ldg(reinterpret_cast<const float4 *>(a.erel + ikq * W));
                    const float4 f4 = __ldg(reinterpret_cast<const float4 *>(a.f32 + ikq * W));
                    emr[0] = e4.x; emr[1] = e4.y; emr[2] = e4.z; emr[3] = e4.w;
                    fmr[0] = f4.x; fmr[1] = f4.y; fmr[2] = f4.z; fmr[3] = f4.w;
                } else {
#pragma unroll
                    for (int x = 0; x < W * W; ++x) Vr[x] = __ldg(Vq + x);
#pragma unroll
                    for (int m = 0; m < W; ++m) {
                        emr[m] = __ldg(a.erel + ikq * W + m);
                        fmr[m] = __ldg(a.f32 + ikq * W + m);
                    }
                }
#pragma unroll
                for (int m = 0; m < W; ++m) {
                    const float em = emr[m];
                    const float fm = fmr[m];
                    // a band with no mode inside c eta of either shell adds exactly zero
                    bool any = false;
#pragma unroll
                    for (int nu = 0; nu < NM; ++nu) {
                        const float w = wq[nu];
                        any |= w >= 0.f && (fabsf((en + w) - em) <= a.ceta32 || fabsf((en - w) - em) <= a.ceta32);
                    }
                    if (!any) continue;
                    float2 h[NM];
#pragma unroll
                    for (int mu = 0; mu < NM; ++mu) {
                        h[mu] = make_float2(0.f, 0.f);
#pragma unroll
                        for (int i = 0; i < W; ++i) h[mu] = cfmacf(Vr[i * W + m], G[mu * W + i], h[mu]);
                    }
                    float gm = 0.f;                  // Gamma capture: sum over modes
#pragma unroll
                    for (int nu = 0; nu < NM; ++nu) {
                        const float w = wq[nu];
                        if (w < 0.f) continue;
                        float2 gv = make_float2(0.f, 0.f);
#pragma unroll
                        for (int mu = 0; mu < NM; ++mu) gv = cfmaf(h[mu], ur[mu * NM + nu], gv);
                        const float g2 = gv.x * gv.x + gv.y * gv.y;
                        const float x1 = (en + w) - em;
                        const float x2 = (en - w) - em;
                        float tt = 0.f;
                        if (fabsf(x1) <= a.ceta32) {
                            const float y = x1 * a.inv_eta32;
                            tt += (nq[nu] + fm) * __expf(-y * y);
                        }
                        if (fabsf(x2) <= a.ceta32) {
                            const float y = x2 * a.inv_eta32;
                            tt += (1.f + nq[nu] - fm) * __expf(-y * y);
                        }
                        rate = fmaf(g2, tt, rate);
                        if constexpr (GAM) gm = fmaf(g2, tt, gm);
                    }
                    if constexpr (GAM) {
                        if (m >= lokq && m < lokq + nwkq) a.gam[grow + m] = gm;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rate += __shfl_xor_sync(0xffffffffu, rate, o);
            wacc += (double)rate;
            __syncwarp();                        // U is rewritten by the next run
        }
        __syncthreads();                         // Y, cq and the runs are rewritten next
        seg0 = seg1;
    }
    if (lane == 0) wsum[wid] = wacc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < kSfWarps; ++w) t += wsum[w];
        a.inv_tau[s] = a.pref * t;
    }
}

size_t sf_smem(int D, int X, int Q, int N1, int N2, int N3) {
    return sizeof(float2) * ((size_t)D * D * D * X + (size_t)D * D * Q * X + (size_t)2 * kSfWarps * D * Q * X +
                             (size_t)(N1 + N2 + N3) * D) +
           sizeof(int) * ((size_t)kSieveBlock + 2 * (size_t)N1);
}

template <int W, int NM, int RC, bool GAM>
void launch_sf_t(epwi_ctx *c, const SfArgs &a, int nitems) {
    const size_t sm = sf_smem(2 * RC + 1, NM * W, a.nq2max, a.g.n1, a.g.n2, a.g.n3);
    EPWI_REQUIRE(sm <= 200 * 1024, EPWI_EUNSUPPORTED,
                 "fp32 mode: the plane-block tables of this grid do not fit in shared memory");
    EPWI_CUDA(cudaFuncSetAttribute(k_scatter_sf<W, NM, RC, GAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    EPWI_CUDA(cudaFuncSetAttribute(k_scatter_sf<W, NM, RC, GAM>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    if (nitems > 0) {
        k_scatter_sf<W, NM, RC, GAM><<<(unsigned)nitems, kSfThreads, sm, c->stream>>>(a);
        EPWI_CHECK_LAUNCH();
    }
}

template <int W, int NM, int RC>
void launch_sf(epwi_ctx *c, const SfArgs &a, int nitems) {
    if (a.gam) launch_sf_t<W, NM, RC, true>(c, a, nitems);
    else launch_sf_t<W, NM, RC, false>(c, a, nitems);
}

}  // namespace

size_t sf_state_bytes(const epwi_ctx *c) { return sizeof(float2) * (size_t)c->nRp * c->nm * c->nw; }

void sf_check(const epwi_ctx *c) {
    const int W = c->nw, NM = c->nm, r = c->rp_cube_r;
    EPWI_REQUIRE(c->nk * std::max(W * W, NM * NM) < (int64_t(1) << 31), EPWI_EUNSUPPORTED,
                 "fp32 mode: grid too large for its 32-bit table offsets");
    EPWI_REQUIRE(r >= 0, EPWI_EUNSUPPORTED, "fp32 mode needs R_p to be the full cube [-r, r]^3");
    EPWI_REQUIRE((W == 4 && NM == 3 && (r == 1 || r == 2)) || (W == 1 && NM == 3 && r == 1),
                 EPWI_EUNSUPPORTED, "fp32 mode built for (nw, modes, R_p half-width) in {(4,3,1), (4,3,2), (1,3,1)}");
}

void sf_restage(epwi_ctx *c, const RestageArgs &ra) {
    const int W = ra.W;
    float2 *out = static_cast<float2 *>(ra.ghat_raw);
    auto go = [&](auto kern, int KG) {
        dim3 grid((ra.nrow + 127) / 128, (unsigned)((ra.nkp + KG - 1) / KG));
        const size_t sm = sizeof(float2) * KG * ra.nRe;
        if (sm > 48 * 1024) EPWI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        kern<<<grid, 128, sm, c->stream>>>(ra, out);
        EPWI_CHECK_LAUNCH();
    };
    if (W == 4) go(k_restage_f32<4, 8>, 8);
    else if (W == 1) go(k_restage_f32<1, 8>, 8);
    else go(k_restage_f32<0, 1>, 1);
}

// Rates of the chunk's states: one CTA per (k-point, band), written straight into inv_tau.
void sf_scatter(epwi_ctx *c, const ScatterArgs &sa, int64_t nkp, const int64_t *kp_pairs_local, int64_t p_off,
                const std::vector<int64_t> &h_kp_state_chunk) {
    const int W = c->nw, NM = c->nm, r = c->rp_cube_r;
    SfArgs a;
    a.g = sa.g;
    a.nplane = (int64_t)sa.g.n2 * sa.g.n3;
    int q2max = 1;
    for (int64_t pb = 0; pb * kSieveBlock < a.nplane; ++pb) {
        const int64_t c0 = pb * kSieveBlock, c1 = std::min<int64_t>(a.nplane, c0 + kSieveBlock) - 1;
        q2max = std::max<int>(q2max, (int)(c1 / sa.g.n3 - c0 / sa.g.n3 + 1));
    }
    a.nq2max = q2max;
    a.ph32 = sa.ph32;
    a.ghat = static_cast<const float2 *>(sa.ghat_raw);
    a.kpts = sa.kpts;
    a.win_lo = sa.win_lo;
    a.win_n = sa.win_n;
    a.kp_state = sa.kp_state;
    a.s_base = sa.s_base;
    a.kp_pairs = kp_pairs_local;
    a.p_off = p_off;
    a.pairs = sa.pairs;
    a.V32 = sa.V32;
    a.u32 = sa.u32;
    a.erel = c->tc_erel.as<float>();
    a.f32 = c->tc_f32.as<float>();
    a.n32 = c->tc_n32.as<float>();
    a.hw32 = c->tc_hw32.as<float>();
    a.ceta32 = (float)sa.ceta;
    a.inv_eta32 = (float)(1.0 / sa.eta);
    a.pref = 2.0 * epc::kPi / epc::kHbarEVs / (double)c->nk / (sqrt(epc::kPi) * sa.eta);
    a.inv_tau = c->inv_tau.as<double>();
    // items: (chunk k-point, band), k-point major
    std::vector<int2> items;
    for (int64_t p = 0; p < nkp; ++p)
        for (int64_t n = 0; n < h_kp_state_chunk[p + 1] - h_kp_state_chunk[p]; ++n) items.push_back(make_int2((int)p, (int)n));
    c->sf_items.ensure(sizeof(int2) * (items.size() + 1));
    if (!items.empty())
        EPWI_CUDA(cudaMemcpyAsync(c->sf_items.p, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice,
                                  c->stream));
    a.items = c->sf_items.as<int2>();
    a.gam = sa.gam32;
    a.goff = sa.goff;
    const int ni = (int)items.size();
    if (W == 4 && NM == 3 && r == 2) launch_sf<4, 3, 2>(c, a, ni);
    else if (W == 4 && NM == 3 && r == 1) launch_sf<4, 3, 1>(c, a, ni);
    else if (W == 1 && NM == 3 && r == 1) launch_sf<1, 3, 1>(c, a, ni);
    else sf_check(c);
    // the host vector of items must outlive the copy
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
}
