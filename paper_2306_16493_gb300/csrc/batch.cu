// Many systems of uneven size in one step.  Each system has its own nw, nat, R-sets and grid.
//
// Planning runs each system's eigensolves, window and sieve count, allocates everything, and
// builds one work queue.  A queue item is (system, k-point, window band, block of M_t
// sieved q).  A step is then one CUDA graph:
//   1. per system: phase table, H(k)/D(q) eigensolves, occupations, sieve fill, and the FP32
//      Re->k stage (Eq. 16, inner bracket);
//   2. ONE persistent kernel.  Its CTAs take queue items through an atomic counter and do,
//      per item, the Rp->q product, the rotations by V(k+q) and u(q), and the Gaussian
//      delta sum of the SERTA rate (Eq. 16, Eq. 10) in FP32.  Each item's sum is written in
//      FP64 to its own slot.  When R_p is a cube the product is factorised along axis 1: an
//      item's pairs come in runs of equal q1 (the sieve order), and per run
//      Z = sum_n1 e^{i q1 n1} ghat[n1][n2 n3] is built once, after which each pair sums only
//      the D^2 terms e^{i(q2 n2 + q3 n3)} Z[n2 n3] (D^3 -> D^2 terms per pair);
//   3. fixed-order FP64 reductions of the slots into 1/tau, then sigma per system (Eq. 12).
// The queue is ordered by per-item cost, largest first.  Results do not depend on which CTA
// takes which item: every item has its own output slot and the sums run in item order.
//
// Each system has its own tile shape: the pairs per item M_t and the K chunk of the Rp sum.
// An autotuner picks it by timing the persistent kernel on a sample of each class
// (W, N_m, n_Rp) and caches the choice per class for the process.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "epwi_internal.cuh"
#include "scatter.cuh"

namespace {

constexpr int kBT = 256;          // threads of the persistent kernel
constexpr int kAcc = 32;          // complex accumulators per thread (Rp->q stage)
constexpr int kMaxMt = 512;       // pairs per item, upper bound
constexpr int kNmB = 18;          // modes, upper bound
constexpr size_t kSmemCap = 100 * 1024;   // two CTAs per SM (228 KB per SM)

struct BSys {
    GridInfo g;
    int W, Nm, nRp, NW;           // NW = Nm * W columns of the Rp->q product
    int rc;                       // R_p is the cube [-rc, rc]^3 in n3-fastest order (else -1)
    int CW, RG;                   // columns per thread group (<= 256), row groups = 256 / CW
    int Mt, KC;                   // tile shape: pairs per item, K chunk
    const int *Rp;
    const float2 *ph32;
    const float2 *V32;
    const float2 *u32;
    const float *erel, *f32, *n32, *hw32;
    const float2 *ghat;           // [state][nRp][Nm][W]
    const int *pairs;             // sieved q of every k-point, grouped by k-point
    const int64_t *kp_pairs;      // [nkp + 1]
    const int *kpts, *win_lo;
    const int64_t *kp_state;      // [nkp + 1]
    float inv_eta, ceta;
};

struct BItem {
    int sys, kp, np, p0, cnt;
    int pad[3];
};

__host__ __device__ inline void col_groups(int NW, int &CW, int &RG) {
    CW = NW < kBT ? NW : kBT;
    RG = kBT / CW;
}

// Re->k stage in FP32, two kernels per chunk of k-points.
// 1. Gk[k][c] = sum_Re w e^{ik.Re} g[Re][c] over the flattened c = (rp, mu, i, j): KB
//    k-points per block share every read of g (one 8-byte load per Re feeds KB complex FMAs).
// 2. ghat(k)[state][rp][mu][i] = sum_j Gk[k][(rp, mu, i), j] V_jn(k) for the window bands n.
constexpr int kKB = 32;           // k-points per block of the first kernel
constexpr int kRC = 64;           // Re per shared-memory chunk

__global__ void __launch_bounds__(256) k_gk_f32(int64_t C, int nRe, GridInfo g,
                                                const int *__restrict__ Re,
                                                const float2 *__restrict__ gw,
                                                const float2 *__restrict__ ph, int nkc,
                                                const int *__restrict__ kpts,
                                                float2 *__restrict__ Gk) {
    __shared__ float2 P[kKB][kRC];
    __shared__ int ka[kKB][3];
    const int t = threadIdx.x;
    const int kb0 = blockIdx.y * kKB;
    const int64_t c = (int64_t)blockIdx.x * 256 + t;
    if (t < kKB) {
        int i1 = 0, i2 = 0, i3 = 0;
        if (kb0 + t < nkc) grid_coords(g, kpts[kb0 + t], i1, i2, i3);
        ka[t][0] = i1 * g.s1 % g.L;
        ka[t][1] = i2 * g.s2 % g.L;
        ka[t][2] = i3 * g.s3 % g.L;
    }
    float2 acc[kKB];
#pragma unroll
    for (int kk = 0; kk < kKB; ++kk) acc[kk] = make_float2(0.f, 0.f);
    for (int r0 = 0; r0 < nRe; r0 += kRC) {
        const int rc = min(kRC, nRe - r0);
        __syncthreads();
        for (int e = t; e < kKB * kRC; e += 256) {
            const int kk = e / kRC, rr = e % kRC;
            float2 v = make_float2(0.f, 0.f);
            if (rr < rc && kb0 + kk < nkc) {
                const int *R = Re + 3 * (r0 + rr);
                v = ph[phase_index(ka[kk][0], ka[kk][1], ka[kk][2], R[0], R[1], R[2], g.L)];
            }
            P[kk][rr] = v;
        }
        __syncthreads();
        if (c < C) {
            const float2 *gc = gw + (int64_t)r0 * C + c;
#pragma unroll 4
            for (int rr = 0; rr < rc; ++rr) {
                const float2 gv = gc[(int64_t)rr * C];
#pragma unroll
                for (int kk = 0; kk < kKB; ++kk) acc[kk] = cfmaf(P[kk][rr], gv, acc[kk]);
            }
        }
    }
    if (c < C)
#pragma unroll
        for (int kk = 0; kk < kKB; ++kk)
            if (kb0 + kk < nkc) Gk[(int64_t)(kb0 + kk) * C + c] = acc[kk];
}

__global__ void k_gk_rotate(int nkc, int nrow, int W, const float2 *__restrict__ Gk,
                            const float2 *__restrict__ V32, const int *__restrict__ kpts,
                            const int64_t *__restrict__ kp_state, const int *__restrict__ win_lo,
                            const int *__restrict__ win_n, float2 *__restrict__ ghat) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nkc * nrow) return;
    const int kk = (int)(e / nrow), row = (int)(e % nrow);
    const int ik = kpts[kk];
    const int lo = win_lo[ik], ns = win_n[ik];
    const float2 *gr = Gk + (int64_t)kk * nrow * W + (int64_t)row * W;
    const float2 *Vk = V32 + (int64_t)ik * W * W;
    const int64_t s0 = kp_state[kk];
    for (int np = 0; np < ns; ++np) {
        float2 o = make_float2(0.f, 0.f);
        for (int j = 0; j < W; ++j) o = cfmaf(gr[j], Vk[j * W + lo + np], o);
        ghat[(s0 + np) * (int64_t)nrow + row] = o;
    }
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async_16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The persistent kernel: CTAs take queue items until the queue is empty.
__global__ void __launch_bounds__(kBT, 2) k_batch_scatter(const BSys *__restrict__ systems,
                                                         const BItem *__restrict__ items,
                                                         const int *__restrict__ order,
                                                         int nitems, int *__restrict__ counter,
                                                         double *__restrict__ part) {
    extern __shared__ float2 sm[];
    __shared__ int s_item;
    __shared__ int sq[kMaxMt];
    __shared__ int sa[3][kMaxMt];
    __shared__ int srun[kMaxMt + 1];             // starts of the runs of equal q1 (factorised path)
    __shared__ int s_nrun;
    __shared__ float2 se1[13];                   // axis-1 phases of the current run (rc <= 6)
    __shared__ double sred[kBT / 32];
    const int t = threadIdx.x;
    for (;;) {
        if (t == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const int slot = order[it];
        const BItem I = items[slot];
        const BSys &S = systems[I.sys];
        const int W = S.W, Nm = S.Nm, NW = S.NW, KC = S.KC, cnt = I.cnt;
        const int ik = S.kpts[I.kp];
        const int64_t st = S.kp_state[I.kp] + I.np;
        const int band = S.win_lo[ik] + I.np;
        const float2 *gh = S.ghat + st * (int64_t)S.nRp * NW;
        const int *pl = S.pairs + S.kp_pairs[I.kp] + I.p0;
        for (int p = t; p < cnt; p += kBT) {
            const int iq = pl[p];
            int i1, i2, i3;
            grid_coords(S.g, iq, i1, i2, i3);
            sq[p] = iq;
            sa[0][p] = i1 * S.g.s1 % S.g.L;
            sa[1][p] = i2 * S.g.s2 % S.g.L;
            sa[2][p] = i3 * S.g.s3 % S.g.L;
        }
        // shared memory: two K chunks of ghat [KC][NW], phases [Mt][KC+1], product [Mt][NW]
        float2 *Gs = sm;
        float2 *P = sm + (size_t)2 * KC * NW;
        float2 *Cs = P + (size_t)S.Mt * (KC + 1);
        const int KP = KC + 1;
        const int cg = t % S.CW, rg = t / S.CW;
        const bool tact = rg < S.RG;
        const int ncol = (NW + S.CW - 1) / S.CW;            // 1 or 2
        const int npt = (cnt + S.RG - 1) / S.RG;            // pairs per thread
        float2 acc[kAcc];
#pragma unroll
        for (int a = 0; a < kAcc; ++a) acc[a] = make_float2(0.f, 0.f);
        __syncthreads();
        // runs of equal q1 (the sieve lists a k-point's pairs by plane block, then q1, so the
        // pairs of one q1 are contiguous): the factorised path needs at least 4 pairs per run
        const bool fac = S.rc >= 0 && S.rc <= 6 &&
                         4 * __syncthreads_count(t < cnt && (t == 0 || sa[0][t] != sa[0][t - 1]) ||
                                                 (t + kBT < cnt && sa[0][t + kBT] != sa[0][t + kBT - 1]))
                             <= cnt;
        if (fac && t < 32) {
            // ordered run starts, by warp 0
            int nr = 0;
            for (int p0 = 0; p0 < cnt; p0 += 32) {
                const int p = p0 + t;
                unsigned bits = __ballot_sync(0xffffffffu, p < cnt && (p == 0 || sa[0][p] != sa[0][p - 1]));
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    if (t == 0) srun[nr] = p0 + b;
                    ++nr;
                }
            }
            if (t == 0) {
                srun[nr] = cnt;
                s_nrun = nr;
            }
        }
        __syncthreads();
        if (fac) {
            // ---- Rp -> q factorised along axis 1: per K chunk of the (n2, n3) plane,
            // C[p] += sum_(n2,n3) e^{i(q2 n2 + q3 n3)} Z_q1[n2 n3], Z_q1 = sum_n1 e^{i q1 n1} ghat[n1][n2 n3],
            // Z built once per run of equal q1 and chunk (the CTA reads ghat from L2)
            const int rc = S.rc, D = 2 * rc + 1, DD = D * D, L = S.g.L;
            float2 *Z = Gs;                                   // [KC][NW]
            const int nchf = (DD + KC - 1) / KC;
            for (int j = 0; j < s_nrun; ++j) {
                const int lo = srun[j], hi = srun[j + 1];
                if (t < D) {
                    int x = (sa[0][lo] * (t - rc)) % L;
                    if (x < 0) x += L;
                    se1[t] = S.ph32[x];                       // e^{i q1 n1}, n1 = t - rc
                }
                // this thread's pairs p = rg + i RG inside [lo, hi)
                unsigned in = 0u;
#pragma unroll
                for (int i = 0; i < kAcc; ++i) {
                    const int pi = rg + i * S.RG;
                    if (i < npt && pi >= lo && pi < hi) in |= 1u << i;
                }
                __syncthreads();
                for (int ch = 0; ch < nchf; ++ch) {
                    const int r0 = ch * KC, kc = min(KC, DD - r0);
                    for (int e = t; e < (hi - lo) * KC; e += kBT) {
                        const int p = lo + e / KC, kk = e % KC;
                        float2 v = make_float2(0.f, 0.f);
                        if (kk < kc) {
                            const int n2 = (r0 + kk) / D - rc, n3 = (r0 + kk) % D - rc;
                            int x = (sa[1][p] * n2 + sa[2][p] * n3) % L;
                            if (x < 0) x += L;
                            v = S.ph32[x];
                        }
                        P[p * KP + kk] = v;
                    }
                    for (int e = t; e < kc * NW; e += kBT) {
                        const int kk = e / NW, col = e - kk * NW;
                        const float2 *src = gh + (int64_t)(r0 + kk) * NW + col;
                        float2 z = make_float2(0.f, 0.f);
                        for (int j1 = 0; j1 < D; ++j1) z = cfmaf(se1[j1], src[(int64_t)j1 * DD * NW], z);
                        Z[kk * NW + col] = z;
                    }
                    __syncthreads();
                    if (tact) {
                        if (ncol == 1) {
                            for (int kk = 0; kk < kc; ++kk) {
                                const float2 g0 = Z[kk * NW + cg];
                                const float2 *pk = P + rg * KP + kk;
#pragma unroll
                                for (int i = 0; i < kAcc; ++i)
                                    if ((in >> i) & 1u) acc[i] = cfmaf(pk[i * S.RG * KP], g0, acc[i]);
                            }
                        } else {
                            const bool c1 = cg + S.CW < NW;
                            for (int kk = 0; kk < kc; ++kk) {
                                const float2 g0 = Z[kk * NW + cg];
                                const float2 g1 = c1 ? Z[kk * NW + cg + S.CW] : make_float2(0.f, 0.f);
                                const float2 *pk = P + rg * KP + kk;
#pragma unroll
                                for (int i = 0; i < kAcc / 2; ++i)
                                    if ((in >> i) & 1u) {
                                        const float2 pv = pk[i * S.RG * KP];
                                        acc[2 * i] = cfmaf(pv, g0, acc[2 * i]);
                                        acc[2 * i + 1] = cfmaf(pv, g1, acc[2 * i + 1]);
                                    }
                            }
                        }
                    }
                    __syncthreads();
                }
            }
        } else {
            // ---- Rp -> q: C[p][mu, i] = sum_Rp e^{i q_p . Rp} ghat[Rp][mu][i]; the K chunks of
            // ghat are copied to shared memory with cp.async, one chunk ahead of the compute
            const int nch = (S.nRp + KC - 1) / KC;
            auto issue = [&](int ch) {
                if (ch < nch) {
                    const int r0 = ch * KC, kc = min(KC, S.nRp - r0);
                    const float2 *src = gh + (int64_t)r0 * NW;
                    float2 *dst = Gs + (size_t)(ch & 1) * KC * NW;
                    if ((NW & 1) == 0) {
                        for (int e = t; e < kc * NW / 2; e += kBT) cp_async_16(dst + 2 * e, src + 2 * e);
                    } else {
                        for (int e = t; e < kc * NW; e += kBT) cp_async_8(dst + e, src + e);
                    }
                }
                cp_async_commit_group();
            };
            issue(0);
            for (int ch = 0; ch < nch; ++ch) {
                issue(ch + 1);
                const int r0 = ch * KC, kc = min(KC, S.nRp - r0);
                for (int e = t; e < cnt * KC; e += kBT) {
                    const int p = e / KC, kk = e - p * KC;
                    float2 v = make_float2(0.f, 0.f);
                    if (kk < kc) {
                        const int *R = S.Rp + 3 * (r0 + kk);
                        v = S.ph32[phase_index(sa[0][p], sa[1][p], sa[2][p], R[0], R[1], R[2], S.g.L)];
                    }
                    P[p * KP + kk] = v;
                }
                cp_async_wait_group<1>();
                __syncthreads();
                if (tact) {
                    const float2 *G = Gs + (size_t)(ch & 1) * KC * NW;
                    const int nv = min(npt, (cnt - rg + S.RG - 1) / S.RG);   // valid pairs
                    if (ncol == 1) {
                        for (int kk = 0; kk < kc; ++kk) {
                            const float2 g0 = G[kk * NW + cg];
                            const float2 *pk = P + rg * KP + kk;
    #pragma unroll
                            for (int i = 0; i < kAcc; ++i)
                                if (i < nv) acc[i] = cfmaf(pk[i * S.RG * KP], g0, acc[i]);
                        }
                    } else {
                        const bool c1 = cg + S.CW < NW;
                        for (int kk = 0; kk < kc; ++kk) {
                            const float2 g0 = G[kk * NW + cg];
                            const float2 g1 = c1 ? G[kk * NW + cg + S.CW] : make_float2(0.f, 0.f);
                            const float2 *pk = P + rg * KP + kk;
    #pragma unroll
                            for (int i = 0; i < kAcc / 2; ++i)
                                if (i < nv) {
                                    const float2 pv = pk[i * S.RG * KP];
                                    acc[2 * i] = cfmaf(pv, g0, acc[2 * i]);
                                    acc[2 * i + 1] = cfmaf(pv, g1, acc[2 * i + 1]);
                                }
                        }
                    }
                }
                __syncthreads();
            }
        }
        cp_async_wait_group<0>();
        if (tact) {
#pragma unroll
            for (int a = 0; a < kAcc; ++a) {
                const int i = ncol == 1 ? a : (a >> 1);
                const int j = ncol == 1 ? 0 : (a & 1);
                const int p = rg + i * S.RG, c = cg + j * S.CW;
                if (i < npt && p < cnt && c < NW) Cs[(size_t)p * NW + c] = acc[a];
            }
        }
        __syncthreads();
        // ---- rotations and the delta sum: one (pair, m) per thread
        const float en = S.erel[(int64_t)ik * W + band];
        float rate = 0.f;
        for (int u = t; u < cnt * W; u += kBT) {
            const int p = u / W, m = u - p * W;
            const int iq = sq[p];
            const int64_t ikq = kplusq(S.g, ik, iq);
            const float2 *Vq = S.V32 + ikq * W * W;
            const float2 *Cp = Cs + (size_t)p * NW;
            float2 h[kNmB];
#pragma unroll
            for (int mu = 0; mu < kNmB; ++mu) h[mu] = make_float2(0.f, 0.f);
            for (int i = 0; i < W; ++i) {             // one load of V_im(k+q) per i
                const float2 v = Vq[i * W + m];
#pragma unroll
                for (int mu = 0; mu < kNmB; ++mu)
                    if (mu < Nm) h[mu] = cfmacf(v, Cp[mu * W + i], h[mu]);
            }
            const float em = S.erel[ikq * W + m];
            const float fm = S.f32[ikq * W + m];
            const float2 *uq = S.u32 + (int64_t)iq * Nm * Nm;
            for (int nu = 0; nu < Nm; ++nu) {
                const float w = S.hw32[(int64_t)iq * Nm + nu];
                if (w < 0.f) continue;
                const float x1 = (en + w) - em, x2 = (en - w) - em;
                const bool t1 = fabsf(x1) <= S.ceta, t2 = fabsf(x2) <= S.ceta;
                if (!t1 && !t2) continue;
                float2 gv = make_float2(0.f, 0.f);
#pragma unroll
                for (int mu = 0; mu < kNmB; ++mu)
                    if (mu < Nm) gv = cfmaf(h[mu], uq[mu * Nm + nu], gv);
                const float g2 = gv.x * gv.x + gv.y * gv.y;
                const float N = S.n32[(int64_t)iq * Nm + nu];
                float term = 0.f;
                if (t1) {
                    const float y = x1 * S.inv_eta;
                    term += (N + fm) * expf(-y * y);
                }
                if (t2) {
                    const float y = x2 * S.inv_eta;
                    term += (1.f + N - fm) * expf(-y * y);
                }
                rate = fmaf(g2, term, rate);
            }
        }
        double r = rate;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
        if ((t & 31) == 0) sred[t >> 5] = r;
        __syncthreads();
        if (t == 0) {
            double s = 0;
            for (int w = 0; w < kBT / 32; ++w) s += sred[w];
            part[slot] = s;
        }
    }
}

// 1/tau of every batch state: pref of its system times the sum of its items' slots in order.
__global__ void k_batch_reduce(int64_t ns, const int64_t *__restrict__ state_item,
                               const int *__restrict__ state_sys, const double *__restrict__ pref,
                               const double *__restrict__ part, double *__restrict__ inv_tau) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    double v = 0;
    for (int64_t i = state_item[s]; i < state_item[s + 1]; ++i) v += part[i];
    inv_tau[s] = pref[state_sys[s]] * v;
}

struct SigmaDesc {
    int64_t ns, s0;               // states of the system, first batch state
    int W;
    const int *st_k, *st_n;
    const double *eps, *vel;
    double mu, kT, pref;
};

// sigma per system (one block each): fixed-order FP64 sums of v_a v_b tau f(1-f)/kT.
__global__ void __launch_bounds__(256) k_batch_sigma(const SigmaDesc *__restrict__ d,
                                                     const double *__restrict__ inv_tau,
                                                     double *__restrict__ sigma) {
    __shared__ double sm[6][256];
    const SigmaDesc D = d[blockIdx.x];
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t s = threadIdx.x; s < D.ns; s += 256) {
        const double r = inv_tau[D.s0 + s];
        if (!(r > 0)) continue;
        const int k = D.st_k[s], n = D.st_n[s];
        const double x = (D.eps[(int64_t)k * D.W + n] - D.mu) / D.kT;
        const double ex = exp(-fabs(x));
        const double f = x > 0 ? ex / (1.0 + ex) : 1.0 / (1.0 + ex);
        const double w = f * (1.0 - f) / r;
        const double *vv = D.vel + ((int64_t)k * D.W + n) * 3;
        v[0] += w * vv[0] * vv[0];
        v[1] += w * vv[1] * vv[1];
        v[2] += w * vv[2] * vv[2];
        v[3] += w * vv[0] * vv[1];
        v[4] += w * vv[0] * vv[2];
        v[5] += w * vv[1] * vv[2];
    }
    for (int j = 0; j < 6; ++j) sm[j][threadIdx.x] = v[j];
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int j = 0; j < 6; ++j) sm[j][threadIdx.x] += sm[j][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double h[6] = {sm[0][0], sm[1][0], sm[2][0], sm[3][0], sm[4][0], sm[5][0]};
        const double tt[9] = {h[0], h[3], h[4], h[3], h[1], h[5], h[4], h[5], h[2]};
        for (int i = 0; i < 9; ++i) sigma[blockIdx.x * 9 + i] = D.pref * tt[i];
    }
}

size_t smem_bytes(int Mt, int KC, int NW) {
    return sizeof(float2) * ((size_t)2 * KC * NW + (size_t)Mt * (KC + 1) + (size_t)Mt * NW);
}

bool tile_ok(int Mt, int KC, int NW) {
    int CW, RG;
    col_groups(NW, CW, RG);
    const int ncol = (NW + CW - 1) / CW;
    const int npt = (Mt + RG - 1) / RG;
    return Mt >= 1 && Mt <= kMaxMt && ncol <= 2 && npt * ncol <= kAcc &&
           smem_bytes(Mt, KC, NW) <= kSmemCap;
}

using TileKey = std::tuple<int, int, int>;           // (W, Nm, nRp)
std::map<TileKey, std::pair<int, int>> g_tile_cache;  // autotuned (Mt, KC) per class

}  // namespace

// ------------------------------------------------------------------------------ batch
struct epwi_batch {
    epwi_options opt{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<epwi_ctx *> sys;
    std::vector<std::array<int, 3>> grids;
    bool planned = false;
    double T = 0, eta = 0;
    std::vector<double> mu, emin, emax;
    // per system device data of the step
    std::vector<DevBuf> pairs, ghat;
    std::vector<std::vector<int64_t>> h_state;
    std::vector<BSys> hsys;
    std::vector<int> tile_src;               // 0 default, 1 autotuned, 2 cached, 3 set
    std::vector<std::pair<int, int>> forced; // tiles set by epwi_batch_set_tile (0: none)
    DevBuf d_sys, d_items, d_order, d_counter, d_part, d_state_item, d_state_sys, d_pref;
    DevBuf d_inv_tau, d_sigdesc, d_sigma;
    DevBuf d_gk;                             // Re->k scratch, reused by every system
    std::vector<int64_t> sys_state0;
    int64_t nitems = 0, nstates = 0, npairs = 0;
    size_t smem = 0;
    int grid_ctas = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    epwi_batch_stats stats{};

    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    ~epwi_batch() {
        drop_graph();
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        for (auto &b : pairs) b.release();
        for (auto &b : ghat) b.release();
        DevBuf *all[] = {&d_sys, &d_items, &d_order, &d_counter, &d_part, &d_state_item,
                         &d_state_sys, &d_pref, &d_inv_tau, &d_sigdesc, &d_sigma, &d_gk};
        for (DevBuf *b : all) b->release();
        for (epwi_ctx *c : sys) epwi_destroy(c);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

template <class F>
epwi_status bguard(epwi_batch *b, F &&f) {
    if (!b) return EPWI_EINVAL;
    try {
        EPWI_CUDA(cudaSetDevice(b->device));
        f();
        b->err.clear();
        return EPWI_OK;
    } catch (const EpwiError &e) {
        b->err = e.msg;
        return e.status;
    } catch (const std::bad_alloc &) {
        b->err = "host allocation failed";
        return EPWI_ENOMEM;
    } catch (...) {
        b->err = "unexpected internal error";
        return EPWI_ECUDA;
    }
}

void check(epwi_ctx *c, epwi_status st, const char *what) {
    if (st != EPWI_OK)
        throw EpwiError{st, std::string(what) + ": " + epwi_last_error(c)};
}

template <class T>
void put(DevBuf &b, const std::vector<T> &v, cudaStream_t st) {
    b.ensure(sizeof(T) * (v.size() + 1));
    if (!v.empty())
        EPWI_CUDA(cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
}

// Chunk of k-points per pass of the two-kernel Re->k stage (the scratch Gk holds
// chunk * nRp * Nm * W^2 complex FP32 values).
int64_t restage_chunk(const epwi_ctx *c) {
    const int64_t C = (int64_t)c->nRp * c->nm * c->nw * c->nw;
    const int64_t kch = std::max<int64_t>(kKB, ((int64_t(1) << 31) / (8 * C)) / kKB * kKB);
    return std::min<int64_t>(kch, std::max<int64_t>(c->nkp, 1));
}

void restage(epwi_batch *b, int s) {
    epwi_ctx *c = b->sys[s];
    const int64_t nrow = (int64_t)c->nRp * c->nm * c->nw;
    const int64_t C = nrow * c->nw;
    GridInfo g = make_grid_info(c);
    const int64_t nkp = c->nkp;
    const int64_t kch = restage_chunk(c);
    for (int64_t k0 = 0; k0 < nkp; k0 += kch) {
        const int nkc = (int)std::min(kch, nkp - k0);
        dim3 grid((unsigned)((C + 255) / 256), (unsigned)((nkc + kKB - 1) / kKB));
        k_gk_f32<<<grid, 256, 0, b->stream>>>(C, c->nRe, g, c->Re.as<int>(), c->gw32.as<float2>(),
                                               c->ph32.as<float2>(), nkc, c->kpts.as<int>() + k0,
                                               b->d_gk.as<float2>());
        EPWI_CHECK_LAUNCH();
        const int64_t n2 = (int64_t)nkc * nrow;
        k_gk_rotate<<<(unsigned)((n2 + 255) / 256), 256, 0, b->stream>>>(
            nkc, (int)nrow, c->nw, b->d_gk.as<float2>(), c->V32.as<float2>(), c->kpts.as<int>() + k0,
            c->kp_state.as<int64_t>() + k0, c->win_lo.as<int>(), c->win_n.as<int>(),
            b->ghat[s].as<float2>());
        EPWI_CHECK_LAUNCH();
    }
}

// The per-system work that precedes the persistent kernel in every step.
void system_prologue(epwi_batch *b, int s) {
    epwi_ctx *c = b->sys[s];
    launch_phase_tables(c);
    launch_eigs(c);
    occupation_tables(c);
    tc_tables(c);
    sieve_fill_chunk(c, 0, c->nkp, b->pairs[s].as<int>());
    restage(b, s);
}

// Items of system s in (k-point, band, q block) order, with their states' item offsets.
void build_items(epwi_batch *b, int s, int Mt, std::vector<BItem> &items,
                 std::vector<int64_t> &state_item) {
    epwi_ctx *c = b->sys[s];
    const auto &hs = b->h_state[s];
    for (int64_t kp = 0; kp < c->nkp; ++kp) {
        const int64_t np = c->h_kp_pairs[kp + 1] - c->h_kp_pairs[kp];
        const int ns = (int)(hs[kp + 1] - hs[kp]);
        for (int n = 0; n < ns; ++n) {
            state_item.push_back((int64_t)items.size());
            for (int64_t p0 = 0; p0 < np; p0 += Mt) {
                BItem it{};
                it.sys = s;
                it.kp = (int)kp;
                it.np = n;
                it.p0 = (int)p0;
                it.cnt = (int)std::min<int64_t>(Mt, np - p0);
                items.push_back(it);
            }
        }
    }
}

void fill_bsys(epwi_batch *b, int s, int Mt, int KC, BSys &d) {
    epwi_ctx *c = b->sys[s];
    d.g = make_grid_info(c);
    d.W = c->nw;
    d.Nm = c->nm;
    d.nRp = c->nRp;
    d.rc = c->rp_cube_r;
    d.NW = c->nw * c->nm;
    col_groups(d.NW, d.CW, d.RG);
    d.Mt = Mt;
    d.KC = KC;
    d.Rp = c->Rp.as<int>();
    d.ph32 = c->ph32.as<float2>();
    d.V32 = c->V32.as<float2>();
    d.u32 = c->u32.as<float2>();
    d.erel = c->tc_erel.as<float>();
    d.f32 = c->tc_f32.as<float>();
    d.n32 = c->tc_n32.as<float>();
    d.hw32 = c->tc_hw32.as<float>();
    d.ghat = b->ghat[s].as<float2>();
    d.pairs = b->pairs[s].as<int>();
    d.kp_pairs = c->kp_pairs.as<int64_t>();
    d.kpts = c->kpts.as<int>();
    d.win_lo = c->win_lo.as<int>();
    d.kp_state = c->kp_state.as<int64_t>();
    d.inv_eta = (float)(1.0 / c->eta);
    d.ceta = (float)(c->opt.sieve_c * c->eta);
}

int persistent_grid(epwi_batch *b, size_t smem) {
    int nsm = 0, per = 0;
    EPWI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
    EPWI_CUDA(cudaFuncSetAttribute(k_batch_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)std::max<size_t>(smem, 1)));
    EPWI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_scatter, kBT, smem));
    EPWI_REQUIRE(per >= 1, EPWI_EUNSUPPORTED, "persistent kernel does not fit on an SM");
    return nsm * per;
}

// Times the persistent kernel for system s with tile (Mt, KC) on up to `sample` items.
float time_tile(epwi_batch *b, int s, int Mt, int KC, int64_t sample, int64_t *pairs_out) {
    std::vector<BItem> items;
    std::vector<int64_t> si;
    build_items(b, s, Mt, items, si);
    if ((int64_t)items.size() > sample) items.resize(sample);
    int64_t pairs = 0;
    for (auto &it : items) pairs += it.cnt;
    *pairs_out = pairs;
    if (items.empty()) return 0.f;
    for (auto &it : items) it.sys = 0;
    BSys d;
    fill_bsys(b, s, Mt, KC, d);
    std::vector<BSys> v(1, d);
    std::vector<int> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    DevBuf ds, di, dord, dc, dp;
    float best = 1e30f;
    try {
        put(ds, v, b->stream);
        put(di, items, b->stream);
        put(dord, order, b->stream);
        dc.ensure(sizeof(int));
        dp.ensure(sizeof(double) * items.size());
        const size_t sm = smem_bytes(Mt, KC, d.NW);
        const int grid = persistent_grid(b, sm);
        for (int rep = 0; rep < 2; ++rep) {
            EPWI_CUDA(cudaMemsetAsync(dc.p, 0, sizeof(int), b->stream));
            cudaEventRecord(b->ev[0], b->stream);
            k_batch_scatter<<<grid, kBT, sm, b->stream>>>(ds.as<BSys>(), di.as<BItem>(),
                                                         dord.as<int>(), (int)items.size(),
                                                         dc.as<int>(), dp.as<double>());
            EPWI_CHECK_LAUNCH();
            cudaEventRecord(b->ev[1], b->stream);
            EPWI_CUDA(cudaEventSynchronize(b->ev[1]));
            float ms = 0;
            cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
            if (rep > 0) best = std::min(best, ms);
        }
    } catch (...) {
        cudaStreamSynchronize(b->stream);
        ds.release(); di.release(); dord.release(); dc.release(); dp.release();
        throw;
    }
    EPWI_CUDA(cudaStreamSynchronize(b->stream));
    ds.release(); di.release(); dord.release(); dc.release(); dp.release();
    return best;
}

std::pair<int, int> default_tile(int NW) {
    static const int mts[] = {128, 64, 32, 16, 8, 4, 2, 1};
    for (int mt : mts)
        for (int kc : {32, 16, 8, 4})
            if (tile_ok(mt, kc, NW)) return {mt, kc};
    return {1, 4};
}

std::pair<int, int> autotune(epwi_batch *b, int s, int &src) {
    epwi_ctx *c = b->sys[s];
    const TileKey key{c->nw, c->nm, c->nRp};
    auto it = g_tile_cache.find(key);
    if (it != g_tile_cache.end()) {
        src = 2;
        return it->second;
    }
    const int NW = c->nw * c->nm;
    std::pair<int, int> best = default_tile(NW);
    double best_t = 1e300;
    for (int mt : {8, 16, 32, 64, 128, 256}) {
        for (int kc : {8, 16, 32}) {
            if (!tile_ok(mt, kc, NW)) continue;
            int64_t pairs = 0;
            const float ms = time_tile(b, s, mt, kc, 1024, &pairs);
            if (pairs == 0) continue;
            const double per = ms / (double)pairs;
            if (per < best_t) {
                best_t = per;
                best = {mt, kc};
            }
        }
    }
    src = 1;
    if (best_t < 1e300) g_tile_cache[key] = best;
    return best;
}

void plan(epwi_batch *b, bool tune) {
    b->drop_graph();
    b->planned = false;
    const int ns = (int)b->sys.size();
    cudaStream_t st = b->stream;
    b->pairs.resize(ns);
    b->ghat.resize(ns);
    b->h_state.assign(ns, {});
    b->hsys.assign(ns, BSys{});
    b->tile_src.assign(ns, 0);
    std::vector<std::pair<int, int>> tiles(ns);
    int64_t npairs = 0, nstates = 0;
    double ms_plan = 0;
    cudaEvent_t p0 = nullptr, p1 = nullptr;
    EPWI_CUDA(cudaEventCreate(&p0));
    EPWI_CUDA(cudaEventCreate(&p1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } evg{p0, p1};
    cudaEventRecord(p0, st);
    for (int s = 0; s < ns; ++s) {
        epwi_ctx *c = b->sys[s];
        c->T = b->T;
        c->mu = b->mu[s];
        c->eta = b->eta;
        c->emin = b->emin[s];
        c->emax = b->emax[s];
        const int g3[3] = {b->grids[s][0], b->grids[s][1], b->grids[s][2]};
        check(c, epwi_eigs(c, g3, g3), "epwi_eigs");
        build_window(c);
        ensure_velocities(c, false);
        sieve_count(c);
        occupation_tables(c);
        tc_tables(c);
        b->h_state[s].resize(c->nkp + 1);
        EPWI_CUDA(cudaMemcpyAsync(b->h_state[s].data(), c->kp_state.p, sizeof(int64_t) * (c->nkp + 1),
                                  cudaMemcpyDeviceToHost, st));
        EPWI_CUDA(cudaStreamSynchronize(st));
        b->pairs[s].ensure(sizeof(int) * (c->npairs + 1));
        const int64_t nrow = (int64_t)c->nRp * c->nm * c->nw;
        b->ghat[s].ensure(sizeof(float2) * (size_t)nrow * (c->nstates + 1));
        {
            // grow-only scratch: sized before any capture so that captured passes never allocate
            const size_t gk = sizeof(float2) * (size_t)restage_chunk(c) * nrow * c->nw;
            if (gk > b->d_gk.bytes) {
                EPWI_CUDA(cudaStreamSynchronize(st));
                b->d_gk.ensure(gk);
            }
        }
        sieve_fill_chunk(c, 0, c->nkp, b->pairs[s].as<int>());
        restage(b, s);
        npairs += c->npairs;
        nstates += c->nstates;
    }
    EPWI_CUDA(cudaStreamSynchronize(st));
    // tile shapes
    for (int s = 0; s < ns; ++s) {
        epwi_ctx *c = b->sys[s];
        const int NW = c->nw * c->nm;
        if ((int)b->forced.size() == ns && b->forced[s].first > 0) {
            tiles[s] = b->forced[s];
            b->tile_src[s] = 3;
        } else if (tune && c->npairs > 0) {
            tiles[s] = autotune(b, s, b->tile_src[s]);
        } else {
            tiles[s] = default_tile(NW);
        }
        EPWI_REQUIRE(tile_ok(tiles[s].first, tiles[s].second, NW), EPWI_EUNSUPPORTED,
                     "no tile shape fits this system (nw * modes too large)");
    }
    // queue: items of every system, state offsets, per-item cost order
    std::vector<BItem> items;
    std::vector<int64_t> state_item;
    std::vector<int> state_sys;
    std::vector<double> pref(ns);
    b->sys_state0.assign(ns + 1, 0);
    size_t smem = 0;
    for (int s = 0; s < ns; ++s) {
        epwi_ctx *c = b->sys[s];
        b->sys_state0[s] = (int64_t)state_item.size();
        build_items(b, s, tiles[s].first, items, state_item);
        state_sys.resize(state_item.size(), s);
        fill_bsys(b, s, tiles[s].first, tiles[s].second, b->hsys[s]);
        pref[s] = 2.0 * epc::kPi / epc::kHbarEVs / (double)c->nk / (std::sqrt(epc::kPi) * c->eta);
        smem = std::max(smem, smem_bytes(tiles[s].first, tiles[s].second, c->nw * c->nm));
    }
    b->sys_state0[ns] = (int64_t)state_item.size();
    state_item.push_back((int64_t)items.size());
    std::vector<double> cost(ns);
    for (int s = 0; s < ns; ++s) {
        const BSys &d = b->hsys[s];
        cost[s] = (double)d.nRp * d.NW + 2.0 * d.W * (d.NW + d.Nm * d.Nm);
    }
    std::vector<int> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return cost[items[x].sys] * items[x].cnt > cost[items[y].sys] * items[y].cnt;
    });
    EPWI_REQUIRE(items.size() < (size_t)INT32_MAX, EPWI_EUNSUPPORTED, "more than 2^31 queue items");
    put(b->d_sys, b->hsys, st);
    put(b->d_items, items, st);
    put(b->d_order, order, st);
    put(b->d_state_item, state_item, st);
    put(b->d_state_sys, state_sys, st);
    put(b->d_pref, pref, st);
    b->d_counter.ensure(sizeof(int));
    b->d_part.ensure(sizeof(double) * (items.size() + 1));
    b->d_inv_tau.ensure(sizeof(double) * (nstates + 1));
    std::vector<SigmaDesc> sd(ns);
    for (int s = 0; s < ns; ++s) {
        epwi_ctx *c = b->sys[s];
        const double kT = epc::kKbEVK * c->T;
        sd[s] = SigmaDesc{c->nstates, b->sys_state0[s], c->nw, c->st_k.as<int>(), c->st_n.as<int>(),
                          c->eps.as<double>(), c->vel.as<double>(), c->mu, kT,
                          2.0 * epc::kECharge * epc::kECharge /
                              ((double)c->nk * c->volume * 1e-30 * kT * epc::kECharge)};
    }
    put(b->d_sigdesc, sd, st);
    b->d_sigma.ensure(sizeof(double) * 9 * ns);
    b->nitems = (int64_t)items.size();
    b->nstates = nstates;
    b->npairs = npairs;
    b->smem = smem;
    b->grid_ctas = persistent_grid(b, smem);
    cudaEventRecord(p1, st);
    EPWI_CUDA(cudaStreamSynchronize(st));
    float ms = 0;
    cudaEventElapsedTime(&ms, p0, p1);
    ms_plan = ms;
    // capture the step
    EPWI_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    try {
        for (int s = 0; s < ns; ++s) system_prologue(b, s);
        EPWI_CUDA(cudaMemsetAsync(b->d_counter.p, 0, sizeof(int), st));
        // external event records become graph nodes (a plain record inside a capture does not)
        EPWI_CUDA(cudaEventRecordWithFlags(b->ev[2], st, cudaEventRecordExternal));
        if (b->nitems > 0) {
            k_batch_scatter<<<b->grid_ctas, kBT, b->smem, st>>>(
                b->d_sys.as<BSys>(), b->d_items.as<BItem>(), b->d_order.as<int>(), (int)b->nitems,
                b->d_counter.as<int>(), b->d_part.as<double>());
            EPWI_CHECK_LAUNCH();
        }
        EPWI_CUDA(cudaEventRecordWithFlags(b->ev[3], st, cudaEventRecordExternal));
        if (nstates > 0) {
            k_batch_reduce<<<(unsigned)((nstates + 255) / 256), 256, 0, st>>>(
                nstates, b->d_state_item.as<int64_t>(), b->d_state_sys.as<int>(),
                b->d_pref.as<double>(), b->d_part.as<double>(), b->d_inv_tau.as<double>());
            EPWI_CHECK_LAUNCH();
        }
        k_batch_sigma<<<ns, 256, 0, st>>>(b->d_sigdesc.as<SigmaDesc>(), b->d_inv_tau.as<double>(),
                                          b->d_sigma.as<double>());
        EPWI_CHECK_LAUNCH();
    } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(st, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    EPWI_CUDA(cudaStreamEndCapture(st, &b->graph));
    EPWI_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    size_t nodes = 0;
    EPWI_CUDA(cudaGraphGetNodes(b->graph, nullptr, &nodes));
    std::memset(&b->stats, 0, sizeof(b->stats));
    b->stats.n_systems = ns;
    b->stats.n_states = nstates;
    b->stats.n_pairs = npairs;
    b->stats.n_items = b->nitems;
    b->stats.graph_nodes = (int64_t)nodes;
    b->stats.persistent_ctas = b->grid_ctas;
    b->stats.smem_bytes = (int64_t)smem;
    b->stats.ms_plan = ms_plan;
    // flops of the algorithm each system runs in the persistent kernel: the Rp->q product (a
    // full R_p sum per pair and band, or for a cube R_p the axis-1 factorisation: D^2 terms per
    // pair and band, plus one D^3 build of Z per item, counting one run of equal q1 per item)
    // and the rotations (per pair, band and final band m: V^dag(k+q) C, N_m W complex
    // multiply-adds, then u(q), N_m^2)
    std::vector<int64_t> sys_items(ns, 0);
    for (const BItem &it : items) ++sys_items[it.sys];
    double fl = 0, rfl = 0;
    for (int s = 0; s < ns; ++s) {
        epwi_ctx *c = b->sys[s];
        const double nbar = (double)c->nstates / std::max<int64_t>(1, c->nkp);
        const double cols = 8.0 * c->nm * c->nw;
        if (c->rp_cube_r >= 0 && c->rp_cube_r <= 6) {
            const double D = 2.0 * c->rp_cube_r + 1;
            fl += cols * (D * D * (double)c->npairs * nbar + D * D * D * (double)sys_items[s]);
        } else {
            fl += cols * c->nRp * (double)c->npairs * nbar;
        }
        fl += 8.0 * c->nw * ((double)c->nm * c->nw + (double)c->nm * c->nm) * (double)c->npairs * nbar;
        rfl += 8.0 * c->nRe * c->nRp * c->nm * (double)c->nw * c->nw * c->nkp;
    }
    b->stats.scatter_flops = fl;
    b->stats.restage_flops = rfl;
    b->planned = true;
}

}  // namespace

extern "C" {

epwi_status epwi_batch_create(epwi_batch **out, const epwi_options *opt) {
    if (!out) return EPWI_EINVAL;
    *out = nullptr;
    epwi_batch *b = nullptr;
    try {
        b = new epwi_batch();
    } catch (...) {
        return EPWI_ENOMEM;
    }
    if (opt) b->opt = *opt;
    else epwi_default_options(&b->opt);
    b->opt.precision = EPWI_FP64;    // the eigen-tables; the batch kernels are FP32
    b->device = b->opt.device;
    epwi_status st = bguard(b, [&] {
        int n = 0;
        EPWI_CUDA(cudaGetDeviceCount(&n));
        EPWI_REQUIRE(b->device >= 0 && b->device < n, EPWI_EINVAL, "no such CUDA device");
        EPWI_CUDA(cudaSetDevice(b->device));
        if (b->opt.cuda_stream) {
            b->stream = (cudaStream_t)b->opt.cuda_stream;
        } else {
            EPWI_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
            b->own_stream = true;
        }
        b->opt.cuda_stream = b->stream;
        for (auto &e : b->ev) EPWI_CUDA(cudaEventCreate(&e));
    });
    if (st != EPWI_OK) {
        delete b;
        return st;
    }
    *out = b;
    return EPWI_OK;
}

void epwi_batch_destroy(epwi_batch *b) { delete b; }

const char *epwi_batch_last_error(const epwi_batch *b) { return b ? b->err.c_str() : "null batch"; }

namespace {
void add_system(epwi_batch *b, const epwi_system *sys, const int32_t *grid) {
    for (int a = 0; a < 3; ++a) EPWI_REQUIRE(grid[a] >= 1, EPWI_EINVAL, "grid sizes must be >= 1");
    b->drop_graph();
    b->planned = false;
    epwi_ctx *c = nullptr;
    EPWI_REQUIRE(epwi_create(&c, &b->opt) == EPWI_OK, EPWI_ECUDA, "context creation failed");
    b->sys.push_back(c);
    c->keep_g64 = false;             // the batch stages g in FP32 only
    check(c, epwi_setup(c, sys), "epwi_setup");
    b->grids.push_back({grid[0], grid[1], grid[2]});
}
}  // namespace

epwi_status epwi_batch_setup(epwi_batch *b, int32_t nsys, const epwi_system *systems,
                             const int32_t *grids) {
    return bguard(b, [&] {
        EPWI_REQUIRE(nsys >= 1 && systems && grids, EPWI_EINVAL, "bad argument");
        b->drop_graph();
        b->planned = false;
        for (epwi_ctx *c : b->sys) epwi_destroy(c);
        b->sys.clear();
        b->grids.clear();
        b->forced.clear();
        for (int s = 0; s < nsys; ++s) add_system(b, &systems[s], grids + 3 * s);
    });
}

epwi_status epwi_batch_add(epwi_batch *b, const epwi_system *sys, const int32_t *grid,
                           int32_t *index) {
    return bguard(b, [&] {
        EPWI_REQUIRE(sys && grid, EPWI_EINVAL, "bad argument");
        add_system(b, sys, grid);
        if (index) *index = (int32_t)b->sys.size() - 1;
    });
}

epwi_status epwi_batch_plan(epwi_batch *b, double T, const double *mu, double smear,
                            const double *emin, const double *emax, int32_t autotune_tiles,
                            int64_t *n_pairs) {
    return bguard(b, [&] {
        EPWI_REQUIRE(!b->sys.empty(), EPWI_ESTATE, "epwi_batch_setup has not been called");
        EPWI_REQUIRE(T > 0 && smear > 0 && mu && emin && emax, EPWI_EINVAL, "bad argument");
        const int ns = (int)b->sys.size();
        b->T = T;
        b->eta = smear;
        b->mu.assign(mu, mu + ns);
        b->emin.assign(emin, emin + ns);
        b->emax.assign(emax, emax + ns);
        for (int s = 0; s < ns; ++s)
            EPWI_REQUIRE(std::isfinite(mu[s]) && !(emin[s] > emax[s]), EPWI_EINVAL,
                         "need finite mu and emin <= emax");
        plan(b, autotune_tiles != 0);
        if (n_pairs) *n_pairs = b->npairs;
    });
}

epwi_status epwi_batch_run(epwi_batch *b, double *sigma) {
    return bguard(b, [&] {
        EPWI_REQUIRE(b->planned && b->exec, EPWI_ESTATE, "epwi_batch_plan has not been called");
        cudaEvent_t e0, e1;
        EPWI_CUDA(cudaEventCreate(&e0));
        EPWI_CUDA(cudaEventCreate(&e1));
        cudaEventRecord(e0, b->stream);
        EPWI_CUDA(cudaGraphLaunch(b->exec, b->stream));
        cudaEventRecord(e1, b->stream);
        const int ns = (int)b->sys.size();
        if (sigma)
            EPWI_CUDA(cudaMemcpyAsync(sigma, b->d_sigma.p, sizeof(double) * 9 * ns,
                                      cudaMemcpyDeviceToHost, b->stream));
        EPWI_CUDA(cudaStreamSynchronize(b->stream));
        float ms = 0, msk = 0;
        EPWI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        EPWI_CUDA(cudaEventElapsedTime(&msk, b->ev[2], b->ev[3]));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->stats.ms_graph = ms;
        b->stats.ms_persistent = msk;
        b->stats.runs += 1;
    });
}

epwi_status epwi_batch_get_rates(epwi_batch *b, int32_t s, int64_t cap, int32_t *k_idx,
                                 int32_t *band, double *rates, int64_t *n) {
    return bguard(b, [&] {
        EPWI_REQUIRE(b->planned && b->stats.runs > 0, EPWI_ESTATE, "epwi_batch_run has not been called");
        EPWI_REQUIRE(s >= 0 && s < (int)b->sys.size(), EPWI_EINVAL, "no such system");
        epwi_ctx *c = b->sys[s];
        const int64_t ns = c->nstates;
        if (n) *n = ns;
        if (!k_idx && !band && !rates) return;
        EPWI_REQUIRE(cap >= ns, EPWI_ETOOSMALL, "capacity below n_states");
        if (ns) {
            if (k_idx) EPWI_CUDA(cudaMemcpyAsync(k_idx, c->st_k.p, 4 * ns, cudaMemcpyDeviceToHost, b->stream));
            if (band) EPWI_CUDA(cudaMemcpyAsync(band, c->st_n.p, 4 * ns, cudaMemcpyDeviceToHost, b->stream));
            if (rates)
                EPWI_CUDA(cudaMemcpyAsync(rates, b->d_inv_tau.as<double>() + b->sys_state0[s], 8 * ns,
                                          cudaMemcpyDeviceToHost, b->stream));
        }
        EPWI_CUDA(cudaStreamSynchronize(b->stream));
    });
}

epwi_status epwi_batch_get_tile(epwi_batch *b, int32_t s, int32_t *mt, int32_t *kc,
                                int32_t *source) {
    return bguard(b, [&] {
        EPWI_REQUIRE(b->planned, EPWI_ESTATE, "epwi_batch_plan has not been called");
        EPWI_REQUIRE(s >= 0 && s < (int)b->sys.size(), EPWI_EINVAL, "no such system");
        if (mt) *mt = b->hsys[s].Mt;
        if (kc) *kc = b->hsys[s].KC;
        if (source) *source = b->tile_src[s];
    });
}

epwi_status epwi_batch_set_tile(epwi_batch *b, int32_t s, int32_t mt, int32_t kc) {
    return bguard(b, [&] {
        EPWI_REQUIRE(s >= 0 && s < (int)b->sys.size(), EPWI_EINVAL, "no such system");
        epwi_ctx *c = b->sys[s];
        EPWI_REQUIRE(mt == 0 || tile_ok(mt, kc, c->nw * c->nm), EPWI_EINVAL,
                     "tile shape does not fit this system");
        b->forced.resize(b->sys.size(), {0, 0});
        b->forced[s] = {mt, kc};
    });
}

epwi_status epwi_batch_band_range(epwi_batch *b, int32_t s, double *emin, double *emax) {
    return bguard(b, [&] {
        EPWI_REQUIRE(s >= 0 && s < (int)b->sys.size(), EPWI_EINVAL, "no such system");
        epwi_ctx *c = b->sys[s];
        const int g3[3] = {b->grids[s][0], b->grids[s][1], b->grids[s][2]};
        check(c, epwi_eigs(c, g3, g3), "epwi_eigs");
        check(c, epwi_band_range(c, emin, emax), "epwi_band_range");
    });
}

epwi_status epwi_batch_get_stats(epwi_batch *b, epwi_batch_stats *out) {
    return bguard(b, [&] {
        EPWI_REQUIRE(out, EPWI_EINVAL, "out is NULL");
        *out = b->stats;
    });
}

}  // extern "C"
