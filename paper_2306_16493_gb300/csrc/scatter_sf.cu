// Sum-factorised Rp->q stage in FP32 (precision EPWI_FP32), fused with the rotations and the
// delta sum of Eq. 10.
//
// Any R_p set is embedded in its bounding cube [-r, r]^3 (vectors outside the set carry zero
// weight), so the phase of Eq. 16 factorises per axis: e^{iq.Rp} = e1(q1,R1) e2(q2,R2)
// e3(q3,R3), e_a(x, R) = e^{i theta R}, theta = 2 pi x / N_a.  Along each axis the values at
// +R and -R are recombined once, at setup, into
//     v'[0] = v[0],  v'[2R-1] = v[R] + v[-R],  v'[2R] = i (v[R] - v[-R])      (R = 1..r)
// so that sum_R e^{i theta R} v[R] = v'[0] + sum_R (cos(theta R) v'[2R-1] + sin(theta R) v'[2R]):
// every stage below is a contraction with REAL coefficients (2 FMAs per complex term instead
// of 4).  The recombination acts on the R_p index only, so it commutes with the Re->k sum and
// the U^dag(k) rotation and is applied to g(Re, Rp) itself (k_sf_transform).
//
// The sieve lists the pairs of a k-point in plane blocks pb of 256 consecutive (q2, q3)
// combinations, then by q1, then by combination.  For the state (k, n) of one CTA:
//   Y[f1][f3][j]  = sum_f2 c2(q2_j)[f2] ghat'[f1][f2][f3]    per plane block and group of q2 values j
//   U[f3][j]      = sum_f1 c1(q1)[f1]  Y[f1][f3][j]           per run (plane block, q1, q2 group)
//   G             = sum_f3 c3(q3)[f3]  U[f3][j(q)]            per pair
// with ghat' = (g' P^el) U^dag(k) from the FP32 Re->k stage, every column (mu, i) at once.
// U is built for a batch of runs by the whole CTA; then every thread takes pairs of the batch
// from one flat list.  Per pair, each lane loops over the final bands m that have a mode within
// c eta of either energy shell (others add exactly zero), and for each band streams the modes
// mu: h = sum_i conj(V_im(k+q)) G[mu][i], g_nu += h u_mu,nu(q); then |g|^2 and the two delta
// terms, in FP32.  With a Gamma capture (iterative BTE) the CTA also writes its band's row of
// every pair's Gamma block (rows of bands out of range stay at the zero the buffer was cleared
// to).  Lane sums are FP32 within a batch, FP64 across batches, and the CTA adds its threads
// in a fixed order, so the result is deterministic and independent of k-point chunking.
#include <algorithm>

#include "epwi_internal.cuh"
#include "scatter.cuh"
#include "sieve.cuh"

namespace {

constexpr int kSfThreads = 256;
constexpr int kSfWarps = kSfThreads / 32;

// Re->k in FP32: ghat32[state][row] = sum_j [sum_Re w e^{ik.Re} g(Re)[row][j]] V_{j, lo+n}(k),
// row = (cube form, mu, i); one thread per row, KG k-points per block row.
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

// The same Re->k stage with one thread per (row, j) and 32 k-points per thread: the phases of
// the block's 32 k-points are staged in shared memory in chunks of 32 R_e and read as
// broadcasts, g'[Re][row][j] is read once per 32 k-points (coalesced over (row, j)), and the
// contraction with V_{j,n}(k) is a shuffle reduction over the W lanes of a row.  Sums over R_e
// run in R_e order; the sum over j is a fixed tree.
template <int W>
__global__ void __launch_bounds__(256) k_restage_f32_kb(RestageArgs a, float2 *__restrict__ out) {
    constexpr int KB = 32, RCH = 32, RPB = 256 / W;   // k-points per block, R_e per chunk, rows per block
    __shared__ float2 Ps[RCH][KB];
    const int tid = threadIdx.x, j = tid % W;
    const int row = blockIdx.x * RPB + tid / W;
    const int k0 = blockIdx.y * KB;
    const bool live = row < a.nrow;
    float2 acc[KB];
#pragma unroll
    for (int x = 0; x < KB; ++x) acc[x] = make_float2(0.f, 0.f);
    for (int re0 = 0; re0 < a.nRe; re0 += RCH) {
        __syncthreads();                          // Ps of the previous chunk is consumed
        for (int e = tid; e < RCH * KB; e += 256) {
            const int rr = e / KB, kk = e % KB, re = re0 + rr;
            float2 p = make_float2(0.f, 0.f);
            if (k0 + kk < a.nkp && re < a.nRe) {
                int i1, i2, i3;
                grid_coords(a.g, a.kpts[k0 + kk], i1, i2, i3);
                p = a.ph32[phase_index(i1 * a.g.s1 % a.g.L, i2 * a.g.s2 % a.g.L, i3 * a.g.s3 % a.g.L,
                                       a.Re[3 * re], a.Re[3 * re + 1], a.Re[3 * re + 2], a.g.L)];
            }
            Ps[rr][kk] = p;
        }
        __syncthreads();
        const int nr = min(RCH, a.nRe - re0);
        if (live) {
            for (int rr = 0; rr < nr; ++rr) {
                const float2 gv = __ldg(a.gw32 + ((size_t)(re0 + rr) * a.nrow + row) * W + j);
#pragma unroll
                for (int x = 0; x < KB; x += 2) {
                    const float4 p2 = reinterpret_cast<const float4 *>(&Ps[rr][x])[0];
                    acc[x] = cfmaf(make_float2(p2.x, p2.y), gv, acc[x]);
                    acc[x + 1] = cfmaf(make_float2(p2.z, p2.w), gv, acc[x + 1]);
                }
            }
        }
    }
    // out[state][row] = sum_j acc[k][j] V_{j, lo+n}(k): lanes j of a row are adjacent
#pragma unroll
    for (int x = 0; x < KB; ++x) {
        const int kp = k0 + x;
        if (kp >= a.nkp) continue;               // uniform over the block
        const int ik = a.kpts[kp];
        const int lo = a.win_lo[ik], ns = a.win_n[ik];
        const int64_t s0 = a.kp_state[kp] - a.s_base;
        const float2 *Vk = a.V32 + (int64_t)ik * W * W;
        for (int np = 0; np < ns; ++np) {
            float2 o = cmulf(acc[x], Vk[j * W + lo + np]);
#pragma unroll
            for (int off = W / 2; off > 0; off >>= 1) {
                o.x += __shfl_xor_sync(0xffffffffu, o.x, off);
                o.y += __shfl_xor_sync(0xffffffffu, o.y, off);
            }
            if (live && j == 0) out[(s0 + np) * a.nrow + row] = o;
        }
    }
}

// g'(Re, f1 f2 f3) = (T x T x T) g(Re, cube): along each axis, form 0 is R = 0, form 2R-1 is
// v[R] + v[-R] and form 2R is i (v[R] - v[-R]).  cube[c] is the index of the R_p vector at
// cube point c, or -1 (zero weight).  One thread per output element; FP64 sums, FP32 output.
__global__ void k_sf_transform(int64_t n, int nRp, int Dc, int rc, int rowlen, const int *__restrict__ cube,
                               const double2 *__restrict__ g64, const float2 *__restrict__ g32,
                               float2 *__restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int e = (int)(idx % rowlen);              // (mu, i, j) within the (Re, form) block
    const int64_t t = idx / rowlen;
    const int D3 = Dc * Dc * Dc;
    const int cf = (int)(t % D3);
    const int64_t re = t / D3;
    const int f[3] = {cf / (Dc * Dc), (cf / Dc) % Dc, cf % Dc};
    int Rv[3][2], nt[3];
    double2 cv[3][2];
    for (int a = 0; a < 3; ++a) {
        if (f[a] == 0) {
            nt[a] = 1;
            Rv[a][0] = 0;
            cv[a][0] = make_double2(1, 0);
        } else {
            const int R = (f[a] + 1) / 2;
            nt[a] = 2;
            Rv[a][0] = R;
            Rv[a][1] = -R;
            if (f[a] & 1) {
                cv[a][0] = make_double2(1, 0);
                cv[a][1] = make_double2(1, 0);
            } else {
                cv[a][0] = make_double2(0, 1);
                cv[a][1] = make_double2(0, -1);
            }
        }
    }
    double2 s = make_double2(0, 0);
    for (int x = 0; x < nt[0]; ++x)
        for (int y = 0; y < nt[1]; ++y)
            for (int z = 0; z < nt[2]; ++z) {
                const int c = ((Rv[0][x] + rc) * Dc + (Rv[1][y] + rc)) * Dc + (Rv[2][z] + rc);
                const int rp = cube[c];
                if (rp < 0) continue;
                const size_t gi = ((size_t)re * nRp + rp) * rowlen + e;
                const double2 v = g64 ? g64[gi] : make_double2(g32[gi].x, g32[gi].y);
                s = cadd(s, cmul(cmul(cmul(cv[0][x], cv[1][y]), cv[2][z]), v));
            }
    out[idx] = make_float2((float)s.x, (float)s.y);
}

// Band-major tables of the k+q side (FP32): Vb[m][k][i] = V[k][i][m] and
// EF[m][k] = (eps_mk - mu, f_mk), so that lanes on consecutive k+q points and one band m read
// contiguous memory.
__global__ void k_band_major_v(int64_t nk, int W, const float2 *__restrict__ V, float2 *__restrict__ Vb) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nk * W * W) return;
    const int i = (int)(idx % W);
    const int64_t t = idx / W;
    const int64_t k = t % nk;
    const int m = (int)(t / nk);
    Vb[idx] = V[k * W * W + i * W + m];
}

// Structure-of-arrays tables of the q side (FP32): uS[mu nu][q] = u_mu,nu(q) and
// wn[nu][q] = (hbar omega, N), so that lanes on consecutive q read contiguous memory.
__global__ void k_soa_q(int64_t nq, int NM, const float2 *__restrict__ u, const float *__restrict__ hw,
                        const float *__restrict__ n, float2 *__restrict__ uS, float2 *__restrict__ wn) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nq * NM * NM) return;
    const int64_t q = idx % nq;
    const int e = (int)(idx / nq);
    uS[idx] = u[q * NM * NM + e];
    if (e < NM) wn[idx] = make_float2(hw[q * NM + e], n[q * NM + e]);
}

__global__ void k_band_major_ef(int64_t nk, int W, const float *__restrict__ erel, const float *__restrict__ f32,
                                float2 *__restrict__ ef) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nk * W) return;
    const int64_t k = idx % nk;
    const int m = (int)(idx / nk);
    ef[idx] = make_float2(erel[k * W + m], f32[k * W + m]);
}

// Division by a divisor fixed at launch (x < 2^31): q = (umulhi(x, m) + x) >> l with
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1 (Granlund & Montgomery, PLDI 1994).
struct FDiv {
    uint32_t d, m, l;
};
FDiv make_fdiv(uint32_t d) {
    FDiv f;
    f.d = d;
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    f.l = l;
    f.m = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
    return f;
}
__device__ __forceinline__ int fdiv(int x, const FDiv &f) {
    return (int)((__umulhi((uint32_t)x, f.m) + (uint32_t)x) >> f.l);
}

struct SfArgs {
    GridInfo g;
    int nplane;                     // N2 N3
    FDiv fplane, fjq;               // division by N2 N3 and by jq
    int jq;                         // q2 values per group (Y and the U buffers hold one group)
    int njg;                        // groups per plane block (over the largest block)
    int pbmax;                      // plane blocks
    const float2 *ph32;             // e^{2 pi i m / L}
    const float2 *ghat;             // [state - s_base][D^3 forms][N_m][W]
    const int *kpts, *win_lo, *win_n;
    const int64_t *kp_state;        // chunk k-points' first states (global)
    int64_t s_base;
    const int64_t *kp_pairs;        // chunk-local pair offsets, minus p_off
    int64_t p_off;
    const int *pairs;               // chunk pair list: q index
    const float2 *Vb32, *u32;       // Vb32[m][k][i]: band-major columns of V
    const float2 *ef;               // [m][k]: (eps - mu, f), band-major
    const float2 *uS;               // [mu nu][q]: u(q), structure of arrays
    const float2 *wn;               // [nu][q]: (hbar omega, N), structure of arrays
    int64_t nk;
    const float *erel, *f32, *n32, *hw32, *hwmax32;
    float ceta32, inv_eta32;
    double pref;                    // 2 pi / (hbar N_q sqrt(pi) eta)
    double *inv_tau;
    const int2 *items;              // {chunk kp, band}
    float *gam;                     // Gamma capture (iterative BTE) or nullptr: row n of each
    const int64_t *goff;            // pair's block, block start goff[chunk pair]
};

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

// Shared-memory layout of k_scatter_sf (float2 units first, then floats, then ints).
struct SfSmem {
    size_t y, u, cs, ints, bytes;
};
__host__ __device__ inline SfSmem sf_smem_layout(int D, int X, int jq, int N1, int N2, int N3, int njg, int pbmax) {
    SfSmem s;
    s.y = (size_t)D * D * jq * X;                          // float2: Y of one q2 group
    s.u = (size_t)kSfWarps * D * jq * X;                   // float2: U of one run per warp
    s.cs = (size_t)(N1 + N2 + N3) * (D - 1);               // float: (cos, sin) per R >= 1
    s.ints = (size_t)kSieveBlock + 2 * (size_t)N1 * njg + (size_t)N1 + (size_t)pbmax + 1 + 4;
    s.bytes = sizeof(float2) * (s.y + s.u) + sizeof(float) * s.cs + sizeof(int) * s.ints;
    return s;
}

template <int W, int NM, int RC, bool GAM>
__global__ void __launch_bounds__(kSfThreads, (W <= 4 ? 3 : 2)) k_scatter_sf(SfArgs a) {
    constexpr int D = 2 * RC + 1;
    constexpr int NF = D - 1;                    // forms with a cos / sin coefficient
    constexpr int X = NM * W;                    // columns (mu, i)
    constexpr bool V2 = (W % 2) == 0;            // rows of W float2 are 16-byte aligned
    constexpr int kMuUnroll = NM <= 3 ? NM : 1;  // wide systems: one mode row at a time (registers)
    constexpr bool kPreG = X <= 12 && X % 2 == 0;  // G of a pair kept in registers for its bands
    extern __shared__ __align__(16) float2 sm[];
    const int N1 = a.g.n1, N2 = a.g.n2, N3 = a.g.n3, L = a.g.L;
    const int JQ = a.jq, NJG = a.njg;
    const SfSmem lay = sf_smem_layout(D, X, JQ, N1, N2, N3, NJG, a.pbmax);
    float2 *Y = sm;                              // [D f1][D f3][JQ][X]
    float *CS = reinterpret_cast<float *>(Y + lay.y + lay.u);   // [N1 + N2 + N3][NF]: cos, sin of theta R
    int *cq = reinterpret_cast<int *>(CS + lay.cs);     // [256]: (j << 16) | q3 of combination t
    int *ss = cq + kSieveBlock;                  // [N1 NJG]: segment start (relative), -1 if none
    int *se = ss + N1 * NJG;                     // [N1 NJG]: segment end
    int *gl = se + N1 * NJG;                     // [N1]: runs (q1) of the current group
    int *pbs = gl + N1;                          // [pbmax + 1]: first pair of each plane block
    int *nglist = pbs + a.pbmax + 1;             // [1]
    __shared__ double wsum[kSfWarps];
    const int2 item = a.items[blockIdx.x];
    const int kp = item.x, n = item.y;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float2 *Uw = Y + lay.y + (size_t)wid * D * JQ * X;   // this warp's run: [D f3][JQ][X]
    const int ik = a.kpts[kp];
    const int lo = a.win_lo[ik];
    const int64_t s = a.kp_state[kp] + n;        // global state
    const float2 *gs = a.ghat + (size_t)(s - a.s_base) * D * D * D * X;
    // cos / sin tables of the three axes (exact integer reduction of x R onto the L roots)
    for (int e = tid; e < (N1 + N2 + N3) * RC; e += kSfThreads) {
        const int R = e % RC + 1, x = e / RC;
        int xx, st;
        if (x < N1) { xx = x; st = a.g.s1; }
        else if (x < N1 + N2) { xx = x - N1; st = a.g.s2; }
        else { xx = x - N1 - N2; st = a.g.s3; }
        const int t = (int)(((int64_t)xx * st % L) * R % L);
        const float2 v = a.ph32[t];
        CS[x * NF + 2 * (R - 1)] = v.x;
        CS[x * NF + 2 * (R - 1) + 1] = v.y;
    }
    const float *CS1 = CS, *CS2 = CS + N1 * NF, *CS3 = CS + (N1 + N2) * NF;
    const int nplane = a.nplane;
    const int pb_n = (nplane + kSieveBlock - 1) / kSieveBlock;
    const int64_t P0 = a.kp_pairs[kp] - a.p_off, P1 = a.kp_pairs[kp + 1] - a.p_off;
    const int *pl = a.pairs + P0;                // this k-point's pairs, relative index
    const int np = (int)(P1 - P0);
    // first pair of every plane block (the list is ordered by plane block)
    for (int pb = tid; pb <= pb_n; pb += kSfThreads)
        pbs[pb] = (int)lower_bound(0, np, pb, [&](int64_t p) {
            const int q = pl[p];
            return (int64_t)((q - fdiv(q, a.fplane) * nplane) / kSieveBlock);
        });
    int k1, k2, k3;
    grid_coords(a.g, ik, k1, k2, k3);
    const float en = a.erel[(int64_t)ik * W + lo + n];
    const float ceta = a.ceta32, ieta = a.inv_eta32;
    double acc = 0;                              // this warp's run sums (lane 0)
    __syncthreads();
    for (int pb = 0; pb < pb_n; ++pb) {
        const int seg0 = pbs[pb], nseg = pbs[pb + 1] - seg0;   // the plane block's pairs
        if (nseg == 0) continue;
        const int *pp = pl + seg0;
        const int c_lo = pb * kSieveBlock, c_hi = min(nplane, c_lo + kSieveBlock) - 1;
        const int q2lo = c_lo / N3, nq2 = c_hi / N3 - q2lo + 1;
        const int njg = (nq2 + JQ - 1) / JQ;
        for (int t = tid; t < kSieveBlock; t += kSfThreads) {
            const int c = c_lo + t, q2 = c / N3;
            cq[t] = ((q2 - q2lo) << 16) | (c - q2 * N3);
        }
        for (int t = tid; t < N1 * NJG; t += kSfThreads) ss[t] = -1;
        __syncthreads();
        // segments: the block's pairs are ordered by q1, then by combination (so by q2 group);
        // key = q1 NJG + group, neighbours' keys by shuffle
        auto keyof = [&](int t) -> int {
            const int q = pp[t];
            const int q1 = fdiv(q, a.fplane);
            const int j = cq[q - q1 * nplane - c_lo] >> 16;
            return q1 * NJG + fdiv(j, a.fjq);
        };
        for (int t0 = wid * 32; t0 < nseg; t0 += kSfThreads) {
            const int t = t0 + lane;
            const bool on = t < nseg;
            const int key = on ? keyof(t) : -1;
            int kprev = __shfl_up_sync(0xffffffffu, key, 1);
            int knext = __shfl_down_sync(0xffffffffu, key, 1);
            if (lane == 0 && t > 0 && on) kprev = keyof(t - 1);
            if (lane == 31 && t + 1 < nseg) knext = keyof(t + 1);
            if (on) {
                if (t == 0 || kprev != key) ss[key] = t;
                if (t == nseg - 1 || knext != key) se[key] = t + 1;
            }
        }
        __syncthreads();
        for (int jg = 0; jg < njg; ++jg) {
            const int j0 = jg * JQ, jn = min(JQ, nq2 - j0);
            // the group's non-empty runs, in q1 order (warp 0)
            if (wid == 0) {
                int cnt = 0;
                for (int q0 = 0; q0 < N1; q0 += 32) {
                    const int q1 = q0 + lane;
                    const bool on = q1 < N1 && ss[q1 * NJG + jg] >= 0;
                    const unsigned b = __ballot_sync(0xffffffffu, on);
                    if (on) gl[cnt + __popc(b & ((1u << lane) - 1u))] = q1;
                    cnt += __popc(b);
                }
                if (lane == 0) *nglist = cnt;
            }
            // Y of this group's q2 values (all threads), read from ghat' (L1 / L2)
            {
                const int per = jn * X;                 // (jj, col) of one (f1, f3)
                for (int e = tid; e < D * D * per; e += kSfThreads) {
                    const int r13 = e / per, e2 = e - r13 * per;
                    const int jj = e2 / X, col = e2 - jj * X;
                    const int f3 = r13 % D, f1 = r13 / D;
                    const float *c2 = CS2 + (q2lo + j0 + jj) * NF;
                    const float2 *src = gs + ((f1 * D) * D + f3) * X + col;
                    float2 v = __ldg(src);                   // form f2 = 0
#pragma unroll
                    for (int f2 = 1; f2 < D; ++f2) {
                        const float c = c2[f2 - 1];
                        const float2 w = __ldg(src + f2 * D * X);
                        v.x = fmaf(c, w.x, v.x);
                        v.y = fmaf(c, w.y, v.y);
                    }
                    Y[(r13 * JQ + jj) * X + col] = v;
                }
            }
            __syncthreads();
            const int ng = *nglist;
            // runs round-robin over the warps (a fixed assignment keeps the sums deterministic)
            for (int r = wid; r < ng; r += kSfWarps) {
                const int q1 = gl[r];
                const int t0 = ss[q1 * NJG + jg], t1 = se[q1 * NJG + jg];
                // U of the run: for each form f3, the contiguous (jj, col) row of Y
                {
                    float c1[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) c1[f] = CS1[q1 * NF + f];
                    if constexpr (X % 2 == 0) {
                        // (f3, e2) over D rows of per4 float4, walked as one list by the lanes
                        const int per4 = jn * X / 2;
                        int f3 = 0, e2 = lane;
                        while (true) {
                            while (e2 >= per4 && f3 < D) {
                                e2 -= per4;
                                ++f3;
                            }
                            if (f3 >= D) break;
                            const float4 *src = reinterpret_cast<const float4 *>(Y + (size_t)f3 * JQ * X) + e2;
                            float4 v = src[0];
#pragma unroll
                            for (int f1 = 1; f1 < D; ++f1) {
                                const float c = c1[f1 - 1];
                                const float4 w = src[f1 * D * JQ * X / 2];
                                v.x = fmaf(c, w.x, v.x);
                                v.y = fmaf(c, w.y, v.y);
                                v.z = fmaf(c, w.z, v.z);
                                v.w = fmaf(c, w.w, v.w);
                            }
                            reinterpret_cast<float4 *>(Uw + (size_t)f3 * JQ * X)[e2] = v;
                            e2 += 32;
                        }
                    } else {
                        const int per = jn * X;
#pragma unroll
                        for (int f3 = 0; f3 < D; ++f3) {
                            const float2 *src = Y + (size_t)f3 * JQ * X;
                            float2 *dst = Uw + (size_t)f3 * JQ * X;
                            for (int e = lane; e < per; e += 32) {
                                float2 v = src[e];
#pragma unroll
                                for (int f1 = 1; f1 < D; ++f1) {
                                    const float c = c1[f1 - 1];
                                    const float2 w = src[e + f1 * D * JQ * X];
                                    v.x = fmaf(c, w.x, v.x);
                                    v.y = fmaf(c, w.y, v.y);
                                }
                                dst[e] = v;
                            }
                        }
                    }
                }
                __syncwarp();
                float rate = 0.f;
                int b1 = k1 + q1;
                if (b1 >= N1) b1 -= N1;
                const int qbase = q1 * nplane + c_lo;
                for (int t = t0 + lane; t < t1; t += 32) {
                    const int q = pp[t];
                    const int jq = cq[q - qbase];
                    const int j = jq >> 16, q3 = jq & 0xffff;
                    int b2 = k2 + q2lo + j, b3 = k3 + q3;
                    if (b2 >= N2) b2 -= N2;
                    if (b3 >= N3) b3 -= N3;
                    const int ikq = (b1 * N2 + b2) * N3 + b3;   // nk W^2 < 2^31 (checked on the host)
                    // final bands within the largest kept mode energy + c eta of e_nk (a superset
                    // of the bands with a mode inside c eta of either shell; the others add zero)
                    const float lim = __ldg(a.hwmax32 + q) + ceta + 1e-5f;
                    float emr[W];
                    if constexpr (W % 4 == 0) {
#pragma unroll
                        for (int m4 = 0; m4 < W / 4; ++m4) {
                            const float4 e4 = __ldg(reinterpret_cast<const float4 *>(a.erel + ikq * W) + m4);
                            emr[4 * m4] = e4.x; emr[4 * m4 + 1] = e4.y; emr[4 * m4 + 2] = e4.z; emr[4 * m4 + 3] = e4.w;
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < W; ++m) emr[m] = __ldg(a.erel + ikq * W + m);
                    }
                    unsigned mask = 0;
#pragma unroll
                    for (int m = 0; m < W; ++m) mask |= (fabsf(en - emr[m]) <= lim ? 1u : 0u) << m;
                    if (!mask) continue;
                    const float2 *Ub = Uw + (j - j0) * X;      // form f3 at + f3 JQ X
                    float c3[NF], wq[NM], nq[NM];
#pragma unroll
                    for (int f = 0; f < NF; ++f) c3[f] = CS3[q3 * NF + f];
#pragma unroll
                    for (int nu = 0; nu < NM; ++nu) {
                        const float2 v = __ldg(a.wn + (int64_t)nu * a.nk + q);
                        wq[nu] = v.x;
                        nq[nu] = v.y;
                    }
                    int lokq = 0, nwkq = 0;
                    int64_t grow = 0;                        // this band's row of the pair's Gamma block
                    if constexpr (GAM) {
                        lokq = __ldg(a.win_lo + ikq);
                        nwkq = __ldg(a.win_n + ikq);
                        grow = a.goff[P0 + seg0 + t] + (int64_t)n * nwkq - lokq;
                    }
                    const float2 *uq = a.uS + q;                     // element e at uq[e * nk]
                    // small shapes: G (every column) once per pair, shared by its bands
                    float2 Gp[kPreG ? X : 1];
                    if constexpr (kPreG) {
#pragma unroll
                        for (int x = 0; x < X; ++x) Gp[x] = Ub[x];
#pragma unroll
                        for (int f = 1; f < D; ++f) {
                            const float c = c3[f - 1];
#pragma unroll
                            for (int x2 = 0; x2 < X / 2; ++x2) {
                                const float4 v = reinterpret_cast<const float4 *>(Ub + f * JQ * X)[x2];
                                Gp[2 * x2].x = fmaf(c, v.x, Gp[2 * x2].x);
                                Gp[2 * x2].y = fmaf(c, v.y, Gp[2 * x2].y);
                                Gp[2 * x2 + 1].x = fmaf(c, v.z, Gp[2 * x2 + 1].x);
                                Gp[2 * x2 + 1].y = fmaf(c, v.w, Gp[2 * x2 + 1].y);
                            }
                        }
                    }
                    while (mask) {
                        const int m = __ffs(mask) - 1;
                        mask &= mask - 1;
                        const float2 emf = __ldg(a.ef + (int64_t)m * a.nk + ikq);
                        const float em = emf.x, fm = emf.y;
                        float2 Vc[W];                        // column m of V(k+q)
                        const float2 *vp = a.Vb32 + ((int64_t)m * a.nk + ikq) * W;
                        if constexpr (V2) {
#pragma unroll
                            for (int i = 0; i < W / 2; ++i) {
                                const float4 v = __ldg(reinterpret_cast<const float4 *>(vp) + i);
                                Vc[2 * i] = make_float2(v.x, v.y);
                                Vc[2 * i + 1] = make_float2(v.z, v.w);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < W; ++i) Vc[i] = __ldg(vp + i);
                        }
                        float2 gv[NM];
#pragma unroll
                        for (int nu = 0; nu < NM; ++nu) gv[nu] = make_float2(0.f, 0.f);
#pragma unroll kMuUnroll
                        for (int mu = 0; mu < NM; ++mu) {
                            float2 G[W];
                            const float2 *u0 = Ub + mu * W;
                            if constexpr (kPreG) {
#pragma unroll
                                for (int i = 0; i < W; ++i) G[i] = Gp[mu * W + i];
                            } else if constexpr (V2) {
#pragma unroll
                                for (int i = 0; i < W / 2; ++i) {
                                    const float4 v = reinterpret_cast<const float4 *>(u0)[i];
                                    G[2 * i] = make_float2(v.x, v.y);
                                    G[2 * i + 1] = make_float2(v.z, v.w);
                                }
#pragma unroll
                                for (int f = 1; f < D; ++f) {
                                    const float c = c3[f - 1];
                                    const float4 *uf = reinterpret_cast<const float4 *>(u0 + f * JQ * X);
#pragma unroll
                                    for (int i = 0; i < W / 2; ++i) {
                                        const float4 v = uf[i];
                                        G[2 * i].x = fmaf(c, v.x, G[2 * i].x);
                                        G[2 * i].y = fmaf(c, v.y, G[2 * i].y);
                                        G[2 * i + 1].x = fmaf(c, v.z, G[2 * i + 1].x);
                                        G[2 * i + 1].y = fmaf(c, v.w, G[2 * i + 1].y);
                                    }
                                }
                            } else {
#pragma unroll
                                for (int i = 0; i < W; ++i) G[i] = u0[i];
#pragma unroll
                                for (int f = 1; f < D; ++f) {
                                    const float c = c3[f - 1];
#pragma unroll
                                    for (int i = 0; i < W; ++i) {
                                        const float2 v = u0[f * JQ * X + i];
                                        G[i].x = fmaf(c, v.x, G[i].x);
                                        G[i].y = fmaf(c, v.y, G[i].y);
                                    }
                                }
                            }
                            float2 h = make_float2(0.f, 0.f);
#pragma unroll
                            for (int i = 0; i < W; ++i) h = cfmacf(Vc[i], G[i], h);
#pragma unroll
                            for (int nu = 0; nu < NM; ++nu)
                                gv[nu] = cfmaf(h, __ldg(uq + (int64_t)(mu * NM + nu) * a.nk), gv[nu]);
                        }
                        float gm = 0.f;                      // Gamma capture: sum over modes
#pragma unroll
                        for (int nu = 0; nu < NM; ++nu) {
                            const float w = wq[nu];
                            if (w < 0.f) continue;
                            const float g2 = gv[nu].x * gv[nu].x + gv[nu].y * gv[nu].y;
                            const float x1 = (en + w) - em;
                            const float x2 = (en - w) - em;
                            float tt = 0.f;
                            if (fabsf(x1) <= ceta) {
                                const float y = x1 * ieta;
                                tt += (nq[nu] + fm) * __expf(-y * y);
                            }
                            if (fabsf(x2) <= ceta) {
                                const float y = x2 * ieta;
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
                acc += (double)rate;                         // runs of this warp in a fixed order
                __syncwarp();                                // Uw is rewritten by the next run
            }
            __syncthreads();                                 // gl, nglist and Y are rewritten next
        }
    }
    if (lane == 0) wsum[wid] = acc;
    __syncthreads();
    if (tid == 0) {
        double t = 0;
        for (int w = 0; w < kSfWarps; ++w) t += wsum[w];
        a.inv_tau[s] = a.pref * t;
    }
}

struct SfPlan {
    int jq, njg, pbmax;
    size_t smem;
};

// q2 values per group (jq): Y of one group and one run's U per warp within budgets that keep
// two or more CTAs per SM.
SfPlan sf_plan(int D, int X, int q2max, int N1, int N2, int N3) {
    const size_t ybudget = 40 * 1024, ubudget = 36 * 1024;
    SfPlan p;
    const size_t per_j = sizeof(float2) * D * X;
    const int jmax = std::max(1, std::min({q2max, (int)(ybudget / (per_j * D)), (int)(ubudget / (per_j * kSfWarps))}));
    p.njg = (q2max + jmax - 1) / jmax;             // groups of equal size
    p.jq = (q2max + p.njg - 1) / p.njg;
    p.pbmax = (N2 * N3 + kSieveBlock - 1) / kSieveBlock;
    p.smem = sf_smem_layout(D, X, p.jq, N1, N2, N3, p.njg, p.pbmax).bytes;
    return p;
}

template <int W, int NM, int RC, bool GAM>
void launch_sf_t(epwi_ctx *c, const SfArgs &a, int nitems, size_t sm) {
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
void launch_sf(epwi_ctx *c, const SfArgs &a, int nitems, size_t sm) {
    if (a.gam) launch_sf_t<W, NM, RC, true>(c, a, nitems, sm);
    else launch_sf_t<W, NM, RC, false>(c, a, nitems, sm);
}

bool sf_shape_built(int W, int NM, int r) {
    return (W == 4 && NM == 3 && r >= 1 && r <= 3) || (W == 1 && NM == 3 && r >= 1 && r <= 2) ||
           (W == 8 && NM == 6 && r >= 1 && r <= 3);
}

}  // namespace

size_t sf_state_bytes(const epwi_ctx *c) {
    const size_t Dc = 2 * (size_t)c->sf_r + 1;
    return sizeof(float2) * Dc * Dc * Dc * c->nm * c->nw;
}

void sf_check(const epwi_ctx *c) {
    const int W = c->nw, NM = c->nm, r = c->sf_r;
    EPWI_REQUIRE(c->nk * std::max(W * W, NM * NM) < (int64_t(1) << 31), EPWI_EUNSUPPORTED,
                 "fp32 mode: grid too large for its 32-bit table offsets");
    EPWI_REQUIRE(sf_shape_built(W, NM, r), EPWI_EUNSUPPORTED,
                 "fp32 mode built for (nw, modes) in {(4,3), (8,6)} with R_p within |n| <= 3, and (1,3) "
                 "within |n| <= 2");
    EPWI_REQUIRE(c->ng[0] * 2 <= 4096 && c->ng[2] <= 0xffff, EPWI_EUNSUPPORTED, "fp32 mode: grid too large");
}

// Builds what the fp32 mode reads besides the eigen-tables: g' (cube embedding and the +-R
// recombination of the R_p axes, once per system) and the band-major FP32 V and (eps - mu, f)
// tables (per rates call).
void sf_prepare(epwi_ctx *c) {
    const int W = c->nw, NM = c->nm;
    const int Dc = 2 * c->sf_r + 1;
    if (!c->sf_g_ready) {
        const int rowlen = NM * W * W;
        const int64_t n = (int64_t)c->nRe * Dc * Dc * Dc * rowlen;
        DevBuf cube;
        upload_ints(c, cube, c->h_rp_cube);
        c->gsf32.ensure(sizeof(float2) * n);
        k_sf_transform<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
            n, c->nRp, Dc, c->sf_r, rowlen, cube.as<int>(), c->keep_g64 ? c->gw64.as<double2>() : nullptr,
            c->gw32.as<float2>(), c->gsf32.as<float2>());
        EPWI_CHECK_LAUNCH();
        EPWI_CUDA(cudaStreamSynchronize(c->stream));   // cube is freed on return
        c->sf_g_ready = true;
    }
    const int64_t nv = c->nk * W * W, ne = c->nk * W;
    c->sf_Vt32.ensure(sizeof(float2) * nv);
    k_band_major_v<<<(unsigned)((nv + 255) / 256), 256, 0, c->stream>>>(c->nk, W, c->V32.as<float2>(),
                                                                       c->sf_Vt32.as<float2>());
    EPWI_CHECK_LAUNCH();
    c->sf_ef.ensure(sizeof(float2) * ne);
    k_band_major_ef<<<(unsigned)((ne + 255) / 256), 256, 0, c->stream>>>(c->nk, W, c->tc_erel.as<float>(),
                                                                        c->tc_f32.as<float>(), c->sf_ef.as<float2>());
    EPWI_CHECK_LAUNCH();
    const int64_t nu = c->nk * NM * NM;
    c->sf_uS.ensure(sizeof(float2) * nu);
    c->sf_wn.ensure(sizeof(float2) * c->nk * NM);
    k_soa_q<<<(unsigned)((nu + 255) / 256), 256, 0, c->stream>>>(c->nk, NM, c->u32.as<float2>(), c->tc_hw32.as<float>(),
                                                                c->tc_n32.as<float>(), c->sf_uS.as<float2>(),
                                                                c->sf_wn.as<float2>());
    EPWI_CHECK_LAUNCH();
}

void sf_restage(epwi_ctx *c, const RestageArgs &ra_in) {
    RestageArgs ra = ra_in;
    const int Dc = 2 * c->sf_r + 1;
    ra.gw32 = c->gsf32.as<float2>();
    ra.nrow = Dc * Dc * Dc * c->nm * c->nw;
    const int W = ra.W;
    float2 *out = static_cast<float2 *>(ra.ghat_raw);
    auto go = [&](auto kern, int KG) {
        dim3 grid((ra.nrow + 127) / 128, (unsigned)((ra.nkp + KG - 1) / KG));
        const size_t sm = sizeof(float2) * KG * ra.nRe;
        if (sm > 48 * 1024) EPWI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        kern<<<grid, 128, sm, c->stream>>>(ra, out);
        EPWI_CHECK_LAUNCH();
    };
    auto kb = [&](auto kern, int rows_per_block) {
        dim3 grid((ra.nrow + rows_per_block - 1) / rows_per_block, (unsigned)((ra.nkp + 31) / 32));
        kern<<<grid, 256, 0, c->stream>>>(ra, out);
        EPWI_CHECK_LAUNCH();
    };
    // measured: the k-blocked kernel pays for the Si-like shape (72 -> 53 ms at 100^3) and not
    // for W = 4 (6.8 -> 9.2 ms at 48^3)
    if (W == 4) go(k_restage_f32<4, 8>, 8);
    else if (W == 8) kb(k_restage_f32_kb<8>, 32);
    else if (W == 1) go(k_restage_f32<1, 8>, 8);
    else go(k_restage_f32<0, 1>, 1);
}

// Rates of the chunk's states: one CTA per (k-point, band), written straight into inv_tau.
void sf_scatter(epwi_ctx *c, const ScatterArgs &sa, int64_t nkp, const int64_t *kp_pairs_local, int64_t p_off,
                const std::vector<int64_t> &h_kp_state_chunk) {
    const int W = c->nw, NM = c->nm, r = c->sf_r;
    const int D = 2 * r + 1, X = NM * W;
    SfArgs a;
    a.g = sa.g;
    a.nplane = sa.g.n2 * sa.g.n3;
    int q2max = 1;
    for (int64_t pb = 0; pb * kSieveBlock < a.nplane; ++pb) {
        const int64_t c0 = pb * kSieveBlock, c1 = std::min<int64_t>(a.nplane, c0 + kSieveBlock) - 1;
        q2max = std::max<int>(q2max, (int)(c1 / sa.g.n3 - c0 / sa.g.n3 + 1));
    }
    const SfPlan plan = sf_plan(D, X, q2max, sa.g.n1, sa.g.n2, sa.g.n3);
    EPWI_REQUIRE((int64_t)sa.g.n1 * plan.njg <= 8192 && plan.pbmax <= 8192, EPWI_EUNSUPPORTED,
                 "fp32 mode: too many runs or plane blocks");
    a.jq = plan.jq;
    a.njg = plan.njg;
    a.pbmax = plan.pbmax;
    a.fplane = make_fdiv((uint32_t)a.nplane);
    a.fjq = make_fdiv((uint32_t)plan.jq);
    a.hwmax32 = c->hwmax32.as<float>();
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
    a.Vb32 = c->sf_Vt32.as<float2>();
    a.ef = c->sf_ef.as<float2>();
    a.uS = c->sf_uS.as<float2>();
    a.wn = c->sf_wn.as<float2>();
    a.nk = c->nk;
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
    const size_t sm = plan.smem;
    if (W == 4 && NM == 3 && r == 1) launch_sf<4, 3, 1>(c, a, ni, sm);
    else if (W == 4 && NM == 3 && r == 2) launch_sf<4, 3, 2>(c, a, ni, sm);
    else if (W == 4 && NM == 3 && r == 3) launch_sf<4, 3, 3>(c, a, ni, sm);
    else if (W == 1 && NM == 3 && r == 1) launch_sf<1, 3, 1>(c, a, ni, sm);
    else if (W == 1 && NM == 3 && r == 2) launch_sf<1, 3, 2>(c, a, ni, sm);
    else if (W == 8 && NM == 6 && r == 1) launch_sf<8, 6, 1>(c, a, ni, sm);
    else if (W == 8 && NM == 6 && r == 2) launch_sf<8, 6, 2>(c, a, ni, sm);
    else if (W == 8 && NM == 6 && r == 3) launch_sf<8, 6, 3>(c, a, ni, sm);
    else sf_check(c);
    // the host vector of items must outlive the copy
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
}
