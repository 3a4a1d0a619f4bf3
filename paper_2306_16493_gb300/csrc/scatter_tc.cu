// Split-precision Rp->q stage on the tcgen05 tensor cores, fused with the rotations and the
// Gaussian delta sum (Sec. III C, Eq. 16, and Sec. II C, Eq. 10).
//
// For one k-point and a tile of 128 kept q (one q per TMEM lane / thread):
//   A = P^ph (128 x Rp), phases e^{i q.Rp} taken from a table of L-th roots of unity by exact
//       integer reduction, written by the threads into shared memory as four operands
//       Pr_hi, Pi_hi, Pr_lo, Pi_lo (x = hi + lo, hi = round(x), lo = round(x - hi));
//   B = ghat(k) (Rp x columns), columns (band n, mode-component mu, Wannier i), split alike;
//   D = A B in TMEM, FP32: Dr = Pr Br - Pi Bi, Di = Pr Bi + Pi Br, each product as
//       hi*hi + hi*lo + lo*hi (the lo*lo term, ~2^-22 relative for fp16/tf32, is dropped).
// K (= Rp) is streamed in chunks of 64 bytes per row through a two-stage shared-memory ring:
// the threads write chunk c+1 while the tensor core multiplies chunk c.  After the last
// chunk every thread loads its row of D (tcgen05.ld), rotates it by V(k+q)^dag and u(q) in
// FP32 and accumulates |g|^2 [(N+f) e^{-(x+/eta)^2} + (1+N-f) e^{-(x-/eta)^2}] with
// x = (e_nk - mu) +/- w - (e_mk+q - mu) in FP32; tile sums are carried in FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "scatter.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr uint64_t kWaitTimeoutNs = 2000000000ull;   // 2 s per mbarrier wait

struct OpF16 {
    static constexpr int kBytes = 2;
    static constexpr uint32_t kFmt = 0;
    static constexpr bool kTF32 = false;
};
struct OpBF16 {
    static constexpr int kBytes = 2;
    static constexpr uint32_t kFmt = 1;
    static constexpr bool kTF32 = false;
};
struct OpTF32 {
    static constexpr int kBytes = 4;
    static constexpr uint32_t kFmt = 2;
    static constexpr bool kTF32 = true;
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// hi/lo split of a value; returns the bit patterns of the operand type.
template <class Op>
__device__ __forceinline__ void split2(double x, uint32_t &hi, uint32_t &lo) {
    if constexpr (Op::kTF32) {
        const float xf = (float)x;
        hi = to_tf32(xf);
        lo = to_tf32((float)(x - (double)__uint_as_float(hi)));
    } else if constexpr (Op::kFmt == 0) {
        const __half h = __double2half(x);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__double2half(x - (double)__half2float(h)));
    } else {
        const __nv_bfloat16 h = __double2bfloat16(x);
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(__double2bfloat16(x - (double)__bfloat162float(h)));
    }
}

template <class Op>
__device__ __forceinline__ void split2f(float x, uint32_t &hi, uint32_t &lo) {
    if constexpr (Op::kTF32) {
        hi = to_tf32(x);
        lo = to_tf32(x - __uint_as_float(hi));
    } else if constexpr (Op::kFmt == 0) {
        const __half h = __float2half_rn(x);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
    }
}

// Pre-split phase table, doubled (index m in [0, 2L) holds e^{2 pi i (m mod L)/L}) so that a
// sum of two reduced indices needs no modulo.  16-bit types: {re_h | im_h << 16, re_l | im_l << 16};
// tf32: {re_h, im_h, re_l, im_l}.
template <class Op>
__global__ void k_phase_split(int L, const double2 *__restrict__ ph64, uint32_t *__restrict__ out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= 2 * L) return;
    const double2 p = ph64[m % L];
    uint32_t rh, rl, ih, il;
    split2<Op>(p.x, rh, rl);
    split2<Op>(p.y, ih, il);
    if constexpr (Op::kTF32) {
        out[4 * m + 0] = rh;
        out[4 * m + 1] = ih;
        out[4 * m + 2] = rl;
        out[4 * m + 3] = il;
    } else {
        out[2 * m + 0] = rh | (ih << 16);
        out[2 * m + 1] = rl | (il << 16);
    }
}

// FP32 per-call tables: energies relative to mu, occupations, mode energies (-1 if dropped).
__global__ void k_tc_tables(int64_t nk, int W, int Nm, const double *__restrict__ eps,
                            const double *__restrict__ hw, const double *__restrict__ focc,
                            const double *__restrict__ nocc, double mu, double omega_min,
                            float *__restrict__ erel, float *__restrict__ f32,
                            float *__restrict__ n32, float *__restrict__ hw32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nk * W) {
        erel[i] = (float)(eps[i] - mu);
        f32[i] = (float)focc[i];
    }
    if (i < nk * Nm) {
        const double w = hw[i];
        const bool keep = w >= omega_min;
        hw32[i] = keep ? (float)w : -1.0f;
        n32[i] = keep ? (float)nocc[i] : 0.0f;
    }
}

// Re->k stage in FP32: ghat32[state][rp][mu][i] = sum_j [sum_Re e^{ik.Re} gw32] V32_jn.
template <int W, int KG>
__global__ void __launch_bounds__(128) k_restage_f32(RestageArgs a, float2 *__restrict__ out) {
    extern __shared__ float2 Pf[];   // [KG][nRe]
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
        Pf[idx] = p;
    }
    __syncthreads();
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= a.nrow) return;
    float2 acc[KG][W];
#pragma unroll
    for (int kk = 0; kk < KG; ++kk)
#pragma unroll
        for (int j = 0; j < W; ++j) acc[kk][j] = make_float2(0.f, 0.f);
    const float2 *gw = a.gw32 + (size_t)row * W;
    for (int r = 0; r < a.nRe; ++r) {
        float2 gv[W];
#pragma unroll
        for (int j = 0; j < W; ++j) gv[j] = __ldg(gw + (size_t)r * a.nrow * W + j);
#pragma unroll
        for (int kk = 0; kk < KG; ++kk) {
            const float2 p = Pf[kk * a.nRe + r];
#pragma unroll
            for (int j = 0; j < W; ++j) acc[kk][j] = cfmaf(p, gv[j], acc[kk][j]);
        }
    }
#pragma unroll
    for (int kk = 0; kk < KG; ++kk) {
        if (kg0 + kk >= a.nkp) break;
        const int ik = a.kpts[kg0 + kk];
        const int lo = a.ovr_nsel >= 0 ? a.ovr_lo : a.win_lo[ik];
        const int ns = a.ovr_nsel >= 0 ? a.ovr_nsel : a.win_n[ik];
        const int64_t s0 = a.kp_state[kg0 + kk] - a.s_base;
        const float2 *Vk = a.V32 + (int64_t)ik * W * W;
        for (int np = 0; np < ns; ++np) {
            float2 o = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < W; ++j) o = cfmaf(acc[kk][j], Vk[j * W + lo + np], o);
            out[(s0 + np) * a.nrow + row] = o;
        }
    }
}

struct TcArgs {
    ScatterArgs s;
    const float2 *ghat32;          // [state][nRp][NM*W]
    const uint32_t *ptab;          // pre-split doubled phase table
    const float *erel32, *f32, *n32, *hw32;
    float scale, scale_inv2;       // B scaled by 2^e before the split; |g|^2 scaled back
    float ceta32, inv_eta32;
    int cube_r;                    // Rp = full cube [-r, r]^3, n3 fastest
    int nchunk;                    // K chunks
    int nbg;                       // bands per column group
    int ncp_max;                   // B rows per stage
    uint32_t tmem_cols;
    int64_t ntiles;
    int *err;                      // [0]: timed-out waits
};

__device__ __forceinline__ int pmod(int x, int L) {
    int r = x % L;
    return r < 0 ? r + L : r;
}

template <class Op, int W, int NM>
__global__ void __launch_bounds__(128, 1) k_scatter_tc(TcArgs a) {
    constexpr int ES = Op::kBytes;
    constexpr int KC = 64 / ES;                 // Rp per chunk (64 bytes per row and operand)
    constexpr int EPV = 16 / ES;                // elements per 16-byte core-matrix row
    constexpr int NMW = NM * W;
    constexpr int NMWP = (NMW + 15) / 16 * 16;  // columns per band, padded to the MMA N granule
    constexpr uint32_t A_ARR = 128 * 64;        // bytes per A operand per stage
    constexpr int TW = Op::kTF32 ? 4 : 2;       // 32-bit words per table entry
    const ScatterArgs &s = a.s;
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t B_ARR = (uint32_t)a.ncp_max * 64;
    uint8_t *sA = smem;
    uint8_t *sB = sA + 2 * 4 * A_ARR;
    uint32_t *sT = reinterpret_cast<uint32_t *>(sB + 2 * 4 * B_ARR);
    const int L = s.g.L;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sT + ((2 * L * TW + 1) & ~1));
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
    float *wred = reinterpret_cast<float *>(tslot + 4);   // [4][kMaxW]

    for (int i = tid; i < 2 * L * TW; i += blockDim.x) sT[i] = a.ptab[i];
    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, a.tmem_cols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);

    const int r = a.cube_r, D = 2 * r + 1, D2 = D * D;
    uint32_t use[2] = {0, 0}, done[2] = {0, 0};
    uint32_t ctr = 0;
    bool failed = false;

    for (int64_t tile = blockIdx.x; tile < a.ntiles && !failed; tile += gridDim.x) {
        const int4 t = s.tiles[tile];
        const int kpl = t.x;
        const int64_t pair = (int64_t)t.y + tid;
        const bool active = pair < t.z;
        const int ik = s.kpts[kpl];
        const int lo = s.ovr_nsel >= 0 ? s.ovr_lo : s.win_lo[ik];
        const int nsel = s.ovr_nsel >= 0 ? s.ovr_nsel : s.win_n[ik];
        const int64_t s0 = s.kp_state[kpl] - s.s_base;
        int iq = 0;
        int64_t ikq = 0;
        int a1 = 0, a2 = 0, a3 = 0;
        if (active) {
            iq = s.pairs[pair];
            ikq = kplusq(s.g, ik, iq);
            int i1, i2, i3;
            grid_coords(s.g, iq, i1, i2, i3);
            a1 = i1 * s.g.s1 % L;
            a2 = i2 * s.g.s2 % L;
            a3 = i3 * s.g.s3 % L;
        }
        const int c3m = pmod(-r * a3, L);

        for (int g0 = 0; g0 < nsel && !failed; g0 += a.nbg) {
            const int nb = min(a.nbg, nsel - g0);
            const int ncp = nb * NMWP;
            const uint32_t idP = tc::idesc(Op::kFmt, 128, ncp, false);
            const uint32_t idN = tc::idesc(Op::kFmt, 128, ncp, true);
            for (int ch = 0; ch < a.nchunk; ++ch) {
                const int st = ctr & 1;
                if (use[st] > done[st]) {
                    if (!tc::mbar_wait_bounded(&bars[st], done[st] & 1, kWaitTimeoutNs)) failed = true;
                    ++done[st];
                }
                if (__syncthreads_or(failed)) {
                    failed = true;
                    break;
                }
                // ---- A: phases of this thread's q for Rp = ch*KC .. ch*KC+KC-1
                const int k0 = ch * KC;
                int n1 = k0 / D2 - r, n2 = (k0 / D) % D - r, n3 = k0 % D - r;
                int b12 = pmod(n1 * a1 + n2 * a2, L);
                int c3 = pmod(n3 * a3, L);
                uint8_t *aSt = sA + st * 4 * A_ARR;
                const uint32_t rowoff = (uint32_t)((tid >> 3) * 4) * 128 + (tid & 7) * 16;
#pragma unroll
                for (int kb = 0; kb < 4; ++kb) {
                    uint32_t e[EPV][TW];
#pragma unroll
                    for (int j = 0; j < EPV; ++j) {
                        const int k = k0 + kb * EPV + j;
                        const bool ok = active && k < s.nRp;
                        const uint32_t *src = sT + (size_t)(b12 + c3) * TW;
#pragma unroll
                        for (int w = 0; w < TW; ++w) e[j][w] = ok ? src[w] : 0u;
                        // advance (n1, n2, n3) with carries
                        ++n3;
                        c3 += a3;
                        if (c3 >= L) c3 -= L;
                        if (n3 > r) {
                            n3 = -r;
                            c3 = c3m;
                            ++n2;
                            b12 += a2;
                            if (b12 >= L) b12 -= L;
                            if (n2 > r) {
                                n2 = -r;
                                ++n1;
                                b12 = pmod(n1 * a1 + n2 * a2, L);
                            }
                        }
                    }
                    uint4 v[4];
                    if constexpr (Op::kTF32) {
                        v[0] = make_uint4(e[0][0], e[1][0], e[2][0], e[3][0]);
                        v[1] = make_uint4(e[0][1], e[1][1], e[2][1], e[3][1]);
                        v[2] = make_uint4(e[0][2], e[1][2], e[2][2], e[3][2]);
                        v[3] = make_uint4(e[0][3], e[1][3], e[2][3], e[3][3]);
                    } else {
                        uint32_t w4[4][4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            w4[0][q] = __byte_perm(e[2 * q][0], e[2 * q + 1][0], 0x5410);
                            w4[1][q] = __byte_perm(e[2 * q][0], e[2 * q + 1][0], 0x7632);
                            w4[2][q] = __byte_perm(e[2 * q][1], e[2 * q + 1][1], 0x5410);
                            w4[3][q] = __byte_perm(e[2 * q][1], e[2 * q + 1][1], 0x7632);
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) v[q] = make_uint4(w4[q][0], w4[q][1], w4[q][2], w4[q][3]);
                    }
#pragma unroll
                    for (int arr = 0; arr < 4; ++arr)
                        *reinterpret_cast<uint4 *>(aSt + arr * A_ARR + rowoff + kb * 128) = v[arr];
                }
                // ---- B: ghat(k) columns of this band group, same chunk of Rp
                uint8_t *bSt = sB + st * 4 * B_ARR;
                for (int idx = tid; idx < KC * ncp; idx += blockDim.x) {
                    const int kk = idx / ncp, c = idx - kk * ncp;
                    const int b = c / NMWP, mi = c - b * NMWP;
                    const int k = k0 + kk;
                    float2 v = make_float2(0.f, 0.f);
                    if (mi < NMW && k < s.nRp)
                        v = __ldg(a.ghat32 + ((s0 + g0 + b) * s.nRp + k) * NMW + mi);
                    uint32_t rh, rl, ih, il;
                    split2f<Op>(v.x * a.scale, rh, rl);
                    split2f<Op>(v.y * a.scale, ih, il);
                    const uint32_t off = (uint32_t)(((c >> 3) * 4 + (kk * ES) / 16) * 128 + (c & 7) * 16 + (kk * ES) % 16);
                    if constexpr (ES == 4) {
                        *reinterpret_cast<uint32_t *>(bSt + 0 * B_ARR + off) = rh;
                        *reinterpret_cast<uint32_t *>(bSt + 1 * B_ARR + off) = ih;
                        *reinterpret_cast<uint32_t *>(bSt + 2 * B_ARR + off) = rl;
                        *reinterpret_cast<uint32_t *>(bSt + 3 * B_ARR + off) = il;
                    } else {
                        *reinterpret_cast<uint16_t *>(bSt + 0 * B_ARR + off) = (uint16_t)rh;
                        *reinterpret_cast<uint16_t *>(bSt + 1 * B_ARR + off) = (uint16_t)ih;
                        *reinterpret_cast<uint16_t *>(bSt + 2 * B_ARR + off) = (uint16_t)rl;
                        *reinterpret_cast<uint16_t *>(bSt + 3 * B_ARR + off) = (uint16_t)il;
                    }
                }
                tc::fence_proxy_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc::tc_fence_after();
                    const uint32_t aB = tc::smem_u32(aSt), bB = tc::smem_u32(bSt);
                    const uint32_t dR = tmem, dI = tmem + (uint32_t)ncp;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        uint64_t A[4], B[4];
#pragma unroll
                        for (int arr = 0; arr < 4; ++arr) {
                            A[arr] = tc::sdesc(aB + arr * A_ARR + ks * 256, 128, 512);
                            B[arr] = tc::sdesc(bB + arr * B_ARR + ks * 256, 128, 512);
                        }
                        const uint32_t acc = (ch == 0 && ks == 0) ? 0u : 1u;
                        // Dr = Pr Br - Pi Bi ; Di = Pr Bi + Pi Br ; each as hh + hl + lh
                        tc::mma<Op::kTF32>(dR, A[0], B[0], idP, acc);
                        tc::mma<Op::kTF32>(dR, A[0], B[2], idP, 1);
                        tc::mma<Op::kTF32>(dR, A[2], B[0], idP, 1);
                        tc::mma<Op::kTF32>(dR, A[1], B[1], idN, 1);
                        tc::mma<Op::kTF32>(dR, A[1], B[3], idN, 1);
                        tc::mma<Op::kTF32>(dR, A[3], B[1], idN, 1);
                        tc::mma<Op::kTF32>(dI, A[0], B[1], idP, acc);
                        tc::mma<Op::kTF32>(dI, A[0], B[3], idP, 1);
                        tc::mma<Op::kTF32>(dI, A[2], B[1], idP, 1);
                        tc::mma<Op::kTF32>(dI, A[1], B[0], idP, 1);
                        tc::mma<Op::kTF32>(dI, A[1], B[2], idP, 1);
                        tc::mma<Op::kTF32>(dI, A[3], B[0], idP, 1);
                    }
                    tc::mma_commit(&bars[st]);
                }
                ++use[st];
                ++ctr;
            }
            if (failed) break;
            // ---- wait for the accumulator, then the epilogue (one thread per q)
            {
                const int st = (ctr - 1) & 1;
                if (!tc::mbar_wait_bounded(&bars[st], done[st] & 1, kWaitTimeoutNs)) failed = true;
                ++done[st];
                if (__syncthreads_or(failed)) {
                    failed = true;
                    break;
                }
            }
            tc::tc_fence_after();
            for (int b = 0; b < nb; ++b) {
                float gr[NMWP], gi[NMWP];
#pragma unroll
                for (int blk = 0; blk < NMWP / 16; ++blk) {
                    float tmp[16];
                    tc::tmem_ld16(tmem_row + (uint32_t)(b * NMWP + blk * 16), tmp);
#pragma unroll
                    for (int x = 0; x < 16; ++x) gr[blk * 16 + x] = tmp[x];
                    tc::tmem_ld16(tmem_row + (uint32_t)(ncp + b * NMWP + blk * 16), tmp);
#pragma unroll
                    for (int x = 0; x < 16; ++x) gi[blk * 16 + x] = tmp[x];
                }
                tc::tmem_wait_ld();
                float rate = 0.f;
                if (active) {
                    const int band = lo + g0 + b;
                    const float en = a.erel32[(int64_t)ik * W + band];
                    const float2 *Vq = s.V32 + ikq * W * W;
                    const float2 *uq = s.u32 + (int64_t)iq * NM * NM;
                    float2 uu[NM][NM];
#pragma unroll
                    for (int x = 0; x < NM; ++x)
#pragma unroll
                        for (int y = 0; y < NM; ++y) uu[x][y] = __ldg(uq + x * NM + y);
                    float wq[NM], nq[NM];
#pragma unroll
                    for (int nu = 0; nu < NM; ++nu) {
                        wq[nu] = __ldg(a.hw32 + (int64_t)iq * NM + nu);
                        nq[nu] = __ldg(a.n32 + (int64_t)iq * NM + nu);
                    }
#pragma unroll
                    for (int m = 0; m < W; ++m) {
                        float2 h[NM];
#pragma unroll
                        for (int mu = 0; mu < NM; ++mu) {
                            h[mu] = make_float2(0.f, 0.f);
#pragma unroll
                            for (int i = 0; i < W; ++i)
                                h[mu] = cfmacf(__ldg(Vq + i * W + m), make_float2(gr[mu * W + i], gi[mu * W + i]), h[mu]);
                        }
                        const float em = __ldg(a.erel32 + ikq * W + m);
                        const float fm = __ldg(a.f32 + ikq * W + m);
#pragma unroll
                        for (int nu = 0; nu < NM; ++nu) {
                            const float w = wq[nu];
                            float2 gv = make_float2(0.f, 0.f);
#pragma unroll
                            for (int mu = 0; mu < NM; ++mu) gv = cfmaf(h[mu], uu[mu][nu], gv);
                            const float g2 = gv.x * gv.x + gv.y * gv.y;
                            if (s.g2out) {
                                s.g2out[(((s.g2_base + pair) * nsel + g0 + b) * NM + nu) * W + m] =
                                    (w >= 0.f) ? (double)g2 * (double)a.scale_inv2 : 0.0;
                                continue;
                            }
                            if (w < 0.f) continue;
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
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) rate += __shfl_down_sync(0xffffffffu, rate, o);
                if (lane == 0) wred[warp * epc::kMaxW + g0 + b] = rate * a.scale_inv2;
            }
            tc::tc_fence_before();
        }
        __syncthreads();
        if (!failed && tid < nsel)
            s.tile_part[tile * epc::kMaxW + tid] =
                ((double)wred[tid] + (double)wred[epc::kMaxW + tid]) +
                ((double)wred[2 * epc::kMaxW + tid] + (double)wred[3 * epc::kMaxW + tid]);
    }
    // wind down: make sure no MMA is still writing TMEM, then free it
    for (int st = 0; st < 2; ++st)
        if (use[st] > done[st]) {
            if (!tc::mbar_wait_bounded(&bars[st], done[st] & 1, kWaitTimeoutNs)) failed = true;
            ++done[st];
        }
    if (failed && tid == 0) atomicAdd(a.err, 1);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, a.tmem_cols);
}

template <class Op>
const uint32_t *phase_table(epwi_ctx *c) {
    const int key = c->L * 8 + c->opt.precision;
    const int TW = Op::kTF32 ? 4 : 2;
    if (c->tc_ptab_key != key) {
        c->tc_ptab.ensure(sizeof(uint32_t) * 2 * c->L * TW);
        k_phase_split<Op><<<(2 * c->L + 127) / 128, 128, 0, c->stream>>>(c->L, c->ph64.as<double2>(),
                                                                        c->tc_ptab.as<uint32_t>());
        EPWI_CHECK_LAUNCH();
        c->tc_ptab_key = key;
    }
    return c->tc_ptab.as<uint32_t>();
}

template <class Op, int W, int NM>
void launch_tc(epwi_ctx *c, const ScatterArgs &sa, int64_t ntiles) {
    constexpr int ES = Op::kBytes;
    constexpr int NMWP = (NM * W + 15) / 16 * 16;
    constexpr int TW = Op::kTF32 ? 4 : 2;
    TcArgs a;
    a.s = sa;
    a.ghat32 = static_cast<const float2 *>(sa.ghat_raw);
    a.ptab = phase_table<Op>(c);
    a.erel32 = c->tc_erel.as<float>();
    a.f32 = c->tc_f32.as<float>();
    a.n32 = c->tc_n32.as<float>();
    a.hw32 = c->tc_hw32.as<float>();
    const int e = (Op::kFmt == 0 && !Op::kTF32) ? c->tc_scale_exp : 0;
    a.scale = std::ldexp(1.0f, e);
    a.scale_inv2 = std::ldexp(1.0f, -2 * e);
    a.ceta32 = (float)sa.ceta;
    a.inv_eta32 = (float)(1.0 / sa.eta);
    a.cube_r = c->rp_cube_r;
    a.nchunk = (c->nRp + 64 / ES - 1) / (64 / ES);
    a.nbg = std::max(1, 128 / NMWP);
    a.ncp_max = std::min(sa.nsel_max, a.nbg) * NMWP;
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * a.ncp_max)) cols <<= 1;
    a.tmem_cols = cols;
    a.ntiles = ntiles;
    c->tc_err.ensure(sizeof(int) * 4);
    EPWI_CUDA(cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream));
    a.err = c->tc_err.as<int>();
    size_t smem = 2 * 4 * 128 * 64 + 2 * 4 * (size_t)a.ncp_max * 64 +
                  sizeof(uint32_t) * ((2 * c->L * TW + 1) & ~1) + 16 + 16 + 4 * epc::kMaxW * 4 + 64;
    auto kern = k_scatter_tc<Op, W, NM>;
    int dev = c->device, nsm = 0;
    EPWI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // keep (resident CTAs per SM) x (TMEM columns) <= 512 so that tcgen05.alloc never waits
    int per_sm = 0;
    for (;;) {
        EPWI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        EPWI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem));
        EPWI_REQUIRE(per_sm >= 1, EPWI_EUNSUPPORTED, "tensor-core kernel does not fit on an SM");
        if ((uint32_t)per_sm * cols <= 512) break;
        smem += 8 * 1024;
    }
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)per_sm * nsm);
    if (grid > 0) {
        kern<<<(unsigned)grid, 128, smem, c->stream>>>(a);
        EPWI_CHECK_LAUNCH();
    }
    c->tc_blocks_per_sm = per_sm;
}

template <class Op>
void dispatch_tc(epwi_ctx *c, const ScatterArgs &sa, int64_t nt) {
    const int W = c->nw, NM = c->nm;
    if (W == 1 && NM == 3) launch_tc<Op, 1, 3>(c, sa, nt);
    else if (W == 4 && NM == 3) launch_tc<Op, 4, 3>(c, sa, nt);
    else if (W == 8 && NM == 6) launch_tc<Op, 8, 6>(c, sa, nt);
    else throw EpwiError{EPWI_EUNSUPPORTED, "split-precision path built for (nw, modes) in {(1,3), (4,3), (8,6)}"};
}

}  // namespace

size_t tc_state_bytes(const epwi_ctx *c) { return sizeof(float2) * (size_t)c->nRp * c->nm * c->nw; }

void tc_tables(epwi_ctx *c) {
    const int64_t nk = c->nk;
    c->tc_erel.ensure(sizeof(float) * nk * c->nw);
    c->tc_f32.ensure(sizeof(float) * nk * c->nw);
    c->tc_n32.ensure(sizeof(float) * nk * c->nm);
    c->tc_hw32.ensure(sizeof(float) * nk * c->nm);
    const int64_t n = nk * std::max(c->nw, c->nm);
    k_tc_tables<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
        nk, c->nw, c->nm, c->eps.as<double>(), c->hw.as<double>(), c->focc.as<double>(),
        c->nocc.as<double>(), c->mu, c->opt.omega_min_eV, c->tc_erel.as<float>(), c->tc_f32.as<float>(),
        c->tc_n32.as<float>(), c->tc_hw32.as<float>());
    EPWI_CHECK_LAUNCH();
}

void tc_restage(epwi_ctx *c, const RestageArgs &ra) {
    float2 *out = static_cast<float2 *>(ra.ghat_raw);
    auto go = [&](auto kern, int KG) {
        dim3 grid((ra.nrow + 127) / 128, (unsigned)((ra.nkp + KG - 1) / KG));
        const size_t sm = sizeof(float2) * KG * ra.nRe;
        if (sm > 48 * 1024)
            EPWI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        kern<<<grid, 128, sm, c->stream>>>(ra, out);
        EPWI_CHECK_LAUNCH();
    };
    if (ra.W == 1) go(k_restage_f32<1, 8>, 8);
    else if (ra.W == 4) go(k_restage_f32<4, 8>, 8);
    else if (ra.W == 8) go(k_restage_f32<8, 4>, 4);
    else throw EpwiError{EPWI_EUNSUPPORTED, "split-precision Re->k stage built for nw in {1, 4, 8}"};
}

void tc_scatter(epwi_ctx *c, const ScatterArgs &sa, int64_t ntiles) {
    EPWI_REQUIRE(c->rp_cube_r >= 0, EPWI_EUNSUPPORTED,
                 "split-precision path needs the phonon R-set to be a full cube [-r, r]^3 (n3 fastest)");
    switch (c->opt.precision) {
        case EPWI_FP16X3: dispatch_tc<OpF16>(c, sa, ntiles); break;
        case EPWI_BF16X3: dispatch_tc<OpBF16>(c, sa, ntiles); break;
        case EPWI_TF32X3: dispatch_tc<OpTF32>(c, sa, ntiles); break;
        default: throw EpwiError{EPWI_EINVAL, "not a split-precision mode"};
    }
}

int tc_check_error(epwi_ctx *c) {
    int h = 0;
    EPWI_CUDA(cudaMemcpyAsync(&h, c->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    return h;
}
