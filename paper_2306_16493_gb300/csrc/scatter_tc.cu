// Split-precision Rp->q stage on the tcgen05 tensor cores, fused with the rotations and the
// Gaussian delta sum (Sec. III C, Eq. 16, and Sec. II C, Eq. 10).
//
// For one k-point and a tile of 128 kept q (one q per TMEM lane / thread):
//   A = P^ph (128 x Rp), phases e^{i q.Rp} taken from a table of L-th roots of unity by exact
//       integer reduction, written by the threads into shared memory as four operands
//       Pr_hi, Pi_hi, Pr_lo, Pi_lo (x = hi + lo, hi = round(x), lo = round(x - hi));
//   B = ghat(k) (Rp x columns), columns (band n, mode-component mu, Wannier i), split alike;
//   D = A B in TMEM, FP32: Dr = Pr Br - Pi Bi, Di = Pr Bi + Pi Br, each product as
//       hi*hi + hi*lo + lo*hi (the lo*lo term, ~2^-22 relative for fp16/tf32, is dropped),
//       issued as four wide MMAs per K step against B concatenated along N (see k_scatter_tc).
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
// sum of two reduced indices needs no modulo, and replicated R = 2^rlog times (entry m, copy g
// at position m*R + g) so that lanes reading different copies never share a bank.
// 16-bit types: {re_h | im_h << 16, re_l | im_l << 16}; tf32: {re_h, im_h, re_l, im_l}.
template <class Op>
__global__ void k_phase_split(int L, int rlog, const double2 *__restrict__ ph64, uint32_t *__restrict__ out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= 2 * L) return;
    const double2 p = ph64[m % L];
    uint32_t rh, rl, ih, il;
    split2<Op>(p.x, rh, rl);
    split2<Op>(p.y, ih, il);
    for (int g = 0; g < (1 << rlog); ++g) {
        const size_t o = (size_t)((m << rlog) | g);
        if constexpr (Op::kTF32) {
            out[4 * o + 0] = rh;
            out[4 * o + 1] = ih;
            out[4 * o + 2] = rl;
            out[4 * o + 3] = il;
        } else {
            out[2 * o + 0] = rh | (ih << 16);
            out[2 * o + 1] = rl | (il << 16);
        }
    }
}

// Split phase rows for the gathered-A mode, one per grid point q: the four operands
// Pr_hi, Pi_hi, Pr_lo, Pi_lo of e^{i q.Rp} for Rp = 0 .. kpad-1 in the cube order of the
// tensor-core kernel (n3 fastest, n in [-RC, RC]), 16-bit types only.  Entries come from the
// same pre-split table as the in-kernel generation (copy 0), so the operand bits are those of
// the TMEM path; K beyond nRp takes entry 0, which meets zero B rows.
template <int RC>
__global__ void k_phase_rows(int64_t nq, GridInfo g, int kpad, int rlog,
                             const uint32_t *__restrict__ ptab, uint8_t *__restrict__ rows) {
    constexpr int D = 2 * RC + 1;
    constexpr int NRP = D * D * D;
    const int npc = kpad / 8;                       // 16-byte pieces per operand
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nq * npc) return;
    const int64_t q = t / npc;
    const int piece = (int)(t % npc);
    int i1, i2, i3;
    grid_coords(g, q, i1, i2, i3);
    const int a1 = i1 * g.s1 % g.L, a2 = i2 * g.s2 % g.L, a3 = i3 * g.s3 % g.L;
    uint16_t v[4][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = piece * 8 + j;
        int idx = 0;
        if (k < NRP) {
            const int n1 = k / (D * D) - RC, n2 = (k / D) % D - RC, n3 = k % D - RC;
            int x = (n1 * a1 + n2 * a2 + n3 * a3) % g.L;
            idx = x < 0 ? x + g.L : x;
        }
        const uint32_t w0 = ptab[(size_t)(idx << rlog) * 2], w1 = ptab[(size_t)(idx << rlog) * 2 + 1];
        v[0][j] = (uint16_t)(w0 & 0xffffu);
        v[1][j] = (uint16_t)(w0 >> 16);
        v[2][j] = (uint16_t)(w1 & 0xffffu);
        v[3][j] = (uint16_t)(w1 >> 16);
    }
    uint8_t *row = rows + q * (int64_t)(4 * kpad * 2);
#pragma unroll
    for (int arr = 0; arr < 4; ++arr) {
        uint4 u;
        u.x = v[arr][0] | ((uint32_t)v[arr][1] << 16);
        u.y = v[arr][2] | ((uint32_t)v[arr][3] << 16);
        u.z = v[arr][4] | ((uint32_t)v[arr][5] << 16);
        u.w = v[arr][6] | ((uint32_t)v[arr][7] << 16);
        *reinterpret_cast<uint4 *>(row + arr * kpad * 2 + piece * 16) = u;
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

// Byte offset of element (row c, k) inside one core-matrix block with 64 bytes of K per
// row (four 8x16-byte core matrices along K per 8-row group).
template <int ES>
__host__ __device__ __forceinline__ uint32_t cm_off(int c, int k) {
    return (uint32_t)(((c >> 3) * 4 + (k * ES) / 16) * 128 + (c & 7) * 16 + (k * ES) % 16);
}

// Re->k stage for the split-precision path.  ghat(k)[rp][mu][i][n] = sum_j [sum_Re e^{ik.Re}
// gw32] V32_jn is accumulated in FP32, scaled by 2^e, split into hi + lo and written as the
// B operand image of the tensor-core kernel:
//   img[ch][arr][state][NMWP rows][64 bytes]  (arr: Br_hi, Bi_hi, Br_lo, Bi_lo, -Bi_hi, -Bi_lo),
// row = mu*W + i (rows NMW..NMWP-1 and K beyond nRp stay zero), K = rp - ch*KC.
template <class Op, int W, int NM, int KG>
__global__ void __launch_bounds__(128) k_restage_tc(RestageArgs a, uint8_t *__restrict__ img,
                                                    int64_t ns, float scale) {
    constexpr int ES = Op::kBytes;
    constexpr int KC = 64 / ES;
    constexpr int NMW = NM * W;
    constexpr int NMWP = (NMW + 15) / 16 * 16;
    constexpr uint32_t BLK = NMWP * 64;
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
    const int rp = row / NMW, c = row - rp * NMW;
    const int ch = rp / KC, kk = rp - ch * KC;
    const uint32_t eoff = cm_off<ES>(c, kk);
#pragma unroll
    for (int q = 0; q < KG; ++q) {
        if (kg0 + q >= a.nkp) break;
        const int ik = a.kpts[kg0 + q];
        const int lo = a.ovr_nsel >= 0 ? a.ovr_lo : a.win_lo[ik];
        const int nsl = a.ovr_nsel >= 0 ? a.ovr_nsel : a.win_n[ik];
        const int64_t s0 = a.kp_state[kg0 + q] - a.s_base;
        const float2 *Vk = a.V32 + (int64_t)ik * W * W;
        for (int np = 0; np < nsl; ++np) {
            float2 o = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < W; ++j) o = cfmaf(acc[q][j], Vk[j * W + lo + np], o);
            uint32_t w6[6];
            split2f<Op>(o.x * scale, w6[0], w6[2]);
            split2f<Op>(o.y * scale, w6[1], w6[3]);
            const uint32_t sign = ES == 4 ? 0x80000000u : 0x8000u;
            w6[4] = w6[1] ^ sign;
            w6[5] = w6[3] ^ sign;
#pragma unroll
            for (int arr = 0; arr < 6; ++arr) {
                uint8_t *dst = img + ((size_t)(ch * 6 + arr) * ns + (s0 + np)) * BLK + eoff;
                if constexpr (ES == 4) *reinterpret_cast<uint32_t *>(dst) = w6[arr];
                else *reinterpret_cast<uint16_t *>(dst) = (uint16_t)w6[arr];
            }
        }
    }
}

// Per-tile metadata gathered once so that every thread starts a tile with one 32-byte load.
struct __align__(16) TileMeta {
    int kpl, begin, end, ik;
    int lo, nsel;
    long long s0;                  // chunk-local state offset of the k-point
};

__global__ void k_tile_meta(int64_t ntiles, const int4 *__restrict__ tiles, const int *__restrict__ kpts,
                            const int *__restrict__ win_lo, const int *__restrict__ win_n,
                            const int64_t *__restrict__ kp_state, int64_t s_base, int ovr_lo,
                            int ovr_nsel, TileMeta *__restrict__ meta) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int4 x = tiles[t];
    TileMeta m;
    m.kpl = x.x;
    m.begin = x.y;
    m.end = x.z;
    m.ik = kpts[x.x];
    m.lo = ovr_nsel >= 0 ? ovr_lo : win_lo[m.ik];
    m.nsel = ovr_nsel >= 0 ? ovr_nsel : win_n[m.ik];
    m.s0 = (long long)(kp_state[x.x] - s_base);
    meta[t] = m;
}

struct TcArgs {
    ScatterArgs s;
    const TileMeta *meta;
    const uint8_t *img;            // B image of the chunk (see k_restage_tc)
    int64_t ns;                    // states in the chunk (image stride)
    const uint32_t *ptab;          // pre-split doubled phase table, replicated 2^rlog times
    int rlog;
    const float *erel32, *f32, *n32, *hw32;
    float scale_inv2;              // |g|^2 scaled back by 2^-2e
    float ceta32, inv_eta32;
    int cube_r;                    // Rp = full cube [-r, r]^3, n3 fastest
    int nchunk;                    // K chunks
    int nbg;                       // bands per column group
    int ncp_max;                   // B rows per stage
    int bres;                      // 1: B of one (k-point, band group) resident in nchunk slots
    int nsa;                       // A stages in TMEM
    uint32_t a_col0;               // first TMEM column of the A stages (after the accumulators)
    uint32_t acc_cols;             // TMEM columns of one accumulator buffer
    uint32_t tmem_cols;
    int64_t ntiles;
    int *err;                      // [0]: timed-out waits
    const uint8_t *arows;          // gathered-A mode: split phase rows [q][4 operands][kpad]
    int64_t arow_bytes;            // bytes per q row (4 * arr_bytes)
    int arr_bytes;                 // bytes per operand (kpad * 2)
};

__device__ __forceinline__ int pmod(int x, int L) {
    int r = x % L;
    return r < 0 ? r + L : r;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void epilogue_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// B slot of one chunk: V1 = [Br_hi | Bi_hi | Br_lo | Bi_lo] then V2 = [-Bi_hi | Br_hi | -Bi_lo | Br_lo],
// each part ncp rows of 64 bytes; these are the image arrays in this order.
__constant__ int kSlotArr[8] = {0, 1, 2, 3, 4, 0, 5, 2};

// Issues the eight bulk copies of (k-point state s0, band group g0, chunk ch) into a slot
// (bytes counted on bar by the caller's expect_tx).
template <int NMWP>
__device__ __forceinline__ void copy_b(const TcArgs &a, long long s0, int g0, int nb, int ch, uint8_t *slot,
                                       uint64_t *bar) {
    const uint32_t bytes = (uint32_t)nb * NMWP * 64;
#pragma unroll
    for (int pos = 0; pos < 8; ++pos)
        tc::bulk_g2s(slot + pos * bytes,
                     a.img + ((size_t)(ch * 6 + kSlotArr[pos]) * a.ns + ((size_t)s0 + g0)) * (NMWP * 64), bytes,
                     bar);
}

template <int NMWP>
__device__ __forceinline__ void issue_b(const TcArgs &a, const TileMeta &m, int g0, int ch, uint8_t *slot,
                                        uint64_t *bar) {
    const int nb = min(a.nbg, m.nsel - g0);
    tc::mbar_arrive_expect_tx(bar, 8u * nb * NMWP * 64);
    copy_b<NMWP>(a, m.s0, g0, nb, ch, slot, bar);
}

// Warp-specialised CTA of 288 threads, one per SM:
//   warps 0-3  A producers: one q row each; phase operands (Pr_hi, Pi_hi, Pr_lo, Pi_lo) written
//              to TMEM with tcgen05.st, K streamed through NSA TMEM stages;
//   warps 4-7  epilogue: one q row each; accumulator rows read with tcgen05.ld, rotated and
//              delta-weighted in FP32, tile sums in FP64;
//   warp 8     lane 0 is the control thread: B operand bulk copies, tcgen05.mma issue/commit.
// The accumulator is double-buffered in TMEM, so the A producers and the MMAs of one band
// group run while the epilogue warps drain the previous one.  Roles talk through mbarriers
// only: a_full (one arrival per producer warp), mma_done (commit per chunk), b_full (bulk-copy
// bytes), acc_full (commit per group) and acc_empty (one arrival per epilogue warp).
// B either stays resident for a (k-point, band group) across consecutive tiles (reloaded
// only when it changes) or, when it does not fit, streams through two slots one chunk ahead.
// 9 warps put at most 3 on a sub-partition: <= 168 registers per thread.
template <class Op, int W, int NM, int RC, bool AG, bool GAM>
__global__ void __maxnreg__(168) k_scatter_tc(TcArgs a) {
    constexpr int ES = Op::kBytes;
    constexpr int KC = 64 / ES;                 // Rp per chunk (64 bytes per row and operand)
    constexpr int EPV = 16 / ES;                // elements per 16-byte core-matrix row
    constexpr int NMW = NM * W;
    constexpr int NMWP = (NMW + 15) / 16 * 16;  // columns per band, padded to the MMA N granule
    constexpr uint32_t A_COLS = 16;             // TMEM columns per A operand per stage (64 bytes)
    constexpr int TW = Op::kTF32 ? 4 : 2;       // 32-bit words per table entry
    constexpr bool PRE = (W * W + NM * NM) <= 32;   // keep the epilogue operands in registers
    constexpr int D = 2 * RC + 1;               // R_p cube side
    constexpr int NRP = D * D * D;
    constexpr int NCH = (NRP + KC - 1) / KC;    // K chunks (compile time)
    const ScatterArgs &s = a.s;
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t B_SLOT = 8u * (uint32_t)a.ncp_max * 64;   // one chunk of V1 and V2
    const int NSA = a.nsa;                      // A stages in TMEM
    // shared memory: B slots, then either the phase table (A generated into TMEM) or the
    // A stages (gathered-A mode: NSA x 4 operands x 128 rows x 64 bytes), then barriers
    constexpr uint32_t A_OP = 128 * 64;                     // one operand of one A stage
    uint8_t *sB = smem;
    uint32_t *sT = reinterpret_cast<uint32_t *>(sB + (a.bres ? a.nchunk : 2) * B_SLOT);
    uint8_t *sA = reinterpret_cast<uint8_t *>(sT);
    const int L = s.g.L;
    const int twords = AG ? 0 : 2 * L * (1 << a.rlog) * TW;
    uint64_t *bars = AG ? reinterpret_cast<uint64_t *>(sA + (size_t)a.nsa * 4 * A_OP)
                        : reinterpret_cast<uint64_t *>(sT + ((twords + 1) & ~1));
    uint64_t *a_full = bars, *mma_done = bars + 3, *b_full = bars + 6, *acc_full = bars + 8,
             *acc_empty = bars + 10, *drained = bars + 12;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 13);
    volatile int *sfail = reinterpret_cast<volatile int *>(tslot + 1);
    float *wred = reinterpret_cast<float *>(tslot + 4);   // [4][kMaxW]

    for (int i = tid; i < twords; i += blockDim.x) sT[i] = a.ptab[i];
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) {
            tc::mbar_init(&a_full[i], 4);     // one elected arrival per producer warp
            tc::mbar_init(&mma_done[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&b_full[i], 1);
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&acc_empty[i], 4);  // one elected arrival per epilogue warp
        }
        tc::mbar_init(drained, 1);
        *sfail = 0;
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
    const uint32_t acc_cols = a.acc_cols;        // columns of one accumulator buffer
    const uint32_t tmem_a = tmem + a.a_col0;     // A stages: NSA x 4 operands x 16 columns
    const int64_t t_begin = blockIdx.x * a.ntiles / gridDim.x;
    const int64_t t_end = (blockIdx.x + 1) * a.ntiles / gridDim.x;
    const unsigned n1 = s.g.n1, n2 = s.g.n2, n3 = s.g.n3;

    if (warp == 8) {
        // ------------------------------------------------------------ control thread
        if (lane == 0) {
            uint32_t aph[3] = {0, 0, 0}, bph[2] = {0, 0}, bpend[2] = {0, 0};
            uint32_t mc[3] = {0, 0, 0}, mw[3] = {0, 0, 0}, eph[2] = {0, 0};
            uint32_t ctr = 0, gctr = 0, dph = 0;
            bool failed = false;
            auto drain_mma = [&]() {
                if (a.bres) {
                    // a commit on its own barrier completes once every MMA issued so far has
                    tc::mma_commit(drained);
                    if (!tc::mbar_wait_bounded(drained, dph, kWaitTimeoutNs)) failed = true;
                    dph ^= 1;
                    return;
                }
                for (int st = 0; st < NSA; ++st)
                    while (mc[st] > mw[st]) {
                        if (!tc::mbar_wait_bounded(&mma_done[st], mw[st] & 1, kWaitTimeoutNs)) failed = true;
                        ++mw[st];
                    }
            };
            // streaming mode: (pt, pg, pc) is the next chunk to fetch into the 2-slot ring
            int64_t pt = t_begin;
            int pg = 0, pc = 0;
            TileMeta pm;
            auto prefetch = [&](int st2) {
                issue_b<NMWP>(a, pm, pg, pc, sB + st2 * B_SLOT, &b_full[st2]);
                ++bpend[st2];
                if (++pc == a.nchunk) {
                    pc = 0;
                    pg += a.nbg;
                    if (pg >= pm.nsel) {
                        pg = 0;
                        if (++pt < t_end) pm = a.meta[pt];
                    }
                }
            };
            if (!a.bres && pt < t_end) {
                pm = a.meta[pt];
                prefetch(0);
            }
            int tag_kp = -1, tag_g0 = -1;
            for (int64_t tile = t_begin; tile < t_end && !failed; ++tile) {
                const TileMeta m = a.meta[tile];
                for (int g0 = 0; g0 < m.nsel && !failed; g0 += a.nbg) {
                    const int ncp = min(a.nbg, m.nsel - g0) * NMWP;
                    const uint32_t id4 = tc::idesc(Op::kFmt, 128, 4 * ncp, false);
                    const uint32_t id2 = tc::idesc(Op::kFmt, 128, 2 * ncp, false);
                    if (a.bres && (m.kpl != tag_kp || g0 != tag_g0)) {
                        drain_mma();   // no MMA may still read the old operand
                        const int nb = min(a.nbg, m.nsel - g0);
                        tc::mbar_arrive_expect_tx(&b_full[0], 8u * nb * NMWP * 64 * a.nchunk);
                        for (int ch = 0; ch < a.nchunk; ++ch) copy_b<NMWP>(a, m.s0, g0, nb, ch, sB + ch * B_SLOT, &b_full[0]);
                        if (!tc::mbar_wait_bounded(&b_full[0], bph[0], kWaitTimeoutNs)) failed = true;
                        bph[0] ^= 1;
                        tag_kp = m.kpl;
                        tag_g0 = g0;
                    }
                    const int ab = gctr & 1;
                    if (gctr >= 2) {   // the epilogue has drained this buffer (two groups ago)
                        if (!tc::mbar_wait_bounded(&acc_empty[ab], eph[ab], kWaitTimeoutNs)) failed = true;
                        eph[ab] ^= 1;
                    }
                    tc::tc_fence_after();
                    const uint32_t dacc = tmem + (uint32_t)ab * acc_cols;
                    for (int ch = 0; ch < a.nchunk && !failed; ++ch) {
                        const int st = ctr % NSA;   // A stage; streaming mode has NSA = 2 = B slots
                        if (!tc::mbar_wait_bounded(&a_full[st], aph[st], kWaitTimeoutNs)) failed = true;
                        aph[st] ^= 1;
                        if (!a.bres) {
                            if (!tc::mbar_wait_bounded(&b_full[st], bph[st], kWaitTimeoutNs)) failed = true;
                            bph[st] ^= 1;
                            --bpend[st];
                        }
                        if (failed) break;
                        tc::tc_fence_after();
                        const uint32_t bV1 = tc::smem_u32(sB + (a.bres ? ch : st) * B_SLOT);
                        const uint32_t bV2 = bV1 + 4u * (uint32_t)ncp * 64;
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks) {
                            const uint64_t B1 = tc::sdesc(bV1 + ks * 256, 128, 512);
                            const uint64_t B2 = tc::sdesc(bV2 + ks * 256, 128, 512);
                            const uint32_t acc = (ch == 0 && ks == 0) ? 0u : 1u;
                            // D = [Dr_hi | Di_hi | Dr_lo | Di_lo]:  Pr_hi V1 + Pi_hi V2 fills all four
                            // (hi*hi and hi*lo), Pr_lo V1 + Pi_lo V2 on the first half adds lo*hi.
                            if constexpr (AG) {
                                // A in shared memory (canonical layout, 32 bytes of K per MMA)
                                const uint32_t aS = tc::smem_u32(sA + (size_t)st * 4 * A_OP) + ks * 256;
                                tc::mma<Op::kTF32>(dacc, tc::sdesc(aS, 128, 512), B1, id4, acc);
                                tc::mma<Op::kTF32>(dacc, tc::sdesc(aS + A_OP, 128, 512), B2, id4, 1);
                                tc::mma<Op::kTF32>(dacc, tc::sdesc(aS + 2 * A_OP, 128, 512), B1, id2, 1);
                                tc::mma<Op::kTF32>(dacc, tc::sdesc(aS + 3 * A_OP, 128, 512), B2, id2, 1);
                            } else {
                                // A in TMEM: Pr_hi, Pi_hi, Pr_lo, Pi_lo
                                const uint32_t aT = tmem_a + (uint32_t)(st * 4 * A_COLS);
                                const uint32_t Arh = aT + ks * 8, Aih = aT + A_COLS + ks * 8;
                                const uint32_t Arl = aT + 2 * A_COLS + ks * 8, Ail = aT + 3 * A_COLS + ks * 8;
                                tc::mma_ta<Op::kTF32>(dacc, Arh, B1, id4, acc);
                                tc::mma_ta<Op::kTF32>(dacc, Aih, B2, id4, 1);
                                tc::mma_ta<Op::kTF32>(dacc, Arl, B1, id2, 1);
                                tc::mma_ta<Op::kTF32>(dacc, Ail, B2, id2, 1);
                            }
                        }
                        tc::mma_commit(&mma_done[st]);
                        ++mc[st];
                        // streaming mode: B of the next chunk into the other slot once its MMAs are done
                        if (!a.bres && pt < t_end) {
                            const int st2 = st ^ 1;
                            if (mc[st2] > mw[st2]) {
                                if (!tc::mbar_wait_bounded(&mma_done[st2], mw[st2] & 1, kWaitTimeoutNs))
                                    failed = true;
                                ++mw[st2];
                            }
                            if (!failed) prefetch(st2);
                        }
                        ++ctr;
                    }
                    if (!failed) tc::mma_commit(&acc_full[ab]);   // this group's accumulator is ready
                    ++gctr;
                }
                if (*sfail) failed = true;
            }
            drain_mma();
            for (int st = 0; st < 2; ++st)
                while (bpend[st] > 0) {
                    if (!tc::mbar_wait_bounded(&b_full[st], bph[st], kWaitTimeoutNs)) failed = true;
                    bph[st] ^= 1;
                    --bpend[st];
                }
            if (failed) {
                *sfail = 1;
                atomicAdd(a.err, 1);
            }
        }
    } else if (warp < 4) {
        // ------------------------------------------------------------ A producers
        const int g = lane & ((1 << a.rlog) - 1);
        uint32_t used[3] = {0, 0, 0}, mw[3] = {0, 0, 0};
        uint32_t ctr = 0;
        bool failed = false;
        TileMeta m_next;
        unsigned q_next = 0;
        if (t_begin < t_end) {
            m_next = a.meta[t_begin];
            if (m_next.begin + tid < m_next.end) q_next = (unsigned)s.pairs[m_next.begin + tid];
        }
        for (int64_t tile = t_begin; tile < t_end && !failed; ++tile) {
            const TileMeta m = m_next;
            const bool active = m.begin + tid < m.end;
            const unsigned iq = q_next;
            if (tile + 1 < t_end) {
                m_next = a.meta[tile + 1];
                q_next = 0;
            }
            if constexpr (AG) {
                // ---- gathered A: copy this row's precomputed split phases chunk by chunk.
                // Inactive rows copy the row of q = 0 (finite values; their results are unread).
                const uint8_t *arow = a.arows + (size_t)(active ? iq : 0u) * a.arow_bytes;
                for (int g0 = 0; g0 < m.nsel && !failed; g0 += a.nbg) {
                    int pend = -1;                  // stage whose copies are in flight
                    for (int ch = 0; ch < NCH; ++ch) {
                        const int st = ctr % NSA;
                        if (used[st] > mw[st]) {
                            if (!tc::mbar_wait_bounded(&mma_done[st], mw[st] & 1, kWaitTimeoutNs)) failed = true;
                            ++mw[st];
                        }
                        if (failed || *sfail) {
                            failed = true;
                            break;
                        }
                        uint8_t *dst = sA + (size_t)st * 4 * A_OP + ((tid >> 3) * 4) * 128 + (tid & 7) * 16;
                        const uint8_t *src = arow + ch * 64;
#pragma unroll
                        for (int arr = 0; arr < 4; ++arr)
#pragma unroll
                            for (int kb = 0; kb < 4; ++kb)
                                cp_async16(dst + arr * A_OP + kb * 128, src + arr * a.arr_bytes + kb * 16);
                        cp_async_commit();
                        if (pend >= 0) {
                            // the previous chunk has landed: make it visible to the tensor core
                            cp_async_wait<1>();
                            tc::fence_proxy_async_smem();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&a_full[pend]);
                        }
                        pend = st;
                        ++used[st];
                        ++ctr;
                        if (ch == 0 && g0 == 0 && tile + 1 < t_end)
                            q_next = (m_next.begin + tid < m_next.end) ? (unsigned)s.pairs[m_next.begin + tid] : 0u;
                    }
                    cp_async_wait<0>();
                    if (pend >= 0 && !failed) {
                        tc::fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&a_full[pend]);
                    }
                }
                continue;
            }
            int a1 = 0, a2 = 0, a3 = 0;
            if (active) {
                const unsigned q3 = iq % n3, qt = iq / n3, q2 = qt % n2, q1 = qt / n2;
                a1 = (int)(q1 * (unsigned)s.g.s1 % (unsigned)L);
                a2 = (int)(q2 * (unsigned)s.g.s2 % (unsigned)L);
                a3 = (int)(q3 * (unsigned)s.g.s3 % (unsigned)L);
            }
            for (int g0 = 0; g0 < m.nsel && !failed; g0 += a.nbg) {
                // Reduced phase-index tables of this q: C3[n3+R] = n3 a3 mod L and
                // B12[(n1+R) D + n2+R] = (n1 a1 + n2 a2) mod L; an R_p index is B12 + C3 < 2L.
                int C3[D], B12[D * D];
                {
                    int B1[D], B2[D];
                    B1[0] = pmod(-RC * a1, L);
                    B2[0] = pmod(-RC * a2, L);
                    C3[0] = pmod(-RC * a3, L);
#pragma unroll
                    for (int j = 1; j < D; ++j) {
                        const int t1 = B1[j - 1] + a1, t2 = B2[j - 1] + a2, t3 = C3[j - 1] + a3;
                        B1[j] = t1 >= L ? t1 - L : t1;
                        B2[j] = t2 >= L ? t2 - L : t2;
                        C3[j] = t3 >= L ? t3 - L : t3;
                    }
#pragma unroll
                    for (int i1 = 0; i1 < D; ++i1)
#pragma unroll
                        for (int i2 = 0; i2 < D; ++i2) {
                            const int t = B1[i1] + B2[i2];
                            B12[i1 * D + i2] = t >= L ? t - L : t;
                        }
                }
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    const int st = ctr % NSA;
                    if (used[st] > mw[st]) {
                        if (!tc::mbar_wait_bounded(&mma_done[st], mw[st] & 1, kWaitTimeoutNs)) failed = true;
                        ++mw[st];
                    }
                    if (failed || *sfail) {
                        failed = true;
                        break;
                    }
                    tc::tc_fence_after();   // the stage's previous MMAs have completed
                    // The tables are re-defined (empty asm) at every chunk so that the compiler
                    // forms each chunk's indices inside the chunk instead of hoisting all of them.
#pragma unroll
                    for (int j = 0; j < D; ++j) asm volatile("" : "+r"(C3[j]));
#pragma unroll
                    for (int j = 0; j < D * D; ++j) asm volatile("" : "+r"(B12[j]));
                    // ---- A: phases of this thread's q for R_p = ch*KC .. ch*KC+KC-1.  Every index
                    // is independent (compile-time (i12, i3)); K beyond nRp reads entry 0, which
                    // meets zero B rows; rows of inactive threads are never read back.
                    const uint32_t aT = tmem_a + ((uint32_t)(warp * 32) << 16) + (uint32_t)(st * 4 * A_COLS);
#pragma unroll
                    for (int kb = 0; kb < 4; ++kb) {
                        uint32_t e[EPV][TW];
#pragma unroll
                        for (int j = 0; j < EPV; ++j) {
                            const int k = ch * KC + kb * EPV + j;
                            const int kk = k < NRP ? k : 0;
                            const int idx = k < NRP ? B12[kk / D] + C3[kk % D] : 0;
                            const uint32_t *src = sT + (((idx << a.rlog) | g) * TW);
                            if constexpr (TW == 4) {
                                const uint4 v4 = *reinterpret_cast<const uint4 *>(src);
                                e[j][0] = v4.x;
                                e[j][1] = v4.y;
                                e[j][2] = v4.z;
                                e[j][3] = v4.w;
                            } else {
                                const uint2 v2 = *reinterpret_cast<const uint2 *>(src);
                                e[j][0] = v2.x;
                                e[j][1] = v2.y;
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
                        for (int arr = 0; arr < 4; ++arr) tc::tmem_st4(aT + (uint32_t)(arr * A_COLS + kb * 4), v[arr]);
                        asm volatile("" ::: "memory");   // keep one 16-byte row block in flight
                    }
                    tc::tmem_wait_st();
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&a_full[st]);
                    ++used[st];
                    ++ctr;
                    if (ch == 0 && g0 == 0 && tile + 1 < t_end)
                        q_next = (m_next.begin + tid < m_next.end) ? (unsigned)s.pairs[m_next.begin + tid] : 0u;
                }
            }
        }
        for (int st = 0; st < NSA; ++st)
            while (used[st] > mw[st]) {
                if (!tc::mbar_wait_bounded(&mma_done[st], mw[st] & 1, kWaitTimeoutNs)) {
                    failed = true;
                    break;
                }
                ++mw[st];
            }
        if (failed) *sfail = 1;
    } else {
        // ------------------------------------------------------------ epilogue
        const int et = tid - 128;                  // row of the tile (TMEM lane)
        const int ew = warp - 4;                   // lane quarter
        const uint32_t tmem_row = tmem + ((uint32_t)(ew * 32) << 16);
        uint32_t fph[2] = {0, 0};
        uint32_t gctr = 0;
        bool failed = false;
        TileMeta m_next;
        unsigned q_next = 0;
        if (t_begin < t_end) {
            m_next = a.meta[t_begin];
            if (m_next.begin + et < m_next.end) q_next = (unsigned)s.pairs[m_next.begin + et];
        }
        for (int64_t tile = t_begin; tile < t_end && !failed; ++tile) {
            const TileMeta m = m_next;
            const int pair = m.begin + et;
            const bool active = pair < m.end;
            const unsigned iq = active ? q_next : 0u;
            if (tile + 1 < t_end) m_next = a.meta[tile + 1];
            unsigned ikq = 0;
            {
                const unsigned q3 = iq % n3, qt = iq / n3, q2 = qt % n2, q1 = qt / n2;
                const unsigned k3 = (unsigned)m.ik % n3, kt = (unsigned)m.ik / n3, k2 = kt % n2, k1 = kt / n2;
                unsigned b1 = q1 + k1, b2 = q2 + k2, b3 = q3 + k3;
                if (b1 >= n1) b1 -= n1;
                if (b2 >= n2) b2 -= n2;
                if (b3 >= n3) b3 -= n3;
                ikq = (b1 * n2 + b2) * n3 + b3;
            }
            // epilogue operands of this pair, fetched while the MMAs of this tile run
            float2 Vr[PRE ? W * W : 1], ur[PRE ? NM * NM : 1];
            float wq[NM], nq[NM], emr[W], fmr[W];
            const float2 *Vq = s.V32 + (size_t)ikq * W * W;
            const float2 *uq = s.u32 + (size_t)iq * NM * NM;
            if constexpr (PRE) {
#pragma unroll
                for (int x = 0; x < W * W; ++x) Vr[x] = __ldg(Vq + x);
#pragma unroll
                for (int x = 0; x < NM * NM; ++x) ur[x] = __ldg(uq + x);
            } else {
                tc::prefetch_l1(Vq);
                tc::prefetch_l1(uq);
            }
#pragma unroll
            for (int nu = 0; nu < NM; ++nu) {
                wq[nu] = __ldg(a.hw32 + (size_t)iq * NM + nu);
                nq[nu] = __ldg(a.n32 + (size_t)iq * NM + nu);
            }
#pragma unroll
            for (int mm = 0; mm < W; ++mm) {
                emr[mm] = __ldg(a.erel32 + (size_t)ikq * W + mm);
                fmr[mm] = __ldg(a.f32 + (size_t)ikq * W + mm);
            }
            int lokq = 0, nwkq = 0;
            int64_t goffp = 0;
            if constexpr (GAM) {
                if (active) {
                    lokq = __ldg(s.win_lo + ikq);
                    nwkq = __ldg(s.win_n + ikq);
                    goffp = s.goff[pair];
                }
            }
            if (tile + 1 < t_end)
                q_next = (m_next.begin + et < m_next.end) ? (unsigned)s.pairs[m_next.begin + et] : 0u;
            for (int g0 = 0; g0 < m.nsel && !failed; g0 += a.nbg) {
                const int nb = min(a.nbg, m.nsel - g0);
                const int ncp = nb * NMWP;
                const int ab = gctr & 1;
                if (!tc::mbar_wait_bounded(&acc_full[ab], fph[ab], kWaitTimeoutNs)) failed = true;
                fph[ab] ^= 1;
                ++gctr;
                if (failed || *sfail) {
                    failed = true;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t arow = tmem_row + (uint32_t)ab * acc_cols;
                for (int b = 0; b < nb; ++b) {
                    float gr[NMWP], gi[NMWP];
#pragma unroll
                    for (int blk = 0; blk < NMWP / 16; ++blk) {
                        float t0[16], t1[16];
                        const uint32_t c0 = arow + (uint32_t)(b * NMWP + blk * 16);
                        tc::tmem_ld16(c0, t0);
                        tc::tmem_ld16(c0 + 2 * ncp, t1);
#pragma unroll
                        for (int x = 0; x < 16; ++x) gr[blk * 16 + x] = t0[x] + t1[x];
                        tc::tmem_ld16(c0 + ncp, t0);
                        tc::tmem_ld16(c0 + 3 * ncp, t1);
#pragma unroll
                        for (int x = 0; x < 16; ++x) gi[blk * 16 + x] = t0[x] + t1[x];
                    }
                    tc::tmem_wait_ld();
                    if (b == nb - 1) {
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&acc_empty[ab]);   // buffer free for the MMAs
                    }
                    float rate = 0.f;
                    if (active) {
                        const float en = a.erel32[(size_t)m.ik * W + m.lo + g0 + b];
#pragma unroll
                        for (int mm = 0; mm < W; ++mm) {
                            float2 h[NM];
#pragma unroll
                            for (int mu = 0; mu < NM; ++mu) {
                                h[mu] = make_float2(0.f, 0.f);
#pragma unroll
                                for (int i = 0; i < W; ++i) {
                                    const float2 vv = PRE ? Vr[(i * W + mm) % (PRE ? W * W : 1)] : __ldg(Vq + i * W + mm);
                                    h[mu] = cfmacf(vv, make_float2(gr[mu * W + i], gi[mu * W + i]), h[mu]);
                                }
                            }
                            const float em = emr[mm];
                            const float fm = fmr[mm];
                            float gm = 0.f;      // Gamma capture: sum over modes
#pragma unroll
                            for (int nu = 0; nu < NM; ++nu) {
                                const float w = wq[nu];
                                float2 gv = make_float2(0.f, 0.f);
#pragma unroll
                                for (int mu = 0; mu < NM; ++mu) {
                                    const float2 uv = PRE ? ur[(mu * NM + nu) % (PRE ? NM * NM : 1)] : __ldg(uq + mu * NM + nu);
                                    gv = cfmaf(h[mu], uv, gv);
                                }
                                const float g2 = gv.x * gv.x + gv.y * gv.y;
                                if (s.g2out) {
                                    s.g2out[(((s.g2_base + pair) * m.nsel + g0 + b) * NM + nu) * W + mm] =
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
                                if constexpr (GAM) gm = fmaf(g2, tt, gm);
                            }
                            if constexpr (GAM) {
                                if (mm >= lokq && mm < lokq + nwkq)
                                    s.gam32[goffp + (int64_t)(g0 + b) * nwkq + (mm - lokq)] = gm * a.scale_inv2;
                            }
                        }
                        if (s.pair_w) rate *= (float)s.pair_w[pair];   // importance-sampling weight
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) rate += __shfl_down_sync(0xffffffffu, rate, o);
                    if (lane == 0) wred[ew * epc::kMaxW + g0 + b] = rate * a.scale_inv2;
                }
            }
            epilogue_sync();
            if (!failed && et < m.nsel)
                s.tile_part[tile * epc::kMaxW + et] =
                    ((double)wred[et] + (double)wred[epc::kMaxW + et]) +
                    ((double)wred[2 * epc::kMaxW + et] + (double)wred[3 * epc::kMaxW + et]);
            epilogue_sync();
        }
        if (failed) *sfail = 1;
    }
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0 && *sfail) atomicAdd(a.err, 1);
    if (warp == 0) tc::tmem_dealloc(tmem, a.tmem_cols);
}

template <class Op>
const uint32_t *phase_table(epwi_ctx *c, int *rlog_out) {
    const int TW = Op::kTF32 ? 4 : 2;
    // replicate the table (copy g serves lanes with lane % R == g) while it stays <= 16 KB;
    // R = 16 (8-byte entries) or 8 (16-byte entries) makes the lookups bank-conflict free
    int rlog = Op::kTF32 ? 3 : 4;
    while (rlog > 0 && (size_t)2 * c->L * (1 << rlog) * TW * 4 > 16384) --rlog;
    const int key = (c->L * 8 + c->opt.precision) * 8 + rlog;
    if (c->tc_ptab_key != key) {
        c->tc_ptab.ensure(sizeof(uint32_t) * 2 * c->L * TW * (1 << rlog));
        k_phase_split<Op><<<(2 * c->L + 127) / 128, 128, 0, c->stream>>>(c->L, rlog, c->ph64.as<double2>(),
                                                                        c->tc_ptab.as<uint32_t>());
        EPWI_CHECK_LAUNCH();
        c->tc_ptab_key = key;
    }
    *rlog_out = rlog;
    return c->tc_ptab.as<uint32_t>();
}

// Gathered-A mode: split phase rows of every grid point (built once per grid and precision).
template <class Op, int RC>
const uint8_t *phase_rows(epwi_ctx *c, int nchunk, int rlog, const uint32_t *ptab) {
    const int kpad = nchunk * (64 / Op::kBytes);
    const int64_t key = ((((int64_t)c->nk * 4096 + c->L) * 8 + c->opt.precision) * 64 + kpad) * 8 + rlog;
    if (c->tc_arows_key != key) {
        c->tc_arows.ensure((size_t)c->nk * 4 * kpad * 2);
        const int64_t nt = c->nk * (kpad / 8);
        k_phase_rows<RC><<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(
            c->nk, make_grid_info(c), kpad, rlog, ptab, c->tc_arows.as<uint8_t>());
        EPWI_CHECK_LAUNCH();
        c->tc_arows_key = key;
    }
    return c->tc_arows.as<uint8_t>();
}

template <class Op, int W, int NM, int RC, bool AG, bool GAM = false>
void launch_tc(epwi_ctx *c, const ScatterArgs &sa, int64_t ntiles) {
    constexpr int NMWP = (NM * W + 15) / 16 * 16;
    constexpr int TW = Op::kTF32 ? 4 : 2;
    constexpr int ES = Op::kBytes;
    TcArgs a;
    a.s = sa;
    c->tc_meta.ensure(sizeof(TileMeta) * (ntiles + 1));
    a.meta = c->tc_meta.as<TileMeta>();
    if (ntiles > 0) {
        k_tile_meta<<<(unsigned)((ntiles + 255) / 256), 256, 0, c->stream>>>(
            ntiles, sa.tiles, sa.kpts, sa.win_lo, sa.win_n, sa.kp_state, sa.s_base, sa.ovr_lo, sa.ovr_nsel,
            c->tc_meta.as<TileMeta>());
        EPWI_CHECK_LAUNCH();
    }
    a.img = static_cast<const uint8_t *>(sa.ghat_raw);
    a.ns = sa.nstates_chunk;
    a.ptab = phase_table<Op>(c, &a.rlog);
    a.erel32 = c->tc_erel.as<float>();
    a.f32 = c->tc_f32.as<float>();
    a.n32 = c->tc_n32.as<float>();
    a.hw32 = c->tc_hw32.as<float>();
    const int e = (Op::kFmt == 0 && !Op::kTF32) ? c->tc_scale_exp : 0;
    a.scale_inv2 = std::ldexp(1.0f, -2 * e);
    a.ceta32 = (float)sa.ceta;
    a.inv_eta32 = (float)(1.0 / sa.eta);
    a.cube_r = tc_rp_r(c);
    a.nchunk = (tc_rp_count(c) + 64 / ES - 1) / (64 / ES);
    a.nbg = std::max(1, 48 / NMWP);   // 4 ncp <= 192: two accumulators + A stages fit 512 columns
    a.ncp_max = std::min(sa.nsel_max, a.nbg) * NMWP;
    // TMEM: two accumulators of 4 ncp_max columns, then (A generated in-kernel) NSA A stages
    // of 4 operands x 16 columns; gathered A lives in shared memory instead
    a.acc_cols = (uint32_t)((4 * a.ncp_max + 15) / 16 * 16);
    a.a_col0 = 2 * a.acc_cols;
    a.nsa = AG ? 3 : ((a.a_col0 + 3 * 64 <= 512) ? 3 : 2);
    uint32_t cols = 32;
    while (cols < a.a_col0 + (AG ? 0u : (uint32_t)(a.nsa * 4 * 16))) cols <<= 1;
    EPWI_REQUIRE(cols <= 512, EPWI_EUNSUPPORTED, "tensor-core kernel needs more than 512 TMEM columns");
    a.tmem_cols = cols;
    a.ntiles = ntiles;
    c->tc_err.ensure(sizeof(int) * 4);
    EPWI_CUDA(cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream));
    a.err = c->tc_err.as<int>();
    const int twords = AG ? 0 : 2 * c->L * (1 << a.rlog) * TW;
    const size_t a_stage = AG ? (size_t)4 * 128 * 64 : 0;          // gathered A, per stage
    const size_t fixed = sizeof(uint32_t) * ((twords + 1) & ~1) + 13 * 8 + 16 + 4 * epc::kMaxW * 4 + 64;
    const size_t bres_bytes = (size_t)a.nchunk * 8 * a.ncp_max * 64;
    const size_t cap = AG ? 220 * 1024 : 200 * 1024;
    a.bres = (fixed + bres_bytes + 2 * a_stage <= cap) ? 1 : 0;
    if (!a.bres) a.nsa = 2;   // streaming B uses the A stage index as its slot index
    else if (AG && fixed + bres_bytes + 3 * a_stage > cap) a.nsa = 2;
    size_t smem = fixed + (a.bres ? bres_bytes : 2 * 8 * (size_t)a.ncp_max * 64) + a.nsa * a_stage;
    a.arows = nullptr;
    a.arow_bytes = 0;
    a.arr_bytes = 0;
    if constexpr (AG) {
        a.arows = phase_rows<Op, RC>(c, a.nchunk, a.rlog, a.ptab);
        a.arr_bytes = a.nchunk * 64;
        a.arow_bytes = 4 * (int64_t)a.arr_bytes;
    }
    auto kern = k_scatter_tc<Op, W, NM, RC, AG, GAM>;
    int nsm = 0;
    EPWI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    EPWI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    // keep (resident CTAs per SM) x (TMEM columns) <= 512 so that tcgen05.alloc never waits
    int per_sm = 0;
    for (;;) {
        EPWI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        EPWI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 288, smem));
        EPWI_REQUIRE(per_sm >= 1, EPWI_EUNSUPPORTED, "tensor-core kernel does not fit on an SM");
        if ((uint32_t)per_sm * cols <= 512) break;
        smem += 8 * 1024;
    }
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)per_sm * nsm);
    if (grid > 0) {
        kern<<<(unsigned)grid, 288, smem, c->stream>>>(a);
        EPWI_CHECK_LAUNCH();
    }
    c->tc_blocks_per_sm = per_sm;
    c->stats_tc_grid = grid;
    c->stats.tc_grid = grid;
    c->stats.tc_ctas_per_sm = per_sm;
    c->stats.sm_count = nsm;
    {
        cudaFuncAttributes fa;
        EPWI_CUDA(cudaFuncGetAttributes(&fa, kern));
        size_t avail = 0;
        if (cudaOccupancyAvailableDynamicSMemPerBlock(&avail, kern, 1, 288) != cudaSuccess) {
            (void)cudaGetLastError();
            avail = 0;
        }
        c->stats.tc_regs = fa.numRegs;
        c->stats.tc_smem = (int64_t)smem;
        c->stats.tc_smem_avail2 = (int64_t)avail;
    }
}

// A generated per tile into TMEM (default), or, when the context asks for it, gathered from
// precomputed split phase rows (16-bit types, rows of the whole grid <= 16 GiB).  On the
// 48^3 Al-like benchmark the gathered mode is slower (583 vs 424 ms per step): the kernel is
// bound by the instruction issue of all roles together, and the gathers add L2 traffic and
// latency in front of every MMA.
template <class Op, int W, int NM, int RC>
void launch_any(epwi_ctx *c, const ScatterArgs &sa, int64_t nt) {
    constexpr int D = 2 * RC + 1;
    const int64_t kpad = ((D * D * D + 64 / Op::kBytes - 1) / (64 / Op::kBytes)) * (64 / Op::kBytes);
    if (sa.gam32) {                          // Gamma capture of the iterative BTE
        launch_tc<Op, W, NM, RC, false, true>(c, sa, nt);
        return;
    }
    if constexpr (!Op::kTF32) {
        if (c->tc_gather && (int64_t)c->nk * 4 * kpad * 2 <= (int64_t(16) << 30)) {
            launch_tc<Op, W, NM, RC, true>(c, sa, nt);
            return;
        }
    }
    launch_tc<Op, W, NM, RC, false>(c, sa, nt);
}

template <class Op>
void dispatch_tc(epwi_ctx *c, const ScatterArgs &sa, int64_t nt) {
    const int W = c->nw, NM = c->nm, r = tc_rp_r(c);
    if (W == 1 && NM == 3 && r == 1) launch_any<Op, 1, 3, 1>(c, sa, nt);
    else if (W == 4 && NM == 3 && r == 1) launch_any<Op, 4, 3, 1>(c, sa, nt);
    else if (W == 4 && NM == 3 && r == 2) launch_any<Op, 4, 3, 2>(c, sa, nt);
    else if (W == 4 && NM == 3 && r == 3) launch_any<Op, 4, 3, 3>(c, sa, nt);
    else if (W == 8 && NM == 6 && r == 3) launch_any<Op, 8, 6, 3>(c, sa, nt);
    else if (W == 8 && NM == 6 && r == 1) launch_any<Op, 8, 6, 1>(c, sa, nt);
    else
        throw EpwiError{EPWI_EUNSUPPORTED,
                        "split-precision path built for (nw, modes, R_p cube half-width) in "
                        "{(1,3,1), (4,3,1), (4,3,2), (4,3,3), (8,6,1), (8,6,3)}"};
}

}  // namespace

size_t tc_state_bytes(const epwi_ctx *c) {
    const int es = c->opt.precision == EPWI_TF32X3 ? 4 : 2;
    const size_t kc = 64 / es;
    const size_t nchunk = (tc_rp_count(c) + kc - 1) / kc;
    const size_t nmwp = (size_t)(c->nm * c->nw + 15) / 16 * 16;
    return nchunk * 6 * nmwp * 64;
}

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

namespace {
template <class Op, int W, int NM, int KG>
void restage_tc_launch(epwi_ctx *c, const RestageArgs &ra) {
    uint8_t *img = static_cast<uint8_t *>(ra.ghat_raw);
    EPWI_CUDA(cudaMemsetAsync(img, 0, tc_state_bytes(c) * (size_t)ra.nstates_chunk, c->stream));
    const int e = (Op::kFmt == 0 && !Op::kTF32) ? c->tc_scale_exp : 0;
    dim3 grid((ra.nrow + 127) / 128, (unsigned)((ra.nkp + KG - 1) / KG));
    const size_t sm = sizeof(float2) * KG * ra.nRe;
    auto kern = k_restage_tc<Op, W, NM, KG>;
    if (sm > 48 * 1024)
        EPWI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    kern<<<grid, 128, sm, c->stream>>>(ra, img, ra.nstates_chunk, std::ldexp(1.0f, e));
    EPWI_CHECK_LAUNCH();
}

template <class Op>
void restage_dispatch(epwi_ctx *c, const RestageArgs &ra) {
    if (c->nw == 1 && c->nm == 3) restage_tc_launch<Op, 1, 3, 8>(c, ra);
    else if (c->nw == 4 && c->nm == 3) restage_tc_launch<Op, 4, 3, 8>(c, ra);
    else if (c->nw == 8 && c->nm == 6) restage_tc_launch<Op, 8, 6, 4>(c, ra);
    else throw EpwiError{EPWI_EUNSUPPORTED, "split-precision path built for (nw, modes) in {(1,3), (4,3), (8,6)}"};
}
}  // namespace

void tc_restage(epwi_ctx *c, const RestageArgs &ra) {
    switch (c->opt.precision) {
        case EPWI_FP16X3: restage_dispatch<OpF16>(c, ra); break;
        case EPWI_BF16X3: restage_dispatch<OpBF16>(c, ra); break;
        case EPWI_TF32X3: restage_dispatch<OpTF32>(c, ra); break;
        default: throw EpwiError{EPWI_EINVAL, "not a split-precision mode"};
    }
}

// A non-cube R_p set embedded in its bounding cube: gcube32[Re][cube point][mu][i][j] = the
// weighted g of the R_p vector at that point, or 0.
__global__ void k_cube_embed(int64_t n, int nRp, int D3, int rowlen, const int *__restrict__ cube,
                             const float2 *__restrict__ g32, float2 *__restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int e = (int)(idx % rowlen);
    const int64_t t = idx / rowlen;
    const int cf = (int)(t % D3);
    const int64_t re = t / D3;
    const int rp = cube[cf];
    out[idx] = rp < 0 ? make_float2(0.f, 0.f) : g32[((size_t)re * nRp + rp) * rowlen + e];
}

// The split-precision view of the R_p set (tc_rp_r, tc_rp_count): for a set that is not a full
// cube, its bounding cube (half-width <= 3) with the weighted g embedded (gcube32).
void tc_prepare(epwi_ctx *c) {
    if (c->rp_cube_r >= 0) return;
    EPWI_REQUIRE(!c->h_rp_cube.empty() && c->sf_r <= 3, EPWI_EUNSUPPORTED,
                 "split-precision path: the bounding cube of R_p must have half-width <= 3");
    if (c->gcube_ready) return;
    const int D = 2 * c->sf_r + 1, D3 = D * D * D, rowlen = c->nm * c->nw * c->nw;
    const int64_t n = (int64_t)c->nRe * D3 * rowlen;
    DevBuf cube;
    upload_ints(c, cube, c->h_rp_cube);
    c->gcube32.ensure(sizeof(float2) * n);
    k_cube_embed<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, c->nRp, D3, rowlen, cube.as<int>(),
                                                                    c->gw32.as<float2>(), c->gcube32.as<float2>());
    EPWI_CHECK_LAUNCH();
    EPWI_CUDA(cudaStreamSynchronize(c->stream));   // cube is freed on return
    c->gcube_ready = true;
}

void tc_scatter(epwi_ctx *c, const ScatterArgs &sa, int64_t ntiles) {
    EPWI_REQUIRE(c->rp_cube_r >= 0 || c->gcube_ready, EPWI_EUNSUPPORTED,
                 "split-precision path: R_p is neither a full cube nor embedded in one");
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
