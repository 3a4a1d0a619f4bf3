// Preprocessing on the device (Sec. III A): the energy window that selects the effective
// states {k_eff}, the effective-process sieve (energy-conservation surface), prefix scans
// and per-chunk pair lists.
//
// Sieve: a pair (k, q) is kept when some window band n at k, some band m at k+q, some
// kept mode nu and a sign s satisfy |(eps_nk + s hbar omega_qnu) - eps_m,k+q| <= c eta.
// Each candidate is first evaluated in FP32 with a rigorous bound delta on the rounding
// error; only candidates whose nearest |x| lies within delta of c eta are re-evaluated in
// FP64 in the oracle's rounding order, so every decision equals the FP64 one.
#include <cstdlib>

#include "epwi_internal.cuh"
#include "sieve.cuh"

namespace {

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of v across the block (blockDim.x multiple of 32, <= 1024).
__device__ int64_t block_excl_scan(int64_t v, int64_t *sm, int64_t &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) sm[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t s = lane < nw ? sm[lane] : 0;
        int64_t si = warp_incl_scan(s);
        if (lane < nw) sm[lane] = si - s;
        if (lane == nw - 1) sm[32] = si;
    }
    __syncthreads();
    int64_t r = inc - v + sm[wid];
    total = sm[32];
    __syncthreads();
    return r;
}

__global__ void k_scan_blocks(const int64_t *in, int64_t n, int64_t *bsum) {
    __shared__ int64_t sm[33];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock * kScanItems + threadIdx.x * kScanItems;
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    int64_t tot;
    block_excl_scan(s, sm, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_apply(const int64_t *in, int64_t n, const int64_t *boff, int64_t *out) {
    __shared__ int64_t sm[33];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock * kScanItems + threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int64_t tot;
    int64_t run = block_excl_scan(s, sm, tot) + boff[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = run;
}

// ------------------------------------------------------------------- window / k_eff
__global__ void k_window(int64_t nk, int W, const double *__restrict__ eps, double emin,
                         double emax, int *__restrict__ lo, int *__restrict__ cnt) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    int l = 0;
    while (l < W && !(eps[k * W + l] >= emin)) ++l;
    int h = l;
    while (h < W && eps[k * W + h] <= emax) ++h;
    lo[k] = l;
    cnt[k] = h - l;
}

// k-points that take part: a window state, and (with symmetry) the representative of its star
__device__ __forceinline__ bool window_kpoint(int64_t k, const int *cnt, const int *rep) {
    return cnt[k] > 0 && (!rep || rep[k] == (int)k);
}

__global__ void k_window_flags(int64_t nk, const int *__restrict__ cnt, const int *__restrict__ rep,
                               int64_t *__restrict__ flag) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nk) flag[k] = window_kpoint(k, cnt, rep) ? 1 : 0;
}

__global__ void k_compact_kpts(int64_t nk, const int64_t *__restrict__ pos,
                               const int *__restrict__ cnt, const int *__restrict__ rep, int *__restrict__ kpts,
                               int64_t *__restrict__ nsel) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk || !window_kpoint(k, cnt, rep)) return;
    kpts[pos[k]] = (int)k;
    nsel[pos[k]] = cnt[k];
}

__global__ void k_states(int64_t nkp, const int *__restrict__ kpts, const int *__restrict__ lo,
                         const int64_t *__restrict__ soff, int *__restrict__ st_k,
                         int *__restrict__ st_n) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nkp) return;
    const int k = kpts[p];
    for (int64_t s = soff[p]; s < soff[p + 1]; ++s) {
        st_k[s] = k;
        st_n[s] = lo[k] + (int)(s - soff[p]);
    }
}

// Candidate order shared by count and fill: the (i2, i3) plane index p runs over blocks of
// blockDim.x (one p per thread), and for each block i1 runs 0..N1-1.  k+q is updated
// incrementally (no division per candidate).
__device__ __forceinline__ int64_t plane_kq(const GridInfo &g, int ka2, int ka3, int64_t p) {
    const int i2 = (int)(p / g.n3), i3 = (int)(p - (int64_t)i2 * g.n3);
    int b2 = ka2 + i2, b3 = ka3 + i3;
    if (b2 >= g.n2) b2 -= g.n2;
    if (b3 >= g.n3) b3 -= g.n3;
    return (int64_t)b2 * g.n3 + b3;
}

// Counts the kept q of each k-point.  With mask != nullptr it also records every decision:
// the candidate of thread t at (plane block pb, i1) is bit t % 32 of word
// ((pb / blockDim.x) * N1 + i1) * (blockDim.x / 32) + t / 32 of the k-point's row.
template <int WT, int NMT>
__global__ void __launch_bounds__(256) k_sieve_count(SieveArgs a, int64_t nkp,
                                                     const int *__restrict__ kpts,
                                                     const int *__restrict__ lo,
                                                     const int *__restrict__ cnt,
                                                     int64_t *__restrict__ counts,
                                                     uint32_t *__restrict__ mask,
                                                     int64_t words_per_kp) {
    __shared__ double en[epc::kMaxW];
    __shared__ float en32[epc::kMaxW];
    __shared__ int64_t sm[33];
    const int ik = kpts[blockIdx.x];
    const int nsel = cnt[ik];
    load_window(a, ik, lo[ik], nsel, en, en32);
    int ka1, ka2, ka3;
    grid_coords(a.g, ik, ka1, ka2, ka3);
    const int64_t nplane = (int64_t)a.g.n2 * a.g.n3;
    const int wpb = blockDim.x >> 5;
    uint32_t *mrow = mask ? mask + (int64_t)blockIdx.x * words_per_kp : nullptr;
    int64_t c = 0;
    for (int64_t pb = 0; pb < nplane; pb += blockDim.x) {
        const int64_t p = pb + threadIdx.x;
        const bool inb = p < nplane;
        const int64_t kqp = inb ? plane_kq(a.g, ka2, ka3, p) : 0;
        int b1 = ka1;
        for (int i1 = 0; i1 < a.g.n1; ++i1) {
            const int64_t iq = (int64_t)i1 * nplane + p;
            const int64_t ikq = (int64_t)b1 * nplane + kqp;
            bool v;
            if constexpr (WT > 0) v = inb && pair_valid_t<WT, NMT>(a, nsel, en, en32, iq, ikq);
            else v = inb && pair_valid(a, nsel, en, en32, iq, ikq);
            c += v;
            if (mrow) {
                const uint32_t bits = __ballot_sync(0xffffffffu, v);
                if ((threadIdx.x & 31) == 0)
                    mrow[((pb / blockDim.x) * a.g.n1 + i1) * wpb + (threadIdx.x >> 5)] = bits;
            }
            if (++b1 == a.g.n1) b1 = 0;
        }
    }
    int64_t tot;
    block_excl_scan(c, sm, tot);
    if (threadIdx.x == 0) counts[blockIdx.x] = tot;
}

// Band energy ranges of each segment of kSegLen consecutive axis-1 points of every column.
__global__ void k_seg_ranges(int N1, int64_t nplane, int W, int nseg, const float *__restrict__ eps32,
                             float2 *__restrict__ segr) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nplane * nseg) return;
    const int64_t col = t / nseg;
    const int sg = (int)(t % nseg);
    const int b0 = sg * kSegLen, b1 = min(N1, b0 + kSegLen);
    for (int m = 0; m < W; ++m) {
        float lo = 3.0e38f, hi = -3.0e38f;
        for (int b = b0; b < b1; ++b) {
            const float e = eps32[((int64_t)b * nplane + col) * W + m];
            lo = fminf(lo, e);
            hi = fmaxf(hi, e);
        }
        segr[t * W + m] = make_float2(lo, hi);
    }
}

// k_sieve_count for compile-time W and N_m, with the same candidates, decisions and mask
// layout.  A candidate is decided from hm = hwmax(q) and the smallest distance
// dmin = min_{n,m} |e_n(k) - e_m(k+q)| (FP32, n over the window bands, m over all bands):
// - dmin > hm + c eta + delta: every (n, m, nu, s) has |(e_n + s w_nu) - e_m| > c eta, since
//   every kept mode has w_nu <= hm and delta bounds the FP32 rounding (reject);
// - hm <= c eta - 2 delta and dmin <= hm + c eta - delta: for the (n, m) of dmin, the mode of
//   energy hm with the sign opposite to d = e_n - e_m gives ||d| - hm| <= c eta - delta
//   (|d| >= hm) or <= hm <= c eta - 2 delta (|d| < hm), so the FP64 test holds (accept);
// - otherwise pair_valid_tail decides (FP32 per mode, FP64 where ambiguous).
// Every outcome therefore equals the FP64 evaluation of pair_valid.  The first two cases cover
// nearly every candidate when the phonon energies lie below c eta (the Gaussian's support is
// wider than the phonon band); the third runs inline for the few others.  The lanes of a warp
// take 32 consecutive (q2, q3) combinations of a plane block and 2-4 consecutive q1 per step,
// with the window's band count a compile-time constant (1 or 2, else a runtime loop); their
// ballots are the plane block's mask words, kept in shared memory ([warp][q1]) and written out
// in k_sieve_count's layout.  Indices are 32-bit (N_k < 2^31, checked).
//
// With FILL the same kernel writes the pair lists of k-points kp0 + blockIdx.x instead (used
// when the whole decision mask would not fit in memory): after each plane block the CTA scans
// the populations of its shared mask words in word order and writes the q of the set bits,
// which is the order of k_sieve_fill_mask.
//
// Segment pruning: the candidates of one k+q column whose axis-1 points lie in one segment of
// kSegLen (aligned in k+q space, so the same for every lane of a warp) are all rejected at once
// when no band's energy range over the segment comes within seglim (>= hwmax(q) + c eta +
// delta for every q, with a margin over FP32 rounding) of the window energies.  A warp whose
// lanes all reject a segment skips its iterations.
template <int WT, int NMT, bool FILL, int NS>
__device__ __forceinline__ int64_t sieve_fast_kp(const SieveArgs &a, int nsel, const double *en, const float *en32,
                                                 int ka1, int ka2, int ka3, uint32_t *words, int64_t *sm,
                                                 uint32_t *mrow, int64_t obase, int *pairs) {
    constexpr int kUnr = WT >= 8 ? 2 : 4;        // candidates per step (registers for their energies)
    constexpr int NSX = NS > 0 ? NS : WT;        // window bands held in registers
    constexpr int V4 = WT / 4;                   // 16-byte loads per k+q point
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float e[NSX];
#pragma unroll
    for (int n = 0; n < NSX; ++n) e[n] = n < nsel ? en32[n] : 3.0e38f;
    float elo = en32[0], ehi = en32[0];
    for (int n = 1; n < nsel; ++n) {
        elo = fminf(elo, en32[n]);
        ehi = fmaxf(ehi, en32[n]);
    }
    const float rej = a.ceta32 + a.delta32, acc = a.ceta32 - a.delta32;
    const float hm_fast = a.ceta32 - 2.f * a.delta32;
    const int N1 = a.g.n1, nplane = a.g.n2 * a.g.n3;
    const int rowv = nplane * V4;                // float4 per axis-1 row of the energy table
    const float4 *eps4 = reinterpret_cast<const float4 *>(a.eps32);
    uint32_t *mw = words + wid * N1;             // this warp's words of the plane block, by q1
    int64_t c = 0;
    for (int pb = 0, pbi = 0; pb < nplane; pb += blockDim.x, ++pbi) {
        const int p = pb + threadIdx.x;
        const bool inb = p < nplane;
        const int kqp = inb ? (int)plane_kq(a.g, ka2, ka3, p) : 0;
        const float *hq = a.hwmax32 + p;         // hwmax of q = (q1, p) at hq[q1 * nplane]
        const float4 *eq = eps4 + (size_t)kqp * V4;   // energies of (b1, kqp) at eq[b1 * rowv]
        for (int i1 = lane; i1 < N1; i1 += 32) mw[i1] = 0u;
        __syncwarp();
        int b1 = ka1;
        for (int i1 = 0; i1 < N1;) {
            // the segment of b1: iterations up to its end (or the wrap of b1 at N1); without the
            // table (nseg = 0) one segment covers the whole column
            const int sg = a.nseg ? b1 / kSegLen : 0;
            const int len = a.nseg ? min(min((sg + 1) * kSegLen, N1) - b1, N1 - i1) : N1 - i1;
            bool segok = inb && !a.nseg;
            if (inb && a.nseg) {
                const float2 *r = a.segr + ((int64_t)kqp * a.nseg + sg) * WT;
#pragma unroll
                for (int m = 0; m < WT; ++m) {
                    const float2 v = r[m];
                    segok |= (v.y >= elo - a.seglim) & (v.x <= ehi + a.seglim);
                }
            }
            if (!__any_sync(0xffffffffu, segok)) {
                i1 += len;
                b1 += len;
                if (b1 >= N1) b1 -= N1;
                continue;
            }
            for (int u = 0; u < len; u += kUnr) {
                // kUnr candidates (q1 = i1 .. i1 + kUnr - 1 of this segment): loads first
                float hm[kUnr];
                float4 em4[kUnr][V4];
#pragma unroll
                for (int j = 0; j < kUnr; ++j) {
                    int bj = b1 + j;
                    if (bj >= N1) bj -= N1;
                    hm[j] = -1.f;
                    if (segok && u + j < len) {
                        hm[j] = hq[(i1 + j) * nplane];
#pragma unroll
                        for (int v = 0; v < V4; ++v) em4[j][v] = eq[bj * rowv + v];
                    }
                }
                unsigned vbits = 0, amb = 0;
#pragma unroll
                for (int j = 0; j < kUnr; ++j) {
                    if (hm[j] >= 0.f) {
                        float d = 3.0e38f;
#pragma unroll
                        for (int n = 0; n < NSX; ++n) {
                            if (NS == 0 && n >= nsel) break;
#pragma unroll
                            for (int v = 0; v < V4; ++v) {
                                d = fminf(d, fabsf(e[n] - em4[j][v].x));
                                d = fminf(d, fabsf(e[n] - em4[j][v].y));
                                d = fminf(d, fabsf(e[n] - em4[j][v].z));
                                d = fminf(d, fabsf(e[n] - em4[j][v].w));
                            }
                        }
                        const bool near = d <= hm[j] + rej;
                        const bool sure = (hm[j] <= hm_fast) & (d <= hm[j] + acc);
                        vbits |= (near & sure ? 1u : 0u) << j;
                        amb |= (near & !sure ? 1u : 0u) << j;
                    }
                }
                // the rest: exact per-mode test (loads repeated: rare)
                while (amb) {
                    const int j = __ffs(amb) - 1;
                    amb &= amb - 1;
                    int bj = b1 + j;
                    if (bj >= N1) bj -= N1;
                    const int64_t ikq = (int64_t)bj * nplane + kqp;
                    const int64_t iqj = (int64_t)(i1 + j) * nplane + p;
                    float emj[WT];
                    load_kq_energies<WT>(a, ikq, emj);
                    if (pair_valid_tail<WT, NMT>(a, nsel, en, en32, iqj, ikq, a.hwmax32[iqj], emj)) vbits |= 1u << j;
                }
                // ballot j is word i1 + j: lane j keeps it and stores it
                uint32_t mine = 0u;
#pragma unroll
                for (int j = 0; j < kUnr; ++j) {
                    const uint32_t bits = __ballot_sync(0xffffffffu, (vbits >> j) & 1u);
                    if (lane == j) mine = bits;
                }
                if (lane < kUnr && u + lane < len) mw[i1 + lane] = mine;
                const int step = min(kUnr, len - u);
                i1 += step;
                b1 += step;
                if (b1 >= N1) b1 -= N1;
            }
        }
        __syncwarp();
        if constexpr (FILL) {
            __syncthreads();                     // every warp's words of this plane block
            const int nw = N1 * 8, per = (nw + blockDim.x - 1) / blockDim.x;
            const int w0 = threadIdx.x * per, w1 = min(nw, w0 + per);
            int pop = 0;
            for (int w = w0; w < w1; ++w) pop += __popc(words[(w & 7) * N1 + (w >> 3)]);
            int64_t tot;
            int64_t o = obase + block_excl_scan((int64_t)pop, sm, tot);
            for (int w = w0; w < w1; ++w) {
                uint32_t b = words[(w & 7) * N1 + (w >> 3)];
                const int q0 = (w >> 3) * nplane + pb + (w & 7) * 32;   // (i1, warp) of the word
                while (b) {
                    const int bit = __ffs(b) - 1;
                    b &= b - 1;
                    pairs[o++] = q0 + bit;
                }
            }
            obase += tot;
            __syncthreads();                     // the words are cleared next
        } else {
            for (int i1 = lane; i1 < N1; i1 += 32) {
                const uint32_t w = mw[i1];
                c += __popc(w);
                if (mrow) mrow[((int64_t)pbi * N1 + i1) * 8] = w;
            }
            __syncwarp();
        }
    }
    return c;
}

template <int WT, int NMT, bool FILL>
__global__ void __launch_bounds__(256, 3) k_sieve_count_fast(SieveArgs a, const int *__restrict__ kpts,
                                                          const int *__restrict__ lo,
                                                          const int *__restrict__ cnt,
                                                          int64_t *__restrict__ counts,
                                                          uint32_t *__restrict__ mask,
                                                          int64_t words_per_kp, int64_t kp0,
                                                          const int64_t *__restrict__ kp_pairs,
                                                          int *__restrict__ pairs) {
    __shared__ double en[epc::kMaxW];
    __shared__ float en32[epc::kMaxW];
    __shared__ int64_t sm[33];
    extern __shared__ uint32_t words[];          // [8][N1]: decisions of the current plane block
    const int64_t kp = FILL ? kp0 + blockIdx.x : blockIdx.x;
    const int ik = kpts[kp];
    const int nsel = cnt[ik];
    load_window(a, ik, lo[ik], nsel, en, en32);
    int ka1, ka2, ka3;
    grid_coords(a.g, ik, ka1, ka2, ka3);
    uint32_t *mrow = (mask && !FILL) ? mask + (int64_t)blockIdx.x * words_per_kp + (threadIdx.x >> 5) : nullptr;
    const int64_t obase = FILL ? kp_pairs[kp] - kp_pairs[kp0] : 0;   // first output position (FILL)
    int64_t c;
    switch (nsel) {                              // the window's band count (uniform over the block)
    case 1: c = sieve_fast_kp<WT, NMT, FILL, 1>(a, nsel, en, en32, ka1, ka2, ka3, words, sm, mrow, obase, pairs); break;
    case 2: c = sieve_fast_kp<WT, NMT, FILL, 2>(a, nsel, en, en32, ka1, ka2, ka3, words, sm, mrow, obase, pairs); break;
    default: c = sieve_fast_kp<WT, NMT, FILL, 0>(a, nsel, en, en32, ka1, ka2, ka3, words, sm, mrow, obase, pairs); break;
    }
    if constexpr (FILL) return;
    int64_t tot;
    block_excl_scan(c, sm, tot);
    if (threadIdx.x == 0) counts[blockIdx.x] = tot;
}

// Pair lists from the decision mask of k_sieve_count, in the same candidate order: each
// thread takes one mask word, the block scans the word populations in word order, every
// thread puts the q of its word's set bits (in bit order) at their places in a shared buffer,
// and the block copies the buffer out with consecutive threads on consecutive pairs.
__global__ void __launch_bounds__(256) k_sieve_fill_mask(GridInfo g, int64_t kp0,
                                                         const uint32_t *__restrict__ mask,
                                                         int64_t words_per_kp, int count_block,
                                                         const int64_t *__restrict__ kp_pairs,
                                                         int *__restrict__ pairs) {
    __shared__ int64_t sm[33];
    __shared__ int buf[256 * 32];
    const int64_t kp = kp0 + blockIdx.x;
    const uint32_t *mrow = mask + kp * words_per_kp;
    const int64_t nplane = (int64_t)g.n2 * g.n3;
    const int wpb = count_block >> 5;
    int *out = pairs + (kp_pairs[kp] - kp_pairs[kp0]);
    for (int64_t w0 = 0; w0 < words_per_kp; w0 += blockDim.x) {
        const int64_t w = w0 + threadIdx.x;
        uint32_t bits = w < words_per_kp ? mrow[w] : 0u;
        int64_t tot;
        int o = (int)block_excl_scan((int64_t)__popc(bits), sm, tot);
        if (bits) {
            const int64_t grp = w / wpb;                 // (plane block, i1) group
            const int64_t pbi = grp / g.n1, i1 = grp % g.n1;
            const int q0 = (int)(i1 * nplane + pbi * count_block + (w % wpb) * 32);
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                buf[o++] = q0 + b;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < (int)tot; i += blockDim.x) out[i] = buf[i];
        out += tot;
        __syncthreads();                                 // buf is refilled next
    }
}

// Writes the kept q of k-points kp0 + blockIdx.x in the candidate order of k_sieve_count.
__global__ void __launch_bounds__(256) k_sieve_fill(SieveArgs a, int64_t kp0,
                                                    const int *__restrict__ kpts,
                                                    const int *__restrict__ lo,
                                                    const int *__restrict__ cnt,
                                                    const int64_t *__restrict__ kp_pairs,
                                                    int *__restrict__ pairs) {
    __shared__ double en[epc::kMaxW];
    __shared__ float en32[epc::kMaxW];
    __shared__ int64_t sm[33];
    const int64_t kp = kp0 + blockIdx.x;
    const int ik = kpts[kp];
    const int nsel = cnt[ik];
    load_window(a, ik, lo[ik], nsel, en, en32);
    int ka1, ka2, ka3;
    grid_coords(a.g, ik, ka1, ka2, ka3);
    const int64_t nplane = (int64_t)a.g.n2 * a.g.n3;
    int64_t base = kp_pairs[kp] - kp_pairs[kp0];
    const int64_t end = kp_pairs[kp + 1] - kp_pairs[kp0];
    for (int64_t pb = 0; pb < nplane; pb += blockDim.x) {
        const int64_t p = pb + threadIdx.x;
        const bool inb = p < nplane;
        const int64_t kqp = inb ? plane_kq(a.g, ka2, ka3, p) : 0;
        int b1 = ka1;
        for (int i1 = 0; i1 < a.g.n1; ++i1) {
            const int64_t iq = (int64_t)i1 * nplane + p;
            const int64_t ikq = (int64_t)b1 * nplane + kqp;
            const int64_t v = inb ? (int64_t)pair_valid(a, nsel, en, en32, iq, ikq) : 0;
            int64_t tot;
            const int64_t off = block_excl_scan(v, sm, tot);
            if (v && base + off < end) pairs[base + off] = (int)iq;
            base += tot;
            if (++b1 == a.g.n1) b1 = 0;
        }
    }
}

}  // namespace

// The fast count / fill kernels keep one plane block's decisions (8 words per q1) in shared
// memory and use 32-bit candidate indices.
static bool sieve_fast_ok(const epwi_ctx *c) {
    return c->ng[0] <= 1024 && c->nk < (int64_t(1) << 31) - c->ng[1] * (int64_t)c->ng[2];
}

SieveArgs make_sieve_args(epwi_ctx *c) {
    SieveArgs a;
    a.g = make_grid_info(c);
    a.W = c->nw;
    a.Nm = c->nm;
    a.eps = c->eps.as<double>();
    a.eps32 = c->eps32.as<float>();
    a.hw = c->hw.as<double>();
    a.hw32 = c->hw32.as<float>();
    a.hwmax32 = c->hwmax32.as<float>();
    a.omega_min = c->opt.omega_min_eV;
    a.ceta = c->opt.sieve_c * c->eta;
    a.ceta32 = (float)a.ceta;
    // FP32 rounding of |e| <= E and of the two operations is < 2^-24 (3E + |w| + |x|) < 4e-7 E'
    a.delta32 = (float)(1e-6 + 4e-7 * (2.0 * c->eabs_max + 1.0));
    a.lim_extra = (float)(a.ceta + a.delta32 + 1e-5);
    // the table pays where a segment spans a small part of the zone (measured: 12% faster at
    // 96^3, 9% slower at 48^3); off below 64 points along axis 1
    a.segr = c->seg_ranges.as<float2>();
    a.nseg = c->ng[0] >= kSegMinGrid ? (c->ng[0] + kSegLen - 1) / kSegLen : 0;
    // >= hwmax(q) + lim_extra + 1e-4 (the prefilter's pad) for every q, plus 1e-4 for rounding
    a.seglim = (float)(c->hw_max + a.lim_extra + 2e-4);
    return a;
}

// The pruning table of the current grid (band ranges per column segment) and the largest mode
// energy; built once per eigs call.
static void seg_ranges(epwi_ctx *c) {
    if (c->seg_ready || c->ng[0] < kSegMinGrid) return;
    const int64_t nplane = (int64_t)c->ng[1] * c->ng[2];
    const int nseg = (c->ng[0] + kSegLen - 1) / kSegLen;
    c->seg_ranges.ensure(sizeof(float2) * nplane * nseg * c->nw);
    const int64_t nt = nplane * nseg;
    k_seg_ranges<<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(c->ng[0], nplane, c->nw, nseg,
                                                                      c->eps32.as<float>(), c->seg_ranges.as<float2>());
    EPWI_CHECK_LAUNCH();
    c->hw_max = std::max(0.0, device_reduce_minmax(c, c->hw.as<double>(), c->nk * c->nm, 1, 0, true));
    c->seg_ready = true;
}

void scan_exclusive_i64(epwi_ctx *c, const int64_t *in, int64_t *out, int64_t n, int64_t *total) {
    // out has n + 1 entries; out[n] = sum.  Recursive over block sums.
    const int64_t per = (int64_t)kScanBlock * kScanItems;
    const int64_t nb = (n + per - 1) / per;
    if (n == 0) {
        EPWI_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), c->stream));
        if (total) *total = 0;
        return;
    }
    DevBuf bs, bo;
    bs.ensure(sizeof(int64_t) * (nb + 1));
    bo.ensure(sizeof(int64_t) * (nb + 1));
    try {
        k_scan_blocks<<<(unsigned)nb, kScanBlock, 0, c->stream>>>(in, n, bs.as<int64_t>());
        EPWI_CHECK_LAUNCH();
        if (nb > 1) {
            scan_exclusive_i64(c, bs.as<int64_t>(), bo.as<int64_t>(), nb, nullptr);
        } else {
            EPWI_CUDA(cudaMemsetAsync(bo.p, 0, sizeof(int64_t), c->stream));
        }
        k_scan_apply<<<(unsigned)nb, kScanBlock, 0, c->stream>>>(in, n, bo.as<int64_t>(), out);
        EPWI_CHECK_LAUNCH();
        if (total) {
            EPWI_CUDA(cudaMemcpyAsync(total, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                      c->stream));
            EPWI_CUDA(cudaStreamSynchronize(c->stream));
        } else {
            EPWI_CUDA(cudaStreamSynchronize(c->stream));   // bs/bo are freed on return
        }
    } catch (...) {
        bs.release();
        bo.release();
        throw;
    }
    bs.release();
    bo.release();
}

void build_window(epwi_ctx *c, const int *rep) {
    const int64_t nk = c->nk;
    c->sym_used = false;
    c->win_lo.ensure(sizeof(int) * nk);
    c->win_n.ensure(sizeof(int) * nk);
    const unsigned nb = (unsigned)((nk + 255) / 256);
    k_window<<<nb, 256, 0, c->stream>>>(nk, c->nw, c->eps.as<double>(), c->emin, c->emax,
                                       c->win_lo.as<int>(), c->win_n.as<int>());
    EPWI_CHECK_LAUNCH();
    if (c->vel_state == 1) c->vel_state = 0;     // velocities of an earlier window
    window_lists(c, rep);
}

void window_lists(epwi_ctx *c, const int *rep) {
    const int64_t nk = c->nk;
    c->counts.ensure(sizeof(int64_t) * (nk + 1));
    c->scan_tmp.ensure(sizeof(int64_t) * (nk + 1));
    const unsigned nb = (unsigned)((nk + 255) / 256);
    k_window_flags<<<nb, 256, 0, c->stream>>>(nk, c->win_n.as<int>(), rep, c->counts.as<int64_t>());
    EPWI_CHECK_LAUNCH();
    int64_t nkp = 0;
    scan_exclusive_i64(c, c->counts.as<int64_t>(), c->scan_tmp.as<int64_t>(), nk, &nkp);
    c->nkp = nkp;
    c->kpts.ensure(sizeof(int) * (nkp + 1));
    c->kp_state.ensure(sizeof(int64_t) * (nkp + 1));
    // reuse counts as the per-kp band count
    k_compact_kpts<<<nb, 256, 0, c->stream>>>(nk, c->scan_tmp.as<int64_t>(), c->win_n.as<int>(), rep,
                                             c->kpts.as<int>(), c->counts.as<int64_t>());
    EPWI_CHECK_LAUNCH();
    int64_t nst = 0;
    scan_exclusive_i64(c, c->counts.as<int64_t>(), c->kp_state.as<int64_t>(), nkp, &nst);
    c->nstates = nst;
    c->st_k.ensure(sizeof(int) * (nst + 1));
    c->st_n.ensure(sizeof(int) * (nst + 1));
    c->inv_tau.ensure(sizeof(double) * (nst + 1));
    if (nkp > 0) {
        k_states<<<(unsigned)((nkp + 255) / 256), 256, 0, c->stream>>>(
            nkp, c->kpts.as<int>(), c->win_lo.as<int>(), c->kp_state.as<int64_t>(),
            c->st_k.as<int>(), c->st_n.as<int>());
        EPWI_CHECK_LAUNCH();
    }
}

void sieve_count(epwi_ctx *c) {
    const int64_t nkp = c->nkp;
    seg_ranges(c);
    c->counts.ensure(sizeof(int64_t) * (nkp + 1));
    c->kp_pairs.ensure(sizeof(int64_t) * (nkp + 1));
    SieveArgs a = make_sieve_args(c);
    // decision mask for the fill when it fits in 2 GiB (else the fill re-evaluates)
    const int64_t nplane = (int64_t)c->ng[1] * c->ng[2];
    const int64_t words = ((nplane + kSieveBlock - 1) / kSieveBlock) * c->ng[0] * (kSieveBlock / 32);
    // EPWI_SIEVE_MASK_MAX_BYTES (default 2 GiB) caps the mask; 0 forces the re-evaluating fill
    int64_t cap = int64_t(1) << 31;
    if (const char *env = std::getenv("EPWI_SIEVE_MASK_MAX_BYTES")) cap = std::strtoll(env, nullptr, 10);
    c->mask_words = (nkp > 0 && words * nkp * 4 <= cap) ? words : 0;
    if (c->mask_words) c->sieve_mask.ensure(sizeof(uint32_t) * words * nkp);
    if (nkp > 0) {
        uint32_t *mk = c->mask_words ? c->sieve_mask.as<uint32_t>() : nullptr;
        auto fast = (c->nw == 4 && c->nm == 3) ? k_sieve_count_fast<4, 3, false>
                    : (c->nw == 8 && c->nm == 6) ? k_sieve_count_fast<8, 6, false> : nullptr;
        if (fast && sieve_fast_ok(c)) {
            fast<<<(unsigned)nkp, kSieveBlock, sizeof(uint32_t) * 8 * (size_t)c->ng[0], c->stream>>>(
                a, c->kpts.as<int>(), c->win_lo.as<int>(), c->win_n.as<int>(), c->counts.as<int64_t>(), mk,
                c->mask_words, 0, nullptr, nullptr);
        } else {
            auto kern = (c->nw == 4 && c->nm == 3) ? k_sieve_count<4, 3> : k_sieve_count<0, 0>;
            kern<<<(unsigned)nkp, kSieveBlock, 0, c->stream>>>(
                a, nkp, c->kpts.as<int>(), c->win_lo.as<int>(), c->win_n.as<int>(), c->counts.as<int64_t>(), mk,
                c->mask_words);
        }
        EPWI_CHECK_LAUNCH();
    }
    int64_t np = 0;
    scan_exclusive_i64(c, c->counts.as<int64_t>(), c->kp_pairs.as<int64_t>(), nkp, &np);
    c->npairs = np;
    c->h_kp_pairs.resize(nkp + 1);
    EPWI_CUDA(cudaMemcpyAsync(c->h_kp_pairs.data(), c->kp_pairs.p, sizeof(int64_t) * (nkp + 1),
                              cudaMemcpyDeviceToHost, c->stream));
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
}

void sieve_fill_chunk(epwi_ctx *c, int64_t kp0, int64_t kp1, int *pairs) {
    if (kp1 <= kp0) return;
    if (c->mask_words) {
        k_sieve_fill_mask<<<(unsigned)(kp1 - kp0), 256, 0, c->stream>>>(
            make_grid_info(c), kp0, c->sieve_mask.as<uint32_t>(), c->mask_words, kSieveBlock,
            c->kp_pairs.as<int64_t>(), pairs);
        EPWI_CHECK_LAUNCH();
        return;
    }
    SieveArgs a = make_sieve_args(c);
    auto fast = (c->nw == 4 && c->nm == 3) ? k_sieve_count_fast<4, 3, true>
                : (c->nw == 8 && c->nm == 6) ? k_sieve_count_fast<8, 6, true> : nullptr;
    if (fast && sieve_fast_ok(c)) {
        fast<<<(unsigned)(kp1 - kp0), kSieveBlock, sizeof(uint32_t) * 8 * (size_t)c->ng[0], c->stream>>>(
            a, c->kpts.as<int>(), c->win_lo.as<int>(), c->win_n.as<int>(), nullptr, nullptr, 0, kp0,
            c->kp_pairs.as<int64_t>(), pairs);
        EPWI_CHECK_LAUNCH();
        return;
    }
    k_sieve_fill<<<(unsigned)(kp1 - kp0), 256, 0, c->stream>>>(
        a, kp0, c->kpts.as<int>(), c->win_lo.as<int>(), c->win_n.as<int>(),
        c->kp_pairs.as<int64_t>(), pairs);
    EPWI_CHECK_LAUNCH();
}
