// Learned q-proposal and importance-sampled SERTA rates.
//
// The paper sums the SERTA rate (Sec. II C, Eq. 10) over every sieved q.  Here a Monte Carlo
// estimate of that q sum is built instead: S grid points q_s are drawn per k from a proposal
// p(q) > 0, and sum_q t(q) is estimated by (1/S) sum_s t(q_s) / p(q_s).  Repeated draws are
// merged, so a distinct q drawn c times gets the weight c / (S p(q)).  The weighted pairs then
// go through the plain interpolation and SERTA kernels of the context's precision.  The
// estimate is unbiased for any p that is positive wherever t is.
//
// Two proposals are available.
//  * uniform: p = 1 / N_q.
//  * learned: the grid is divided into cells of s^3 points around every s-th grid point.  For
//    each window state (k, n) the network scores every cell centre and mode.  The cell
//    probability is P_n(c) = sum_nu e^{a yhat} / (the same sum over all cells), where a is
//    the std of the training targets.  Then p_n(q) = alpha / N_q + (1 - alpha) P_n(c(q)) / s^3.
//    The bands of one k share one draw from the band mixture (1/n_win) sum_n p_n.
//
// Training data are the terms t_nu(k, q, n) of Eq. 10 on the current (coarse) grid.  They
// cover every sieved pair plus uniformly drawn background pairs, and come from the FP64
// terms mode of the plain kernels.  The network regresses the normalised log(t + floor).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "mlp.cuh"
#include "scatter.cuh"
#include "sieve.cuh"

namespace {
using namespace mlp;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {     // SplitMix64 output function
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double u53(uint64_t h) {          // uniform in [0, 1)
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double centred(int i, int n) {   // i / n mapped to [-1/2, 1/2)
    const double f = (double)i / (double)n;
    return 2 * i < n ? f : f - 1.0;
}

// Network inputs of one sample: k and q coordinates (centred, doubled), (eps - mu) / 0.25 eV,
// n / W, nu / Nm.  Computed in FP64 and rounded once to FP32.
__device__ __forceinline__ void make_features(const GridInfo &g, int64_t ik, int64_t iq,
                                              double e_rel, int n, int nu, int W, int Nm,
                                              float *x) {
    int a1, a2, a3, b1, b2, b3;
    grid_coords(g, ik, a1, a2, a3);
    grid_coords(g, iq, b1, b2, b3);
    x[0] = (float)(2.0 * centred(a1, g.n1));
    x[1] = (float)(2.0 * centred(a2, g.n2));
    x[2] = (float)(2.0 * centred(a3, g.n3));
    x[3] = (float)(2.0 * centred(b1, g.n1));
    x[4] = (float)(2.0 * centred(b2, g.n2));
    x[5] = (float)(2.0 * centred(b3, g.n3));
    x[6] = (float)(e_rel / kEScale);
    x[7] = (float)((double)n / (double)W);
    x[8] = (float)((double)nu / (double)Nm);
}

// ------------------------------------------------------------------ training set
__global__ void k_train_set(int64_t npairs, const int *__restrict__ pair_kp,
                            const int *__restrict__ pairs, const int *__restrict__ kpts,
                            const int *__restrict__ win_lo, const int *__restrict__ win_n,
                            const int64_t *__restrict__ kp_pairs,
                            const int64_t *__restrict__ entry_off, const double *__restrict__ tout,
                            int tstride, const double *__restrict__ eps, double mu, GridInfo g,
                            int W, int Nm, float *__restrict__ X, double *__restrict__ T64,
                            int4 *__restrict__ ids) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const int kp = pair_kp[p];
    const int ik = kpts[kp];
    const int lo = win_lo[ik], ns = win_n[ik];
    const int iq = pairs[p];
    const int64_t base = entry_off[kp] + (p - kp_pairs[kp]) * ns * Nm;
    for (int np = 0; np < ns; ++np) {
        const double e_rel = eps[(int64_t)ik * W + lo + np] - mu;
        for (int nu = 0; nu < Nm; ++nu) {
            const int64_t e = base + (int64_t)np * Nm + nu;
            T64[e] = tout[(p * tstride + np) * Nm + nu];
            ids[e] = make_int4(ik, iq, lo + np, nu);
            make_features(g, ik, iq, e_rel, lo + np, nu, W, Nm, X + e * kIn);
        }
    }
}

// Y = log(t + floor), with per-block FP64 sums of Y and Y^2.
__global__ void __launch_bounds__(256) k_log_targets(int64_t n, const double *__restrict__ T64,
                                                     double floor_, float *__restrict__ Y,
                                                     double *__restrict__ part) {
    __shared__ double s1[256], s2[256];
    const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
    double y = 0;
    if (e < n) {
        y = log(T64[e] + floor_);
        Y[e] = (float)y;
    }
    s1[threadIdx.x] = y;
    s2[threadIdx.x] = y * y;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            s1[threadIdx.x] += s1[threadIdx.x + s];
            s2[threadIdx.x] += s2[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1[0];
        part[2 * blockIdx.x + 1] = s2[0];
    }
}

__global__ void k_normalise(int64_t n, float shift, float inv_scale, float *__restrict__ Y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) Y[e] = (Y[e] - shift) * inv_scale;
}

// ------------------------------------------------------------------ proposal
struct PropArgs {
    GridInfo g;
    int W, Nm, s;                 // s = cell stride
    int c2, c3;                   // cells per axis 2, 3
    int64_t ncell;
    const int *st_k, *st_n;
    const double *eps;
    double mu;
};

// Features of proposal rows r0 .. r0+n-1 of the chunk's states starting at global state s0;
// row = (state * ncell + cell) * Nm + nu.
__global__ void k_prop_features(PropArgs a, int64_t s0, int64_t r0, int64_t n,
                                float *__restrict__ X) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t r = r0 + j;
    const int nu = (int)(r % a.Nm);
    const int64_t sc = r / a.Nm;
    const int64_t cell = sc % a.ncell;
    const int64_t st = s0 + sc / a.ncell;
    const int ik = a.st_k[st], bn = a.st_n[st];
    const int c3 = (int)(cell % a.c3), c2 = (int)((cell / a.c3) % a.c2), c1 = (int)(cell / ((int64_t)a.c3 * a.c2));
    const int64_t iq = grid_index(a.g, a.s * c1, a.s * c2, a.s * c3);
    make_features(a.g, ik, iq, a.eps[(int64_t)ik * a.W + bn] - a.mu, bn, nu, a.W, a.Nm, X + j * kIn);
}

// logit[(row0 / Nm) + j] = log sum_nu exp(scale * yhat) over the Nm rows of each (state, cell).
__global__ void k_prop_lse(int64_t ngroups, int Nm, float scale, const float *__restrict__ yhat,
                           float *__restrict__ logit) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ngroups) return;
    float m = -INFINITY;
    for (int nu = 0; nu < Nm; ++nu) m = fmaxf(m, scale * yhat[j * Nm + nu]);
    float s = 0.f;
    for (int nu = 0; nu < Nm; ++nu) s += expf(scale * yhat[j * Nm + nu] - m);
    logit[j] = m + logf(s);
}

// Per state (one block): cdf[c] = sum_{c' <= c} exp(logit[c'] - max) in FP64; tot = cdf[last].
__global__ void __launch_bounds__(1024) k_state_cdf(int64_t ncell, const float *__restrict__ logit,
                                                    double *__restrict__ cdf,
                                                    double *__restrict__ tot) {
    __shared__ float smax[32];
    __shared__ double ssum[32];
    __shared__ double carry;
    const int64_t st = blockIdx.x;
    const float *lg = logit + st * ncell;
    double *cd = cdf + st * ncell;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float m = -INFINITY;
    for (int64_t c = threadIdx.x; c < ncell; c += 1024) m = fmaxf(m, lg[c]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) smax[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mm = smax[0];
        for (int w = 1; w < 32; ++w) mm = fmaxf(mm, smax[w]);
        smax[0] = mm;
        carry = 0.0;
    }
    __syncthreads();
    const float mx = smax[0];
    for (int64_t c0 = 0; c0 < ncell; c0 += 1024) {
        const int64_t c = c0 + threadIdx.x;
        const double v = c < ncell ? exp((double)lg[c] - (double)mx) : 0.0;
        double x = v;                                   // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ssum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            double w = ssum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const double y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            ssum[lane] = w;                             // inclusive over warps
        }
        __syncthreads();
        const double before = carry + (wid > 0 ? ssum[wid - 1] : 0.0);
        if (c < ncell) cd[c] = before + x;
        __syncthreads();
        if (threadIdx.x == 0) carry += ssum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) tot[st] = carry;
}

struct SampleArgs {
    GridInfo g;
    int s, c2, c3;
    int64_t ncell, nq;
    int64_t S;                     // draws per k-point
    double alpha;
    uint64_t seed;
    const int *kpts;               // chunk k-points
    const int64_t *kp_state;       // global state offsets of the chunk k-points
    int64_t s_base;                // first state of the chunk
    const int *win_lo, *win_n;
    const double *cdf, *tot;       // per chunk state (learned proposal only)
    int *counts;                   // [kp_local][nq]
    SieveArgs sv;                  // drawn q failing the sieve have t = 0 and are dropped
};

__device__ __forceinline__ uint64_t draw_key(uint64_t seed, int ik, int64_t s) {
    return mix64(mix64(seed ^ (0x9e3779b97f4a7c15ull * (uint64_t)(ik + 1))) +
                 0xd1b54a32d192ed03ull * (uint64_t)(s + 1));
}

__global__ void k_is_sample(SampleArgs a, int64_t nkpc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nkpc * a.S) return;
    const int64_t kpl = t / a.S, s = t % a.S;
    const int ik = a.kpts[kpl];
    const uint64_t key = draw_key(a.seed, ik, s);
    const double u0 = u53(mix64(key + 1)), u1 = u53(mix64(key + 2)), u2 = u53(mix64(key + 3)),
                 u3 = u53(mix64(key + 4));
    int64_t iq;
    if (u1 < a.alpha || !a.cdf) {
        iq = min((int64_t)(u2 * (double)a.nq), a.nq - 1);
    } else {
        const int nwin = a.win_n[ik];
        const int b = min((int)(u0 * nwin), nwin - 1);
        const int64_t st = a.kp_state[kpl] - a.s_base + b;
        const double *cd = a.cdf + st * a.ncell;
        const double target = u2 * a.tot[st];
        int64_t lo = 0, hi = a.ncell - 1;               // first c with cdf[c] > target
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cd[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        const int64_t cell = lo;
        const int c3 = (int)(cell % a.c3), c2 = (int)((cell / a.c3) % a.c2),
                  c1 = (int)(cell / ((int64_t)a.c3 * a.c2));
        const int s3 = a.s * a.s * a.s;
        const int o = min((int)(u3 * s3), s3 - 1);
        const int o1 = o / (a.s * a.s), o2 = (o / a.s) % a.s, o3 = o % a.s;
        const int h = a.s / 2;
        const int i1 = (a.s * c1 - h + o1 + a.g.n1) % a.g.n1;
        const int i2 = (a.s * c2 - h + o2 + a.g.n2) % a.g.n2;
        const int i3 = (a.s * c3 - h + o3 + a.g.n3) % a.g.n3;
        iq = grid_index(a.g, i1, i2, i3);
    }
    atomicAdd(&a.counts[kpl * a.nq + iq], 1);
}

__device__ __forceinline__ int64_t block_excl_scan_i64(int64_t v, int64_t *sm, int64_t &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t r = 0;
        for (int w = 0; w < nw; ++w) {
            const int64_t t = sm[w];
            sm[w] = r;
            r += t;
        }
        sm[32] = r;
    }
    __syncthreads();
    const int64_t ex = sm[wid] + x - v;
    total = sm[32];
    __syncthreads();
    return ex;
}

// A drawn q is evaluated when the sieve keeps (k, q); otherwise every term t(k, q) is zero.
__device__ __forceinline__ bool keep_draw(const SampleArgs &a, int ik, int nsel, const double *en,
                                          const float *en32, int64_t q) {
    return pair_valid(a.sv, nsel, en, en32, q, kplusq(a.g, ik, q));
}

__global__ void __launch_bounds__(256) k_is_count(SampleArgs a, int64_t *__restrict__ out) {
    __shared__ int64_t sm[33];
    __shared__ double en[epc::kMaxW];
    __shared__ float en32[epc::kMaxW];
    const int ik = a.kpts[blockIdx.x];
    const int nsel = a.win_n[ik];
    load_window(a.sv, ik, a.win_lo[ik], nsel, en, en32);
    const int *cn = a.counts + (int64_t)blockIdx.x * a.nq;
    int64_t c = 0;
    for (int64_t q = threadIdx.x; q < a.nq; q += blockDim.x)
        c += cn[q] > 0 && keep_draw(a, ik, nsel, en, en32, q);
    int64_t tot;
    block_excl_scan_i64(c, sm, tot);
    if (threadIdx.x == 0) out[blockIdx.x] = tot;
}

// Ordered compaction of the drawn q of each chunk k-point (one block each) with their
// weights c / (S p(q)).
__global__ void __launch_bounds__(256) k_is_fill(SampleArgs a, const int64_t *__restrict__ off,
                                                 int *__restrict__ pairs, double *__restrict__ w) {
    __shared__ int64_t sm[33];
    __shared__ double en[epc::kMaxW];
    __shared__ float en32[epc::kMaxW];
    const int64_t kpl = blockIdx.x;
    const int ik = a.kpts[kpl];
    const int nwin = a.win_n[ik];
    load_window(a.sv, ik, a.win_lo[ik], nwin, en, en32);
    const int64_t st0 = a.kp_state[kpl] - a.s_base;
    const int *cn = a.counts + kpl * a.nq;
    int64_t base = off[kpl];
    const double inv_s3 = 1.0 / ((double)a.s * a.s * a.s);
    for (int64_t q0 = 0; q0 < a.nq; q0 += blockDim.x) {
        const int64_t q = q0 + threadIdx.x;
        const int cnt = q < a.nq && cn[q] > 0 && keep_draw(a, ik, nwin, en, en32, q) ? cn[q] : 0;
        int64_t tot;
        const int64_t ex = block_excl_scan_i64(cnt > 0, sm, tot);
        if (cnt > 0) {
            double p = 1.0 / (double)a.nq;
            if (a.cdf) {
                int i1, i2, i3;
                grid_coords(a.g, q, i1, i2, i3);
                const int h = a.s / 2;
                const int64_t cell = ((int64_t)(((i1 + h) % a.g.n1) / a.s) * a.c2 +
                                      ((i2 + h) % a.g.n2) / a.s) * a.c3 +
                                     ((i3 + h) % a.g.n3) / a.s;
                double pm = 0;
                for (int b = 0; b < nwin; ++b) {
                    const double *cd = a.cdf + (st0 + b) * a.ncell;
                    const double pc = (cd[cell] - (cell > 0 ? cd[cell - 1] : 0.0)) / a.tot[st0 + b];
                    pm += a.alpha / (double)a.nq + (1.0 - a.alpha) * pc * inv_s3;
                }
                p = pm / nwin;
            }
            pairs[base + ex] = (int)q;
            w[base + ex] = (double)cnt / ((double)a.S * p);
        }
        base += tot;
    }
}

template <class T>
void upload_vec(DevBuf &b, const std::vector<T> &v, cudaStream_t st) {
    b.ensure(sizeof(T) * (v.size() + 1));
    if (!v.empty())
        EPWI_CUDA(cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
}

template <class T>
std::vector<T> download_vec(const DevBuf &b, size_t n, cudaStream_t st) {
    std::vector<T> v(n);
    if (n) EPWI_CUDA(cudaMemcpyAsync(v.data(), b.p, sizeof(T) * n, cudaMemcpyDeviceToHost, st));
    EPWI_CUDA(cudaStreamSynchronize(st));
    return v;
}

uint64_t host_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

void set_transport_params(epwi_ctx *c, double T, double mu, double eta, double emin, double emax) {
    c->have_rates = c->have_sigma = c->have_is = false;
    c->T = T;
    c->mu = mu;
    c->eta = eta;
    c->emin = emin;
    c->emax = emax;
}

struct PrecisionGuard {            // runs the plain kernels in FP64 and restores the mode
    epwi_ctx *c;
    int saved;
    explicit PrecisionGuard(epwi_ctx *cc) : c(cc), saved(cc->opt.precision) {
        c->opt.precision = EPWI_FP64;
    }
    ~PrecisionGuard() { c->opt.precision = (epwi_precision)saved; }
};

}  // namespace

// Builds the training set on the current grid and trains the network.
void mlp_train(epwi_ctx *c, double T, double mu, double eta, double emin, double emax,
               const epwi_mlp_train_options &o, double *final_loss) {
    set_transport_params(c, T, mu, eta, emin, emax);
    PrecisionGuard pg(c);
    if (!c->mlp || !c->mlp->ready) mlp_init(c, o.seed);
    build_window(c);
    ensure_velocities(c, false);
    sieve_count(c);
    occupation_tables(c);
    const int64_t nkp = c->nkp;
    EPWI_REQUIRE(nkp > 0, EPWI_EINVAL, "no states in the training window");
    EPWI_REQUIRE(c->npairs <= (int64_t(1) << 26), EPWI_EUNSUPPORTED,
                 "training grid too large (more than 2^26 sieved pairs)");
    cudaStream_t st = c->stream;
    // sieved pairs of every k-point, then uniformly drawn background pairs
    DevBuf sp;
    sp.ensure(sizeof(int) * (c->npairs + 1));
    sieve_fill_chunk(c, 0, nkp, sp.as<int>());
    std::vector<int> h_sp = download_vec<int>(sp, (size_t)c->npairs, st);
    sp.release();
    std::vector<int64_t> h_state = download_vec<int64_t>(c->kp_state, (size_t)nkp + 1, st);
    const int64_t nbg_total = (int64_t)std::ceil(o.background * (double)c->npairs);
    const int64_t nbg = nkp > 0 ? (nbg_total + nkp - 1) / nkp : 0;
    std::vector<int> pairs, pair_kp;
    std::vector<int64_t> kp_pairs(nkp + 1, 0), entry_off(nkp + 1, 0);
    int tstride = 1;
    for (int64_t kp = 0; kp < nkp; ++kp) {
        kp_pairs[kp] = (int64_t)pairs.size();
        for (int64_t p = c->h_kp_pairs[kp]; p < c->h_kp_pairs[kp + 1]; ++p) {
            pairs.push_back(h_sp[p]);
            pair_kp.push_back((int)kp);
        }
        for (int64_t j = 0; j < nbg; ++j) {
            const uint64_t h = host_mix64(host_mix64(o.seed ^ 0x5851f42d4c957f2dull) +
                                          0x9e3779b97f4a7c15ull * (uint64_t)(kp * nbg + j + 1));
            pairs.push_back((int)((h >> 11) % (uint64_t)c->nk));
            pair_kp.push_back((int)kp);
        }
        const int ns = (int)(h_state[kp + 1] - h_state[kp]);
        tstride = std::max(tstride, ns);
        entry_off[kp + 1] = entry_off[kp] +
                            ((int64_t)pairs.size() - kp_pairs[kp]) * ns * c->nm;
    }
    kp_pairs[nkp] = (int64_t)pairs.size();
    const int64_t np = (int64_t)pairs.size();
    const int64_t n = entry_off[nkp];
    MlpState &m = *c->mlp;
    DevBuf d_pairs, d_pair_kp, d_kp_pairs, d_off, d_tout;
    auto cleanup = [&] {
        d_pairs.release(); d_pair_kp.release(); d_kp_pairs.release(); d_off.release();
        d_tout.release();
    };
    try {
        upload_vec(d_pairs, pairs, st);
        upload_vec(d_pair_kp, pair_kp, st);
        upload_vec(d_kp_pairs, kp_pairs, st);
        upload_vec(d_off, entry_off, st);
        const size_t ntout = (size_t)np * tstride * c->nm;
        d_tout.ensure(sizeof(double) * (ntout + 1));
        EPWI_CUDA(cudaMemsetAsync(d_tout.p, 0, sizeof(double) * (ntout + 1), st));
        WorkSet ws;
        ws.nkp = nkp;
        ws.kpts = c->kpts.as<int>();
        ws.kp_state = c->kp_state.as<int64_t>();
        ws.kp_pairs = d_kp_pairs.as<int64_t>();
        ws.h_kp_state = h_state;
        ws.h_kp_pairs = kp_pairs;
        ws.pairs_dev = d_pairs.as<int>();
        epwi_stats keep = c->stats;
        process_workset(c, ws, nullptr, d_tout.as<double>(), tstride);
        c->stats = keep;
        // samples: features, raw terms, log targets
        m.n_train = n;
        m.X.ensure(sizeof(float) * (n * kIn + 4));
        m.Y.ensure(sizeof(float) * (n + 4));
        m.T64.ensure(sizeof(double) * (n + 1));
        m.ids.ensure(sizeof(int4) * (n + 1));
        GridInfo g = make_grid_info(c);
        k_train_set<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(
            np, d_pair_kp.as<int>(), d_pairs.as<int>(), c->kpts.as<int>(), c->win_lo.as<int>(),
            c->win_n.as<int>(), d_kp_pairs.as<int64_t>(), d_off.as<int64_t>(), d_tout.as<double>(),
            tstride, c->eps.as<double>(), mu, g, c->nw, c->nm, m.X.as<float>(), m.T64.as<double>(),
            m.ids.as<int4>());
        EPWI_CHECK_LAUNCH();
        EPWI_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        cudaStreamSynchronize(st);
        cleanup();
        throw;
    }
    cleanup();
    const double tmax = device_reduce_minmax(c, m.T64.as<double>(), n, 1, 0, true);
    EPWI_REQUIRE(tmax > 0, EPWI_ENUMERIC, "all training targets are zero");
    const double floor_ = o.floor_rel * tmax;
    const int64_t nb = (n + 255) / 256;
    DevBuf part;
    part.ensure(sizeof(double) * 2 * (nb + 1));
    k_log_targets<<<(unsigned)nb, 256, 0, st>>>(n, m.T64.as<double>(), floor_, m.Y.as<float>(),
                                                 part.as<double>());
    EPWI_CHECK_LAUNCH();
    std::vector<double> hp = download_vec<double>(part, (size_t)(2 * nb), st);
    part.release();
    double s1 = 0, s2 = 0;
    for (int64_t b = 0; b < nb; ++b) {
        s1 += hp[2 * b];
        s2 += hp[2 * b + 1];
    }
    const double mean = s1 / (double)n;
    const double sd = std::sqrt(std::max(1e-30, s2 / (double)n - mean * mean));
    k_normalise<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, (float)mean, (float)(1.0 / sd),
                                                            m.Y.as<float>());
    EPWI_CHECK_LAUNCH();
    m.out_scale = sd;
    m.out_shift = mean;
    // Adam on shuffled mini-batches of B samples (the last batch of an epoch wraps around the
    // permutation); the learning rate follows a cosine from lr to lr / 20.  The per-step
    // scalars go into a table; one captured graph replays every step.
    const int64_t B = std::min<int64_t>(std::min<int64_t>(std::max<int64_t>(o.batch, 1), kMaxBatch), n);
    const int64_t steps_per_epoch = (n + B - 1) / B;
    const int64_t total = steps_per_epoch * std::max(o.epochs, 0);
    std::vector<StepParams> steps;
    steps.reserve((size_t)total);
    const int64_t t0 = m.step;                       // Adam steps taken before this call
    for (int ep = 0; ep < o.epochs; ++ep) {
        // shuffle: i -> (a i + b) mod n with gcd(a, n) = 1
        uint64_t h = host_mix64(o.seed + 0x632be59bd9b4e019ull * (uint64_t)(ep + 1));
        uint64_t a = 1 + (h % (uint64_t)n);
        while (std::gcd(a, (uint64_t)n) != 1) a = a % (uint64_t)n + 1;
        const uint64_t b = host_mix64(h) % (uint64_t)n;
        for (int64_t i0 = 0; i0 < n; i0 += B) {
            const int64_t step = (int64_t)steps.size();
            const double frac = total > 1 ? (double)step / (double)(total - 1) : 1.0;
            const double t = (double)(t0 + step + 1);
            StepParams sp{};
            sp.i0 = i0;
            sp.a = a;
            sp.b = b;
            sp.lr = (float)(o.lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(epc::kPi * frac))));
            sp.bc1 = (float)(1.0 - std::pow(0.9, t));
            sp.bc2 = (float)(1.0 - std::pow(0.999, t));
            steps.push_back(sp);
        }
    }
    mlp_train_graph(c, steps, B);
    const double L = mlp_dataset_loss(c);
    if (final_loss) *final_loss = L;
}

// Importance-sampled rates: draws, weights, then the plain FP64 kernels on the weighted pairs.
void run_is(epwi_ctx *c, double T, double mu, double eta, double emin, double emax,
            int64_t S, double alpha, int stride, int proposal, uint64_t seed) {
    set_transport_params(c, T, mu, eta, emin, emax);
    cudaStream_t st = c->stream;
    cudaEvent_t e0, e1, e2;
    EPWI_CUDA(cudaEventCreate(&e0));
    EPWI_CUDA(cudaEventCreate(&e1));
    EPWI_CUDA(cudaEventCreate(&e2));
    cudaEventRecord(e0, st);
    build_window(c);
    ensure_velocities(c, false);
    occupation_tables(c);
    const int64_t nkp = c->nkp, nq = c->nk;
    const bool learned = proposal == EPWI_PROPOSAL_LEARNED;
    const int s = learned ? stride : 1;
    GridInfo g = make_grid_info(c);
    const int c1 = g.n1 / s, c2 = g.n2 / s, c3 = g.n3 / s;
    const int64_t ncell = (int64_t)c1 * c2 * c3;
    std::vector<int64_t> h_state = download_vec<int64_t>(c->kp_state, (size_t)nkp + 1, st);
    // chunk: counts <= 1 GiB, proposal tables <= 2 GiB
    const int64_t max_w = std::max<int64_t>(1, c->nstates > 0 ? (c->nstates + nkp - 1) / nkp : 1);
    int64_t kpc = std::max<int64_t>(1, (int64_t(1) << 30) / (4 * nq));
    if (learned) kpc = std::min<int64_t>(kpc, std::max<int64_t>(1, (int64_t(1) << 31) / (12 * ncell * max_w)));
    kpc = std::min<int64_t>(kpc, std::max<int64_t>(1, (int64_t(1) << 30) / std::max<int64_t>(1, S)));
    DevBuf counts, cdf, tot, logit, xb, yb, cnt, off;
    std::vector<DevBuf> chunk_pairs, chunk_w;
    std::vector<int64_t> kp_off(nkp + 1, 0);
    double flops = 0;
    float ms_prop = 0;
    auto cleanup = [&] {
        counts.release(); cdf.release(); tot.release(); logit.release(); xb.release();
        yb.release(); cnt.release(); off.release();
        for (auto &b : chunk_pairs) b.release();
        for (auto &b : chunk_w) b.release();
    };
    try {
        const int64_t rows_per_batch = (((int64_t)1 << 22) / c->nm) * c->nm;
        for (int64_t kp0 = 0; kp0 < nkp; kp0 += kpc) {
            const int64_t kp1 = std::min(nkp, kp0 + kpc), nkc = kp1 - kp0;
            const int64_t s0 = h_state[kp0], nsc = h_state[kp1] - s0;
            SampleArgs sa;
            sa.g = g;
            sa.s = s;
            sa.c2 = c2;
            sa.c3 = c3;
            sa.ncell = ncell;
            sa.nq = nq;
            sa.S = S;
            sa.alpha = learned ? alpha : 1.0;
            sa.seed = seed;
            sa.kpts = c->kpts.as<int>() + kp0;
            sa.kp_state = c->kp_state.as<int64_t>() + kp0;
            sa.s_base = s0;
            sa.win_lo = c->win_lo.as<int>();
            sa.win_n = c->win_n.as<int>();
            sa.sv = make_sieve_args(c);
            sa.cdf = nullptr;
            sa.tot = nullptr;
            if (learned && nsc > 0) {
                cudaEvent_t p0, p1;
                EPWI_CUDA(cudaEventCreate(&p0));
                EPWI_CUDA(cudaEventCreate(&p1));
                cudaEventRecord(p0, st);
                logit.ensure(sizeof(float) * nsc * ncell);
                cdf.ensure(sizeof(double) * nsc * ncell);
                tot.ensure(sizeof(double) * (nsc + 1));
                xb.ensure(sizeof(float) * rows_per_batch * kIn);
                yb.ensure(sizeof(float) * rows_per_batch);
                PropArgs pa;
                pa.g = g;
                pa.W = c->nw;
                pa.Nm = c->nm;
                pa.s = s;
                pa.c2 = c2;
                pa.c3 = c3;
                pa.ncell = ncell;
                pa.st_k = c->st_k.as<int>();
                pa.st_n = c->st_n.as<int>();
                pa.eps = c->eps.as<double>();
                pa.mu = mu;
                const int64_t rows = nsc * ncell * c->nm;
                for (int64_t r0 = 0; r0 < rows; r0 += rows_per_batch) {
                    const int64_t nr = std::min(rows_per_batch, rows - r0);
                    k_prop_features<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(pa, s0, r0, nr,
                                                                                   xb.as<float>());
                    EPWI_CHECK_LAUNCH();
                    mlp_forward_fast(c, nr, xb.as<float>(), yb.as<float>());
                    const int64_t ng = nr / c->nm;
                    k_prop_lse<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(
                        ng, c->nm, (float)c->mlp->out_scale, yb.as<float>(),
                        logit.as<float>() + r0 / c->nm);
                    EPWI_CHECK_LAUNCH();
                }
                flops += 2.0 * (double)rows * (kIn * kHid + 2.0 * kHid * kHid + kHid);
                k_state_cdf<<<(unsigned)nsc, 1024, 0, st>>>(ncell, logit.as<float>(), cdf.as<double>(),
                                                           tot.as<double>());
                EPWI_CHECK_LAUNCH();
                cudaEventRecord(p1, st);
                EPWI_CUDA(cudaEventSynchronize(p1));
                float ms = 0;
                cudaEventElapsedTime(&ms, p0, p1);
                ms_prop += ms;
                cudaEventDestroy(p0);
                cudaEventDestroy(p1);
                sa.cdf = cdf.as<double>();
                sa.tot = tot.as<double>();
            }
            counts.ensure(sizeof(int) * nkc * nq);
            EPWI_CUDA(cudaMemsetAsync(counts.p, 0, sizeof(int) * nkc * nq, st));
            sa.counts = counts.as<int>();
            const int64_t nt = nkc * S;
            if (nt > 0) {
                k_is_sample<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(sa, nkc);
                EPWI_CHECK_LAUNCH();
            }
            cnt.ensure(sizeof(int64_t) * (nkc + 1));
            off.ensure(sizeof(int64_t) * (nkc + 1));
            k_is_count<<<(unsigned)nkc, 256, 0, st>>>(sa, cnt.as<int64_t>());
            EPWI_CHECK_LAUNCH();
            int64_t npc = 0;
            scan_exclusive_i64(c, cnt.as<int64_t>(), off.as<int64_t>(), nkc, &npc);
            std::vector<int64_t> ho = download_vec<int64_t>(off, (size_t)nkc + 1, st);
            for (int64_t k = 0; k < nkc; ++k) kp_off[kp0 + k + 1] = kp_off[kp0] + ho[k + 1];
            chunk_pairs.emplace_back();
            chunk_w.emplace_back();
            chunk_pairs.back().ensure(sizeof(int) * (npc + 1));
            chunk_w.back().ensure(sizeof(double) * (npc + 1));
            k_is_fill<<<(unsigned)nkc, 256, 0, st>>>(sa, off.as<int64_t>(), chunk_pairs.back().as<int>(),
                                                     chunk_w.back().as<double>());
            EPWI_CHECK_LAUNCH();
            EPWI_CUDA(cudaStreamSynchronize(st));
        }
        const int64_t npairs = kp_off[nkp];
        c->is_pairs.ensure(sizeof(int) * (npairs + 1));
        c->is_w.ensure(sizeof(double) * (npairs + 1));
        {
            int64_t k = 0;
            for (size_t ci = 0; ci < chunk_pairs.size(); ++ci) {
                const int64_t kp0 = (int64_t)ci * kpc, kp1 = std::min(nkp, kp0 + kpc);
                const int64_t m = kp_off[kp1] - kp_off[kp0];
                if (m > 0) {
                    EPWI_CUDA(cudaMemcpyAsync(c->is_pairs.as<int>() + k, chunk_pairs[ci].p,
                                              sizeof(int) * m, cudaMemcpyDeviceToDevice, st));
                    EPWI_CUDA(cudaMemcpyAsync(c->is_w.as<double>() + k, chunk_w[ci].p,
                                              sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
                }
                k += m;
            }
        }
        upload_vec(c->is_kp_pairs, kp_off, st);
        c->h_is_kp_pairs = kp_off;
        EPWI_CUDA(cudaStreamSynchronize(st));
        cleanup();
        cudaEventRecord(e1, st);
        if (c->nstates > 0)
            EPWI_CUDA(cudaMemsetAsync(c->inv_tau.p, 0, sizeof(double) * c->nstates, st));
        std::memset(&c->stats, 0, sizeof(c->stats));
        c->stats.precision = c->opt.precision;
        c->stats.ms_eigs = c->ms_eigs;
        EPWI_CUDA(cudaDeviceGetAttribute(&c->stats.sm_count, cudaDevAttrMultiProcessorCount, c->device));
        WorkSet ws;
        ws.nkp = nkp;
        ws.kpts = c->kpts.as<int>();
        ws.kp_state = c->kp_state.as<int64_t>();
        ws.kp_pairs = c->is_kp_pairs.as<int64_t>();
        ws.h_kp_state = h_state;
        ws.h_kp_pairs = kp_off;
        ws.pairs_dev = c->is_pairs.as<int>();
        ws.pair_w = c->is_w.as<double>();
        process_workset(c, ws, nullptr);
        cudaEventRecord(e2, st);
        EPWI_CUDA(cudaEventSynchronize(e2));
        float ms_draw = 0;
        cudaEventElapsedTime(&ms_draw, e0, e1);
        c->npairs = npairs;
        c->stats.n_kpoints = nkp;
        c->stats.n_states = c->nstates;
        c->stats.n_pairs = npairs;
        c->stats.ms_proposal = ms_prop;
        c->stats.ms_sampling = ms_draw - ms_prop;
        c->stats.proposal_flops = flops;
        c->stats.scatter_flops = 8.0 * c->nRp * c->nm * c->nw * (double)npairs *
                                 ((double)c->nstates / std::max<int64_t>(1, nkp));
    } catch (...) {
        cudaStreamSynchronize(st);
        cleanup();
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    c->have_rates = true;
    c->have_is = true;
}
