// Training kernels of the learned q-proposal network (SIMT, FP32 arithmetic on BF16-rounded
// weights): dense layers with SiLU, the least-squares loss, back-propagation by the chain
// rule, Adam (Kingma & Ba 2015, Algorithm 1), initialisation and the batch gather.  One
// training step (gather, forward, back-propagation, Adam) is captured as a CUDA graph and
// replayed for every step; the step-dependent scalars come from a per-step table indexed by
// a device counter.  The same dense-layer kernels give the reference forward pass.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mlp.cuh"

namespace {
using namespace mlp;

constexpr int kRowsPerBlock = 64;     // dense layers: rows per block
constexpr int kSliceRows = 64;        // weight gradients: rows per batch slice

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// SplitMix64 output function (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// out[r][c] = sum_{j<K} X[r][j] Wop(j, c), c < 128.
//   TW = false: Wop(j, c) = W[c][j]  (W stored [128][K]: a layer's forward product)
//   TW = true : Wop(j, c) = W[j][c]  (W stored [K][128]: product with the transposed layer)
// EPI = 0: z = acc + bias[c]; Z[r][c] = z (if Z); H[r][c] = silu(z)
// EPI = 1: H[r][c] = acc * silu'(Zp[r][c])      (back-propagation through the activation)
template <int K, bool TW, int EPI>
__global__ void __launch_bounds__(256) k_dense(int64_t n, const float *__restrict__ X,
                                               const float *__restrict__ W,
                                               const float *__restrict__ bias,
                                               const float *__restrict__ Zp, float *__restrict__ Z,
                                               float *__restrict__ H) {
    constexpr int KC = K < 32 ? K : 32;
    __shared__ float Xs[kRowsPerBlock][KC + 1];
    __shared__ float Ws[kHid][KC + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += KC) {
        for (int e = threadIdx.x; e < kRowsPerBlock * KC; e += 256) {
            const int rr = e / KC, kk = e % KC;
            const int64_t r = r0 + rr;
            Xs[rr][kk] = r < n ? X[r * K + k0 + kk] : 0.f;
        }
        for (int e = threadIdx.x; e < kHid * KC; e += 256) {
            if (TW) {
                const int kk = e / kHid, cc = e % kHid;
                Ws[cc][kk] = W[(k0 + kk) * kHid + cc];
            } else {
                const int cc = e / KC, kk = e % KC;
                Ws[cc][kk] = W[cc * K + k0 + kk];
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KC; ++kk) {
            float a[8], b[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = Xs[ty * 8 + i][kk];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Ws[tx + 32 * j][kk];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = r0 + ty * 8 + i;
        if (r >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = tx + 32 * j;
            if (EPI == 0) {
                const float z = acc[i][j] + bias[c];
                if (Z) Z[r * kHid + c] = z;
                H[r * kHid + c] = silu_f(z);
            } else {
                H[r * kHid + c] = acc[i][j] * dsilu_f(Zp[r * kHid + c]);
            }
        }
    }
}

// yhat[r] = H3[r] . w4 + b4 (one warp per row); with Y: dy[r] = (yhat - Y) * inv_b.
__global__ void __launch_bounds__(256) k_out(int64_t n, const float *__restrict__ H3,
                                             const float *__restrict__ w4,
                                             const float *__restrict__ b4,
                                             const float *__restrict__ Y, float inv_b,
                                             float *__restrict__ yhat, float *__restrict__ dy) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float4 h = reinterpret_cast<const float4 *>(H3 + r * kHid)[lane];
    const float4 w = reinterpret_cast<const float4 *>(w4)[lane];
    float s = h.x * w.x;
    s = fmaf(h.y, w.y, s);
    s = fmaf(h.z, w.z, s);
    s = fmaf(h.w, w.w, s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const float y = s + b4[0];
        yhat[r] = y;
        if (Y) dy[r] = (y - Y[r]) * inv_b;
    }
}

// Per-block sums of (yhat - Y)^2 in FP64.
__global__ void __launch_bounds__(256) k_sq_partial(int64_t n, const float *__restrict__ yhat,
                                                    const float *__restrict__ Y,
                                                    double *__restrict__ part) {
    __shared__ double sm[256];
    const int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x;
    double v = 0;
    if (r < n) {
        const double d = (double)yhat[r] - (double)Y[r];
        v = d * d;
    }
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// dZ3[r][c] = dy[r] w4[c] silu'(Z3[r][c])
__global__ void k_dz_last(int64_t n, const float *__restrict__ dy, const float *__restrict__ w4,
                          const float *__restrict__ Z3, float *__restrict__ D3) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * kHid) return;
    const int c = (int)(e % kHid);
    D3[e] = dy[e / kHid] * w4[c] * dsilu_f(Z3[e]);
}

// Split-batch weight gradients: part[s][c][j] = sum_{r in slice s} D[r][c] X[r][j] and
// partb[s][c] = sum_{r in slice s} D[r][c] (c < 128, j < K).  Thread (ty, tx) owns
// c in [8 ty, 8 ty + 8), j in [8 tx, 8 tx + 8).
template <int K>
__global__ void __launch_bounds__(256) k_wgrad(int64_t n, const float *__restrict__ D,
                                               const float *__restrict__ X,
                                               float *__restrict__ part,
                                               float *__restrict__ partb) {
    constexpr int KP = ((K + 7) / 8) * 8 + 4;
    __shared__ __align__(16) float Ds[32][kHid + 4];
    __shared__ __align__(16) float Xs[32][KP];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const bool jact = tx * 8 < K;
    const int64_t rb0 = (int64_t)blockIdx.x * kSliceRows;
    const int64_t rb1 = min(n, rb0 + kSliceRows);
    float acc[8][8], accb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        accb[i] = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    }
    for (int64_t rb = rb0; rb < rb1; rb += 32) {
        for (int e = threadIdx.x; e < 32 * kHid; e += 256) {
            const int rr = e / kHid, cc = e % kHid;
            Ds[rr][cc] = rb + rr < rb1 ? D[(rb + rr) * kHid + cc] : 0.f;
        }
        for (int e = threadIdx.x; e < 32 * KP; e += 256) {
            const int rr = e / KP, jj = e % KP;
            Xs[rr][jj] = (rb + rr < rb1 && jj < K) ? X[(rb + rr) * K + jj] : 0.f;
        }
        __syncthreads();
        for (int rr = 0; rr < 32; ++rr) {
            float a[8], x[8];
            const float4 a0 = *reinterpret_cast<const float4 *>(&Ds[rr][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&Ds[rr][ty * 8 + 4]);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
            if (jact) {
                const float4 x0 = *reinterpret_cast<const float4 *>(&Xs[rr][tx * 8]);
                const float4 x1 = *reinterpret_cast<const float4 *>(&Xs[rr][tx * 8 + 4]);
                x[0] = x0.x; x[1] = x0.y; x[2] = x0.z; x[3] = x0.w;
                x[4] = x1.x; x[5] = x1.y; x[6] = x1.z; x[7] = x1.w;
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) x[j] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                accb[i] += a[i];
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], x[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
    float *ps = part + (int64_t)blockIdx.x * kHid * K;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = ty * 8 + i;
        if (jact)
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (tx * 8 + j < K) ps[c * K + tx * 8 + j] = acc[i][j];
        if (tx == 0) partb[(int64_t)blockIdx.x * kHid + c] = accb[i];
    }
}

// out[i] = sum over slices s (in order) of part[s * len + i]
__global__ void k_reduce_slices(int64_t len, int nslices, const float *__restrict__ part,
                                float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    float s = 0.f;
    for (int k = 0; k < nslices; ++k) s += part[(int64_t)k * len + i];
    out[i] = s;
}

// bf16 copy of the master weights (round to nearest even)
__device__ __forceinline__ void store_rounded(int64_t i, float x, float *__restrict__ w,
                                              uint16_t *__restrict__ wbf) {
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    w[i] = __bfloat162float(b);
    wbf[i] = __bfloat16_as_ushort(b);
}

__global__ void k_round(int64_t np, const float *__restrict__ master, float *__restrict__ w,
                        uint16_t *__restrict__ wbf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) store_rounded(i, master[i], w, wbf);
}

// Glorot-uniform weights from a counter-based generator, zero biases.
__global__ void k_init(uint64_t seed, float *__restrict__ master) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParam) return;
    float lim = 0.f;
    if (i < ob1) lim = sqrtf(6.0f / (kIn + kHid));
    else if ((i >= oW2 && i < ob2) || (i >= oW3 && i < ob3)) lim = sqrtf(6.0f / (kHid + kHid));
    else if (i >= ow4 && i < ob4) lim = sqrtf(6.0f / (kHid + 1));
    const uint64_t h = mix64(seed * 0x9e3779b97f4a7c15ull + (uint64_t)i + 1);
    const double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);   // [0, 1)
    master[i] = (float)((2.0 * u - 1.0) * lim);
}


// Training-step kernels driven by a per-step parameter table and a device step counter, so
// that one captured graph replays every step.
__global__ void k_gather_step(const StepParams *__restrict__ sp, const int64_t *__restrict__ ctr,
                              int64_t n, int64_t bsz, const float *__restrict__ X,
                              const float *__restrict__ Y, float *__restrict__ bx,
                              float *__restrict__ by) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= bsz) return;
    const StepParams p = sp[*ctr];
    // a full batch every step: positions past the end of the permutation wrap around
    const uint64_t i = (uint64_t)((p.i0 + j) % n);
    const uint64_t idx = (p.a * i + p.b) % (uint64_t)n;
    for (int f = 0; f < kIn; ++f) bx[j * kIn + f] = X[idx * kIn + f];
    by[j] = Y[idx];
}

__global__ void k_adam_step(const StepParams *__restrict__ sp, const int64_t *__restrict__ ctr,
                            int64_t np, float *__restrict__ master, const float *__restrict__ grad,
                            float *__restrict__ m, float *__restrict__ v, float b1, float b2, float eps,
                            float *__restrict__ w, uint16_t *__restrict__ wbf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const StepParams p = sp[*ctr];
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float x = master[i] - p.lr * (mi / p.bc1) / (sqrtf(vi / p.bc2) + eps);
    master[i] = x;
    const __nv_bfloat16 bv = __float2bfloat16_rn(x);
    w[i] = __bfloat162float(bv);
    wbf[i] = __bfloat16_as_ushort(bv);
}

__global__ void k_step_advance(int64_t *ctr) { *ctr += 1; }

MlpState &state(epwi_ctx *c) {
    if (!c->mlp) c->mlp = new MlpState();
    return *c->mlp;
}

// Activation slots of one batch of up to `cap` rows.
struct Act {
    float *Z1, *H1, *Z2, *H2, *Z3, *H3, *D3, *D2, *D1, *yhat, *dy;
};

Act act_slots(epwi_ctx *c, int64_t rows) {
    MlpState &s = state(c);
    const size_t per = (size_t)rows * kHid;
    s.act.ensure(sizeof(float) * (9 * per + 2 * (size_t)rows + 64));
    float *p = s.act.as<float>();
    Act a;
    a.Z1 = p;
    a.H1 = p + per;
    a.Z2 = p + 2 * per;
    a.H2 = p + 3 * per;
    a.Z3 = p + 4 * per;
    a.H3 = p + 5 * per;
    a.D3 = p + 6 * per;
    a.D2 = p + 7 * per;
    a.D1 = p + 8 * per;
    a.yhat = p + 9 * per;
    a.dy = a.yhat + rows;
    return a;
}

void round_params(epwi_ctx *c) {
    MlpState &s = state(c);
    k_round<<<(unsigned)((kNParam + 255) / 256), 256, 0, c->stream>>>(
        kNParam, s.master.as<float>(), s.w.as<float>(), s.wbf.as<uint16_t>());
    EPWI_CHECK_LAUNCH();
}

void alloc_params(epwi_ctx *c) {
    MlpState &s = state(c);
    s.master.ensure(sizeof(float) * kNParam);
    s.w.ensure(sizeof(float) * kNParam);
    s.wbf.ensure(sizeof(uint16_t) * kNParam + 16);
    s.m.ensure(sizeof(float) * kNParam);
    s.v.ensure(sizeof(float) * kNParam);
    s.grad.ensure(sizeof(float) * kNParam);
    EPWI_CUDA(cudaMemsetAsync(s.m.p, 0, sizeof(float) * kNParam, c->stream));
    EPWI_CUDA(cudaMemsetAsync(s.v.p, 0, sizeof(float) * kNParam, c->stream));
    s.step = 0;
}

// Forward pass of n <= cap rows; Z buffers are written when keep is set.
void forward_rows(epwi_ctx *c, const Act &a, int64_t n, const float *X, const float *Y,
                  bool keep) {
    MlpState &s = state(c);
    const float *w = s.w.as<float>();
    const unsigned nb = (unsigned)((n + kRowsPerBlock - 1) / kRowsPerBlock);
    k_dense<kIn, false, 0><<<nb, 256, 0, c->stream>>>(n, X, w + oW1, w + ob1, nullptr,
                                                        keep ? a.Z1 : nullptr, a.H1);
    EPWI_CHECK_LAUNCH();
    k_dense<kHid, false, 0><<<nb, 256, 0, c->stream>>>(n, a.H1, w + oW2, w + ob2, nullptr,
                                                         keep ? a.Z2 : nullptr, a.H2);
    EPWI_CHECK_LAUNCH();
    k_dense<kHid, false, 0><<<nb, 256, 0, c->stream>>>(n, a.H2, w + oW3, w + ob3, nullptr,
                                                         keep ? a.Z3 : nullptr, a.H3);
    EPWI_CHECK_LAUNCH();
    k_out<<<(unsigned)((n * 32 + 255) / 256), 256, 0, c->stream>>>(
        n, a.H3, w + ow4, w + ob4, Y, 1.0f / (float)n, a.yhat, a.dy);
    EPWI_CHECK_LAUNCH();
}

double sum_sq(epwi_ctx *c, int64_t n, const float *yhat, const float *Y) {
    MlpState &s = state(c);
    const int64_t nb = (n + 255) / 256;
    s.lossbuf.ensure(sizeof(double) * (nb + 1));
    k_sq_partial<<<(unsigned)nb, 256, 0, c->stream>>>(n, yhat, Y, s.lossbuf.as<double>());
    EPWI_CHECK_LAUNCH();
    std::vector<double> h(nb);
    EPWI_CUDA(cudaMemcpyAsync(h.data(), s.lossbuf.p, sizeof(double) * nb, cudaMemcpyDeviceToHost,
                              c->stream));
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    double t = 0;
    for (double v : h) t += v;
    return t;
}

template <int K>
void weight_grad(epwi_ctx *c, int64_t n, const float *D, const float *X, int64_t oW, int64_t ob) {
    MlpState &s = state(c);
    const int nsl = (int)((n + kSliceRows - 1) / kSliceRows);
    s.part.ensure(sizeof(float) * ((size_t)nsl * kHid * (K + 1) + 16));
    float *part = s.part.as<float>();
    float *partb = part + (size_t)nsl * kHid * K;
    k_wgrad<K><<<(unsigned)nsl, 256, 0, c->stream>>>(n, D, X, part, partb);
    EPWI_CHECK_LAUNCH();
    float *g = s.grad.as<float>();
    k_reduce_slices<<<(unsigned)((kHid * K + 255) / 256), 256, 0, c->stream>>>(kHid * K, nsl, part,
                                                                              g + oW);
    EPWI_CHECK_LAUNCH();
    k_reduce_slices<<<1, kHid, 0, c->stream>>>(kHid, nsl, partb, g + ob);
    EPWI_CHECK_LAUNCH();
}

}  // namespace

void mlp_free(MlpState *m) {
    if (!m) return;
    m->release();
    delete m;
}

void mlp_init(epwi_ctx *c, uint64_t seed) {
    alloc_params(c);
    MlpState &s = state(c);
    k_init<<<(unsigned)((kNParam + 255) / 256), 256, 0, c->stream>>>(seed, s.master.as<float>());
    EPWI_CHECK_LAUNCH();
    round_params(c);
    s.out_scale = 1.0;
    s.out_shift = 0.0;
    s.ready = true;
}

void mlp_set_master(epwi_ctx *c, const float *host_params) {
    alloc_params(c);
    MlpState &s = state(c);
    EPWI_CUDA(cudaMemcpyAsync(s.master.p, host_params, sizeof(float) * kNParam,
                              cudaMemcpyHostToDevice, c->stream));
    round_params(c);
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    s.ready = true;
}

void mlp_forward(epwi_ctx *c, int64_t n, const float *X, float *yhat) {
    const int64_t cap = std::min<int64_t>(n, kMaxBatch);
    for (int64_t r0 = 0; r0 < n; r0 += cap) {
        const int64_t m = std::min(cap, n - r0);
        Act a = act_slots(c, cap);
        forward_rows(c, a, m, X + r0 * kIn, nullptr, false);
        EPWI_CUDA(cudaMemcpyAsync(yhat + r0, a.yhat, sizeof(float) * m, cudaMemcpyDeviceToDevice,
                                  c->stream));
    }
}

// One forward and backward pass over n <= kMaxBatch rows (device X, Y); leaves dL/dparams in
// the gradient buffer and returns L = (1/2n) sum (yhat - y)^2.
double mlp_loss_grad(epwi_ctx *c, int64_t n, const float *X, const float *Y, bool want_loss) {
    MlpState &s = state(c);
    Act a = act_slots(c, n);
    const float *w = s.w.as<float>();
    float *g = s.grad.as<float>();
    forward_rows(c, a, n, X, Y, true);
    const unsigned nb = (unsigned)((n + kRowsPerBlock - 1) / kRowsPerBlock);
    // output layer: dL/dz3 = dy w4 silu'(z3), dL/dw4 = sum_r h3[r] dy[r], dL/db4 = sum_r dy[r]
    k_dz_last<<<(unsigned)((n * kHid + 255) / 256), 256, 0, c->stream>>>(n, a.dy, w + ow4, a.Z3,
                                                                       a.D3);
    EPWI_CHECK_LAUNCH();
    {
        const int nsl = (int)((n + kSliceRows - 1) / kSliceRows);
        s.part.ensure(sizeof(float) * ((size_t)nsl * kHid * (kHid + 1) + 16));
        float *part = s.part.as<float>();
        float *partb = part + (size_t)nsl * kHid * kHid;
        // the weight-gradient kernel with D = h3 and a one-column input dy: part[s][c][0] =
        // sum over the slice of h3[r][c] dy[r]
        k_wgrad<1><<<(unsigned)nsl, 256, 0, c->stream>>>(n, a.H3, a.dy, part, partb);
        EPWI_CHECK_LAUNCH();
        k_reduce_slices<<<1, kHid, 0, c->stream>>>(kHid, nsl, part, g + ow4);
        EPWI_CHECK_LAUNCH();
        // db4: the slice reduction with one element per "slice" sums dy in row order
        k_reduce_slices<<<1, 32, 0, c->stream>>>(1, (int)n, a.dy, g + ob4);
        EPWI_CHECK_LAUNCH();
    }
    weight_grad<kHid>(c, n, a.D3, a.H2, oW3, ob3);
    k_dense<kHid, true, 1><<<nb, 256, 0, c->stream>>>(n, a.D3, w + oW3, nullptr, a.Z2, nullptr,
                                                        a.D2);
    EPWI_CHECK_LAUNCH();
    weight_grad<kHid>(c, n, a.D2, a.H1, oW2, ob2);
    k_dense<kHid, true, 1><<<nb, 256, 0, c->stream>>>(n, a.D2, w + oW2, nullptr, a.Z1, nullptr,
                                                        a.D1);
    EPWI_CHECK_LAUNCH();
    weight_grad<kIn>(c, n, a.D1, X, oW1, ob1);
    return want_loss ? 0.5 * sum_sq(c, n, a.yhat, Y) / (double)n : 0.0;
}

// Mean squared residual (1/2n) sum (yhat - y)^2 over the whole training set.
double mlp_dataset_loss(epwi_ctx *c) {
    MlpState &s = state(c);
    const int64_t n = s.n_train;
    if (n == 0) return 0.0;
    const int64_t cap = std::min<int64_t>(n, kMaxBatch);
    double t = 0;
    for (int64_t r0 = 0; r0 < n; r0 += cap) {
        const int64_t m = std::min(cap, n - r0);
        Act a = act_slots(c, cap);
        forward_rows(c, a, m, s.X.as<float>() + r0 * kIn, nullptr, false);
        t += sum_sq(c, m, a.yhat, s.Y.as<float>() + r0);
    }
    return 0.5 * t / (double)n;
}

void mlp_forward_fast(epwi_ctx *c, int64_t n, const float *X, float *y) {
    MlpState &s = state(c);
    s.err.ensure(sizeof(int));
    EPWI_CUDA(cudaMemsetAsync(s.err.p, 0, sizeof(int), c->stream));
    mlp_forward_tc(c, n, X, y, s.err.as<int>());
    int h = 0;
    EPWI_CUDA(cudaMemcpyAsync(&h, s.err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    EPWI_REQUIRE(h == 0, EPWI_ETIMEOUT, "tensor-core inference: a bounded mbarrier wait timed out");
}

// Replays one captured training step (gather, forward, back-propagation, Adam, counter) for
// every entry of the step table.
void mlp_train_graph(epwi_ctx *c, const std::vector<StepParams> &steps, int64_t B) {
    MlpState &s = state(c);
    const int64_t n = s.n_train;
    if (steps.empty() || n == 0) return;
    // capture and replay on a private stream (the legacy default stream cannot be captured);
    // it first waits for the work already queued on the context's stream
    struct StreamSwap {
        epwi_ctx *c;
        cudaStream_t saved, own = nullptr;
        explicit StreamSwap(epwi_ctx *cc) : c(cc), saved(cc->stream) {
            EPWI_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
            cudaEvent_t ev;
            EPWI_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            EPWI_CUDA(cudaEventRecord(ev, saved));
            EPWI_CUDA(cudaStreamWaitEvent(own, ev, 0));
            cudaEventDestroy(ev);
            c->stream = own;
        }
        ~StreamSwap() {
            cudaStreamSynchronize(own);
            c->stream = saved;
            cudaStreamDestroy(own);
        }
    } swap(c);
    s.bx.ensure(sizeof(float) * kIn * kMaxBatch);
    s.by.ensure(sizeof(float) * kMaxBatch);
    DevBuf sp, ctr;
    sp.ensure(sizeof(StepParams) * steps.size());
    ctr.ensure(sizeof(int64_t));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&] {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        sp.release();
        ctr.release();
    };
    try {
        EPWI_CUDA(cudaMemcpyAsync(sp.p, steps.data(), sizeof(StepParams) * steps.size(),
                                  cudaMemcpyHostToDevice, c->stream));
        EPWI_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(int64_t), c->stream));
        // one un-captured pass sizes every buffer of the step
        mlp_loss_grad(c, B, s.bx.as<float>(), s.by.as<float>(), false);
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
        EPWI_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
        try {
            k_gather_step<<<(unsigned)((B + 255) / 256), 256, 0, c->stream>>>(
                sp.as<StepParams>(), ctr.as<int64_t>(), n, B, s.X.as<float>(), s.Y.as<float>(),
                s.bx.as<float>(), s.by.as<float>());
            EPWI_CHECK_LAUNCH();
            mlp_loss_grad(c, B, s.bx.as<float>(), s.by.as<float>(), false);
            k_adam_step<<<(unsigned)((kNParam + 255) / 256), 256, 0, c->stream>>>(
                sp.as<StepParams>(), ctr.as<int64_t>(), kNParam, s.master.as<float>(), s.grad.as<float>(),
                s.m.as<float>(), s.v.as<float>(), 0.9f, 0.999f, 1e-8f, s.w.as<float>(), s.wbf.as<uint16_t>());
            EPWI_CHECK_LAUNCH();
            k_step_advance<<<1, 1, 0, c->stream>>>(ctr.as<int64_t>());
            EPWI_CHECK_LAUNCH();
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(c->stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        EPWI_CUDA(cudaStreamEndCapture(c->stream, &graph));
        EPWI_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        for (size_t k = 0; k < steps.size(); ++k) EPWI_CUDA(cudaGraphLaunch(exec, c->stream));
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
        s.step += (int64_t)steps.size();
    } catch (...) {
        cudaStreamSynchronize(c->stream);
        cleanup();
        throw;
    }
    cleanup();
}
