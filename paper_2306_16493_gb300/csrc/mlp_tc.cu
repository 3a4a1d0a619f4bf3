// Inference of the q-proposal network on the tensor cores (tcgen05).
//
// One 128-row tile at a time per CTA (persistent over tiles, two CTAs per SM), 128 threads:
// thread r owns row r of the tile and TMEM lane r.
//   layer 1 (K = 9) on the CUDA cores in FP32: h1 = silu(W1 x + b1), rounded to BF16 and
//           written to shared memory as the A operand;
//   layer 2 h2 = silu(W2 h1 + b2): eight tcgen05.mma kind::f16 (BF16, M = N = 128, K = 16
//           each) with the FP32 accumulator in TMEM, read back by tcgen05.ld, bias and SiLU
//           in FP32, rounded to BF16 into the same A buffer;
//   layer 3 the same with W3, then y = w4 . silu(W3 h2 + b3) + b4 in FP32.
// Weights stay in shared memory for the whole launch.  Operands use the no-swizzle K-major
// canonical layout (core matrices of 8 rows x 16 bytes; LBO = 128 bytes between core matrices
// along K, SBO = 2048 bytes between 8-row groups for K = 128).  Every mbarrier wait is
// bounded; on a timeout the kernel records the error, drains and frees its TMEM.
#include <cuda_bf16.h>

#include <algorithm>

#include "mlp.cuh"
#include "tc_ptx.cuh"

namespace {
using namespace mlp;

constexpr int kRows = 128;
constexpr uint32_t kTileBytes = 128 * 128 * 2;      // one 128 x 128 BF16 operand
constexpr uint64_t kWaitNs = 2000000000ull;          // 2 s

__device__ __forceinline__ uint32_t cm_offset(int row, int k) {   // bytes, K = 128 BF16
    return (uint32_t)(((row >> 3) * 16 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

struct MlpTcArgs {
    int64_t n;                   // rows
    const float *X;              // [n][9]
    float *y;                    // [n]
    const uint16_t *wbf;         // BF16 parameters (storage order of mlp.cuh)
    const float *w;              // the same values as FP32 (biases, W1, w4)
    int *err;
};

__global__ void __launch_bounds__(kRows, 2) k_mlp_infer_tc(MlpTcArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sW2 = smem;
    uint8_t *sW3 = smem + kTileBytes;
    uint8_t *sA = smem + 2 * kTileBytes;
    float *sW1 = reinterpret_cast<float *>(smem + 3 * kTileBytes);     // [128][9]
    float *sB1 = sW1 + kHid * kIn, *sB2 = sB1 + kHid, *sB3 = sB2 + kHid, *sW4 = sB3 + kHid;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sW4 + kHid + 2);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    volatile int *sfail = reinterpret_cast<volatile int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5;

    // weights into shared memory: W2, W3 as canonical BF16 tiles; the rest in FP32
    for (int e = tid; e < kHid * kHid / 8; e += kRows) {
        const int n = e / (kHid / 8), k8 = (e % (kHid / 8)) * 8;
        const uint4 v2 = *reinterpret_cast<const uint4 *>(a.wbf + oW2 + n * kHid + k8);
        const uint4 v3 = *reinterpret_cast<const uint4 *>(a.wbf + oW3 + n * kHid + k8);
        *reinterpret_cast<uint4 *>(sW2 + cm_offset(n, k8)) = v2;
        *reinterpret_cast<uint4 *>(sW3 + cm_offset(n, k8)) = v3;
    }
    for (int e = tid; e < kHid * kIn; e += kRows) sW1[e] = a.w[oW1 + e];
    for (int e = tid; e < kHid; e += kRows) {
        sB1[e] = a.w[ob1 + e];
        sB2[e] = a.w[ob2 + e];
        sB3[e] = a.w[ob3 + e];
        sW4[e] = a.w[ow4 + e];
    }
    const float b4 = a.w[ob4];
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        *sfail = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, 128);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t idesc = tc::idesc(1, 128, 128, false);            // BF16 x BF16 -> FP32
    const uint32_t aA = tc::smem_u32(sA), aW2 = tc::smem_u32(sW2), aW3 = tc::smem_u32(sW3);
    uint32_t phase = 0;
    bool failed = false;
    const int64_t ntiles = (a.n + kRows - 1) / kRows;

    auto layer_mma = [&](uint32_t aB) -> bool {
        // all threads: the A buffer is written and visible to the tensor core
        tc::fence_proxy_async_smem();
        tc::tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < kHid / 16; ++ks)
                tc::mma<false>(tmem, tc::sdesc(aA + ks * 256, 128, 2048),
                               tc::sdesc(aB + ks * 256, 128, 2048), idesc, ks > 0 ? 1u : 0u);
            tc::mma_commit(bar);
        }
        const bool ok = tc::mbar_wait_bounded(bar, phase, kWaitNs);
        phase ^= 1;
        tc::tc_fence_after();
        return ok;
    };

    for (int64_t t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
        const int64_t row = t * kRows + tid;
        // ---- layer 1 on the CUDA cores
        float x[kIn];
#pragma unroll
        for (int f = 0; f < kIn; ++f) x[f] = row < a.n ? a.X[row * kIn + f] : 0.f;
#pragma unroll 1
        for (int k8 = 0; k8 < kHid; k8 += 8) {
            float h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float *wr = sW1 + (k8 + j) * kIn;
                float z = sB1[k8 + j];
#pragma unroll
                for (int f = 0; f < kIn; ++f) z = fmaf(wr[f], x[f], z);
                h[j] = silu_fast(z);
            }
            *reinterpret_cast<uint4 *>(sA + cm_offset(tid, k8)) =
                make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]),
                           pack_bf16(h[6], h[7]));
        }
        // ---- layers 2 and 3 on the tensor cores
        float out = b4;
        for (int layer = 0; layer < 2 && !failed; ++layer) {
            if (!layer_mma(layer == 0 ? aW2 : aW3)) *sfail = 1;
            __syncthreads();
            if (*sfail) {
                failed = true;
                break;
            }
            const float *bias = layer == 0 ? sB2 : sB3;
#pragma unroll 1
            for (int c0 = 0; c0 < kHid; c0 += 16) {
                float v[16];
                tc::tmem_ld16(trow + (uint32_t)c0, v);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = silu_fast(v[j] + bias[c0 + j]);
                if (layer == 0) {
                    *reinterpret_cast<uint4 *>(sA + cm_offset(tid, c0)) =
                        make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                   pack_bf16(v[6], v[7]));
                    *reinterpret_cast<uint4 *>(sA + cm_offset(tid, c0 + 8)) =
                        make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]),
                                   pack_bf16(v[12], v[13]), pack_bf16(v[14], v[15]));
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) out = fmaf(sW4[c0 + j], v[j], out);
                }
            }
            // the accumulator is read: the next MMA may overwrite it
            tc::tc_fence_before();
        }
        if (!failed && row < a.n) a.y[row] = out;
        __syncthreads();
    }
    if (failed) {
        // let the MMA whose wait gave up finish before the TMEM is released (its parity is
        // the one before the flip in layer_mma)
        tc::mbar_wait_bounded(bar, phase ^ 1u, kWaitNs);
        if (tid == 0) atomicAdd(a.err, 1);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

size_t infer_smem() {
    return 3 * (size_t)kTileBytes + sizeof(float) * (kHid * kIn + 4 * kHid + 2) + 64;
}

}  // namespace

// y[n] = network(X[n][9]) on the tensor cores (BF16 activations between layers).  Returns the
// number of CTAs that timed out (0 on success).
int mlp_forward_tc(epwi_ctx *c, int64_t n, const float *X, float *y, int *err_dev) {
    if (n <= 0) return 0;
    MlpState &m = *c->mlp;
    static bool attr = false;
    const size_t sm = infer_smem();
    if (!attr) {
        EPWI_CUDA(cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr = true;
    }
    int nsm = 0;
    EPWI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    const int64_t ntiles = (n + kRows - 1) / kRows;
    const int grid = (int)std::min<int64_t>(ntiles, 2 * (int64_t)nsm);
    MlpTcArgs a{n, X, y, m.wbf.as<uint16_t>(), m.w.as<float>(), err_dev};
    k_mlp_infer_tc<<<grid, kRows, sm, c->stream>>>(a);
    EPWI_CHECK_LAUNCH();
    return 0;
}
