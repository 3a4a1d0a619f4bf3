// Symmetry-reduced k grids (Sec. III A: the CPU flow reduces the k grid with the crystal's
// symmetry before the scattering loops).
//
// A crystal invariant under a point group G has eps(S k) = eps(k), omega(S q) = omega(q) and
// 1/tau_n(S k) = 1/tau_n(k) for every operation S (k -> K_S k on the grid index vectors).  The
// rates are then computed once per star of window k-points, for its representative (the
// lowest grid index of the star), and copied to every member.  sigma sums over all window
// states with each state's own velocity, so it needs no rotation of tensors.
//
// Every member of a star takes its representative's band window, so the states of a star
// agree exactly (eps may differ in the last bits between separately diagonalised points).
#include <algorithm>
#include <array>
#include <cstring>
#include <string>

#include "epwi_internal.cuh"

namespace {

constexpr int kMaxOps = 48;

struct SymOps {
    int n;
    int m[kMaxOps][9];
};

__device__ __forceinline__ int64_t apply_op(const int *m, int i1, int i2, int i3, int N) {
    int a[3];
    for (int r = 0; r < 3; ++r) {
        int t = (m[3 * r] * i1 + m[3 * r + 1] * i2 + m[3 * r + 2] * i3) % N;
        a[r] = t < 0 ? t + N : t;
    }
    return ((int64_t)a[0] * N + a[1]) * N + a[2];
}

// rep[k] = the lowest grid index of k's star
__global__ void k_sym_rep(int64_t nk, int N, SymOps ops, int *__restrict__ rep) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    const int i3 = (int)(k % N), i2 = (int)((k / N) % N), i1 = (int)(k / ((int64_t)N * N));
    int64_t best = k;
    for (int o = 0; o < ops.n; ++o) best = min(best, apply_op(ops.m[o], i1, i2, i3, N));
    rep[k] = (int)best;
}

// max over k and operations of |eps(S k) - eps(k)| and |omega(S k) - omega(k)| (bit patterns of
// non-negative doubles order like the values)
__global__ void k_sym_check(int64_t nk, int N, int W, int Nm, SymOps ops, const double *__restrict__ eps,
                            const double *__restrict__ hw, unsigned long long *__restrict__ red) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    const int i3 = (int)(k % N), i2 = (int)((k / N) % N), i1 = (int)(k / ((int64_t)N * N));
    double de = 0, dw = 0;
    for (int o = 0; o < ops.n; ++o) {
        const int64_t j = apply_op(ops.m[o], i1, i2, i3, N);
        for (int n = 0; n < W; ++n) de = fmax(de, fabs(eps[j * W + n] - eps[k * W + n]));
        for (int v = 0; v < Nm; ++v) dw = fmax(dw, fabs(hw[j * Nm + v] - hw[k * Nm + v]));
    }
    if (de > 0) atomicMax(&red[0], (unsigned long long)__double_as_longlong(de));
    if (dw > 0) atomicMax(&red[1], (unsigned long long)__double_as_longlong(dw));
}

// every k takes the band window of its representative (in place: a representative keeps its own)
__global__ void k_sym_window(int64_t nk, const int *__restrict__ rep, int *__restrict__ lo, int *__restrict__ cnt) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    const int r = rep[k];
    if (r == (int)k) return;
    lo[k] = lo[r];
    cnt[k] = cnt[r];
}

__global__ void k_sym_kpos(int64_t nkp, const int *__restrict__ kpts, int *__restrict__ kpos) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nkp) kpos[kpts[p]] = (int)p;
}

// 1/tau of every window state from its star's representative
__global__ void k_sym_expand(int64_t ns, const int *__restrict__ st_k, const int *__restrict__ st_n,
                             const int *__restrict__ rep, const int *__restrict__ kpos_rep,
                             const int64_t *__restrict__ kp_state_rep, const int *__restrict__ lo,
                             const double *__restrict__ inv_tau_rep, double *__restrict__ inv_tau) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const int r = rep[st_k[s]];
    inv_tau[s] = inv_tau_rep[kp_state_rep[kpos_rep[r]] + (st_n[s] - lo[r])];
}

SymOps device_ops(const epwi_ctx *c) {
    SymOps o;
    o.n = (int)(c->sym_ops.size() / 9);
    std::memcpy(o.m, c->sym_ops.data(), sizeof(int) * c->sym_ops.size());
    return o;
}

}  // namespace

// Representatives of the current grid and a check that the crystal has the symmetry.
void sym_prepare(epwi_ctx *c) {
    const int N = c->ng[0];
    EPWI_REQUIRE(c->ng[1] == N && c->ng[2] == N, EPWI_EUNSUPPORTED,
                 "symmetry-reduced grids need an N x N x N grid");
    const SymOps ops = device_ops(c);
    const int64_t nk = c->nk;
    const unsigned nb = (unsigned)((nk + 255) / 256);
    c->sym_rep.ensure(sizeof(int) * nk);
    k_sym_rep<<<nb, 256, 0, c->stream>>>(nk, N, ops, c->sym_rep.as<int>());
    EPWI_CHECK_LAUNCH();
    DevBuf red;
    unsigned long long h[2] = {0, 0};
    try {
        red.ensure(sizeof(unsigned long long) * 2);
        EPWI_CUDA(cudaMemsetAsync(red.p, 0, sizeof(unsigned long long) * 2, c->stream));
        k_sym_check<<<nb, 256, 0, c->stream>>>(nk, N, c->nw, c->nm, ops, c->eps.as<double>(), c->hw.as<double>(),
                                              red.as<unsigned long long>());
        EPWI_CHECK_LAUNCH();
        EPWI_CUDA(cudaMemcpyAsync(h, red.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
    } catch (...) {
        red.release();
        throw;
    }
    red.release();
    double de, dw;
    std::memcpy(&de, &h[0], sizeof(double));
    std::memcpy(&dw, &h[1], sizeof(double));
    EPWI_REQUIRE(de <= 1e-9 * std::max(1.0, c->eabs_max) && dw <= 1e-9, EPWI_EINVAL,
                 "the crystal is not invariant under the symmetry operations (max |eps(Sk) - eps(k)| = " +
                     std::to_string(de) + " eV, max |omega(Sq) - omega(q)| = " + std::to_string(dw) + " eV)");
}

// After the rates of the representatives: the full window (every member of every star, each
// with its representative's bands) and its 1/tau.
void sym_expand(epwi_ctx *c) {
    const int64_t nk = c->nk;
    const unsigned nb = (unsigned)((nk + 255) / 256);
    DevBuf kpts_r, kp_state_r, inv_tau_r, kpos;
    std::swap(kpts_r, c->kpts);
    std::swap(kp_state_r, c->kp_state);
    std::swap(inv_tau_r, c->inv_tau);
    const int64_t nkp_r = c->nkp;
    auto done = [&] {
        kpts_r.release();
        kp_state_r.release();
        inv_tau_r.release();
        kpos.release();
    };
    try {
        kpos.ensure(sizeof(int) * nk);
        if (nkp_r > 0) {
            k_sym_kpos<<<(unsigned)((nkp_r + 255) / 256), 256, 0, c->stream>>>(nkp_r, kpts_r.as<int>(), kpos.as<int>());
            EPWI_CHECK_LAUNCH();
        }
        k_sym_window<<<nb, 256, 0, c->stream>>>(nk, c->sym_rep.as<int>(), c->win_lo.as<int>(), c->win_n.as<int>());
        EPWI_CHECK_LAUNCH();
        if (c->vel_state == 1) c->vel_state = 0;  // members took their representatives' windows
        ensure_velocities(c, false);
        window_lists(c, nullptr);
        if (c->nstates > 0) {
            k_sym_expand<<<(unsigned)((c->nstates + 255) / 256), 256, 0, c->stream>>>(
                c->nstates, c->st_k.as<int>(), c->st_n.as<int>(), c->sym_rep.as<int>(), kpos.as<int>(),
                kp_state_r.as<int64_t>(), c->win_lo.as<int>(), inv_tau_r.as<double>(), c->inv_tau.as<double>());
            EPWI_CHECK_LAUNCH();
        }
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
    } catch (...) {
        done();
        throw;
    }
    done();
}

extern "C" epwi_status epwi_set_symmetry(epwi_ctx *c, int32_t nops, const int32_t *kops) {
    if (!c) return EPWI_EINVAL;
    if (nops < 0 || nops > kMaxOps || (nops > 0 && !kops)) {
        c->err = "nops must be in [0, 48] and kops non-NULL";
        return EPWI_EINVAL;
    }
    std::vector<int> ops(kops, kops + 9 * (size_t)nops);
    // the operations must form a group (closure, identity) of unimodular integer matrices
    auto mul = [&](int a, int b) {
        std::array<int, 9> r{};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) r[3 * i + j] += ops[9 * a + 3 * i + k] * ops[9 * b + 3 * k + j];
        return r;
    };
    auto find = [&](const std::array<int, 9> &m) {
        for (int o = 0; o < nops; ++o)
            if (std::equal(m.begin(), m.end(), ops.begin() + 9 * o)) return true;
        return false;
    };
    if (nops > 0) {
        const std::array<int, 9> id{1, 0, 0, 0, 1, 0, 0, 0, 1};
        bool ok = find(id);
        for (int a = 0; a < nops && ok; ++a)
            for (int b = 0; b < nops && ok; ++b) ok = find(mul(a, b));
        if (!ok) {
            c->err = "the symmetry operations do not form a group (identity and closure)";
            return EPWI_EINVAL;
        }
    }
    c->sym_ops = ops;
    c->err.clear();
    return EPWI_OK;
}
