// Occupations and transport reductions (Sec. II C): Fermi-Dirac and Bose-Einstein tables,
// sigma (Eq. 12 with F = v tau), conduction-electron density for the chemical potential
// (Sec. III A), band extrema.  All reductions are two-pass with a fixed block count and a
// fixed tree order, so results are bitwise reproducible for a given input size.
#include "epwi_internal.cuh"
#include "scatter.cuh"

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 1024;

__device__ __forceinline__ double fermi(double e, double mu, double kT) {
    const double x = (e - mu) / kT;
    const double ex = exp(-fabs(x));
    return x > 0 ? ex / (1.0 + ex) : 1.0 / (1.0 + ex);
}

template <int NV>
__device__ void block_sum(double (&v)[NV], double *sm) {
    // sm: [NV][kRedThreads]
    for (int j = 0; j < NV; ++j) sm[j * kRedThreads + threadIdx.x] = v[j];
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int j = 0; j < NV; ++j)
                sm[j * kRedThreads + threadIdx.x] += sm[j * kRedThreads + threadIdx.x + s];
        __syncthreads();
    }
    for (int j = 0; j < NV; ++j) v[j] = sm[j * kRedThreads];
    __syncthreads();
}

__global__ void k_occupations(int64_t nk, int W, int Nm, const double *__restrict__ eps,
                              const double *__restrict__ hw, double mu, double kT,
                              double omega_min, double *__restrict__ focc,
                              double *__restrict__ nocc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nk * W) focc[i] = fermi(eps[i], mu, kT);
    if (i < nk * Nm) {
        const double w = hw[i];
        nocc[i] = (w >= omega_min) ? 1.0 / expm1(w / kT) : 0.0;
    }
}

// sigma partial sums: xx yy zz xy xz yz
__global__ void __launch_bounds__(kRedThreads) k_sigma_part(
    int64_t ns, int W, const int *__restrict__ st_k, const int *__restrict__ st_n,
    const double *__restrict__ inv_tau, const double *__restrict__ eps,
    const double *__restrict__ vel, double mu, double kT, double *__restrict__ part) {
    __shared__ double sm[6 * kRedThreads];
    const int64_t per = (ns + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = per * blockIdx.x, b1 = min(ns, b0 + per);
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t s = b0 + threadIdx.x; s < b1; s += blockDim.x) {
        const double r = inv_tau[s];
        if (!(r > 0)) continue;
        const int64_t idx = (int64_t)st_k[s] * W + st_n[s];
        const double f = fermi(eps[idx], mu, kT);
        const double w = f * (1.0 - f) / r;
        const double vx = vel[idx * 3], vy = vel[idx * 3 + 1], vz = vel[idx * 3 + 2];
        v[0] += w * vx * vx;
        v[1] += w * vy * vy;
        v[2] += w * vz * vz;
        v[3] += w * vx * vy;
        v[4] += w * vx * vz;
        v[5] += w * vy * vz;
    }
    block_sum<6>(v, sm);
    if (threadIdx.x == 0)
        for (int j = 0; j < 6; ++j) part[blockIdx.x * 6 + j] = v[j];
}

// Energy moments p = 0, 1, 2 of the SERTA transport sum (Sec. II C, Eqs. 12-14): for each
// state, w = tau f(1-f) and x = eps - mu (eV); sums of w x^p v_a v_b for the six components
// xx yy zz xy xz yz, stored p-major.
__global__ void __launch_bounds__(kRedThreads) k_moments_part(
    int64_t ns, int W, const int *__restrict__ st_k, const int *__restrict__ st_n,
    const double *__restrict__ inv_tau, const double *__restrict__ eps,
    const double *__restrict__ vel, double mu, double kT, double *__restrict__ part) {
    __shared__ double sm[18 * kRedThreads];
    const int64_t per = (ns + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = per * blockIdx.x, b1 = min(ns, b0 + per);
    double v[18];
    for (int j = 0; j < 18; ++j) v[j] = 0;
    for (int64_t s = b0 + threadIdx.x; s < b1; s += blockDim.x) {
        const double r = inv_tau[s];
        if (!(r > 0)) continue;
        const int64_t idx = (int64_t)st_k[s] * W + st_n[s];
        const double f = fermi(eps[idx], mu, kT);
        const double w0 = f * (1.0 - f) / r;
        const double x = eps[idx] - mu;
        const double vx = vel[idx * 3], vy = vel[idx * 3 + 1], vz = vel[idx * 3 + 2];
        const double c[6] = {vx * vx, vy * vy, vz * vz, vx * vy, vx * vz, vy * vz};
        double w = w0;
        for (int p = 0; p < 3; ++p) {
            for (int j = 0; j < 6; ++j) v[p * 6 + j] += w * c[j];
            w *= x;
        }
    }
    block_sum<18>(v, sm);
    if (threadIdx.x == 0)
        for (int j = 0; j < 18; ++j) part[blockIdx.x * 18 + j] = v[j];
}

// Energy moment p of the transport sum with the mean free paths F (iterative BTE): sums of
// f(1-f) x^p v_a F_b over the window states, nine components a-major.
__global__ void __launch_bounds__(kRedThreads) k_moments_F_part(
    int64_t ns, int W, int p, const int *__restrict__ st_k, const int *__restrict__ st_n,
    const double *__restrict__ eps, const double *__restrict__ vel, const double *__restrict__ F,
    double mu, double kT, double *__restrict__ part) {
    __shared__ double sm[9 * kRedThreads];
    const int64_t per = (ns + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = per * blockIdx.x, b1 = min(ns, b0 + per);
    double v[9];
    for (int j = 0; j < 9; ++j) v[j] = 0;
    for (int64_t s = b0 + threadIdx.x; s < b1; s += blockDim.x) {
        const int64_t idx = (int64_t)st_k[s] * W + st_n[s];
        const double f = fermi(eps[idx], mu, kT);
        const double x = eps[idx] - mu;
        double w = f * (1.0 - f);
        for (int q = 0; q < p; ++q) w *= x;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) v[a * 3 + b] += w * vel[idx * 3 + a] * F[s * 3 + b];
    }
    block_sum<9>(v, sm);
    if (threadIdx.x == 0)
        for (int j = 0; j < 9; ++j) part[blockIdx.x * 9 + j] = v[j];
}

template <int NV>
__global__ void __launch_bounds__(kRedThreads) k_final_sum(int nb, const double *__restrict__ part,
                                                           double *__restrict__ out) {
    __shared__ double sm[NV * kRedThreads];
    double v[NV];
    for (int j = 0; j < NV; ++j) v[j] = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int j = 0; j < NV; ++j) v[j] += part[b * NV + j];
    block_sum<NV>(v, sm);
    if (threadIdx.x == 0)
        for (int j = 0; j < NV; ++j) out[j] = v[j];
}

__global__ void __launch_bounds__(kRedThreads) k_density_part(int64_t nk, int W, int nv,
                                                              const double *__restrict__ eps,
                                                              double mu, double kT,
                                                              double *__restrict__ part) {
    __shared__ double sm[kRedThreads];
    const int nc = W - nv;
    const int64_t n = nk * nc;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = per * blockIdx.x, b1 = min(n, b0 + per);
    double v[1] = {0};
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const int64_t k = i / nc;
        const int b = nv + (int)(i % nc);
        v[0] += fermi(eps[k * W + b], mu, kT);
    }
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

__global__ void __launch_bounds__(kRedThreads) k_minmax_part(const double *__restrict__ x,
                                                             int64_t n, int64_t stride,
                                                             int64_t off, double *__restrict__ part) {
    __shared__ double smn[kRedThreads], smx[kRedThreads];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = per * blockIdx.x, b1 = min(n, b0 + per);
    double mn = INFINITY, mx = -INFINITY;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const double v = x[i * stride + off];
        mn = fmin(mn, v);
        mx = fmax(mx, v);
    }
    smn[threadIdx.x] = mn;
    smx[threadIdx.x] = mx;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + s]);
            smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = smn[0];
        part[2 * blockIdx.x + 1] = smx[0];
    }
}

__global__ void k_minmax_final(int nb, const double *__restrict__ part, double *__restrict__ out) {
    if (threadIdx.x != 0) return;
    double mn = INFINITY, mx = -INFINITY;
    for (int b = 0; b < nb; ++b) {
        mn = fmin(mn, part[2 * b]);
        mx = fmax(mx, part[2 * b + 1]);
    }
    out[0] = mn;
    out[1] = mx;
}

int red_blocks(int64_t n) {
    int64_t b = (n + 4 * kRedThreads - 1) / (4 * kRedThreads);
    if (b < 1) b = 1;
    if (b > kRedMaxBlocks) b = kRedMaxBlocks;
    return (int)b;
}

}  // namespace

void occupation_tables(epwi_ctx *c) {
    const int64_t nk = c->nk;
    c->focc.ensure(sizeof(double) * nk * c->nw);
    c->nocc.ensure(sizeof(double) * nk * c->nm);
    const int64_t n = nk * (c->nw > c->nm ? c->nw : c->nm);
    k_occupations<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
        nk, c->nw, c->nm, c->eps.as<double>(), c->hw.as<double>(), c->mu, epc::kKbEVK * c->T,
        c->opt.omega_min_eV, c->focc.as<double>(), c->nocc.as<double>());
    EPWI_CHECK_LAUNCH();
    if (c->opt.precision != EPWI_FP64) tc_tables(c);
}

double device_reduce_minmax(epwi_ctx *c, const double *x, int64_t n, int64_t stride, int64_t off,
                            bool want_max) {
    const int nb = red_blocks(n);
    c->red_tmp.ensure(sizeof(double) * (2 * nb + 16));
    double *part = c->red_tmp.as<double>();
    double *out = part + 2 * nb;
    k_minmax_part<<<nb, kRedThreads, 0, c->stream>>>(x, n, stride, off, part);
    EPWI_CHECK_LAUNCH();
    k_minmax_final<<<1, 32, 0, c->stream>>>(nb, part, out);
    EPWI_CHECK_LAUNCH();
    double h[2];
    EPWI_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    return want_max ? h[1] : h[0];
}

double carrier_density(epwi_ctx *c, double T, double mu, int nv) {
    const int64_t n = c->nk * (c->nw - nv);
    const int nb = red_blocks(n);
    c->red_tmp.ensure(sizeof(double) * (nb + 16));
    double *part = c->red_tmp.as<double>();
    double *out = part + nb;
    k_density_part<<<nb, kRedThreads, 0, c->stream>>>(c->nk, c->nw, nv, c->eps.as<double>(), mu,
                                                      epc::kKbEVK * T, part);
    EPWI_CHECK_LAUNCH();
    k_final_sum<1><<<1, kRedThreads, 0, c->stream>>>(nb, part, out);
    EPWI_CHECK_LAUNCH();
    double h;
    EPWI_CUDA(cudaMemcpyAsync(&h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    // (2 / (N_k V)) sum f, per cm^3
    return 2.0 * h / ((double)c->nk * c->volume * 1e-24);
}

void conductivity(epwi_ctx *c, double sigma[9]) {
    const int64_t ns = c->nstates;
    const int nb = red_blocks(ns);
    c->red_tmp.ensure(sizeof(double) * (6 * nb + 16));
    double *part = c->red_tmp.as<double>();
    double *out = part + 6 * nb;
    const double kT = epc::kKbEVK * c->T;
    k_sigma_part<<<nb, kRedThreads, 0, c->stream>>>(ns, c->nw, c->st_k.as<int>(), c->st_n.as<int>(),
                                                    c->inv_tau.as<double>(), c->eps.as<double>(),
                                                    c->vel.as<double>(), c->mu, kT, part);
    EPWI_CHECK_LAUNCH();
    k_final_sum<6><<<1, kRedThreads, 0, c->stream>>>(nb, part, out);
    EPWI_CHECK_LAUNCH();
    double h[6];
    EPWI_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    const double kT_J = kT * epc::kECharge;
    const double pref = 2.0 * epc::kECharge * epc::kECharge / ((double)c->nk * c->volume * 1e-30 * kT_J);
    const double s[9] = {h[0], h[3], h[4], h[3], h[1], h[5], h[4], h[5], h[2]};
    for (int i = 0; i < 9; ++i) sigma[i] = pref * s[i];
}

// sum over states of tau f(1-f) (eps - mu)^p v_a v_b, p = 0, 1, 2 (eV^p m^2/s), as three
// symmetric 3x3 tensors m[p][9].
void transport_moments(epwi_ctx *c, double m[3][9]) {
    const int64_t ns = c->nstates;
    const int nb = red_blocks(ns);
    c->red_tmp.ensure(sizeof(double) * (18 * nb + 32));
    double *part = c->red_tmp.as<double>();
    double *out = part + 18 * nb;
    const double kT = epc::kKbEVK * c->T;
    k_moments_part<<<nb, kRedThreads, 0, c->stream>>>(ns, c->nw, c->st_k.as<int>(), c->st_n.as<int>(),
                                                      c->inv_tau.as<double>(), c->eps.as<double>(),
                                                      c->vel.as<double>(), c->mu, kT, part);
    EPWI_CHECK_LAUNCH();
    k_final_sum<18><<<1, kRedThreads, 0, c->stream>>>(nb, part, out);
    EPWI_CHECK_LAUNCH();
    double h[18];
    EPWI_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    for (int p = 0; p < 3; ++p) {
        const double *q = h + 6 * p;
        const double t[9] = {q[0], q[3], q[4], q[3], q[1], q[5], q[4], q[5], q[2]};
        for (int i = 0; i < 9; ++i) m[p][i] = t[i];
    }
}

// Moments p = 0, 1, 2 of the transport sum with v tau replaced by the mean free paths F
// (iterative BTE): m[p][a*3+b] = sum f(1-f) (eps - mu)^p v_a F_b.
void transport_moments_F(epwi_ctx *c, const double *F, double m[3][9]) {
    const int64_t ns = c->nstates;
    const int nb = red_blocks(ns);
    c->red_tmp.ensure(sizeof(double) * (9 * nb + 32));
    double *part = c->red_tmp.as<double>();
    double *out = part + 9 * nb;
    const double kT = epc::kKbEVK * c->T;
    for (int p = 0; p < 3; ++p) {
        k_moments_F_part<<<nb, kRedThreads, 0, c->stream>>>(ns, c->nw, p, c->st_k.as<int>(),
                                                            c->st_n.as<int>(), c->eps.as<double>(),
                                                            c->vel.as<double>(), F, c->mu, kT, part);
        EPWI_CHECK_LAUNCH();
        k_final_sum<9><<<1, kRedThreads, 0, c->stream>>>(nb, part, out);
        EPWI_CHECK_LAUNCH();
        EPWI_CUDA(cudaMemcpyAsync(m[p], out, sizeof(double) * 9, cudaMemcpyDeviceToHost, c->stream));
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
    }
}
