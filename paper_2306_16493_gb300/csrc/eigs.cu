// Interpolated electrons and phonons on the full grid (Sec. II B, Eqs. 4-6; Sec. III A
// preprocessing): H(k) and D(q) Fourier sums with exact integer phase reduction, FP64
// cyclic complex Jacobi, band velocities and phonon displacement vectors.
//
// One thread owns one grid point.  Each point is diagonalised once (Nk + Nq solves); the
// scattering loops gather V(k+q), u(q) from these tables instead of re-diagonalising per
// pair.
#include "epwi_internal.cuh"
#include "jacobi.cuh"

namespace {

__global__ void k_phase_tables(int L, double2 *ph64, float2 *ph32) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= L) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)L, &s, &c);   // e^{2 pi i m / L}
    ph64[m] = make_double2(c, s);
    ph32[m] = make_float2((float)c, (float)s);
}

// Electrons: eps (ascending), V (columns), velocities, FP32 copies.
template <int WMAX>
__global__ void __launch_bounds__(128) k_eig_el(GridInfo g, int64_t nk, int W, int nR,
                                                const int *__restrict__ R,
                                                const double *__restrict__ Rcart,
                                                const double2 *__restrict__ Hw,
                                                const double2 *__restrict__ ph,
                                                double *__restrict__ eps, float *__restrict__ eps32,
                                                double2 *__restrict__ Vout,
                                                float2 *__restrict__ V32,
                                                double *__restrict__ vel, int *__restrict__ flag) {
    int64_t ik = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ik >= nk) return;
    int i1, i2, i3;
    grid_coords(g, ik, i1, i2, i3);
    const int a1 = (int)((int64_t)i1 * g.s1 % g.L), a2 = (int)((int64_t)i2 * g.s2 % g.L),
              a3 = (int)((int64_t)i3 * g.s3 % g.L);
    double2 A[WMAX * WMAX], Vm[WMAX * WMAX];
    const int WW = W * W;
    for (int e = 0; e < WW; ++e) A[e] = make_double2(0, 0);
    for (int r = 0; r < nR; ++r) {
        const double2 p = ph[phase_index(a1, a2, a3, R[3 * r], R[3 * r + 1], R[3 * r + 2], g.L)];
        const double2 *h = Hw + (size_t)r * WW;
        for (int e = 0; e < WW; ++e) A[e] = cfma(p, h[e], A[e]);
    }
    double w[WMAX];
    int ok = jacobi_hermitian<WMAX>(A, Vm, W, w);
    if (!ok) atomicAdd(flag, 1);
    for (int n = 0; n < W; ++n) {
        eps[ik * W + n] = w[n];
        eps32[ik * W + n] = (float)w[n];
    }
    for (int e = 0; e < WW; ++e) {
        Vout[ik * WW + e] = Vm[e];
        V32[ik * WW + e] = make_float2((float)Vm[e].x, (float)Vm[e].y);
    }
    // v_n,a = (1/hbar) Re[V^dag (sum_R w_R i R_a e^{ik.R} H(R)) V]_nn, one axis at a time
    for (int ax = 0; ax < 3; ++ax) {
        for (int e = 0; e < WW; ++e) A[e] = make_double2(0, 0);
        for (int r = 0; r < nR; ++r) {
            const double2 p = ph[phase_index(a1, a2, a3, R[3 * r], R[3 * r + 1], R[3 * r + 2], g.L)];
            const double ra = Rcart[3 * r + ax];
            const double2 ip = make_double2(-ra * p.y, ra * p.x);   // i R_a e^{ik.R}
            const double2 *h = Hw + (size_t)r * WW;
            for (int e = 0; e < WW; ++e) A[e] = cfma(ip, h[e], A[e]);
        }
        for (int n = 0; n < W; ++n) {
            double acc = 0;
            for (int i = 0; i < W; ++i) {
                double2 t = make_double2(0, 0);
                for (int j = 0; j < W; ++j) t = cfma(A[i * W + j], Vm[j * W + n], t);
                acc += Vm[i * W + n].x * t.x + Vm[i * W + n].y * t.y;   // Re(conj(V_in) t)
            }
            vel[(ik * W + n) * 3 + ax] = acc / epc::kHbarEVs * 1e-10;
        }
    }
}

// Phonons: hbar*omega, u = e (hbar^2 / (2 m hbar omega))^{1/2}, FP32 copies.
template <int NMAX>
__global__ void __launch_bounds__(128) k_eig_ph(GridInfo g, int64_t nq, int Nm, int nR,
                                                const int *__restrict__ R,
                                                const double *__restrict__ Phiw,
                                                const double *__restrict__ mode_mass,
                                                const double2 *__restrict__ ph, double omega_min,
                                                double *__restrict__ hw, float *__restrict__ hwmax32,
                                                float *__restrict__ hw32,
                                                double2 *__restrict__ uout,
                                                float2 *__restrict__ u32, int *__restrict__ flag) {
    int64_t iq = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (iq >= nq) return;
    int i1, i2, i3;
    grid_coords(g, iq, i1, i2, i3);
    const int a1 = (int)((int64_t)i1 * g.s1 % g.L), a2 = (int)((int64_t)i2 * g.s2 % g.L),
              a3 = (int)((int64_t)i3 * g.s3 % g.L);
    double2 A[NMAX * NMAX], E[NMAX * NMAX];
    const int MM = Nm * Nm;
    for (int e = 0; e < MM; ++e) A[e] = make_double2(0, 0);
    for (int r = 0; r < nR; ++r) {
        const double2 p = ph[phase_index(a1, a2, a3, R[3 * r], R[3 * r + 1], R[3 * r + 2], g.L)];
        const double *f = Phiw + (size_t)r * MM;
        for (int e = 0; e < MM; ++e) {
            A[e].x = fma(p.x, f[e], A[e].x);
            A[e].y = fma(p.y, f[e], A[e].y);
        }
    }
    double lam[NMAX];
    int ok = jacobi_hermitian<NMAX>(A, E, Nm, lam);
    if (!ok) atomicAdd(flag, 1);
    float wmax = -1.f;
    for (int nu = 0; nu < Nm; ++nu) {
        const double l = lam[nu];
        const double w = (l >= 0 ? 1.0 : -1.0) * sqrt(fabs(l) * epc::kHbar2AmuA2);
        hw[iq * Nm + nu] = w;
        const bool keep = w >= omega_min;
        hw32[iq * Nm + nu] = keep ? (float)w : -1.0f;
        if (keep) wmax = fmaxf(wmax, (float)w);
        for (int m = 0; m < Nm; ++m) {
            double amp = keep ? sqrt(epc::kHbar2AmuA2 / (2.0 * mode_mass[m] * w)) : 0.0;
            double2 v = make_double2(E[m * Nm + nu].x * amp, E[m * Nm + nu].y * amp);
            uout[iq * MM + m * Nm + nu] = v;
            u32[iq * MM + m * Nm + nu] = make_float2((float)v.x, (float)v.y);
        }
    }
    hwmax32[iq] = wmax;
}

}  // namespace

GridInfo make_grid_info(const epwi_ctx *c) {
    GridInfo g;
    g.n1 = c->ng[0];
    g.n2 = c->ng[1];
    g.n3 = c->ng[2];
    g.L = c->L;
    g.s1 = c->L / c->ng[0];
    g.s2 = c->L / c->ng[1];
    g.s3 = c->L / c->ng[2];
    return g;
}

void launch_phase_tables(epwi_ctx *c) {
    c->ph64.ensure(sizeof(double2) * c->L);
    c->ph32.ensure(sizeof(float2) * c->L);
    k_phase_tables<<<(c->L + 127) / 128, 128, 0, c->stream>>>(c->L, c->ph64.as<double2>(),
                                                               c->ph32.as<float2>());
    EPWI_CHECK_LAUNCH();
}

void launch_eigs(epwi_ctx *c) {
    const int64_t nk = c->nk;
    const int W = c->nw, Nm = c->nm;
    c->eps.ensure(sizeof(double) * nk * W);
    c->eps32.ensure(sizeof(float) * nk * W);
    c->V.ensure(sizeof(double2) * nk * W * W);
    c->V32.ensure(sizeof(float2) * nk * W * W);
    c->vel.ensure(sizeof(double) * nk * W * 3);
    c->hw.ensure(sizeof(double) * nk * Nm);
    c->hwmax32.ensure(sizeof(float) * nk);
    c->hw32.ensure(sizeof(float) * nk * Nm);
    c->u.ensure(sizeof(double2) * nk * Nm * Nm);
    c->u32.ensure(sizeof(float2) * nk * Nm * Nm);
    c->eig_flag.ensure(sizeof(int) * 2);
    EPWI_CUDA(cudaMemsetAsync(c->eig_flag.p, 0, sizeof(int) * 2, c->stream));
    GridInfo g = make_grid_info(c);
    const int bs = 128;
    const unsigned nb = (unsigned)((nk + bs - 1) / bs);
#define EL_ARGS                                                                              \
    g, nk, W, c->nRe, c->Re.as<int>(), c->Rcart.as<double>(), c->Hw.as<double2>(),            \
        c->ph64.as<double2>(), c->eps.as<double>(), c->eps32.as<float>(), c->V.as<double2>(), \
        c->V32.as<float2>(), c->vel.as<double>(), c->eig_flag.as<int>()
    if (W <= 1) k_eig_el<1><<<nb, bs, 0, c->stream>>>(EL_ARGS);
    else if (W <= 4) k_eig_el<4><<<nb, bs, 0, c->stream>>>(EL_ARGS);
    else if (W <= 8) k_eig_el<8><<<nb, bs, 0, c->stream>>>(EL_ARGS);
    else if (W <= 16) k_eig_el<16><<<nb, bs, 0, c->stream>>>(EL_ARGS);
    else k_eig_el<24><<<nb, bs, 0, c->stream>>>(EL_ARGS);
#undef EL_ARGS
    EPWI_CHECK_LAUNCH();
#define PH_ARGS                                                                             \
    g, nk, Nm, c->nRp, c->Rp.as<int>(), c->Phiw.as<double>(), c->mode_mass.as<double>(),     \
        c->ph64.as<double2>(), c->opt.omega_min_eV, c->hw.as<double>(), c->hwmax32.as<float>(), \
        c->hw32.as<float>(),                                                                   \
        c->u.as<double2>(), c->u32.as<float2>(), c->eig_flag.as<int>() + 1
    if (Nm <= 3) k_eig_ph<3><<<nb, bs, 0, c->stream>>>(PH_ARGS);
    else if (Nm <= 6) k_eig_ph<6><<<nb, bs, 0, c->stream>>>(PH_ARGS);
    else if (Nm <= 12) k_eig_ph<12><<<nb, bs, 0, c->stream>>>(PH_ARGS);
    else k_eig_ph<18><<<nb, bs, 0, c->stream>>>(PH_ARGS);
#undef PH_ARGS
    EPWI_CHECK_LAUNCH();
}
