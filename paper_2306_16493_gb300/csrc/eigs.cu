// Interpolated electrons and phonons on the full grid (Sec. II B, Eqs. 4-6; Sec. III A
// preprocessing): H(k) and D(q) Fourier sums with exact integer phase reduction, FP64
// cyclic complex Jacobi, band velocities and phonon displacement vectors.
//
// One thread owns one grid point.  Each point is diagonalised once (Nk + Nq solves); the
// scattering loops gather V(k+q), u(q) from these tables instead of re-diagonalising per
// pair.
#include <algorithm>
#include <utility>
#include <vector>

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

// Sum-factorised Fourier builds (Eqs. 4-5 reordered, exact in real arithmetic).  With the
// R-set embedded in its bounding cube [-r, r]^3 (absent vectors carry zero), e^{ik.R} =
// e1(k1, n1) e2(k2, n2) e3(k3, n3) and X(k) = sum_n1 e1 sum_n2 e2 sum_n3 e3 X(n) is done in
// three stages, each shared by every grid point that needs it: axis 3 per (n1, n2, k3), axis 2
// per (n1, k2, k3), axis 1 inside the eigensolve kernels per k.  For the band velocities the
// n_b-weighted sums sum_n n_b e^{ik.R} H(R) ride along (VEL): dH/dk_a = i sum_b A_ba S_b with
// R_cart = sum_b n_b a_b.  E = entries per matrix; all FP64.
//   T[s][n1][n2][k3][e]:  s = 0: sum_n3 e3 X;   s = 1 (VEL): sum_n3 n3 e3 X
//   U[s][n1][k2][k3][e]:  s = 0: sum_n2 e2 T0;  s = 1: sum_n2 n2 e2 T0;  s = 2: sum_n2 e2 T1
__device__ __forceinline__ double2 axis_ph(const double2 *ph, int n, int a, int L) {
    int t = (n * a) % L;
    if (t < 0) t += L;
    return ph[t];
}

template <bool VEL>
__global__ void k_fac_axis3(int D, int rc, int N3, int s3, int L, int E, const double2 *__restrict__ Xc,
                            const double2 *__restrict__ ph, double2 *__restrict__ T) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)D * D * N3 * E;
    if (idx >= total) return;
    const int e = (int)(idx % E);
    const int64_t t = idx / E;
    const int k3 = (int)(t % N3);
    const int r12 = (int)(t / N3);
    const int a3 = (int)((int64_t)k3 * s3 % L);
    double2 s0 = make_double2(0, 0), s1 = make_double2(0, 0);
    for (int j = 0; j < D; ++j) {
        const int n3 = j - rc;
        const double2 v = cmul(axis_ph(ph, n3, a3, L), Xc[((int64_t)r12 * D + j) * E + e]);
        s0 = cadd(s0, v);
        if (VEL) s1 = make_double2(fma((double)n3, v.x, s1.x), fma((double)n3, v.y, s1.y));
    }
    T[((int64_t)r12 * N3 + k3) * E + e] = s0;
    if (VEL) T[(((int64_t)D * D + r12) * N3 + k3) * E + e] = s1;
}

template <bool VEL>
__global__ void k_fac_axis2(int D, int rc, int N2, int N3, int s2, int L, int E, const double2 *__restrict__ T,
                            const double2 *__restrict__ ph, double2 *__restrict__ U) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t plane = (int64_t)N2 * N3;
    const int64_t total = (int64_t)D * plane * E;
    if (idx >= total) return;
    const int e = (int)(idx % E);
    int64_t t = idx / E;
    const int k3 = (int)(t % N3);
    t /= N3;
    const int k2 = (int)(t % N2);
    const int r1 = (int)(t / N2);
    const int a2 = (int)((int64_t)k2 * s2 % L);
    double2 u0 = make_double2(0, 0), u1 = make_double2(0, 0), u2 = make_double2(0, 0);
    for (int j = 0; j < D; ++j) {
        const int n2 = j - rc;
        const double2 p = axis_ph(ph, n2, a2, L);
        const double2 v = cmul(p, T[(((int64_t)r1 * D + j) * N3 + k3) * E + e]);
        u0 = cadd(u0, v);
        if (VEL) {
            u1 = make_double2(fma((double)n2, v.x, u1.x), fma((double)n2, v.y, u1.y));
            u2 = cadd(u2, cmul(p, T[((((int64_t)D + r1) * D + j) * N3 + k3) * E + e]));
        }
    }
    const int64_t o = ((int64_t)r1 * plane + (int64_t)k2 * N3 + k3) * E + e;
    U[o] = u0;
    if (VEL) {
        U[(int64_t)D * plane * E + o] = u1;
        U[2 * (int64_t)D * plane * E + o] = u2;
    }
}

// The axis-2 stage output U[s][n1][k2 k3][e] of a factorised build (sources s = 0, 1, 2).
struct FacDesc {
    const double2 *U;
    int D, rc;
    int64_t plane;                   // N2 N3
};
struct Lattice {
    double a[3][3];                  // rows a_1, a_2, a_3 (A)
};

// Electrons: eps (ascending), V (columns), velocities, FP32 copies.  FAC: H(k) and dH/dk from
// the factorised stages (fac, lattice rows lat) instead of direct sums over the R-set.
template <int WMAX, bool FAC>
__global__ void __launch_bounds__(128) k_eig_el(GridInfo g, int64_t nk, int W, int nR,
                                                const int *__restrict__ R,
                                                const double *__restrict__ Rcart,
                                                const double2 *__restrict__ Hw,
                                                const double2 *__restrict__ ph,
                                                double *__restrict__ eps, float *__restrict__ eps32,
                                                double2 *__restrict__ Vout,
                                                float2 *__restrict__ V32,
                                                double *__restrict__ vel, int *__restrict__ flag,
                                                FacDesc fac, Lattice lat, int do_vel) {
    int64_t ik = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ik >= nk) return;
    int i1, i2, i3;
    grid_coords(g, ik, i1, i2, i3);
    const int a1 = (int)((int64_t)i1 * g.s1 % g.L), a2 = (int)((int64_t)i2 * g.s2 % g.L),
              a3 = (int)((int64_t)i3 * g.s3 % g.L);
    double2 A[WMAX * WMAX], Vm[WMAX * WMAX];
    const int WW = W * W;
    const int64_t pp = (int64_t)i2 * g.n3 + i3;   // (k2, k3) of this point (factorised build)
    for (int e = 0; e < WW; ++e) A[e] = make_double2(0, 0);
    if constexpr (FAC) {
        for (int j = 0; j < fac.D; ++j) {
            const double2 p = axis_ph(ph, j - fac.rc, a1, g.L);
            const double2 *u = fac.U + ((int64_t)j * fac.plane + pp) * WW;
            for (int e = 0; e < WW; ++e) A[e] = cfma(p, u[e], A[e]);
        }
    } else {
        for (int r = 0; r < nR; ++r) {
            const double2 p = ph[phase_index(a1, a2, a3, R[3 * r], R[3 * r + 1], R[3 * r + 2], g.L)];
            const double2 *h = Hw + (size_t)r * WW;
            for (int e = 0; e < WW; ++e) A[e] = cfma(p, h[e], A[e]);
        }
    }
    double w[WMAX];
    // FP64 results either way; the mixed solver where the FP64 Jacobi binds (8 x 8)
    int ok = WMAX >= 8 ? jacobi_hermitian_mixed<WMAX>(A, Vm, W, w) : jacobi_hermitian<WMAX>(A, Vm, W, w);
    if (!ok) atomicAdd(flag, 1);
    for (int n = 0; n < W; ++n) {
        eps[ik * W + n] = w[n];
        eps32[ik * W + n] = (float)w[n];
    }
    for (int e = 0; e < WW; ++e) {
        Vout[ik * WW + e] = Vm[e];
        V32[ik * WW + e] = make_float2((float)Vm[e].x, (float)Vm[e].y);
    }
    if (!do_vel) return;                 // velocities later, for the k-points that need them
    // v_n,a = (1/hbar) Re[V^dag (sum_R w_R i R_a e^{ik.R} H(R)) V]_nn, one axis at a time
    for (int ax = 0; ax < 3; ++ax) {
        for (int e = 0; e < WW; ++e) A[e] = make_double2(0, 0);
        if constexpr (FAC) {
            // i R_a = i (n1 A_1a + n2 A_2a + n3 A_3a): U_0 weighted by n1, U_1 (n2 sums), U_2 (n3 sums)
            const int64_t src = (int64_t)fac.D * fac.plane * WW;
            for (int j = 0; j < fac.D; ++j) {
                const int n1 = j - fac.rc;
                const double2 p = axis_ph(ph, n1, a1, g.L);
                const double2 ip = make_double2(-p.y, p.x);   // i e1
                const double c0 = n1 * lat.a[0][ax], c1 = lat.a[1][ax], c2 = lat.a[2][ax];
                const double2 *u = fac.U + ((int64_t)j * fac.plane + pp) * WW;
                for (int e = 0; e < WW; ++e) {
                    const double2 sr = make_double2(c0 * u[e].x + c1 * u[src + e].x + c2 * u[2 * src + e].x,
                                                    c0 * u[e].y + c1 * u[src + e].y + c2 * u[2 * src + e].y);
                    A[e] = cfma(ip, sr, A[e]);
                }
            }
        } else {
            for (int r = 0; r < nR; ++r) {
                const double2 p = ph[phase_index(a1, a2, a3, R[3 * r], R[3 * r + 1], R[3 * r + 2], g.L)];
                const double ra = Rcart[3 * r + ax];
                const double2 ip = make_double2(-ra * p.y, ra * p.x);   // i R_a e^{ik.R}
                const double2 *h = Hw + (size_t)r * WW;
                for (int e = 0; e < WW; ++e) A[e] = cfma(ip, h[e], A[e]);
            }
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

// Band velocities from the factorised stages and the stored eigenvectors (the velocity part of
// k_eig_el<WMAX, true>, same arithmetic), for the grid points with win_n > 0 (every point when
// win_n is NULL).
template <int WMAX>
__global__ void __launch_bounds__(128) k_vel_fac(GridInfo g, int64_t nk, int W, const int *__restrict__ win_n,
                                                 const double2 *__restrict__ ph, const double2 *__restrict__ Vin,
                                                 double *__restrict__ vel, FacDesc fac, Lattice lat) {
    const int64_t ik = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ik >= nk || (win_n && win_n[ik] == 0)) return;
    int i1, i2, i3;
    grid_coords(g, ik, i1, i2, i3);
    const int a1 = (int)((int64_t)i1 * g.s1 % g.L);
    const int WW = W * W;
    const int64_t pp = (int64_t)i2 * g.n3 + i3;
    double2 A[WMAX * WMAX], Vm[WMAX * WMAX];
    for (int e = 0; e < WW; ++e) Vm[e] = Vin[ik * WW + e];
    const int64_t src = (int64_t)fac.D * fac.plane * WW;
    for (int ax = 0; ax < 3; ++ax) {
        for (int e = 0; e < WW; ++e) A[e] = make_double2(0, 0);
        for (int j = 0; j < fac.D; ++j) {
            const int n1 = j - fac.rc;
            const double2 p = axis_ph(ph, n1, a1, g.L);
            const double2 ip = make_double2(-p.y, p.x);   // i e1
            const double c0 = n1 * lat.a[0][ax], c1 = lat.a[1][ax], c2 = lat.a[2][ax];
            const double2 *u = fac.U + ((int64_t)j * fac.plane + pp) * WW;
            for (int e = 0; e < WW; ++e) {
                const double2 sr = make_double2(c0 * u[e].x + c1 * u[src + e].x + c2 * u[2 * src + e].x,
                                                c0 * u[e].y + c1 * u[src + e].y + c2 * u[2 * src + e].y);
                A[e] = cfma(ip, sr, A[e]);
            }
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

// Phonons: hbar*omega, u = e (hbar^2 / (2 m hbar omega))^{1/2}, FP32 copies.  FAC: D(q) from
// the factorised stages.
template <int NMAX, bool FAC>
__global__ void __launch_bounds__(128) k_eig_ph(GridInfo g, int64_t nq, int Nm, int nR,
                                                const int *__restrict__ R,
                                                const double *__restrict__ Phiw,
                                                const double *__restrict__ mode_mass,
                                                const double2 *__restrict__ ph, double omega_min,
                                                double *__restrict__ hw, float *__restrict__ hwmax32,
                                                float *__restrict__ hw32,
                                                double2 *__restrict__ uout,
                                                float2 *__restrict__ u32, int *__restrict__ flag,
                                                FacDesc fac) {
    int64_t iq = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (iq >= nq) return;
    int i1, i2, i3;
    grid_coords(g, iq, i1, i2, i3);
    const int a1 = (int)((int64_t)i1 * g.s1 % g.L), a2 = (int)((int64_t)i2 * g.s2 % g.L),
              a3 = (int)((int64_t)i3 * g.s3 % g.L);
    double2 A[NMAX * NMAX], E[NMAX * NMAX];
    const int MM = Nm * Nm;
    for (int e = 0; e < MM; ++e) A[e] = make_double2(0, 0);
    if constexpr (FAC) {
        const int64_t pp = (int64_t)i2 * g.n3 + i3;
        for (int j = 0; j < fac.D; ++j) {
            const double2 p = axis_ph(ph, j - fac.rc, a1, g.L);
            const double2 *u = fac.U + ((int64_t)j * fac.plane + pp) * MM;
            for (int e = 0; e < MM; ++e) A[e] = cfma(p, u[e], A[e]);
        }
    } else {
        for (int r = 0; r < nR; ++r) {
            const double2 p = ph[phase_index(a1, a2, a3, R[3 * r], R[3 * r + 1], R[3 * r + 2], g.L)];
            const double *f = Phiw + (size_t)r * MM;
            for (int e = 0; e < MM; ++e) {
                A[e].x = fma(p.x, f[e], A[e].x);
                A[e].y = fma(p.y, f[e], A[e].y);
            }
        }
    }
    double lam[NMAX];
    int ok = NMAX >= 6 ? jacobi_hermitian_mixed<NMAX>(A, E, Nm, lam) : jacobi_hermitian<NMAX>(A, E, Nm, lam);
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

// Warp-per-matrix variants for large matrices (W >= 16, Nm >= 12): the matrix lives in
// shared memory (row stride n + 1), lane r builds row r of the Fourier sum, and the
// warp-parallel Jacobi diagonalises it.  Outputs are those of the one-thread kernels.
constexpr int kWarpsPerBlock = 4;

struct WarpScratch {
    double2 *A, *V;
    double *w;
    int *perm;
    JRot *rot;
};

__device__ inline WarpScratch warp_scratch(uint8_t *base, int n) {
    const int ld = n + 1;
    const size_t per = sizeof(double2) * 2 * n * ld + sizeof(double) * 32 + sizeof(int) * 32 +
                       sizeof(JRot) * 16;
    uint8_t *b = base + (threadIdx.x >> 5) * ((per + 15) & ~size_t(15));
    WarpScratch ws;
    ws.A = reinterpret_cast<double2 *>(b);
    ws.V = ws.A + n * ld;
    ws.w = reinterpret_cast<double *>(ws.V + n * ld);
    ws.perm = reinterpret_cast<int *>(ws.w + 32);
    ws.rot = reinterpret_cast<JRot *>(ws.perm + 32);
    return ws;
}

size_t warp_scratch_bytes(int n) {
    const size_t per = sizeof(double2) * 2 * n * (n + 1) + sizeof(double) * 32 + sizeof(int) * 32 +
                       sizeof(JRot) * 16;
    return kWarpsPerBlock * ((per + 15) & ~size_t(15));
}

// FAC: H(k) and dH/dk from the factorised stages (as in k_eig_el), each lane building its row.
template <bool FAC>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_eig_el_warp(
    GridInfo g, int64_t nk, int W, int nR, const int *__restrict__ R, const double *__restrict__ Rcart,
    const double2 *__restrict__ Hw, const double2 *__restrict__ ph, double *__restrict__ eps,
    float *__restrict__ eps32, double2 *__restrict__ Vout, float2 *__restrict__ V32,
    double *__restrict__ vel, int *__restrict__ flag, FacDesc fac, Lattice lat) {
    extern __shared__ __align__(16) uint8_t wsm[];
    const int lane = threadIdx.x & 31;
    const int64_t ik = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (ik >= nk) return;                      // whole warps leave together
    WarpScratch S = warp_scratch(wsm, W);
    const int ld = W + 1;
    int i1, i2, i3;
    grid_coords(g, ik, i1, i2, i3);
    const int a1 = (int)((int64_t)i1 * g.s1 % g.L), a2 = (int)((int64_t)i2 * g.s2 % g.L),
              a3 = (int)((int64_t)i3 * g.s3 % g.L);
    const int64_t WW = (int64_t)W * W;
    const int64_t pp = (int64_t)i2 * g.n3 + i3;   // (k2, k3) of this point (factorised build)
    if (lane < W) {
        for (int j = 0; j < W; ++j) S.A[lane * ld + j] = make_double2(0, 0);
        if constexpr (FAC) {
            for (int j1 = 0; j1 < fac.D; ++j1) {
                const double2 p = axis_ph(ph, j1 - fac.rc, a1, g.L);
                const double2 *u = fac.U + ((int64_t)j1 * fac.plane + pp) * WW + lane * W;
                for (int j = 0; j < W; ++j) S.A[lane * ld + j] = cfma(p, u[j], S.A[lane * ld + j]);
            }
        } else {
            for (int r = 0; r < nR; ++r) {
                const double2 p = ph[phase_index(a1, a2, a3, R[3 * r], R[3 * r + 1], R[3 * r + 2], g.L)];
                const double2 *h = Hw + (size_t)r * W * W + lane * W;
                for (int j = 0; j < W; ++j) S.A[lane * ld + j] = cfma(p, h[j], S.A[lane * ld + j]);
            }
        }
    }
    __syncwarp();
    const int ok = jacobi_hermitian_warp(S.A, S.V, W, ld, S.w, S.rot, S.perm);
    if (lane == 0 && !ok) atomicAdd(flag, 1);
    if (lane < W) {
        eps[ik * W + lane] = S.w[lane];
        eps32[ik * W + lane] = (float)S.w[lane];
        for (int n = 0; n < W; ++n) {
            const double2 v = S.V[lane * ld + n];
            Vout[ik * W * W + lane * W + n] = v;
            V32[ik * W * W + lane * W + n] = make_float2((float)v.x, (float)v.y);
        }
    }
    // v_n,a = (1/hbar) Re[V^dag (sum_R w_R i R_a e^{ik.R} H(R)) V]_nn, one axis at a time;
    // the derivative matrix reuses A (lane = row), then lane n contracts column n
    for (int ax = 0; ax < 3; ++ax) {
        __syncwarp();
        if (lane < W) {
            for (int j = 0; j < W; ++j) S.A[lane * ld + j] = make_double2(0, 0);
            if constexpr (FAC) {
                // i R_a = i (n1 A_1a + n2 A_2a + n3 A_3a): U_0 weighted by n1, U_1 (n2 sums), U_2 (n3 sums)
                const int64_t src = (int64_t)fac.D * fac.plane * WW;
                for (int j1 = 0; j1 < fac.D; ++j1) {
                    const int n1 = j1 - fac.rc;
                    const double2 p = axis_ph(ph, n1, a1, g.L);
                    const double2 ip = make_double2(-p.y, p.x);   // i e1
                    const double c0 = n1 * lat.a[0][ax], c1 = lat.a[1][ax], c2 = lat.a[2][ax];
                    const double2 *u = fac.U + ((int64_t)j1 * fac.plane + pp) * WW + lane * W;
                    for (int j = 0; j < W; ++j) {
                        const double2 sr = make_double2(c0 * u[j].x + c1 * u[src + j].x + c2 * u[2 * src + j].x,
                                                        c0 * u[j].y + c1 * u[src + j].y + c2 * u[2 * src + j].y);
                        S.A[lane * ld + j] = cfma(ip, sr, S.A[lane * ld + j]);
                    }
                }
            } else {
                for (int r = 0; r < nR; ++r) {
                    const double2 p = ph[phase_index(a1, a2, a3, R[3 * r], R[3 * r + 1], R[3 * r + 2], g.L)];
                    const double ra = Rcart[3 * r + ax];
                    const double2 ip = make_double2(-ra * p.y, ra * p.x);
                    const double2 *h = Hw + (size_t)r * W * W + lane * W;
                    for (int j = 0; j < W; ++j) S.A[lane * ld + j] = cfma(ip, h[j], S.A[lane * ld + j]);
                }
            }
        }
        __syncwarp();
        if (lane < W) {
            const int n = lane;
            double acc = 0;
            for (int i = 0; i < W; ++i) {
                double2 t = make_double2(0, 0);
                for (int j = 0; j < W; ++j) t = cfma(S.A[i * ld + j], S.V[j * ld + n], t);
                acc += S.V[i * ld + n].x * t.x + S.V[i * ld + n].y * t.y;
            }
            vel[(ik * W + n) * 3 + ax] = acc / epc::kHbarEVs * 1e-10;
        }
    }
}

template <bool FAC>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_eig_ph_warp(
    GridInfo g, int64_t nq, int Nm, int nR, const int *__restrict__ R, const double *__restrict__ Phiw,
    const double *__restrict__ mode_mass, const double2 *__restrict__ ph, double omega_min,
    double *__restrict__ hw, float *__restrict__ hwmax32, float *__restrict__ hw32,
    double2 *__restrict__ uout, float2 *__restrict__ u32, int *__restrict__ flag, FacDesc fac) {
    extern __shared__ __align__(16) uint8_t wsm[];
    const int lane = threadIdx.x & 31;
    const int64_t iq = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (iq >= nq) return;
    WarpScratch S = warp_scratch(wsm, Nm);
    const int ld = Nm + 1;
    int i1, i2, i3;
    grid_coords(g, iq, i1, i2, i3);
    const int a1 = (int)((int64_t)i1 * g.s1 % g.L), a2 = (int)((int64_t)i2 * g.s2 % g.L),
              a3 = (int)((int64_t)i3 * g.s3 % g.L);
    if (lane < Nm) {
        for (int j = 0; j < Nm; ++j) S.A[lane * ld + j] = make_double2(0, 0);
        if constexpr (FAC) {
            const int64_t pp = (int64_t)i2 * g.n3 + i3;
            for (int j1 = 0; j1 < fac.D; ++j1) {
                const double2 p = axis_ph(ph, j1 - fac.rc, a1, g.L);
                const double2 *u = fac.U + ((int64_t)j1 * fac.plane + pp) * Nm * Nm + lane * Nm;
                for (int j = 0; j < Nm; ++j) S.A[lane * ld + j] = cfma(p, u[j], S.A[lane * ld + j]);
            }
        } else {
            for (int r = 0; r < nR; ++r) {
                const double2 p = ph[phase_index(a1, a2, a3, R[3 * r], R[3 * r + 1], R[3 * r + 2], g.L)];
                const double *f = Phiw + (size_t)r * Nm * Nm + lane * Nm;
                for (int j = 0; j < Nm; ++j) {
                    S.A[lane * ld + j].x = fma(p.x, f[j], S.A[lane * ld + j].x);
                    S.A[lane * ld + j].y = fma(p.y, f[j], S.A[lane * ld + j].y);
                }
            }
        }
    }
    __syncwarp();
    const int ok = jacobi_hermitian_warp(S.A, S.V, Nm, ld, S.w, S.rot, S.perm);
    if (lane == 0 && !ok) atomicAdd(flag, 1);
    // lane = mode nu
    float wmax = -1.f;
    if (lane < Nm) {
        const int nu = lane;
        const double l = S.w[nu];
        const double w = (l >= 0 ? 1.0 : -1.0) * sqrt(fabs(l) * epc::kHbar2AmuA2);
        hw[iq * Nm + nu] = w;
        const bool keep = w >= omega_min;
        hw32[iq * Nm + nu] = keep ? (float)w : -1.0f;
        if (keep) wmax = (float)w;
        for (int m = 0; m < Nm; ++m) {
            const double amp = keep ? sqrt(epc::kHbar2AmuA2 / (2.0 * mode_mass[m] * w)) : 0.0;
            const double2 e = S.V[m * ld + nu];
            const double2 v = make_double2(e.x * amp, e.y * amp);
            uout[iq * Nm * Nm + m * Nm + nu] = v;
            u32[iq * Nm * Nm + m * Nm + nu] = make_float2((float)v.x, (float)v.y);
        }
    }
    for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    if (lane == 0) hwmax32[iq] = wmax;
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

// Raises a kernel's dynamic shared-memory limit the first time a larger size is needed
// (the first launch of each size happens outside any stream capture).  The limit set so far is
// kept per kernel: kernels of one signature share the template instance.
template <class K>
void set_smem_once(K kern, size_t bytes) {
    static std::vector<std::pair<const void *, size_t>> set;
    const void *key = reinterpret_cast<const void *>(kern);
    size_t *have = nullptr;
    for (auto &e : set)
        if (e.first == key) have = &e.second;
    if (!have) {
        set.emplace_back(key, size_t(48 * 1024));
        have = &set.back().second;
    }
    if (bytes > *have) {
        EPWI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        *have = bytes;
    }
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
    const int64_t plane = (int64_t)g.n2 * g.n3;
    // factorised build: axis-3 and axis-2 stages into fac_U (sources 0..nsrc-1), axis 1 in the
    // eigensolve kernel
    auto fac_sizes = [&](int rc, int E, bool vel, int64_t &nT, int64_t &nU) {
        const int D = 2 * rc + 1;
        nT = (int64_t)(vel ? 2 : 1) * D * D * g.n3 * E;
        nU = (int64_t)(vel ? 3 : 1) * D * plane * E;
    };
    auto fac_stages = [&](const DevBuf &Xc, int rc, int E, bool vel, DevBuf &Uout) {
        const int D = 2 * rc + 1;
        const int64_t t3 = (int64_t)D * D * g.n3 * E, t2 = (int64_t)D * plane * E;
        if (vel) {
            k_fac_axis3<true><<<(unsigned)((t3 + 255) / 256), 256, 0, c->stream>>>(
                D, rc, g.n3, g.s3, g.L, E, Xc.as<double2>(), c->ph64.as<double2>(), c->fac_T.as<double2>());
            EPWI_CHECK_LAUNCH();
            k_fac_axis2<true><<<(unsigned)((t2 + 255) / 256), 256, 0, c->stream>>>(
                D, rc, g.n2, g.n3, g.s2, g.L, E, c->fac_T.as<double2>(), c->ph64.as<double2>(), Uout.as<double2>());
        } else {
            k_fac_axis3<false><<<(unsigned)((t3 + 255) / 256), 256, 0, c->stream>>>(
                D, rc, g.n3, g.s3, g.L, E, Xc.as<double2>(), c->ph64.as<double2>(), c->fac_T.as<double2>());
            EPWI_CHECK_LAUNCH();
            k_fac_axis2<false><<<(unsigned)((t2 + 255) / 256), 256, 0, c->stream>>>(
                D, rc, g.n2, g.n3, g.s2, g.L, E, c->fac_T.as<double2>(), c->ph64.as<double2>(), Uout.as<double2>());
        }
        EPWI_CHECK_LAUNCH();
        FacDesc f;
        f.U = Uout.as<double2>();
        f.D = D;
        f.rc = rc;
        f.plane = plane;
        return f;
    };
    Lattice lat;
    for (int i = 0; i < 9; ++i) lat.a[i / 3][i % 3] = c->lattice[i];
    const bool fac_el = c->fac_re_r >= 0, fac_ph = c->fac_rp_r >= 0;
    {
        // both builds share the stage buffers: size them once, before any launch
        int64_t nT = 1, nU = 1, t, u;
        if (fac_el) {
            fac_sizes(c->fac_re_r, W * W, true, t, u);
            nT = std::max(nT, t);
            nU = std::max(nU, u);
        }
        if (fac_ph) {
            fac_sizes(c->fac_rp_r, Nm * Nm, false, t, u);
            nT = std::max(nT, t);
            nU = std::max(nU, u);
        }
        if (fac_el || fac_ph) {
            c->fac_T.ensure(sizeof(double2) * nT);
            c->fac_U.ensure(sizeof(double2) * nU);
        }
    }
    // deferred velocities (thread-per-point solver with the factorised build): the electron
    // stage output stays in fac_Uel for ensure_velocities
    const bool defer = c->vel_defer && fac_el && W <= 8;
    if (defer) {
        int64_t t, u;
        fac_sizes(c->fac_re_r, W * W, true, t, u);
        c->fac_Uel.ensure(sizeof(double2) * u);
    }
    FacDesc fe{}, fp{};
    if (fac_el) fe = fac_stages(c->fac_Hc, c->fac_re_r, W * W, true, defer ? c->fac_Uel : c->fac_U);
    const int do_vel = defer ? 0 : 1;
    c->vel_state = defer ? 0 : 2;
#define EL_ARGS                                                                              \
    g, nk, W, c->nRe, c->Re.as<int>(), c->Rcart.as<double>(), c->Hw.as<double2>(),            \
        c->ph64.as<double2>(), c->eps.as<double>(), c->eps32.as<float>(), c->V.as<double2>(), \
        c->V32.as<float2>(), c->vel.as<double>(), c->eig_flag.as<int>()
    const unsigned nbw = (unsigned)((nk + kWarpsPerBlock - 1) / kWarpsPerBlock);
    if (W <= 1) {
        if (fac_el) k_eig_el<1, true><<<nb, bs, 0, c->stream>>>(EL_ARGS, fe, lat, do_vel);
        else k_eig_el<1, false><<<nb, bs, 0, c->stream>>>(EL_ARGS, fe, lat, 1);
    } else if (W <= 4) {
        if (fac_el) k_eig_el<4, true><<<nb, bs, 0, c->stream>>>(EL_ARGS, fe, lat, do_vel);
        else k_eig_el<4, false><<<nb, bs, 0, c->stream>>>(EL_ARGS, fe, lat, 1);
    } else if (W <= 8) {
        if (fac_el) k_eig_el<8, true><<<nb, bs, 0, c->stream>>>(EL_ARGS, fe, lat, do_vel);
        else k_eig_el<8, false><<<nb, bs, 0, c->stream>>>(EL_ARGS, fe, lat, 1);
    } else {
        const size_t sm = warp_scratch_bytes(W);
        if (fac_el) {
            set_smem_once(k_eig_el_warp<true>, sm);
            k_eig_el_warp<true><<<nbw, 32 * kWarpsPerBlock, sm, c->stream>>>(EL_ARGS, fe, lat);
        } else {
            set_smem_once(k_eig_el_warp<false>, sm);
            k_eig_el_warp<false><<<nbw, 32 * kWarpsPerBlock, sm, c->stream>>>(EL_ARGS, fe, lat);
        }
    }
#undef EL_ARGS
    EPWI_CHECK_LAUNCH();
#define PH_ARGS                                                                             \
    g, nk, Nm, c->nRp, c->Rp.as<int>(), c->Phiw.as<double>(), c->mode_mass.as<double>(),     \
        c->ph64.as<double2>(), c->opt.omega_min_eV, c->hw.as<double>(), c->hwmax32.as<float>(), \
        c->hw32.as<float>(),                                                                   \
        c->u.as<double2>(), c->u32.as<float2>(), c->eig_flag.as<int>() + 1
    // the electron kernel above has read fac_U; the phonon stages reuse the buffers (same stream)
    if (fac_ph) fp = fac_stages(c->fac_Pc, c->fac_rp_r, Nm * Nm, false, c->fac_U);
    if (Nm <= 3) {
        if (fac_ph) k_eig_ph<3, true><<<nb, bs, 0, c->stream>>>(PH_ARGS, fp);
        else k_eig_ph<3, false><<<nb, bs, 0, c->stream>>>(PH_ARGS, fp);
    } else if (Nm <= 6) {
        if (fac_ph) k_eig_ph<6, true><<<nb, bs, 0, c->stream>>>(PH_ARGS, fp);
        else k_eig_ph<6, false><<<nb, bs, 0, c->stream>>>(PH_ARGS, fp);
    } else {
        const size_t sm = warp_scratch_bytes(Nm);
        if (fac_ph) {
            set_smem_once(k_eig_ph_warp<true>, sm);
            k_eig_ph_warp<true><<<nbw, 32 * kWarpsPerBlock, sm, c->stream>>>(PH_ARGS, fp);
        } else {
            set_smem_once(k_eig_ph_warp<false>, sm);
            k_eig_ph_warp<false><<<nbw, 32 * kWarpsPerBlock, sm, c->stream>>>(PH_ARGS, fp);
        }
    }
#undef PH_ARGS
    EPWI_CHECK_LAUNCH();
}

void ensure_velocities(epwi_ctx *c, bool all) {
    if (c->vel_state == 2 || (!all && c->vel_state == 1)) return;
    const int W = c->nw;
    GridInfo g = make_grid_info(c);
    FacDesc f;
    f.U = c->fac_Uel.as<double2>();
    f.rc = c->fac_re_r;
    f.D = 2 * f.rc + 1;
    f.plane = (int64_t)g.n2 * g.n3;
    Lattice lat;
    for (int i = 0; i < 9; ++i) lat.a[i / 3][i % 3] = c->lattice[i];
    const int *win = all ? nullptr : c->win_n.as<int>();
    const unsigned nb = (unsigned)((c->nk + 127) / 128);
#define VEL_ARGS g, c->nk, W, win, c->ph64.as<double2>(), c->V.as<double2>(), c->vel.as<double>(), f, lat
    if (W <= 1) k_vel_fac<1><<<nb, 128, 0, c->stream>>>(VEL_ARGS);
    else if (W <= 4) k_vel_fac<4><<<nb, 128, 0, c->stream>>>(VEL_ARGS);
    else k_vel_fac<8><<<nb, 128, 0, c->stream>>>(VEL_ARGS);
#undef VEL_ARGS
    EPWI_CHECK_LAUNCH();
    c->vel_state = all ? 2 : 1;
}
