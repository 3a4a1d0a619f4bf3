// C ABI of libepwi (declared in include/epwi.h): argument checks, input validation,
// weight folding and the orchestration of the device stages.  No C++ exception crosses
// the ABI; every entry point returns an epwi_status and records a message.
#include <algorithm>
#include <array>
#include <cmath>
#include <chrono>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "epwi_internal.cuh"
#include "mlp.cuh"
#include "scatter.cuh"

namespace {

template <class F>
epwi_status guard(epwi_ctx *c, F &&f) {
    if (!c) return EPWI_EINVAL;
    try {
        EPWI_CUDA(cudaSetDevice(c->device));
        f();
        c->err.clear();
        return EPWI_OK;
    } catch (const EpwiError &e) {
        c->err = e.msg;
        return e.status;
    } catch (const std::bad_alloc &) {
        c->err = "host allocation failed";
        return EPWI_ENOMEM;
    } catch (...) {
        c->err = "unexpected internal error";
        return EPWI_ECUDA;
    }
}

// f(i) for i in [0, n) on the host's hardware threads (static contiguous split).
template <class F>
void parallel_for(int n, F &&f) {
    const int nt = std::max(1, std::min<int>(n, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (int i = (int)((int64_t)n * t / nt); i < (int)((int64_t)n * (t + 1) / nt); ++i) f(i);
        });
    for (auto &x : th) x.join();
}

template <class T>
void upload(DevBuf &b, const T *h, size_t n, cudaStream_t st) {
    b.ensure(sizeof(T) * (n ? n : 1));
    if (n) EPWI_CUDA(cudaMemcpyAsync(b.p, h, sizeof(T) * n, cudaMemcpyHostToDevice, st));
}

std::vector<int> minus_index(const int32_t *R, int n, const char *what) {
    std::map<std::array<int, 3>, int> lut;
    for (int i = 0; i < n; ++i) lut[{R[3 * i], R[3 * i + 1], R[3 * i + 2]}] = i;
    std::vector<int> mi(n);
    for (int i = 0; i < n; ++i) {
        auto it = lut.find({-R[3 * i], -R[3 * i + 1], -R[3 * i + 2]});
        EPWI_REQUIRE(it != lut.end(), EPWI_EINVAL, std::string(what) + ": -R missing from the set");
        mi[i] = it->second;
    }
    return mi;
}

long long lcm3(long long a, long long b, long long c) {
    auto l = [](long long x, long long y) { return x / std::gcd(x, y) * y; };
    return l(l(a, b), c);
}

void require_sys(epwi_ctx *c) { EPWI_REQUIRE(c->have_sys, EPWI_ESTATE, "epwi_setup has not been called"); }
void require_eigs(epwi_ctx *c) {
    require_sys(c);
    EPWI_REQUIRE(c->have_eigs, EPWI_ESTATE, "epwi_eigs has not been called");
}
void require_rates(epwi_ctx *c) {
    require_eigs(c);
    EPWI_REQUIRE(c->have_rates, EPWI_ESTATE, "epwi_scatter_rates has not been called");
}

}  // namespace

int64_t g_epwi_launches = 0;

extern "C" {

int64_t epwi_kernel_launches(void) { return g_epwi_launches; }

void epwi_default_options(epwi_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = EPWI_FP64;
    opt->sieve_c = 6.0;
    opt->omega_min_eV = 1e-4;
    opt->device = 0;
    opt->cuda_stream = nullptr;
    opt->kpoint_chunk = 0;
    opt->tc_a_operand = 0;
    opt->ordering = 0;
}

epwi_status epwi_create(epwi_ctx **out, const epwi_options *opt) {
    if (!out) return EPWI_EINVAL;
    *out = nullptr;
    epwi_ctx *c = nullptr;
    try {
        c = new epwi_ctx();
    } catch (...) {
        return EPWI_ENOMEM;
    }
    if (opt) c->opt = *opt;
    else epwi_default_options(&c->opt);
    if (!(c->opt.sieve_c > 0) || !(c->opt.omega_min_eV >= 0) || c->opt.precision < 0 ||
        c->opt.precision > EPWI_FP32) {
        delete c;
        return EPWI_EINVAL;
    }
    c->device = c->opt.device;
    c->stream = (cudaStream_t)c->opt.cuda_stream;
    c->tc_gather = c->opt.tc_a_operand == 1;
    epwi_status st = guard(c, [&] {
        int n = 0;
        EPWI_CUDA(cudaGetDeviceCount(&n));
        EPWI_REQUIRE(c->device >= 0 && c->device < n, EPWI_EINVAL, "no such CUDA device");
        EPWI_CUDA(cudaSetDevice(c->device));
        EPWI_CUDA(cudaFree(nullptr));   // create the primary context now
    });
    if (st != EPWI_OK) {
        delete c;
        return st;
    }
    *out = c;
    return EPWI_OK;
}

void epwi_destroy(epwi_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    delete c;
}

const char *epwi_last_error(const epwi_ctx *c) { return c ? c->err.c_str() : "null context"; }

epwi_status epwi_set_precision(epwi_ctx *c, int32_t p) {
    return guard(c, [&] {
        EPWI_REQUIRE(p >= EPWI_FP64 && p <= EPWI_FP32, EPWI_EINVAL, "unknown precision");
        c->opt.precision = p;
    });
}

epwi_status epwi_set_stream(epwi_ctx *c, void *s) {
    return guard(c, [&] {
        c->stream = (cudaStream_t)s;
        c->opt.cuda_stream = s;
    });
}

epwi_status epwi_setup(epwi_ctx *c, const epwi_system *s) {
    return guard(c, [&] {
        EPWI_REQUIRE(s, EPWI_EINVAL, "system is NULL");
        EPWI_REQUIRE(s->nat >= 1 && 3 * s->nat <= epc::kMaxNm, EPWI_EUNSUPPORTED,
                     "nat must be in [1, 6]");
        EPWI_REQUIRE(s->nw >= 1 && s->nw <= epc::kMaxW, EPWI_EUNSUPPORTED, "nw must be in [1, 24]");
        EPWI_REQUIRE(s->nRe >= 1 && s->nRp >= 1, EPWI_EINVAL, "empty lattice-vector set");
        EPWI_REQUIRE(s->mass && s->Re && s->we && s->H && s->Rp && s->wp && s->Phi && s->g,
                     EPWI_EINVAL, "NULL array in epwi_system");
        const int W = s->nw, Nm = 3 * s->nat, nRe = s->nRe, nRp = s->nRp;
        for (int a = 0; a < s->nat; ++a)
            EPWI_REQUIRE(s->mass[a] > 0 && std::isfinite(s->mass[a]), EPWI_EINVAL, "mass must be > 0");
        int rmax = 0;
        for (int i = 0; i < 3 * nRe; ++i) rmax = std::max(rmax, std::abs(s->Re[i]));
        for (int i = 0; i < 3 * nRp; ++i) rmax = std::max(rmax, std::abs(s->Rp[i]));
        EPWI_REQUIRE(rmax <= 64, EPWI_EUNSUPPORTED, "lattice coordinates beyond |n| = 64");
        auto mie = minus_index(s->Re, nRe, "Re");
        auto mip = minus_index(s->Rp, nRp, "Rp");
        // Hermiticity of H and symmetry of the weights
        double hmax = 0, herr = 0;
        for (int r = 0; r < nRe; ++r) {
            EPWI_REQUIRE(s->we[r] == s->we[mie[r]], EPWI_EINVAL, "we(R) != we(-R)");
            for (int i = 0; i < W; ++i)
                for (int j = 0; j < W; ++j) {
                    const epwi_c64 a = s->H[((size_t)r * W + i) * W + j];
                    const epwi_c64 b = s->H[((size_t)mie[r] * W + j) * W + i];
                    hmax = std::max(hmax, std::hypot(a.re, a.im));
                    herr = std::max(herr, std::hypot(a.re - b.re, a.im + b.im));
                }
        }
        EPWI_REQUIRE(herr <= 1e-10 * std::max(hmax, 1e-300), EPWI_EINVAL,
                     "H(-R) != H(R)^dagger (relative error " + std::to_string(herr / hmax) + ")");
        // Phi symmetry and acoustic sum rule
        double pmax = 0, perr = 0;
        for (int r = 0; r < nRp; ++r) {
            EPWI_REQUIRE(s->wp[r] == s->wp[mip[r]], EPWI_EINVAL, "wp(R) != wp(-R)");
            for (int i = 0; i < Nm; ++i)
                for (int j = 0; j < Nm; ++j) {
                    const double a = s->Phi[((size_t)r * Nm + i) * Nm + j];
                    const double b = s->Phi[((size_t)mip[r] * Nm + j) * Nm + i];
                    pmax = std::max(pmax, std::fabs(a));
                    perr = std::max(perr, std::fabs(a - b));
                }
        }
        EPWI_REQUIRE(perr <= 1e-10 * std::max(pmax, 1e-300), EPWI_EINVAL, "Phi(-R) != Phi(R)^T");
        double asr = 0;
        for (int i = 0; i < Nm; ++i)
            for (int beta = 0; beta < 3; ++beta) {
                double sum = 0;
                for (int r = 0; r < nRp; ++r)
                    for (int b = 0; b < s->nat; ++b)
                        sum += s->wp[r] * s->Phi[((size_t)r * Nm + i) * Nm + 3 * b + beta];
                asr = std::max(asr, std::fabs(sum));
            }
        EPWI_REQUIRE(asr <= 1e-8 * std::max(pmax, 1e-300), EPWI_EINVAL, "acoustic sum rule violated");

        c->have_sys = c->have_eigs = c->have_rates = c->have_sigma = false;
        c->nat = s->nat;
        c->nw = W;
        c->nm = Nm;
        c->nRe = nRe;
        c->nRp = nRp;
        c->rmax = rmax;
        std::memcpy(c->lattice, s->lattice, sizeof(c->lattice));
        const double *A = s->lattice;
        c->volume = std::fabs(A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                              A[2] * (A[3] * A[7] - A[4] * A[6]));
        EPWI_REQUIRE(c->volume > 0, EPWI_EINVAL, "singular lattice");
        // fold weights
        std::vector<double2> Hw((size_t)nRe * W * W);
        std::vector<double> Rc((size_t)nRe * 3);
        for (int r = 0; r < nRe; ++r) {
            for (int e = 0; e < W * W; ++e) {
                const epwi_c64 h = s->H[(size_t)r * W * W + e];
                Hw[(size_t)r * W * W + e] = make_double2(s->we[r] * h.re, s->we[r] * h.im);
            }
            for (int ax = 0; ax < 3; ++ax)
                Rc[3 * r + ax] = s->Re[3 * r] * A[ax] + s->Re[3 * r + 1] * A[3 + ax] +
                                 s->Re[3 * r + 2] * A[6 + ax];
        }
        std::vector<double> Pw((size_t)nRp * Nm * Nm), mm(Nm);
        for (int i = 0; i < Nm; ++i) mm[i] = s->mass[i / 3];
        for (int r = 0; r < nRp; ++r)
            for (int i = 0; i < Nm; ++i)
                for (int j = 0; j < Nm; ++j)
                    Pw[((size_t)r * Nm + i) * Nm + j] =
                        s->wp[r] * s->Phi[((size_t)r * Nm + i) * Nm + j] / std::sqrt(mm[i] * mm[j]);
        const size_t ng = (size_t)nRe * nRp * Nm * W * W;
        const size_t per_re = (size_t)nRp * Nm * W * W;
        std::vector<double2> g64(c->keep_g64 ? ng : 0);
        std::vector<float2> g32(ng);
        parallel_for(nRe, [&](int re) {
            for (int rp = 0; rp < nRp; ++rp) {
                const double w = s->we[re] * s->wp[rp];
                const size_t base = (size_t)re * per_re + (size_t)rp * Nm * W * W;
                for (size_t e = 0; e < (size_t)Nm * W * W; ++e) {
                    const epwi_c64 v = s->g[base + e];
                    if (c->keep_g64) g64[base + e] = make_double2(w * v.re, w * v.im);
                    g32[base + e] = make_float2((float)(w * v.re), (float)(w * v.im));
                }
            }
        });
        // Rp as a full cube [-r, r]^3 with n3 fastest enables the incremental phase index
        // of the tensor-core kernel.
        c->rp_cube_r = -1;
        for (int rr = 0; rr <= 64; ++rr) {
            const int Dd = 2 * rr + 1;
            if ((long long)Dd * Dd * Dd != nRp) continue;
            bool ok = true;
            for (int k = 0; k < nRp && ok; ++k)
                ok = s->Rp[3 * k] == k / (Dd * Dd) - rr && s->Rp[3 * k + 1] == (k / Dd) % Dd - rr &&
                     s->Rp[3 * k + 2] == k % Dd - rr;
            if (ok) c->rp_cube_r = rr;
            break;
        }
        // factorised H(k) / D(q) builds (eigs.cu): weighted H and Phi in the bounding cubes
        {
            auto embed = [](const int32_t *R, int n, size_t ne, auto value, int &rout, std::vector<double2> &out) {
                int r = 0;
                for (int i = 0; i < 3 * n; ++i) r = std::max(r, std::abs(R[i]));
                rout = -1;
                out.clear();
                if (r > 6) return;
                const int Dc = 2 * r + 1;
                out.assign((size_t)Dc * Dc * Dc * ne, make_double2(0, 0));
                for (int k = 0; k < n; ++k) {
                    const size_t cf = ((size_t)(R[3 * k] + r) * Dc + (R[3 * k + 1] + r)) * Dc + (R[3 * k + 2] + r);
                    for (size_t e = 0; e < ne; ++e) out[cf * ne + e] = value(k, e);
                }
                rout = r;
            };
            std::vector<double2> hc, pc;
            embed(s->Re, nRe, (size_t)W * W, [&](int k, size_t e) { return Hw[(size_t)k * W * W + e]; },
                  c->fac_re_r, hc);
            embed(s->Rp, nRp, (size_t)Nm * Nm,
                  [&](int k, size_t e) { return make_double2(Pw[(size_t)k * Nm * Nm + e], 0.0); }, c->fac_rp_r, pc);
            if (c->fac_re_r >= 0) upload(c->fac_Hc, hc.data(), hc.size(), c->stream);
            if (c->fac_rp_r >= 0) upload(c->fac_Pc, pc.data(), pc.size(), c->stream);
            EPWI_CUDA(cudaStreamSynchronize(c->stream));   // hc, pc are freed on return
        }
        // fp32 mode: R_p embedded in its bounding cube [-r, r]^3 (points outside the set carry
        // zero weight); g' is built from the weighted g on the first fp32 rates call
        {
            int r = 0;
            for (int i = 0; i < 3 * nRp; ++i) r = std::max(r, std::abs(s->Rp[i]));
            c->sf_r = r;
            c->sf_g_ready = false;
            c->gcube_ready = false;
            c->gcube32.release();
            c->h_rp_cube.clear();
            if (r <= 6) {
                const int Dc = 2 * r + 1;
                c->h_rp_cube.assign((size_t)Dc * Dc * Dc, -1);
                for (int k = 0; k < nRp; ++k)
                    c->h_rp_cube[((size_t)(s->Rp[3 * k] + r) * Dc + (s->Rp[3 * k + 1] + r)) * Dc +
                                 (s->Rp[3 * k + 2] + r)] = k;
            }
            c->gsf32.release();
        }
        // |ghat(k)[rp][mu][i][n]| <= sum_Re sum_j |w g| (|V_jn| <= 1): scale fp16 operands so
        // that this bound maps to 2^14 (no overflow, full mantissa for the split).
        std::vector<double> rp_bound(nRp, 0.0);
        parallel_for(nRp, [&](int rp) {
            for (int mi = 0; mi < Nm * W; ++mi) {
                double sum = 0;
                for (int re = 0; re < nRe; ++re) {
                    const double w = s->we[re] * s->wp[rp];
                    for (int j = 0; j < W; ++j) {
                        const epwi_c64 v = s->g[(size_t)re * per_re + ((size_t)rp * Nm * W + mi) * W + j];
                        sum += std::hypot(w * v.re, w * v.im);
                    }
                }
                rp_bound[rp] = std::max(rp_bound[rp], sum);
            }
        });
        double gbound = 0;
        for (double v : rp_bound) gbound = std::max(gbound, v);
        c->tc_scale_exp = gbound > 0 ? 14 - (int)std::ceil(std::log2(gbound)) : 0;
        c->tc_ptab_key = -1;
        c->tc_arows_key = -1;
        upload(c->Re, s->Re, 3 * (size_t)nRe, c->stream);
        upload(c->Rp, s->Rp, 3 * (size_t)nRp, c->stream);
        upload(c->Rcart, Rc.data(), Rc.size(), c->stream);
        upload(c->Hw, Hw.data(), Hw.size(), c->stream);
        upload(c->Phiw, Pw.data(), Pw.size(), c->stream);
        upload(c->mode_mass, mm.data(), mm.size(), c->stream);
        if (c->keep_g64) upload(c->gw64, g64.data(), g64.size(), c->stream);
        else c->gw64.release();
        upload(c->gw32, g32.data(), g32.size(), c->stream);
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
        c->have_sys = true;
    });
}

epwi_status epwi_eigs(epwi_ctx *c, const int32_t kgrid[3], const int32_t qgrid[3]) {
    return guard(c, [&] {
        require_sys(c);
        EPWI_REQUIRE(kgrid && qgrid, EPWI_EINVAL, "grid is NULL");
        for (int a = 0; a < 3; ++a) {
            EPWI_REQUIRE(kgrid[a] >= 1 && kgrid[a] == qgrid[a], EPWI_EINVAL,
                         "qgrid must equal kgrid and be >= 1");
        }
        const long long L = lcm3(kgrid[0], kgrid[1], kgrid[2]);
        EPWI_REQUIRE(L <= epc::kMaxL, EPWI_EUNSUPPORTED, "lcm of grid sizes exceeds 4096");
        const int64_t nk = (int64_t)kgrid[0] * kgrid[1] * kgrid[2];
        EPWI_REQUIRE(nk < (int64_t(1) << 31), EPWI_EUNSUPPORTED, "grid larger than 2^31 points");
        c->have_eigs = c->have_rates = c->have_sigma = false;
        c->tc_ptab_key = -1;
        c->tc_arows_key = -1;
        c->seg_ready = false;
        for (int a = 0; a < 3; ++a) c->ng[a] = kgrid[a];
        c->nk = nk;
        c->L = (int)L;
        cudaEvent_t e0, e1;
        EPWI_CUDA(cudaEventCreate(&e0));
        EPWI_CUDA(cudaEventCreate(&e1));
        cudaEventRecord(e0, c->stream);
        launch_phase_tables(c);
        c->vel_defer = true;                 // velocities where a window or epwi_get_bands needs them
        launch_eigs(c);
        cudaEventRecord(e1, c->stream);
        int flag[2];
        EPWI_CUDA(cudaMemcpyAsync(flag, c->eig_flag.p, sizeof(flag), cudaMemcpyDeviceToHost, c->stream));
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
        cudaEventElapsedTime(&c->ms_eigs, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        EPWI_REQUIRE(flag[0] == 0 && flag[1] == 0, EPWI_ENUMERIC,
                     "Jacobi did not converge on " + std::to_string(flag[0]) + " H(k) and " +
                         std::to_string(flag[1]) + " D(q) matrices");
        {
            const double lo = device_reduce_minmax(c, c->eps.as<double>(), nk * c->nw, 1, 0, false);
            const double hi = device_reduce_minmax(c, c->eps.as<double>(), nk * c->nw, 1, 0, true);
            c->eabs_max = std::max(std::fabs(lo), std::fabs(hi));
        }
        c->have_eigs = true;
    });
}

epwi_status epwi_band_range(epwi_ctx *c, double *emin, double *emax) {
    return guard(c, [&] {
        require_eigs(c);
        const double *e = c->eps.as<double>();
        const int64_t n = c->nk * c->nw;
        if (emin) *emin = device_reduce_minmax(c, e, n, 1, 0, false);
        if (emax) *emax = device_reduce_minmax(c, e, n, 1, 0, true);
    });
}

epwi_status epwi_band_edges(epwi_ctx *c, int32_t nv, double *vbm, double *cbm) {
    return guard(c, [&] {
        require_eigs(c);
        EPWI_REQUIRE(nv >= 1 && nv < c->nw, EPWI_EINVAL, "n_valence must be in [1, nw-1]");
        const double *e = c->eps.as<double>();
        if (vbm) *vbm = device_reduce_minmax(c, e, c->nk, c->nw, nv - 1, true);
        if (cbm) *cbm = device_reduce_minmax(c, e, c->nk, c->nw, nv, false);
    });
}

epwi_status epwi_carrier_density(epwi_ctx *c, double T, double mu, int32_t nv, double *n) {
    return guard(c, [&] {
        require_eigs(c);
        EPWI_REQUIRE(T > 0 && n && nv >= 0 && nv < c->nw, EPWI_EINVAL, "bad argument");
        *n = carrier_density(c, T, mu, nv);
    });
}

epwi_status epwi_find_mu(epwi_ctx *c, double T, double n_c, int32_t nv, double *mu_out) {
    return guard(c, [&] {
        require_eigs(c);
        EPWI_REQUIRE(T > 0 && n_c > 0 && mu_out && nv >= 0 && nv < c->nw, EPWI_EINVAL, "bad argument");
        const double *e = c->eps.as<double>();
        double lo = device_reduce_minmax(c, e, c->nk, c->nw, nv, false) - 3.0;
        double hi = device_reduce_minmax(c, e, c->nk, c->nw, c->nw - 1, true) + 3.0;
        // n(mu) is increasing and nearly exponential below the band edge, so the root of
        // h(mu) = ln n(mu) - ln n_c is bracketed and found by regula falsi with the Illinois
        // modification (a retained end's h is halved), falling back to bisection where h is not
        // finite (n underflowed); stop at the same residual as a bisection: |n - n_c| <= 1e-13 n_c.
        auto h = [&](double mu, double &n) {
            n = carrier_density(c, T, mu, nv);
            return n > 0 ? std::log(n / n_c) : -HUGE_VAL;
        };
        double nlo, nhi;
        double hlo = h(lo, nlo), hhi = h(hi, nhi);
        double mid = 0.5 * (lo + hi);
        int side = 0;
        for (int it = 0; it < 400; ++it) {
            if (std::isfinite(hlo) && std::isfinite(hhi) && hhi > hlo) {
                mid = hi - hhi * (hi - lo) / (hhi - hlo);
                if (!(mid > lo && mid < hi)) mid = 0.5 * (lo + hi);
            } else {
                mid = 0.5 * (lo + hi);
            }
            double n;
            const double hm = h(mid, n);
            if (std::fabs(n - n_c) <= 1e-13 * n_c || hi - lo <= 1e-15) break;
            if (n < n_c) {
                lo = mid;
                hlo = hm;
                if (side == -1 && std::isfinite(hhi)) hhi *= 0.5;
                side = -1;
            } else {
                hi = mid;
                hhi = hm;
                if (side == 1 && std::isfinite(hlo)) hlo *= 0.5;
                side = 1;
            }
        }
        *mu_out = mid;
    });
}

static void solve3(const double A_[9], const double B_[9], double X[9]);

namespace {

// Window, sieve count, occupation tables and the work set of a rates call (Sec. III A);
// 1/tau is zeroed.
WorkSet begin_rates(epwi_ctx *c, double T, double mu, double eta, double emin, double emax,
                    bool sym = false) {
    require_eigs(c);
    EPWI_REQUIRE(T > 0 && eta > 0 && std::isfinite(mu) && !(emin > emax), EPWI_EINVAL,
                 "need T > 0, smear > 0, finite mu and emin <= emax");
    c->have_rates = c->have_sigma = c->have_is = c->have_ibte = false;
    c->T = T;
    c->mu = mu;
    c->eta = eta;
    c->emin = emin;
    c->emax = emax;
    std::memset(&c->stats, 0, sizeof(c->stats));
    c->stats.precision = c->opt.precision;
    c->stats.ms_eigs = c->ms_eigs;
    EPWI_CUDA(cudaDeviceGetAttribute(&c->stats.sm_count, cudaDevAttrMultiProcessorCount, c->device));
    // window and sieve (ms_sieve); the window's deferred band velocities count as eigensolve
    // work (ms_eigs)
    cudaEvent_t ev[4];
    for (auto &e : ev) EPWI_CUDA(cudaEventCreate(&e));
    cudaEventRecord(ev[0], c->stream);
    if (sym) sym_prepare(c);                 // representatives of the stars; invariance check
    build_window(c, sym ? c->sym_rep.as<int>() : nullptr);
    cudaEventRecord(ev[1], c->stream);
    ensure_velocities(c, false);
    cudaEventRecord(ev[2], c->stream);
    sieve_count(c);
    cudaEventRecord(ev[3], c->stream);
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    float ms_w = 0, ms_v = 0, ms_s = 0;
    cudaEventElapsedTime(&ms_w, ev[0], ev[1]);
    cudaEventElapsedTime(&ms_v, ev[1], ev[2]);
    cudaEventElapsedTime(&ms_s, ev[2], ev[3]);
    for (auto &e : ev) cudaEventDestroy(e);
    c->stats.ms_sieve = ms_w + ms_s;
    c->stats.ms_eigs += ms_v;
    occupation_tables(c);
    if (c->nstates > 0)
        EPWI_CUDA(cudaMemsetAsync(c->inv_tau.p, 0, sizeof(double) * c->nstates, c->stream));
    WorkSet ws;
    ws.nkp = c->nkp;
    ws.kpts = c->kpts.as<int>();
    ws.kp_state = c->kp_state.as<int64_t>();
    ws.kp_pairs = c->kp_pairs.as<int64_t>();
    ws.h_kp_pairs = c->h_kp_pairs;
    ws.h_kp_state.resize(c->nkp + 1);
    EPWI_CUDA(cudaMemcpyAsync(ws.h_kp_state.data(), c->kp_state.p, sizeof(int64_t) * (c->nkp + 1),
                              cudaMemcpyDeviceToHost, c->stream));
    EPWI_CUDA(cudaStreamSynchronize(c->stream));
    return ws;
}

void end_rates(epwi_ctx *c) {
    c->stats.n_kpoints = c->nkp;
    c->stats.n_states = c->nstates;
    c->stats.n_pairs = c->npairs;
    c->stats.restage_bytes = (int64_t)c->stats.n_chunks * c->nRe * c->nRp * c->nm * c->nw *
                             c->nw * (c->opt.precision == EPWI_FP64 ? 16 : 8);
    const double nbar = (double)c->nstates / std::max<int64_t>(1, c->nkp);
    c->stats.scatter_flops = 8.0 * c->nRp * c->nm * c->nw * (double)c->npairs * nbar;
    if (c->opt.precision == EPWI_FP32) {
        // per (pair, band): the last factor of the R_p sum (real coefficients on 2r recombined
        // forms, 4 flop each per column) and the rotations of one final band, the least any
        // pair needs (the per-block and per-run sums are shared, bands out of range are
        // skipped; neither is counted)
        const double NF = 2.0 * c->sf_r, X = (double)c->nm * c->nw;
        c->stats.scatter_flops = (4.0 * NF * X + 8.0 * ((double)c->nw * c->nm + (double)c->nm * c->nm)) *
                                 (double)c->npairs * nbar;
    }
    c->have_rates = true;
}

// sigma, S and kappa_e from the three energy moments (Sec. II C, Eqs. 12-14)
void finish_transport(epwi_ctx *c, const double (&m)[3][9], double *sigma, double *seebeck,
                      double *kappa_e) {
    const double e = epc::kECharge;
    const double kT_J = epc::kKbEVK * c->T * e;
    const double vol = (double)c->nk * c->volume * 1e-30;
    const double pref = 2.0 * e * e / (vol * kT_J);   // sigma per unit of the zeroth moment
    double sig[9], nu[9], k0[9];
    for (int i = 0; i < 9; ++i) {
        sig[i] = pref * m[0][i];
        nu[i] = -pref * m[1][i] / c->T;                // q = -e: electrons
        k0[i] = pref * m[2][i] / c->T;
    }
    double S[9];
    solve3(sig, nu, S);
    for (int i = 0; i < 9; ++i) {
        EPWI_REQUIRE(std::isfinite(sig[i]) && std::isfinite(S[i]), EPWI_ENUMERIC, "non-finite result");
        if (sigma) sigma[i] = sig[i];
        if (seebeck) seebeck[i] = S[i];
    }
    if (kappa_e)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double t = 0;
                for (int k = 0; k < 3; ++k) t += nu[i * 3 + k] * S[k * 3 + j];
                kappa_e[i * 3 + j] = k0[i * 3 + j] - c->T * t;
            }
}

}  // namespace

epwi_status epwi_scatter_rates(epwi_ctx *c, double T, double mu, double eta, double emin,
                               double emax, int64_t *n_states, int64_t *n_pairs) {
    return guard(c, [&] {
        EPWI_REQUIRE(c->opt.ordering == 0 || c->opt.ordering == 1, EPWI_EINVAL, "ordering must be 0 or 1");
        EPWI_REQUIRE(c->opt.ordering == 0 || c->opt.precision == EPWI_FP64, EPWI_EUNSUPPORTED,
                     "the k-batch ordering is FP64 only");
        const bool sym = !c->sym_ops.empty();
        WorkSet ws = begin_rates(c, T, mu, eta, emin, emax, sym);
        if (c->opt.ordering == 1) process_kbatch(c);
        else process_workset(c, ws, nullptr);
        end_rates(c);
        if (c->opt.ordering == 1)      // per pair: n_Re x N_m x W x W complex MACs instead
            c->stats.scatter_flops = 8.0 * c->nRe * c->nm * c->nw * c->nw * (double)c->npairs;
        if (sym) {
            // rates of the representatives -> every window state (Sec. III A symmetry)
            c->stats.sym_kpoints = c->nkp;
            c->stats.sym_states = c->nstates;
            sym_expand(c);
            c->sym_used = true;
            c->stats.n_kpoints = c->nkp;
            c->stats.n_states = c->nstates;
        }
        if (n_states) *n_states = c->nstates;
        if (n_pairs) *n_pairs = c->npairs;
    });
}

epwi_status epwi_ibte(epwi_ctx *c, double T, double mu, double eta, double emin, double emax,
                      int32_t max_iter, double tol, int32_t *iters, double *change) {
    return guard(c, [&] {
        EPWI_REQUIRE(max_iter >= 0 && tol >= 0 && std::isfinite(tol), EPWI_EINVAL,
                     "need max_iter >= 0 and a finite tol >= 0");
        EPWI_REQUIRE(c->sym_ops.empty(), EPWI_EUNSUPPORTED,
                     "the iterative BTE couples every k-point: clear the symmetry operations first");
        cudaEvent_t e0, e1;
        EPWI_CUDA(cudaEventCreate(&e0));
        EPWI_CUDA(cudaEventCreate(&e1));
        try {
            std::memset(&c->ib_stats, 0, sizeof(c->ib_stats));
            cudaEventRecord(e0, c->stream);
            WorkSet ws = begin_rates(c, T, mu, eta, emin, emax);
            ibte_prepare(c, ws);
            process_workset(c, ws, nullptr);
            cudaEventRecord(e1, c->stream);
            EPWI_CUDA(cudaStreamSynchronize(c->stream));
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            end_rates(c);
            c->ib_stats.ms_rates = ms;
            c->ib_stats.n_states = c->nstates;
            c->ib_stats.n_pairs = c->npairs;
            const auto t0 = std::chrono::steady_clock::now();
            ibte_iterate(c, max_iter, tol);
            c->ib_stats.ms_iterate =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->have_ibte = true;
        if (iters) *iters = c->ib_stats.iters;
        if (change) *change = c->ib_stats.change;
    });
}

epwi_status epwi_get_mfp(epwi_ctx *c, int64_t cap, double *F) {
    return guard(c, [&] {
        EPWI_REQUIRE(c->have_ibte, EPWI_ESTATE, "epwi_ibte has not been called");
        EPWI_REQUIRE(cap >= c->nstates, EPWI_ETOOSMALL, "capacity below n_states");
        EPWI_REQUIRE(F || c->nstates == 0, EPWI_EINVAL, "F is NULL");
        if (c->nstates)
            EPWI_CUDA(cudaMemcpyAsync(F, c->ib_F.p, sizeof(double) * 3 * c->nstates, cudaMemcpyDeviceToHost,
                                      c->stream));
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
    });
}

epwi_status epwi_ibte_transport(epwi_ctx *c, double sigma[9], double seebeck[9], double kappa_e[9]) {
    return guard(c, [&] {
        EPWI_REQUIRE(c->have_ibte, EPWI_ESTATE, "epwi_ibte has not been called");
        double m[3][9];
        transport_moments_F(c, c->ib_F.as<double>(), m);
        finish_transport(c, m, sigma, seebeck, kappa_e);
    });
}

epwi_status epwi_get_ibte_stats(epwi_ctx *c, epwi_ibte_stats *out) {
    return guard(c, [&] {
        EPWI_REQUIRE(out, EPWI_EINVAL, "out is NULL");
        *out = c->ib_stats;
    });
}

epwi_status epwi_get_rates(epwi_ctx *c, int64_t cap, int32_t *k_idx, int32_t *band, double *rates) {
    return guard(c, [&] {
        require_rates(c);
        EPWI_REQUIRE(cap >= c->nstates, EPWI_ETOOSMALL, "capacity below n_states");
        const size_t n = (size_t)c->nstates;
        if (n) {
            if (k_idx) EPWI_CUDA(cudaMemcpyAsync(k_idx, c->st_k.p, 4 * n, cudaMemcpyDeviceToHost, c->stream));
            if (band) EPWI_CUDA(cudaMemcpyAsync(band, c->st_n.p, 4 * n, cudaMemcpyDeviceToHost, c->stream));
            if (rates) EPWI_CUDA(cudaMemcpyAsync(rates, c->inv_tau.p, 8 * n, cudaMemcpyDeviceToHost, c->stream));
        }
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
    });
}

epwi_status epwi_conductivity(epwi_ctx *c, double sigma[9]) {
    return guard(c, [&] {
        require_rates(c);
        EPWI_REQUIRE(sigma, EPWI_EINVAL, "sigma is NULL");
        conductivity(c, c->sigma);
        for (int i = 0; i < 9; ++i) {
            EPWI_REQUIRE(std::isfinite(c->sigma[i]), EPWI_ENUMERIC, "non-finite conductivity");
            sigma[i] = c->sigma[i];
        }
        c->have_sigma = true;
    });
}

// 3x3 solve x = A^-1 b (row-major, all three columns of b), Gaussian elimination with
// partial pivoting.
static void solve3(const double A_[9], const double B_[9], double X[9]) {
    double A[9], B[9];
    std::memcpy(A, A_, sizeof(A));
    std::memcpy(B, B_, sizeof(B));
    int piv[3] = {0, 1, 2};
    for (int col = 0; col < 3; ++col) {
        int best = col;
        for (int r = col + 1; r < 3; ++r)
            if (std::fabs(A[piv[r] * 3 + col]) > std::fabs(A[piv[best] * 3 + col])) best = r;
        std::swap(piv[col], piv[best]);
        const double d = A[piv[col] * 3 + col];
        EPWI_REQUIRE(d != 0.0, EPWI_ENUMERIC, "singular conductivity tensor");
        for (int r = col + 1; r < 3; ++r) {
            const double f = A[piv[r] * 3 + col] / d;
            for (int j = 0; j < 3; ++j) {
                A[piv[r] * 3 + j] -= f * A[piv[col] * 3 + j];
                B[piv[r] * 3 + j] -= f * B[piv[col] * 3 + j];
            }
        }
    }
    for (int j = 0; j < 3; ++j)
        for (int col = 2; col >= 0; --col) {
            double v = B[piv[col] * 3 + j];
            for (int k = col + 1; k < 3; ++k) v -= A[piv[col] * 3 + k] * X[k * 3 + j];
            X[col * 3 + j] = v / A[piv[col] * 3 + col];
        }
}

epwi_status epwi_transport(epwi_ctx *c, double sigma[9], double seebeck[9], double kappa_e[9]) {
    return guard(c, [&] {
        require_rates(c);
        double m[3][9];
        transport_moments(c, m);
        finish_transport(c, m, sigma, seebeck, kappa_e);
    });
}

epwi_status epwi_mobility(epwi_ctx *c, double n_c, double mob[9]) {
    return guard(c, [&] {
        EPWI_REQUIRE(c->have_sigma, EPWI_ESTATE, "epwi_conductivity has not been called");
        EPWI_REQUIRE(n_c > 0 && mob, EPWI_EINVAL, "bad argument");
        for (int i = 0; i < 9; ++i) mob[i] = c->sigma[i] / (n_c * 1e6 * epc::kECharge) * 1e4;
    });
}

epwi_status epwi_get_bands(epwi_ctx *c, double *eps, epwi_c64 *V, double *vel) {
    return guard(c, [&] {
        require_eigs(c);
        const size_t nk = (size_t)c->nk, W = (size_t)c->nw;
        if (eps) EPWI_CUDA(cudaMemcpyAsync(eps, c->eps.p, 8 * nk * W, cudaMemcpyDeviceToHost, c->stream));
        if (V) EPWI_CUDA(cudaMemcpyAsync(V, c->V.p, 16 * nk * W * W, cudaMemcpyDeviceToHost, c->stream));
        if (vel) {
            ensure_velocities(c, true);
            EPWI_CUDA(cudaMemcpyAsync(vel, c->vel.p, 24 * nk * W, cudaMemcpyDeviceToHost, c->stream));
        }
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
    });
}

epwi_status epwi_get_phonons(epwi_ctx *c, double *omega, epwi_c64 *u) {
    return guard(c, [&] {
        require_eigs(c);
        const size_t nq = (size_t)c->nk, Nm = (size_t)c->nm;
        if (omega) EPWI_CUDA(cudaMemcpyAsync(omega, c->hw.p, 8 * nq * Nm, cudaMemcpyDeviceToHost, c->stream));
        if (u) EPWI_CUDA(cudaMemcpyAsync(u, c->u.p, 16 * nq * Nm * Nm, cudaMemcpyDeviceToHost, c->stream));
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
    });
}

epwi_status epwi_get_sieve(epwi_ctx *c, int64_t cap, int32_t *kpts, int64_t *counts) {
    return guard(c, [&] {
        require_rates(c);
        EPWI_REQUIRE(!c->have_is, EPWI_ESTATE, "the last rates came from importance sampling");
        EPWI_REQUIRE(!c->sym_used, EPWI_EUNSUPPORTED,
                     "the last rates were computed per star: the sieve lists are those of the representatives");
        EPWI_REQUIRE(cap >= c->nkp, EPWI_ETOOSMALL, "capacity below n_kpoints");
        if (kpts && c->nkp)
            EPWI_CUDA(cudaMemcpyAsync(kpts, c->kpts.p, 4 * (size_t)c->nkp, cudaMemcpyDeviceToHost, c->stream));
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
        if (counts)
            for (int64_t p = 0; p < c->nkp; ++p) counts[p] = c->h_kp_pairs[p + 1] - c->h_kp_pairs[p];
    });
}

epwi_status epwi_g2(epwi_ctx *c, int64_t npairs, const int32_t *ik, const int32_t *iq,
                    int32_t band_lo, int32_t nsel, double *g2) {
    return guard(c, [&] {
        require_eigs(c);
        EPWI_REQUIRE(npairs >= 1 && ik && iq && g2, EPWI_EINVAL, "bad argument");
        EPWI_REQUIRE(band_lo >= 0 && nsel >= 1 && band_lo + nsel <= c->nw, EPWI_EINVAL, "bad band window");
        for (int64_t p = 0; p < npairs; ++p)
            EPWI_REQUIRE(ik[p] >= 0 && ik[p] < c->nk && iq[p] >= 0 && iq[p] < c->nk, EPWI_EINVAL,
                         "grid index out of range");
        std::vector<int64_t> order(npairs);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return ik[a] < ik[b]; });
        std::vector<int> kp, pq(npairs);
        std::vector<int64_t> kst, kpr;
        for (int64_t t = 0; t < npairs; ++t) {
            const int64_t p = order[t];
            if (kp.empty() || kp.back() != ik[p]) {
                kp.push_back(ik[p]);
                kpr.push_back(t);
            }
            pq[t] = iq[p];
        }
        kpr.push_back(npairs);
        const int64_t nkp = (int64_t)kp.size();
        for (int64_t p = 0; p <= nkp; ++p) kst.push_back(p * nsel);
        DevBuf dk, ds, dp, dq, dout;
        auto cleanup = [&] { dk.release(); ds.release(); dp.release(); dq.release(); dout.release(); };
        try {
            upload(dk, kp.data(), kp.size(), c->stream);
            upload(ds, kst.data(), kst.size(), c->stream);
            upload(dp, kpr.data(), kpr.size(), c->stream);
            upload(dq, pq.data(), pq.size(), c->stream);
            const size_t nout = (size_t)npairs * nsel * c->nm * c->nw;
            dout.ensure(sizeof(double) * nout);
            if (c->eta <= 0) c->eta = 1.0;   // unused by g2 mode, kept finite
            if (c->opt.precision != EPWI_FP64) {
                // the tensor-core epilogue reads the FP32 mode-energy table; build the per-call
                // tables if no scatter_rates call has (occupations are unused in g2 mode)
                if (!(c->T > 0)) {
                    c->T = 300.0;
                    c->mu = 0.0;
                }
                occupation_tables(c);
            }
            WorkSet ws;
            ws.nkp = nkp;
            ws.kpts = dk.as<int>();
            ws.kp_state = ds.as<int64_t>();
            ws.kp_pairs = dp.as<int64_t>();
            ws.h_kp_state = kst;
            ws.h_kp_pairs = kpr;
            ws.pairs_dev = dq.as<int>();
            ws.ovr_lo = band_lo;
            ws.ovr_nsel = nsel;
            epwi_stats keep = c->stats;
            process_workset(c, ws, dout.as<double>());
            c->stats = keep;
            std::vector<double> h(nout);
            EPWI_CUDA(cudaMemcpyAsync(h.data(), dout.p, 8 * nout, cudaMemcpyDeviceToHost, c->stream));
            EPWI_CUDA(cudaStreamSynchronize(c->stream));
            const size_t per = (size_t)nsel * c->nm * c->nw;
            for (int64_t t = 0; t < npairs; ++t)
                std::memcpy(g2 + (size_t)order[t] * per, h.data() + (size_t)t * per, 8 * per);
        } catch (...) {
            cleanup();
            throw;
        }
        cleanup();
    });
}

void epwi_mlp_default_train_options(epwi_mlp_train_options *o) {
    if (!o) return;
    o->epochs = 100;
    o->batch = 512;
    o->lr = 2e-3;
    o->background = 1.0;
    o->floor_rel = 1e-8;
    o->seed = 1;
}

epwi_status epwi_mlp_train(epwi_ctx *c, double T, double mu, double eta, double emin, double emax,
                           const epwi_mlp_train_options *opt, double *final_loss) {
    return guard(c, [&] {
        require_eigs(c);
        EPWI_REQUIRE(T > 0 && eta > 0 && std::isfinite(mu) && !(emin > emax), EPWI_EINVAL,
                     "need T > 0, smear > 0, finite mu and emin <= emax");
        epwi_mlp_train_options o;
        epwi_mlp_default_train_options(&o);
        if (opt) o = *opt;
        EPWI_REQUIRE(o.epochs >= 0 && o.batch >= 1 && o.batch <= mlp::kMaxBatch && o.lr > 0 &&
                         o.background >= 0 && o.floor_rel > 0,
                     EPWI_EINVAL, "bad training options");
        mlp_train(c, T, mu, eta, emin, emax, o, final_loss);
    });
}

epwi_status epwi_mlp_set_params(epwi_ctx *c, const float *params) {
    return guard(c, [&] {
        EPWI_REQUIRE(params, EPWI_EINVAL, "params is NULL");
        mlp_set_master(c, params);
        c->mlp->out_scale = 1.0;
        c->mlp->out_shift = 0.0;
    });
}

epwi_status epwi_mlp_get_params(epwi_ctx *c, float *params, double *scale, double *shift) {
    return guard(c, [&] {
        EPWI_REQUIRE(c->mlp && c->mlp->ready, EPWI_ESTATE, "the network has no parameters yet");
        if (params) {
            EPWI_CUDA(cudaMemcpyAsync(params, c->mlp->w.p, sizeof(float) * mlp::kNParam,
                                      cudaMemcpyDeviceToHost, c->stream));
            EPWI_CUDA(cudaStreamSynchronize(c->stream));
        }
        if (scale) *scale = c->mlp->out_scale;
        if (shift) *shift = c->mlp->out_shift;
    });
}

epwi_status epwi_mlp_forward(epwi_ctx *c, int64_t n, const float *x, float *y) {
    return guard(c, [&] {
        EPWI_REQUIRE(c->mlp && c->mlp->ready, EPWI_ESTATE, "the network has no parameters yet");
        EPWI_REQUIRE(n >= 0 && (n == 0 || (x && y)), EPWI_EINVAL, "bad argument");
        if (n == 0) return;
        DevBuf dx, dy;
        try {
            upload(dx, x, (size_t)n * mlp::kIn, c->stream);
            dy.ensure(sizeof(float) * n);
            mlp_forward(c, n, dx.as<float>(), dy.as<float>());
            EPWI_CUDA(cudaMemcpyAsync(y, dy.p, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
            EPWI_CUDA(cudaStreamSynchronize(c->stream));
        } catch (...) {
            cudaStreamSynchronize(c->stream);
            dx.release();
            dy.release();
            throw;
        }
        dx.release();
        dy.release();
    });
}

epwi_status epwi_mlp_forward_tc(epwi_ctx *c, int64_t n, const float *x, float *y) {
    return guard(c, [&] {
        EPWI_REQUIRE(c->mlp && c->mlp->ready, EPWI_ESTATE, "the network has no parameters yet");
        EPWI_REQUIRE(n >= 0 && (n == 0 || (x && y)), EPWI_EINVAL, "bad argument");
        if (n == 0) return;
        DevBuf dx, dy;
        try {
            upload(dx, x, (size_t)n * mlp::kIn, c->stream);
            dy.ensure(sizeof(float) * n);
            mlp_forward_fast(c, n, dx.as<float>(), dy.as<float>());
            EPWI_CUDA(cudaMemcpyAsync(y, dy.p, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
            EPWI_CUDA(cudaStreamSynchronize(c->stream));
        } catch (...) {
            cudaStreamSynchronize(c->stream);
            dx.release();
            dy.release();
            throw;
        }
        dx.release();
        dy.release();
    });
}

epwi_status epwi_mlp_loss_grad(epwi_ctx *c, int64_t n, const float *x, const float *y,
                               double *loss, float *grad) {
    return guard(c, [&] {
        EPWI_REQUIRE(c->mlp && c->mlp->ready, EPWI_ESTATE, "the network has no parameters yet");
        EPWI_REQUIRE(n >= 1 && n <= mlp::kMaxBatch && x && y, EPWI_EINVAL, "bad argument");
        DevBuf dx, dy;
        try {
            upload(dx, x, (size_t)n * mlp::kIn, c->stream);
            upload(dy, y, (size_t)n, c->stream);
            const double L = mlp_loss_grad(c, n, dx.as<float>(), dy.as<float>(), true);
            if (loss) *loss = L;
            if (grad)
                EPWI_CUDA(cudaMemcpyAsync(grad, c->mlp->grad.p, sizeof(float) * mlp::kNParam,
                                          cudaMemcpyDeviceToHost, c->stream));
            EPWI_CUDA(cudaStreamSynchronize(c->stream));
        } catch (...) {
            cudaStreamSynchronize(c->stream);
            dx.release();
            dy.release();
            throw;
        }
        dx.release();
        dy.release();
    });
}

epwi_status epwi_mlp_get_training_set(epwi_ctx *c, int64_t cap, int32_t *ids, double *t,
                                      float *x, float *y, int64_t *n) {
    return guard(c, [&] {
        EPWI_REQUIRE(c->mlp && c->mlp->n_train > 0, EPWI_ESTATE, "epwi_mlp_train has not been called");
        const int64_t nt = c->mlp->n_train;
        if (n) *n = nt;
        if (!ids && !t && !x && !y) return;
        EPWI_REQUIRE(cap >= nt, EPWI_ETOOSMALL, "capacity below the training-set size");
        MlpState &m = *c->mlp;
        if (ids) EPWI_CUDA(cudaMemcpyAsync(ids, m.ids.p, 16 * (size_t)nt, cudaMemcpyDeviceToHost, c->stream));
        if (t) EPWI_CUDA(cudaMemcpyAsync(t, m.T64.p, 8 * (size_t)nt, cudaMemcpyDeviceToHost, c->stream));
        if (x) EPWI_CUDA(cudaMemcpyAsync(x, m.X.p, 4 * (size_t)nt * mlp::kIn, cudaMemcpyDeviceToHost, c->stream));
        if (y) EPWI_CUDA(cudaMemcpyAsync(y, m.Y.p, 4 * (size_t)nt, cudaMemcpyDeviceToHost, c->stream));
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
    });
}

epwi_status epwi_scatter_rates_is(epwi_ctx *c, double T, double mu, double eta, double emin,
                                  double emax, int64_t S, double alpha, int32_t stride,
                                  int32_t proposal, uint64_t seed, int64_t *n_states,
                                  int64_t *n_pairs) {
    return guard(c, [&] {
        require_eigs(c);
        EPWI_REQUIRE(T > 0 && eta > 0 && std::isfinite(mu) && !(emin > emax), EPWI_EINVAL,
                     "need T > 0, smear > 0, finite mu and emin <= emax");
        EPWI_REQUIRE(S >= 1 && S <= (int64_t(1) << 30), EPWI_EINVAL, "samples_per_k out of range");
        EPWI_REQUIRE(proposal == EPWI_PROPOSAL_UNIFORM || proposal == EPWI_PROPOSAL_LEARNED,
                     EPWI_EINVAL, "unknown proposal");
        if (proposal == EPWI_PROPOSAL_LEARNED) {
            EPWI_REQUIRE(c->mlp && c->mlp->ready, EPWI_ESTATE, "the network has no parameters yet");
            EPWI_REQUIRE(alpha > 0 && alpha <= 1, EPWI_EINVAL, "alpha must be in (0, 1]");
            EPWI_REQUIRE(stride >= 1 && c->ng[0] % stride == 0 && c->ng[1] % stride == 0 &&
                             c->ng[2] % stride == 0,
                         EPWI_EINVAL, "cell_stride must divide every grid dimension");
        }
        run_is(c, T, mu, eta, emin, emax, S, alpha, stride, proposal, seed);
        if (n_states) *n_states = c->nstates;
        if (n_pairs) *n_pairs = c->npairs;
    });
}

epwi_status epwi_get_is_pairs(epwi_ctx *c, int64_t cap, int32_t *ik, int32_t *iq, double *w,
                              int64_t *n) {
    return guard(c, [&] {
        EPWI_REQUIRE(c->have_is, EPWI_ESTATE, "epwi_scatter_rates_is has not been called");
        const int64_t np = c->npairs;
        if (n) *n = np;
        if (!ik && !iq && !w) return;
        EPWI_REQUIRE(cap >= np, EPWI_ETOOSMALL, "capacity below the pair count");
        if (iq && np) EPWI_CUDA(cudaMemcpyAsync(iq, c->is_pairs.p, 4 * (size_t)np, cudaMemcpyDeviceToHost, c->stream));
        if (w && np) EPWI_CUDA(cudaMemcpyAsync(w, c->is_w.p, 8 * (size_t)np, cudaMemcpyDeviceToHost, c->stream));
        std::vector<int> kp(c->nkp);
        if (c->nkp) EPWI_CUDA(cudaMemcpyAsync(kp.data(), c->kpts.p, 4 * (size_t)c->nkp, cudaMemcpyDeviceToHost, c->stream));
        EPWI_CUDA(cudaStreamSynchronize(c->stream));
        if (ik)
            for (int64_t p = 0; p < c->nkp; ++p)
                for (int64_t j = c->h_is_kp_pairs[p]; j < c->h_is_kp_pairs[p + 1]; ++j) ik[j] = kp[p];
    });
}

epwi_status epwi_get_stats(epwi_ctx *c, epwi_stats *out) {
    return guard(c, [&] {
        EPWI_REQUIRE(out, EPWI_EINVAL, "out is NULL");
        *out = c->stats;
    });
}

}  // extern "C"
