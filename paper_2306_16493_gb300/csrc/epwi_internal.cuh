// Internal declarations shared by the translation units of libepwi (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "epwi.h"

// ----------------------------------------------------------------------------- constants
// CODATA 2018.
namespace epc {
constexpr double kHbarEVs = 6.582119569e-16;           // eV s
constexpr double kHbarJs = 1.054571817e-34;            // J s
constexpr double kKbEVK = 8.617333262e-5;              // eV / K
constexpr double kECharge = 1.602176634e-19;           // C
constexpr double kAmuKg = 1.66053906660e-27;           // kg
// hbar^2 / (amu A^2) in eV: (hbar omega)^2 = lambda[eV/A^2/amu] * kHbar2AmuA2
constexpr double kHbar2AmuA2 = kHbarJs * kHbarJs / (kAmuKg * 1e-20) / kECharge;
constexpr double kPi = 3.14159265358979323846;
constexpr int kTile = 128;        // pairs per work tile (one tcgen05 M=128 tile)
constexpr int kMaxW = 24;
constexpr int kMaxNm = 18;
constexpr int kMaxL = 4096;       // lcm of the grid sizes (phase-table length)
}  // namespace epc

// ----------------------------------------------------------------------------- errors
struct EpwiError {
    epwi_status status;
    std::string msg;
};

#define EPWI_CUDA(call)                                                                    \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            throw EpwiError{e_ == cudaErrorMemoryAllocation ? EPWI_ENOMEM : EPWI_ECUDA,    \
                            std::string(#call) + ": " + cudaGetErrorString(e_)};          \
        }                                                                                  \
    } while (0)

// Every kernel launch site ends with this check; it also counts the launch.
extern int64_t g_epwi_launches;
#define EPWI_CHECK_LAUNCH()                                                                \
    do {                                                                                   \
        ++g_epwi_launches;                                                                 \
        EPWI_CUDA(cudaGetLastError());                                                     \
    } while (0)

#define EPWI_REQUIRE(cond, st, m)                                                          \
    do {                                                                                   \
        if (!(cond)) throw EpwiError{st, m};                                               \
    } while (0)

// ----------------------------------------------------------------------------- buffers
// Device buffer that grows on demand and is freed with the context.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    void ensure(size_t n) {
        if (n <= bytes && p) return;
        release();
        if (n == 0) n = 16;
        EPWI_CUDA(cudaMalloc(&p, n));
        bytes = n;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// ----------------------------------------------------------------------------- context
struct MlpState;                    // learned q-proposal network (mlp.cuh)
void mlp_free(MlpState *m);

struct epwi_ctx {
    epwi_options opt{};
    cudaStream_t stream = nullptr;
    std::string err;
    int device = 0;

    // system (after epwi_setup)
    bool have_sys = false;
    int nat = 0, nw = 0, nm = 0, nRe = 0, nRp = 0;
    double lattice[9] = {0};
    double volume = 0;             // A^3
    int rmax = 0;                  // max |n_a| over both R-sets
    DevBuf Re, Rp;                 // int32 [nR][3]
    DevBuf Rcart;                  // double [nRe][3]
    DevBuf Hw;                     // double2 [nRe][W][W], weight folded
    DevBuf Phiw;                   // double [nRp][Nm][Nm], w_R / sqrt(m_a m_b) folded
    DevBuf mode_mass;              // double [Nm] mass of the atom of each Cartesian mode
    DevBuf gw64;                   // double2 [nRe][nRp*Nm*W*W], c = ((rp*Nm+mu)*W+i)*W+j
    DevBuf gw32;                   // float2, same layout
    bool keep_g64 = true;          // false: FP32 copy only (members of a batch)

    // eigen-tables (after epwi_eigs)
    bool have_eigs = false;
    int ng[3] = {0, 0, 0};
    int64_t nk = 0;
    int L = 0;                     // lcm(N1, N2, N3)
    DevBuf ph64;                   // double2 [L]: e^{2 pi i m / L}
    DevBuf ph32;                   // float2 [L]
    DevBuf eps;                    // double [Nk][W]
    DevBuf eps32;                  // float  [Nk][W]
    DevBuf V;                      // double2 [Nk][W][W] (row i, column n)
    DevBuf V32;                    // float2 [Nk][W][W]
    DevBuf vel;                    // double [Nk][W][3] m/s
    DevBuf hw;                     // double [Nq][Nm] eV (dropped modes keep their value)
    DevBuf hwmax32;                // float [Nq] largest kept mode energy, -1 if none
    DevBuf hw32;                   // float [Nq][Nm] mode energy, -1 for dropped modes
    double eabs_max = 0;           // max |eps| over the grid (FP32 error bounds)
    DevBuf u;                      // double2 [Nq][Nm][Nm] A (row mu, column nu), 0 if dropped
    DevBuf u32;                    // float2 [Nq][Nm][Nm]
    DevBuf eig_flag;               // int [1] non-converged count
    float ms_eigs = 0;

    // scatter-rate results
    bool have_rates = false;
    double T = 0, mu = 0, eta = 0, emin = 0, emax = 0;
    int64_t nkp = 0, nstates = 0, npairs = 0;
    DevBuf kpts;                   // int32 [nkp] k index
    DevBuf win_lo, win_n;          // int32 [Nk] first window band, count
    DevBuf kp_state;               // int64 [nkp+1] state offsets
    DevBuf kp_pairs;               // int64 [nkp+1] pair offsets
    DevBuf sieve_mask;             // uint32 [nkp][mask_words]: sieve decisions of the count
    int64_t mask_words = 0;        // words per k-point (0: no mask, the fill re-evaluates)
    DevBuf inv_tau;                // double [nstates]
    DevBuf st_k, st_n;             // int32 [nstates]
    DevBuf focc;                   // double [Nk][W] Fermi-Dirac
    DevBuf nocc;                   // double [Nq][Nm] Bose-Einstein (0 for dropped modes)
    std::vector<int64_t> h_kp_pairs;
    epwi_stats stats{};

    // scratch
    DevBuf pairs;                  // int32 q index per pair of the chunk
    DevBuf ghat;                   // per-chunk Re->k output
    DevBuf tiles;                  // int4 per tile {kp_local, pair_begin, pair_end, 0}
    DevBuf tile_part;              // double [tile][W] partial sums
    DevBuf kp_tile;                // int64 [chunk kp + 1]
    DevBuf scan_tmp;               // scan workspace
    DevBuf red_tmp;                // reduction workspace
    DevBuf counts;                 // int64 per kp

    // split-precision (tcgen05) path
    int rp_cube_r = -1;            // Rp is the full cube [-r, r]^3 in n3-fastest order, else -1
    int tc_scale_exp = 0;          // fp16 operands: B scaled by 2^e (bound of |ghat| -> 2^14)
    int tc_ptab_key = -1;
    int tc_blocks_per_sm = 0;
    DevBuf tc_ptab;                // pre-split phase table
    DevBuf tc_erel, tc_f32;        // float [Nk][W]: eps - mu, Fermi-Dirac
    DevBuf tc_n32, tc_hw32;        // float [Nq][Nm]: Bose-Einstein, mode energy (-1 dropped)
    DevBuf tc_err;                 // int: timed-out waits in the tensor-core kernel
    DevBuf tc_meta;                // per-tile metadata of the tensor-core kernel
    DevBuf tc_arows;               // gathered-A mode: split phase rows of every grid point
    DevBuf sf_items;               // fp32 mode: (k-point, band) work items of a chunk
    int sf_r = 0;                  // fp32 mode: half-width of the bounding cube of R_p
    std::vector<int> h_rp_cube;    // fp32 mode: R_p index of each bounding-cube point, -1 if absent
    DevBuf gsf32;                  // fp32 mode: g' [Re][cube forms][Nm][W][W] (+-R recombined)
    bool sf_g_ready = false;       // gsf32 built for the current system
    DevBuf sf_Vt32;                // fp32 mode: float2 [m][Nk][i], columns of V band-major
    DevBuf sf_ef;                  // fp32 mode: float2 [m][Nk]: (eps - mu, f), band-major
    DevBuf sf_uS, sf_wn;           // fp32 mode: float2 [mu nu][Nq] u(q), [nu][Nq] (hbar omega, N)
    DevBuf gcube32;                // split modes, R_p not a cube: weighted g in the bounding cube
    bool gcube_ready = false;      // gcube32 built for the current system
    // factorised H(k) / D(q) builds: weighted H and Phi/sqrt(m m) embedded in the bounding cubes
    // of the two R-sets (half-widths fac_re_r, fac_rp_r; -1: direct sums), stage buffers
    int fac_re_r = -1, fac_rp_r = -1;
    DevBuf fac_Hc, fac_Pc;         // double2 [Dc^3][W W], [Dc^3][Nm Nm]
    DevBuf fac_T, fac_U;           // stage outputs (see eigs.cu)
    // band velocities: with vel_defer (set by epwi_eigs) the eigensolve leaves them out and
    // they are formed from the kept electron stage output fac_Uel for the k-points that need
    // them: those of each new window, or every point on request (ensure_velocities)
    bool vel_defer = false;
    int vel_state = 0;             // 0: none, 1: the current window's k-points, 2: every point
    DevBuf fac_Uel;
    int64_t tc_arows_key = -1;
    bool tc_gather = false;        // use the gathered-A mode where it applies
    int64_t stats_tc_grid = 0;

    // conductivity
    bool have_sigma = false;
    double sigma[9] = {0};

    // learned proposal and importance-sampled rates
    MlpState *mlp = nullptr;
    bool have_is = false;
    DevBuf is_pairs;               // int32 q index per sampled pair (all k-points)
    DevBuf is_w;                   // double weight count / (S p(q)) per sampled pair
    DevBuf is_kp_pairs;            // int64 [nkp+1] pair offsets of the sampled pairs
    std::vector<int64_t> h_is_kp_pairs;

    // iterative BTE: Gamma in pair blocks, mean free paths
    bool have_ibte = false;
    DevBuf ib_pairs;               // int32 q index per pair (all k-points of the window; capture only)
    DevBuf ib_goff;                // int64 [npairs + 1] first Gamma entry of each pair (capture only)
    DevBuf ib_col;                 // uint32 per Gamma entry: (final state << 5) | band of k (step only)
    DevBuf ib_ent;                 // int64 [nkp + 1] first Gamma entry of each window k-point

    // point-group symmetry of the rates (epwi_set_symmetry, sym.cu)
    std::vector<int> sym_ops;      // [nops][3][3] k-space operations on grid index vectors
    DevBuf sym_rep;                // int [Nk]: representative (lowest index) of each star
    // sieve pruning table (sieve.cu): band ranges per column segment, built once per eigs call
    DevBuf seg_ranges;
    bool seg_ready = false;
    double hw_max = 0;             // largest mode energy on the grid
    bool sym_used = false;         // the last rates call computed representatives only
    DevBuf ib_gam;                 // double (FP64 path) or float: per pair [n][m in window(k+q)]
    DevBuf ib_kpos;                // int32 [Nk] window k-point of each grid point, -1 outside
    DevBuf ib_F0, ib_F, ib_Fn;     // double [nstates][3] m: v tau, current and next iterate
    DevBuf ib_F32, ib_Fn32;        // float4 [nstates]: FP32 copies of ib_F, ib_Fn (split paths)
    DevBuf ib_red;                 // uint64 [2]: bit patterns of max |dF| and max |F|
    epwi_ibte_stats ib_stats{};

    ~epwi_ctx() {
        DevBuf *all[] = {&Re, &Rp, &Rcart, &Hw, &Phiw, &mode_mass, &gw64, &gw32, &ph64, &ph32,
                         &eps, &eps32, &V, &V32, &vel, &hw, &hwmax32, &hw32, &u, &u32, &eig_flag,
                         &kpts, &win_lo, &win_n, &kp_state, &kp_pairs, &inv_tau, &st_k,
                         &st_n, &focc, &nocc, &pairs, &ghat, &tiles, &tile_part, &kp_tile,
                         &scan_tmp, &red_tmp, &counts, &tc_ptab, &tc_erel, &tc_f32,
                         &tc_n32, &tc_hw32, &tc_err, &tc_meta, &is_pairs, &is_w,
                         &is_kp_pairs, &sieve_mask, &tc_arows, &ib_pairs, &ib_goff, &ib_gam,
                         &ib_kpos, &ib_F0, &ib_F, &ib_Fn, &ib_red, &ib_F32, &ib_Fn32, &sf_items, &ib_col, &ib_ent, &sym_rep, &seg_ranges,
                         &gsf32, &sf_Vt32, &sf_ef, &sf_uS, &sf_wn, &gcube32, &fac_Hc, &fac_Pc, &fac_T, &fac_U, &fac_Uel};
        for (DevBuf *b : all) b->release();
        mlp_free(mlp);
    }
};

// The R_p set the split-precision path works on: the set itself when it is a full cube
// [-r, r]^3 in n3-fastest order, else its bounding cube with zero-weight padding (gcube32).
inline int tc_rp_r(const epwi_ctx *c) { return c->rp_cube_r >= 0 ? c->rp_cube_r : c->sf_r; }
inline int tc_rp_count(const epwi_ctx *c) {
    const int D = 2 * tc_rp_r(c) + 1;
    return c->rp_cube_r >= 0 ? c->nRp : D * D * D;
}

// Uploads a host int vector into b (synchronously ordered on the context stream).
inline void upload_ints(epwi_ctx *c, DevBuf &b, const std::vector<int> &h) {
    b.ensure(sizeof(int) * (h.size() + 1));
    if (!h.empty())
        EPWI_CUDA(cudaMemcpyAsync(b.p, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice, c->stream));
}

// ----------------------------------------------------------------------------- complex
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 c) {  // conj(a)*b + c
    return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cfmaf(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ float2 cfmacf(float2 a, float2 b, float2 c) {  // conj(a)*b + c
    return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, c.y)));
}

// ----------------------------------------------------------------------------- grids
// Per-axis phase strides of a grid point: a_x = (i_x * L / N_x) mod L, so that
// e^{2 pi i k.R} = table[(n1 a1 + n2 a2 + n3 a3) mod L] exactly (integer reduction).
struct GridInfo {
    int n1, n2, n3, L, s1, s2, s3;   // s_x = L / N_x
};

__host__ __device__ __forceinline__ void grid_coords(const GridInfo &g, int64_t idx, int &i1,
                                                     int &i2, int &i3) {
    i3 = (int)(idx % g.n3);
    int64_t t = idx / g.n3;
    i2 = (int)(t % g.n2);
    i1 = (int)(t / g.n2);
}

__host__ __device__ __forceinline__ int64_t grid_index(const GridInfo &g, int i1, int i2, int i3) {
    return ((int64_t)i1 * g.n2 + i2) * g.n3 + i3;
}

__host__ __device__ __forceinline__ int64_t kplusq(const GridInfo &g, int64_t ik, int64_t iq) {
    int a1, a2, a3, b1, b2, b3;
    grid_coords(g, ik, a1, a2, a3);
    grid_coords(g, iq, b1, b2, b3);
    a1 += b1; if (a1 >= g.n1) a1 -= g.n1;
    a2 += b2; if (a2 >= g.n2) a2 -= g.n2;
    a3 += b3; if (a3 >= g.n3) a3 -= g.n3;
    return grid_index(g, a1, a2, a3);
}

__host__ __device__ __forceinline__ int phase_index(int a1, int a2, int a3, int n1, int n2, int n3,
                                                    int L) {
    int t = n1 * a1 + n2 * a2 + n3 * a3;   // |n| <= 64, a < 4096: fits in int32
    t %= L;
    return t < 0 ? t + L : t;
}

// ----------------------------------------------------------------------------- launches
GridInfo make_grid_info(const epwi_ctx *c);
void launch_phase_tables(epwi_ctx *c);
void launch_eigs(epwi_ctx *c);
// Band velocities of the window's k-points (all = false; needs win_n) or of every grid point,
// where the eigensolve deferred them; a no-op otherwise.  Every builder of a rates window calls
// it (all = false) after build_window.
void ensure_velocities(epwi_ctx *c, bool all);
void scan_exclusive_i64(epwi_ctx *c, const int64_t *in, int64_t *out, int64_t n, int64_t *total);
double device_reduce_minmax(epwi_ctx *c, const double *x, int64_t n, int64_t stride, int64_t off,
                            bool want_max);
// Window of the current rates call: lo/count per k from eps, then the lists of k-points and
// states.  rep (optional, symmetry): only k-points that represent their star take part.
void build_window(epwi_ctx *c, const int *rep = nullptr);
// The k-point and state lists from the current win_lo / win_n (rep as above).
void window_lists(epwi_ctx *c, const int *rep = nullptr);
// Point-group symmetry (sym.cu): representatives and invariance check of the current grid, and
// the expansion of the representatives' rates to every window state.
void sym_prepare(epwi_ctx *c);
void sym_expand(epwi_ctx *c);
void sieve_count(epwi_ctx *c);
void occupation_tables(epwi_ctx *c);
void run_scatter(epwi_ctx *c);
double carrier_density(epwi_ctx *c, double T, double mu, int n_valence);
void conductivity(epwi_ctx *c, double sigma[9]);
void transport_moments(epwi_ctx *c, double m[3][9]);
void transport_moments_F(epwi_ctx *c, const double *F, double m[3][9]);
void run_g2(epwi_ctx *c, int64_t npairs, const int32_t *ik, const int32_t *iq, int band_lo,
            int nsel, double *g2);
