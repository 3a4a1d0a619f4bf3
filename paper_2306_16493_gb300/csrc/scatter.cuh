// Argument blocks of the Re->k and Rp->q kernels and the chunked work set (internal).
#pragma once

#include <vector>

#include "epwi_internal.cuh"

struct RestageArgs {
    GridInfo g;
    int W, Nm, nRe, nRp, nrow;            // nrow = nRp * Nm * W
    const int *Re;
    const double2 *gw64;                  // [nRe][nrow][W]
    const float2 *gw32;
    const double2 *ph64;
    const float2 *ph32;
    const double2 *V64;
    const float2 *V32;
    int nkp;                              // k-points of the chunk
    const int *kpts;                      // [nkp] k index
    const int64_t *kp_state;              // [nkp+1] global state offsets
    int64_t s_base;                       // state offset of the chunk
    const int *win_lo, *win_n;            // per k index
    int ovr_lo, ovr_nsel;                 // >= 0: fixed band window (g2 mode)
    double2 *ghat64;                      // FP64 output [state][nrow]
    void *ghat_raw;                       // split-precision output (layout of the TC kernel)
    int precision;
    int64_t nstates_chunk;                // states of the chunk
};

struct ScatterArgs {
    GridInfo g;
    int W, Nm, nRp, nrow;
    const int *Rp;
    const double2 *ph64;
    const float2 *ph32;
    const int4 *tiles;                    // {kp_local, pair_begin, pair_end, 0} chunk-local
    const int *kpts;
    const int64_t *kp_state;
    int64_t s_base;
    const int *win_lo, *win_n;
    int ovr_lo, ovr_nsel;
    const int *pairs;                     // chunk pair list: q index
    const double2 *ghat64;
    const void *ghat_raw;
    const double2 *V64;
    const float2 *V32;
    const double2 *u64;
    const float2 *u32;
    const double *eps;
    const double *hw;
    const double *focc, *nocc;
    double omega_min, eta, ceta;
    double *tile_part;                    // [tile][kMaxW]
    double *g2out;                        // g2 mode output or nullptr
    int64_t g2_base;                      // global index of the chunk's first pair
    const double *pair_w;                 // per chunk pair weight (importance sampling) or nullptr
    double *tout;                         // terms mode output or nullptr:
                                          // tout[(pair * tstride + np) * Nm + nu]
    int tstride;
    float *gam32;                         // Gamma capture (split paths) or nullptr
    double *gam64;                        // Gamma capture (FP64 path) or nullptr
    const int64_t *goff;                  // chunk pair -> first Gamma entry (with a capture)
    int precision;
    int nsel_max;                         // largest band window of the chunk
    int64_t nstates_chunk;                // states of the chunk
};

struct WorkSet {
    int64_t nkp = 0;
    const int *kpts = nullptr;
    const int64_t *kp_state = nullptr;
    const int64_t *kp_pairs = nullptr;
    std::vector<int64_t> h_kp_state, h_kp_pairs;
    const int *pairs_dev = nullptr;       // all pairs, or nullptr: sieve fill per chunk
    const double *pair_w = nullptr;       // per pair weight of pairs_dev (FP64 path only)
    // Gamma capture of the iterative BTE (rates mode): for every pair, the block
    // [n in window(k)][m in window(k+q)] of sum_nu |g|^2 [occupation x exp] starting at
    // goff[pair] (global pair index), in gam64 (FP64 path) or gam32 (split paths)
    float *gam32 = nullptr;
    double *gam64 = nullptr;
    const int64_t *goff = nullptr;
    int ovr_lo = -1, ovr_nsel = -1;
};

// Rates mode (g2out == tout == nullptr): writes inv_tau for every state of the work set.
// g2 mode: |g|^2 per pair.  Terms mode (FP64 path): the summand of the SERTA rate per pair,
// band and mode, tout[(pair * tstride + np) * Nm + nu].
void process_workset(epwi_ctx *c, const WorkSet &ws, double *g2out, double *tout = nullptr,
                     int tstride = 0);
void sieve_fill_chunk(epwi_ctx *c, int64_t kp0, int64_t kp1, int *pairs);

// split-precision (tcgen05) path
size_t tc_state_bytes(const epwi_ctx *c);
void tc_restage(epwi_ctx *c, const RestageArgs &ra);
void tc_scatter(epwi_ctx *c, const ScatterArgs &sa, int64_t ntiles);
void tc_tables(epwi_ctx *c);
void tc_prepare(epwi_ctx *c);
int tc_check_error(epwi_ctx *c);

// Iterative BTE: pair list, Gamma layout and storage of the current window (sets the Gamma
// capture of ws); iteration from F0 = v tau into ib_F.
void ibte_prepare(epwi_ctx *c, WorkSet &ws);
void ibte_iterate(epwi_ctx *c, int max_iter, double tol);

// Rates of the current window by the k-batch ordering (FP64 ablation); fills inv_tau.
void process_kbatch(epwi_ctx *c);

// fp32 mode (sum-factorised Rp->q, scatter_sf.cu)
size_t sf_state_bytes(const epwi_ctx *c);
void sf_check(const epwi_ctx *c);
void sf_prepare(epwi_ctx *c);
void sf_restage(epwi_ctx *c, const RestageArgs &ra);
void sf_scatter(epwi_ctx *c, const ScatterArgs &sa, int64_t nkp, const int64_t *kp_pairs_local, int64_t p_off,
                const std::vector<int64_t> &h_kp_state_chunk);
