/*
 * epwi.h - C ABI of the GB300 (sm_103a) electron-phonon Wannier interpolation (EPWI)
 * transport hot path.
 *
 * The calls follow the problem statement of the paper (arXiv:2306.16493): Sec. III A
 * describes the inputs (lattice, mesh density, temperature, doping; H(R_e), Phi(R_p)
 * and g(R_e, R_p) in the Wannier basis), the preprocessing (interpolated electrons and
 * phonons, velocities, the chemical potential, the energy-conservation sieve) and the
 * on-the-fly EPWI loops; Sec. II B gives the interpolation formulas (Eqs. 4-7) and
 * Sec. II C the SERTA scattering rate (Eq. 10), the conductivity (Eq. 12) and the
 * mobility (Eq. 15).  Sec. III C (Eq. 16) fixes the evaluation order
 * {U(k+q)[(g P^el U^dag(k)) P^ph]} u(q).
 *
 * Conventions for every call:
 *  - Units: eV, Angstrom, amu, K.  Outputs: 1/tau in 1/s, sigma in S/m, mobility in
 *    cm^2/(V s), velocities in m/s.
 *  - All pointers are HOST pointers unless a name ends in _dev.  Arrays are C row-major.
 *    The caller owns every input and output buffer; inputs are copied, never retained.
 *    The context owns all device memory it allocates; epwi_destroy frees it.
 *  - Grids are Gamma-centred Monkhorst-Pack grids; the flat index of the point
 *    (i1, i2, i3) is (i1 * N2 + i2) * N3 + i3 and k+q is taken component-wise modulo N.
 *  - Every call returns an epwi_status.  No C++ exception crosses the ABI.  On error the
 *    context keeps a message (epwi_last_error).  A call made before the calls it depends
 *    on returns EPWI_ESTATE.  A context is not thread safe: use one per host thread.
 *  - Work is enqueued on the context's CUDA stream (epwi_options.cuda_stream, or the
 *    legacy default stream when NULL).  Calls that return host data synchronise that
 *    stream; the others only enqueue work unless stated.
 */
#ifndef EPWI_H
#define EPWI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct epwi_ctx epwi_ctx;

typedef enum {
    EPWI_OK = 0,
    EPWI_EINVAL = 1,      /* bad argument (NULL pointer, size, non-Hermitian H, ASR broken, ...) */
    EPWI_ENOMEM = 2,      /* device allocation failed */
    EPWI_ECUDA = 3,       /* a CUDA runtime call or kernel failed */
    EPWI_ESTATE = 4,      /* call out of order (e.g. scatter_rates before eigs) */
    EPWI_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
    EPWI_ENUMERIC = 6,    /* non-finite result or eigensolver did not converge */
    EPWI_ETOOSMALL = 7,   /* output capacity smaller than the result */
    EPWI_EUNSUPPORTED = 8 /* size or mode outside what the library supports */
} epwi_status;

/* Arithmetic of the g(k,q) interpolation (steps Re->k, Rp->q and the rotations).
 * Eigensolves, delta functions, occupations and the 1/tau and sigma sums are FP64 in
 * every mode.  EPWI_FP64 is the reference path. */
typedef enum {
    EPWI_FP64 = 0,   /* FP64 throughout */
    EPWI_TF32X3 = 1, /* Rp->q GEMM on tcgen05 kind::tf32, 3-term hi/lo split, FP32 accumulate */
    EPWI_BF16X3 = 2, /* Rp->q GEMM on tcgen05 kind::f16 with bf16 operands, 3-term split */
    EPWI_FP16X3 = 3, /* Rp->q GEMM on tcgen05 kind::f16 with fp16 operands, 3-term split */
    EPWI_FP32 = 4    /* FP32 Re->k, then the Rp->q sum factorised over the axes of the R_p cube
                        (D N_m W complex MACs per pair instead of D^3 N_m W), FP32 rotations and
                        delta terms, FP64 sums per state.  epwi_scatter_rates and epwi_ibte
                        (EUNSUPPORTED for importance sampling and epwi_g2); needs R_p to be a
                        full cube and
                        (nw, modes, half-width) in {(4,3,1), (4,3,2), (1,3,1)} */
} epwi_precision;

typedef struct { double re, im; } epwi_c64;

/* One crystal in the Wannier basis (Sec. III A inputs).  Arrays are unweighted; the
 * lattice-vector weights we/wp multiply every Fourier sum. */
typedef struct {
    double lattice[9];          /* rows a1, a2, a3 in Angstrom */
    int32_t nat;                /* atoms per cell; modes Nm = 3 nat */
    const double *mass;         /* [nat] amu, > 0 */
    int32_t nw;                 /* Wannier functions W */
    int32_t nRe;                /* electron lattice vectors */
    const int32_t *Re;          /* [nRe][3] integer lattice coordinates; -R must be present */
    const double *we;           /* [nRe] weights */
    const epwi_c64 *H;          /* [nRe][nw][nw] eV; H(-R) = H(R)^dagger required */
    int32_t nRp;                /* phonon lattice vectors */
    const int32_t *Rp;          /* [nRp][3] */
    const double *wp;           /* [nRp] */
    const double *Phi;          /* [nRp][3nat][3nat] eV/A^2, real; Phi(-R) = Phi(R)^T and the
                                   acoustic sum rule sum_R w_R sum_b Phi_ab(R) = 0 required */
    const epwi_c64 *g;          /* [nRe][nRp][3nat][nw][nw] eV/A, index [mu][i][j]: i pairs
                                   with k+q and j with k (Eq. 7) */
} epwi_system;

typedef struct {
    int32_t precision;          /* epwi_precision (default EPWI_FP64) */
    double sieve_c;             /* delta cut-off |x| <= c*eta, also the sieve (default 6) */
    double omega_min_eV;        /* modes below this energy are dropped (default 1e-4) */
    int32_t device;             /* CUDA device ordinal (default 0) */
    void *cuda_stream;          /* cudaStream_t, NULL = legacy default stream */
    int32_t kpoint_chunk;       /* k-points per on-the-fly chunk, 0 = automatic */
    int32_t tc_a_operand;       /* split modes, phase operand A: 0 = generated per tile into
                                   TMEM (default); 1 = precomputed split rows of every q gathered
                                   into shared memory (fp16x3, bf16x3, when the rows take
                                   <= 16 GiB; measured slower on the 48^3 benchmark) */
    int32_t ordering;           /* interpolation order of epwi_scatter_rates (Sec. III C):
                                   0 = q-batch (default): Re->k once per k-point, Rp->q per pair;
                                   1 = k-batch, the ordering the paper compares against (Table 3):
                                   Rp->q (with u(q)) once per q-point, Re->k and both rotations
                                   per pair.  k-batch is FP64 only (EUNSUPPORTED otherwise), for
                                   nw <= 8 and <= 6 modes; same rates within rounding */
} epwi_options;

/* Per-call statistics of the last epwi_scatter_rates (and what precedes it). */
typedef struct {
    int64_t n_kpoints;          /* k-points with at least one state in the window */
    int64_t n_states;           /* states (n,k) in the window */
    int64_t n_pairs;            /* (k,q) pairs kept by the sieve */
    int64_t n_tiles;            /* 128-pair work tiles processed */
    int64_t n_chunks;           /* on-the-fly k-point chunks */
    double ms_eigs, ms_sieve, ms_restage, ms_scatter, ms_reduce;   /* device time per stage */
    int64_t restage_bytes;      /* algorithmic bytes of the Re->k stage (g read once per chunk) */
    double scatter_flops;       /* algorithmic flops of the Rp->q GEMM (one pass, no padding) */
    int32_t precision;
    int32_t sm_count;           /* multiprocessors of the device */
    int64_t tc_grid;            /* CTAs of the last tensor-core launch (0 in FP64 mode) */
    int32_t tc_ctas_per_sm;     /* resident CTAs per SM of that launch */
    int32_t tc_regs;            /* registers per thread of that kernel */
    int64_t tc_smem;            /* dynamic shared memory per CTA (bytes) */
    int64_t tc_smem_avail2;     /* dynamic shared memory available to one CTA on an SM */
    double ms_proposal;         /* importance sampling: network scores and cell tables */
    double ms_sampling;         /* importance sampling: draws, merge and weights */
    double proposal_flops;      /* importance sampling: network flops (2 per multiply-add) */
    int64_t sym_kpoints;        /* symmetry-reduced call: k-points computed (star representatives), else 0 */
    int64_t sym_states;         /* symmetry-reduced call: states computed, else 0 */
} epwi_stats;

/* Statistics of the last epwi_ibte. */
typedef struct {
    int64_t n_states;           /* states (n,k) in the window */
    int64_t n_pairs;            /* (k,q) pairs kept by the sieve */
    int64_t n_entries;          /* stored Gamma values: sum over pairs of n_window(k) x
                                   n_window(k+q) */
    int32_t entry_bytes;        /* 8 (FP64 path) or 4 (split-precision paths) */
    int32_t iters;              /* iterations done */
    double change;              /* max |F^i - F^(i-1)| / max |F^i| after the last iteration */
    double ms_rates;            /* window, sieve, interpolation, 1/tau and the Gamma capture */
    double ms_iterate;          /* every iteration: step kernels and convergence reads */
    double ms_step;             /* mean device time of one step kernel */
    double bytes_per_step;      /* algorithmic bytes of one step: the index, Gamma, F0, tau,
                                   F read and written once */
    int64_t index_bytes;        /* the step's index: a 4-byte column word per Gamma entry and
                                   an 8-byte offset per window k-point */
} epwi_ibte_stats;

/* Fills *opt with the defaults listed above. */
void epwi_default_options(epwi_options *opt);

/* Creates a context on opt->device (opt may be NULL for defaults).  Errors: EINVAL, ECUDA. */
epwi_status epwi_create(epwi_ctx **ctx, const epwi_options *opt);

/* Frees all device memory of the context.  NULL is ignored. */
void epwi_destroy(epwi_ctx *ctx);

/* Message of the last failed call on this context ("" if none).  Valid until the next call. */
const char *epwi_last_error(const epwi_ctx *ctx);

/* Switches the interpolation arithmetic for subsequent epwi_scatter_rates calls. */
epwi_status epwi_set_precision(epwi_ctx *ctx, int32_t precision);

/* Switches the CUDA stream used by subsequent calls. */
epwi_status epwi_set_stream(epwi_ctx *ctx, void *cuda_stream);

/* Copies the system to the device and folds the weights in: w_R into H(R) (Eq. 4),
 * w_R/sqrt(m_a m_b) into Phi(R) (Eq. 5), w_e w_p into g (Eq. 7); reorders g into the
 * per-R_p column layout of the Re->k stage and keeps an FP32 copy for the split-precision
 * modes.  Validates Hermiticity of H (1e-10 relative), Phi(-R) = Phi(R)^T, the acoustic
 * sum rule (1e-8 relative), masses > 0 and that -R is in each set.  Replaces any previous
 * system (eigen-tables and rates are discarded).  Synchronous. */
epwi_status epwi_setup(epwi_ctx *ctx, const epwi_system *sys);

/* Interpolates and diagonalises H(k) and D(q) on the full grids (Sec. II B, Eqs. 4-6):
 * eps_nk (ascending), V(k) (columns), v_nk = (1/hbar) Re[V^dag dH/dk V]_nn, hbar*omega_qnu
 * and u_{mu nu}(q) = (hbar / 2 m_mu omega_nu)^{1/2} e_{mu nu}(q) (FP64 Jacobi, one matrix per
 * grid point).  qgrid must equal kgrid (k+q is a grid point, Sec. III E).  The least
 * common multiple of the three grid sizes must be <= 4096.  Errors: ESTATE (no setup),
 * EINVAL, ENUMERIC (Jacobi did not converge). */
epwi_status epwi_eigs(epwi_ctx *ctx, const int32_t kgrid[3], const int32_t qgrid[3]);

/* Smallest and largest band energy on the k grid (eV).  Synchronises. */
epwi_status epwi_band_range(epwi_ctx *ctx, double *emin_eV, double *emax_eV);

/* Valence maximum (band n_valence-1) and conduction minimum (band n_valence) over the grid. */
epwi_status epwi_band_edges(epwi_ctx *ctx, int32_t n_valence, double *vbm_eV, double *cbm_eV);

/* Chemical potential for a conduction-electron density n_c (per cm^3) at T (Sec. III A):
 * bisection on n(mu) = (2/(N_k V)) sum_{n >= n_valence, k} f(eps_nk) to a relative
 * residual of 1e-13.  Synchronises. */
epwi_status epwi_find_mu(epwi_ctx *ctx, double T_K, double carriers_per_cm3,
                         int32_t n_valence, double *mu_eV);

/* Conduction-electron density (per cm^3) at mu and T, same sum as epwi_find_mu. */
epwi_status epwi_carrier_density(epwi_ctx *ctx, double T_K, double mu_eV, int32_t n_valence,
                                 double *n_cm3);

/* SERTA scattering rates (Sec. II C, Eq. 10) for every state with emin <= eps_nk <= emax:
 * 1/tau_nk = (2 pi/hbar)(1/N_q) sum_{q m nu} |g^nu_mn(k,q)|^2 [(N + f) delta(e_nk + w - e_mk+q)
 *            + (1 + N - f) delta(e_nk - w - e_mk+q)],
 * delta(x) = exp(-(x/eta)^2)/(sqrt(pi) eta) for |x| <= c eta, eta = smear_eV.
 * Runs the sieve (Sec. III A), then the on-the-fly q-batched interpolation (Sec. III D) in
 * k-point chunks.  Results stay on the device (see epwi_get_rates); n_states and n_pairs
 * (either may be NULL) receive the state and sieved-pair counts.  Synchronises.
 * Memory: the sieve keeps its decisions as a bit mask (one bit per (k-point, q) candidate)
 * when that mask fits in EPWI_SIEVE_MASK_MAX_BYTES (environment variable, bytes, default
 * 2 GiB); otherwise each chunk's pair lists are rebuilt by evaluating the sieve again.  Both
 * give the same pair lists and rates. */
epwi_status epwi_scatter_rates(epwi_ctx *ctx, double T_K, double mu_eV, double smear_eV,
                               double emin_eV, double emax_eV,
                               int64_t *n_states, int64_t *n_pairs);

/* Point-group symmetry of the crystal for epwi_scatter_rates: the symmetry-reduced k grids of
 * the paper's preprocessing (Sec. III A).  kops: nops integer 3x3 matrices (row-major) acting
 * on grid index vectors, k -> K k modulo N (for lattice operations n -> M n on the lattice
 * coordinates of the R-sets, K = M^-T).  They must form a group (identity and closure;
 * nops <= 48); nops = 0 switches the reduction off.  Copied.
 * With operations set, epwi_scatter_rates needs an N x N x N grid, checks on the device that
 * eps and hbar omega are invariant on the grid (max |eps(Kk) - eps(k)| <= 1e-9 max(1, |eps|),
 * |omega(Kq) - omega(q)| <= 1e-9 eV; EINVAL otherwise), computes the sieve and 1/tau only for
 * the window k-points that represent their star (the lowest grid index), and gives every
 * member of a star its representative's band window and rates.  epwi_get_rates then returns
 * every window state; sigma, mobility and transport sum over all of them with each state's own
 * velocity.  n_pairs counts the pairs computed; epwi_stats.sym_kpoints / sym_states the
 * representatives.  The iterative BTE refuses to run with operations set (EUNSUPPORTED), and
 * epwi_get_sieve after a reduced call too.  Errors: EINVAL (nops, NULL kops, not a group). */
epwi_status epwi_set_symmetry(epwi_ctx *ctx, int32_t nops, const int32_t *kops);

/* Copies the states of the last epwi_scatter_rates (ordered by k index, then band) and
 * their rates to host arrays of capacity >= n_states.  Any output pointer may be NULL.
 * Errors: ESTATE (no rates), ETOOSMALL (capacity). */
epwi_status epwi_get_rates(epwi_ctx *ctx, int64_t capacity, int32_t *k_idx, int32_t *band,
                           double *inv_tau_s);

/* sigma_ab = (2 e^2/(N_k V)) sum_{nk in window} v_a v_b tau f(1-f)/(k_B T) (Sec. II C,
 * Eq. 12 with F = v tau), over the states of the last epwi_scatter_rates with 1/tau > 0,
 * at the T and mu of that call.  sigma_Sm is 3x3 row-major.  Synchronises. */
epwi_status epwi_conductivity(epwi_ctx *ctx, double sigma_Sm[9]);

/* mu_ab = sigma_ab / (n e) (Sec. II C, Eq. 15) using the last conductivity. */
epwi_status epwi_mobility(epwi_ctx *ctx, double carriers_per_cm3, double mu_cm2Vs[9]);

/* Copies the eigen-tables: eps [Nk][nw], V [Nk][nw][nw] (row i, column n), vel
 * [Nk][nw][3].  Any pointer may be NULL.  Synchronises.  (epwi_eigs forms the velocities of
 * the k-points that a rates window needs; the first request for vel forms the rest.) */
epwi_status epwi_get_bands(epwi_ctx *ctx, double *eps, epwi_c64 *V, double *vel);

/* Copies hbar*omega [Nq][Nm] (eV) and u [Nq][Nm][Nm] (A, row mu, column nu; zero columns
 * for dropped modes).  Any pointer may be NULL.  Synchronises. */
epwi_status epwi_get_phonons(epwi_ctx *ctx, double *omega, epwi_c64 *u);

/* Sieve output of the last epwi_scatter_rates: the k-points with window states
 * (kpts[n_kpoints]) and per k-point pair counts (counts[n_kpoints]).  Pair lists are not
 * kept (they are built per chunk).  Errors: ESTATE, ETOOSMALL. */
epwi_status epwi_get_sieve(epwi_ctx *ctx, int64_t capacity, int32_t *kpts, int64_t *counts);

/* |g^nu_mn(k,q)|^2 (eV^2) for explicit pairs, through the same Re->k, Rp->q and rotation
 * kernels as epwi_scatter_rates in the current precision: g2 has layout
 * [pair][nsel][nu][m] for the bands n = band_lo .. band_lo+nsel-1 at each k.
 * ik, iq: [npairs] grid indices; band_lo, nsel: window per pair (nsel <= nw).  For tests. */
epwi_status epwi_g2(epwi_ctx *ctx, int64_t npairs, const int32_t *ik, const int32_t *iq,
                    int32_t band_lo, int32_t nsel, double *g2);

/* Conductivity from per-state DEVICE arrays, allocating no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc, such as a
 * host framework that owns all device memory through its own pool, or a service that must
 * not allocate after start-up (cudaMalloc/cudaFree may synchronise the device and can fail
 * under memory pressure mid-run).  Same sum as epwi_conductivity:
 *   sigma_ab = (2 e^2/(N_k V)) sum_s v_a v_b f(1-f)/(k_B T) / (1/tau_s), states with 1/tau_s = 0
 *   skipped, f = Fermi-Dirac(eps_s; mu, T).
 * eps_dev [n_states] eV, vel_dev [n_states][3] m/s, inv_tau_dev [n_states] 1/s, all device
 * pointers owned by the caller; sigma_dev: 9 doubles (3x3 row-major) in device memory, written
 * on cuda_stream (NULL = legacy default stream); the call only enqueues work.  nk is N_k of the
 * grid, volume_A3 the cell volume.  Scratch is a fixed 48 KiB device array in the library
 * (held by every GPU that loads it until exit); n_states above 4,194,304 returns
 * EPWI_EUNSUPPORTED.  The first call on each device resolves the array's device address
 * (cudaGetSymbolAddress) and caches it, so make that first call before any stream capture;
 * two host threads making that first call together store the same address (harmless).  A
 * device reset in the process (cudaDeviceReset) invalidates the cached address: do not call
 * this entry point after one.  All calls share the array: calls that overlap on the GPU race.  Errors: EINVAL (NULL pointer, T <= 0,
 * volume <= 0, nk < 1), EUNSUPPORTED (too many states), ECUDA (launch or symbol lookup). */
epwi_status epwi_conductivity_noalloc(int64_t n_states, const double *eps_dev, const double *vel_dev,
                                      const double *inv_tau_dev, double mu_eV, double T_K,
                                      double volume_A3, int64_t nk, void *cuda_stream,
                                      double *sigma_dev);

/* ---------------------------------------------------------------------------------------
 * Learned q-proposal and importance-sampled rates.  The paper has no learned part: it sums
 * the SERTA rate (Sec. II C, Eq. 10) over every sieved q.  These calls estimate that q sum by
 * importance sampling instead.  Per k-point, S grid points q are drawn from a proposal p > 0,
 * and the rate is (2 pi/hbar)(1/N_q) sum over the distinct drawn q of c_q / (S p(q)) t(q),
 * where c_q is how often q was drawn and t is the summand of Eq. 10.  This is unbiased for
 * any proposal that is positive wherever t is.
 *
 * The learned proposal uses a network 9 -> 128 -> 128 -> 128 -> 1 with SiLU hidden
 * activations, BF16 weights and FP32 arithmetic.  Its inputs are:
 *   - k and q as fractional coordinates mapped to [-1/2, 1/2) and doubled;
 *   - (eps_nk - mu) / 0.25 eV;
 *   - n / nw;
 *   - nu / (3 nat).
 * It is trained on the normalised log(t + floor) of the terms on the context's current grid.
 *
 * Parameters are EPWI_MLP_NPARAM floats, stored in this order: W1 [128][9], b1 [128],
 * W2 [128][128], b2, W3 [128][128], b3, w4 [128], b4 [1].
 * ------------------------------------------------------------------------------------- */
#define EPWI_MLP_NPARAM 34433

typedef enum { EPWI_PROPOSAL_UNIFORM = 0, EPWI_PROPOSAL_LEARNED = 1 } epwi_proposal;

typedef struct {
    int32_t epochs;             /* passes over the training set (default 100) */
    int32_t batch;              /* samples per Adam step, <= 65536 (default 512) */
    double lr;                  /* Adam step size; cosine decay to lr/20 (default 2e-3) */
    double background;          /* uniformly drawn (k,q) pairs per sieved pair (default 1) */
    double floor_rel;           /* targets are log(t + floor_rel * max t) (default 1e-8) */
    uint64_t seed;              /* initialisation, background draw and shuffles (default 1) */
} epwi_mlp_train_options;

void epwi_mlp_default_train_options(epwi_mlp_train_options *opt);

/* Builds the training set on the current grid and trains the network with Adam.
 * Needs epwi_eigs.  The training set is every sieved (k,q) pair of the window [emin, emax],
 * plus background pairs drawn uniformly, times every window band and mode.  Its targets come
 * from the FP64 kernels at (T, mu, smear).  The network is initialised from opt->seed unless
 * parameters were set or trained before.  final_loss (may be NULL) receives the mean of
 * (yhat - y)^2 / 2 over the training set.
 * The terms are Gaussians of width smear in energy, so on a coarse grid they are spikes at
 * its q points.  A network trained on them transfers poorly to a finer grid.  Training with a
 * smear of 2-4x the production one spreads them into a shell the network can learn; the
 * estimate stays unbiased whatever the proposal.
 * Errors: ESTATE, EINVAL (empty window), EUNSUPPORTED (more than 2^26 sieved pairs). */
epwi_status epwi_mlp_train(epwi_ctx *ctx, double T_K, double mu_eV, double smear_eV,
                           double emin_eV, double emax_eV, const epwi_mlp_train_options *opt,
                           double *final_loss);

/* Sets the parameters (host, EPWI_MLP_NPARAM floats, layout above).  They become the FP32
 * master copy; the network computes with their BF16 rounding.  The output scale becomes 1 and
 * the shift 0. */
epwi_status epwi_mlp_set_params(epwi_ctx *ctx, const float *params);
/* The BF16-rounded parameters the network computes with (host, EPWI_MLP_NPARAM floats), and the
 * output affine map log t = scale * yhat + shift (either pointer may be NULL). */
epwi_status epwi_mlp_get_params(epwi_ctx *ctx, float *params, double *scale, double *shift);
/* Network output yhat for n host samples x [n][9] -> y [n] (reference SIMT kernels). */
epwi_status epwi_mlp_forward(epwi_ctx *ctx, int64_t n, const float *x, float *y);
/* The same on the tensor cores, as the proposal uses it: layer 1 in FP32, layers 2-3 as BF16
 * tcgen05 products with FP32 accumulation, activations rounded to BF16 between layers.
 * Errors: ESTATE, EINVAL, ETIMEOUT (a bounded wait in the kernel gave up). */
epwi_status epwi_mlp_forward_tc(epwi_ctx *ctx, int64_t n, const float *x, float *y);
/* One forward and backward pass over n <= 65536 host samples: loss = (1/2n) sum (yhat - y)^2,
 * grad [EPWI_MLP_NPARAM] = dloss/dparams (host), with respect to the BF16-rounded parameters. */
epwi_status epwi_mlp_loss_grad(epwi_ctx *ctx, int64_t n, const float *x, const float *y,
                               double *loss, float *grad);
/* The training set of the last epwi_mlp_train.  A size query when every pointer is NULL;
 * otherwise capacity must be >= n.  Per sample it gives:
 *   ids [n][4]: (k index, q index, band, mode);
 *   t [n]: the FP64 term of Eq. 10 (eV);
 *   x [n][9]: the features;
 *   y [n]: the normalised log target. */
epwi_status epwi_mlp_get_training_set(epwi_ctx *ctx, int64_t capacity, int32_t *ids, double *t,
                                      float *x, float *y, int64_t *n);

/* Importance-sampled 1/tau for every state in the window [emin, emax], S = samples_per_k draws
 * per k-point.  Needs epwi_eigs; for EPWI_PROPOSAL_LEARNED also a trained or set network.
 *   - Proposal EPWI_PROPOSAL_UNIFORM: p = 1/N_q.
 *   - Proposal EPWI_PROPOSAL_LEARNED: cells of cell_stride^3 grid points, one around every
 *     cell_stride-th point.  cell_stride must divide every grid dimension.  For each state
 *     the network scores every cell centre and mode, and
 *       p_n(q) = alpha/N_q + (1 - alpha) P_n(cell(q)) / cell_stride^3, with 0 < alpha <= 1.
 *     The bands of one k share one draw from the band mixture.
 * The weighted pairs run through the kernels of the context's precision (FP64, or a split
 * tensor-core mode with the weight applied per pair in FP32).  The result
 * replaces the rates of epwi_scatter_rates: epwi_get_rates, epwi_conductivity and
 * epwi_get_stats (n_pairs = distinct drawn pairs) read it.  Errors: ESTATE, EINVAL. */
epwi_status epwi_scatter_rates_is(epwi_ctx *ctx, double T_K, double mu_eV, double smear_eV,
                                  double emin_eV, double emax_eV, int64_t samples_per_k,
                                  double alpha, int32_t cell_stride, int32_t proposal,
                                  uint64_t seed, int64_t *n_states, int64_t *n_pairs);
/* The distinct drawn pairs of the last epwi_scatter_rates_is: k index, q index and weight
 * c_q / (S p(q)) per pair, grouped by k-point in window order and ascending q within a k-point.
 * A size query when every output pointer is NULL; otherwise capacity must be >= n. */
epwi_status epwi_get_is_pairs(epwi_ctx *ctx, int64_t capacity, int32_t *ik, int32_t *iq,
                              double *weight, int64_t *n);

/* ---------------------------------------------------------------------------------------
 * Batches of uneven systems.  Each system brings its own nw, nat, R-sets and grid.
 *
 * epwi_batch_plan runs each system's eigensolves, window and sieve count, then picks a tile
 * shape per system: the pairs per work item M_t and the K chunk of the Rp sum.  The
 * autotuner chooses it by timing candidates on a sample of each class (nw, 3 nat, n_Rp) and
 * caches the choice per class for the process.  The plan then captures one CUDA graph.  In
 * the graph, each system gets its eigensolves, sieve fill and FP32 Re->k stage.  Then ONE
 * persistent kernel works through a queue of (system, k-point, band, block of q) items
 * covering every system.  Per item it runs the Rp->q product, the rotations and the delta
 * sum of Eq. 10 in FP32, writing one FP64 sum per item.  Fixed-order FP64 reductions then
 * give 1/tau and sigma (Eq. 12) per system.  epwi_batch_run launches the graph.
 *
 * Limits: nw * 3 nat <= 512, states with an item queue below 2^31 items.
 * ------------------------------------------------------------------------------------- */
typedef struct epwi_batch epwi_batch;

typedef struct {
    int64_t n_systems, n_states, n_pairs, n_items;
    int64_t graph_nodes;        /* nodes of the captured step */
    int64_t persistent_ctas;    /* CTAs of the persistent kernel */
    int64_t smem_bytes;         /* its dynamic shared memory per CTA */
    int64_t runs;               /* graph launches so far */
    double ms_plan;             /* device time of the planning pass (incl. autotuning) */
    double ms_graph;            /* last graph launch, whole step */
    double ms_persistent;       /* last graph launch, the persistent kernel */
    double scatter_flops;       /* algorithmic flops of the persistent kernel (one pass): the
                                   Rp->q products (for a cube R_p of side D the axis-1
                                   factorisation, 8 D^2 N_m W per pair and band plus
                                   8 D^3 N_m W per item; otherwise 8 n_Rp N_m W per pair and
                                   band) and the rotations (8 W (N_m W + N_m^2) per pair and
                                   band) */
    double restage_flops;       /* algorithmic flops of the Re->k stages */
} epwi_batch_stats;

/* Creates a batch on opt->device (NULL: defaults).  With opt->cuda_stream NULL the batch makes
 * its own non-blocking stream. */
epwi_status epwi_batch_create(epwi_batch **batch, const epwi_options *opt);
void epwi_batch_destroy(epwi_batch *batch);
const char *epwi_batch_last_error(const epwi_batch *batch);
/* Copies and validates nsys systems (as epwi_setup) with their Gamma-centred grids
 * grids[nsys][3]. */
epwi_status epwi_batch_setup(epwi_batch *batch, int32_t nsys, const epwi_system *systems,
                             const int32_t *grids);
/* Appends one system with its grid[3]; its host arrays may be freed when the call returns.
 * index (may be NULL) receives its position in the batch. */
epwi_status epwi_batch_add(epwi_batch *batch, const epwi_system *sys, const int32_t *grid,
                           int32_t *index);
/* Band range (min, max of eps over all bands) of system s on its grid, for choosing mu and
 * windows before planning (runs that system's eigensolves). */
epwi_status epwi_batch_band_range(epwi_batch *batch, int32_t s, double *emin, double *emax);
/* Plans the step for temperature T, chemical potentials mu[nsys], smearing and per-system
 * windows [emin, emax]; autotune_tiles != 0 runs the autotuner (otherwise a default shape,
 * or the one set by epwi_batch_set_tile).  n_pairs (may be NULL) receives the sieved pairs
 * of all systems. */
epwi_status epwi_batch_plan(epwi_batch *batch, double T_K, const double *mu_eV, double smear_eV,
                            const double *emin_eV, const double *emax_eV, int32_t autotune_tiles,
                            int64_t *n_pairs);
/* One step (one graph launch); sigma (host, [nsys][9] S/m, may be NULL) receives every
 * system's conductivity. */
epwi_status epwi_batch_run(epwi_batch *batch, double *sigma);
/* 1/tau of system s after a run (layout as epwi_get_rates; size query with NULL outputs). */
epwi_status epwi_batch_get_rates(epwi_batch *batch, int32_t s, int64_t capacity, int32_t *k_idx,
                                 int32_t *band, double *inv_tau_s, int64_t *n_states);
/* Forces the tile shape of system s for the next plan (mt = 0 clears it). */
epwi_status epwi_batch_set_tile(epwi_batch *batch, int32_t s, int32_t mt, int32_t kc);
/* Tile shape of system s in the current plan; source: 0 default, 1 autotuned now, 2 from
 * the autotuner's cache, 3 set by epwi_batch_set_tile. */
epwi_status epwi_batch_get_tile(epwi_batch *batch, int32_t s, int32_t *mt, int32_t *kc,
                                int32_t *source);
epwi_status epwi_batch_get_stats(epwi_batch *batch, epwi_batch_stats *out);

/* Transport tensors of the last epwi_scatter_rates or epwi_scatter_rates_is (Sec. II C,
 * Eqs. 12-14, with F = v tau).  Let w = tau f(1-f)/(k_B T).  Then:
 *   sigma        = (2 e^2/(N_k V)) sum w v v                      [S/m];
 *   nu = sigma S = (2 q/(T V N_k)) sum (eps - mu) w v v, q = -e   [A/(m K)];
 *   kappa_0      = (2/(T V N_k)) sum (eps - mu)^2 w v v           [W/(m K)];
 *   S = sigma^-1 nu                                               [V/K];
 *   kappa_e = kappa_0 - T nu sigma^-1 nu, the tensor form of kappa_0 - T sigma S^2.
 * Outputs are row-major 3x3 (any pointer may be NULL).  The three moments come from one
 * fixed-order FP64 device reduction.  Errors: ESTATE; ENUMERIC (singular sigma). */
epwi_status epwi_transport(epwi_ctx *ctx, double sigma[9], double seebeck[9], double kappa_e[9]);

/* Iterative Boltzmann transport equation (Sec. II C, the iteration equation after Eq. 10).
 *   F^0_nk = v_nk tau_nk;
 *   F^(i+1)_nk = F^0_nk + tau_nk sum_{q p m} Gamma_{nk -> m,k+q} F^i_{m,k+q}.
 * Gamma is the equilibrium transition rate with f_nk (1 - f_nk) divided out.  By detailed
 * balance it equals the summand of Eq. 10 for the final state (m, k+q) and mode p, summed
 * over the two signs.  1/tau_nk is therefore the sum of Gamma over all final states.
 *
 * The call runs what epwi_scatter_rates runs for (T, mu, smear, emin, emax), which also
 * leaves 1/tau for epwi_get_rates and epwi_transport.  During the interpolation it stores
 * Gamma for final states inside the window, as one block [n in window(k)][m in
 * window(k+q)] per sieved pair, in pair order.  Blocks are FP64 on the FP64 path and FP32
 * on the split paths.  Final states outside the window keep their share of 1/tau and carry
 * F = 0.  States with 1/tau = 0 have F = 0.
 *
 * The step is one kernel per iteration: one block per window k-point, fixed-order sums, so
 * the result is deterministic.  It stops when max |F^(i+1) - F^i| <= tol max |F^(i+1)|, or
 * after max_iter steps (max_iter = 0: F = F^0).
 *
 * iters, change: steps done and the last relative change (either may be NULL).
 * Errors: ESTATE (no eigs); EINVAL (T, smear, window, max_iter < 0, tol < 0); ENOMEM. */
epwi_status epwi_ibte(epwi_ctx *ctx, double T, double mu, double smear, double emin, double emax,
                      int32_t max_iter, double tol, int32_t *iters, double *change);
/* Mean free paths F [n_states][3] in m after epwi_ibte, in the state order of epwi_get_rates.
 * Errors: ESTATE; ETOOSMALL (capacity below n_states). */
epwi_status epwi_get_mfp(epwi_ctx *ctx, int64_t capacity, double *F);
/* sigma, Seebeck and kappa_e from F (Sec. II C, Eqs. 12-14): the moments of epwi_transport
 * with tau v_a v_b replaced by v_a F_b (a full 3x3 tensor; v_a is the row).  Errors: ESTATE;
 * ENUMERIC. */
epwi_status epwi_ibte_transport(epwi_ctx *ctx, double sigma[9], double seebeck[9], double kappa_e[9]);
epwi_status epwi_get_ibte_stats(epwi_ctx *ctx, epwi_ibte_stats *out);

/* Number of kernels this library has launched in the process so far (all contexts). */
int64_t epwi_kernel_launches(void);

/* Measured FMA throughput of the device, the denominator of the roofline fractions of the
 * SIMT kernels (the paper has no counterpart; it reports no roofline).  fp64 = 0 times FP32
 * FMAs, fp64 = 1 FP64 FMAs: every thread of 8 CTAs per SM runs 8 independent register-only
 * FMA chains, the launch is sized from a calibration run to about target_ms, and the best of
 * three timed launches (CUDA events on cuda_stream, NULL = legacy default stream) is returned
 * in *tflops (2 flop per FMA) and its duration in *ms (may be NULL).  Synchronises the stream.
 * Allocates a 2 KiB sink buffer for the duration of the call.  Errors: EINVAL (NULL tflops,
 * target_ms <= 0, fp64 not 0 or 1), ECUDA. */
epwi_status epwi_fma_peak(int32_t fp64, int32_t device, void *cuda_stream, double target_ms,
                          double *tflops, double *ms);

/* Statistics of the last epwi_scatter_rates. */
epwi_status epwi_get_stats(epwi_ctx *ctx, epwi_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* EPWI_H */
