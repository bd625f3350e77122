/*
 * sps.h - C ABI of the GB300 (sm_103a) SPS photometry / likelihood / HMC library.
 *
 * The library evaluates, for every (galaxy, chain) row, the stellar population
 * synthesis model of arXiv 2506.19919 and its Gaussian photometric likelihood:
 *
 *   L_gal(lambda) = M_star sum_ij L_SSP(lambda | tau_i, Z_j) F_att(lambda) P_SFH(tau_i) P_met(Z_j)
 *                                                      (Eq. galSEDdef, Eq. galSED_decomposed)
 *   c_b = int dlambda T_b(lambda | z) L_gal(lambda)     (Eq. photo_integral_exact)
 *   c_b ~ F_att(lambda_eff,b) sum_ij P_ij c_SSP,b,ij(z) (Eq. lambda_eff, Eq. photo_integral_approx)
 *   log L = -1/2 sum_b ((m_b - m_obs,b) / sigma_b)^2    (App. D.1)
 *
 * and runs batched Hamiltonian Monte Carlo over it (Sec. 4, App. D.2).
 *
 * Conventions shared by every entry point:
 *  - Parameters: 12 physical columns per row, in this order (App. A.1-A.3):
 *      0 lgM       log10 SFR amplitude M_formed [M_sun/yr] (Eq. SFRsmooth)
 *      1 tau       double-power-law turnover time [Gyr]
 *      2 alpha     falling slope          3 beta   rising slope
 *      4 F_burst   burst mass fraction (Eq. composite_age_weights)
 *      5 lgT_peak  log10 burst peak age [yr] (Eq. triweight)
 *      6 dlgT      log10 T_max - log10 T_peak [dex] (sigma_burst = dlgT / 3)
 *      7 lgZ       mean of the Gaussian in log10 Z/Z_sun (App. A.2)
 *      8 sigma_lgZ width of that Gaussian [dex]
 *      9 A_V       10 delta   11 F_floor   (Eq. DustAtt and the F_floor equation)
 *    The redshift is per galaxy and fixed (it is data, not a parameter).
 *  - Rows are (galaxy, chain) pairs.  A row refers to a galaxy of the set given
 *    to sps_set_galaxies, either by gal_idx[row] or, when gal_idx is NULL, by
 *    row == galaxy (then n must equal the galaxy count).
 *  - Every array argument may be a host pointer or a device pointer of the
 *    context's device; the library detects which (cudaPointerGetAttributes)
 *    and stages host arrays through its own device buffers.  An array in the
 *    memory of another device gives SPS_E_INVALID_ARG.  Each call makes the
 *    context's device current and restores the caller's current device before
 *    it returns.  With device
 *    pointers the call is asynchronous on `stream` (a cudaStream_t, NULL =
 *    legacy default stream); with any host pointer it synchronises `stream`
 *    before returning.  The caller keeps ownership of every array.
 *  - Row-major, C-contiguous layouts; float32 unless stated.
 *  - Errors are returned as sps_status; nothing is thrown across the ABI.
 *    Shapes and arguments are checked on the host before any launch.  After
 *    SPS_E_CUDA the context should be destroyed.  sps_last_error_message()
 *    gives a human-readable reason for the last failure of this thread.
 *  - A context is not thread-safe: use one context per host thread.
 */
#ifndef SPS_GB300_H
#define SPS_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPS_NPARAM 12
#define SPS_MAX_BANDS 32
#define SPS_MAX_AGES 128
#define SPS_MAX_METS 32

typedef struct sps_ctx sps_ctx; /* opaque; owned by the library */

typedef enum {
    SPS_OK = 0,
    SPS_E_INVALID_ARG = 1, /* NULL pointer, bad enum, non-increasing grid, bad band */
    SPS_E_SHAPE = 2,       /* sizes out of range or inconsistent                   */
    SPS_E_NONFINITE = 3,   /* some output rows are NaN because inputs were         */
    SPS_E_CUDA = 4,        /* a CUDA runtime call failed                          */
    SPS_E_TIMEOUT = 5,     /* a bounded device wait gave up (HMC work queue)       */
    SPS_E_UNSUPPORTED = 6, /* mode / precision / device not supported              */
    SPS_E_STATE = 7,       /* call order: e.g. no galaxy set, or no approx tables */
    SPS_E_NOMEM = 8        /* device allocation failed                             */
} sps_status;

typedef enum { SPS_EXACT = 0, SPS_APPROX = 1 } sps_mode;
/* Arithmetic of the exact path's SSP contraction:
 *  SPS_FP32   FP32 SIMT (the reference precision: ~4e-6 mag, gradients ~1e-5);
 *  SPS_BF16   BF16 operands with per-age-row power-of-two scaling, FP32
 *             accumulation on the tensor cores (~1e-3 mag);
 *  SPS_TF32X3 FP32 operands split into TF32 halves, hi*hi + hi*lo + lo*hi on
 *             the tensor cores (~3e-5 mag, gradients ~1e-3: the tensor-core
 *             accumulation over the 1284-term contraction limits it). */
typedef enum { SPS_FP32 = 0, SPS_BF16 = 1, SPS_TF32X3 = 2 } sps_prec;
typedef enum { SPS_BAND_TOPHAT = 0, SPS_BAND_GAUSS = 1, SPS_BAND_TABLE = 2 } sps_band_kind;

/* Model grids, SSP table and filters (host memory, float64; copied in).
 *  age_yr[n_age]  strictly increasing SSP ages [yr]
 *  lgZ[n_met]     strictly increasing log10(Z/Z_sun) grid
 *  lam_ang[n_lam] strictly increasing rest-frame wavelengths [Angstrom]
 *  ssp[n_age*n_met*n_lam] L_SSP[i][j][n] in L_sun/Hz per solar mass formed
 *  band_kind[n_band], band_p0, band_p1: observed-frame filters;
 *    TOPHAT: transmission 1 on [p0, p1) Angstrom;
 *    GAUSS:  transmission exp(-(l - p0)^2 / (2 s^2)), s = p1 / (2 sqrt(2 ln 2)) (p1 = FWHM),
 *            integrated over |l - p0| < 6 s (the rest is 2e-9 of the band's weight);
 *    TABLE:  a measured throughput curve (Sec. 5 uses LSST's): band_tab_n[b] >= 2
 *            samples T_m >= 0 at l = p0 + m p1 Angstrom (p0 > 0, p1 > 0), the
 *            transmission their linear interpolant, zero outside the samples.
 *  band_tab_n[n_band]: samples per TABLE band (ignored for the others; the
 *    pointer may be NULL when no band is tabulated); band_tab_T: the TABLE
 *    bands' samples, concatenated in band order.  Resample curves with uneven
 *    steps onto a uniform grid first (paper_2506_19919_gb300.loaders does).
 *  mdf_offset[n_age] or NULL: a non-separable SSP weighting (Sec. 2: the MDF
 *    following the time evolution of the mass-metallicity relation): the
 *    metallicity distribution of stars in age bin i has mean lgZ +
 *    mdf_offset[i] (width sigma_lgZ shared), so W_ij = M_star P_SFH,i
 *    P_met,ij is a general [n_age x n_met] matrix.  NULL: the separable model.
 *    The forward-mode comparison baselines support only the separable model. */
typedef struct {
    int32_t n_age, n_met, n_lam, n_band;
    const double* age_yr;
    const double* lgZ;
    const double* lam_ang;
    const double* ssp;
    const int32_t* band_kind;
    const double* band_p0;
    const double* band_p1;
    const int32_t* band_tab_n;
    const double* band_tab_T;
    const double* mdf_offset;
} sps_tables;

/* Prior on the unbounded parameters x (App. C).  SPS_PRIOR_UNIFORM: uniform in
 * each bounded parameter theta = F_B(x), i.e. the log of the Jacobian of Eq.
 * BoundingFunction, log s (1 - s) with s = 1 / (1 + exp(-k (x - x0))) (the
 * constant log(k (hi - lo)) dropped).  SPS_PRIOR_SKEWNORMAL: the skew-normal
 * of Eq. SkewNormPrior on x, log(2 / omega) + log N((x - xi) / omega)
 * + log Phi(s (x - xi) / omega), a normalised density (the paper fits xi,
 * omega, s to prior draws mapped through F_B^-1; paper_2506_19919_gb300.priors
 * does that on the host). */
typedef enum { SPS_PRIOR_UNIFORM = 0, SPS_PRIOR_SKEWNORMAL = 1 } sps_prior;

/* Context configuration.  sps_config_default() fills the declared defaults:
 * flat LambdaCDM with H0 = 70 km/s/Mpc, Omega_m = 0.3 (the paper states none),
 * the package's prior bounds, device 0, Gauss-Legendre order 6 and panel width
 * 0.25 in ln t for the SFH bin integrals, bounding functions with k = 1,
 * x0 = 0 and the uniform prior.  The SFH bin integrals use panels of
 * sfh_panel * 10 / kappa in ln t, kappa = max(alpha + beta, beta + 1), clamped
 * to [1, 8] x sfh_panel, with the sfh_gl_order rule on each; a bin that fits in
 * one panel and is narrow against 1 / kappa takes a 2- or 3-node rule (never
 * more nodes than sfh_gl_order). */
typedef struct {
    double h0_kms_mpc;
    double omega_m;
    double prior_lo[SPS_NPARAM];
    double prior_hi[SPS_NPARAM];
    int32_t device;
    int32_t sfh_gl_order; /* 2..16 */
    double sfh_panel;     /* panel width in ln t at kappa = 10, (0, 2] */
    double sigmoid_k[SPS_NPARAM];   /* Eq. BoundingFunction k per parameter, > 0 (1)   */
    double sigmoid_x0[SPS_NPARAM];  /* Eq. BoundingFunction x0 per parameter (0)       */
    int32_t prior;                  /* sps_prior (SPS_PRIOR_UNIFORM)                   */
    double skew_xi[SPS_NPARAM];     /* Eq. SkewNormPrior location per parameter (0)    */
    double skew_omega[SPS_NPARAM];  /* Eq. SkewNormPrior scale per parameter, > 0 (1)  */
    double skew_s[SPS_NPARAM];      /* Eq. SkewNormPrior shape per parameter (0)       */
} sps_config;

sps_status sps_config_default(sps_config* cfg);

/* Create a context on cfg->device: validates and uploads the tables (FP32,
 * BF16 row-scaled and per-wavelength dust constants).  On success *out owns
 * device memory until sps_destroy.  Sec. 2 (fixed SSP library), App. A.3.
 * cfg may be NULL (the defaults).  The tables are read, not kept.
 * Errors (*out stays NULL; sps_last_error_message() names the failed check).
 * Every table and config check runs on the host before any device work:
 *   SPS_E_SHAPE       n_age outside [2, 128], n_met outside [1, 32],
 *                     n_lam < 2, n_band outside [1, 32], n_age * n_met > 1312;
 *   SPS_E_INVALID_ARG a NULL pointer; a grid that is not positive and
 *                     increasing (ages, wavelengths) or not increasing (lgZ);
 *                     an SSP value that is negative or not finite; a bad band
 *                     (unknown kind, top-hat without 0 < p0 < p1, Gaussian
 *                     without positive centre and FWHM, tabulated without
 *                     start > 0, step > 0, 2..2^20 finite samples >= 0);
 *                     an mdf_offset that is not finite or exceeds 10 dex;
 *                     a config field out of range (sfh_gl_order, sfh_panel or
 *                     a panel too small for the panel budget, H0 <= 0,
 *                     Omega_m outside (0, 1), prior_hi <= prior_lo,
 *                     sigmoid_k <= 0 or not finite, sigmoid_x0 not finite,
 *                     an unknown prior, and for the skew-normal prior
 *                     omega <= 0 or a parameter that is not finite);
 *   SPS_E_UNSUPPORTED no CUDA device, or one older than sm_100;
 *   SPS_E_INVALID_ARG a device ordinal out of range;
 *   SPS_E_CUDA / SPS_E_NOMEM a failed device call or allocation. */
sps_status sps_create(sps_ctx** out, const sps_tables* tables, const sps_config* cfg);
sps_status sps_destroy(sps_ctx* ctx);

/* Set the galaxies (their redshifts z[n_gal], float32) that later rows refer to.
 * Computes per galaxy, in FP64: t_obs(z), d_L(z), the age bins in cosmic time
 * (Eq. smoothPsfh), band supports, band normalisations and AB zero points, and,
 * if build_approx != 0, lambda_eff (Eq. lambda_eff) and the per-galaxy table
 * c_SSP[g][b][ij] (the c_SSP definition of Sec. 3, "at a fixed z if the
 * redshift is known").  Replaces any previous set.  Synchronous. */
sps_status sps_set_galaxies(sps_ctx* ctx, const float* z, int64_t n_gal, int32_t build_approx,
                            void* stream);

/* AB magnitudes of n rows: theta[n][12] -> mag_out[n][n_band].
 * mode EXACT: Eq. photo_integral_exact (SSP contraction over the full
 * wavelength grid, dust and filters applied per wavelength); prec selects the
 * contraction arithmetic (sps_prec).  mode APPROX: Eq. photo_integral_approx
 * (FP32; prec must be SPS_FP32).  Rows whose theta is non-finite give NaN
 * magnitudes and SPS_E_NONFINITE (the other rows are still valid). */
sps_status sps_photometry(sps_ctx* ctx, const float* theta, const int32_t* gal_idx, int64_t n,
                          sps_mode mode, sps_prec prec, float* mag_out, void* stream);

/* Gaussian log-likelihood (App. D.1) of n rows and its gradient with respect
 * to the 12 physical parameters, by a hand-written adjoint that recomputes the
 * per-SSP products instead of storing them.
 *  mag_obs[n_gal][n_band], sigma[n_gal][n_band]: per-galaxy data;
 *  mask[n_gal]: bit b set <=> band b enters the likelihood;
 *  loglike_out[n]; grad_out[n][12] or NULL (value only). */
sps_status sps_loglike_grad(sps_ctx* ctx, const float* theta, const int32_t* gal_idx, int64_t n,
                            const float* mag_obs, const float* sigma, const uint32_t* mask,
                            sps_mode mode, sps_prec prec, float* loglike_out, float* grad_out,
                            void* stream);

/* sps_loglike_grad with a 13th gradient column: the derivative of each row's
 * log L with respect to its galaxy's redshift z, for fits that free z (the
 * SPS redshift parameter; Sec. 3 T(lambda | z) and c_SSP(z), App. A.1
 * t_obs(z)).  grad_out[n][13]: columns 0-11 as sps_loglike_grad, column 12
 * d log L / dz through the observed-frame filters T((1+z) lambda), the band
 * normalisation N_b(z), d_L(z), the (1+z) bandwidth factor, lambda_eff(z) and
 * c_SSP(z) (approximate path), and t_obs(z) (age bins, mass formed, burst
 * clipping).  Needs a filter set without top-hat bands (the rest-grid filter
 * sum of a top-hat is piecewise constant in z): SPS_E_UNSUPPORTED otherwise.
 * The approximate path builds, on its first call after sps_set_galaxies, a
 * d c_SSP / dz table the size of c_SSP (SPS_E_NOMEM if it does not fit).
 * Arguments, precisions and errors otherwise as sps_loglike_grad; grad_out
 * must not be NULL. */
sps_status sps_loglike_grad_z(sps_ctx* ctx, const float* theta, const int32_t* gal_idx, int64_t n,
                              const float* mag_obs, const float* sigma, const uint32_t* mask,
                              sps_mode mode, sps_prec prec, float* loglike_out, float* grad_out,
                              void* stream);

/* Comparison baseline, not a product path: the same approximate-path log L and
 * gradient as sps_loglike_grad (SPS_APPROX), computed the plain way a direct
 * GPU port would: unfused kernels with their intermediates in HBM and the
 * gradient by forward-mode tangents (one contraction per weight parameter,
 * 9 in all, against ~2 for the hand-written adjoint).  Same arguments and
 * layouts as sps_loglike_grad. */
sps_status sps_loglike_grad_forward_mode(sps_ctx* ctx, const float* theta, const int32_t* gal_idx,
                                         int64_t n, const float* mag_obs, const float* sigma,
                                         const uint32_t* mask, float* loglike_out, float* grad_out,
                                         void* stream);

/* Batched HMC configuration (Sec. 4, App. D.2). */
typedef struct {
    int32_t chains_per_gal; /* C >= 1; chain c of galaxy g is row g*C + c          */
    int32_t n_warm;         /* adaptation iterations (dual-averaged step size)      */
    int32_t n_samp;         /* sampling iterations                                 */
    int32_t L_min, L_max;   /* leapfrog steps per trajectory ~ U{L_min..L_max}      */
    float target_accept;    /* dual-averaging target (0.8)                        */
    float eps0;             /* initial step size (0.1)                            */
    uint64_t seed;          /* Philox-4x32-10 key                                 */
    int32_t mode;           /* sps_mode (APPROX runs the persistent fused kernel)  */
    int32_t prec;           /* sps_prec (EXACT only)                              */
    int32_t use_graph;      /* capture the device work in a CUDA graph             */
    int32_t autotune;       /* pick the launch shape by timing candidates          */
    int32_t adapt_mass;     /* warm-up metric: 0 identity (default), 1 diagonal, 2 dense */
    int32_t sampler;        /* sps_sampler: SPS_HMC (default) or SPS_NUTS             */
    int32_t max_depth;      /* NUTS tree depth limit, 1..10 (10): <= 2^depth - 1 leaves */
} sps_hmc_config;

/* Sampler of sps_hmc_run.  SPS_NUTS is the No-U-Turn Sampler the paper sets
 * beside HMC (Sec. 4, App. D.2): multinomial NUTS with the generalised U-turn
 * criterion (Hoffman & Gelman 2014; Betancourt 2017), identity metric; every
 * aligned block of leaves of a new subtree is checked as it completes, a
 * subtree is taken with probability min(1, W_subtree / W_trajectory), a leaf
 * inside it by progressive multinomial sampling, divergence at dH > 1000.
 * Step size by dual averaging on the mean over the leaves built of
 * min(1, exp(-dH)).  L_min / L_max are ignored; adapt_mass must be 0.
 * Draws: Philox-4x32-10 counters (iteration, 0..2, chain, 0) for the momentum
 * (as HMC), (iteration, 16 + j, chain, 0) for the direction (word 0, top bit
 * set = forward) and subtree uniform (word 1) at depth j, and
 * (iteration, 64 + j, chain, n) word 0 for leaf n of that subtree.
 * stats->grad_evals counts the leaves built (+1); accept_prob is the mean of
 * that statistic over the sampling phase. */
typedef enum { SPS_HMC = 0, SPS_NUTS = 1 } sps_sampler;

sps_status sps_hmc_config_default(sps_hmc_config* cfg);

/* Per-chain statistics (each pointer may be NULL; host or device). */
typedef struct {
    float* accept_prob;   /* [G*C] mean Metropolis acceptance probability, sampling phase */
    float* step_size;     /* [G*C] step size used for sampling                           */
    int32_t* divergences; /* [G*C] trajectories with non-finite or > 1000 energy error    */
    int64_t* grad_evals;  /* [G*C] log-posterior gradient evaluations                     */
    int32_t* status;      /* [G*C] 0 finished, 1 not finished (timeout)                   */
} sps_hmc_stats;

/* Run batched HMC (or NUTS, cfg->sampler) for every chain of every galaxy of
 * the current set.  Warm-up adapts, per chain, the step size by dual averaging (Hoffman & Gelman
 * 2014) and, if adapt_mass is 1 (2), a diagonal (dense) inverse metric in
 * windows (75-iteration initial buffer, slow windows of 25, 50, 100, ...,
 * 50-iteration terminal buffer; regularised variances (covariance) of each
 * window's positions; a dense metric M^-1 = L L^T gives momenta L^-T z).
 * The target is log L (App. D.1) plus the log prior the context's sps_config
 * selects on the unbounded parameters x, where theta = lo + (hi - lo) /
 * (1 + exp(-k (x - x0))) (Eq. BoundingFunction with the config's per-parameter
 * sigmoid_k and sigmoid_x0): by default the log-Jacobian of that map, i.e. a
 * prior uniform in each bounded parameter, else the skew-normal of
 * Eq. SkewNormPrior (sps_prior); sampling is in x.
 *  theta0_unb[G*C][12]: start points in unbounded space;
 *  samples_out[G*C][n_samp][12]: bounded (physical) draws, or NULL.
 * cfg->mode APPROX (Eq. photo_integral_approx) runs the persistent fused
 * kernel (HMC or NUTS, any metric).  cfg->mode EXACT (Eq. photo_integral_exact;
 * the paper's exact-photometry HMC, Sec. 3) runs HMC with the identity metric
 * in rounds: each round evaluates every chain's log L and gradient through the
 * exact path in cfg->prec (the tensor-core contractions for SPS_BF16 and
 * SPS_TF32X3) and takes one leapfrog step of every chain, a chain whose
 * trajectory has ended starting its next iteration at once; same draws and
 * sampler as the approximate path's HMC.  Synchronous; SPS_E_UNSUPPORTED for
 * NUTS or an adapted metric in this mode.
 * Random numbers: Philox-4x32-10 keyed by seed, counter (iteration, block,
 * chain, 0) (NUTS: the counters listed at sps_sampler); a run is a pure
 * function of its inputs.  NUTS state takes 1.3 KB of device memory per chain. */
sps_status sps_hmc_run(sps_ctx* ctx, const sps_hmc_config* cfg, const float* theta0_unb,
                       const float* mag_obs, const float* sigma, const uint32_t* mask,
                       float* samples_out, sps_hmc_stats* stats, void* stream);

/* Comparison baseline for sps_hmc_run (not a product path): the same sampler
 * (identity metric, same Philox streams, dual averaging, FP64 accept) run the
 * way a vectorised port of the paper's batched HMC (Sec. 4, App. D.2) runs it.
 * All chains advance in lock step; each iteration takes L_max rounds, and every
 * round evaluates every chain with the unfused forward-mode gradient of
 * sps_loglike_grad_forward_mode whether or not its trajectory has ended.
 * Arguments, layouts and outputs as sps_hmc_run; stats->grad_evals counts the
 * evaluations performed (1 + (n_warm + n_samp) L_max per chain).
 * SPS_E_UNSUPPORTED unless cfg->adapt_mass == 0, cfg->sampler == SPS_HMC and
 * cfg->mode == SPS_APPROX. */
sps_status sps_hmc_run_forward_mode(sps_ctx* ctx, const sps_hmc_config* cfg, const float* theta0_unb,
                                    const float* mag_obs, const float* sigma, const uint32_t* mask,
                                    float* samples_out, sps_hmc_stats* stats, void* stream);

/* Deterministic leapfrog trajectories (the HMC integrator of App. D.2 without
 * the random draws): for each row, L[row] steps of size eps[row] from
 * (x0, p0) in unbounded space; writes the end point, its momentum and log
 * posterior.  Uses the same device code as sps_hmc_run (APPROX mode). */
sps_status sps_leapfrog(sps_ctx* ctx, const float* x0, const float* p0, const float* eps,
                        const int32_t* L, const int32_t* gal_idx, int64_t n, const float* mag_obs,
                        const float* sigma, const uint32_t* mask, float* x_out, float* p_out,
                        double* logp_out, void* stream);

/* Test hook for failure detection without a GPU fault: runs the bounded
 * mbarrier wait of the tensor-core pipeline on a barrier that is completed
 * (ready != 0) or never completed (ready == 0).  The wait polls at most
 * spin_limit times (1 .. 2^26), then flags the timeout and the kernel returns,
 * so the context stays usable.  Returns SPS_OK or SPS_E_TIMEOUT. */
sps_status sps_wait_probe(sps_ctx* ctx, int32_t ready, uint32_t spin_limit, void* stream);

/* The device Philox-4x32-10 generator: out[n][4] = philox(ctr[n][4], key).
 * (Salmon et al. 2011; the generator behind every HMC draw.) */
sps_status sps_philox(sps_ctx* ctx, const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out,
                      void* stream);

/* SSP weights of n rows: W[n][n_age*n_met] = M_star P_SFH,i P_met,j (Eq.
 * galSED_decomposed with Eq. composite_age_weights) and M_star[n] in M_sun. */
sps_status sps_weights(sps_ctx* ctx, const float* theta, const int32_t* gal_idx, int64_t n,
                       float* W_out, double* mstar_out, void* stream);

/* Host-side diagnostics (FP64): multi-chain effective sample size with Geyer's
 * initial monotone sequence and split R-hat (Gelman-Rubin, Sec. 4), per galaxy
 * and parameter, of samples[G*C][N][P] (host memory).  ess_out, rhat_out:
 * [G][P] (either may be NULL). */
sps_status sps_diagnostics(const float* samples, int64_t n_gal, int32_t chains_per_gal,
                           int32_t n_draws, int32_t n_param, double* ess_out, double* rhat_out);

/* Host-side split of a galaxy catalogue over n_parts processes (one per GPU).
 * Galaxies are independent units (Sec. 4 fits them in parallel with no
 * exchange), so the split is into contiguous blocks; a galaxy weighs
 * base_weight plus its observed bands (the set bits of mask[g]), the part of
 * an evaluation's cost that varies between galaxies, and the heaviest block is
 * made as light as possible (exact for these integer weights).  While
 * n_gal >= n_parts every block holds at least one galaxy; with fewer galaxies
 * each has its own block and the trailing blocks are empty.  If every weight
 * is 0 the counts are balanced.
 *   mask        host [n_gal] band bitmasks, or NULL (weights base_weight)
 *   starts_out  host [n_parts + 1]: block p is galaxies [starts_out[p],
 *               starts_out[p + 1]); starts_out[0] = 0, starts_out[n_parts] = n_gal
 * Errors: SPS_E_INVALID_ARG (starts_out NULL, base_weight < 0), SPS_E_SHAPE
 * (n_gal < 0, n_parts < 1).  No device work. */
sps_status sps_partition_galaxies(const uint32_t* mask, int64_t n_gal, int32_t base_weight, int32_t n_parts,
                                  int64_t* starts_out);

/* Sizes and a few derived quantities of a context (host integers). */
typedef struct {
    int32_t n_age, n_met, n_lam, n_band, k_pad;
    int64_t n_gal;
    int32_t has_approx;
    int32_t device;
    int32_t sfh_gl_order;
    int32_t max_panels;
    int32_t hmc_launches;   /* sampler-kernel launches of the last approximate-path
                               sps_hmc_run: 1, or 2 when its last wave of two-chain
                               teams ran as one-chain teams (0 before any run) */
} sps_info;
sps_status sps_get_info(const sps_ctx* ctx, sps_info* out);

/* Gauss-Legendre rule the library built for the SFH integrals (host copy):
 * nodes[order], weights[order] on [-1, 1]. */
sps_status sps_gl_rule(const sps_ctx* ctx, double* nodes, double* weights);

/* Exact FP32 photometry (the computation of sps_photometry with SPS_EXACT,
 * SPS_FP32) for callers that cannot allocate device memory while running:
 * services that reserve a fixed device-memory budget at start-up, hosts whose
 * allocator owns the device memory, and loops where cudaMalloc would
 * synchronise the device or fail on a fragmented heap.  This call performs no
 * cudaMalloc, cudaFree or other allocation: its scratch is a fixed 32 MiB
 * array compiled into the library (resident on every GPU that loads the
 * library until the process exits), so at most
 * floor(32 MiB / (4 * k_pad + 16 * n_band)) rows fit in one call, about 6,100
 * rows for a 107 x 12 x 5994 grid with 6 bands; larger n returns SPS_E_SHAPE
 * with a message.  theta, gal_idx and mag_out must be device pointers (host
 * arrays would need staging buffers): SPS_E_INVALID_ARG otherwise.  The first
 * call on a device looks the array's device address up (cudaGetSymbolAddress)
 * and should come before any stream capture (it looks it up again if the
 * device's context has been reset since).  All calls share the array;
 * calls that overlap on the GPU race.  The call synchronises `stream` to
 * report SPS_E_NONFINITE, and restores the caller's current device.  The
 * paper has no counterpart. */
sps_status sps_photometry_exact_noalloc(sps_ctx* ctx, const float* theta, const int32_t* gal_idx,
                                        int64_t n, float* mag_out, void* stream);

const char* sps_error_string(sps_status status);
const char* sps_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* SPS_GB300_H */
