// Internal declarations shared by the host runtime and the CUDA kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sps.h"

namespace sps {

constexpr int kMaxAges = SPS_MAX_AGES;   // bins per row held in shared memory
constexpr int kMaxMets = SPS_MAX_METS;
constexpr int kMaxBands = SPS_MAX_BANDS;
constexpr int kMaxGL = 16;
constexpr int kMaxPanels = 512;          // SFH panels per row (checked on the host)
constexpr int kKTileMax = 41;            // ceil(K / 32) held in registers: K <= 1312
constexpr int kWarpsApprox = 4;          // warps per block of the fused approximate kernel

// Tables-wide constants handed to every kernel by value.
struct Consts {
    int n_age, n_met, n_lam, n_band, K, k_pad;
    int lam_pad;                          // wavelength stride of the padded tables
    int gl_order;
    float panel;                          // panel width in ln t at kappa = 10 (SFH quadrature)
    float gl_x[kMaxGL], gl_w[kMaxGL];     // Gauss-Legendre rule on [-1, 1] for full panels
    float gl2_x[2], gl2_w[2];             // 2- and 3-node rules for narrow bins
    float gl3_x[3], gl3_w[3];
    float log_age_edge[kMaxAges + 1];     // log10 age-bin edges [yr]; [0] = -100 stand-in
    float lgz_edge[kMaxMets + 1];         // metallicity-bin edges; outer +-inf
    float prior_lo[SPS_NPARAM], prior_span[SPS_NPARAM];
    float sig_k[SPS_NPARAM], sig_x0[SPS_NPARAM];   // Eq. BoundingFunction slope and centre
    int prior_kind;                                // sps_prior
    float sn_xi[SPS_NPARAM], sn_iom[SPS_NPARAM];   // Eq. SkewNormPrior: xi, 1 / omega,
    float sn_s[SPS_NPARAM], sn_c[SPS_NPARAM];      // s, log(2 / omega) - log(2 pi) / 2
    int band_kind[kMaxBands];
    int tab_off[kMaxBands], tab_n[kMaxBands];      // TABLE bands: offset and count in Grid::band_T
    int mdf_age;                                   // 1: MDF mean shifted per age bin (non-separable W)
    float mdf_off[kMaxAges];                       // the shift of age bin i
};

// Per-galaxy tables built by sps_set_galaxies (device, structure of arrays).
struct Galaxies {
    int64_t n;
    const float* z;          // [G]
    const float* lnT;        // [G] ln(t_obs / Gyr)
    const float* lT10;       // [G] log10(t_obs / yr)
    const float2* bins;      // [G][A] (centre, half-width) in ln(t/Gyr); Big-Bang bin: (ln t_hi, -1)
    const double* zp;        // [G][B] AB zero point: m = zp - 2.5 log10(c)
    const int2* support;     // [G][B] wavelength index range [lo, hi) of the redshifted band
    const float2* gauss;     // [G][B] (rest centre, (1+z)/s) of a Gaussian band
    const float* cssp;       // [G][B][K] per-galaxy c_SSP (approximate path) or nullptr
    const float4* dust_eff;  // [G][B] (k0, ln(l/lV), Drude, lambda_eff) at lambda_eff
    // redshift derivatives (the z column of sps_loglike_grad_z)
    const float* dtdz;       // [G] d t_obs / dz [Gyr]
    const float* dzp;        // [G][B] d zp / dz [mag]
    const float4* ddust;     // [G][B] d(k0, ln(l/lV), Drude) / dz at lambda_eff, unused
    const float* dcssp;      // [G][B][K] d c_SSP / dz (approximate path) or nullptr
};

// Per-wavelength constants of the rest grid (device).
struct Grid {
    const float* lam;        // [L] Angstrom
    const float4* lamc;      // [L] (q_n / lambda_n, k0, ln(lambda/lambda_V), Drude shape)
    const float2* lamq;      // [L] (lambda, q_n / lambda_n) in FP32
    const double* lam64;     // [L] Angstrom, FP64
    const float* ssp_t;      // [lam_pad][k_pad] SSP table transposed, FP32 (zero padded)
    const float* ssp;        // [k_pad][lam_pad] SSP table, FP32 (zero padded)
    const uint16_t* ssp_bf;  // [k_pad][lam_pad] SSP table, BF16 bits, row-scaled by 2^-e_i
    const uint16_t* ssp_t_bf;// [lam_pad][k_pad] transposed BF16 row-scaled
    const float* row_scale;  // [A] 2^e_i
    const float* col_scale;  // [k_pad] 2^e_i of column k = i Zn + j, 0 past K
    const float* band_T;     // tabulated transmission samples, all TABLE bands (FP32)
    const double* band_T64;  // the same in FP64 (per-galaxy set-up kernels)
};

// Metric-adaptation state of one HMC chain, kept in global memory (read at
// trajectory ends; chol every leapfrog step with the dense metric).
struct ChainMetric {
    float wmean[SPS_NPARAM], wm2[SPS_NPARAM];    // Welford moments of the window
    float chol[78];                              // dense inverse metric L L^T, packed lower
    float wcov[78];                              // window co-moments (dense)
};

// Tree state of one NUTS chain (hmc_team.cu), kept in global memory: the
// trajectory's two ends, the subtree's proposal, the merged trajectory's
// momentum sum and, per level k = 1..kNutsMaxDepth-1 of the subtree being
// built, the subtree's momentum prefix sum before its current aligned block
// of 2^k leaves and that block's first momentum (a block's momentum sum is
// the prefix sum at its last leaf minus the one before its first).
constexpr int kNutsMaxDepth = 10;
struct NutsChain {
    float xe[2][SPS_NPARAM], pe[2][SPS_NPARAM], ge[2][SPS_NPARAM];   // [0] backward end, [1] forward end
    float xq[SPS_NPARAM], gq[SPS_NPARAM];                            // subtree proposal
    float rho[SPS_NPARAM];                                           // momentum sum of the trajectory
    float sk[kNutsMaxDepth - 1][SPS_NPARAM], pk[kNutsMaxDepth - 1][SPS_NPARAM];
    double lpq;                                                      // log density of the subtree proposal
};

// State of one chain of the plain lock-step HMC (hmc_plain.cu).
struct PlainChain {
    float x[SPS_NPARAM], p[SPS_NPARAM], g[SPS_NPARAM], xs[SPS_NPARAM], gs[SPS_NPARAM];
    double lp, lps, h0, uacc;        // log posterior, energies, log of the accept uniform
    float mu, hbar, leb, acc, eps;   // dual averaging, accept sum, step size
    int L, l, it, mda, ndiv, active;
    long long nev;
};

// Records the message returned by sps_last_error_message() on this thread.
void set_last_error(const char* msg);
// Where an array argument lives: 1 in the memory of `device` (or managed
// memory), 0 in host memory, -1 in the memory of another device.
int pointer_location(const void* p, int device);

// Launchers (defined in the .cu files); all return cudaError_t of the launch.
cudaError_t launch_prepare_galaxies(const Consts& c, const Grid& grid, const double* lam64,
                                    const double* band_p0, const double* band_p1,
                                    const double* age_edges_yr, const float* z, int64_t n_gal,
                                    double h0, double om, float* lnT, float* lT10, float2* bins,
                                    double* zp, int2* support, float2* gauss, float4* dust_eff,
                                    float* dtdz, float* dzp, float4* ddust, cudaStream_t s);
// c_SSP (deriv = 0) or its redshift derivative d c_SSP / dz (deriv = 1)
cudaError_t launch_cssp(const Consts& c, const Grid& grid, const Galaxies& g,
                        const double* band_p0, const double* band_p1, float* cssp, cudaStream_t s,
                        int deriv = 0);

// Row evaluation of the approximate path (photometry / log-likelihood + gradient).
cudaError_t launch_approx_rows(const Consts& c, const Galaxies& g, const float* theta,
                               int theta_unbounded, const int32_t* gal_idx, int64_t n,
                               const float* mag_obs, const float* sigma, const uint32_t* mask,
                               float* mag_out, float* loglike_out, float* grad_out,
                               double* logp_out, int* nonfinite, cudaStream_t s);
// log L and the 13-column gradient (12 parameters and the redshift) of the
// approximate path, one row per warp; needs g.dcssp
cudaError_t launch_approx_rows_z(const Consts& c, const Galaxies& g, const float* theta,
                                 const int32_t* gal_idx, int64_t n, const float* mag_obs,
                                 const float* sigma, const uint32_t* mask, float* loglike_out,
                                 float* grad_out, int* nonfinite, cudaStream_t s);

// Exact path pieces.
cudaError_t launch_exact_weights(const Consts& c, const Grid& grid, const Galaxies& g,
                                 const float* theta, const int32_t* gal_idx, int64_t n,
                                 int bf16, float* W32, uint16_t* Wbf, cudaStream_t s,
                                 const int32_t* pos_of = nullptr,    // W row of each row (or itself)
                                 float* W32lo = nullptr,             // with W32lo: W32 = TF32 hi, W32lo = lo
                                 float* keep = nullptr);             // with keep: the row's weight arrays
                                                                     // (keep_stride floats per row)
cudaError_t launch_exact_fwd(const Consts& c, const Grid& grid, const Galaxies& g,
                             const float* theta, const int32_t* gal_idx, int64_t n, int bf16,
                             const float* W32, const uint16_t* Wbf, float* cJ, cudaStream_t s,
                             float* cJz = nullptr);   // with cJz: [r][b][2] sum_n wb' S (1, E)
cudaError_t launch_lambda_consts(const double* lam, int L, float4* out, float* lam32, float2* lamq,
                                 cudaStream_t s);
cudaError_t launch_exact_like(const Consts& c, const Galaxies& g, const float* theta,
                              const int32_t* gal_idx, int64_t n, const float* cJ, float* rowinfo,
                              const float* mag_obs, const float* sigma, const uint32_t* mask,
                              float* mag_out, float* loglike_out, float* gbar, int* nonfinite,
                              cudaStream_t s,
                              const float* cJz = nullptr,   // with cJz: rowz[r] = the explicit
                              float* rowz = nullptr,        // (fixed-weights) part of dlogL/dz
                              double* ll64_out = nullptr);  // log L in FP64 (the samplers' accept)
cudaError_t launch_exact_vgen(const Consts& c, const Grid& grid, const Galaxies& g,
                              const float* theta, const int32_t* gal_idx, int64_t n,
                              const float* gbar, float* V32, uint16_t* Vbf, cudaStream_t s,
                              float* V32lo = nullptr);   // with V32lo: V32 = TF32 hi, V32lo = lo
cudaError_t launch_exact_adj(const Consts& c, const Grid& grid, int64_t n, int bf16,
                             const float* V32, float* Wbar, cudaStream_t s);
cudaError_t launch_exact_grad(const Consts& c, const Galaxies& g, const float* theta,
                              const int32_t* gal_idx, int64_t n, const float* rowinfo,
                              const float* Wbar, float* grad_out, cudaStream_t s,
                              const float* rowz = nullptr,    // with rowz: 13 columns, z last
                              const float* keep = nullptr);   // weight arrays kept by the weights kernel
// Floats per row of the kept weight arrays: M (FP64, two floats), then
// m, dm/dtau, dm/dalpha, dm/dbeta, pi, w over the age bins and q over the
// metallicity bins; a multiple of 4 floats, so that every row's M is 8-byte
// aligned.
__host__ __device__ inline int64_t keep_stride(const Consts& c) { return (2 + 6 * (int64_t)c.n_age + c.n_met + 3) / 4 * 4; }

// Tensor-core (tcgen05) contractions; the tensor maps describe the operands:
// a[0], b[0] the A (rows) and B (table) operands, and for 3xTF32 (tf) a[1],
// b[1] their low parts.
struct TcMaps {
    CUtensorMap a[2], b[2];
};
size_t tc_fwd_smem(bool tf);
size_t tc_adj_smem(bool tf);
cudaError_t launch_fwd_tc(const TcMaps& tm, bool tf, const Consts& c, const Grid& grid, const Galaxies& g,
                          const float* theta, const int32_t* gal_idx, const int32_t* perm, int64_t n, float* cJ,
                          int* err, cudaStream_t s, float* cJz = nullptr);
cudaError_t launch_fwd_tc_z(const TcMaps& tm, bool tf, const Consts& c, const Grid& grid, const Galaxies& g,
                            const float* theta, const int32_t* gal_idx, const int32_t* perm, int64_t n,
                            float* cJ, int* err, cudaStream_t s, float* cJz);   // exact_tc_z.cu
cudaError_t launch_adj_tc(const TcMaps& tm, bool tf, const Consts& c, const Grid& grid, int64_t n, float* Wbar,
                          int* err, cudaStream_t s);
// Rows ordered by redshift (bucketed in log(1+z)): perm[pos] = row,
// pos_of[row] = pos; counts is scratch of zsort_buckets() ints.
int zsort_buckets();
cudaError_t launch_zsort(const Galaxies& g, const int32_t* gal_idx, int64_t n, int32_t* perm,
                         int32_t* pos_of, int32_t* counts, cudaStream_t s);

// Plain per-galaxy forward-mode path (comparison baseline).
size_t plain_scratch_bytes_per_row(const Consts& c);
cudaError_t launch_plain(const Consts& c, const Galaxies& g, const float* theta,
                         const int32_t* gal_idx, int64_t n, const float* mag_obs,
                         const float* sigma, const uint32_t* mask, float* ll_out, float* grad_out,
                         float* T, float* cd, cudaStream_t s, double* ll64_out = nullptr);

cudaError_t launch_weights_rows(const Consts& c, const Galaxies& g, const float* theta,
                                const int32_t* gal_idx, int64_t n, float* W_out,
                                double* mstar_out, cudaStream_t s);

cudaError_t launch_philox(const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out,
                          cudaStream_t s);

// HMC.
struct HmcParams {
    int chains_per_gal, n_warm, n_samp, L_min, L_max;
    float target_accept, eps0;
    uint64_t seed;
    int adapt_mass;         // 0 identity, 1 windowed diagonal, 2 windowed dense metric
    int sync_every;         // passes between the block barriers of the team kernel (>= 1)
    int max_depth;          // NUTS tree depth limit (1..kNutsMaxDepth)
    NutsChain* nuts;        // per-chain NUTS state; null runs HMC
    // team kernel: the launch takes work items [item0, item_end) of its own
    // grouping (item_end < 0: all of them)
    int64_t item0 = 0, item_end = -1;
};
// log L + gradient of independent rows through the team evaluation (n_met <= 12);
// see hmc_team.cu
cudaError_t launch_like_team(const Consts& c, const Galaxies& g, const float* theta, const int32_t* gal_idx,
                             int64_t n, const float* mag_obs, const float* sigma, const uint32_t* mask,
                             float* ll_out, float* grad_out, int* nonfinite, cudaStream_t s);
// approximate-path magnitudes of independent rows through the team layout,
// forward only (separable model, n_met <= 12); see hmc_team.cu
cudaError_t launch_phot_team(const Consts& c, const Galaxies& g, const float* theta, const int32_t* gal_idx,
                             int64_t n, float* mag_out, int* nonfinite, cudaStream_t s);
// rows: the age-dependent-MDF variant (one chain per warp, per-age q matrix); see hmc_team.cu
size_t hmc_team_smem_per_warp(int cpw, bool rows);
cudaError_t hmc_team_occupancy(int cpw, bool rows, bool nuts, int warps, int* blocks_per_sm);
cudaError_t launch_hmc_team(int cpw, bool rows, const Consts& c, const Galaxies& g, const HmcParams& hp,
                            const float* theta0, const float* mag_obs, const float* sigma,
                            const uint32_t* mask, const int32_t* gal_order, float* samples,
                            float* acc, float* eps_out, int32_t* div, int64_t* nevals,
                            int32_t* status, int* queue, ChainMetric* metric, int blocks, int warps,
                            cudaStream_t s);
cudaError_t plain_hmc_init(const Consts& c, int64_t n, int C, const float* x0, float eps0, PlainChain* st,
                           float* theta, int32_t* gal_idx, cudaStream_t s);
cudaError_t plain_hmc_absorb(const Consts& c, int64_t n, PlainChain* st, const double* ll, const float* gth,
                             cudaStream_t s);
cudaError_t plain_hmc_start(const Consts& c, const HmcParams& hp, int64_t n, PlainChain* st, float* theta,
                            cudaStream_t s);
cudaError_t plain_hmc_step(const Consts& c, const HmcParams& hp, int64_t n, PlainChain* st, const double* ll,
                           const float* gth, float* theta, float* samples, cudaStream_t s);
// exact-path sampler: trajectory-asynchronous rounds (hmc_plain.cu)
cudaError_t async_hmc_step(const Consts& c, const HmcParams& hp, int64_t n, PlainChain* st, const double* ll,
                           const float* gth, float* theta, float* samples, cudaStream_t s);
cudaError_t async_hmc_rounds(const HmcParams& hp, int64_t n, int* max_out, cudaStream_t s);
cudaError_t plain_hmc_stats(const HmcParams& hp, int64_t n, const PlainChain* st, float* acc, float* eps_out,
                            int32_t* div_out, int64_t* nev_out, int32_t* status_out, cudaStream_t s);
cudaError_t launch_leapfrog(const Consts& c, const Galaxies& g, const float* x0,
                            const float* p0, const float* eps, const int32_t* L,
                            const int32_t* gal_idx, int64_t n, const float* mag_obs,
                            const float* sigma, const uint32_t* mask, float* x_out,
                            float* p_out, double* logp_out, cudaStream_t s);

}  // namespace sps
