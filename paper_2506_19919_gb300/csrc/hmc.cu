// Deterministic leapfrog trajectories through the per-row evaluator (test
// hook of the HMC integrator of Sec. 4 / App. D.2).  The batched sampler
// itself is in hmc_team.cu.
//
// Per iteration: p = z / sqrt(minv), z ~ N(0, I), L ~ U{L_min..L_max}; L
// leapfrog steps (half kick, drift x += eps minv p, gradient, half kick);
// Metropolis accept on the FP64 energy difference.  Warm-up: the step size
// follows the dual averaging of Hoffman & Gelman (2014, Sec. 3.2.1); the
// diagonal inverse metric minv is adapted in the windowed scheme of the Stan
// reference manual (75-iteration initial buffer, slow windows of 25, 50, 100,
// ... iterations, 50-iteration terminal buffer; regularised Welford variance
// n/(n+5) var + 1e-3 * 5/(n+5) of each window's positions, after which dual
// averaging restarts at mu = log(10 eps)).  Sampling uses the averaged step
// size.  Draws: Philox-4x32-10, counter (iteration, block, chain, 0),
// key = seed; Box-Muller in FP64.
#include "philox.cuh"
#include "sps_eval.cuh"

namespace sps {

namespace {

struct ChainCtx {
    const Consts* c;
    WarpWork* ww;
    const float2* bins;
    float lnT, lT10;
    int nb;
};

// log posterior in unbounded space and its gradient; x, g warp-uniform.
__device__ __forceinline__ double logp_grad(const ChainCtx& cc, const float* x, float* g) {
    RowParams p;
    load_params(*cc.c, x, true, p);
    float gr[SPS_NPARAM];
    double ll = eval_row(*cc.c, *cc.ww, cc.bins, cc.lnT, cc.lT10, p, cc.nb, true, true, gr);
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) g[k] = gr[k] * p.dth[k] + p.dlp[k];
    return ll + p.logprior;
}

// Deterministic leapfrog (test hook): one warp per row.
__global__ void __launch_bounds__(32 * kWarpsApprox)
k_leapfrog(const __grid_constant__ Consts c, const Galaxies g, const float* __restrict__ x0,
           const float* __restrict__ p0, const float* __restrict__ epsv, const int32_t* __restrict__ Lv,
           const int32_t* __restrict__ gal_idx, int64_t n, const float* __restrict__ mag_obs,
           const float* __restrict__ sigma, const uint32_t* __restrict__ mask,
           float* __restrict__ x_out, float* __restrict__ p_out, double* __restrict__ lp_out) {
    __shared__ WarpWork work[kWarpsApprox];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int B = c.n_band;
    const uint32_t all = (B >= 32) ? 0xffffffffu : ((1u << B) - 1u);
    for (int64_t row = (int64_t)blockIdx.x * kWarpsApprox + warp; row < n;
         row += (int64_t)gridDim.x * kWarpsApprox) {
        const int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
        if (gi < 0 || gi >= g.n) continue;
        WarpWork& ww = work[warp];
        const uint32_t bits = mask[gi] & all;
        const int nb = fill_slots(c, g, ww.d, gi, bits, mag_obs, sigma, g.cssp + (size_t)gi * B * c.K, false);
        ChainCtx cc{&c, &ww, g.bins + (size_t)gi * c.n_age, g.lnT[gi], g.lT10[gi], nb};
        float x[SPS_NPARAM], p[SPS_NPARAM], gr[SPS_NPARAM];
#pragma unroll
        for (int k = 0; k < SPS_NPARAM; ++k) {
            x[k] = x0[row * SPS_NPARAM + k];
            p[k] = p0[row * SPS_NPARAM + k];
        }
        const float eps = epsv[row];
        double lp = logp_grad(cc, x, gr);
        for (int l = 0; l < Lv[row]; ++l) {
#pragma unroll
            for (int k = 0; k < SPS_NPARAM; ++k) {
                p[k] = fmaf(0.5f * eps, gr[k], p[k]);
                x[k] = fmaf(eps, p[k], x[k]);
            }
            lp = logp_grad(cc, x, gr);
#pragma unroll
            for (int k = 0; k < SPS_NPARAM; ++k) p[k] = fmaf(0.5f * eps, gr[k], p[k]);
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < SPS_NPARAM; ++k) {
                x_out[row * SPS_NPARAM + k] = x[k];
                p_out[row * SPS_NPARAM + k] = p[k];
            }
            lp_out[row] = lp;
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_leapfrog(const Consts& c, const Galaxies& g, const float* x0, const float* p0,
                            const float* eps, const int32_t* L, const int32_t* gal_idx, int64_t n,
                            const float* mag_obs, const float* sigma, const uint32_t* mask,
                            float* x_out, float* p_out, double* logp_out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t b = (n + kWarpsApprox - 1) / kWarpsApprox;
    if (b > 152LL * 64) b = 152LL * 64;
    k_leapfrog<<<(unsigned)b, 32 * kWarpsApprox, 0, s>>>(c, g, x0, p0, eps, L, gal_idx, n, mag_obs,
                                                         sigma, mask, x_out, p_out, logp_out);
    return cudaGetLastError();
}

}  // namespace sps
