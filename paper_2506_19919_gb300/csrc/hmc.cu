// Batched HMC on the approximate path in one persistent launch (Sec. 4,
// App. D.2).  Blocks pull galaxies from a global work queue (atomic counter,
// no waiting); a block stages the galaxy's observed-band c_SSP rows in shared
// memory and runs each chain of that galaxy on one warp.  Chains are
// trajectory-asynchronous: each warp advances its own chain through its own
// trajectory lengths; uneven band counts and trajectory lengths are balanced
// by the queue.
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
    for (int k = 0; k < SPS_NPARAM; ++k) {
        float sg = sigmoidf_(x[k]);
        g[k] = gr[k] * p.dth[k] + (1.0f - 2.0f * sg);
    }
    return ll + p.logprior;
}

// Draws of one iteration for one chain: momenta (FP64 Box-Muller -> float),
// accept uniform and trajectory length.  Warp-uniform results.
__device__ __forceinline__ void draws(uint64_t seed, uint32_t chain, uint32_t it, int L_min,
                                      int L_max, float* p, double& u_acc, int& L) {
    const int lane = lane_id();
    uint4 w = make_uint4(0, 0, 0, 0);
    if (lane < 4)
        w = philox4x32_10(make_uint4(it, (uint32_t)lane, chain, 0u), (uint32_t)(seed & 0xffffffffu),
                          (uint32_t)(seed >> 32));
    // pair m uses uniforms u[2m], u[2m+1]: word (2m) and (2m+1) of blocks 0-2
    double z0 = 0.0, z1 = 0.0;
    uint32_t wa = 0, wb = 0;
    {
        // every lane fetches the two words of pair (lane % 6)
        const int m = lane % 6;
        const int ia = 2 * m, ib = 2 * m + 1;
        uint32_t ax = __shfl_sync(kFull, w.x, ia >> 2), ay = __shfl_sync(kFull, w.y, ia >> 2);
        uint32_t az = __shfl_sync(kFull, w.z, ia >> 2), aw = __shfl_sync(kFull, w.w, ia >> 2);
        uint32_t bx = __shfl_sync(kFull, w.x, ib >> 2), by = __shfl_sync(kFull, w.y, ib >> 2);
        uint32_t bz = __shfl_sync(kFull, w.z, ib >> 2), bw = __shfl_sync(kFull, w.w, ib >> 2);
        const int sa = ia & 3, sb = ib & 3;
        wa = sa == 0 ? ax : sa == 1 ? ay : sa == 2 ? az : aw;
        wb = sb == 0 ? bx : sb == 1 ? by : sb == 2 ? bz : bw;
        double u1 = u01_d(wa), u2 = u01_d(wb);
        double r = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        z0 = r * cs;
        z1 = r * sn;
    }
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        p[2 * m] = (float)__shfl_sync(kFull, z0, m);
        p[2 * m + 1] = (float)__shfl_sync(kFull, z1, m);
    }
    uint32_t w30 = __shfl_sync(kFull, w.x, 3), w31 = __shfl_sync(kFull, w.y, 3);
    u_acc = u01_d(w30);
    const uint64_t span = (uint64_t)(L_max - L_min + 1);
    L = L_min + (int)(((uint64_t)w31 * span) >> 32);
}

// Windowed metric-adaptation schedule for n_warm warm-up iterations.
struct Windows {
    int start, end, width, stop;
    __device__ void init(int n_warm) {
        int init_b, term_b;
        if (n_warm >= 150) {
            init_b = 75;
            term_b = 50;
            width = 25;
        } else {
            init_b = (int)(0.15 * n_warm);
            term_b = (int)(0.1 * n_warm);
            width = n_warm - init_b - term_b;
        }
        stop = n_warm - term_b;
        start = init_b;
        set_end();
    }
    __device__ void set_end() {
        end = start + width;
        if (end + 2 * width > stop) end = stop;
        if (width <= 0 || start >= stop) start = end = 0x7fffffff;
    }
    __device__ void next() {
        start = end;
        width *= 2;
        set_end();
    }
};

__device__ void run_chain(const ChainCtx& cc, const HmcParams hp, uint32_t chain,
                          const float* __restrict__ x0, float* __restrict__ samples,
                          float* acc_out, float* eps_out, int32_t* div_out, int64_t* nev_out,
                          int32_t* status_out) {
    const Consts& c = *cc.c;
    const int lane = lane_id();
    float x[SPS_NPARAM], g[SPS_NPARAM], minv[SPS_NPARAM];
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) {
        x[k] = x0[(size_t)chain * SPS_NPARAM + k];
        minv[k] = 1.0f;
    }
    double lp = logp_grad(cc, x, g);
    float eps = hp.eps0;
    double mu = log(10.0 * (double)hp.eps0);
    double hbar = 0.0, log_eps_bar = 0.0;
    int m_da = 0;
    Windows win;
    win.init(hp.adapt_mass ? hp.n_warm : 0);
    int wn = 0;
    double wmean = 0.0, wm2 = 0.0;          // lane k < 12: Welford state of parameter k
    double acc_sum = 0.0;
    int ndiv = 0;
    long long nev = 1;
    const int n_it = hp.n_warm + hp.n_samp;
    for (int it = 0; it < n_it; ++it) {
        float p[SPS_NPARAM];
        double u_acc;
        int L;
        draws(hp.seed, chain, (uint32_t)it, hp.L_min, hp.L_max, p, u_acc, L);
        float x1[SPS_NPARAM], p1[SPS_NPARAM], g1[SPS_NPARAM];
#pragma unroll
        for (int k = 0; k < SPS_NPARAM; ++k) {
            p[k] = p[k] * rsqrtf(minv[k]);
            x1[k] = x[k];
            p1[k] = p[k];
            g1[k] = g[k];
        }
        double lp1 = lp;
        for (int l = 0; l < L; ++l) {
#pragma unroll
            for (int k = 0; k < SPS_NPARAM; ++k) {
                p1[k] = fmaf(0.5f * eps, g1[k], p1[k]);
                x1[k] = fmaf(eps * minv[k], p1[k], x1[k]);
            }
            lp1 = logp_grad(cc, x1, g1);
#pragma unroll
            for (int k = 0; k < SPS_NPARAM; ++k) p1[k] = fmaf(0.5f * eps, g1[k], p1[k]);
        }
        nev += L;
        double k0 = 0.0, k1 = 0.0;
#pragma unroll
        for (int k = 0; k < SPS_NPARAM; ++k) {
            k0 += (double)minv[k] * (double)p[k] * (double)p[k];
            k1 += (double)minv[k] * (double)p1[k] * (double)p1[k];
        }
        const double dH = (-lp1 + 0.5 * k1) - (-lp + 0.5 * k0);
        const bool fin = isfinite(dH);
        const double a = fin ? fmin(1.0, exp(-dH)) : 0.0;
        if (!fin || dH > 1000.0) ++ndiv;
        if (fin && log(u_acc) < -dH) {
#pragma unroll
            for (int k = 0; k < SPS_NPARAM; ++k) {
                x[k] = x1[k];
                g[k] = g1[k];
            }
            lp = lp1;
        }
        float xs = x[0];                      // this lane's parameter (lanes < 12)
#pragma unroll
        for (int k = 1; k < SPS_NPARAM; ++k)
            if (lane == k) xs = x[k];
        if (it < hp.n_warm) {
            const double m = (double)(++m_da);
            hbar = (1.0 - 1.0 / (m + 10.0)) * hbar + ((double)hp.target_accept - a) / (m + 10.0);
            const double log_eps = mu - sqrt(m) / 0.05 * hbar;
            const double wgt = pow(m, -0.75);
            log_eps_bar = wgt * log_eps + (1.0 - wgt) * log_eps_bar;
            eps = (float)exp(it < hp.n_warm - 1 ? log_eps : log_eps_bar);
            if (it >= win.start && it < win.end) {
                ++wn;
                const double d = (double)xs - wmean;
                wmean += d / (double)wn;
                wm2 += d * ((double)xs - wmean);
                if (it == win.end - 1) {
                    const double var = wm2 / ((double)wn - 1.0);
                    const float mk = (float)(((double)wn / (wn + 5.0)) * var + 1e-3 * (5.0 / (wn + 5.0)));
#pragma unroll
                    for (int k = 0; k < SPS_NPARAM; ++k) minv[k] = __shfl_sync(kFull, mk, k);
                    wn = 0;
                    wmean = wm2 = 0.0;
                    mu = log(10.0 * (double)eps);
                    hbar = 0.0;
                    log_eps_bar = 0.0;
                    m_da = 0;
                    win.next();
                }
            }
        } else {
            acc_sum += a;
            if (samples && lane < SPS_NPARAM)
                samples[((size_t)chain * hp.n_samp + (it - hp.n_warm)) * SPS_NPARAM + lane] =
                    c.prior_lo[lane] + c.prior_span[lane] * sigmoidf_(xs);
        }
    }
    if (lane == 0) {
        if (acc_out) acc_out[chain] = (float)(acc_sum / (double)max(hp.n_samp, 1));
        if (eps_out) eps_out[chain] = eps;
        if (div_out) div_out[chain] = ndiv;
        if (nev_out) nev_out[chain] = nev;
        if (status_out) status_out[chain] = 0;
    }
}

__global__ void k_hmc_approx(const __grid_constant__ Consts c, const Galaxies g, const HmcParams hp,
                             const float* __restrict__ theta0, const float* __restrict__ mag_obs,
                             const float* __restrict__ sigma, const uint32_t* __restrict__ mask,
                             const int32_t* __restrict__ gal_order, float* __restrict__ samples,
                             float* acc, float* eps_out, int32_t* div, int64_t* nev, int32_t* status,
                             int* queue) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nwarps = blockDim.x >> 5;
    WarpWork* work = reinterpret_cast<WarpWork*>(smem);
    float* table = reinterpret_cast<float*>(smem + sizeof(WarpWork) * nwarps);
    __shared__ int s_q;
    __shared__ int s_band[kMaxBands];
    const int warp = threadIdx.x >> 5;
    const int B = c.n_band, K = c.K;
    const uint32_t all = (B >= 32) ? 0xffffffffu : ((1u << B) - 1u);
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(queue, 1);
        __syncthreads();
        const int q = s_q;
        if (q >= g.n) break;
        const int64_t gi = gal_order ? (int64_t)gal_order[q] : (int64_t)q;
        const uint32_t bits = mask[gi] & all;
        const int nb = __popc(bits);
        if (threadIdx.x < B && ((bits >> threadIdx.x) & 1u))
            s_band[__popc(bits & ((1u << threadIdx.x) - 1u))] = threadIdx.x;
        __syncthreads();
        const float* src = g.cssp + (size_t)gi * B * K;
        for (int e = threadIdx.x; e < nb * K; e += blockDim.x) {
            int sl = e / K, k = e - sl * K;
            table[e] = src[(size_t)s_band[sl] * K + k];
        }
        __syncthreads();
        WarpWork& ww = work[warp];
        fill_slots(c, g, ww.d, gi, bits, mag_obs, sigma, table, true);
        ChainCtx cc{&c, &ww, g.bins + (size_t)gi * c.n_age, g.lnT[gi], g.lT10[gi], nb};
        for (int ch = warp; ch < hp.chains_per_gal; ch += nwarps) {
            const uint32_t chain = (uint32_t)(gi * hp.chains_per_gal + ch);
            run_chain(cc, hp, chain, theta0, samples, acc, eps_out, div, nev, status);
        }
        __syncthreads();
    }
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

size_t hmc_warp_smem_bytes() { return sizeof(WarpWork); }

cudaError_t hmc_set_smem(size_t bytes) {
    return cudaFuncSetAttribute(k_hmc_approx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t hmc_occupancy(int warps, size_t smem, int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_hmc_approx, warps * 32, smem);
}

cudaError_t launch_hmc_approx(const Consts& c, const Galaxies& g, const HmcParams& hp,
                              const float* theta0, const float* mag_obs, const float* sigma,
                              const uint32_t* mask, const int32_t* gal_order, float* samples,
                              float* acc, float* eps_out, int32_t* div, int64_t* nevals,
                              int32_t* status, int* queue, int* err, int grid_blocks,
                              int warps_per_block, size_t smem_cssp_bytes, cudaStream_t s) {
    (void)err;
    const size_t smem = sizeof(WarpWork) * warps_per_block + smem_cssp_bytes;
    k_hmc_approx<<<grid_blocks, warps_per_block * 32, smem, s>>>(
        c, g, hp, theta0, mag_obs, sigma, mask, gal_order, samples, acc, eps_out, div, nevals,
        status, queue);
    return cudaGetLastError();
}

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
