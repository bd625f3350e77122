// Plain batched HMC: the comparison baseline for the fused persistent sampler
// (Sec. 4, App. D.2), run as a straightforward GPU port of the paper's
// vectorised sampler would run it.
//
// Every chain advances in lock step, one leapfrog step per round of kernel
// launches: all chains start their trajectory together, and every round
// evaluates the gradient of every chain with the unfused forward-mode path
// (plain.cu) whether or not the chain's trajectory has already ended, up to
// L_max rounds per iteration (a vectorised loop over chains runs until its
// longest member finishes).  The sampler itself is the fused kernel's, step for
// step: identity metric, Philox-4x32-10 draws with counter (iteration, block,
// chain, 0), Box-Muller momenta, L = L_min + (w n) >> 32, leapfrog with half
// kicks around each drift, accept on the FP64 energy difference, dual-averaged
// step size in the warm-up and its average in the sampling phase.  One thread
// per chain.
#include <math.h>

#include "philox.cuh"
#include "sps_device.cuh"

namespace sps {

namespace {

// theta = F_B(x) for the next gradient evaluation.
__device__ __forceinline__ void write_theta(const Consts& c, const PlainChain& s, float* __restrict__ th) {
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) th[k] = bound_theta(c, k, s.x[k]);
}

// log posterior and its gradient in unbounded space from the physical-space
// log-likelihood and gradient at s.x.
__device__ __forceinline__ void absorb(const Consts& c, PlainChain& s, double ll, const float* __restrict__ gth) {
    double lpri = 0.0;
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) {
        float t, d, l, q;
        bound_prior(c, k, s.x[k], t, d, l, q);
        lpri += (double)l;
        s.g[k] = gth[k] * d + q;
    }
    s.lp = ll + lpri;
}

__global__ void k_plain_init(const __grid_constant__ Consts c, int64_t n, int C, const float* __restrict__ x0,
                             float eps0, PlainChain* __restrict__ st, float* __restrict__ theta,
                             int32_t* __restrict__ gal_idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PlainChain s;
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) s.x[k] = x0[i * SPS_NPARAM + k];
    s.eps = eps0;
    s.mu = logf(10.0f * eps0);
    s.hbar = s.leb = s.acc = 0.0f;
    s.it = s.mda = s.ndiv = s.l = s.L = 0;
    s.active = 0;
    s.nev = 1;
    st[i] = s;
    write_theta(c, s, theta + i * SPS_NPARAM);
    gal_idx[i] = (int32_t)(i / C);
}

__global__ void k_plain_absorb(const __grid_constant__ Consts c, int64_t n, PlainChain* __restrict__ st,
                               const double* __restrict__ ll, const float* __restrict__ gth) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PlainChain s = st[i];
    absorb(c, s, ll[i], gth + i * SPS_NPARAM);
    st[i] = s;
}

// Start of iteration s.it of chain i: momentum, start state, half kick, drift.
// Returns false (and leaves the chain inactive) once every iteration is done.
__device__ __forceinline__ bool begin_iteration(const HmcParams& hp, int64_t i, PlainChain& s) {
    if (s.it >= hp.n_warm + hp.n_samp) {
        s.active = 0;
        return false;
    }
    const uint32_t k0 = (uint32_t)(hp.seed & 0xffffffffu), k1 = (uint32_t)(hp.seed >> 32);
    uint32_t w[16];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)s.it, (uint32_t)b, (uint32_t)i, 0u), k0, k1);
        w[4 * b] = r.x;
        w[4 * b + 1] = r.y;
        w[4 * b + 2] = r.z;
        w[4 * b + 3] = r.w;
    }
    float kin = 0.0f;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        const float rr = sqrtf(-2.0f * logf(u01_f(w[2 * m])));
        float sn, cs;
        sincospif(2.0f * u01_f(w[2 * m + 1]), &sn, &cs);
        s.p[2 * m] = rr * cs;
        s.p[2 * m + 1] = rr * sn;
    }
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) {
        kin = fmaf(s.p[k], s.p[k], kin);
        s.xs[k] = s.x[k];
        s.gs[k] = s.g[k];
    }
    s.uacc = (double)logf(u01_f(w[12]));
    s.L = hp.L_min + (int)(((uint64_t)w[13] * (uint64_t)(hp.L_max - hp.L_min + 1)) >> 32);
    s.l = 0;
    s.lps = s.lp;
    s.h0 = -s.lp + 0.5 * (double)kin;
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) {
        s.p[k] = fmaf(0.5f * s.eps, s.g[k], s.p[k]);
        s.x[k] = fmaf(s.eps, s.p[k], s.x[k]);
    }
    s.active = 1;
    return true;
}

__global__ void k_plain_start(const __grid_constant__ Consts c, const HmcParams hp, int64_t n,
                              PlainChain* __restrict__ st, float* __restrict__ theta) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PlainChain s = st[i];
    const bool on = begin_iteration(hp, i, s);
    st[i] = s;
    if (on) write_theta(c, s, theta + i * SPS_NPARAM);
}

// End of chain i's trajectory at s.x (after its last half kick): accept or
// reject on the FP64 energy difference, step-size adaptation in the warm-up,
// the sample in the sampling phase; the chain is then inactive.
__device__ __forceinline__ void end_trajectory(const Consts& c, const HmcParams& hp, int64_t i, PlainChain& s,
                                               float* __restrict__ samples) {
    float kin = 0.0f;
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) kin = fmaf(s.p[k], s.p[k], kin);
    const double dH = (-s.lp + 0.5 * (double)kin) - s.h0;
    const bool fin = isfinite(dH);
    const float a = fin ? fminf(1.0f, __expf(-(float)dH)) : 0.0f;
    const bool take = fin && s.uacc < -dH;
    if (!take) {
#pragma unroll
        for (int k = 0; k < SPS_NPARAM; ++k) {
            s.x[k] = s.xs[k];
            s.g[k] = s.gs[k];
        }
        s.lp = s.lps;
    }
    if (!fin || dH > 1000.0) s.ndiv += 1;
    const int it = s.it;
    if (it < hp.n_warm) {
        const float m = (float)(s.mda + 1);
        const float im = __frcp_rn(m + 10.0f);
        const float hbar = (1.0f - im) * s.hbar + (hp.target_accept - a) * im;
        const float log_eps = s.mu - sqrtf(m) * 20.0f * hbar;
        const float wgt = exp2f(-0.75f * log2f(m));
        const float leb = wgt * log_eps + (1.0f - wgt) * s.leb;
        s.eps = expf(it < hp.n_warm - 1 ? log_eps : leb);
        s.mda += 1;
        s.hbar = hbar;
        s.leb = leb;
    } else {
        s.acc += a;
        if (samples) {
            float* o = samples + ((size_t)i * hp.n_samp + (it - hp.n_warm)) * SPS_NPARAM;
#pragma unroll
            for (int k = 0; k < SPS_NPARAM; ++k)
                o[k] = bound_theta(c, k, s.x[k]);
        }
    }
    s.it = it + 1;
    s.active = 0;
}

// One leapfrog round after the gradient evaluation at every chain's x.
__global__ void k_plain_step(const __grid_constant__ Consts c, const HmcParams hp, int64_t n,
                             PlainChain* __restrict__ st, const double* __restrict__ ll,
                             const float* __restrict__ gth, float* __restrict__ theta,
                             float* __restrict__ samples) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PlainChain s = st[i];
    s.nev += 1;                                   // every round evaluates every chain
    if (!s.active) {
        st[i] = s;
        return;
    }
    absorb(c, s, ll[i], gth + i * SPS_NPARAM);
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) s.p[k] = fmaf(0.5f * s.eps, s.g[k], s.p[k]);
    if (s.l + 1 < s.L) {
#pragma unroll
        for (int k = 0; k < SPS_NPARAM; ++k) {
            s.p[k] = fmaf(0.5f * s.eps, s.g[k], s.p[k]);
            s.x[k] = fmaf(s.eps, s.p[k], s.x[k]);
        }
        s.l += 1;
        st[i] = s;
        write_theta(c, s, theta + i * SPS_NPARAM);
        return;
    }
    end_trajectory(c, hp, i, s, samples);
    st[i] = s;
}

// Trajectory-asynchronous round of the exact-path sampler: after the
// gradient evaluation at every chain's x, one leapfrog step of every active
// chain; a chain whose trajectory ends starts its next iteration at once
// (same draws and sampler as above), so every round's evaluations are used
// until the chain has run all its iterations.
__global__ void k_async_step(const __grid_constant__ Consts c, const HmcParams hp, int64_t n,
                             PlainChain* __restrict__ st, const double* __restrict__ ll,
                             const float* __restrict__ gth, float* __restrict__ theta,
                             float* __restrict__ samples) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PlainChain s = st[i];
    if (!s.active) return;
    s.nev += 1;
    absorb(c, s, ll[i], gth + i * SPS_NPARAM);
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) s.p[k] = fmaf(0.5f * s.eps, s.g[k], s.p[k]);
    if (s.l + 1 < s.L) {
#pragma unroll
        for (int k = 0; k < SPS_NPARAM; ++k) {
            s.p[k] = fmaf(0.5f * s.eps, s.g[k], s.p[k]);
            s.x[k] = fmaf(s.eps, s.p[k], s.x[k]);
        }
        s.l += 1;
        st[i] = s;
        write_theta(c, s, theta + i * SPS_NPARAM);
        return;
    }
    end_trajectory(c, hp, i, s, samples);
    if (begin_iteration(hp, i, s)) write_theta(c, s, theta + i * SPS_NPARAM);
    st[i] = s;
}

// Rounds the asynchronous sampler needs: the largest, over chains, of the
// chain's leapfrog steps over all its iterations, sum_it L(it), from the same
// Philox words that draw L.
__global__ void k_traj_rounds(const HmcParams hp, int64_t n, int* __restrict__ max_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k0 = (uint32_t)(hp.seed & 0xffffffffu), k1 = (uint32_t)(hp.seed >> 32);
    const uint64_t span = (uint64_t)(hp.L_max - hp.L_min + 1);
    long long tot = 0;
    for (int it = 0; it < hp.n_warm + hp.n_samp; ++it) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)it, 3u, (uint32_t)i, 0u), k0, k1);
        tot += hp.L_min + (int)(((uint64_t)r.y * span) >> 32);
    }
    atomicMax(max_out, (int)min(tot, (long long)0x7fffffff));
}

__global__ void k_plain_stats(const HmcParams hp, int64_t n, const PlainChain* __restrict__ st, float* acc,
                              float* eps_out, int32_t* div_out, int64_t* nev_out, int32_t* status_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const PlainChain& s = st[i];
    if (acc) acc[i] = s.acc / (float)max(hp.n_samp, 1);
    if (eps_out) eps_out[i] = s.eps;
    if (div_out) div_out[i] = s.ndiv;
    if (nev_out) nev_out[i] = s.nev;
    if (status_out) status_out[i] = 0;
}

inline unsigned grid_for(int64_t n) { return (unsigned)((n + 127) / 128); }

}  // namespace

cudaError_t plain_hmc_init(const Consts& c, int64_t n, int C, const float* x0, float eps0, PlainChain* st,
                           float* theta, int32_t* gal_idx, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_plain_init<<<grid_for(n), 128, 0, s>>>(c, n, C, x0, eps0, st, theta, gal_idx);
    return cudaGetLastError();
}

cudaError_t plain_hmc_absorb(const Consts& c, int64_t n, PlainChain* st, const double* ll, const float* gth,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_plain_absorb<<<grid_for(n), 128, 0, s>>>(c, n, st, ll, gth);
    return cudaGetLastError();
}

cudaError_t plain_hmc_start(const Consts& c, const HmcParams& hp, int64_t n, PlainChain* st, float* theta,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_plain_start<<<grid_for(n), 128, 0, s>>>(c, hp, n, st, theta);
    return cudaGetLastError();
}

cudaError_t plain_hmc_step(const Consts& c, const HmcParams& hp, int64_t n, PlainChain* st, const double* ll,
                           const float* gth, float* theta, float* samples, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_plain_step<<<grid_for(n), 128, 0, s>>>(c, hp, n, st, ll, gth, theta, samples);
    return cudaGetLastError();
}

cudaError_t async_hmc_step(const Consts& c, const HmcParams& hp, int64_t n, PlainChain* st, const double* ll,
                           const float* gth, float* theta, float* samples, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_async_step<<<grid_for(n), 128, 0, s>>>(c, hp, n, st, ll, gth, theta, samples);
    return cudaGetLastError();
}

cudaError_t async_hmc_rounds(const HmcParams& hp, int64_t n, int* max_out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(max_out, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_traj_rounds<<<grid_for(n), 128, 0, s>>>(hp, n, max_out);
    return cudaGetLastError();
}

cudaError_t plain_hmc_stats(const HmcParams& hp, int64_t n, const PlainChain* st, float* acc, float* eps_out,
                            int32_t* div_out, int64_t* nev_out, int32_t* status_out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_plain_stats<<<grid_for(n), 128, 0, s>>>(hp, n, st, acc, eps_out, div_out, nev_out, status_out);
    return cudaGetLastError();
}

}  // namespace sps
