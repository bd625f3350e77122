// Approximate photometry, log-likelihood and adjoint gradient, one warp per
// row (Eq. photo_integral_approx, App. D.1), plus the SSP-weights and Philox
// test hooks.
#include "sps_eval.cuh"
#include "philox.cuh"

namespace sps {

namespace {

__global__ void __launch_bounds__(32 * kWarpsApprox)
k_approx_rows(const __grid_constant__ Consts c, const Galaxies g, const float* __restrict__ theta,
              int unbounded, const int32_t* __restrict__ gal_idx, int64_t n,
              const float* __restrict__ mag_obs, const float* __restrict__ sigma,
              const uint32_t* __restrict__ mask, float* __restrict__ mag_out,
              float* __restrict__ ll_out, float* __restrict__ grad_out,
              double* __restrict__ logp_out, int* __restrict__ nonfinite) {
    __shared__ WarpWork work[kWarpsApprox];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    WarpWork& ww = work[warp];
    const bool like = (ll_out != nullptr) || (logp_out != nullptr);
    const bool grad = grad_out != nullptr;
    const int B = c.n_band;
    const uint32_t all = (B >= 32) ? 0xffffffffu : ((1u << B) - 1u);
    for (int64_t row = (int64_t)blockIdx.x * kWarpsApprox + warp; row < n;
         row += (int64_t)gridDim.x * kWarpsApprox) {
        const int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
        RowParams p;
        load_params(c, theta + row * SPS_NPARAM, unbounded != 0, p);
        if (gi < 0 || gi >= g.n) p.finite = false;      // out-of-range galaxy: NaN row
        if (!p.finite) {
            if (lane == 0) atomicOr(nonfinite, 1);
            if (mag_out && lane < B) mag_out[row * B + lane] = __int_as_float(0x7fc00000);
            if (ll_out && lane == 0) ll_out[row] = __int_as_float(0x7fc00000);
            if (logp_out && lane == 0) logp_out[row] = __longlong_as_double(0x7ff8000000000000ll);
            if (grad && lane < SPS_NPARAM) grad_out[row * SPS_NPARAM + lane] = __int_as_float(0x7fc00000);
            continue;
        }
        const uint32_t bits = like ? (mask[gi] & all) : all;
        const int nb = fill_slots(c, g, ww.d, gi, bits, like ? mag_obs : nullptr, sigma,
                                  g.cssp + (size_t)gi * B * c.K, false);
        float gr[SPS_NPARAM];
        double ll = eval_row(c, ww, g.bins + (size_t)gi * c.n_age, g.lnT[gi], g.lT10[gi], p, nb,
                             like, grad, gr);
        if (mag_out && lane < nb) mag_out[row * B + ww.d.band[lane]] = (float)ww.d.mag[lane];
        if (ll_out && lane == 0) ll_out[row] = (float)ll;
        if (logp_out && lane == 0) logp_out[row] = ll + p.logprior;
        if (grad && lane == 0) {
            bool bad = !isfinite(ll);
#pragma unroll
            for (int k = 0; k < SPS_NPARAM; ++k) {
                float v = gr[k];
                if (unbounded) v = v * p.dth[k] + p.dlp[k];
                bad = bad || !isfinite(v);
                grad_out[row * SPS_NPARAM + k] = v;
            }
            if (bad) atomicOr(nonfinite, 1);
        } else if (lane == 0 && !isfinite(ll) && like) {
            atomicOr(nonfinite, 1);
        }
        __syncwarp();
    }
}

// log L and d log L / d(theta, z) of the approximate path, one warp per row:
// grad_out[row][13], the last column the derivative in the galaxy's redshift.
__global__ void __launch_bounds__(32 * kWarpsApprox)
k_approx_rows_z(const __grid_constant__ Consts c, const Galaxies g, const float* __restrict__ theta,
                const int32_t* __restrict__ gal_idx, int64_t n, const float* __restrict__ mag_obs,
                const float* __restrict__ sigma, const uint32_t* __restrict__ mask,
                float* __restrict__ ll_out, float* __restrict__ grad_out, int* __restrict__ nonfinite) {
    __shared__ WarpWork work[kWarpsApprox];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    WarpWork& ww = work[warp];
    const int B = c.n_band;
    constexpr int NG = SPS_NPARAM + 1;
    const uint32_t all = (B >= 32) ? 0xffffffffu : ((1u << B) - 1u);
    for (int64_t row = (int64_t)blockIdx.x * kWarpsApprox + warp; row < n;
         row += (int64_t)gridDim.x * kWarpsApprox) {
        const int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
        RowParams p;
        load_params(c, theta + row * SPS_NPARAM, false, p);
        if (gi < 0 || gi >= g.n) p.finite = false;
        if (!p.finite) {
            if (lane == 0) atomicOr(nonfinite, 1);
            if (lane == 0) ll_out[row] = __int_as_float(0x7fc00000);
            if (lane < NG) grad_out[row * NG + lane] = __int_as_float(0x7fc00000);
            continue;
        }
        const size_t gb0 = (size_t)gi * B;
        const int nb = fill_slots(c, g, ww.d, gi, mask[gi] & all, mag_obs, sigma, g.cssp + gb0 * c.K, false);
        const ZRow zr{g.dcssp + gb0 * c.K, g.dzp + gb0, g.ddust + gb0, g.dtdz[gi]};
        float gr[NG];
        const double ll = eval_row<true>(c, ww, g.bins + (size_t)gi * c.n_age, g.lnT[gi], g.lT10[gi], p,
                                         nb, true, true, gr, &zr);
        if (lane == 0) {
            ll_out[row] = (float)ll;
            bool bad = !isfinite(ll);
#pragma unroll
            for (int k = 0; k < NG; ++k) {
                bad = bad || !isfinite(gr[k]);
                grad_out[row * NG + k] = gr[k];
            }
            if (bad) atomicOr(nonfinite, 1);
        }
        __syncwarp();
    }
}

// W[row][i*Zn + j] = M_star P_SFH,i P_met,j and M_star (test hook).
__global__ void __launch_bounds__(32 * kWarpsApprox)
k_weights_rows(const __grid_constant__ Consts c, const Galaxies g, const float* __restrict__ theta,
               const int32_t* __restrict__ gal_idx, int64_t n, float* __restrict__ W_out,
               double* __restrict__ mstar_out) {
    __shared__ WarpWork work[kWarpsApprox];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    RowScratch& s = work[warp].r;
    for (int64_t row = (int64_t)blockIdx.x * kWarpsApprox + warp; row < n;
         row += (int64_t)gridDim.x * kWarpsApprox) {
        const int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
        if (gi < 0 || gi >= g.n) continue;
        RowParams p;
        load_params(c, theta + row * SPS_NPARAM, false, p);
        double M = age_met_weights(c, s, g.bins + (size_t)gi * c.n_age, g.lnT[gi], g.lT10[gi], p,
                                   false);
        const double scale = 1e9 * exp10((double)p.th[0]);
        if (mstar_out && lane == 0) mstar_out[row] = scale * M;
        if (W_out) {
            if (c.mdf_age) mdf_rows_fill(c, c.lgz_edge, p.th[7], p.th[8], s.u.kbuf);
            for (int k = lane; k < c.K; k += 32) {
                int i = k / c.n_met, j = k % c.n_met;
                const float q = c.mdf_age ? s.u.kbuf[k] : s.q[j];
                W_out[row * c.K + k] = (float)(scale * (double)s.w[i] * (double)q);
            }
        }
        __syncwarp();
    }
}

__global__ void k_philox(const uint32_t* __restrict__ ctr, int64_t n, uint64_t key,
                         uint32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint4 c4 = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
        uint4 r = philox4x32_10(c4, (uint32_t)(key & 0xffffffffu), (uint32_t)(key >> 32));
        out[4 * i] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    }
}

int blocks_for(int64_t rows, int per_block) {
    int64_t b = (rows + per_block - 1) / per_block;
    if (b > 152LL * 64) b = 152LL * 64;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_approx_rows(const Consts& c, const Galaxies& g, const float* theta,
                               int theta_unbounded, const int32_t* gal_idx, int64_t n,
                               const float* mag_obs, const float* sigma, const uint32_t* mask,
                               float* mag_out, float* loglike_out, float* grad_out,
                               double* logp_out, int* nonfinite, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_approx_rows<<<blocks_for(n, kWarpsApprox), 32 * kWarpsApprox, 0, s>>>(
        c, g, theta, theta_unbounded, gal_idx, n, mag_obs, sigma, mask, mag_out, loglike_out,
        grad_out, logp_out, nonfinite);
    return cudaGetLastError();
}

cudaError_t launch_approx_rows_z(const Consts& c, const Galaxies& g, const float* theta,
                                 const int32_t* gal_idx, int64_t n, const float* mag_obs,
                                 const float* sigma, const uint32_t* mask, float* loglike_out,
                                 float* grad_out, int* nonfinite, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_approx_rows_z<<<blocks_for(n, kWarpsApprox), 32 * kWarpsApprox, 0, s>>>(
        c, g, theta, gal_idx, n, mag_obs, sigma, mask, loglike_out, grad_out, nonfinite);
    return cudaGetLastError();
}

cudaError_t launch_weights_rows(const Consts& c, const Galaxies& g, const float* theta,
                                const int32_t* gal_idx, int64_t n, float* W_out,
                                double* mstar_out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_weights_rows<<<blocks_for(n, kWarpsApprox), 32 * kWarpsApprox, 0, s>>>(
        c, g, theta, gal_idx, n, W_out, mstar_out);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out,
                          cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_philox<<<blocks, 256, 0, s>>>(ctr, n, key, out);
    return cudaGetLastError();
}

}  // namespace sps
