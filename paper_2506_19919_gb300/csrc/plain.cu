// Plain per-galaxy forward-mode path: the comparison baseline for the fused
// adjoint (Sec. 3 approximate photometry, App. D.1 likelihood).
//
// Three unfused kernels per batch of rows, each a separate launch with its
// intermediate in HBM, as a straightforward GPU port of the model would be
// written:
//   k_plain_tangents : W[r][k] and its tangents dW/dtheta for the 8 parameters
//                      that enter the weights (tau, alpha, beta, F_burst,
//                      lgT_peak, dlgT, lgZ, sigma_lgZ) -> T[r][9][K] in HBM
//   k_plain_contract : c[r][b][d] = sum_k T[r][d][k] c_SSP[g][b][k] for the 9
//                      directions (one warp per (row, band))
//   k_plain_like     : magnitudes, log L and the gradient by the chain rule
//                      (lgM and dust directions analytic)
// Forward mode costs one contraction per direction, so 9x the forward work
// of the fused kernel's forward pass, against ~2x for the hand-written
// adjoint.
#include "sps_device.cuh"

namespace sps {

namespace {

constexpr int kDir = 9;   // value + 8 weight-parameter tangents

// tangent of the metallicity weights: dq_j/d(lgZ), dq_j/d(sigma_lgZ)
__device__ __forceinline__ void met_tangents(const Consts& c, float mu, float sd, int j, float& dmu,
                                             float& dsd) {
    const float yl = (c.lgz_edge[j] - mu) / sd, yh = (c.lgz_edge[j + 1] - mu) / sd;
    dmu = -(phi_(yh) - phi_(yl)) / sd;
    dsd = -(phi_y(yh) - phi_y(yl)) / sd;
}

__global__ void __launch_bounds__(32 * kWarpsApprox)
k_plain_tangents(const __grid_constant__ Consts c, const Galaxies g, const float* __restrict__ theta,
                 const int32_t* __restrict__ gal_idx, int64_t n, float* __restrict__ T) {
    __shared__ RowScratch scratch[kWarpsApprox];
    __shared__ float sdpi[kWarpsApprox][2][kMaxAges];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    RowScratch& s = scratch[warp];
    const int A = c.n_age, Zn = c.n_met, K = c.K;
    for (int64_t row = (int64_t)blockIdx.x * kWarpsApprox + warp; row < n;
         row += (int64_t)gridDim.x * kWarpsApprox) {
        int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
        if (gi < 0 || gi >= g.n) gi = 0;
        RowParams p;
        load_params(c, theta + row * SPS_NPARAM, false, p);
        const double M = age_met_weights(c, s, g.bins + (size_t)gi * A, g.lnT[gi], g.lT10[gi], p, true);
        const float fb = p.th[4], Mf = (float)M;
        // burst tangents d pi_i / d(mu, sigma) with the renormalisation
        const float lT = g.lT10[gi], mu = p.th[5], sig = p.th[6] * (1.0f / 3.0f);
        const float xT = (lT - mu) / sig, D = tri_cdf(xT), tT = tri_pdf(xT);
        for (int i = lane; i < A; i += 32) {
            const float lo = fminf(c.log_age_edge[i], lT), hi = fminf(c.log_age_edge[i + 1], lT);
            const float xl = (lo - mu) / sig, xh = (hi - mu) / sig;
            const float tl = tri_pdf(xl), th = tri_pdf(xh);
            const float draw_mu = -(th - tl) / sig, draw_sg = -(xh * th - xl * tl) / sig;
            sdpi[warp][0][i] = (draw_mu - s.pi[i] * (-tT / sig)) / D;
            sdpi[warp][1][i] = (draw_sg - s.pi[i] * (-xT * tT / sig)) / D * (1.0f / 3.0f);
        }
        // d M / d(tau, alpha, beta)
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int i = lane; i < A; i += 32) {
            a0 += s.dm[0][i];
            a1 += s.dm[1][i];
            a2 += s.dm[2][i];
        }
        const float dM0 = warp_sum(a0), dM1 = warp_sum(a1), dM2 = warp_sum(a2);
        __syncwarp();
        float* out = T + (size_t)row * kDir * K;
        for (int k = lane; k < K; k += 32) {
            const int i = k / Zn, j = k - (k / Zn) * Zn;
            const float qj = s.q[j], wi = s.w[i];
            float dqm, dqs;
            met_tangents(c, p.th[7], p.th[8], j, dqm, dqs);
            const float pib = s.pi[i];
            out[0 * K + k] = wi * qj;
            out[1 * K + k] = ((1.0f - fb) * s.dm[0][i] + fb * pib * dM0) * qj;
            out[2 * K + k] = ((1.0f - fb) * s.dm[1][i] + fb * pib * dM1) * qj;
            out[3 * K + k] = ((1.0f - fb) * s.dm[2][i] + fb * pib * dM2) * qj;
            out[4 * K + k] = (pib * Mf - s.m[i]) * qj;
            out[5 * K + k] = fb * Mf * sdpi[warp][0][i] * qj;
            out[6 * K + k] = fb * Mf * sdpi[warp][1][i] * qj;
            out[7 * K + k] = wi * dqm;
            out[8 * K + k] = wi * dqs;
        }
        __syncwarp();
    }
}

// One warp per (row, band): the 9 contractions with the galaxy's c_SSP row.
__global__ void __launch_bounds__(256)
k_plain_contract(const __grid_constant__ Consts c, const Galaxies g, const int32_t* __restrict__ gal_idx,
                 int64_t n, const float* __restrict__ T, float* __restrict__ cd) {
    const int B = c.n_band, K = c.K;
    const int64_t item = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = lane_id();
    if (item >= n * B) return;
    const int64_t row = item / B;
    const int b = (int)(item - row * B);
    int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
    if (gi < 0 || gi >= g.n) gi = 0;
    const float* C = g.cssp + ((size_t)gi * B + b) * K;
    const float* Tr = T + (size_t)row * kDir * K;
    float acc[kDir];
#pragma unroll
    for (int d = 0; d < kDir; ++d) acc[d] = 0.0f;
    for (int k = lane; k < K; k += 32) {
        const float cv = __ldg(C + k);
#pragma unroll
        for (int d = 0; d < kDir; ++d) acc[d] = fmaf(__ldg(Tr + d * K + k), cv, acc[d]);
    }
#pragma unroll
    for (int d = 0; d < kDir; ++d) {
        const float v = warp_sum(acc[d]);
        if (lane == 0) cd[(row * B + b) * kDir + d] = v;
    }
}

// One thread per row: magnitudes, log L, gradient by the chain rule.
__global__ void k_plain_like(const __grid_constant__ Consts c, const Galaxies g,
                             const float* __restrict__ theta, const int32_t* __restrict__ gal_idx,
                             int64_t n, const float* __restrict__ cd, const float* __restrict__ mag_obs,
                             const float* __restrict__ sigma, const uint32_t* __restrict__ mask,
                             float* __restrict__ ll_out, float* __restrict__ grad_out,
                             double* __restrict__ ll64_out) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int B = c.n_band;
    int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
    if (gi < 0 || gi >= g.n) gi = 0;
    const float* t = theta + row * SPS_NPARAM;
    const uint32_t bits = mask[gi];
    double ll = 0.0;
    float gr[SPS_NPARAM];
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) gr[k] = 0.0f;
    for (int b = 0; b < B; ++b) {
        if (!((bits >> b) & 1u)) continue;
        const float* v = cd + (row * B + b) * kDir;
        const float4 dc = g.dust_eff[gi * B + b];
        const DustTerms d = dust_eval(dc.x, dc.y, dc.z, t[9], t[10], t[11]);
        const double lc = log10((double)d.F * (double)v[0]) + (double)t[0] + 9.0;
        const double m = g.zp[gi * B + b] - 2.5 * lc;
        const double is2 = 1.0 / ((double)sigma[gi * B + b] * (double)sigma[gi * B + b]);
        const double r = m - (double)mag_obs[gi * B + b];
        ll += -0.5 * r * r * is2;
        const float gam = (float)(2.5 * r * is2 / 2.302585092994046);
        gr[0] += gam * kLn10f;
        const float gS = gam / v[0];
        gr[1] += gS * v[1];
        gr[2] += gS * v[2];
        gr[3] += gS * v[3];
        gr[4] += gS * v[4];
        gr[5] += gS * v[5];
        gr[6] += gS * v[6];
        gr[7] += gS * v[7];
        gr[8] += gS * v[8];
        const float gF = gam / d.F;
        gr[9] += gF * d.dF_AV;
        gr[10] += gF * d.dF_delta;
        gr[11] += gF * d.dF_floor;
    }
    if (ll_out) ll_out[row] = (float)ll;
    if (ll64_out) ll64_out[row] = ll;
    if (grad_out)
#pragma unroll
        for (int k = 0; k < SPS_NPARAM; ++k) grad_out[row * SPS_NPARAM + k] = gr[k];
}

}  // namespace

size_t plain_scratch_bytes_per_row(const Consts& c) {
    return (size_t)kDir * c.K * sizeof(float) + (size_t)c.n_band * kDir * sizeof(float);
}

cudaError_t launch_plain(const Consts& c, const Galaxies& g, const float* theta,
                         const int32_t* gal_idx, int64_t n, const float* mag_obs,
                         const float* sigma, const uint32_t* mask, float* ll_out, float* grad_out,
                         float* T, float* cd, cudaStream_t s, double* ll64_out) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + kWarpsApprox - 1) / kWarpsApprox;
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    k_plain_tangents<<<(unsigned)blocks, 32 * kWarpsApprox, 0, s>>>(c, g, theta, gal_idx, n, T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t items = n * c.n_band;
    k_plain_contract<<<(unsigned)((items + 7) / 8), 256, 0, s>>>(c, g, gal_idx, n, T, cd);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_plain_like<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(c, g, theta, gal_idx, n, cd, mag_obs, sigma,
                                                             mask, ll_out, grad_out, ll64_out);
    return cudaGetLastError();
}

}  // namespace sps
