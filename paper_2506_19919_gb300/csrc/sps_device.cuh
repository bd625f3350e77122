// Device-side model of arXiv 2506.19919 (App. A) evaluated by one warp per
// (galaxy, chain) row, and its hand-written adjoint.
//
// Forward, per row (App. A.1-A.3):
//   m_i    = int_{bin i} SFR shape dt  (Eq. SFRsmooth, Eq. smoothPsfh), by
//            Gauss-Legendre panels in x = ln t with the substitution
//            t = tau e^u:  m_i = tau int hh(u) du, hh = 1 / (e^{(a-1)u} + e^{-(b+1)u}).
//            The integrand is analytic in a strip of half-width pi/(a+b) around
//            the real axis, so panels of width <= 0.25 give ~1e-9 accuracy.
//            Below x_min = min(ln t_obs - ln tau, 0) - 30/(b+1) the remaining
//            mass is < 1e-10 of the total and is dropped.
//   M      = sum_i m_i in FP64 (the cumulative mass integral, Eq. totalMstarFormed)
//   pi_i   = triweight CDF mass of bin i in log age, clipped at t_obs and
//            renormalised (Eq. triweight)
//   q_j    = Gaussian (log10 Z) mass of metallicity bin j (App. A.2)
//   w_i    = (1 - F_burst) m_i + F_burst pi_i M  (Eq. composite_age_weights x M_star)
//   W_ij   = 1e9 10^lgM w_i q_j                    (Eq. galSED_decomposed)
//   S_b    = sum_ij w_i q_j c_SSP[b][ij]           (Eq. photo_integral_approx)
//   c_b    = 1e9 10^lgM F_att(lambda_eff,b) S_b;  m_b = zp_b - 2.5 log10 c_b (FP64)
//
// Adjoint (reverse order; recomputes the per-SSP products):
//   gamma_b = dlogL / dln c_b = 2.5 r_b / (sigma_b^2 ln 10)
//   v_ij    = sum_b (gamma_b / S_b) c_SSP[b][ij]
//   wbar_i  = sum_j v_ij q_j,   qbar_j = sum_i v_ij w_i
//   mbar_l  = (1 - F_b) wbar_l + F_b sum_i wbar_i pi_i
//   then through the bin integrals, the triweight CDF and the normal CDF.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sps_internal.h"

namespace sps {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kLn10f = 2.302585092994046f;
constexpr float kLog2_10f = 3.321928094887362f;
constexpr float kInvSqrt2Pi = 0.3989422804014327f;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ---------------------------------------------------------------- triweight
// CDF of Eq. triweight: with u = x/3 clipped to [-1, 1],
// 1/2 + (35/32)(u - u^3 + 3u^5/5 - u^7/7).
__device__ __forceinline__ float tri_cdf(float x) {
    float u = fminf(fmaxf(x * (1.0f / 3.0f), -1.0f), 1.0f);
    float u2 = u * u;
    float p = u * (1.0f - u2 * (1.0f - u2 * (0.6f - u2 * (1.0f / 7.0f))));
    return 0.5f + (35.0f / 32.0f) * p;
}
__device__ __forceinline__ float tri_pdf(float x) {
    float t = 1.0f - (x * x) * (1.0f / 9.0f);
    return (fabsf(x) <= 3.0f) ? (35.0f / 96.0f) * t * t * t : 0.0f;
}

// ---------------------------------------------------------------- dust
// F_att = F_floor + (1 - F_floor) 10^{-0.4 A},  A = (A_V/4.05)(k0 (l/l_V)^delta + E_b D),
// E_b = max(0.85 - 1.9 delta, 0)  (Eq. DustAtt, App. A.3).
struct DustTerms {
    float F, dF_AV, dF_delta, dF_floor;
};
__device__ __forceinline__ DustTerms dust_eval(float k0, float lnr, float drude, float AV,
                                              float delta, float ffl) {
    float eb = fmaxf(0.85f - 1.9f * delta, 0.0f);
    float pw = __expf(delta * lnr);
    float base = k0 * pw + eb * drude;
    float A = AV * (1.0f / 4.05f) * base;
    float E = exp2f(-0.4f * kLog2_10f * A);
    DustTerms d;
    d.F = ffl + (1.0f - ffl) * E;
    float g = (1.0f - ffl) * E * (-0.4f * kLn10f);
    d.dF_AV = g * base * (1.0f / 4.05f);
    d.dF_delta = g * AV * (1.0f / 4.05f) * (k0 * pw * lnr - (eb > 0.0f ? 1.9f * drude : 0.0f));
    d.dF_floor = 1.0f - E;
    return d;
}

// ---------------------------------------------------------------- per-warp scratch
// Panel bookkeeping of the SFH quadrature of one row.
struct PanelScratch {
    float px0[kMaxAges];        // first panel centre (ln t)
    float php[kMaxAges];        // panel half-width
    unsigned short pn[kMaxAges];
    unsigned short pstart[kMaxAges + 1];
    unsigned char pmap[kMaxPanels];
};

// Where the age / metallicity stage of one row keeps its arrays.
struct AgeView {
    float* m;          // [A] bin integrals
    float* dm0;        // [A] d m / d tau
    float* dm1;        // [A] d m / d alpha
    float* dm2;        // [A] d m / d beta
    float* pi;         // [A] burst weights
    float* w;          // [A] age weights
    float* wb;         // [A] adjoint of w
    float* q;          // [Zn] metallicity weights
    float* qb;         // [Zn] adjoint of q
    PanelScratch* ps;
};

struct RowScratch {
    float m[kMaxAges];          // bin integrals tau * int hh du [Gyr]
    float dm[3][kMaxAges];      // d m / d(tau, alpha, beta)
    float pi[kMaxAges];         // burst weights
    float w[kMaxAges];          // age weights w_i
    float wb[kMaxAges];         // adjoint of w_i
    union {
        PanelScratch s;
        float kbuf[kKTileMax * 32];     // v_ij during the adjoint
    } u;
    float q[kMaxMets];
    float qb[kMaxMets];
    int slot_band[kMaxBands];
    float slot_S[kMaxBands];
    float slot_F[kMaxBands];
    float slot_g[kMaxBands];    // gamma_b
    __device__ AgeView view() {
        return AgeView{m, dm[0], dm[1], dm[2], pi, w, wb, q, qb, &u.s};
    }
};

// ---------------------------------------------------------------- SFH bins
// Panel count ceil(w / panel) clamped to [1, kMaxPanels]; NaN or inf give a
// bounded count so that no input can index outside the scratch arrays.
__device__ __forceinline__ int panel_count(float w, float panel) {
    float f = ceilf(w / panel);
    return (f >= 1.0f) ? ((f < (float)kMaxPanels) ? (int)f : kMaxPanels) : 1;
}

// Fills s.m and (if grad) s.dm; returns M = sum_i m_i (FP64).
__device__ __forceinline__ double sfh_bins(const Consts& c, const AgeView& v, const float2* __restrict__ bins,
                           float lnT, float tau, float alpha, float beta, bool grad) {
    PanelScratch& ps = *v.ps;
    const int lane = lane_id();
    const int A = c.n_age;
    const float lntau = __logf(tau);
    const float xmin = lntau + fminf(lnT - lntau, 0.0f) - 30.0f / (beta + 1.0f);
    const float panel = c.panel;
    for (int i = lane; i < A; i += 32) {
        float2 b = bins[i];
        int n = 0;
        float x0 = 0.0f, hp = 0.0f;
        if (b.y < 0.0f) {                          // reaches t = 0
            float w = b.x - xmin;
            if (w > 0.0f) {
                n = panel_count(w, panel);
                hp = 0.5f * w / (float)n;
                x0 = xmin + hp;
            }
        } else if (b.y > 0.0f) {
            float hi = b.x + b.y;
            float lo = b.x - b.y;
            if (hi > xmin) {
                if (lo < xmin) {
                    float w = hi - xmin;
                    n = panel_count(w, panel);
                    hp = 0.5f * w / (float)n;
                    x0 = xmin + hp;
                } else {
                    n = panel_count(2.0f * b.y, panel);
                    hp = b.y / (float)n;
                    x0 = b.x + (float)(1 - n) * hp;
                }
            }
        }
        ps.pn[i] = (unsigned short)n;
        ps.px0[i] = x0;
        ps.php[i] = hp;
        v.m[i] = 0.0f;
        v.dm0[i] = 0.0f;
        v.dm1[i] = 0.0f;
        v.dm2[i] = 0.0f;
    }
    __syncwarp();
    int carry = 0;
    for (int base = 0; base < A; base += 32) {
        int i = base + lane;
        int n = (i < A) ? (int)ps.pn[i] : 0;
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (i < A) ps.pstart[i] = (unsigned short)min(carry + incl - n, kMaxPanels);
        carry += __shfl_sync(kFull, incl, 31);
    }
    const int P = min(carry, kMaxPanels);
    __syncwarp();
    for (int i = lane; i < A; i += 32) {
        int p0 = ps.pstart[i];
        int p1 = min(p0 + (int)ps.pn[i], kMaxPanels);
        for (int p = p0; p < p1; ++p) ps.pmap[p] = (unsigned char)i;
    }
    __syncwarp();
    const float am1 = alpha - 1.0f, bp1 = beta + 1.0f;
    for (int base = 0; base < P; base += 32) {
        const int p = base + lane;
        const bool act = p < P;
        int bin = act ? (int)ps.pmap[p] : -1;
        float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
        if (act) {
            const int k = p - (int)ps.pstart[bin];
            const float hp = ps.php[bin];
            const float xc = ps.px0[bin] + 2.0f * (float)k * hp - lntau;
            for (int gq = 0; gq < c.gl_order; ++gq) {
                float uu = fmaf(hp, c.gl_x[gq], xc);
                float P_ = __expf(am1 * uu);
                float Q_ = __expf(-bp1 * uu);
                float hh = __frcp_rn(P_ + Q_);
                float wq = c.gl_w[gq] * hp;
                v0 = fmaf(wq, hh, v0);
                if (grad) {
                    float h2 = hh * hh * wq;
                    v1 = fmaf(h2, alpha * P_ - beta * Q_, v1);
                    v2 = fmaf(-h2 * P_, uu, v2);
                    v3 = fmaf(h2 * Q_, uu, v3);
                }
            }
        }
        // segmented inclusive scan over panels of the same bin (bins are sorted)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            float t0 = __shfl_up_sync(kFull, v0, o);
            float t1 = __shfl_up_sync(kFull, v1, o);
            float t2 = __shfl_up_sync(kFull, v2, o);
            float t3 = __shfl_up_sync(kFull, v3, o);
            int bo = __shfl_up_sync(kFull, bin, o);
            if (lane >= o && bo == bin) {
                v0 += t0; v1 += t1; v2 += t2; v3 += t3;
            }
        }
        int bnext = __shfl_down_sync(kFull, bin, 1);
        if (act && (lane == 31 || bnext != bin)) {
            v.m[bin] += v0 * tau;
            if (grad) {
                v.dm0[bin] += v1;
                v.dm1[bin] += v2 * tau;
                v.dm2[bin] += v3 * tau;
            }
        }
        __syncwarp();
    }
    double acc = 0.0;
    for (int i = lane; i < A; i += 32) acc += (double)v.m[i];
    return warp_sum_d(acc);
}

// ---------------------------------------------------------------- burst + MDF
__device__ __forceinline__ float burst_weights(const Consts& c, const AgeView& v, float lT10,
                                               float mu, float sig) {
    const float xT = (lT10 - mu) / sig;
    const float D = tri_cdf(xT);
    const float invD = 1.0f / D;
    for (int i = lane_id(); i < c.n_age; i += 32) {
        float lo = fminf(c.log_age_edge[i], lT10);
        float hi = fminf(c.log_age_edge[i + 1], lT10);
        v.pi[i] = (tri_cdf((hi - mu) / sig) - tri_cdf((lo - mu) / sig)) * invD;
    }
    return D;
}

__device__ __forceinline__ void met_weights(const Consts& c, const AgeView& v, float mu, float sd) {
    int j = lane_id();
    if (j < c.n_met) {
        float ylo = (c.lgz_edge[j] - mu) / sd;
        float yhi = (c.lgz_edge[j + 1] - mu) / sd;
        v.q[j] = (ylo > 0.0f) ? normcdff(-ylo) - normcdff(-yhi) : normcdff(yhi) - normcdff(ylo);
    }
}

__device__ __forceinline__ float phi_y(float y) {  // y phi(y), 0 at +-inf
    return isinf(y) ? 0.0f : y * kInvSqrt2Pi * __expf(-0.5f * y * y);
}
__device__ __forceinline__ float phi_(float y) {
    return isinf(y) ? 0.0f : kInvSqrt2Pi * __expf(-0.5f * y * y);
}

// ---------------------------------------------------------------- bounding map
// theta = lo + span / (1 + exp(-x))  (Eq. BoundingFunction, k = 1, x0 = 0).
__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + __expf(-x)); }

// Parameters of one row held uniformly by the warp.
struct RowParams {
    float th[SPS_NPARAM];
    float dth[SPS_NPARAM];   // d theta / d x (unbounded input) or 1
    double logprior;         // log Jacobian of the bounding map (unbounded input) or 0
    bool finite;
};

__device__ __forceinline__ void load_params(const Consts& c, const float* __restrict__ src,
                                            bool unbounded, RowParams& p) {
    p.finite = true;
    p.logprior = 0.0;
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) {
        float x = src[k];
        p.finite = p.finite && isfinite(x);
        if (unbounded) {
            float sg = sigmoidf_(x);
            p.th[k] = c.prior_lo[k] + c.prior_span[k] * sg;
            p.dth[k] = c.prior_span[k] * sg * (1.0f - sg);
            float ax = fabsf(x);
            p.logprior += (double)(-ax - 2.0f * log1pf(__expf(-ax)));
        } else {
            p.th[k] = x;
            p.dth[k] = 1.0f;
        }
    }
}

// ---------------------------------------------------------------- weights stage
// Fills v.m/dm, v.pi, v.q, v.w for parameters th[12]; returns M (FP64).
__device__ __forceinline__ double age_met_weights(const Consts& c, const AgeView& v,
                                                  const float2* __restrict__ bins, float lnT,
                                                  float lT10, const float* th, bool grad) {
    double M = sfh_bins(c, v, bins, lnT, th[1], th[2], th[3], grad);
    burst_weights(c, v, lT10, th[5], th[6] * (1.0f / 3.0f));
    met_weights(c, v, th[7], th[8]);
    __syncwarp();
    const float fb = th[4];
    const float Mf = (float)M;
    for (int i = lane_id(); i < c.n_age; i += 32) v.w[i] = (1.0f - fb) * v.m[i] + fb * v.pi[i] * Mf;
    __syncwarp();
    return M;
}
__device__ __forceinline__ double age_met_weights(const Consts& c, RowScratch& s,
                                                  const float2* __restrict__ bins, float lnT,
                                                  float lT10, const RowParams& p, bool grad) {
    return age_met_weights(c, s.view(), bins, lnT, lT10, p.th, grad);
}

// Adjoint of age_met_weights: given s.wb (dlogL/dw_i) and s.qb (dlogL/dq_j)
// returns d/dtheta for columns 1-8 added into g[].
__device__ __forceinline__ void age_met_adjoint(const Consts& c, const AgeView& s, float lT10, double M,
                                             const float* th, float* g) {
    const int lane = lane_id();
    const int A = c.n_age;
    const float fb = th[4];
    const float Mf = (float)M;
    // sum_i wbar_i pi_i  and  F_burst-bar
    float a_wp = 0.f, a_fb = 0.f;
    for (int i = lane; i < A; i += 32) {
        float wb = s.wb[i];
        a_wp += wb * s.pi[i];
        a_fb += wb * (s.pi[i] * Mf - s.m[i]);
    }
    a_wp = warp_sum(a_wp);
    a_fb = warp_sum(a_fb);
    // smooth SFH: mbar_l = (1 - fb) wbar_l + fb sum_i wbar_i pi_i
    float gt = 0.f, ga = 0.f, gbt = 0.f;
    for (int i = lane; i < A; i += 32) {
        float mb = (1.0f - fb) * s.wb[i] + fb * a_wp;
        gt += mb * s.dm0[i];
        ga += mb * s.dm1[i];
        gbt += mb * s.dm2[i];
    }
    g[1] += warp_sum(gt);
    g[2] += warp_sum(ga);
    g[3] += warp_sum(gbt);
    g[4] += a_fb;
    // burst: pi_i = raw_i / D, pibar_i = fb M wbar_i
    const float mu = th[5], sig = th[6] * (1.0f / 3.0f);
    const float xT = (lT10 - mu) / sig;
    const float D = tri_cdf(xT);
    float s_mu = 0.f, s_sg = 0.f, s_pp = 0.f;
    for (int i = lane; i < A; i += 32) {
        float lo = fminf(c.log_age_edge[i], lT10);
        float hi = fminf(c.log_age_edge[i + 1], lT10);
        float xl = (lo - mu) / sig, xh = (hi - mu) / sig;
        float pib = fb * Mf * s.wb[i];
        float tl = tri_pdf(xl), th = tri_pdf(xh);
        s_mu += pib * (-(th - tl));
        s_sg += pib * (-(xh * th - xl * tl));
        s_pp += pib * s.pi[i];
    }
    s_mu = warp_sum(s_mu);
    s_sg = warp_sum(s_sg);
    s_pp = warp_sum(s_pp);
    const float tT = tri_pdf(xT);
    // d raw/d mu = -(T(xh) - T(xl))/sig ; dD/dmu = -T(xT)/sig  (and x T(x) for sigma)
    float gmu = (s_mu - s_pp * (-tT)) / (sig * D);
    float gsg = (s_sg - s_pp * (-xT * tT)) / (sig * D);
    g[5] += gmu;
    g[6] += gsg * (1.0f / 3.0f);
    // metallicity: q_j = Phi(yh) - Phi(yl)
    const float mz = th[7], sz = th[8];
    float gz = 0.f, gs = 0.f;
    int j = lane;
    if (j < c.n_met) {
        float yl = (c.lgz_edge[j] - mz) / sz, yh = (c.lgz_edge[j + 1] - mz) / sz;
        float qb = s.qb[j];
        gz = qb * (-(phi_(yh) - phi_(yl)) / sz);
        gs = qb * (-(phi_y(yh) - phi_y(yl)) / sz);
    }
    g[7] += warp_sum(gz);
    g[8] += warp_sum(gs);
}
__device__ inline void age_met_adjoint(const Consts& c, RowScratch& s, float lT10, double M,
                                       const RowParams& p, float* g) {
    age_met_adjoint(c, s.view(), lT10, M, p.th, g);
}

}  // namespace sps
