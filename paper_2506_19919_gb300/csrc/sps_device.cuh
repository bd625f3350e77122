// Device-side model of arXiv 2506.19919 (App. A) evaluated by one warp per
// (galaxy, chain) row, and its hand-written adjoint.
//
// Forward, per row (App. A.1-A.3):
//   m_i    = int_{bin i} SFR shape dt  (Eq. SFRsmooth, Eq. smoothPsfh), by
//            Gauss-Legendre rules in x = ln t with the substitution
//            t = tau e^u:  m_i = tau int hh(u) du, hh = 1 / (e^{(a-1)u} + e^{-(b+1)u}).
//            Narrow bins take one 2- or 3-node panel, wide bins panels of the
//            full rule sized by the analyticity strip (see sfh_bins); the part
//            of the oldest bin below e^-22 of the peak integrand is dropped.
//   q_j, pi_i are differences of CDFs at the bin edges, one CDF per edge.
//   M      = sum_i m_i in FP64 (the cumulative mass integral, Eq. totalMstarFormed)
//   pi_i   = triweight CDF mass of bin i in log age, clipped at t_obs and
//            renormalised (Eq. triweight)
//   q_j    = Gaussian (log10 Z) mass of metallicity bin j (App. A.2)
//   w_i    = (1 - F_burst) m_i + F_burst pi_i M  (Eq. composite_age_weights x M_star)
//   W_ij   = 1e9 10^lgM w_i q_j                    (Eq. galSED_decomposed)
//   S_b    = sum_ij w_i q_j c_SSP[b][ij]           (Eq. photo_integral_approx)
//   c_b    = 1e9 10^lgM F_att(lambda_eff,b) S_b;  m_b = zp_b - 2.5 log10 c_b (FP64
//            magnitude; the log's exponent part exact, its mantissa part FP32)
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

// ---------------------------------------------------------------- 3xTF32 split
// hi = x rounded to TF32 (10 mantissa bits, the low 13 bits zero), lo = x - hi
// (exact in FP32): the operand halves of a 3xTF32 tensor-core product.
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    hi = __uint_as_float(r);
    lo = x - hi;
}

// ---------------------------------------------------------------- magnitudes
// log10 of a positive FP32 flux for the magnitude m = zp - 2.5 log10 c: with
// x = f 2^e, f in [0.5, 1), the exponent part e log10(2) is exact in FP64 and
// log10(f) (|.| < 0.31) is an FP32 log, so the result is good to ~5e-8 at any
// flux, faint or bright; x = 0 gives -inf.
__device__ __forceinline__ double log10_flux(float x) {
    int e;
    const float f = frexpf(x, &e);
    return fma((double)e, 0.30102999566398120, (double)logf(f) * 0.43429448190325182);
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
    float4 info[kMaxAges];            // per queued bin: (first panel centre, half-width,
                                      //  first panel index as int bits or -1, unused)
    unsigned char pmap[kMaxPanels];   // bin index at each queued bin's first panel
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
    const float* age_edge;   // [A + 1] log10 age-bin edges (shared or parameter memory)
    const float* lgz_edge;   // [Zn + 1] metallicity-bin edges
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
    float slot_D[kMaxBands];    // sum_k W_k d c_SSP[b][k] / dz (redshift gradient)
    float slot_g[kMaxBands];    // gamma_b
    __device__ AgeView view(const Consts& c) {
        return AgeView{m, dm[0], dm[1], dm[2], pi, w, wb, q, qb, &u.s, c.log_age_edge, c.lgz_edge};
    }
};

// ---------------------------------------------------------------- SFH bins
// Panel count ceil(f) clamped to [1, kMaxPanels]; NaN or inf give a bounded
// count so that no input can index outside the scratch arrays.
__device__ __forceinline__ int panel_count(float f) {
    f = ceilf(f);
    return (f >= 1.0f) ? ((f < (float)kMaxPanels) ? (int)f : kMaxPanels) : 1;
}

// One panel of an N-node Gauss-Legendre rule (nodes gx, weights gw on [-1, 1])
// centred at u = xc with half-width hp: accumulates int hh du into v0 and, if
// grad, the integrands of d/d(alpha), d/d(ln tau-free parts) into v1..v3, with
// hh = 1 / (P + Q), P = e^{(alpha-1)u}, Q = e^{-(beta+1)u}.  Written with the
// exponent of the ratio Q/P or P/Q kept <= 0 (no overflow):
//   u < 0:  hh = e^{(beta+1)u} r,  r = 1 / (1 + e^{(alpha+beta)u}),  hh P = 1 - r, hh Q = r
//   u >= 0: hh = e^{(1-alpha)u} r, r = 1 / (1 + e^{-(alpha+beta)u}), hh P = r,     hh Q = 1 - r
// so that dhh/dalpha = -u hh (hh P), dhh/dbeta = u hh (hh Q) and
// alpha P - beta Q = (alpha hhP - beta hhQ) / hh.  kPack takes the nodes in pairs
// with packed FP32x2 arithmetic (faster in the HMC team kernel, slower in the
// one-row-per-warp kernels, which keep the scalar loop).
template <int N, bool kPack = false>
__device__ __forceinline__ void gl_panel(const float* __restrict__ gx, const float* __restrict__ gw,
                                         float hp, float xc, float alpha, float beta, bool grad,
                                         float& v0, float& v1, float& v2, float& v3) {
    const float kL2E = 1.4426950408889634f;
    const float cneg = (beta + 1.0f) * kL2E, cpos = (1.0f - alpha) * kL2E, cs = -(alpha + beta) * kL2E;
    if constexpr (kPack) {
        // nodes in pairs with packed FP32x2 arithmetic (MUFU per element)
        const float2 hp2 = make_float2(hp, hp), xc2 = make_float2(xc, xc);
        const float2 one2 = make_float2(1.0f, 1.0f);
        float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
#pragma unroll
        for (int q = 0; q + 1 < N; q += 2) {
            const float2 uu = __ffma2_rn(hp2, make_float2(gx[q], gx[q + 1]), xc2);
            const bool px = uu.x >= 0.0f, py = uu.y >= 0.0f;
            const float2 Ea = __fmul2_rn(uu, make_float2(px ? cpos : cneg, py ? cpos : cneg));
            const float2 Ra = __fmul2_rn(make_float2(fabsf(uu.x), fabsf(uu.y)), make_float2(cs, cs));
            const float2 E = make_float2(exp2f(Ea.x), exp2f(Ea.y));
            const float2 R = make_float2(exp2f(Ra.x), exp2f(Ra.y));
            const float2 d = __fadd2_rn(one2, R);
            const float2 r = make_float2(__fdividef(1.0f, d.x), __fdividef(1.0f, d.y));
            const float2 wh = __fmul2_rn(__fmul2_rn(make_float2(gw[q], gw[q + 1]), hp2), __fmul2_rn(E, r));
            a0 = __fadd2_rn(a0, wh);
            if (grad) {
                const float2 hP = make_float2(px ? r.x : 1.0f - r.x, py ? r.y : 1.0f - r.y);   // hh P
                const float2 hQ = __fadd2_rn(one2, make_float2(-hP.x, -hP.y));              // hh Q
                const float2 tt = __ffma2_rn(make_float2(alpha, alpha), hP, __fmul2_rn(make_float2(-beta, -beta), hQ));
                a1 = __ffma2_rn(wh, tt, a1);
                const float2 whu = __fmul2_rn(wh, uu);
                a2 = __ffma2_rn(make_float2(-whu.x, -whu.y), hP, a2);
                a3 = __ffma2_rn(whu, hQ, a3);
            }
        }
        if (N & 1) {
            const int q = N - 1;
            const float uu = fmaf(hp, gx[q], xc);
            const bool pos = uu >= 0.0f;
            const float E = exp2f(uu * (pos ? cpos : cneg));
            const float R = exp2f(fabsf(uu) * cs);
            const float r = __fdividef(1.0f, 1.0f + R);
            const float wh = gw[q] * hp * E * r;
            a0.x += wh;
            if (grad) {
                const float hP = pos ? r : 1.0f - r;
                const float hQ = 1.0f - hP;
                a1.x = fmaf(wh, alpha * hP - beta * hQ, a1.x);
                const float whu = wh * uu;
                a2.x = fmaf(-whu, hP, a2.x);
                a3.x = fmaf(whu, hQ, a3.x);
            }
        }
        v0 += a0.x + a0.y;
        if (grad) {
            v1 += a1.x + a1.y;
            v2 += a2.x + a2.y;
            v3 += a3.x + a3.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            const float uu = fmaf(hp, gx[q], xc);
            const bool pos = uu >= 0.0f;
            const float E = exp2f(uu * (pos ? cpos : cneg));
            const float R = exp2f(fabsf(uu) * cs);
            const float r = __fdividef(1.0f, 1.0f + R);
            const float wh = gw[q] * hp * E * r;                      // w hh
            v0 += wh;
            if (grad) {
                const float hP = pos ? r : 1.0f - r;                  // hh P
                const float hQ = 1.0f - hP;                           // hh Q
                v1 = fmaf(wh, alpha * hP - beta * hQ, v1);
                const float whu = wh * uu;
                v2 = fmaf(-whu, hP, v2);
                v3 = fmaf(whu, hQ, v3);
            }
        }
    }
}
__device__ __forceinline__ void gl_panel_any(int n, const float* __restrict__ gx,
                                             const float* __restrict__ gw, float hp, float xc,
                                             float alpha, float beta, bool grad, float& v0,
                                             float& v1, float& v2, float& v3) {
#pragma unroll 1
    for (int q = 0; q < n; ++q) gl_panel<1>(gx + q, gw + q, hp, xc, alpha, beta, grad, v0, v1, v2, v3);
}

// Fills v.m and (if grad) v.dm0..2; returns M = sum_i m_i (FP64).
//
// Quadrature rule.  In u = ln(t / tau) the integrand hh(u) is analytic in the
// strip |Im u| < pi / (alpha + beta) and grows at most like e^{kappa |u|},
// kappa = max(alpha + beta, beta + 1).  Panels of the full rule (order
// c.gl_order) are c.panel * 10 / kappa wide, clamped to [1, 8] x c.panel, so the
// ratio of singularity distance to half-width stays >= 2.5 and kappa x
// half-width <= 1.25: a relative error below 1e-8 per panel for order 6.  A bin
// that fits in one panel with kappa x half-width <= 0.25 uses 3 nodes, <= 0.04
// 2 nodes (relative error below 1e-8 by the same bounds).  Below x_min =
// ln tau + min(ln t_obs - ln tau, 0) - 22 / (beta + 1) the integrand is below
// e^-22 of its value at the peak or at t_obs, and the remaining mass (< 1e-9
// of the total) is dropped.
template <bool kPack = false>
__device__ __forceinline__ void sfh_bins_raw(const Consts& c, const AgeView& v, const float2* __restrict__ bins,
                                             float lnT, float tau, float alpha, float beta, bool grad) {
    PanelScratch& ps = *v.ps;
    const int lane = lane_id();
    const int A = c.n_age;
    const float lntau = __logf(tau);
    const float bp1 = beta + 1.0f;
    const float xmin = lntau + fminf(lnT - lntau, 0.0f) - 22.0f / bp1;
    const float kap = fmaxf(alpha + beta, bp1);
    const float pw = fminf(fmaxf(c.panel * 10.0f / kap, c.panel), 8.0f * c.panel);
    const float ipw = 1.0f / pw;
    const int G = c.gl_order;
    const int o2 = min(2, G), o3 = min(3, G);
    // Pass 1, bins i = lane + 32 k: panel layout; a bin that fits one panel is
    // integrated here, a bin of several panels is queued for pass 2.
    int base = 0;                               // panels queued so far (warp-uniform)
#pragma unroll 1
    for (int i0 = 0; i0 < A; i0 += 32) {
        const int i = i0 + lane;
        int n = 0;
        float x0 = 0.0f, hp = 0.0f;
        if (i < A) {
            const float2 b = bins[i];
            if (b.y < 0.0f) {                          // reaches t = 0
                const float w = b.x - xmin;
                if (w > 0.0f) {
                    n = panel_count(w * ipw);
                    hp = 0.5f * w * __frcp_rn((float)n);
                    x0 = xmin + hp;
                }
            } else if (b.y > 0.0f) {
                const float hi = b.x + b.y;
                const float lo = b.x - b.y;
                if (hi > xmin) {
                    if (lo < xmin) {
                        const float w = hi - xmin;
                        n = panel_count(w * ipw);
                        hp = 0.5f * w * __frcp_rn((float)n);
                        x0 = xmin + hp;
                    } else {                           // centre / half-width kept exact
                        n = panel_count(2.0f * b.y * ipw);
                        hp = b.y * __frcp_rn((float)n);
                        x0 = b.x + (float)(1 - n) * hp;
                    }
                }
            }
        }
        const float hk = hp * kap;
        const int ord = (n == 1) ? (hk <= 0.04f ? o2 : (hk <= 0.25f ? o3 : G)) : 0;
        const int oc = __reduce_max_sync(kFull, ord);
        float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
        if (oc > 0 && ord > 0) {
            const float xc = x0 - lntau;
            if (oc <= 2)
                gl_panel<2, kPack>(c.gl2_x, c.gl2_w, hp, xc, alpha, beta, grad, v0, v1, v2, v3);
            else if (oc == 3)
                gl_panel<3, kPack>(c.gl3_x, c.gl3_w, hp, xc, alpha, beta, grad, v0, v1, v2, v3);
            else if (oc == 6)
                gl_panel<6, kPack>(c.gl_x, c.gl_w, hp, xc, alpha, beta, grad, v0, v1, v2, v3);
            else
                gl_panel_any(G, c.gl_x, c.gl_w, hp, xc, alpha, beta, grad, v0, v1, v2, v3);
        }
        if (i < A) {
            v.m[i] = v0 * tau;
            if (grad) {
                v.dm0[i] = v1;
                v.dm1[i] = v2 * tau;
                v.dm2[i] = v3 * tau;
            }
        }
        // queue the panels of multi-panel bins: exclusive scan of their counts
        const int nq = (n >= 2) ? n : 0;
        int incl = nq;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        const int st = base + incl - nq;
        if (nq > 0) {
            ps.info[i] = make_float4(x0, hp, __int_as_float(st), 0.0f);
            if (st < kMaxPanels) ps.pmap[st] = (unsigned char)i;
        } else if (i < A) {
            ps.info[i].z = __int_as_float(-1);       // not queued in this call
        }
        base += __shfl_sync(kFull, incl, 31);
    }
    const int P = min(base, kMaxPanels);
    __syncwarp();
    // Pass 2: the queued panels, 32 per chunk, full rule; the panels of a bin
    // are consecutive and summed by a segmented scan.
    int carry = -1;
    for (int c0 = 0; c0 < P; c0 += 32) {
        const int p = c0 + lane;
        const bool act = p < P;
        // flag = bin index at a bin's first panel; the running max gives the bin
        int f = -1;
        if (act) {
            const int cand = ps.pmap[p];
            if (cand < A && __float_as_int(ps.info[cand].z) == p) f = cand;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, f, o);
            if (lane >= o) f = max(f, t);
        }
        f = max(f, carry);
        carry = __shfl_sync(kFull, f, 31);
        const int bin = (act && f >= 0) ? f : -1;
        float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
        if (bin >= 0) {
            const float4 inf = ps.info[bin];
            const float hp = inf.y;
            const float xc = inf.x + 2.0f * (float)(p - __float_as_int(inf.z)) * hp - lntau;
            if (G == 6)
                gl_panel<6, kPack>(c.gl_x, c.gl_w, hp, xc, alpha, beta, grad, v0, v1, v2, v3);
            else
                gl_panel_any(G, c.gl_x, c.gl_w, hp, xc, alpha, beta, grad, v0, v1, v2, v3);
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float t0 = __shfl_up_sync(kFull, v0, o);
            const float t1 = __shfl_up_sync(kFull, v1, o);
            const float t2 = __shfl_up_sync(kFull, v2, o);
            const float t3 = __shfl_up_sync(kFull, v3, o);
            const int bo = __shfl_up_sync(kFull, bin, o);
            if (lane >= o && bo == bin) {
                v0 += t0; v1 += t1; v2 += t2; v3 += t3;
            }
        }
        const int bnext = __shfl_down_sync(kFull, bin, 1);
        if (bin >= 0 && (lane == 31 || bnext != bin)) {
            v.m[bin] += v0 * tau;
            if (grad) {
                v.dm0[bin] += v1;
                v.dm1[bin] += v2 * tau;
                v.dm2[bin] += v3 * tau;
            }
        }
        __syncwarp();
    }
}

// This lane's FP64 partial of M = sum_i m_i (the cumulative mass integral);
// warp_sum_d of it gives M.
// The lane's (at most 4) bins are summed in FP32 with two-sum error terms, so
// hi + lo carries their sum to ~2^-47; the FP64 accumulation starts from it.
__device__ __forceinline__ double mass_partial(const Consts& c, const AgeView& v) {
    float hi = 0.0f, lo = 0.0f;
#pragma unroll 4
    for (int i = lane_id(); i < c.n_age; i += 32) {
        const float x = v.m[i];
        const float sum = hi + x;
        const float bp = sum - hi;
        lo += (hi - (sum - bp)) + (x - bp);       // Knuth two-sum error term
        hi = sum;
    }
    return (double)hi + (double)lo;
}

__device__ __forceinline__ double sfh_bins(const Consts& c, const AgeView& v, const float2* __restrict__ bins,
                                           float lnT, float tau, float alpha, float beta, bool grad) {
    sfh_bins_raw(c, v, bins, lnT, tau, alpha, beta, grad);
    return warp_sum_d(mass_partial(c, v));
}

// ---------------------------------------------------------------- burst + MDF
// Burst weights pi_i = (T(x_{i+1}) - T(x_i)) / D over the log-age edges
// clipped at t_obs, T the triweight CDF.  Each lane evaluates the CDF at one
// edge; the lower edge of a bin comes from the neighbouring lane.
__device__ __forceinline__ float burst_weights(const Consts& c, const AgeView& v, float lT10,
                                               float mu, float sig) {
    const int lane = lane_id();
    const int A = c.n_age;
    const float isig = 1.0f / sig;
    const float D = tri_cdf((lT10 - mu) * isig);
    const float invD = 1.0f / D;
    float carry = 0.0f;                          // CDF at the last edge of the previous group
#pragma unroll 1
    for (int e0 = 0; e0 <= A; e0 += 32) {
        const int e = e0 + lane;
        const float F = (e <= A) ? tri_cdf((fminf(v.age_edge[e], lT10) - mu) * isig) : 0.0f;
        float Fl = __shfl_up_sync(kFull, F, 1);
        if (lane == 0) Fl = carry;
        if (e >= 1 && e <= A) v.pi[e - 1] = (F - Fl) * invD;
        carry = __shfl_sync(kFull, F, 31);
    }
    return D;
}

// Metallicity weights q_j = Phi(y_{j+1}) - Phi(y_j), y = (edge - mu) / sd.
// Each lane takes one edge and the smaller tail T = Phi(-|y|) there, so that a
// bin in either tail is a difference of small numbers.
__device__ __forceinline__ void met_weights(const Consts& c, const AgeView& v, float mu, float sd) {
    const int e = lane_id();
    const int Zn = c.n_met;
    const float isd = 1.0f / sd;
    float T = 0.0f;
    bool pos = false;
    if (e <= Zn) {
        const float y = (v.lgz_edge[e] - mu) * isd;
        T = 0.5f * erfcf(fabsf(y) * 0.70710678118654752f);
        pos = y >= 0.0f;
    }
    float Th = __shfl_down_sync(kFull, T, 1);
    bool ph = __shfl_down_sync(kFull, pos ? 1 : 0, 1) != 0;
    if (e == Zn - 1) {                           // the top edge is +inf
        Th = 0.0f;
        ph = true;
    }
    if (e < Zn) v.q[e] = pos ? (T - Th) : (ph ? (1.0f - Th) - T : Th - T);
}

// ---------------------------------------------------------------- non-separable MDF
// With c.mdf_age the MDF of age bin i has mean mu_i = lgZ + c.mdf_off[i] and
// the common width sigma: q_ij = Phi(y_{i,j+1}) - Phi(y_ij), y = (edge - mu_i)
// / sigma, so W_ij = w_i q_ij is a general [A x Zn] matrix.  One lane takes
// one age row and walks its edges, each cell from the smaller tails at its two
// edges (as met_weights).
__device__ __forceinline__ void mdf_edge(const float* __restrict__ lgz_edge, int e, float mu, float isd,
                                         float& y, float& T, bool& pos) {
    y = (lgz_edge[e] - mu) * isd;
    T = 0.5f * erfcf(fabsf(y) * 0.70710678118654752f);
    pos = y >= 0.0f;
}
__device__ __forceinline__ float mdf_cell(float Tl, bool pl, float Th, bool ph) {
    return pl ? (Tl - Th) : (ph ? (1.0f - Th) - Tl : Th - Tl);
}

// qm[i * Zn + j] = q_ij for every age row (lanes over rows).
__device__ __forceinline__ void mdf_rows_fill(const Consts& c, const float* __restrict__ lgz_edge, float mz,
                                              float sz, float* __restrict__ qm) {
    const int Zn = c.n_met;
    const float isd = 1.0f / sz;
    for (int i = lane_id(); i < c.n_age; i += 32) {
        const float mu = mz + c.mdf_off[i];
        float y, Tl, Th;
        bool pl, ph;
        mdf_edge(lgz_edge, 0, mu, isd, y, Tl, pl);
#pragma unroll 1
        for (int j = 0; j < Zn; ++j) {
            mdf_edge(lgz_edge, j + 1, mu, isd, y, Th, ph);
            qm[i * Zn + j] = mdf_cell(Tl, pl, Th, ph);
            Tl = Th;
            pl = ph;
        }
    }
    __syncwarp();
}

__device__ __forceinline__ float phi_(float y);
__device__ __forceinline__ float phi_y(float y);

// Adjoint through the non-separable MDF.  vbuf[i * Zn + j] holds dlogL/dW'_ij
// for W'_ij = w_i q_ij: writes wb_i = sum_j v_ij q_ij and adds
// dlogL/d(lgZ, sigma) = sum_i (1/sigma) sum_e (phi_e, y_e phi_e)(qb_ie - qb_i,e-1),
// qb_ij = w_i v_ij, into g[7], g[8] (warp-uniform).  The MDF part of
// age_met_adjoint must then see qb = 0.
__device__ __forceinline__ void mdf_rows_adjoint(const Consts& c, const AgeView& v, const float* __restrict__ vbuf,
                                                 float mz, float sz, float* g) {
    const int Zn = c.n_met;
    const float isd = 1.0f / sz;
    float gz = 0.0f, gs = 0.0f;
    for (int i = lane_id(); i < c.n_age; i += 32) {
        const float mu = mz + c.mdf_off[i];
        const float wi = v.w[i];
        const float* vr = vbuf + i * Zn;
        float y, Tl, Th;
        bool pl, ph;
        mdf_edge(v.lgz_edge, 0, mu, isd, y, Tl, pl);
        float a = 0.0f, vprev = 0.0f;
#pragma unroll 1
        for (int e = 0; e <= Zn; ++e) {
            if (e > 0) mdf_edge(v.lgz_edge, e, mu, isd, y, Th, ph);
            const float ve = (e < Zn) ? vr[e] : 0.0f;
            if (e > 0) {
                a = fmaf(vprev, mdf_cell(Tl, pl, Th, ph), a);
                Tl = Th;
                pl = ph;
            }
            const float d = wi * (ve - vprev);
            gz = fmaf(phi_(y), d, gz);
            gs = fmaf(phi_y(y), d, gs);
            vprev = ve;
        }
        v.wb[i] = a;
    }
    gz = warp_sum(gz);
    gs = warp_sum(gs);
    if (lane_id() < Zn) v.qb[lane_id()] = 0.0f;
    __syncwarp();
    g[7] += gz * isd;
    g[8] += gs * isd;
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

// Eq. BoundingFunction for parameter k: theta = lo + span / (1 + exp(-k_s (x - x0))).
__device__ __forceinline__ float bound_theta(const Consts& c, int k, float x) {
    return c.prior_lo[k] + c.prior_span[k] * sigmoidf_(c.sig_k[k] * (x - c.sig_x0[k]));
}

// Eq. BoundingFunction for parameter k with its derivative, and the log prior
// density of x with its derivative: uniform in theta (log of the Jacobian,
// log s (1 - s), constant log(k_s span) dropped), or the skew-normal of Eq.
// SkewNormPrior on x, log(2/omega) + log N(u) + log Phi(s u), u = (x - xi) /
// omega.  log Phi(z) and phi(z) / Phi(z) for z < 0 through the scaled
// complementary error function: Phi(z) = erfcx(-z/sqrt2) e^{-z^2/2} / 2.
__device__ __forceinline__ void bound_prior(const Consts& c, int k, float x, float& th, float& dth, float& lpe,
                                            float& dlpe) {
    const float ks = c.sig_k[k];
    const float y = ks * (x - c.sig_x0[k]);
    const float ey = __expf(-fabsf(y));
    const float r = __frcp_rn(1.0f + ey);
    const float sg = (y >= 0.0f) ? r : ey * r;              // 1 / (1 + e^-y)
    th = c.prior_lo[k] + c.prior_span[k] * sg;
    dth = c.prior_span[k] * ks * sg * (1.0f - sg);
    if (c.prior_kind == SPS_PRIOR_SKEWNORMAL) {
        const float u = (x - c.sn_xi[k]) * c.sn_iom[k];
        const float z = c.sn_s[k] * u;
        float lphi, ratio;
        if (z < 0.0f) {
            const float e = erfcxf(-z * 0.70710678f);
            lphi = __logf(0.5f * e) - 0.5f * z * z;
            ratio = 0.79788456f / e;                             // sqrt(2 / pi) / erfcx
        } else {
            const float q = 0.5f * erfcf(z * 0.70710678f);      // 1 - Phi(z)
            lphi = log1pf(-q);
            ratio = 0.39894228f * __expf(-0.5f * z * z) / (1.0f - q);
        }
        lpe = c.sn_c[k] - 0.5f * u * u + lphi;
        dlpe = (c.sn_s[k] * ratio - u) * c.sn_iom[k];
    } else {
        lpe = -fabsf(y) - 2.0f * log1pf(ey);
        dlpe = ks * (1.0f - 2.0f * sg);
    }
}

// Parameters of one row held uniformly by the warp.
struct RowParams {
    float th[SPS_NPARAM];
    float dth[SPS_NPARAM];   // d theta / d x (unbounded input) or 1
    float dlp[SPS_NPARAM];   // d log prior / d x (unbounded input) or 0
    double logprior;         // log prior density of x (unbounded input) or 0
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
            float lpe;
            bound_prior(c, k, x, p.th[k], p.dth[k], lpe, p.dlp[k]);
            p.logprior += (double)lpe;
        } else {
            p.th[k] = x;
            p.dth[k] = 1.0f;
            p.dlp[k] = 0.0f;
        }
    }
}

// ---------------------------------------------------------------- weights stage
// Bin integrals, burst and metallicity weights (everything but M and w).
template <bool kPack = false>
__device__ __forceinline__ void age_met_parts(const Consts& c, const AgeView& v, const float2* __restrict__ bins,
                                              float lnT, float lT10, const float* th, bool grad) {
    sfh_bins_raw<kPack>(c, v, bins, lnT, th[1], th[2], th[3], grad);
    burst_weights(c, v, lT10, th[5], th[6] * (1.0f / 3.0f));
    met_weights(c, v, th[7], th[8]);
}
// w_i = (1 - F_burst) m_i + F_burst pi_i M.
__device__ __forceinline__ void age_weights(const Consts& c, const AgeView& v, const float* th, double M) {
    __syncwarp();
    const float fb = th[4];
    const float Mf = (float)M;
#pragma unroll 4
    for (int i = lane_id(); i < c.n_age; i += 32) v.w[i] = (1.0f - fb) * v.m[i] + fb * v.pi[i] * Mf;
    __syncwarp();
}
// Fills v.m/dm, v.pi, v.q, v.w for parameters th[12]; returns M (FP64).
__device__ __forceinline__ double age_met_weights(const Consts& c, const AgeView& v,
                                                  const float2* __restrict__ bins, float lnT,
                                                  float lT10, const float* th, bool grad) {
    age_met_parts(c, v, bins, lnT, lT10, th, grad);
    __syncwarp();
    const double M = warp_sum_d(mass_partial(c, v));
    age_weights(c, v, th, M);
    return M;
}
__device__ __forceinline__ double age_met_weights(const Consts& c, RowScratch& s,
                                                  const float2* __restrict__ bins, float lnT,
                                                  float lT10, const RowParams& p, bool grad) {
    return age_met_weights(c, s.view(c), bins, lnT, lT10, p.th, grad);
}

// Adjoint of age_met_weights: given s.wb (dlogL/dw_i) and s.qb (dlogL/dq_j)
// returns d/dtheta for columns 1-8 added into g[].  Every bin sum is taken in
// one pass and reduced in one round:
//   mbar_l = (1 - F_b) wbar_l + F_b sum_i wbar_i pi_i   (smooth SFH)
//   pibar_i = F_b M wbar_i                               (burst, through pi = raw / D)
//   F_b-bar = sum_i wbar_i (pi_i M - m_i)
__device__ __forceinline__ void age_met_adjoint(const Consts& c, const AgeView& s, float lT10, double M,
                                                const float* th, float* g) {
    const int lane = lane_id();
    const int A = c.n_age;
    const float fb = th[4];
    const float Mf = (float)M;
    const float mu = th[5], sig = th[6] * (1.0f / 3.0f);
    const float isig = 1.0f / sig;
    float s_wp = 0.f, s_wm = 0.f, s_w0 = 0.f, s_w1 = 0.f, s_w2 = 0.f;
    float s_d0 = 0.f, s_d1 = 0.f, s_d2 = 0.f, s_mu = 0.f, s_sg = 0.f;
#pragma unroll 4
    for (int i = lane; i < A; i += 32) {
        const float wb = s.wb[i];
        const float d0 = s.dm0[i], d1 = s.dm1[i], d2 = s.dm2[i];
        s_wp = fmaf(wb, s.pi[i], s_wp);
        s_wm = fmaf(wb, s.m[i], s_wm);
        s_w0 = fmaf(wb, d0, s_w0);
        s_w1 = fmaf(wb, d1, s_w1);
        s_w2 = fmaf(wb, d2, s_w2);
        s_d0 += d0;
        s_d1 += d1;
        s_d2 += d2;
    }
    // burst, edge by edge: sum_i wbar_i (T(x_i) - T(x_{i+1})) = sum_e T(x_e) (wbar_e - wbar_{e-1})
#pragma unroll 1
    for (int e = lane; e <= A; e += 32) {
        const float x = (fminf(s.age_edge[e], lT10) - mu) * isig;
        const float d = ((e < A) ? s.wb[e] : 0.0f) - ((e > 0) ? s.wb[e - 1] : 0.0f);
        const float tp = tri_pdf(x) * d;
        s_mu += tp;
        s_sg = fmaf(x, tp, s_sg);
    }
    // metallicity: q_j = Phi(y_{j+1}) - Phi(y_j), edge by edge
    const float mz = th[7], sz = th[8];
    const float isz = 1.0f / sz;
    float s_gz = 0.f, s_gs = 0.f;
    if (lane <= c.n_met) {
        const float y = (s.lgz_edge[lane] - mz) * isz;
        const float d = ((lane < c.n_met) ? s.qb[lane] : 0.0f) - ((lane > 0) ? s.qb[lane - 1] : 0.0f);
        s_gz = phi_(y) * d;
        s_gs = phi_y(y) * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s_wp += __shfl_xor_sync(kFull, s_wp, o);
        s_wm += __shfl_xor_sync(kFull, s_wm, o);
        s_w0 += __shfl_xor_sync(kFull, s_w0, o);
        s_w1 += __shfl_xor_sync(kFull, s_w1, o);
        s_w2 += __shfl_xor_sync(kFull, s_w2, o);
        s_d0 += __shfl_xor_sync(kFull, s_d0, o);
        s_d1 += __shfl_xor_sync(kFull, s_d1, o);
        s_d2 += __shfl_xor_sync(kFull, s_d2, o);
        s_mu += __shfl_xor_sync(kFull, s_mu, o);
        s_sg += __shfl_xor_sync(kFull, s_sg, o);
        s_gz += __shfl_xor_sync(kFull, s_gz, o);
        s_gs += __shfl_xor_sync(kFull, s_gs, o);
    }
    const float omf = 1.0f - fb, fa = fb * s_wp;
    g[1] += omf * s_w0 + fa * s_d0;
    g[2] += omf * s_w1 + fa * s_d1;
    g[3] += omf * s_w2 + fa * s_d2;
    g[4] += Mf * s_wp - s_wm;
    // burst: d raw_i/d mu = -(T(xh) - T(xl)) / sig, dD/dmu = -T(xT) / sig; x T(x) for sigma
    const float xT = (lT10 - mu) * isig;
    const float D = tri_cdf(xT);
    const float tT = tri_pdf(xT);
    const float k = fb * Mf / (sig * D);
    g[5] += k * (s_mu + s_wp * tT);
    g[6] += k * (s_sg + s_wp * xT * tT) * (1.0f / 3.0f);
    g[7] += s_gz * isz;
    g[8] += s_gs * isz;
}
__device__ inline void age_met_adjoint(const Consts& c, RowScratch& s, float lT10, double M,
                                       const RowParams& p, float* g) {
    age_met_adjoint(c, s.view(c), lT10, M, p.th, g);
}

// ---------------------------------------------------------------- redshift through t_obs
// SFR shape of Eq. SFRsmooth at ln t (t in Gyr): [(t/tau)^alpha + (t/tau)^-beta]^-1,
// written as exp(beta v - softplus((alpha + beta) v)), v = ln(t / tau).
__device__ __forceinline__ float sfr_shape_ln(float lnt, float ltau, float alpha, float beta) {
    const float v = lnt - ltau;
    const float x = (alpha + beta) * v;
    const float sp = fmaxf(x, 0.0f) + log1pf(__expf(-fabsf(x)));
    return __expf(beta * v - sp);
}

// sum_i wbar_i d w_i / d t_obs (t_obs in Gyr), given s.wb (dlogL/dw_i) and the
// weights of age_met_weights, w_i = (1 - F_b) m_i + F_b pi_i M.  The bin
// integrals m_i run over [t_obs - E_{i+1}, t_obs - E_i], so d m_i / d t_obs is
// the SFR shape at the upper limit minus that at the lower one (a limit pinned
// at t = 0 does not move); M = sum m_i moves by the shape at t_obs.  The burst
// edges are clipped at lT = log10 t_obs: with x_T = (lT - mu) / sigma and
// D = T(x_T), d pi_i / d lT = t(x_T) / (sigma D) ([i holds t_obs] - pi_i).
// Bins are (centre c, half-width hw) in ln t; (ln t_hi, -1) reaches t = 0;
// (0, 0) is empty.  The youngest bins are ~1e-5 wide in ln t, so forming
// c +- hw in FP32 would lose most of the difference of the two shapes; it is
// taken instead around the centre, h(c + s) / h(c) = exp(a(s)) with
// a(s) = beta s - log1p(expm1(k s) sigma(k v)), k = alpha + beta, v = c - ln tau
// (the softplus difference written exactly), so the difference is
// h(c) (expm1(a(hw)) - expm1(a(-hw))).  Returns the warp-uniform sum.
__device__ __forceinline__ float tobs_adjoint(const Consts& c, const AgeView& s, const float2* __restrict__ bins,
                                              float lnT, float lT10, double M, const float* th) {
    const int lane = lane_id();
    const float ltau = __logf(th[1]), al = th[2], be = th[3], fb = th[4];
    float s_m = 0.0f, s_p = 0.0f, wT = 0.0f;
    for (int i = lane; i < c.n_age; i += 32) {
        const float2 b = bins[i];
        const float wb = s.wb[i];
        float dm = 0.0f;
        if (b.y > 0.0f) {
            const float kk = al + be;
            if (kk * b.y < 20.0f) {
                const float sg = 1.0f / (1.0f + __expf(-kk * (b.x - ltau)));
                const float ap = be * b.y - log1pf(expm1f(kk * b.y) * sg);
                const float am = -be * b.y - log1pf(expm1f(-kk * b.y) * sg);
                dm = sfr_shape_ln(b.x, ltau, al, be) * (expm1f(ap) - expm1f(am));
            } else {            // a wide bin: no cancellation in the plain difference
                dm = sfr_shape_ln(b.x + b.y, ltau, al, be) - sfr_shape_ln(b.x - b.y, ltau, al, be);
            }
        } else if (b.y < 0.0f) {
            dm = sfr_shape_ln(b.x, ltau, al, be);
            wT = wb;
        }
        s_m = fmaf(wb, dm, s_m);
        s_p = fmaf(wb, s.pi[i], s_p);
    }
    s_m = warp_sum(s_m);
    s_p = warp_sum(s_p);
    wT = warp_sum(wT);
    const float sig = th[6] * (1.0f / 3.0f);
    const float xT = (lT10 - th[5]) / sig;
    const float D = tri_cdf(xT);
    const float dlT = 1.0f / (__expf(lnT) * kLn10f);              // d lT / d t_obs
    const float dpi = tri_pdf(xT) / (sig * D) * dlT;
    const float shT = sfr_shape_ln(lnT, ltau, al, be);
    return (1.0f - fb) * s_m + fb * (shT * s_p + (float)M * dpi * (wT - s_p));
}

}  // namespace sps
