// Warp-level evaluation of one (galaxy, chain) row on the approximate path
// (Eq. photo_integral_approx) with its Gaussian log-likelihood (App. D.1)
// and hand-written adjoint gradient.  Shared by the row kernel and the
// persistent HMC kernel; the c_SSP rows of the bands being evaluated are
// reached through generic pointers (global memory or shared memory).
#pragma once

#include "sps_device.cuh"

namespace sps {

struct SlotData {
    const float* ptr[kMaxBands];   // c_SSP row of the band in slot s ([K])
    float4 dust[kMaxBands];        // dust constants at lambda_eff
    double zp[kMaxBands];          // AB zero point
    float mobs[kMaxBands];
    float isig2[kMaxBands];
    int band[kMaxBands];
    double mag[kMaxBands];
};

struct WarpWork {
    RowScratch r;
    SlotData d;
};

// Fill the slot table of galaxy gi for the bands set in `bits` (lane-parallel).
__device__ __forceinline__ int fill_slots(const Consts& c, const Galaxies& g, SlotData& d,
                                          int64_t gi, uint32_t bits, const float* mag_obs,
                                          const float* sigma, const float* cssp_base,
                                          bool compact_table) {
    const int lane = lane_id();
    const int B = c.n_band;
    const int nb = __popc(bits);
    if (lane < B && ((bits >> lane) & 1u)) {
        int slot = __popc(bits & ((1u << lane) - 1u));
        size_t gb = (size_t)gi * B + lane;
        d.band[slot] = lane;
        d.ptr[slot] = compact_table ? cssp_base + (size_t)slot * c.K : cssp_base + (size_t)lane * c.K;
        d.dust[slot] = g.dust_eff[gb];
        d.zp[slot] = g.zp[gb];
        if (mag_obs) {
            float sg = sigma[gb];
            d.mobs[slot] = mag_obs[gb];
            d.isig2[slot] = 1.0f / (sg * sg);
        }
    }
    __syncwarp();
    return nb;
}

// Per-galaxy redshift derivatives for the z column (kZ): d c_SSP / dz rows,
// d zp / dz, the dust constants' d/dz at lambda_eff, and d t_obs / dz.
struct ZRow {
    const float* dcssp;     // [B][K]
    const float* dzp;       // [B]
    const float4* ddust;    // [B]
    float dtdz;
};

// Evaluate one row.  Returns log L (FP64, warp-uniform; 0 if !like), writes
// d.mag[slot] (FP64) and, if grad, the physical-parameter gradient into g[12]
// (warp-uniform).  kZ (with like and grad): also d log L / dz into g[12] (13
// entries), the explicit part (filter, zero point, lambda_eff, c_SSP(z)) plus
// the part through t_obs(z) (age bins, M, burst clipping).
template <bool kZ = false>
__device__ inline double eval_row(const Consts& c, WarpWork& ww, const float2* __restrict__ bins,
                           float lnT, float lT10, const RowParams& p, int nb, bool like,
                           bool grad, float* gout, const ZRow* zr = nullptr) {
    RowScratch& s = ww.r;
    SlotData& d = ww.d;
    const int lane = lane_id();
    const int K = c.K, Zn = c.n_met, A = c.n_age;
    const double M = age_met_weights(c, s, bins, lnT, lT10, p, grad);

    // W_ij / (1e9 10^lgM) = w_i q_j, one register tile per lane (k = lane + 32 t);
    // with an age-dependent MDF, w_i q_ij with q_ij staged in kbuf
    const bool nonsep = c.mdf_age != 0;
    if (nonsep) mdf_rows_fill(c, c.lgz_edge, p.th[7], p.th[8], s.u.kbuf);
    float wreg[kKTileMax];
#pragma unroll
    for (int t = 0; t < kKTileMax; ++t) {
        int k = lane + 32 * t;
        wreg[t] = (k < K) ? s.w[k / Zn] * (nonsep ? s.u.kbuf[k] : s.q[k % Zn]) : 0.0f;
    }
    __syncwarp();
    for (int sl = 0; sl < nb; ++sl) {
        const float* C = d.ptr[sl];
        float a = 0.0f;
#pragma unroll
        for (int t = 0; t < kKTileMax; ++t) {
            int k = lane + 32 * t;
            if (k < K) a = fmaf(wreg[t], C[k], a);
        }
        a = warp_sum(a);
        if (lane == 0) s.slot_S[sl] = a;
        if (kZ) {
            const float* Cd = zr->dcssp + (size_t)d.band[sl] * K;
            float b = 0.0f;
#pragma unroll
            for (int t = 0; t < kKTileMax; ++t) {
                int k = lane + 32 * t;
                if (k < K) b = fmaf(wreg[t], Cd[k], b);
            }
            b = warp_sum(b);
            if (lane == 0) s.slot_D[sl] = b;
        }
    }
    __syncwarp();

    double ll = 0.0;
    float gam = 0.0f;
    float gz = 0.0f;             // kZ: this band's explicit d log L / dz
    DustTerms dt{1.f, 0.f, 0.f, 0.f};
    float S = 1.0f;
    if (lane < nb) {
        float4 dc = d.dust[lane];
        dt = dust_eval(dc.x, dc.y, dc.z, p.th[9], p.th[10], p.th[11]);
        S = s.slot_S[lane];
        double lc = log10_flux(dt.F * S) + (double)p.th[0] + 9.0;
        double m = d.zp[lane] - 2.5 * lc;
        d.mag[lane] = m;
        if (like) {
            double r = m - (double)d.mobs[lane];
            double is2 = (double)d.isig2[lane];
            ll = -0.5 * r * r * is2;
            gam = (float)(2.5 * r * is2 / 2.302585092994046);
            if (kZ) {
                // m = zp - 2.5 log10(F S ...): dlogL/dm = -r is2, dlogL/dln c = gam;
                // dF/dz through the dust curve at lambda_eff(z)
                const int band = d.band[lane];
                const float4 dd = zr->ddust[band];
                const float AV = p.th[9], dl = p.th[10], ff = p.th[11];
                const float eb = fmaxf(0.85f - 1.9f * dl, 0.0f);
                const float pw = __expf(dl * dc.y);
                const float E = exp2f(-0.4f * kLog2_10f * AV * (1.0f / 4.05f) * (dc.x * pw + eb * dc.z));
                const float dA = AV * (1.0f / 4.05f) * (dd.x * pw + dc.x * pw * dl * dd.y + eb * dd.z);
                const float dF = (1.0f - ff) * E * (-0.4f * kLn10f) * dA;
                gz = (float)(-r * is2) * zr->dzp[band] + gam * (dF / dt.F + s.slot_D[lane] / S);
            }
        }
    }
    ll = warp_sum_d(ll);
    if (!grad) {
        __syncwarp();
        return ll;
    }
    // d/dlgM and dust gradients: c_b = 1e9 10^lgM F_b S_b
    float g0 = gam * kLn10f;
    float gF = (lane < nb) ? gam / dt.F : 0.0f;
    float gAV = gF * dt.dF_AV, gdl = gF * dt.dF_delta, gff = gF * dt.dF_floor;
    if (lane < nb) s.slot_g[lane] = gam / S;
    g0 = warp_sum(g0);
    gAV = warp_sum(gAV);
    gdl = warp_sum(gdl);
    gff = warp_sum(gff);
    __syncwarp();
    // v_k = sum_b (gamma_b / S_b) c_SSP[b][k]
#pragma unroll 4
    for (int t = 0; t < kKTileMax; ++t) {
        int k = lane + 32 * t;
        if (k < K) {
            float v = 0.0f;
            for (int sl = 0; sl < nb; ++sl) v = fmaf(s.slot_g[sl], d.ptr[sl][k], v);
            s.u.kbuf[k] = v;
        }
    }
    __syncwarp();
    float g[SPS_NPARAM];
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) g[k] = 0.0f;
    g[0] = g0;
    g[9] = gAV;
    g[10] = gdl;
    g[11] = gff;
    if (nonsep) {
        mdf_rows_adjoint(c, s.view(c), s.u.kbuf, p.th[7], p.th[8], g);
    } else {
        for (int i = lane; i < A; i += 32) {
            float a = 0.0f;
            const float* vr = s.u.kbuf + i * Zn;
            for (int j = 0; j < Zn; ++j) a = fmaf(vr[j], s.q[j], a);
            s.wb[i] = a;
        }
        if (lane < Zn) {
            float a = 0.0f;
            for (int i = 0; i < A; ++i) a = fmaf(s.u.kbuf[i * Zn + lane], s.w[i], a);
            s.qb[lane] = a;
        }
        __syncwarp();
    }
    age_met_adjoint(c, s, lT10, M, p, g);
#pragma unroll
    for (int k = 0; k < SPS_NPARAM; ++k) gout[k] = g[k];
    if (kZ) {
        gz = warp_sum(gz);
        gout[SPS_NPARAM] = gz + zr->dtdz * tobs_adjoint(c, s.view(c), bins, lnT, lT10, M, p.th);
    }
    __syncwarp();
    return ll;
}

}  // namespace sps
