// Batched HMC on the approximate path with the chains of one galaxy in lock
// step on one warp (Sec. 4, App. D.2).
//
// A warp ("team") takes up to kCPW chains of one galaxy from a global work
// queue (atomic counter, no waiting) and advances all of them one gradient
// evaluation per step.  Chains stay trajectory-asynchronous: each has its own
// trajectory length, step size, inverse metric and iteration count, and ends
// and restarts its trajectories on its own; a chain that has finished keeps
// its last position until the team's other chains are done.  The contraction
// with the galaxy's c_SSP table is organised by age bin: every table row
// c_SSP[b][i][0..Zn) is loaded once and used by all chains of the team for
// R = sum_j q_j C_ij (forward), and again in the adjoint pass for
// wbar_i += g_b R and qbar_j += g_b w_i C_ij.  Warps never wait on one another.
//
// Sampler (same definition as the per-chain kernel): p = z / sqrt(minv),
// leapfrog (half kick, drift x += eps minv p, gradient, half kick), FP64
// energy accept, dual-averaged step size and windowed diagonal metric in the
// warm-up, Philox-4x32-10 draws with counter (iteration, block, chain, 0).
#include <algorithm>

#include "philox.cuh"
#include "sps_device.cuh"

namespace sps {

namespace {

constexpr int kZnReg = 12;   // metallicity bins held in registers (Zn <= 12)

template <int CPW>
struct TeamWork {
    float m[CPW][kMaxAges], dm0[CPW][kMaxAges], dm1[CPW][kMaxAges], dm2[CPW][kMaxAges];
    float pi[CPW][kMaxAges];
    float w[CPW][kMaxAges];                 // age weights; their adjoint overwrites them
    float q[CPW][kMaxMets], qb[CPW][kMaxMets];
    union {
        PanelScratch ps;
        float red[32][kZnReg + 1];          // qbar partials of one chain
        struct {                            // per (chain, band) of the contraction
            float F[CPW][kMaxBands];        // dust factor at lambda_eff
            float Ah[CPW][kMaxBands], Al[CPW][kMaxBands];   // zp - m_obs - 2.5 (lgM + 9), hi + lo
            float res[CPW][kMaxBands], gam[CPW][kMaxBands]; // residual m - m_obs, dlogL / dln c
            float gh[CPW][kMaxBands];                       // gamma_b / S_b (age-dependent MDF pass)
        } t;
    } u;
    float th[CPW][SPS_NPARAM], dth[CPW][SPS_NPARAM];
    float lpe[CPW][SPS_NPARAM];             // log prior terms, then their x-derivatives
    double M[CPW], lpri[CPW], ll[CPW];
    float gd[CPW][4];                       // d logL / d(lgM, A_V, delta, F_floor)
    // galaxy slots
    float2 bins[kMaxAges];                  // age bins of the galaxy (centre, half-width in ln t)
    float lnT, lT10;                        // ln t_obs [Gyr], log10 t_obs [yr]
    const float* ptr[kMaxBands];
    float4 dust[kMaxBands];
    double zp[kMaxBands];
    float mobs[kMaxBands], isig2[kMaxBands];
    // chain state
    float x[CPW][SPS_NPARAM], p[CPW][SPS_NPARAM], g[CPW][SPS_NPARAM];
    float xs[CPW][SPS_NPARAM], gs[CPW][SPS_NPARAM], minv[CPW][SPS_NPARAM];
    double lp[CPW], lps[CPW], h0[CPW];
    float mu[CPW], hbar[CPW], leb[CPW], acc[CPW];   // dual averaging, accept sum
    ChainMetric* cm[CPW];                   // metric-adaptation state (global memory)
    float v[CPW][SPS_NPARAM], lu[CPW][SPS_NPARAM], dv[CPW][2][SPS_NPARAM];
    double uacc[CPW];                       // log of the accept uniform
    float eps[CPW];
    int L[CPW], l[CPW], it[CPW], mda[CPW], wn[CPW], ndiv[CPW], done[CPW];
    int wstart[CPW], wend[CPW], wwidth[CPW], wstop[CPW];
    long long nev[CPW];
    uint32_t chain[CPW];
    // NUTS: log weights of the trajectory and of the subtree (relative to
    // exp(-H0)), statistic sum, leaves built, subtree depth, leaf index in the
    // subtree, direction, the subtree's acceptance uniform
    float lw[CPW], lws[CPW], nacc[CPW], utree[CPW];
    int nleaf[CPW], nj[CPW], nn[CPW], dir[CPW];
    float nS[CPW][SPS_NPARAM];              // momentum prefix sum of the subtree
    float nu[CPW][32];                      // uniforms of the subtree's next 32 leaves
};

// Age and metallicity bin edges of the tables, staged once per block.
struct EdgeTables {
    float age[kMaxAges + 1];
    float lgz[kMaxMets + 1];
};

template <int CPW>
__device__ __forceinline__ AgeView age_view(TeamWork<CPW>& t, int ch, const EdgeTables& et) {
    return AgeView{t.m[ch], t.dm0[ch], t.dm1[ch], t.dm2[ch], t.pi[ch], t.w[ch], t.w[ch],
                   t.q[ch], t.qb[ch], &t.u.ps, et.age, et.lgz};
}

// Row i of a band's c_SSP table: Zn consecutive floats.
__device__ __forceinline__ void load_row(const float* __restrict__ p, int Zn, float* cv) {
    if (Zn == 12) {
        const float4* v = reinterpret_cast<const float4*>(p);
        float4 a = v[0], b = v[1], c = v[2];
        cv[0] = a.x; cv[1] = a.y; cv[2] = a.z; cv[3] = a.w;
        cv[4] = b.x; cv[5] = b.y; cv[6] = b.z; cv[7] = b.w;
        cv[8] = c.x; cv[9] = c.y; cv[10] = c.z; cv[11] = c.w;
    } else {
#pragma unroll
        for (int j = 0; j < kZnReg; ++j) cv[j] = (j < Zn) ? p[j] : 0.0f;
    }
}

// log posterior (unbounded space) and its gradient for every chain of the
// team at t.x; writes t.lp and t.g.
// kNonsep (one chain per warp): the MDF mean depends on the age bin, so q is
// a matrix qm[i * Zn + j] (shared memory, filled here); the forward takes
// R_i = sum_j q_ij C_bij and S_b = sum_i w_i R_i, and a second pass over the
// c_SSP rows forms V_ij = sum_b g_b C_bij for the MDF gradient (qbar_ij =
// w_i V_ij through the edge pdfs of each row).
template <int CPW, bool kPhys = false, bool kNonsep = false>
__device__ __forceinline__ void team_eval(const Consts& c, TeamWork<CPW>& t, const EdgeTables& et,
                                          float lnT, float lT10, int nb, float* __restrict__ qm = nullptr) {
    static_assert(!kNonsep || CPW == 1, "the age-dependent MDF takes one chain per warp");
    const int lane = lane_id();
    const int A = c.n_age, Zn = c.n_met;
    float dlp[(CPW * SPS_NPARAM + 31) / 32];
#pragma unroll
    for (int r = 0; r < (CPW * SPS_NPARAM + 31) / 32; ++r) {
        const int e = lane + 32 * r;
        if (e < CPW * SPS_NPARAM) {
            const int ch = e / SPS_NPARAM, k = e - ch * SPS_NPARAM;
            if (kPhys) {                                     // physical parameters, no prior
                t.th[ch][k] = t.x[ch][k];
                t.dth[ch][k] = 1.0f;
                t.lpe[ch][k] = 0.0f;
                dlp[r] = 0.0f;
            } else {
                bound_prior(c, k, t.x[ch][k], t.th[ch][k], t.dth[ch][k], t.lpe[ch][k], dlp[r]);
            }
        }
    }
    __syncwarp();
    // log prior, FP64: two chains per round, 16 lanes each
#pragma unroll
    for (int c0 = 0; c0 < CPW; c0 += 2) {
        const int ch = c0 + (lane >> 4), k = lane & 15;
        double s = (ch < CPW && k < SPS_NPARAM) ? (double)t.lpe[ch][k] : 0.0;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (k == 0 && ch < CPW) t.lpri[ch] = s;
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < (CPW * SPS_NPARAM + 31) / 32; ++r) {     // lpe now holds d log prior / dx
        const int e = lane + 32 * r;
        if (e < CPW * SPS_NPARAM) t.lpe[e / SPS_NPARAM][e % SPS_NPARAM] = dlp[r];
    }
#pragma unroll 1
    for (int ch = 0; ch < CPW; ++ch) age_met_parts<true>(c, age_view(t, ch, et), t.bins, lnT, lT10, t.th[ch], true);
    __syncwarp();
    if constexpr (kNonsep) mdf_rows_fill(c, et.lgz, t.th[0][7], t.th[0][8], qm);
    // M = sum_i m_i in FP64, the chains' reductions interleaved
    {
        double mp[CPW];
#pragma unroll
        for (int ch = 0; ch < CPW; ++ch) mp[ch] = mass_partial(c, age_view(t, ch, et));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int ch = 0; ch < CPW; ++ch) mp[ch] += __shfl_xor_sync(kFull, mp[ch], o);
#pragma unroll
        for (int ch = 0; ch < CPW; ++ch) {
            if (lane == 0) t.M[ch] = mp[ch];
            age_weights(c, age_view(t, ch, et), t.th[ch], mp[ch]);
        }
    }
    // ---- per (chain, band): dust factor and the magnitude offset
    //      A = zp - m_obs - 2.5 (lgM + 9) as an FP32 hi + lo pair
#pragma unroll 1
    for (int e = lane; e < CPW * nb; e += 32) {
        const int ch = e / nb, b = e - ch * nb;
        const float4 dc = t.dust[b];
        t.u.t.F[ch][b] = dust_eval(dc.x, dc.y, dc.z, t.th[ch][9], t.th[ch][10], t.th[ch][11]).F;
        const double Aoff = t.zp[b] - (double)t.mobs[b] - 2.5 * ((double)t.th[ch][0] + 9.0);
        const float ah = (float)Aoff;
        t.u.t.Ah[ch][b] = ah;
        t.u.t.Al[ch][b] = (float)(Aoff - (double)ah);
    }
    __syncwarp();
    // ---- one pass over the galaxy's c_SSP rows, band by band, forward and adjoint:
    //      R_i = sum_j q_j C_bij, U_j = sum_i w_i C_bij (lane partials over its rows),
    //      S_b = sum_j q_j U_j; then with g_b = gamma_b / S_b:
    //      wbar_i += g_b R_i, qbar_j += g_b U_j.
    // The residual that gives gamma_b is taken in FP32: with F S = f 2^e,
    // r = (A - 2.5 e log10 2) - 2.5 log10 f, the bracket exact in hi + lo parts
    // (~1e-7 mag); the FP64 log likelihood is formed afterwards from S_b.
    constexpr float kL2hi = 0.301025390625f;            // log10(2), 11 bits
    constexpr float kL2lo = 4.6050389811952137e-6f;     // log10(2) - kL2hi
    // Metallicity columns are taken in pairs with packed FP32x2 FMAs.
    constexpr int kZ2 = kZnReg / 2;
    float2 qr[CPW][kZ2], qbr[CPW][kZ2];
    float wbl[CPW][4];
#pragma unroll
    for (int ch = 0; ch < CPW; ++ch) {
#pragma unroll
        for (int j = 0; j < kZ2; ++j) {
            qr[ch][j] = make_float2((2 * j < Zn) ? t.q[ch][2 * j] : 0.0f, (2 * j + 1 < Zn) ? t.q[ch][2 * j + 1] : 0.0f);
            qbr[ch][j] = make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) wbl[ch][tt] = 0.0f;
    }
#pragma unroll 1
    for (int b = 0; b < nb; ++b) {
        const float* C = t.ptr[b];
        float2 U[CPW][kZ2];
        float R[CPW][4];
        float spn = 0.0f;                                   // kNonsep: lane partial of S_b
#pragma unroll
        for (int ch = 0; ch < CPW; ++ch)
#pragma unroll
            for (int j = 0; j < kZ2; ++j) U[ch][j] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) {
            const int i = lane + 32 * tt;
            float cs[kZnReg];
#pragma unroll
            for (int j = 0; j < kZnReg; ++j) cs[j] = 0.0f;
            if (i < A) load_row(C + i * Zn, Zn, cs);
            float2 cv[kZ2];
#pragma unroll
            for (int j = 0; j < kZ2; ++j) cv[j] = make_float2(cs[2 * j], cs[2 * j + 1]);
            if constexpr (kNonsep) {
                const float wi = (i < A) ? t.w[0][i] : 0.0f;
                float2 r2 = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int j = 0; j < kZ2; ++j) {
                    const float2 q2 = (i < A) ? make_float2((2 * j < Zn) ? qm[i * Zn + 2 * j] : 0.0f,
                                                            (2 * j + 1 < Zn) ? qm[i * Zn + 2 * j + 1] : 0.0f)
                                              : make_float2(0.0f, 0.0f);
                    r2 = __ffma2_rn(q2, cv[j], r2);
                }
                R[0][tt] = r2.x + r2.y;
                spn = fmaf(wi, R[0][tt], spn);
            } else {
#pragma unroll
                for (int ch = 0; ch < CPW; ++ch) {
                    const float wi = (i < A) ? t.w[ch][i] : 0.0f;
                    const float2 w2 = make_float2(wi, wi);
                    float2 r2 = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int j = 0; j < kZ2; ++j) {
                        r2 = __ffma2_rn(qr[ch][j], cv[j], r2);
                        U[ch][j] = __ffma2_rn(w2, cv[j], U[ch][j]);
                    }
                    R[ch][tt] = r2.x + r2.y;
                }
            }
        }
        float sp[CPW];
#pragma unroll
        for (int ch = 0; ch < CPW; ++ch) {
            if constexpr (kNonsep) {
                sp[ch] = spn;
            } else {
                float2 v = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int j = 0; j < kZ2; ++j) v = __ffma2_rn(qr[ch][j], U[ch][j], v);
                sp[ch] = v.x + v.y;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int ch = 0; ch < CPW; ++ch) sp[ch] += __shfl_xor_sync(kFull, sp[ch], o);
#pragma unroll
        for (int ch = 0; ch < CPW; ++ch) {
            const float S = sp[ch];
            int e2;
            const float f = frexpf(t.u.t.F[ch][b] * S, &e2);
            const float fe = (float)e2;
            const float bh = t.u.t.Ah[ch][b] - 2.5f * (fe * kL2hi);
            const float bl = t.u.t.Al[ch][b] - 2.5f * (fe * kL2lo);
            const float r = (bh + bl) - 2.5f * log10f(f);
            const float gam = r * t.isig2[b] * 1.0857362047581294f;     // 2.5 / ln 10
            const float gh = __fdividef(gam, S);
            if (lane == 0) {
                t.u.t.res[ch][b] = r;
                t.u.t.gam[ch][b] = gam;
                if (kNonsep) t.u.t.gh[ch][b] = gh;
            }
            if constexpr (!kNonsep) {
                const float2 g2 = make_float2(gh, gh);
#pragma unroll
                for (int j = 0; j < kZ2; ++j) qbr[ch][j] = __ffma2_rn(g2, U[ch][j], qbr[ch][j]);
            }
#pragma unroll
            for (int tt = 0; tt < 4; ++tt) wbl[ch][tt] = fmaf(gh, R[ch][tt], wbl[ch][tt]);
        }
    }
    __syncwarp();
    // kNonsep: V_ij = sum_b g_b C_bij row by row, and the MDF gradient
    // sum_ij w_i V_ij dq_ij/d(lgZ, sigma) edge by edge (q_ij = Phi(y_i,j+1) - Phi(y_ij))
    float mdf_gz = 0.0f, mdf_gs = 0.0f;
    if constexpr (kNonsep) {
        const float isd = 1.0f / t.th[0][8], mz = t.th[0][7];
#pragma unroll 1
        for (int tt = 0; tt < 4; ++tt) {
            const int i = lane + 32 * tt;
            if (i >= A) break;
            float v[kZnReg];
#pragma unroll
            for (int j = 0; j < kZnReg; ++j) v[j] = 0.0f;
#pragma unroll 1
            for (int b = 0; b < nb; ++b) {
                float cs[kZnReg];
                load_row(t.ptr[b] + i * Zn, Zn, cs);
                const float gb = t.u.t.gh[0][b];
#pragma unroll
                for (int j = 0; j < kZnReg; ++j) v[j] = fmaf(gb, cs[j], v[j]);
            }
            const float wi = t.w[0][i], mu = mz + c.mdf_off[i];
            float vprev = 0.0f;
#pragma unroll
            for (int e = 0; e <= kZnReg; ++e) {
                if (e > Zn) break;
                const float ve = (e < Zn) ? v[e < kZnReg ? e : kZnReg - 1] : 0.0f;
                const float y = (et.lgz[e] - mu) * isd;
                const float d = wi * (ve - vprev);
                mdf_gz = fmaf(phi_(y), d, mdf_gz);
                mdf_gs = fmaf(phi_y(y), d, mdf_gs);
                vprev = ve;
            }
        }
        mdf_gz = warp_sum(mdf_gz) * isd;
        mdf_gs = warp_sum(mdf_gs) * isd;
    }
    // ---- log likelihood (FP64 sum of the band terms) and the dust / lgM
    //      gradients: two chains per round, 16 lanes each, bands strided by 16
#pragma unroll
    for (int c0 = 0; c0 < CPW; c0 += 2) {
        const int ch = c0 + (lane >> 4), k = lane & 15;
        double s = 0.0;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
        if (ch < CPW) {
#pragma unroll 1
            for (int b = k; b < nb; b += 16) {
                const float4 dc = t.dust[b];
                const DustTerms d = dust_eval(dc.x, dc.y, dc.z, t.th[ch][9], t.th[ch][10], t.th[ch][11]);
                const float r = t.u.t.res[ch][b];
                s -= 0.5 * (double)(r * r * t.isig2[b]);
                const float gam = t.u.t.gam[ch][b];
                const float gF = __fdividef(gam, d.F);
                g0 = fmaf(gam, kLn10f, g0);
                g1 = fmaf(gF, d.dF_AV, g1);
                g2 = fmaf(gF, d.dF_delta, g2);
                g3 = fmaf(gF, d.dF_floor, g3);
            }
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            s += __shfl_xor_sync(kFull, s, o);
            g0 += __shfl_xor_sync(kFull, g0, o);
            g1 += __shfl_xor_sync(kFull, g1, o);
            g2 += __shfl_xor_sync(kFull, g2, o);
            g3 += __shfl_xor_sync(kFull, g3, o);
        }
        if (k == 0 && ch < CPW) {
            t.ll[ch] = s;
            t.gd[ch][0] = g0;
            t.gd[ch][1] = g1;
            t.gd[ch][2] = g2;
            t.gd[ch][3] = g3;
        }
    }
    // wbar_i replaces w_i (each lane its own rows)
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) {
        const int i = lane + 32 * tt;
        if (i < A)
#pragma unroll
            for (int ch = 0; ch < CPW; ++ch) t.w[ch][i] = wbl[ch][tt];
    }
    __syncwarp();
    // qbar: sum the lanes' partials, one chain per round (two half sums);
    // with kNonsep the MDF gradient is already formed and qbar is zero
    if constexpr (kNonsep) {
#pragma unroll
        for (int ch = 0; ch < CPW; ++ch)
            if (lane < Zn) t.qb[ch][lane] = 0.0f;
        __syncwarp();
    } else {
#pragma unroll
        for (int ch = 0; ch < CPW; ++ch) {
#pragma unroll
            for (int j = 0; j < kZ2; ++j) {
                t.u.red[lane][2 * j] = qbr[ch][j].x;
                t.u.red[lane][2 * j + 1] = qbr[ch][j].y;
            }
            __syncwarp();
            const int j = lane & 15, h = lane >> 4;
            float s = 0.0f;
            if (j < kZnReg) {
#pragma unroll 8
                for (int r = 0; r < 16; ++r) s += t.u.red[16 * h + r][j];
            }
            s += __shfl_down_sync(kFull, s, 16);
            if (lane < Zn) t.qb[ch][lane] = s;
            __syncwarp();
        }
    }
    // ---- through the SFH, burst and MDF weights; then to unbounded space
#pragma unroll 1
    for (int ch = 0; ch < CPW; ++ch) {
        float gr[SPS_NPARAM];
#pragma unroll
        for (int k = 0; k < SPS_NPARAM; ++k) gr[k] = 0.0f;
        gr[0] = t.gd[ch][0];
        gr[9] = t.gd[ch][1];
        gr[10] = t.gd[ch][2];
        gr[11] = t.gd[ch][3];
        age_met_adjoint(c, age_view(t, ch, et), lT10, t.M[ch], t.th[ch], gr);
        if constexpr (kNonsep) {
            gr[7] += mdf_gz;
            gr[8] += mdf_gs;
        }
        if (lane < SPS_NPARAM) {
            float v = gr[0];
#pragma unroll
            for (int k = 1; k < SPS_NPARAM; ++k)
                if (lane == k) v = gr[k];
            t.g[ch][lane] = v * t.dth[ch][lane] + t.lpe[ch][lane];
        }
        if (lane == 0) t.lp[ch] = t.ll[ch] + t.lpri[ch];
    }
    __syncwarp();
}

// Draws of iteration `it` for one chain (FP64 Box-Muller): z[12] and, in
// lane 0's view, the accept uniform and L (all lanes get them).
__device__ __forceinline__ void team_draws(uint64_t seed, uint32_t chain, uint32_t it, int L_min,
                                           int L_max, float* z, double& log_u, int& L) {
    const int lane = lane_id();
    uint4 w = make_uint4(0, 0, 0, 0);
    if (lane < 4)
        w = philox4x32_10(make_uint4(it, (uint32_t)lane, chain, 0u), (uint32_t)(seed & 0xffffffffu),
                          (uint32_t)(seed >> 32));
    const int m = lane % 6;
    const int ia = 2 * m, ib = 2 * m + 1;
    const uint32_t ax = __shfl_sync(kFull, w.x, ia >> 2), ay = __shfl_sync(kFull, w.y, ia >> 2);
    const uint32_t az = __shfl_sync(kFull, w.z, ia >> 2), aw = __shfl_sync(kFull, w.w, ia >> 2);
    const uint32_t bx = __shfl_sync(kFull, w.x, ib >> 2), by = __shfl_sync(kFull, w.y, ib >> 2);
    const uint32_t bz = __shfl_sync(kFull, w.z, ib >> 2), bw = __shfl_sync(kFull, w.w, ib >> 2);
    const int sa = ia & 3, sb = ib & 3;
    const uint32_t wa = sa == 0 ? ax : sa == 1 ? ay : sa == 2 ? az : aw;
    const uint32_t wb = sb == 0 ? bx : sb == 1 ? by : sb == 2 ? bz : bw;
    const float r = sqrtf(-2.0f * logf(u01_f(wa)));
    float sn, cs;
    sincospif(2.0f * u01_f(wb), &sn, &cs);
    const float z0 = r * cs, z1 = r * sn;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        z[2 * k] = (float)__shfl_sync(kFull, z0, k);
        z[2 * k + 1] = (float)__shfl_sync(kFull, z1, k);
    }
    const uint32_t w30 = __shfl_sync(kFull, w.x, 3), w31 = __shfl_sync(kFull, w.y, 3);
    log_u = (double)logf(u01_f(w30));
    L = L_min + (int)(((uint64_t)w31 * (uint64_t)(L_max - L_min + 1)) >> 32);
}

__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// v = L L^T p for chain ch (dense metric).
template <int CPW>
__device__ __noinline__ void metric_apply_dense(TeamWork<CPW>& t, int ch) {
    const int lane = lane_id();
    if (lane < SPS_NPARAM) {
        float a = 0.0f;
        for (int k = lane; k < SPS_NPARAM; ++k) a = fmaf(t.cm[ch]->chol[tri(k, lane)], t.p[ch][k], a);
        t.lu[ch][lane] = a;                                      // (L^T p)_j
    }
    __syncwarp();
    if (lane < SPS_NPARAM) {
        float a = 0.0f;
        for (int j = 0; j <= lane; ++j) a = fmaf(t.cm[ch]->chol[tri(lane, j)], t.lu[ch][j], a);
        t.v[ch][lane] = a;                                       // (L L^T p)_k
    }
    __syncwarp();
}

// v = Minv p for chain ch (diagonal minv, or dense L L^T).
template <int CPW>
__device__ __forceinline__ void metric_apply(TeamWork<CPW>& t, int ch, bool dense) {
    if (dense) {
        metric_apply_dense(t, ch);
        return;
    }
    const int lane = lane_id();
    if (lane < SPS_NPARAM) t.v[ch][lane] = t.minv[ch][lane] * t.p[ch][lane];
    __syncwarp();
}

// p = L^-T p by back substitution (dense metric; one thread).
template <int CPW>
__device__ __noinline__ void dense_momentum(TeamWork<CPW>& t, int ch) {
#pragma unroll 1
    for (int i = SPS_NPARAM - 1; i >= 0; --i) {
        float a = t.p[ch][i];
#pragma unroll 1
        for (int k = i + 1; k < SPS_NPARAM; ++k) a -= t.cm[ch]->chol[tri(k, i)] * t.p[ch][k];
        t.p[ch][i] = a / t.cm[ch]->chol[tri(i, i)];
    }
}

// p^T Minv p / 2 (needs metric_apply first).
template <int CPW>
__device__ __forceinline__ double kinetic(TeamWork<CPW>& t, int ch) {
    const int lane = lane_id();
    float v = 0.0f;
    if (lane < SPS_NPARAM) v = t.p[ch][lane] * t.v[ch][lane];
    return 0.5 * (double)warp_sum(v);
}

// Start a trajectory for chain ch: draws, momentum, record the start state,
// first half kick and drift.
template <int CPW>
__device__ __noinline__ void start_traj(TeamWork<CPW>& t, int ch, const HmcParams& hp) {
    const int lane = lane_id();
    float z[SPS_NPARAM];
    double u;
    int L;
    team_draws(hp.seed, t.chain[ch], (uint32_t)t.it[ch], hp.L_min, hp.L_max, z, u, L);
    const bool dense = hp.adapt_mass == 2;
    if (lane < SPS_NPARAM) {
        float zz = z[0];
#pragma unroll
        for (int k = 1; k < SPS_NPARAM; ++k)
            if (lane == k) zz = z[k];
        t.p[ch][lane] = dense ? zz : zz * rsqrtf(t.minv[ch][lane]);
        t.xs[ch][lane] = t.x[ch][lane];
        t.gs[ch][lane] = t.g[ch][lane];
    }
    __syncwarp();
    if (dense && lane == 0) dense_momentum(t, ch);     // p = L^-T z
    __syncwarp();
    metric_apply(t, ch, dense);
    const double h0 = -t.lp[ch] + kinetic(t, ch);
    if (lane == 0) {
        t.uacc[ch] = u;
        t.L[ch] = L;
        t.l[ch] = 0;
        t.lps[ch] = t.lp[ch];
        t.h0[ch] = h0;
    }
    if (lane < SPS_NPARAM) t.p[ch][lane] = fmaf(0.5f * t.eps[ch], t.g[ch][lane], t.p[ch][lane]);
    __syncwarp();
    metric_apply(t, ch, dense);
    if (lane < SPS_NPARAM) t.x[ch][lane] = fmaf(t.eps[ch], t.v[ch][lane], t.x[ch][lane]);
    __syncwarp();
}

__device__ __forceinline__ void win_set_end(int& start, int& end, int width, int stop) {
    end = start + width;
    if (end + 2 * width > stop) end = stop;
    if (width <= 0 || start >= stop) start = end = 0x7fffffff;
}

// Window end of the dense metric: regularised covariance (n/(n+5)) S + 1e-3
// (5/(n+5)) I of the window's co-moments, replaced by its Cholesky factor in
// place; a factorisation that fails keeps the previous metric.  One thread.
__device__ __noinline__ void dense_metric_update(ChainMetric* cm, int wn) {
    const float a = (float)wn / (wn + 5.0f), b = 1e-3f * (5.0f / (wn + 5.0f));
    const float inv = 1.0f / ((float)wn - 1.0f);
    float Lm[78];
#pragma unroll 1
    for (int e = 0; e < 78; ++e) Lm[e] = a * cm->wcov[e] * inv;
#pragma unroll 1
    for (int i = 0; i < SPS_NPARAM; ++i) Lm[tri(i, i)] += b;
#pragma unroll 1
    for (int j = 0; j < SPS_NPARAM; ++j) {
        float dgl = Lm[tri(j, j)];
#pragma unroll 1
        for (int k = 0; k < j; ++k) dgl -= Lm[tri(j, k)] * Lm[tri(j, k)];
        if (!(dgl > 0.0f)) return;
        const float ljj = sqrtf(dgl);
        Lm[tri(j, j)] = ljj;
#pragma unroll 1
        for (int i = j + 1; i < SPS_NPARAM; ++i) {
            float sv = Lm[tri(i, j)];
#pragma unroll 1
            for (int k = 0; k < j; ++k) sv -= Lm[tri(i, k)] * Lm[tri(j, k)];
            Lm[tri(i, j)] = sv / ljj;
        }
    }
#pragma unroll 1
    for (int e = 0; e < 78; ++e) cm->chol[e] = Lm[e];
}

// End of iteration t.it[ch] once the chain's new state is in t.x / t.g /
// t.lp: step-size and metric adaptation (warm-up) with statistic a, or the
// sample (sampling phase); advances the iteration count.
template <int CPW>
__device__ __noinline__ void iter_finish(const Consts& c, TeamWork<CPW>& t, int ch, const HmcParams& hp,
                                         float a, float* __restrict__ samples) {
    const int lane = lane_id();
    const bool dense = hp.adapt_mass == 2;
    const int it = t.it[ch];
    if (it < hp.n_warm) {
        const float m = (float)(t.mda[ch] + 1);
        const float im = __frcp_rn(m + 10.0f);
        const float hbar = (1.0f - im) * t.hbar[ch] + (hp.target_accept - a) * im;
        const float log_eps = t.mu[ch] - sqrtf(m) * 20.0f * hbar;        // gamma = 0.05
        const float wgt = exp2f(-0.75f * log2f(m));                        // kappa = 0.75
        const float leb = wgt * log_eps + (1.0f - wgt) * t.leb[ch];
        const float eps = expf(it < hp.n_warm - 1 ? log_eps : leb);
        __syncwarp();
        if (lane == 0) {
            t.mda[ch] += 1;
            t.hbar[ch] = hbar;
            t.leb[ch] = leb;
            t.eps[ch] = eps;
        }
        __syncwarp();
        if (it >= t.wstart[ch] && it < t.wend[ch]) {
            const int wn = t.wn[ch] + 1;
            if (lane < SPS_NPARAM) {
                const float xv = t.x[ch][lane];
                ChainMetric* cm = t.cm[ch];
                const float d = xv - cm->wmean[lane];
                const float mean = cm->wmean[lane] + d * __frcp_rn((float)wn);
                cm->wmean[lane] = mean;
                cm->wm2[lane] += d * (xv - mean);
                t.dv[ch][0][lane] = d;
                t.dv[ch][1][lane] = xv - mean;
            }
            __syncwarp();
            if (dense) {
                for (int e = lane; e < 78; e += 32) {
                    int i = 0;
                    while (tri(i + 1, 0) <= e) ++i;
                    const int j = e - tri(i, 0);
                    t.cm[ch]->wcov[e] += t.dv[ch][0][i] * t.dv[ch][1][j];
                }
            }
            __syncwarp();
            if (lane == 0) t.wn[ch] = wn;
            if (it == t.wend[ch] - 1) {
                if (wn >= 2 && !dense && lane < SPS_NPARAM) {
                    const float var = t.cm[ch]->wm2[lane] / ((float)wn - 1.0f);
                    const float iw = __frcp_rn((float)wn + 5.0f);
                    t.minv[ch][lane] = ((float)wn * iw) * var + 1e-3f * (5.0f * iw);
                }
                if (wn >= 2 && dense && lane == 0) dense_metric_update(t.cm[ch], wn);
                if (lane < SPS_NPARAM) {
                    t.cm[ch]->wmean[lane] = 0.0f;
                    t.cm[ch]->wm2[lane] = 0.0f;
                }
                for (int e = lane; e < 78; e += 32) t.cm[ch]->wcov[e] = 0.0f;
                __syncwarp();
                if (lane == 0) {
                    t.wn[ch] = 0;
                    t.mu[ch] = logf(10.0f * t.eps[ch]);
                    t.hbar[ch] = 0.0f;
                    t.leb[ch] = 0.0f;
                    t.mda[ch] = 0;
                    int s = t.wend[ch], e = 0, wdt = 2 * t.wwidth[ch];
                    win_set_end(s, e, wdt, t.wstop[ch]);
                    t.wstart[ch] = s;
                    t.wend[ch] = e;
                    t.wwidth[ch] = wdt;
                }
            }
        }
    } else {
        if (lane == 0) t.acc[ch] += a;
        if (samples && lane < SPS_NPARAM)
            samples[((size_t)t.chain[ch] * hp.n_samp + (it - hp.n_warm)) * SPS_NPARAM + lane] =
                bound_theta(c, lane, t.x[ch][lane]);
    }
    __syncwarp();
    if (lane == 0) t.it[ch] = it + 1;
    __syncwarp();
}

// End of chain ch's HMC trajectory: accept / reject, then iter_finish.
template <int CPW>
__device__ __noinline__ void end_traj(const Consts& c, TeamWork<CPW>& t, int ch, const HmcParams& hp,
                                      float* __restrict__ samples) {
    const int lane = lane_id();
    metric_apply(t, ch, hp.adapt_mass == 2);
    const double dH = (-t.lp[ch] + kinetic(t, ch)) - t.h0[ch];
    const bool fin = isfinite(dH);
    const float a = fin ? fminf(1.0f, __expf(-(float)dH)) : 0.0f;
    const bool take = fin && t.uacc[ch] < -dH;
    if (!take && lane < SPS_NPARAM) {
        t.x[ch][lane] = t.xs[ch][lane];
        t.g[ch][lane] = t.gs[ch][lane];
    }
    __syncwarp();
    if (lane == 0) {
        if (!take) t.lp[ch] = t.lps[ch];
        if (!fin || dH > 1000.0) t.ndiv[ch] += 1;
        t.nev[ch] += t.L[ch];
    }
    iter_finish<CPW>(c, t, ch, hp, a, samples);
}

// ---------------------------------------------------------------- NUTS
// Multinomial NUTS with the generalised no-U-turn criterion (Hoffman & Gelman
// 2014; Betancourt 2017), identity metric, the comparison sampler of Sec. 4 /
// App. D.2.  A chain's trajectory grows by doubling: at depth j a subtree of
// 2^j leapfrog steps is built from the trajectory's end in a drawn direction,
// one leaf per evaluation of the team.  Leaves are weighted by exp(H0 - H);
// a leaf replaces the subtree's proposal with probability w / (sum of the
// subtree's weights so far), a completed subtree replaces the trajectory's
// proposal with probability min(1, W_subtree / W_trajectory).  Every aligned
// block of 2^k leaves of the subtree is checked for a U-turn (rho . p_first
// <= 0 or rho . p_last <= 0) as it completes; a U-turn or a divergence
// (H - H0 > 1000) discards the subtree and ends the iteration.  A merged
// trajectory that U-turns, or reaches the depth limit, ends it too.  Draws:
// Philox-4x32-10 with counter (iteration, 16 + j, chain, 0) for the
// direction (word 0, top bit set = forward) and the subtree's uniform
// (word 1), (iteration, 64 + j, chain, n) word 0 for leaf n of the depth-j
// subtree (drawn 32 leaves at a time, one per lane); momenta as HMC.

__device__ __forceinline__ float log_add(float a, float b) {
    const float m = fmaxf(a, b);
    return (m == -INFINITY) ? m : m + log1pf(expf(-fabsf(a - b)));
}

// Uniforms of leaves n .. n+31 of the chain's current subtree (n = t.nn[ch]).
template <int CPW>
__device__ __forceinline__ void nuts_fill(TeamWork<CPW>& t, int ch, const HmcParams& hp) {
    const int lane = lane_id();
    const uint4 w = philox4x32_10(make_uint4((uint32_t)t.it[ch], 64u + (uint32_t)t.nj[ch], t.chain[ch],
                                             (uint32_t)(t.nn[ch] + lane)),
                                  (uint32_t)(hp.seed & 0xffffffffu), (uint32_t)(hp.seed >> 32));
    t.nu[ch][lane] = u01_f(w.x);
    __syncwarp();
}

// New subtree at depth t.nj[ch]: direction, acceptance uniform, empty
// weight and momentum sum, its first 32 leaf uniforms.
template <int CPW>
__device__ __forceinline__ void nuts_level(TeamWork<CPW>& t, int ch, const HmcParams& hp) {
    const int lane = lane_id();
    if (lane == 0) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)t.it[ch], 16u + (uint32_t)t.nj[ch], t.chain[ch], 0u),
                                      (uint32_t)(hp.seed & 0xffffffffu), (uint32_t)(hp.seed >> 32));
        t.dir[ch] = (w.x >> 31) ? 1 : -1;
        t.utree[ch] = u01_f(w.y);
        t.nn[ch] = 0;
        t.lws[ch] = -INFINITY;
    }
    if (lane < SPS_NPARAM) t.nS[ch][lane] = 0.0f;
    __syncwarp();
    nuts_fill(t, ch, hp);
}

// First half kick and drift of the next leaf, in the chain's direction.
template <int CPW>
__device__ __forceinline__ void nuts_advance(TeamWork<CPW>& t, int ch) {
    const int lane = lane_id();
    const float ve = (float)t.dir[ch] * t.eps[ch];
    if (lane < SPS_NPARAM) {
        const float pp = fmaf(0.5f * ve, t.g[ch][lane], t.p[ch][lane]);
        t.p[ch][lane] = pp;
        t.x[ch][lane] = fmaf(ve, pp, t.x[ch][lane]);
    }
    __syncwarp();
}

// Start of iteration t.it[ch]: momentum, H0, the one-state trajectory
// (its ends, momentum sum and proposal), depth 0, first leaf's drift.
template <int CPW>
__device__ __noinline__ void nuts_start(TeamWork<CPW>& t, int ch, const HmcParams& hp) {
    const int lane = lane_id();
    float z[SPS_NPARAM];
    double u;
    int L;
    team_draws(hp.seed, t.chain[ch], (uint32_t)t.it[ch], 1, 1, z, u, L);
    NutsChain* ns = hp.nuts + t.chain[ch];
    float pl = 0.0f;
    if (lane < SPS_NPARAM) {
        pl = z[0];
#pragma unroll
        for (int k = 1; k < SPS_NPARAM; ++k)
            if (lane == k) pl = z[k];
        const float xl = t.x[ch][lane], gl = t.g[ch][lane];
        t.p[ch][lane] = pl;
        t.xs[ch][lane] = xl;
        t.gs[ch][lane] = gl;
        ns->xe[0][lane] = xl;
        ns->xe[1][lane] = xl;
        ns->pe[0][lane] = pl;
        ns->pe[1][lane] = pl;
        ns->ge[0][lane] = gl;
        ns->ge[1][lane] = gl;
        ns->rho[lane] = pl;
    }
    const double h0 = -t.lp[ch] + 0.5 * (double)warp_sum(pl * pl);
    if (lane == 0) {
        t.h0[ch] = h0;
        t.lps[ch] = t.lp[ch];
        t.lw[ch] = 0.0f;
        t.nacc[ch] = 0.0f;
        t.nleaf[ch] = 0;
        t.nj[ch] = 0;
    }
    __syncwarp();
    nuts_level(t, ch, hp);
    nuts_advance(t, ch);
}

// End of the iteration: the trajectory's proposal becomes the state; step
// size adaptation or sample; the next iteration starts (or the chain is done).
template <int CPW>
__device__ __noinline__ void nuts_end_iter(const Consts& c, TeamWork<CPW>& t, int ch, const HmcParams& hp,
                                           float* __restrict__ samples) {
    const int lane = lane_id();
    if (lane < SPS_NPARAM) {
        t.x[ch][lane] = t.xs[ch][lane];
        t.g[ch][lane] = t.gs[ch][lane];
    }
    __syncwarp();
    const float a = t.nacc[ch] / (float)t.nleaf[ch];
    if (lane == 0) {
        t.lp[ch] = t.lps[ch];
        t.nev[ch] += t.nleaf[ch];
    }
    __syncwarp();
    iter_finish<CPW>(c, t, ch, hp, a, samples);
    if (t.it[ch] >= hp.n_warm + hp.n_samp) {
        if (lane == 0) t.done[ch] = 1;
        __syncwarp();
    } else {
        nuts_start<CPW>(t, ch, hp);
    }
}

// The subtree at depth t.nj[ch] is complete and free of U-turns: merge it
// (proposal, weight, momentum sum, end), then check the whole trajectory and
// either end the iteration or start the next subtree from the drawn end.
template <int CPW>
__device__ __noinline__ void nuts_merge(const Consts& c, TeamWork<CPW>& t, int ch, const HmcParams& hp,
                                        float* __restrict__ samples) {
    const int lane = lane_id();
    NutsChain* ns = hp.nuts + t.chain[ch];
    const int j = t.nj[ch];
    const float lws = t.lws[ch];
    const bool take = lws >= t.lw[ch] || t.utree[ch] < expf(lws - t.lw[ch]);
    const int e = t.dir[ch] > 0 ? 1 : 0;
    float d0 = 0.0f, d1 = 0.0f;
    if (lane < SPS_NPARAM) {
        if (take) {
            t.xs[ch][lane] = ns->xq[lane];
            t.gs[ch][lane] = ns->gq[lane];
        }
        const float pl = t.p[ch][lane];
        const float rho = ns->rho[lane] + t.nS[ch][lane];
        ns->rho[lane] = rho;
        ns->xe[e][lane] = t.x[ch][lane];
        ns->pe[e][lane] = pl;
        ns->ge[e][lane] = t.g[ch][lane];
        d0 = rho * (e == 0 ? pl : ns->pe[0][lane]);
        d1 = rho * (e == 1 ? pl : ns->pe[1][lane]);
    }
    d0 = warp_sum(d0);
    d1 = warp_sum(d1);
    if (lane == 0) {
        if (take) t.lps[ch] = ns->lpq;
        t.lw[ch] = log_add(t.lw[ch], lws);
        t.nj[ch] = j + 1;
    }
    __syncwarp();
    if (d0 <= 0.0f || d1 <= 0.0f || j + 1 >= hp.max_depth) {
        nuts_end_iter<CPW>(c, t, ch, hp, samples);
        return;
    }
    nuts_level(t, ch, hp);
    const int e2 = t.dir[ch] > 0 ? 1 : 0;
    if (lane < SPS_NPARAM) {
        t.x[ch][lane] = ns->xe[e2][lane];
        t.p[ch][lane] = ns->pe[e2][lane];
        t.g[ch][lane] = ns->ge[e2][lane];
    }
    __syncwarp();
    nuts_advance(t, ch);
}

// Chain ch after the evaluation at its newest leaf n of the depth-j subtree:
// second half kick, the leaf's weight and proposal draw, the U-turn checks of
// the aligned blocks it completes, then the next leaf (or merge / end).
template <int CPW>
__device__ __forceinline__ void nuts_leaf(const Consts& c, TeamWork<CPW>& t, int ch, const HmcParams& hp,
                                          float* __restrict__ samples) {
    const int lane = lane_id();
    const float ve = (float)t.dir[ch] * t.eps[ch];
    float pl = 0.0f;
    if (lane < SPS_NPARAM) {
        pl = fmaf(0.5f * ve, t.g[ch][lane], t.p[ch][lane]);
        t.p[ch][lane] = pl;
    }
    const double dh = (-t.lp[ch] + 0.5 * (double)warp_sum(pl * pl)) - t.h0[ch];
    if (!isfinite(dh) || dh > 1000.0) {                       // divergence
        if (lane == 0) {
            t.ndiv[ch] += 1;
            t.nleaf[ch] += 1;
        }
        __syncwarp();
        nuts_end_iter<CPW>(c, t, ch, hp, samples);
        return;
    }
    NutsChain* ns = hp.nuts + t.chain[ch];
    const int j = t.nj[ch], n = t.nn[ch];
    const float mdh = -(float)dh;
    const float lws = log_add(t.lws[ch], mdh);
    if (n == 0 || t.nu[ch][n & 31] < expf(mdh - lws)) {     // u01_f can round to 1
        if (lane < SPS_NPARAM) {
            ns->xq[lane] = t.x[ch][lane];
            ns->gq[lane] = t.g[ch][lane];
        }
        if (lane == 0) ns->lpq = t.lp[ch];
    }
    // momentum prefix sum of the subtree; blocks of 2^k leaves starting here
    // record it, blocks ending here are checked (rho = prefix - recorded)
    bool turn = false;
    if (j > 0) {
        const int starts = (n == 0) ? j : __ffs(n) - 1;       // levels k with n % 2^k == 0
        const int ends = __ffs(n + 1) - 1;                     // levels k with (n + 1) % 2^k == 0
        float sb = 0.0f, sa = 0.0f;
        if (lane < SPS_NPARAM) {
            sb = t.nS[ch][lane];
            sa = sb + pl;
            t.nS[ch][lane] = sa;
#pragma unroll 1
            for (int k = 1; k <= starts; ++k) {
                ns->sk[k - 1][lane] = sb;
                ns->pk[k - 1][lane] = pl;
            }
        }
#pragma unroll 1
        for (int k = 1; k <= ends; ++k) {
            float r = 0.0f, f = 0.0f;
            if (lane < SPS_NPARAM) {
                r = sa - ns->sk[k - 1][lane];
                f = ns->pk[k - 1][lane];
            }
            const float d0 = warp_sum(r * f), d1 = warp_sum(r * pl);
            turn = turn || d0 <= 0.0f || d1 <= 0.0f;
        }
    } else if (lane < SPS_NPARAM) {
        t.nS[ch][lane] = pl;
    }
    if (lane == 0) {
        t.nacc[ch] += fminf(1.0f, __expf(mdh));
        t.nleaf[ch] += 1;
        t.lws[ch] = lws;
        t.nn[ch] = n + 1;
    }
    __syncwarp();
    if (turn) {
        nuts_end_iter<CPW>(c, t, ch, hp, samples);
    } else if (n + 1 == (1 << j)) {
        nuts_merge<CPW>(c, t, ch, hp, samples);
    } else {
        if (((n + 1) & 31) == 0) nuts_fill(t, ch, hp);
        nuts_advance(t, ch);
    }
}

// The galaxy's age bins, ln t_obs and, for the observed bands in `bits`, the
// slot table (c_SSP row pointer, dust constants, zero point, data).
template <int CPW>
__device__ __forceinline__ void team_galaxy(const Consts& c, const Galaxies& g, TeamWork<CPW>& t, int64_t gi,
                                            uint32_t bits, const float* __restrict__ mag_obs,
                                            const float* __restrict__ sigma) {
    const int lane = lane_id();
    const int B = c.n_band, K = c.K;
    for (int i = lane; i < c.n_age; i += 32) t.bins[i] = g.bins[(size_t)gi * c.n_age + i];
    if (lane == 0) {
        t.lnT = g.lnT[gi];
        t.lT10 = g.lT10[gi];
    }
    if (lane < B && ((bits >> lane) & 1u)) {
        const int slot = __popc(bits & ((1u << lane) - 1u));
        const size_t gb = (size_t)gi * B + lane;
        t.ptr[slot] = g.cssp + gb * K;
        t.dust[slot] = g.dust_eff[gb];
        t.zp[slot] = g.zp[gb];
        t.mobs[slot] = mag_obs[gb];
        const float sg = sigma[gb];
        t.isig2[slot] = 1.0f / (sg * sg);
    }
    __syncwarp();
}

// Take work item q (a galaxy and a group of CPW of its chains) into the
// team: the galaxy's observed-band slots and the chains' initial state.
// Returns the galaxy index; *nch / *nb get the live chains and observed bands.
template <int CPW>
__device__ __noinline__ int64_t team_init(const Consts& c, const Galaxies& g, const HmcParams& hp,
                                          TeamWork<CPW>& t, int q, const float* __restrict__ theta0,
                                          const float* __restrict__ mag_obs, const float* __restrict__ sigma,
                                          const uint32_t* __restrict__ mask, const int32_t* __restrict__ gal_order,
                                          ChainMetric* __restrict__ metric, int* nch_out, int* nb_out) {
    const int lane = lane_id();
    const int B = c.n_band;
    const uint32_t all = (B >= 32) ? 0xffffffffu : ((1u << B) - 1u);
    const int C = hp.chains_per_gal;
    const int groups = (C + CPW - 1) / CPW;
    const int n_it = hp.n_warm + hp.n_samp;
    const int64_t gi = gal_order ? (int64_t)gal_order[q / groups] : (int64_t)(q / groups);
    const int c0 = (q % groups) * CPW;
    const int nch = min(CPW, C - c0);
    const uint32_t bits = mask[gi] & all;
    team_galaxy<CPW>(c, g, t, gi, bits, mag_obs, sigma);
    // chain state; unused chain slots mirror the first chain and never write
    for (int e = lane; e < CPW * SPS_NPARAM; e += 32) {
        const int ch = e / SPS_NPARAM, k = e - ch * SPS_NPARAM;
        const int cc = (ch < nch) ? ch : 0;
        t.x[ch][k] = theta0[((size_t)gi * C + c0 + cc) * SPS_NPARAM + k];
        t.minv[ch][k] = 1.0f;
        if (ch < nch && hp.adapt_mass) {
            ChainMetric* cm = metric + (gi * C + c0 + ch);
            cm->wmean[k] = 0.0f;
            cm->wm2[k] = 0.0f;
        }
    }
    if (hp.adapt_mass == 2) {
        for (int e = lane; e < nch * 78; e += 32) {
            const int ch = e / 78, r = e - ch * 78;
            int i = 0;
            while (tri(i + 1, 0) <= r) ++i;
            ChainMetric* cm = metric + (gi * C + c0 + ch);
            cm->chol[r] = (r == tri(i, i)) ? 1.0f : 0.0f;
            cm->wcov[r] = 0.0f;
        }
    }
    if (lane < CPW) {
        const int ch = lane;
        t.chain[ch] = (uint32_t)(gi * C + c0 + ((ch < nch) ? ch : 0));
        t.cm[ch] = metric + t.chain[ch];
        t.eps[ch] = hp.eps0;
        t.mu[ch] = logf(10.0f * hp.eps0);
        t.hbar[ch] = t.leb[ch] = t.acc[ch] = 0.0f;
        t.it[ch] = 0;
        t.mda[ch] = t.wn[ch] = t.ndiv[ch] = 0;
        t.nev[ch] = 1;
        t.done[ch] = (ch < nch) ? (n_it <= 0) : 1;
        int init_b, term_b, width;
        const int nw = hp.adapt_mass ? hp.n_warm : 0;
        if (nw >= 150) {
            init_b = 75;
            term_b = 50;
            width = 25;
        } else {
            init_b = (int)(0.15 * nw);
            term_b = (int)(0.1 * nw);
            width = nw - init_b - term_b;
        }
        int s = init_b, e = 0;
        win_set_end(s, e, width, nw - term_b);
        t.wstart[ch] = s;
        t.wend[ch] = e;
        t.wwidth[ch] = width;
        t.wstop[ch] = nw - term_b;
    }
    __syncwarp();
    *nch_out = nch;
    *nb_out = __popc(bits);
    return gi;
}

// One leapfrog step of every live chain after the team's evaluation.
template <int CPW, bool kNuts>
__device__ __forceinline__ void team_step(const Consts& c, TeamWork<CPW>& t, const HmcParams& hp, int nch,
                                          float* __restrict__ samples) {
    if constexpr (kNuts) {
#pragma unroll 1
        for (int ch = 0; ch < CPW; ++ch)
            if (!t.done[ch]) nuts_leaf<CPW>(c, t, ch, hp, (ch < nch) ? samples : nullptr);
    } else {
        const int lane = lane_id();
        const int n_it = hp.n_warm + hp.n_samp;
#pragma unroll 1
        for (int ch = 0; ch < CPW; ++ch) {
            if (t.done[ch]) continue;
            if (lane < SPS_NPARAM) t.p[ch][lane] = fmaf(0.5f * t.eps[ch], t.g[ch][lane], t.p[ch][lane]);
            __syncwarp();
            const int l = t.l[ch] + 1;
            if (l == t.L[ch]) {
                end_traj<CPW>(c, t, ch, hp, (ch < nch) ? samples : nullptr);
                if (t.it[ch] >= n_it) {
                    if (lane == 0) t.done[ch] = 1;
                    __syncwarp();
                } else {
                    start_traj<CPW>(t, ch, hp);
                }
            } else {
                if (lane < SPS_NPARAM) t.p[ch][lane] = fmaf(0.5f * t.eps[ch], t.g[ch][lane], t.p[ch][lane]);
                __syncwarp();
                metric_apply(t, ch, hp.adapt_mass == 2);
                if (lane < SPS_NPARAM) t.x[ch][lane] = fmaf(t.eps[ch], t.v[ch][lane], t.x[ch][lane]);
                __syncwarp();
                if (lane == 0) t.l[ch] = l;
                __syncwarp();
            }
        }
    }
}

// Shared memory of one warp: the team state, and with an age-dependent MDF
// (kNonsep, one chain per warp) the q matrix of the chain.
constexpr int kQmFloats = kKTileMax * 32;
template <int CPW, bool kNonsep>
__host__ __device__ constexpr size_t team_stride() {
    return kNonsep ? sizeof(TeamWork<CPW>) + sizeof(float) * kQmFloats : sizeof(TeamWork<CPW>);
}

// Persistent kernel: each warp is a team working through the queue of
// (galaxy, chain group) items; the warps of a block advance one evaluation per
// pass together (one block barrier per pass), so that they run the same code
// at the same time and share the instruction cache.
template <int CPW, bool kNonsep, bool kNuts>
__global__ void __launch_bounds__(512, 1)
k_hmc_team(const __grid_constant__ Consts c, const Galaxies g, const HmcParams hp,
           const float* __restrict__ theta0, const float* __restrict__ mag_obs,
           const float* __restrict__ sigma, const uint32_t* __restrict__ mask,
           const int32_t* __restrict__ gal_order, float* __restrict__ samples, float* acc_out,
           float* eps_out, int32_t* div_out, int64_t* nev_out, int32_t* status_out, int* queue,
           ChainMetric* __restrict__ metric) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ EdgeTables et;
    unsigned char* mine = smem + (size_t)(threadIdx.x >> 5) * team_stride<CPW, kNonsep>();
    TeamWork<CPW>& t = *reinterpret_cast<TeamWork<CPW>*>(mine);
    float* qm = kNonsep ? reinterpret_cast<float*>(mine + sizeof(TeamWork<CPW>)) : nullptr;
    const int lane = lane_id();
    const int C = hp.chains_per_gal;
    for (int i = threadIdx.x; i <= c.n_age; i += blockDim.x) et.age[i] = c.log_age_edge[i];
    for (int i = threadIdx.x; i <= c.n_met; i += blockDim.x) et.lgz[i] = c.lgz_edge[i];
    __syncthreads();
    const int groups = (C + CPW - 1) / CPW;
    bool have = false, drained = false;     // warp-uniform
    int64_t gi = 0;
    int nch = 0, nb = 0, pass = 0;
    const int sync_every = max(hp.sync_every, 1);
    // every warp meets the block barrier once per sync_every of its own
    // iterations (a warp without work iterates without evaluating)
    for (int iter = 0;; ++iter) {
        if (!have && !drained) {
            int q = 0;
            if (lane == 0) q = atomicAdd(queue, 1);
            q = __shfl_sync(kFull, q, 0);
            const int64_t qe = (int64_t)q + hp.item0;
            if (qe >= (hp.item_end >= 0 ? hp.item_end : g.n * groups)) {
                drained = true;
            } else {
                gi = team_init<CPW>(c, g, hp, t, (int)qe, theta0, mag_obs, sigma, mask, gal_order, metric, &nch,
                                    &nb);
                have = true;
                pass = 0;
            }
        }
        if (iter % sync_every == 0 && !__syncthreads_or(have ? 1 : 0)) break;
        if (!have) continue;
        team_eval<CPW, false, kNonsep>(c, t, et, t.lnT, t.lT10, nb, qm);
        if (pass == 0) {
#pragma unroll 1
            for (int ch = 0; ch < CPW; ++ch)
                if (!t.done[ch]) {
                    if constexpr (kNuts)
                        nuts_start<CPW>(t, ch, hp);
                    else
                        start_traj<CPW>(t, ch, hp);
                }
        } else {
            team_step<CPW, kNuts>(c, t, hp, nch, samples);
        }
        ++pass;
        bool any = false;
        for (int ch = 0; ch < CPW; ++ch) any = any || !t.done[ch];
        if (!any) {
            if (lane < nch) {
                const uint32_t chn = t.chain[lane];
                if (acc_out) acc_out[chn] = t.acc[lane] / (float)max(hp.n_samp, 1);
                if (eps_out) eps_out[chn] = t.eps[lane];
                if (div_out) div_out[chn] = t.ndiv[lane];
                if (nev_out) nev_out[chn] = t.nev[lane];
                if (status_out) status_out[chn] = 0;
            }
            __syncwarp();
            have = false;
        }
    }
}

// log L and its gradient (physical parameters) for n independent rows, one
// row per warp through the team evaluation (the fused single-pass contraction
// and lane-parallel reductions of the sampler); every warp of a block takes
// its next row after one block barrier, so the block's warps stay in phase.
// Non-finite parameters or a galaxy index out of range give NaN outputs;
// any non-finite output raises *nonfinite.
template <bool kNonsep>
__global__ void __launch_bounds__(512, 1)
k_like_team(const __grid_constant__ Consts c, const Galaxies g, const float* __restrict__ theta,
            const int32_t* __restrict__ gal_idx, int64_t n, const float* __restrict__ mag_obs,
            const float* __restrict__ sigma, const uint32_t* __restrict__ mask, float* __restrict__ ll_out,
            float* __restrict__ grad_out, int* __restrict__ nonfinite) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ EdgeTables et;
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5;
    unsigned char* mine = smem + (size_t)warp * team_stride<1, kNonsep>();
    TeamWork<1>& t = *reinterpret_cast<TeamWork<1>*>(mine);
    float* qm = kNonsep ? reinterpret_cast<float*>(mine + sizeof(TeamWork<1>)) : nullptr;
    const int lane = lane_id();
    const int B = c.n_band;
    const uint32_t all = (B >= 32) ? 0xffffffffu : ((1u << B) - 1u);
    for (int i = threadIdx.x; i <= c.n_age; i += blockDim.x) et.age[i] = c.log_age_edge[i];
    for (int i = threadIdx.x; i <= c.n_met; i += blockDim.x) et.lgz[i] = c.lgz_edge[i];
    const int64_t per_round = (int64_t)gridDim.x * warps;
    const int64_t rounds = (n + per_round - 1) / per_round;
    for (int64_t r = 0; r < rounds; ++r) {
        __syncthreads();
        const int64_t row = (r * gridDim.x + blockIdx.x) * warps + warp;
        if (row >= n) continue;
        const int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
        float xk = (lane < SPS_NPARAM) ? theta[row * SPS_NPARAM + lane] : 0.0f;
        const bool ok = __all_sync(kFull, isfinite(xk)) && gi >= 0 && gi < g.n;
        if (!ok) {
            if (lane == 0) {
                atomicOr(nonfinite, 1);
                ll_out[row] = __int_as_float(0x7fc00000);
            }
            if (grad_out && lane < SPS_NPARAM) grad_out[row * SPS_NPARAM + lane] = __int_as_float(0x7fc00000);
            continue;
        }
        const uint32_t bits = mask[gi] & all;
        team_galaxy<1>(c, g, t, gi, bits, mag_obs, sigma);
        if (lane < SPS_NPARAM) t.x[0][lane] = xk;
        __syncwarp();
        team_eval<1, true, kNonsep>(c, t, et, t.lnT, t.lT10, __popc(bits), qm);
        const double ll = t.ll[0];
        const float gk = (lane < SPS_NPARAM) ? t.g[0][lane] : 0.0f;
        if (lane == 0) ll_out[row] = (float)ll;
        if (grad_out && lane < SPS_NPARAM) grad_out[row * SPS_NPARAM + lane] = gk;
        const bool bad = __any_sync(kFull, !isfinite(gk)) || !isfinite(ll);
        if (bad && lane == 0) atomicOr(nonfinite, 1);
        __syncwarp();
    }
}

// AB magnitudes of n independent rows (separable model), one row per warp
// through the team layout without the adjoint: SFH, burst and MDF weights,
// then per band one pass over the galaxy's c_SSP rows, S_b = sum_j q_j
// sum_i w_i C_bij, and m_b = zp_b - 2.5 log10(1e9 10^lgM F_b S_b)
// (Eq. photo_integral_approx).  Every warp of a block takes its next row
// after one block barrier, as k_like_team.  Non-finite parameters or a
// galaxy index out of range give NaN rows and raise *nonfinite.
__global__ void __launch_bounds__(512, 1)
k_phot_team(const __grid_constant__ Consts c, const Galaxies g, const float* __restrict__ theta,
            const int32_t* __restrict__ gal_idx, int64_t n, float* __restrict__ mag_out,
            int* __restrict__ nonfinite) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ EdgeTables et;
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5;
    TeamWork<1>& t = *reinterpret_cast<TeamWork<1>*>(smem + (size_t)warp * sizeof(TeamWork<1>));
    const int lane = lane_id();
    const int B = c.n_band, A = c.n_age, Zn = c.n_met, K = c.K;
    for (int i = threadIdx.x; i <= c.n_age; i += blockDim.x) et.age[i] = c.log_age_edge[i];
    for (int i = threadIdx.x; i <= c.n_met; i += blockDim.x) et.lgz[i] = c.lgz_edge[i];
    const int64_t per_round = (int64_t)gridDim.x * warps;
    const int64_t rounds = (n + per_round - 1) / per_round;
    constexpr int kZ2 = kZnReg / 2;
    for (int64_t r = 0; r < rounds; ++r) {
        __syncthreads();
        const int64_t row = (r * gridDim.x + blockIdx.x) * warps + warp;
        if (row >= n) continue;
        const int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
        const float xk = (lane < SPS_NPARAM) ? theta[row * SPS_NPARAM + lane] : 0.0f;
        const bool ok = __all_sync(kFull, isfinite(xk)) && gi >= 0 && gi < g.n;
        if (!ok) {
            if (lane == 0) atomicOr(nonfinite, 1);
            if (lane < B) mag_out[row * B + lane] = __int_as_float(0x7fc00000);
            continue;
        }
        for (int i = lane; i < A; i += 32) t.bins[i] = g.bins[(size_t)gi * A + i];
        if (lane < SPS_NPARAM) t.th[0][lane] = xk;
        __syncwarp();
        const float lnT = g.lnT[gi], lT10 = g.lT10[gi];
        age_met_parts<true>(c, age_view(t, 0, et), t.bins, lnT, lT10, t.th[0], false);
        __syncwarp();
        const double M = warp_sum_d(mass_partial(c, age_view(t, 0, et)));
        age_weights(c, age_view(t, 0, et), t.th[0], M);
        float2 qr[kZ2];
#pragma unroll
        for (int j = 0; j < kZ2; ++j)
            qr[j] = make_float2((2 * j < Zn) ? t.q[0][2 * j] : 0.0f, (2 * j + 1 < Zn) ? t.q[0][2 * j + 1] : 0.0f);
        float wl[4];
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) {
            const int i = lane + 32 * tt;
            wl[tt] = (i < A) ? t.w[0][i] : 0.0f;
        }
        const double lgm = (double)t.th[0][0] + 9.0;
        const float AV = t.th[0][9], dl = t.th[0][10], ff = t.th[0][11];
        const float* Cg = g.cssp + (size_t)gi * B * K;
#pragma unroll 1
        for (int b = 0; b < B; ++b) {
            const float* C = Cg + (size_t)b * K;
            float2 U[kZ2];
#pragma unroll
            for (int j = 0; j < kZ2; ++j) U[j] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int tt = 0; tt < 4; ++tt) {
                const int i = lane + 32 * tt;
                float cs[kZnReg];
#pragma unroll
                for (int j = 0; j < kZnReg; ++j) cs[j] = 0.0f;
                if (i < A) load_row(C + i * Zn, Zn, cs);
                const float2 w2 = make_float2(wl[tt], wl[tt]);
#pragma unroll
                for (int j = 0; j < kZ2; ++j) U[j] = __ffma2_rn(w2, make_float2(cs[2 * j], cs[2 * j + 1]), U[j]);
            }
            float2 v = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int j = 0; j < kZ2; ++j) v = __ffma2_rn(qr[j], U[j], v);
            const float S = warp_sum(v.x + v.y);
            if (lane == 0) {
                const size_t gb = (size_t)gi * B + b;
                const float4 dc = g.dust_eff[gb];
                const float F = dust_eval(dc.x, dc.y, dc.z, AV, dl, ff).F;
                const double m = g.zp[gb] - 2.5 * (log10_flux(F * S) + lgm);
                mag_out[row * B + b] = (float)m;
                if (!isfinite(m)) atomicOr(nonfinite, 1);
            }
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_phot_team(const Consts& c, const Galaxies& g, const float* theta, const int32_t* gal_idx,
                             int64_t n, float* mag_out, int* nonfinite, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    constexpr int kWarps = 8;
    const size_t smem = sizeof(TeamWork<1>) * kWarps;
    cudaError_t e = cudaFuncSetAttribute(k_phot_team, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phot_team, 32 * kWarps, smem)) != cudaSuccess)
        return e;
    const int64_t need = (n + kWarps - 1) / kWarps;
    const int blocks = (int)std::min<int64_t>(need, (int64_t)std::max(per_sm, 1) * sms);
    k_phot_team<<<blocks, 32 * kWarps, smem, s>>>(c, g, theta, gal_idx, n, mag_out, nonfinite);
    return cudaGetLastError();
}

template <bool kNonsep>
static cudaError_t like_launch(const Consts& c, const Galaxies& g, const float* theta, const int32_t* gal_idx,
                               int64_t n, const float* mag_obs, const float* sigma, const uint32_t* mask,
                               float* ll_out, float* grad_out, int* nonfinite, cudaStream_t s) {
    constexpr int kWarps = 8;
    const size_t smem = team_stride<1, kNonsep>() * kWarps;
    cudaError_t e = cudaFuncSetAttribute(k_like_team<kNonsep>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_like_team<kNonsep>, 32 * kWarps, smem)) !=
        cudaSuccess)
        return e;
    const int64_t need = (n + kWarps - 1) / kWarps;
    const int blocks = (int)std::min<int64_t>(need, (int64_t)std::max(per_sm, 1) * sms);
    k_like_team<kNonsep><<<blocks, 32 * kWarps, smem, s>>>(c, g, theta, gal_idx, n, mag_obs, sigma, mask, ll_out,
                                                           grad_out, nonfinite);
    return cudaGetLastError();
}

cudaError_t launch_like_team(const Consts& c, const Galaxies& g, const float* theta, const int32_t* gal_idx,
                             int64_t n, const float* mag_obs, const float* sigma, const uint32_t* mask,
                             float* ll_out, float* grad_out, int* nonfinite, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (c.mdf_age)
        return like_launch<true>(c, g, theta, gal_idx, n, mag_obs, sigma, mask, ll_out, grad_out, nonfinite, s);
    return like_launch<false>(c, g, theta, gal_idx, n, mag_obs, sigma, mask, ll_out, grad_out, nonfinite, s);
}

size_t hmc_team_smem_per_warp(int cpw, bool rows) {
    if (rows) return team_stride<1, true>();
    return cpw >= 4 ? sizeof(TeamWork<4>) : cpw == 2 ? sizeof(TeamWork<2>) : sizeof(TeamWork<1>);
}

template <int CPW, bool kNonsep, bool kNuts>
static cudaError_t team_launch(const Consts& c, const Galaxies& g, const HmcParams& hp,
                               const float* theta0, const float* mag_obs, const float* sigma,
                               const uint32_t* mask, const int32_t* gal_order, float* samples,
                               float* acc, float* eps_out, int32_t* div, int64_t* nevals,
                               int32_t* status, int* queue, ChainMetric* metric, int blocks, int warps,
                               cudaStream_t s) {
    const size_t smem = team_stride<CPW, kNonsep>() * warps;
    auto kern = k_hmc_team<CPW, kNonsep, kNuts>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, warps * 32, smem, s>>>(c, g, hp, theta0, mag_obs, sigma, mask, gal_order, samples, acc, eps_out,
                                          div, nevals, status, queue, metric);
    return cudaGetLastError();
}

template <int CPW, bool kNonsep, bool kNuts>
static cudaError_t team_occupancy(int warps, int* blocks_per_sm) {
    const size_t smem = team_stride<CPW, kNonsep>() * warps;
    auto kern = k_hmc_team<CPW, kNonsep, kNuts>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, warps * 32, smem);
}

// The sampler is a template parameter (HMC or NUTS code only in each kernel);
// chains per warp: 1, 2 or 4; the age-dependent MDF takes one chain per warp.
template <bool kNuts>
static cudaError_t occupancy_of(int cpw, bool rows, int warps, int* blocks_per_sm) {
    if (rows) return team_occupancy<1, true, kNuts>(warps, blocks_per_sm);
    if (cpw >= 4) return team_occupancy<4, false, kNuts>(warps, blocks_per_sm);
    if (cpw == 2) return team_occupancy<2, false, kNuts>(warps, blocks_per_sm);
    return team_occupancy<1, false, kNuts>(warps, blocks_per_sm);
}

cudaError_t hmc_team_occupancy(int cpw, bool rows, bool nuts, int warps, int* blocks_per_sm) {
    return nuts ? occupancy_of<true>(cpw, rows, warps, blocks_per_sm)
                : occupancy_of<false>(cpw, rows, warps, blocks_per_sm);
}

template <bool kNuts>
static cudaError_t launch_of(int cpw, bool rows, const Consts& c, const Galaxies& g, const HmcParams& hp,
                             const float* theta0, const float* mag_obs, const float* sigma, const uint32_t* mask,
                             const int32_t* gal_order, float* samples, float* acc, float* eps_out, int32_t* div,
                             int64_t* nevals, int32_t* status, int* queue, ChainMetric* metric, int blocks,
                             int warps, cudaStream_t s) {
    if (rows)
        return team_launch<1, true, kNuts>(c, g, hp, theta0, mag_obs, sigma, mask, gal_order, samples, acc,
                                           eps_out, div, nevals, status, queue, metric, blocks, warps, s);
    if (cpw >= 4)
        return team_launch<4, false, kNuts>(c, g, hp, theta0, mag_obs, sigma, mask, gal_order, samples, acc,
                                            eps_out, div, nevals, status, queue, metric, blocks, warps, s);
    if (cpw == 2)
        return team_launch<2, false, kNuts>(c, g, hp, theta0, mag_obs, sigma, mask, gal_order, samples, acc,
                                            eps_out, div, nevals, status, queue, metric, blocks, warps, s);
    return team_launch<1, false, kNuts>(c, g, hp, theta0, mag_obs, sigma, mask, gal_order, samples, acc, eps_out,
                                        div, nevals, status, queue, metric, blocks, warps, s);
}

cudaError_t launch_hmc_team(int cpw, bool rows, const Consts& c, const Galaxies& g, const HmcParams& hp,
                            const float* theta0, const float* mag_obs, const float* sigma,
                            const uint32_t* mask, const int32_t* gal_order, float* samples,
                            float* acc, float* eps_out, int32_t* div, int64_t* nevals,
                            int32_t* status, int* queue, ChainMetric* metric, int blocks, int warps,
                            cudaStream_t s) {
    if (hp.nuts)
        return launch_of<true>(cpw, rows, c, g, hp, theta0, mag_obs, sigma, mask, gal_order, samples, acc, eps_out,
                               div, nevals, status, queue, metric, blocks, warps, s);
    return launch_of<false>(cpw, rows, c, g, hp, theta0, mag_obs, sigma, mask, gal_order, samples, acc, eps_out,
                            div, nevals, status, queue, metric, blocks, warps, s);
}

}  // namespace sps
