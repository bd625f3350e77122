// Exact photometry (Eq. photo_integral_exact) and its adjoint, as a chain of
// kernels over a block of rows:
//   weights : W[r][ij] = w_i q_j (FP32, or BF16 scaled by 2^{e_i})
//   fwd     : S = W L over the wavelength grid, reduced in the epilogue with
//             the dust curve and the redshifted band weights into
//             A[r][b][0..3] = sum_n wb S (1, E, E base, E dterm)   (10^-0.4A = E)
//   like    : magnitudes, log L, gamma_b / c_b, dust and lgM gradients
//   vgen    : v[r][n] = F_att(n) sum_b (gamma_b / c_b) wb(n)
//   adj     : Wbar = v L^T (the second contraction: recomputed, not stored)
//   grad    : Wbar -> d logL / d theta through the SFH, burst and MDF weights
// This file holds the SIMT contraction kernels.
#include <cuda_bf16.h>

#include "band_tab.cuh"
#include "sps_device.cuh"

namespace sps {

namespace {

constexpr int kBM = 64, kBN = 128, kBK = 16, kThreads = 256;

__device__ __forceinline__ float bf16_to_f(uint16_t h) { return __uint_as_float(((uint32_t)h) << 16); }
__device__ __forceinline__ uint16_t f_to_bf16(float f) {
    __nv_bfloat16 b = __float2bfloat16_rn(f);
    return *reinterpret_cast<uint16_t*>(&b);
}
template <typename T>
__device__ __forceinline__ float ld_elem(const T* p);
template <>
__device__ __forceinline__ float ld_elem<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ld_elem<uint16_t>(const uint16_t* p) { return bf16_to_f(__ldg(p)); }

// ---------------------------------------------------------------- weights
__global__ void __launch_bounds__(32 * kWarpsApprox)
k_weights(const __grid_constant__ Consts c, const Grid grid, const Galaxies g,
          const float* __restrict__ theta, const int32_t* __restrict__ gal_idx, int64_t n,
          int bf16, float* __restrict__ W32, uint16_t* __restrict__ Wbf,
          const int32_t* __restrict__ pos_of, float* __restrict__ W32lo, float* __restrict__ keep) {
    __shared__ RowScratch scratch[kWarpsApprox];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    RowScratch& s = scratch[warp];
    for (int64_t row = (int64_t)blockIdx.x * kWarpsApprox + warp; row < n;
         row += (int64_t)gridDim.x * kWarpsApprox) {
        const int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
        RowParams p;
        load_params(c, theta + row * SPS_NPARAM, false, p);
        if (gi < 0 || gi >= g.n) p.finite = false;
        if (p.finite) {
            // with keep (a gradient follows): the derivative integrals too, and the
            // arrays the adjoint needs are kept for it (m and w are the same
            // either way: the derivatives are separate accumulators)
            const double M = age_met_weights(c, s, g.bins + (size_t)gi * c.n_age, g.lnT[gi], g.lT10[gi], p,
                                             keep != nullptr);
            if (keep) {
                const int A = c.n_age;
                float* kr = keep + row * keep_stride(c);
                if (lane == 0) *reinterpret_cast<double*>(kr) = M;
                float* ka = kr + 2;
                for (int i = lane; i < A; i += 32) {
                    ka[i] = s.m[i];
                    ka[A + i] = s.dm[0][i];
                    ka[2 * A + i] = s.dm[1][i];
                    ka[3 * A + i] = s.dm[2][i];
                    ka[4 * A + i] = s.pi[i];
                    ka[5 * A + i] = s.w[i];
                }
                if (lane < c.n_met) ka[6 * A + lane] = s.q[lane];
            }
        } else {
            for (int i = lane; i < c.n_age; i += 32) s.w[i] = __int_as_float(0x7fc00000);
            if (lane < c.n_met) s.q[lane] = 1.0f;
            __syncwarp();
        }
        const int64_t wr = pos_of ? (int64_t)pos_of[row] : row;
        const bool nonsep = c.mdf_age != 0 && p.finite;
        if (nonsep) mdf_rows_fill(c, c.lgz_edge, p.th[7], p.th[8], s.u.kbuf);
        // W_k = w_i q_j, k = i Zn + j: a lane writes the pair (k, k + 1) for
        // k = 2 lane + 64 t (k_pad is even), with (i, j) of k kept incrementally
        const int Zn = c.n_met;
        int k = 2 * lane;
        int i = k / Zn, j = k - i * Zn;
        const int di = 64 / Zn, dj = 64 - di * Zn;
        for (; k < c.k_pad; k += 64) {
            int i1 = i, j1 = j + 1;
            if (j1 == Zn) {
                j1 = 0;
                ++i1;
            }
            float v0 = 0.0f, v1 = 0.0f;
            if (k < c.K) v0 = s.w[i] * (nonsep ? s.u.kbuf[k] : s.q[j]);
            if (k + 1 < c.K) v1 = s.w[i1] * (nonsep ? s.u.kbuf[k + 1] : s.q[j1]);
            const int64_t o = wr * c.k_pad + k;
            if (bf16) {
                const float b0 = k < c.K ? v0 * grid.row_scale[i] : 0.0f;
                const float b1 = k + 1 < c.K ? v1 * grid.row_scale[i1] : 0.0f;
                *reinterpret_cast<uint32_t*>(Wbf + o) = (uint32_t)f_to_bf16(b0) | ((uint32_t)f_to_bf16(b1) << 16);
            } else if (W32lo) {                        // 3xTF32 operand halves
                float h0, l0, h1, l1;
                tf32_split(v0, h0, l0);
                tf32_split(v1, h1, l1);
                *reinterpret_cast<float2*>(W32 + o) = make_float2(h0, h1);
                *reinterpret_cast<float2*>(W32lo + o) = make_float2(l0, l1);
            } else {
                *reinterpret_cast<float2*>(W32 + o) = make_float2(v0, v1);
            }
            i += di;
            j += dj;
            if (j >= Zn) {
                j -= Zn;
                ++i;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- SIMT NN tile
// acc[4][8] of thread (ty, tx) = rows m0 + 4 ty + i, columns n0 + 8 tx + j of
// A[m][0:red] * B[0:red][n]; A rows red-contiguous (lda), B rows n-contiguous (ldb).
template <typename TA, typename TB>
__device__ __forceinline__ void tile_contract(const TA* __restrict__ A, int64_t lda, int64_t m0,
                                              int64_t M, const TB* __restrict__ Bm, int64_t ldb,
                                              int n0, int N, int red, float (&As)[kBK][kBM + 4],
                                              float (&Bs)[kBK][kBN], float (&acc)[4][8]) {
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < red; k0 += kBK) {
        for (int e = tid; e < kBM * kBK; e += kThreads) {
            int mm = e / kBK, kk = e % kBK;
            int64_t m = m0 + mm;
            int k = k0 + kk;
            As[kk][mm] = (m < M && k < red) ? ld_elem<TA>(A + m * lda + k) : 0.0f;
        }
        for (int e = tid; e < kBK * kBN; e += kThreads) {
            int kk = e / kBN, nn = e % kBN;
            int k = k0 + kk, nidx = n0 + nn;
            Bs[kk][nn] = (k < red && nidx < N) ? ld_elem<TB>(Bm + (int64_t)k * ldb + nidx) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float a[4], b[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = Bs[kk][tx * 8 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- forward + epilogue
// One block per 64 rows, looping over every wavelength tile; the epilogue
// folds each tile into A[r][b][4] in shared memory (fixed order).  KZ also
// folds the redshift derivative of the band weights, wb' = d wb / dz =
// q_n T'((1+z) l_n), into Az[r][b][2] = sum_n wb' S (1, E).
template <typename T, bool KZ = false>
__global__ void __launch_bounds__(kThreads)
k_exact_fwd(const __grid_constant__ Consts c, const Grid grid, const Galaxies g,
            const float* __restrict__ theta, const int32_t* __restrict__ gal_idx, int64_t n,
            const T* __restrict__ W, const T* __restrict__ Ltab, float* __restrict__ cJ,
            float* __restrict__ cJz) {
    __shared__ float As[kBK][kBM + 4];
    __shared__ float Bs[kBK][kBN];
    __shared__ float4 lc[kBN];
    __shared__ float lamt[kBN];
    __shared__ float4 rdust[kBM];  // A_V/4.05, delta, F_floor, E_b
    extern __shared__ float dyn[];
    const int B = c.n_band;
    float* accsm = dyn;                                              // [kBM][B][4]
    int2* sup = reinterpret_cast<int2*>(dyn + kBM * B * 4);          // [kBM][B]
    float2* ga = reinterpret_cast<float2*>(sup + kBM * B);           // [kBM][B]
    float* accz = reinterpret_cast<float*>(ga + kBM * B);            // KZ: [kBM][B][2]
    float* gzf = accz + kBM * B * 2;                                 // KZ: [kBM][B] 1/sigma or 1/step
    const int64_t m0 = (int64_t)blockIdx.x * kBM;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    for (int e = tid; e < kBM * B * 4; e += kThreads) accsm[e] = 0.0f;
    if (KZ)
        for (int e = tid; e < kBM * B * 2; e += kThreads) accz[e] = 0.0f;
    for (int e = tid; e < kBM * B; e += kThreads) {
        int r = e / B, b = e % B;
        int64_t row = m0 + r;
        int64_t gi = (row < n) ? (gal_idx ? (int64_t)gal_idx[row] : row) : -1;
        if (gi >= 0 && gi < g.n) {
            sup[e] = g.support[gi * B + b];
            ga[e] = g.gauss[gi * B + b];
            if (KZ) gzf[e] = fabsf(ga[e].y) / (1.0f + g.z[gi]);   // (1+z)/s / (1+z)
        } else {
            sup[e] = make_int2(0, 0);
            ga[e] = make_float2(0.f, 0.f);
            if (KZ) gzf[e] = 0.0f;
        }
    }
    for (int r = tid; r < kBM; r += kThreads) {
        int64_t row = m0 + r;
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < n) {
            const float* t = theta + row * SPS_NPARAM;
            d = make_float4(t[9] * (1.0f / 4.05f), t[10], t[11], fmaxf(0.85f - 1.9f * t[10], 0.0f));
        }
        rdust[r] = d;
    }
    __syncthreads();
    float acc[4][8];
    for (int n0 = 0; n0 < c.n_lam; n0 += kBN) {
        tile_contract<T, T>(W, c.k_pad, m0, n, Ltab, c.lam_pad, n0, c.n_lam, c.K, As, Bs, acc);
        for (int t = tid; t < kBN; t += kThreads) {
            int nn = n0 + t;
            lc[t] = (nn < c.n_lam) ? grid.lamc[nn] : make_float4(0.f, 0.f, 0.f, 0.f);
            lamt[t] = (nn < c.n_lam) ? grid.lam[nn] : 0.0f;
        }
        __syncthreads();
        for (int b = 0; b < B; ++b) {
            const int kind = c.band_kind[b];
            const float* tabT = grid.band_T + c.tab_off[b];
            const int tabn = c.tab_n[b];
            float v[4][4];
            float vz[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                v[i][0] = v[i][1] = v[i][2] = v[i][3] = 0.0f;
                vz[i][0] = vz[i][1] = 0.0f;
                const int r = ty * 4 + i;
                const int2 sp = sup[r * B + b];
                const float2 gg = ga[r * B + b];
                const float4 rd = rdust[r];
                const float fz = KZ ? gzf[r * B + b] : 0.0f;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int nl = tx * 8 + j, nn = n0 + nl;
                    if (nn >= sp.x && nn < sp.y) {
                        const float4 L4 = lc[nl];
                        float wb = L4.x;
                        float wz = 0.0f;
                        if (kind == 1) {
                            float u = (lamt[nl] - gg.x) * gg.y;
                            wb *= __expf(-0.5f * u * u);
                            if (KZ) wz = -wb * lamt[nl] * u * fz;       // q T' with T' = -u T / s
                        } else if (kind == 2) {
                            const float ut = (lamt[nl] - gg.x) * -gg.y;
                            wb *= tab_T32(tabT, tabn, ut);
                            if (KZ) wz = L4.x * lamt[nl] * tab_dT32(tabT, tabn, ut) * fz;
                        }
                        float pw = __expf(rd.y * L4.z);
                        float base = L4.y * pw + rd.w * L4.w;
                        float E = exp2f(-0.4f * kLog2_10f * rd.x * base);
                        float dterm = L4.y * pw * L4.z - (rd.w > 0.0f ? 1.9f * L4.w : 0.0f);
                        float S = acc[i][j] * wb;
                        float es = S * E;
                        v[i][0] += S;
                        v[i][1] += es;
                        v[i][2] += es * base;
                        v[i][3] += es * dterm;
                        if (KZ) {
                            const float Sz = acc[i][j] * wz;
                            vz[i][0] += Sz;
                            vz[i][1] += Sz * E;
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float x = v[i][q];
                    x += __shfl_xor_sync(kFull, x, 8);
                    x += __shfl_xor_sync(kFull, x, 4);
                    x += __shfl_xor_sync(kFull, x, 2);
                    x += __shfl_xor_sync(kFull, x, 1);
                    v[i][q] = x;
                }
                if (KZ) {
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        float x = vz[i][q];
                        x += __shfl_xor_sync(kFull, x, 8);
                        x += __shfl_xor_sync(kFull, x, 4);
                        x += __shfl_xor_sync(kFull, x, 2);
                        x += __shfl_xor_sync(kFull, x, 1);
                        vz[i][q] = x;
                    }
                }
            }
            if (tx == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) accsm[((ty * 4 + i) * B + b) * 4 + q] += v[i][q];
                    if (KZ) {
                        accz[((ty * 4 + i) * B + b) * 2 + 0] += vz[i][0];
                        accz[((ty * 4 + i) * B + b) * 2 + 1] += vz[i][1];
                    }
                }
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < kBM * B * 4; e += kThreads) {
        int64_t row = m0 + e / (B * 4);
        if (row < n) cJ[m0 * B * 4 + e] = accsm[e];
    }
    if (KZ)
        for (int e = tid; e < kBM * B * 2; e += kThreads) {
            int64_t row = m0 + e / (B * 2);
            if (row < n) cJz[m0 * B * 2 + e] = accz[e];
        }
}

// ---------------------------------------------------------------- likelihood
// One thread per row.  cJ -> magnitudes, log L, gbar[r][b] = gamma_b / c_b
// and rowinfo[r] = (dlogL/dlgM, dA_V, ddelta, dF_floor).
__global__ void k_exact_like(const __grid_constant__ Consts c, const Galaxies g,
                             const float* __restrict__ theta, const int32_t* __restrict__ gal_idx,
                             int64_t n, const float* __restrict__ cJ,
                             const float* __restrict__ mag_obs, const float* __restrict__ sigma,
                             const uint32_t* __restrict__ mask, float* __restrict__ mag_out,
                             float* __restrict__ ll_out, float* __restrict__ gbar,
                             float* __restrict__ rowinfo, int* __restrict__ nonfinite,
                             const float* __restrict__ cJz, float* __restrict__ rowz,
                             double* __restrict__ ll64_out) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int B = c.n_band;
    const int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
    if (gi < 0 || gi >= g.n) {
        atomicOr(nonfinite, 1);
        if (rowz) rowz[row] = 0.0f;
        if (ll_out) ll_out[row] = __int_as_float(0x7fc00000);
        if (ll64_out) ll64_out[row] = __longlong_as_double(0x7ff8000000000000ll);
        for (int b = 0; b < B; ++b) {
            if (mag_out) mag_out[row * B + b] = __int_as_float(0x7fc00000);
            if (gbar) gbar[row * B + b] = 0.0f;
        }
        if (rowinfo)
            for (int q = 0; q < 4; ++q) rowinfo[row * 4 + q] = 0.0f;
        return;
    }
    const float* t = theta + row * SPS_NPARAM;
    const float lgM = t[0], AV = t[9], ff = t[11];
    const uint32_t bits = mask ? mask[gi] : 0u;
    double ll = 0.0;
    float g0 = 0.f, gAV = 0.f, gdl = 0.f, gff = 0.f;
    float gz = 0.f;     // explicit d log L / dz (zero point, band weights; weights W fixed)
    bool bad = false;
    for (int b = 0; b < B; ++b) {
        const float* a = cJ + (row * B + b) * 4;
        float cprime = ff * a[0] + (1.0f - ff) * a[1];
        double m = g.zp[gi * B + b] - 2.5 * (log10_flux(cprime) + (double)lgM + 9.0);
        bad = bad || !isfinite(m);
        if (mag_out) mag_out[row * B + b] = (float)m;
        float gb = 0.0f;
        if ((bits >> b) & 1u) {
            double is2 = 1.0 / ((double)sigma[gi * B + b] * (double)sigma[gi * B + b]);
            double r = m - (double)mag_obs[gi * B + b];
            ll += -0.5 * r * r * is2;
            float gam = (float)(2.5 * r * is2 / 2.302585092994046);
            gb = gam / cprime;
            g0 += gam * kLn10f;
            gAV += gb * (1.0f - ff) * (-0.4f * kLn10f / 4.05f) * a[2];
            gdl += gb * (1.0f - ff) * (-0.4f * kLn10f) * (AV / 4.05f) * a[3];
            gff += gb * (a[0] - a[1]);
            if (cJz) {
                const float* az = cJz + (row * B + b) * 2;
                gz += (float)(-r * is2) * g.dzp[gi * B + b] + gb * (ff * az[0] + (1.0f - ff) * az[1]);
            }
        }
        if (gbar) gbar[row * B + b] = gb;
    }
    if (rowz) rowz[row] = gz;
    if (ll_out) ll_out[row] = (float)ll;
    if (ll64_out) ll64_out[row] = ll;
    if (rowinfo) {
        rowinfo[row * 4 + 0] = g0;
        rowinfo[row * 4 + 1] = gAV;
        rowinfo[row * 4 + 2] = gdl;
        rowinfo[row * 4 + 3] = gff;
    }
    if (bad || (mask && !isfinite(ll))) atomicOr(nonfinite, 1);
}

// ---------------------------------------------------------------- adjoint source
// One block per row: v[n] = F_att(n) sum_b gbar_b wb(n), zero beyond the grid.
// The band sum is built band by band over each band's support only (a row
// buffer in shared memory, bands in order, so each v[n] sums its bands in
// the same order as a per-wavelength loop would), then the dust factor is
// applied once per wavelength.
__global__ void __launch_bounds__(256)
k_exact_vgen(const __grid_constant__ Consts c, const Grid grid, const Galaxies g,
             const float* __restrict__ theta, const int32_t* __restrict__ gal_idx, int64_t n,
             const float* __restrict__ gbar, float* __restrict__ V, uint16_t* __restrict__ Vbf,
             float* __restrict__ Vlo) {
    extern __shared__ __align__(16) float ssum[];  // [lam_pad]
    __shared__ float gb[kMaxBands];
    __shared__ int2 sp[kMaxBands];
    __shared__ float2 gg[kMaxBands];
    const int64_t row = blockIdx.x;
    if (row >= n) return;
    const int B = c.n_band;
    int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
    if (gi < 0 || gi >= g.n) gi = 0;          // row already flagged; gbar is zero
    if (threadIdx.x < B) {
        gb[threadIdx.x] = gbar[row * B + threadIdx.x];
        sp[threadIdx.x] = g.support[gi * B + threadIdx.x];
        gg[threadIdx.x] = g.gauss[gi * B + threadIdx.x];
    }
    for (int nn = threadIdx.x; nn < c.lam_pad; nn += blockDim.x) ssum[nn] = 0.0f;
    __syncthreads();
    for (int b = 0; b < B; ++b) {
        const float gbb = gb[b];
        if (gbb == 0.0f) continue;                 // block-uniform
        const int kind = c.band_kind[b];
        const int lo = sp[b].x, hi = min(sp[b].y, c.n_lam);
        const float2 gp = gg[b];
        const float gsv = gp.y * 0.84932180028801904f;   // e^{-u^2 / 2} = 2^{-(u sqrt(log2(e) / 2))^2}
        for (int nn = lo + threadIdx.x; nn < hi; nn += blockDim.x) {
            const float2 lq = __ldg(grid.lamq + nn);      // (lambda, q / lambda)
            float wb = lq.y;
            if (kind == 1) {
                const float u = (lq.x - gp.x) * gsv;
                wb *= exp2f(-(u * u));
            } else if (kind == 2) {
                wb *= tab_T32(grid.band_T + c.tab_off[b], c.tab_n[b], (lq.x - gp.x) * -gp.y);
            }
            ssum[nn] = fmaf(gbb, wb, ssum[nn]);
        }
        __syncthreads();
    }
    const float* t = theta + row * SPS_NPARAM;
    const float AV = t[9], dl = t[10], ff = t[11];
    if (Vbf) {
        // BF16 v in column pairs: F = F_floor + (1 - F_floor) 2^{cA (k0 e^{delta lnr} + E_b D)}
        // in packed FP32x2 (the terms of dust_eval), one 32-bit store per pair
        const float eb = fmaxf(0.85f - 1.9f * dl, 0.0f);
        const float cA = -0.4f * kLog2_10f * AV * (1.0f / 4.05f);
        const float dlg = dl * 1.4426950408889634f;     // delta log2(e)
        const float2 dl2 = make_float2(dlg, dlg), eb2 = make_float2(eb, eb), cA2 = make_float2(cA, cA);
        const float2 ff2 = make_float2(ff, ff), omf2 = make_float2(1.0f - ff, 1.0f - ff);
        uint32_t* vrow = reinterpret_cast<uint32_t*>(Vbf + row * c.lam_pad);
        const float2* s2 = reinterpret_cast<const float2*>(ssum);
        for (int p = threadIdx.x; 2 * p < c.lam_pad; p += blockDim.x) {
            const float2 sum = s2[p];
            uint32_t out = 0u;
            if (sum.x != 0.0f || sum.y != 0.0f) {
                const int nn = 2 * p;
                const float4 La = grid.lamc[nn];
                const float4 Lb = (nn + 1 < c.n_lam) ? grid.lamc[nn + 1] : La;
                const float2 pa = __fmul2_rn(dl2, make_float2(La.z, Lb.z));
                const float2 pw = make_float2(exp2f(pa.x), exp2f(pa.y));
                const float2 base = __ffma2_rn(make_float2(La.y, Lb.y), pw, __fmul2_rn(eb2, make_float2(La.w, Lb.w)));
                const float2 ea = __fmul2_rn(cA2, base);
                const float2 E = make_float2(exp2f(ea.x), exp2f(ea.y));
                const float2 F = __ffma2_rn(omf2, E, ff2);
                const float2 v = __fmul2_rn(F, sum);
                out = (uint32_t)f_to_bf16(v.x) | ((uint32_t)f_to_bf16(v.y) << 16);
            }
            vrow[p] = out;
        }
        return;
    }
    for (int nn = threadIdx.x; nn < c.lam_pad; nn += blockDim.x) {
        const float sum = ssum[nn];
        float v = 0.0f;
        if (sum != 0.0f) {
            const float4 L4 = grid.lamc[nn];
            v = dust_eval(L4.y, L4.z, L4.w, AV, dl, ff).F * sum;
        }
        if (Vbf) {
            Vbf[row * c.lam_pad + nn] = f_to_bf16(v);
        } else if (Vlo) {                              // 3xTF32 operand halves
            float hi, lo;
            tf32_split(v, hi, lo);
            V[row * c.lam_pad + nn] = hi;
            Vlo[row * c.lam_pad + nn] = lo;
        } else {
            V[row * c.lam_pad + nn] = v;
        }
    }
}

// ---------------------------------------------------------------- adjoint contraction
// Wbar[m][k] = sum_n V[m][n] Lt[n][k] (x 2^{e_i} for the scaled BF16 table).
template <typename TB>
__global__ void __launch_bounds__(kThreads)
k_exact_adj(const __grid_constant__ Consts c, const Grid grid, int64_t n,
            const float* __restrict__ V, const TB* __restrict__ Lt, int scaled,
            float* __restrict__ Wbar) {
    __shared__ float As[kBK][kBM + 4];
    __shared__ float Bs[kBK][kBN];
    const int64_t m0 = (int64_t)blockIdx.x * kBM;
    const int n0 = blockIdx.y * kBN;
    float acc[4][8];
    tile_contract<float, TB>(V, c.lam_pad, m0, n, Lt, c.k_pad, n0, c.K, c.n_lam, As, Bs, acc);
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t row = m0 + ty * 4 + i;
        if (row >= n) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int k = n0 + tx * 8 + j;
            if (k < c.K) {
                float v = acc[i][j];
                if (scaled) v *= grid.row_scale[k / c.n_met];
                Wbar[row * c.k_pad + k] = v;
            }
        }
    }
}

// ---------------------------------------------------------------- gradient assembly
__global__ void __launch_bounds__(32 * kWarpsApprox)
k_exact_grad(const __grid_constant__ Consts c, const Galaxies g, const float* __restrict__ theta,
             const int32_t* __restrict__ gal_idx, int64_t n, const float* __restrict__ rowinfo,
             const float* __restrict__ Wbar, float* __restrict__ grad_out, const float* __restrict__ rowz,
             const float* __restrict__ keep) {
    __shared__ RowScratch scratch[kWarpsApprox];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    RowScratch& s = scratch[warp];
    const int A = c.n_age, Zn = c.n_met, K = c.K;
    const int NG = rowz ? SPS_NPARAM + 1 : SPS_NPARAM;       // with rowz: d/dz last
    for (int64_t row = (int64_t)blockIdx.x * kWarpsApprox + warp; row < n;
         row += (int64_t)gridDim.x * kWarpsApprox) {
        const int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
        RowParams p;
        load_params(c, theta + row * SPS_NPARAM, false, p);
        if (gi < 0 || gi >= g.n) p.finite = false;
        if (!p.finite) {
            if (lane < NG) grad_out[row * NG + lane] = __int_as_float(0x7fc00000);
            continue;
        }
        double M;
        if (keep) {                                // the weights kernel's arrays of this row
            const float* kr = keep + row * keep_stride(c);
            M = *reinterpret_cast<const double*>(kr);
            const float* ka = kr + 2;
            for (int i = lane; i < A; i += 32) {
                s.m[i] = ka[i];
                s.dm[0][i] = ka[A + i];
                s.dm[1][i] = ka[2 * A + i];
                s.dm[2][i] = ka[3 * A + i];
                s.pi[i] = ka[4 * A + i];
                s.w[i] = ka[5 * A + i];
            }
            if (lane < Zn) s.q[lane] = ka[6 * A + lane];
        } else {
            M = age_met_weights(c, s, g.bins + (size_t)gi * A, g.lnT[gi], g.lT10[gi], p, true);
        }
        for (int k = lane; k < K; k += 32) s.u.kbuf[k] = Wbar[row * c.k_pad + k];
        __syncwarp();
        float gr[SPS_NPARAM];
#pragma unroll
        for (int k = 0; k < SPS_NPARAM; ++k) gr[k] = 0.0f;
        if (c.mdf_age) {
            mdf_rows_adjoint(c, s.view(c), s.u.kbuf, p.th[7], p.th[8], gr);
        } else {
            for (int i = lane; i < A; i += 32) {
                float a = 0.0f;
                for (int j = 0; j < Zn; ++j) a = fmaf(s.u.kbuf[i * Zn + j], s.q[j], a);
                s.wb[i] = a;
            }
            if (lane < Zn) {
                float a = 0.0f;
                for (int i = 0; i < A; ++i) a = fmaf(s.u.kbuf[i * Zn + lane], s.w[i], a);
                s.qb[lane] = a;
            }
            __syncwarp();
        }
        gr[0] = rowinfo[row * 4 + 0];
        gr[9] = rowinfo[row * 4 + 1];
        gr[10] = rowinfo[row * 4 + 2];
        gr[11] = rowinfo[row * 4 + 3];
        age_met_adjoint(c, s, g.lT10[gi], M, p, gr);
        float gzt = 0.0f;          // d log L / dz through t_obs (age bins, M, burst clipping)
        if (rowz)
            gzt = rowz[row] + g.dtdz[gi] * tobs_adjoint(c, s.view(c), g.bins + (size_t)gi * A, g.lnT[gi],
                                                         g.lT10[gi], M, p.th);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < SPS_NPARAM; ++k) grad_out[row * NG + k] = gr[k];
            if (rowz) grad_out[row * NG + SPS_NPARAM] = gzt;
        }
        __syncwarp();
    }
}

int blocks_rows(int64_t rows, int per_block) {
    int64_t b = (rows + per_block - 1) / per_block;
    if (b > 152LL * 64) b = 152LL * 64;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_exact_weights(const Consts& c, const Grid& grid, const Galaxies& g,
                                 const float* theta, const int32_t* gal_idx, int64_t n, int bf16,
                                 float* W32, uint16_t* Wbf, cudaStream_t s, const int32_t* pos_of,
                                 float* W32lo, float* keep) {
    if (n <= 0) return cudaSuccess;
    k_weights<<<blocks_rows(n, kWarpsApprox), 32 * kWarpsApprox, 0, s>>>(c, grid, g, theta, gal_idx,
                                                                         n, bf16, W32, Wbf, pos_of, W32lo,
                                                                         keep);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- redshift order
// Rows bucketed by log(1 + z) of their galaxy (2048 buckets over [0, 2.5]),
// so that the rows of a tensor-core tile see nearly the same band supports.
constexpr int kZBuckets = 2048;

int zsort_buckets() { return kZBuckets; }

namespace {
__device__ __forceinline__ int zbucket(const Galaxies& g, const int32_t* gal_idx, int64_t row) {
    const int64_t gi = gal_idx ? (int64_t)gal_idx[row] : row;
    const float z = (gi >= 0 && gi < g.n) ? g.z[gi] : 0.0f;
    const float u = log1pf(fmaxf(z, 0.0f)) * ((float)kZBuckets / 2.5f);
    return (u < (float)(kZBuckets - 1)) ? (int)u : kZBuckets - 1;   // NaN goes last
}
__global__ void k_zcount(const Galaxies g, const int32_t* __restrict__ gal_idx, int64_t n, int32_t* counts) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row < n) atomicAdd(&counts[zbucket(g, gal_idx, row)], 1);
}
// Exclusive scan of the bucket counts in place (one block of 1024 threads).
__global__ void __launch_bounds__(1024) k_zscan(int32_t* counts) {
    __shared__ int32_t part[1024];
    const int t = threadIdx.x;
    const int a = counts[2 * t], b = counts[2 * t + 1];
    part[t] = a + b;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = (t >= o) ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    const int base = part[t] - (a + b);
    counts[2 * t] = base;
    counts[2 * t + 1] = base + a;
}
__global__ void k_zscatter(const Galaxies g, const int32_t* __restrict__ gal_idx, int64_t n, int32_t* cursor,
                           int32_t* __restrict__ perm, int32_t* __restrict__ pos_of) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int pos = atomicAdd(&cursor[zbucket(g, gal_idx, row)], 1);
    perm[pos] = (int32_t)row;
    pos_of[row] = pos;
}
}  // namespace

cudaError_t launch_zsort(const Galaxies& g, const int32_t* gal_idx, int64_t n, int32_t* perm,
                         int32_t* pos_of, int32_t* counts, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    static_assert(kZBuckets == 2 * 1024, "scan layout");
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * kZBuckets, s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_zcount<<<blocks, 256, 0, s>>>(g, gal_idx, n, counts);
    k_zscan<<<1, 1024, 0, s>>>(counts);
    k_zscatter<<<blocks, 256, 0, s>>>(g, gal_idx, n, counts, perm, pos_of);
    return cudaGetLastError();
}

cudaError_t launch_exact_fwd(const Consts& c, const Grid& grid, const Galaxies& g,
                             const float* theta, const int32_t* gal_idx, int64_t n, int bf16,
                             const float* W32, const uint16_t* Wbf, float* cJ, cudaStream_t s,
                             float* cJz) {
    if (n <= 0) return cudaSuccess;
    const bool kz = cJz != nullptr;
    const size_t dyn = (size_t)kBM * c.n_band *
                       (4 * sizeof(float) + sizeof(int2) + sizeof(float2) + (kz ? 3 * sizeof(float) : 0));
    const unsigned grid_m = (unsigned)((n + kBM - 1) / kBM);
    auto go = [&](auto kern, const auto* Wp, const auto* Lp) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        kern<<<grid_m, kThreads, dyn, s>>>(c, grid, g, theta, gal_idx, n, Wp, Lp, cJ, cJz);
    };
    if (bf16)
        kz ? go(k_exact_fwd<uint16_t, true>, Wbf, grid.ssp_bf) : go(k_exact_fwd<uint16_t, false>, Wbf, grid.ssp_bf);
    else
        kz ? go(k_exact_fwd<float, true>, W32, grid.ssp) : go(k_exact_fwd<float, false>, W32, grid.ssp);
    return cudaGetLastError();
}

cudaError_t launch_exact_like(const Consts& c, const Galaxies& g, const float* theta,
                              const int32_t* gal_idx, int64_t n, const float* cJ, float* rowinfo,
                              const float* mag_obs, const float* sigma, const uint32_t* mask,
                              float* mag_out, float* loglike_out, float* gbar, int* nonfinite,
                              cudaStream_t s, const float* cJz, float* rowz, double* ll64_out) {
    if (n <= 0) return cudaSuccess;
    k_exact_like<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(c, g, theta, gal_idx, n, cJ, mag_obs,
                                                             sigma, mask, mag_out, loglike_out, gbar,
                                                             rowinfo, nonfinite, cJz, rowz, ll64_out);
    return cudaGetLastError();
}

cudaError_t launch_exact_vgen(const Consts& c, const Grid& grid, const Galaxies& g,
                              const float* theta, const int32_t* gal_idx, int64_t n,
                              const float* gbar, float* V32, uint16_t* Vbf, cudaStream_t s, float* V32lo) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * (size_t)c.lam_pad;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_exact_vgen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_exact_vgen<<<(unsigned)n, 256, smem, s>>>(c, grid, g, theta, gal_idx, n, gbar, V32, Vbf, V32lo);
    return cudaGetLastError();
}

cudaError_t launch_exact_adj(const Consts& c, const Grid& grid, int64_t n, int bf16,
                             const float* V32, float* Wbar, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    dim3 grd((unsigned)((n + kBM - 1) / kBM), (unsigned)((c.K + kBN - 1) / kBN));
    if (bf16)
        k_exact_adj<uint16_t><<<grd, kThreads, 0, s>>>(c, grid, n, V32, grid.ssp_t_bf, 1, Wbar);
    else
        k_exact_adj<float><<<grd, kThreads, 0, s>>>(c, grid, n, V32, grid.ssp_t, 0, Wbar);
    return cudaGetLastError();
}

cudaError_t launch_exact_grad(const Consts& c, const Galaxies& g, const float* theta,
                              const int32_t* gal_idx, int64_t n, const float* rowinfo,
                              const float* Wbar, float* grad_out, cudaStream_t s, const float* rowz,
                              const float* keep) {
    if (n <= 0) return cudaSuccess;
    k_exact_grad<<<blocks_rows(n, kWarpsApprox), 32 * kWarpsApprox, 0, s>>>(c, g, theta, gal_idx, n,
                                                                            rowinfo, Wbar, grad_out, rowz, keep);
    return cudaGetLastError();
}

}  // namespace sps
