// Per-galaxy preparation (once per galaxy set, FP64) and the per-galaxy
// c_SSP table of the approximate path (the c_SSP definition of Sec. 3).
#include <cuda_runtime.h>
#include <math.h>

#include "band_tab.cuh"
#include "sps_internal.h"

namespace sps {

namespace {

constexpr double kMpcCm = 3.0856775814913673e24;
constexpr double kMpcKm = 3.0856775814913673e19;
constexpr double kGyrS = 3.15576e16;
constexpr double kCkms = 299792.458;
constexpr double kLsun = 3.828e33;
constexpr double kAbZp = 3631e-23;
constexpr double kFwhmToSigma = 0.42466090014400953;  // 1 / (2 sqrt(2 ln 2))
constexpr int kPrepThreads = 256;

// Calzetti et al. (2000) k'(lambda), R_V = 4.05, clamped at zero; Drude bump
// of unit amplitude at 0.2175 um with width 0.035 um (App. A.3).
__device__ double calzetti_k0(double lum) {
    double k = (lum < 0.63)
                   ? 2.659 * (-2.156 + 1.509 / lum - 0.198 / (lum * lum) + 0.011 / (lum * lum * lum)) + 4.05
                   : 2.659 * (-1.857 + 1.040 / lum) + 4.05;
    return k > 0.0 ? k : 0.0;
}
__device__ double drude_shape(double lum) {
    double x = (lum * 0.035) * (lum * 0.035);
    double d = lum * lum - 0.2175 * 0.2175;
    return x / (d * d + x);
}

// d k0 / d lambda and d D / d lambda [per um] of the two curves above.
__device__ double calzetti_dk0(double lum) {
    if (calzetti_k0(lum) <= 0.0) return 0.0;
    const double i1 = 1.0 / lum, i2 = i1 * i1;
    return (lum < 0.63) ? 2.659 * (-1.509 * i2 + 2.0 * 0.198 * i2 * i1 - 3.0 * 0.011 * i2 * i2)
                        : 2.659 * (-1.040 * i2);
}
__device__ double drude_dshape(double lum) {
    const double x = (lum * 0.035) * (lum * 0.035);
    const double dx = 2.0 * 0.035 * 0.035 * lum;
    const double d = lum * lum - 0.2175 * 0.2175;
    const double dd = 2.0 * lum;
    const double den = d * d + x;
    return (dx * d * d - 2.0 * x * d * dd) / (den * den);
}

template <typename T>
__device__ T block_sum(T v, T* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    T t = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : (T)0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    T r = sh[0];
    __syncthreads();
    return r;
}

// Per-wavelength constants: (q_n / lambda_n, k0, ln(lambda/lambda_V), Drude).
__global__ void k_lambda_consts(const double* __restrict__ lam, int L, float4* __restrict__ out,
                                float* __restrict__ lam32, float2* __restrict__ lamq) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= L) return;
    double l = lam[n];
    double q = (n == 0) ? 0.5 * (lam[1] - lam[0])
             : (n == L - 1) ? 0.5 * (lam[L - 1] - lam[L - 2])
                            : 0.5 * (lam[n + 1] - lam[n - 1]);
    double lum = l * 1e-4;
    out[n] = make_float4((float)(q / l), (float)calzetti_k0(lum), (float)log(l / 5500.0),
                         (float)drude_shape(lum));
    lam32[n] = (float)l;
    lamq[n] = make_float2((float)l, (float)(q / l));
}

// One block per galaxy.
__global__ void __launch_bounds__(kPrepThreads)
k_prepare(const __grid_constant__ Consts c, const double* __restrict__ lam,
          const double* __restrict__ band_p0, const double* __restrict__ band_p1,
          const double* __restrict__ tabT, const double* __restrict__ age_edges_yr,
          const float* __restrict__ zin, int64_t G,
          double h0, double om, float* __restrict__ lnT_out, float* __restrict__ lT10_out,
          float2* __restrict__ bins, double* __restrict__ zp, int2* __restrict__ support,
          float2* __restrict__ gauss, float4* __restrict__ dust_eff, float* __restrict__ dtdz,
          float* __restrict__ dzp, float4* __restrict__ ddust) {
    __shared__ double shd[32];
    __shared__ int shmin, shmax;
    const int64_t g = blockIdx.x;
    if (g >= G) return;
    const double z = (double)zin[g];
    const double opz = 1.0 + z;
    const double ol = 1.0 - om;
    const double th = kMpcKm / h0 / kGyrS;                    // Hubble time [Gyr]
    // age of a flat matter + Lambda universe (closed form)
    const double t_obs = (2.0 / (3.0 * sqrt(ol))) * th * asinh(sqrt(ol / om) * pow(opz, -1.5));
    // comoving distance: composite Simpson on 2 * kPrepThreads intervals of 1/E(z)
    double part = 0.0;
    {
        const int nint = 2 * kPrepThreads;
        const double h = z / nint;
        for (int k = threadIdx.x; k <= nint; k += blockDim.x) {
            double x = h * k;
            double f = 1.0 / sqrt(om * (1 + x) * (1 + x) * (1 + x) + ol);
            double wgt = (k == 0 || k == nint) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
            part += wgt * f;
        }
        part *= h / 3.0;
    }
    const double dc = block_sum(part, shd) * (kCkms / h0);    // Mpc
    const double dl_cm = opz * dc * kMpcCm;
    const double T_yr = t_obs * 1e9;
    // redshift derivatives: dt/dz = -1 / ((1+z) H(z)); d ln d_L / dz = 1/(1+z) + (c/H0) / (E d_C)
    const double Ez = sqrt(om * opz * opz * opz + ol);
    const double dlnDL = 1.0 / opz + (kCkms / h0) / (Ez * dc);
    if (threadIdx.x == 0) {
        lnT_out[g] = (float)log(t_obs);
        lT10_out[g] = (float)log10(T_yr);
        dtdz[g] = (float)(-th / (opz * Ez));
    }
    // age bins in cosmic time (Eq. smoothPsfh): ages [min(E_i,T), min(E_{i+1},T)]
    for (int i = threadIdx.x; i < c.n_age; i += blockDim.x) {
        double e0 = age_edges_yr[i], e1 = age_edges_yr[i + 1];
        float2 b = make_float2(0.f, 0.f);
        if (e0 < T_yr) {
            double lo_age = e0;
            double hi_age = (e1 < T_yr) ? e1 : T_yr;
            double t_hi = (T_yr - lo_age) * 1e-9;
            if (e1 >= T_yr) {
                b = make_float2((float)log(t_hi), -1.0f);               // reaches t = 0
            } else {
                double t_lo = (T_yr - hi_age) * 1e-9;
                double c0 = 0.5 * (log(t_lo) + log(t_hi));
                double hw = 0.5 * log1p((hi_age - lo_age) / (T_yr - hi_age));
                b = make_float2((float)c0, (float)hw);
            }
        }
        bins[g * c.n_age + i] = b;
    }
    // bands: support, N_b, lambda_eff, zero point
    const int L = c.n_lam;
    for (int b = 0; b < c.n_band; ++b) {
        const double p0 = band_p0[b], p1 = band_p1[b];
        const int kind = c.band_kind[b];
        const double sg = p1 * kFwhmToSigma;
        if (threadIdx.x == 0) {
            shmin = L;
            shmax = -1;
        }
        __syncthreads();
        double sN = 0.0, sQT = 0.0, sQTL = 0.0;
        double sNd = 0.0, sQTd = 0.0, sQTLd = 0.0;              // their z derivatives over lambda
        int lo = L, hi = -1;
        for (int n = threadIdx.x; n < L; n += blockDim.x) {
            const double l = lam[n];
            const double lo_ = opz * l;                             // observed wavelength
            double T, Td;                                           // T and dT / d lambda_obs
            bool in;
            if (kind == 0) {
                in = (lo_ >= p0) && (lo_ < p1);
                T = in ? 1.0 : 0.0;
                Td = 0.0;
            } else if (kind == 1) {
                // Gaussian support: |u| < 6 drops 2e-9 of the band's weight, below
                // FP32 rounding; zero point and fluxes use the same support
                double u = (lo_ - p0) / sg;
                in = fabs(u) < 6.0;
                T = in ? exp(-0.5 * u * u) : 0.0;
                Td = -u / sg * T;
            } else {
                const double u = (lo_ - p0) / p1;
                in = u >= 0.0 && u <= (double)(c.tab_n[b] - 1);
                T = tab_T64(tabT + c.tab_off[b], c.tab_n[b], u);
                Td = tab_dT64(tabT + c.tab_off[b], c.tab_n[b], u) / p1;
            }
            if (in) {
                double q = (n == 0) ? 0.5 * (lam[1] - lam[0])
                         : (n == L - 1) ? 0.5 * (lam[L - 1] - lam[L - 2])
                                        : 0.5 * (lam[n + 1] - lam[n - 1]);
                sN += q * T / l;
                sQT += q * T;
                sQTL += q * T * l;
                // d T((1+z) l) / dz = l T'
                sNd += q * Td;
                sQTd += q * Td * l;
                sQTLd += q * Td * l * l;
                lo = min(lo, n);
                hi = max(hi, n);
            }
        }
        if (lo < L) atomicMin(&shmin, lo);
        if (hi >= 0) atomicMax(&shmax, hi);
        sN = block_sum(sN, shd);
        sQT = block_sum(sQT, shd);
        sQTL = block_sum(sQTL, shd);
        sNd = block_sum(sNd, shd);
        sQTd = block_sum(sQTd, shd);
        sQTLd = block_sum(sQTLd, shd);
        if (threadIdx.x == 0) {
            const size_t gb = (size_t)g * c.n_band + b;
            const double K = opz * kLsun / (4.0 * M_PI * dl_cm * dl_cm * kAbZp * sN);
            zp[gb] = -2.5 * log10(K);
            support[gb] = (shmax >= 0) ? make_int2(shmin, shmax + 1) : make_int2(0, 0);
            // (rest centre, (1+z)/s) of a Gaussian; (rest start, -(1+z)/step) of a table
            gauss[gb] = (kind == 2) ? make_float2((float)(p0 / opz), (float)(-opz / p1))
                                    : make_float2((float)(p0 / opz), (float)(opz / sg));
            const double le = sQTL / sQT;                           // rest-frame lambda_eff
            const double lum = le * 1e-4;
            dust_eff[gb] = make_float4((float)calzetti_k0(lum), (float)log(le / 5500.0),
                                       (float)drude_shape(lum), (float)le);
            // zp = -2.5 log10((1+z) L_sun / (4 pi d_L^2 3631 Jy N_b))
            dzp[gb] = (float)(-2.5 / M_LN10 * (1.0 / opz - 2.0 * dlnDL - sNd / sN));
            const double dle = (sQTLd * sQT - sQTL * sQTd) / (sQT * sQT);   // d lambda_eff / dz
            ddust[gb] = make_float4((float)(calzetti_dk0(lum) * 1e-4 * dle), (float)(dle / le),
                                    (float)(drude_dshape(lum) * 1e-4 * dle), 0.0f);
        }
        __syncthreads();
    }
}

// c_SSP[g][b][k] = sum_n (q_n/lambda_n) T_b((1+z_g) lambda_n) L[k][n]: one block
// per (galaxy, 128-wide k tile), band weights staged in shared memory.  This
// runs once per galaxy set, so it is written for accuracy: the Gaussian
// argument is formed in FP64, the weight uses the accurate expf, and FP32
// partial sums of 32 terms are accumulated in FP64.
constexpr int kCsspK = 128;
constexpr int kCsspChunk = 256;
__global__ void __launch_bounds__(kCsspK)
k_cssp(const __grid_constant__ Consts c, const Grid grid, const Galaxies gal,
       const double* __restrict__ band_p0, const double* __restrict__ band_p1, float* __restrict__ out,
       int deriv) {
    __shared__ float wsh[kCsspChunk];
    const int64_t g = blockIdx.x;
    const int k = blockIdx.y * kCsspK + threadIdx.x;
    const double opz = 1.0 + (double)gal.z[g];
    for (int b = 0; b < c.n_band; ++b) {
        const size_t gb = (size_t)g * c.n_band + b;
        const int2 sup = gal.support[gb];
        const double crest = band_p0[b] / opz;
        const double inv = (double)gal.gauss[gb].y;
        const int kind = c.band_kind[b];
        double acc = 0.0;
        for (int n0 = sup.x; n0 < sup.y; n0 += kCsspChunk) {
            __syncthreads();
            for (int t = threadIdx.x; t < kCsspChunk; t += blockDim.x) {
                int n = n0 + t;
                float w = 0.0f;
                if (n < sup.y && !deriv) {
                    float4 lc = grid.lamc[n];
                    if (kind == 0) {
                        w = lc.x;
                    } else if (kind == 1) {
                        float u = (float)((grid.lam64[n] - crest) * inv);
                        w = lc.x * expf(-0.5f * u * u);
                    } else {
                        const double u = (opz * grid.lam64[n] - band_p0[b]) / band_p1[b];
                        w = (float)((double)lc.x * tab_T64(grid.band_T64 + c.tab_off[b], c.tab_n[b], u));
                    }
                } else if (n < sup.y) {
                    // d/dz of (q_n / l_n) T((1+z) l_n) = q_n T'((1+z) l_n): zero for a top-hat
                    const double ql = (double)grid.lamc[n].x * grid.lam64[n];
                    if (kind == 1) {
                        const double u = (grid.lam64[n] - crest) * inv;
                        w = (float)(-ql * u * (inv / opz) * exp(-0.5 * u * u));
                    } else if (kind == 2) {
                        const double u = (opz * grid.lam64[n] - band_p0[b]) / band_p1[b];
                        w = (float)(ql * tab_dT64(grid.band_T64 + c.tab_off[b], c.tab_n[b], u) / band_p1[b]);
                    }
                }
                wsh[t] = w;
            }
            __syncthreads();
            if (k < c.K) {
                const int nn = min(kCsspChunk, sup.y - n0);
                const float* col = grid.ssp_t + (size_t)n0 * c.k_pad + k;
                for (int t0 = 0; t0 < nn; t0 += 32) {
                    float part = 0.0f;
                    const int te = min(t0 + 32, nn);
                    for (int t = t0; t < te; ++t) part = fmaf(wsh[t], col[(size_t)t * c.k_pad], part);
                    acc += (double)part;
                }
            }
        }
        if (k < c.K) out[gb * c.K + k] = (float)acc;
    }
}

}  // namespace

cudaError_t launch_lambda_consts(const double* lam, int L, float4* out, float* lam32, float2* lamq,
                                 cudaStream_t s) {
    k_lambda_consts<<<(L + 255) / 256, 256, 0, s>>>(lam, L, out, lam32, lamq);
    return cudaGetLastError();
}

cudaError_t launch_prepare_galaxies(const Consts& c, const Grid& grid, const double* lam64,
                                    const double* band_p0, const double* band_p1,
                                    const double* age_edges_yr, const float* z, int64_t n_gal,
                                    double h0, double om, float* lnT, float* lT10, float2* bins,
                                    double* zp, int2* support, float2* gauss, float4* dust_eff,
                                    float* dtdz, float* dzp, float4* ddust, cudaStream_t s) {
    if (n_gal <= 0) return cudaSuccess;
    k_prepare<<<(unsigned)n_gal, kPrepThreads, 0, s>>>(c, lam64, band_p0, band_p1, grid.band_T64, age_edges_yr,
                                                       z, n_gal, h0, om, lnT, lT10, bins, zp, support,
                                                       gauss, dust_eff, dtdz, dzp, ddust);
    return cudaGetLastError();
}

cudaError_t launch_cssp(const Consts& c, const Grid& grid, const Galaxies& g,
                        const double* band_p0, const double* band_p1, float* cssp, cudaStream_t s,
                        int deriv) {
    if (g.n <= 0) return cudaSuccess;
    dim3 grd((unsigned)g.n, (c.K + kCsspK - 1) / kCsspK);
    k_cssp<<<grd, kCsspK, 0, s>>>(c, grid, g, band_p0, band_p1, cssp, deriv);
    return cudaGetLastError();
}

}  // namespace sps
