// Host runtime behind the C ABI of include/sps.h: context and table upload,
// argument checks, host/device pointer detection and staging, chunked
// dispatch of the exact path, the HMC launch (graph capture, autotuned launch
// shape) and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "ctx.h"
#include "sps_internal.h"

using namespace sps;

namespace {

thread_local std::string g_last_error;

sps_status fail(sps_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}
}  // namespace

void sps::set_last_error(const char* msg) { g_last_error = msg; }

namespace {

sps_status cuda_fail(cudaError_t e, const char* where) {
    return fail(SPS_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(call)                                              \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);   \
    } while (0)

}  // namespace

int sps::pointer_location(const void* p, int device) {
    if (!p) return 0;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    if (a.type == cudaMemoryTypeDevice) return a.device == device ? 1 : -1;
    return 0;
}

namespace {

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

uint16_t bf16_rne(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2D BF16 tensor [rows][inner] (row stride `ld` elements), box {64, box_rows},
// 128-byte swizzle, zero fill outside the tensor.
bool make_tmap_bf16(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint64_t ld,
                    uint32_t box_rows) {
    auto enc = tmap_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {ld * 2};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2D FP32 tensor [rows][inner] (row stride `ld` elements), box {32, box_rows}
// (128-byte rows), 128-byte swizzle, zero fill outside the tensor.
bool make_tmap_f32(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint64_t ld,
                   uint32_t box_rows) {
    auto enc = tmap_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {ld * 4};
    cuuint32_t box[2] = {32, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// hi = x rounded to nearest (ties away) to TF32, lo = x - hi.
void tf32_split_host(float x, float& hi, float& lo) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) {      // finite: round at mantissa bit 13
        u += 0x1000u;
        u &= 0xffffe000u;
    }
    std::memcpy(&hi, &u, 4);
    lo = x - hi;
}

}  // namespace

namespace {

// Staging of host arrays: in() returns a device pointer holding the data,
// out() a device pointer whose contents are copied back by finish().
struct Stager {
    sps_ctx* ctx;
    cudaStream_t s;
    int slot = 0;
    bool any_host = false;
    struct Back {
        void* host;
        const void* dev;
        size_t bytes;
    };
    std::vector<Back> back;
    cudaError_t err = cudaSuccess;
    bool foreign = false;    // an argument lives in another device's memory

    // 1: use p as it is; 0: stage it; -1: reject it
    int where(const void* p, size_t count) {
        if (!p || count == 0) return 1;
        const int w = pointer_location(p, ctx->device);
        if (w < 0) foreign = true;
        return w;
    }
    template <typename T>
    const T* in(const T* p, size_t count) {
        const int w = where(p, count);
        if (w != 0) return w > 0 ? p : nullptr;
        any_host = true;
        DevBuf& b = ctx->stage[slot++];
        if ((err = b.reserve(count * sizeof(T))) != cudaSuccess) return nullptr;
        if ((err = cudaMemcpyAsync(b.p, p, count * sizeof(T), cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return nullptr;
        return b.as<T>();
    }
    template <typename T>
    T* out(T* p, size_t count) {
        const int w = where(p, count);
        if (w != 0) return w > 0 ? p : nullptr;
        any_host = true;
        DevBuf& b = ctx->stage[slot++];
        if ((err = b.reserve(count * sizeof(T))) != cudaSuccess) return nullptr;
        back.push_back({p, b.p, count * sizeof(T)});
        return b.as<T>();
    }
    sps_status check() const {
        if (foreign)
            return fail(SPS_E_INVALID_ARG, "an array argument lives in the memory of another device "
                                           "than the context's");
        if (err != cudaSuccess) return cuda_fail(err, "staging");
        return SPS_OK;
    }
    cudaError_t finish() {
        for (auto& bk : back) {
            cudaError_t e = cudaMemcpyAsync(bk.host, bk.dev, bk.bytes, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return e;
        }
        if (any_host) return cudaStreamSynchronize(s);
        return cudaSuccess;
    }
};

sps_status check_rows(const sps_ctx* ctx, const float* theta, const int32_t* gal_idx, int64_t n) {
    if (!ctx) return fail(SPS_E_INVALID_ARG, "null context");
    if (ctx->n_gal <= 0) return fail(SPS_E_STATE, "no galaxy set: call sps_set_galaxies first");
    if (n < 0) return fail(SPS_E_SHAPE, "negative row count");
    if (n == 0) return SPS_OK;
    if (!theta) return fail(SPS_E_INVALID_ARG, "theta is NULL");
    if (!gal_idx && n != ctx->n_gal)
        return fail(SPS_E_SHAPE, "gal_idx is NULL but n differs from the galaxy count");
    const int gw = gal_idx && n > 0 ? pointer_location(gal_idx, ctx->device) : 1;
    if (gw < 0) return fail(SPS_E_INVALID_ARG, "gal_idx lives in the memory of another device");
    if (gw == 0) {
        for (int64_t i = 0; i < n; ++i)
            if (gal_idx[i] < 0 || gal_idx[i] >= ctx->n_gal)
                return fail(SPS_E_SHAPE, "gal_idx out of range at row " + std::to_string(i));
    }
    return SPS_OK;
}

}  // namespace

extern "C" {

const char* sps_error_string(sps_status s) {
    switch (s) {
        case SPS_OK: return "ok";
        case SPS_E_INVALID_ARG: return "invalid argument";
        case SPS_E_SHAPE: return "shape or size out of range";
        case SPS_E_NONFINITE: return "non-finite inputs gave NaN rows";
        case SPS_E_CUDA: return "CUDA error";
        case SPS_E_TIMEOUT: return "bounded device wait timed out";
        case SPS_E_UNSUPPORTED: return "unsupported mode, precision or device";
        case SPS_E_STATE: return "call order (state) error";
        case SPS_E_NOMEM: return "device allocation failed";
    }
    return "unknown status";
}

const char* sps_last_error_message(void) { return g_last_error.c_str(); }

sps_status sps_config_default(sps_config* cfg) {
    if (!cfg) return fail(SPS_E_INVALID_ARG, "null config");
    static const double lo[SPS_NPARAM] = {-1.5, 0.5, 0.1, 0.1, 0.0, 6.0, 0.05, -2.0, 0.05, 0.0, -1.0, 0.0};
    static const double hi[SPS_NPARAM] = {2.5, 12.0, 5.0, 5.0, 0.2, 8.5, 1.5, 0.2, 0.5, 3.0, 0.4, 0.5};
    cfg->h0_kms_mpc = 70.0;
    cfg->omega_m = 0.3;
    for (int k = 0; k < SPS_NPARAM; ++k) {
        cfg->prior_lo[k] = lo[k];
        cfg->prior_hi[k] = hi[k];
    }
    cfg->device = 0;
    cfg->sfh_gl_order = 6;
    cfg->sfh_panel = 0.25;
    for (int k = 0; k < SPS_NPARAM; ++k) {
        cfg->sigmoid_k[k] = 1.0;
        cfg->sigmoid_x0[k] = 0.0;
        cfg->skew_xi[k] = 0.0;
        cfg->skew_omega[k] = 1.0;
        cfg->skew_s[k] = 0.0;
    }
    cfg->prior = SPS_PRIOR_UNIFORM;
    return SPS_OK;
}

sps_status sps_hmc_config_default(sps_hmc_config* cfg) {
    if (!cfg) return fail(SPS_E_INVALID_ARG, "null config");
    cfg->chains_per_gal = 4;
    cfg->n_warm = 500;
    cfg->n_samp = 500;
    cfg->L_min = 8;
    cfg->L_max = 64;
    cfg->target_accept = 0.8f;
    cfg->eps0 = 0.1f;
    cfg->seed = 2506199190ull;
    cfg->mode = SPS_APPROX;
    cfg->prec = SPS_FP32;
    cfg->use_graph = 1;
    cfg->autotune = 1;
    cfg->adapt_mass = 0;
    cfg->sampler = SPS_HMC;
    cfg->max_depth = 10;
    return SPS_OK;
}

sps_status sps_create(sps_ctx** out, const sps_tables* t, const sps_config* cfg_in) {
    if (!out || !t) return fail(SPS_E_INVALID_ARG, "null argument");
    *out = nullptr;
    sps_config cfg;
    if (cfg_in) cfg = *cfg_in;
    else sps_config_default(&cfg);
    const int A = t->n_age, Zn = t->n_met, L = t->n_lam, B = t->n_band;
    if (A < 2 || A > SPS_MAX_AGES) return fail(SPS_E_SHAPE, "n_age must be in [2, 128]");
    if (Zn < 1 || Zn > SPS_MAX_METS) return fail(SPS_E_SHAPE, "n_met must be in [1, 32]");
    if (L < 2) return fail(SPS_E_SHAPE, "n_lam must be >= 2");
    if (B < 1 || B > SPS_MAX_BANDS) return fail(SPS_E_SHAPE, "n_band must be in [1, 32]");
    if (A * Zn > kKTileMax * 32) return fail(SPS_E_SHAPE, "n_age * n_met must be <= 1312");
    if (!t->age_yr || !t->lgZ || !t->lam_ang || !t->ssp || !t->band_kind || !t->band_p0 || !t->band_p1)
        return fail(SPS_E_INVALID_ARG, "null table pointer");
    for (int i = 0; i < A; ++i)
        if (!(t->age_yr[i] > 0) || (i && !(t->age_yr[i] > t->age_yr[i - 1])))
            return fail(SPS_E_INVALID_ARG, "age grid must be positive and increasing");
    for (int j = 1; j < Zn; ++j)
        if (!(t->lgZ[j] > t->lgZ[j - 1])) return fail(SPS_E_INVALID_ARG, "lgZ grid must increase");
    for (int n = 0; n < L; ++n)
        if (!(t->lam_ang[n] > 0) || (n && !(t->lam_ang[n] > t->lam_ang[n - 1])))
            return fail(SPS_E_INVALID_ARG, "wavelength grid must be positive and increasing");
    if (t->mdf_offset)
        for (int i = 0; i < A; ++i)
            if (!std::isfinite(t->mdf_offset[i]) || std::fabs(t->mdf_offset[i]) > 10.0)
                return fail(SPS_E_INVALID_ARG, "mdf_offset must be finite, |offset| <= 10 dex");
    int64_t n_tab = 0;                        // tabulated samples in all
    for (int b = 0; b < B; ++b) {
        int k = t->band_kind[b];
        if (k != SPS_BAND_TOPHAT && k != SPS_BAND_GAUSS && k != SPS_BAND_TABLE)
            return fail(SPS_E_INVALID_ARG, "bad band kind");
        if (k == SPS_BAND_TOPHAT && !(t->band_p1[b] > t->band_p0[b] && t->band_p0[b] > 0))
            return fail(SPS_E_INVALID_ARG, "top-hat band needs 0 < p0 < p1");
        if (k == SPS_BAND_GAUSS && !(t->band_p1[b] > 0 && t->band_p0[b] > 0))
            return fail(SPS_E_INVALID_ARG, "Gaussian band needs positive centre and FWHM");
        if (k == SPS_BAND_TABLE) {
            if (!t->band_tab_n || !t->band_tab_T) return fail(SPS_E_INVALID_ARG, "tabulated band without samples");
            if (!(t->band_p0[b] > 0 && t->band_p1[b] > 0) || t->band_tab_n[b] < 2 || t->band_tab_n[b] > (1 << 20))
                return fail(SPS_E_INVALID_ARG, "tabulated band needs start > 0, step > 0 and 2..2^20 samples");
            for (int m = 0; m < t->band_tab_n[b]; ++m) {
                const double v = t->band_tab_T[n_tab + m];
                if (!std::isfinite(v) || v < 0) return fail(SPS_E_INVALID_ARG, "tabulated transmission must be finite and >= 0");
            }
            n_tab += t->band_tab_n[b];
        }
    }
    const size_t K = (size_t)A * Zn;
    for (size_t e = 0; e < K * L; ++e)
        if (!std::isfinite(t->ssp[e]) || t->ssp[e] < 0) return fail(SPS_E_INVALID_ARG, "SSP table must be finite and >= 0");
    if (cfg.sfh_gl_order < 2 || cfg.sfh_gl_order > kMaxGL) return fail(SPS_E_INVALID_ARG, "sfh_gl_order in [2, 16]");
    if (!(cfg.sfh_panel > 0 && cfg.sfh_panel <= 2.0)) return fail(SPS_E_INVALID_ARG, "sfh_panel in (0, 2]");
    if (!(cfg.h0_kms_mpc > 0) || !(cfg.omega_m > 0 && cfg.omega_m < 1))
        return fail(SPS_E_INVALID_ARG, "cosmology out of range");
    for (int k = 0; k < SPS_NPARAM; ++k) {
        if (!(cfg.prior_hi[k] > cfg.prior_lo[k])) return fail(SPS_E_INVALID_ARG, "prior_hi must exceed prior_lo");
        if (!(cfg.sigmoid_k[k] > 0) || !std::isfinite(cfg.sigmoid_k[k]) || !std::isfinite(cfg.sigmoid_x0[k]))
            return fail(SPS_E_INVALID_ARG, "sigmoid_k must be finite and > 0, sigmoid_x0 finite");
        if (cfg.prior == SPS_PRIOR_SKEWNORMAL &&
            (!(cfg.skew_omega[k] > 0) || !std::isfinite(cfg.skew_omega[k]) || !std::isfinite(cfg.skew_xi[k]) ||
             !std::isfinite(cfg.skew_s[k])))
            return fail(SPS_E_INVALID_ARG, "skew-normal prior needs finite xi, s and omega > 0");
    }
    if (cfg.prior != SPS_PRIOR_UNIFORM && cfg.prior != SPS_PRIOR_SKEWNORMAL)
        return fail(SPS_E_INVALID_ARG, "prior");
    // Worst-case SFH panel count per row: every bin one panel plus the log-time
    // range down to the truncation point (at most ~45 in ln t) in panels.
    const int max_panels = A + (int)std::ceil(48.0 / cfg.sfh_panel) + 2;
    if (max_panels > kMaxPanels) return fail(SPS_E_INVALID_ARG, "sfh_panel too small for the panel budget");

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(SPS_E_UNSUPPORTED, "no CUDA device");
    }
    if (cfg.device < 0 || cfg.device >= ndev) return fail(SPS_E_INVALID_ARG, "bad device ordinal");
    DeviceGuard dg(cfg.device);
    CK(dg.err);
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, cfg.device));
    if (prop.major < 10) return fail(SPS_E_UNSUPPORTED, "needs a Blackwell (sm_100+) device");

    sps_ctx* ctx = new sps_ctx();
    ctx->device = cfg.device;
    ctx->h0 = cfg.h0_kms_mpc;
    ctx->om = cfg.omega_m;
    Consts& c = ctx->c;
    c.n_age = A;
    c.n_met = Zn;
    c.n_lam = L;
    c.n_band = B;
    c.K = (int)K;
    c.k_pad = (int)((K + 63) / 64 * 64);   // k-blocks of 64 BF16 (128-byte TMA rows)
    c.lam_pad = (L + 31) / 32 * 32;
    c.gl_order = cfg.sfh_gl_order;
    c.panel = (float)cfg.sfh_panel;
    gauss_legendre(c.gl_order, ctx->gl_x, ctx->gl_w);
    for (int i = 0; i < c.gl_order; ++i) {
        c.gl_x[i] = (float)ctx->gl_x[i];
        c.gl_w[i] = (float)ctx->gl_w[i];
    }
    {
        double x2[2], w2[2], x3[3], w3[3];
        gauss_legendre(2, x2, w2);
        gauss_legendre(3, x3, w3);
        for (int i = 0; i < 2; ++i) {
            c.gl2_x[i] = (float)x2[i];
            c.gl2_w[i] = (float)w2[i];
        }
        for (int i = 0; i < 3; ++i) {
            c.gl3_x[i] = (float)x3[i];
            c.gl3_w[i] = (float)w3[i];
        }
    }
    std::vector<double> edges(A + 1);
    edges[0] = 0.0;
    for (int i = 1; i < A; ++i) edges[i] = std::sqrt(t->age_yr[i - 1] * t->age_yr[i]);
    edges[A] = INFINITY;
    c.log_age_edge[0] = -100.0f;
    for (int i = 1; i < A; ++i) c.log_age_edge[i] = (float)std::log10(edges[i]);
    c.log_age_edge[A] = 100.0f;
    c.lgz_edge[0] = -INFINITY;
    for (int j = 1; j < Zn; ++j) c.lgz_edge[j] = (float)(0.5 * (t->lgZ[j - 1] + t->lgZ[j]));
    c.lgz_edge[Zn] = INFINITY;
    for (int k = 0; k < SPS_NPARAM; ++k) {
        c.prior_lo[k] = (float)cfg.prior_lo[k];
        c.prior_span[k] = (float)(cfg.prior_hi[k] - cfg.prior_lo[k]);
        c.sig_k[k] = (float)cfg.sigmoid_k[k];
        c.sig_x0[k] = (float)cfg.sigmoid_x0[k];
        c.sn_xi[k] = (float)cfg.skew_xi[k];
        c.sn_iom[k] = (float)(1.0 / cfg.skew_omega[k]);
        c.sn_s[k] = (float)cfg.skew_s[k];
        c.sn_c[k] = (float)(std::log(2.0 / cfg.skew_omega[k]) - 0.5 * std::log(2.0 * M_PI));
    }
    c.prior_kind = cfg.prior;
    c.mdf_age = t->mdf_offset ? 1 : 0;
    for (int i = 0; i < kMaxAges; ++i) c.mdf_off[i] = (t->mdf_offset && i < A) ? (float)t->mdf_offset[i] : 0.0f;
    std::vector<double> tab64;
    for (int b = 0; b < B; ++b) {
        c.band_kind[b] = t->band_kind[b];
        c.tab_off[b] = (int)tab64.size();
        c.tab_n[b] = 0;
        if (t->band_kind[b] == SPS_BAND_TABLE) {
            c.tab_n[b] = t->band_tab_n[b];
            tab64.insert(tab64.end(), t->band_tab_T + c.tab_off[b], t->band_tab_T + c.tab_off[b] + c.tab_n[b]);
        }
    }
    if (tab64.empty()) tab64.push_back(0.0);
    std::vector<float> tab32(tab64.begin(), tab64.end());
    ctx->band_p0.assign(t->band_p0, t->band_p0 + B);
    ctx->band_p1.assign(t->band_p1, t->band_p1 + B);

    // tables: FP32 [k_pad][lam_pad], transposed, BF16 row-scaled versions
    const int kp = c.k_pad, lp = c.lam_pad;
    std::vector<float> s32((size_t)kp * lp, 0.f), st32((size_t)lp * kp, 0.f);
    std::vector<uint16_t> sbf((size_t)kp * lp, 0), stbf((size_t)lp * kp, 0);
    std::vector<float> rscale(A);
    for (int i = 0; i < A; ++i) {
        double mx = 0.0;
        for (int j = 0; j < Zn; ++j)
            for (int n = 0; n < L; ++n) mx = std::max(mx, t->ssp[((size_t)i * Zn + j) * L + n]);
        int e = (mx > 0) ? (int)std::lround(std::log2(mx)) : 0;
        rscale[i] = std::ldexp(1.0f, e);
        for (int j = 0; j < Zn; ++j) {
            size_t k = (size_t)i * Zn + j;
            for (int n = 0; n < L; ++n) {
                double v = t->ssp[k * L + n];
                float f = (float)v;
                s32[k * lp + n] = f;
                st32[(size_t)n * kp + k] = f;
                uint16_t h = bf16_rne((float)std::ldexp(v, -e));
                sbf[k * lp + n] = h;
                stbf[(size_t)n * kp + k] = h;
            }
        }
    }
    auto upload = [&](DevBuf& b, const void* src, size_t bytes) -> cudaError_t {
        cudaError_t e = b.reserve(bytes);
        if (e != cudaSuccess) return e;
        return cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice);
    };
    // per-column copy of the row scales (the adjoint epilogue's factor)
    std::vector<float> cscale((size_t)c.k_pad, 0.0f);
    for (int k = 0; k < c.K; ++k) cscale[(size_t)k] = rscale[(size_t)(k / c.n_met)];
    // 3xTF32 halves of the FP32 tables
    std::vector<float> s_hi(s32.size()), s_lo(s32.size()), st_hi(st32.size()), st_lo(st32.size());
    for (size_t i = 0; i < s32.size(); ++i) tf32_split_host(s32[i], s_hi[i], s_lo[i]);
    for (size_t i = 0; i < st32.size(); ++i) tf32_split_host(st32[i], st_hi[i], st_lo[i]);
    cudaError_t e = cudaSuccess;
    if ((e = upload(ctx->lam64, t->lam_ang, sizeof(double) * L)) != cudaSuccess ||
        (e = upload(ctx->ssp_hi, s_hi.data(), s_hi.size() * 4)) != cudaSuccess ||
        (e = upload(ctx->ssp_lo, s_lo.data(), s_lo.size() * 4)) != cudaSuccess ||
        (e = upload(ctx->ssp_t_hi, st_hi.data(), st_hi.size() * 4)) != cudaSuccess ||
        (e = upload(ctx->ssp_t_lo, st_lo.data(), st_lo.size() * 4)) != cudaSuccess ||
        (e = upload(ctx->ssp, s32.data(), s32.size() * 4)) != cudaSuccess ||
        (e = upload(ctx->ssp_t, st32.data(), st32.size() * 4)) != cudaSuccess ||
        (e = upload(ctx->ssp_bf, sbf.data(), sbf.size() * 2)) != cudaSuccess ||
        (e = upload(ctx->ssp_t_bf, stbf.data(), stbf.size() * 2)) != cudaSuccess ||
        (e = upload(ctx->row_scale, rscale.data(), rscale.size() * 4)) != cudaSuccess ||
        (e = upload(ctx->col_scale, cscale.data(), cscale.size() * 4)) != cudaSuccess ||
        (e = upload(ctx->age_edges, edges.data(), edges.size() * 8)) != cudaSuccess ||
        (e = upload(ctx->bp0, t->band_p0, sizeof(double) * B)) != cudaSuccess ||
        (e = upload(ctx->bp1, t->band_p1, sizeof(double) * B)) != cudaSuccess ||
        (e = upload(ctx->tabT, tab32.data(), sizeof(float) * tab32.size())) != cudaSuccess ||
        (e = upload(ctx->tabT64, tab64.data(), sizeof(double) * tab64.size())) != cudaSuccess ||
        (e = ctx->lam32.reserve(sizeof(float) * L)) != cudaSuccess ||
        (e = ctx->lamc.reserve(sizeof(float4) * L)) != cudaSuccess ||
        (e = ctx->lamq.reserve(sizeof(float2) * L)) != cudaSuccess ||
        (e = ctx->nonfinite.reserve(64)) != cudaSuccess || (e = ctx->queue.reserve(64)) != cudaSuccess ||
        (e = ctx->err.reserve(64)) != cudaSuccess) {
        delete ctx;
        return (e == cudaErrorMemoryAllocation) ? fail(SPS_E_NOMEM, "table upload: out of memory")
                                                : cuda_fail(e, "table upload");
    }
    if ((e = launch_lambda_consts(ctx->lam64.as<double>(), L, ctx->lamc.as<float4>(),
                                  ctx->lam32.as<float>(), ctx->lamq.as<float2>(), 0)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        delete ctx;
        return cuda_fail(e, "lambda constants");
    }
    if (const char* v = std::getenv("SPS_NO_TCGEN05")) ctx->use_tc = (v[0] == '0');
    *out = ctx;
    return SPS_OK;
}

sps_status sps_destroy(sps_ctx* ctx) {
    delete ctx;
    return SPS_OK;
}

sps_status sps_set_galaxies(sps_ctx* ctx, const float* z, int64_t n_gal, int32_t build_approx,
                            void* stream) {
    if (!ctx || (!z && n_gal > 0)) return fail(SPS_E_INVALID_ARG, "null argument");
    if (n_gal <= 0 || n_gal > (int64_t)1 << 31) return fail(SPS_E_SHAPE, "n_gal out of range");
    DeviceGuard dg(ctx->device);
    CK(dg.err);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<float> zh((size_t)n_gal);
    if (pointer_location(z, ctx->device) != 0) CK(cudaMemcpy(zh.data(), z, n_gal * 4, cudaMemcpyDeviceToHost));
    else std::memcpy(zh.data(), z, n_gal * 4);
    for (int64_t i = 0; i < n_gal; ++i)
        if (!(zh[i] > 0.0f && zh[i] < 20.0f)) return fail(SPS_E_INVALID_ARG, "redshift must be in (0, 20)");
    const Consts& c = ctx->c;
    const size_t G = (size_t)n_gal, B = c.n_band;
    CK(ctx->gz.reserve(G * 4));
    CK(ctx->glnT.reserve(G * 4));
    CK(ctx->glT10.reserve(G * 4));
    CK(ctx->gbins.reserve(G * c.n_age * sizeof(float2)));
    CK(ctx->gzp.reserve(G * B * 8));
    CK(ctx->gsup.reserve(G * B * sizeof(int2)));
    CK(ctx->ggauss.reserve(G * B * sizeof(float2)));
    CK(ctx->gdust.reserve(G * B * sizeof(float4)));
    CK(ctx->gdtdz.reserve(G * 4));
    CK(ctx->gdzp.reserve(G * B * 4));
    CK(ctx->gddust.reserve(G * B * sizeof(float4)));
    CK(cudaMemcpyAsync(ctx->gz.p, zh.data(), G * 4, cudaMemcpyHostToDevice, s));
    ctx->n_gal = n_gal;
    ctx->has_approx = false;
    ctx->has_dcssp = false;
    CK(launch_prepare_galaxies(c, ctx->grid(), ctx->lam64.as<double>(), ctx->bp0.as<double>(),
                               ctx->bp1.as<double>(), ctx->age_edges.as<double>(), ctx->gz.as<float>(),
                               n_gal, ctx->h0, ctx->om, ctx->glnT.as<float>(), ctx->glT10.as<float>(),
                               ctx->gbins.as<float2>(), ctx->gzp.as<double>(), ctx->gsup.as<int2>(),
                               ctx->ggauss.as<float2>(), ctx->gdust.as<float4>(), ctx->gdtdz.as<float>(),
                               ctx->gdzp.as<float>(), ctx->gddust.as<float4>(), s));
    if (build_approx) {
        cudaError_t e = ctx->gcssp.reserve(G * B * c.K * sizeof(float));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SPS_E_NOMEM, "c_SSP table does not fit in device memory");
        }
        ctx->has_approx = true;
        CK(launch_cssp(c, ctx->grid(), ctx->gal(), ctx->bp0.as<double>(), ctx->bp1.as<double>(),
                       ctx->gcssp.as<float>(), s));
    }
    CK(cudaStreamSynchronize(s));
    return SPS_OK;
}

// want_z: grad_out has 13 columns, d log L / dz last.
static sps_status run_exact(sps_ctx* ctx, const float* theta, const int32_t* gidx, int64_t n,
                            const float* mobs, const float* sigma, const uint32_t* mask, sps_prec prec,
                            float* mag_out, float* ll_out, float* grad_out, cudaStream_t s,
                            bool want_z = false, double* ll64_out = nullptr) {
    const Consts& c = ctx->c;
    const int NG = want_z ? SPS_NPARAM + 1 : SPS_NPARAM;
    // tcgen05 for BF16 operands (SIMT when disabled) and for 3xTF32; FP32 is SIMT
    if (prec == SPS_TF32X3 && !ctx->use_tc) return fail(SPS_E_UNSUPPORTED, "3xTF32 needs the tensor cores");
    const int bf16 = prec == SPS_BF16 ? 1 : 0;
    const bool tf = prec == SPS_TF32X3;
    const bool tc = tf || (bf16 && ctx->use_tc);
    const int64_t chunk = tc ? (tf ? 65536 : 131072) : 32768;
    const int64_t rows = std::min<int64_t>(n, chunk);
    CK(ctx->W.reserve((size_t)rows * c.k_pad * 4));
    if (tf) CK(ctx->Wlo.reserve((size_t)rows * c.k_pad * 4));
    CK(ctx->cJ.reserve((size_t)rows * c.n_band * 4 * 4));
    CK(ctx->rowinfo.reserve((size_t)rows * 4 * 4));
    CK(ctx->gbar.reserve((size_t)rows * c.n_band * 4));
    if (tc) CK(ctx->zperm.reserve(sizeof(int32_t) * (2 * (size_t)rows + (size_t)zsort_buckets())));
    int32_t* perm = tc ? ctx->zperm.as<int32_t>() : nullptr;
    int32_t* pos_of = tc ? perm + rows : nullptr;
    int32_t* zcounts = tc ? perm + 2 * rows : nullptr;
    if (grad_out) {
        CK(ctx->V.reserve((size_t)rows * c.lam_pad * 4));
        CK(ctx->Wbar.reserve((size_t)rows * c.k_pad * 4));
        if (tf) CK(ctx->Vlo.reserve((size_t)rows * c.lam_pad * 4));
        CK(ctx->keep.reserve((size_t)rows * (size_t)keep_stride(c) * 4));
    }
    float* keep = grad_out ? ctx->keep.as<float>() : nullptr;
    if (want_z) {
        CK(ctx->cJz.reserve((size_t)rows * c.n_band * 2 * 4));
        CK(ctx->rowz.reserve((size_t)rows * 4));
    }
    float* cJz = want_z ? ctx->cJz.as<float>() : nullptr;
    float* rowz = want_z ? ctx->rowz.as<float>() : nullptr;
    const Grid grid = ctx->grid();
    const Galaxies gal = ctx->gal();
    int* nf = ctx->nonfinite.as<int>();
    int* terr = ctx->nonfinite.as<int>() + 1;
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t m = std::min(chunk, n - r0);
        const float* th = theta + r0 * SPS_NPARAM;
        const int32_t* gi = gidx ? gidx + r0 : nullptr;
        // rows of a chunk without gal_idx map to galaxies r0 + row: pass an
        // offset view of the galaxy tables instead of an index array
        Galaxies gv = gal;
        const float* mo = mobs;
        const float* sg = sigma;
        const uint32_t* mk = mask;
        if (!gidx) {
            if (mo) mo += r0 * c.n_band;
            if (sg) sg += r0 * c.n_band;
            if (mk) mk += r0;
            gv.z += r0; gv.lnT += r0; gv.lT10 += r0;
            gv.bins += r0 * c.n_age; gv.zp += r0 * c.n_band; gv.support += r0 * c.n_band;
            gv.gauss += r0 * c.n_band; gv.dust_eff += r0 * c.n_band;
            if (gv.cssp) gv.cssp += r0 * c.n_band * c.K;
            gv.dtdz += r0; gv.dzp += r0 * c.n_band; gv.ddust += r0 * c.n_band;
            if (gv.dcssp) gv.dcssp += r0 * c.n_band * c.K;
            gv.n = m;
        }
        if (tc) CK(launch_zsort(gv, gi, m, perm, pos_of, zcounts, s));
        CK(launch_exact_weights(c, grid, gv, th, gi, m, bf16, ctx->W.as<float>(), ctx->W.as<uint16_t>(), s,
                                pos_of, tf ? ctx->Wlo.as<float>() : nullptr, keep));
        if (tc) {
            TcMaps tm;
            const bool ok = tf ? (make_tmap_f32(&tm.a[0], ctx->W.p, c.k_pad, m, c.k_pad, 128) &&
                                  make_tmap_f32(&tm.a[1], ctx->Wlo.p, c.k_pad, m, c.k_pad, 128) &&
                                  make_tmap_f32(&tm.b[0], ctx->ssp_t_hi.p, c.k_pad, c.n_lam, c.k_pad, 128) &&
                                  make_tmap_f32(&tm.b[1], ctx->ssp_t_lo.p, c.k_pad, c.n_lam, c.k_pad, 128))
                               : (make_tmap_bf16(&tm.a[0], ctx->W.p, c.k_pad, m, c.k_pad, 128) &&
                                  make_tmap_bf16(&tm.b[0], ctx->ssp_t_bf.p, c.k_pad, c.n_lam, c.k_pad, 256));
            if (!ok) return fail(SPS_E_CUDA, "tensor map encoding failed");
            if (!tf) tm.a[1] = tm.a[0], tm.b[1] = tm.b[0];
            CK(launch_fwd_tc(tm, tf, c, grid, gv, th, gi, perm, m, ctx->cJ.as<float>(), terr, s, cJz));
        } else {
            CK(launch_exact_fwd(c, grid, gv, th, gi, m, bf16, ctx->W.as<float>(), ctx->W.as<uint16_t>(),
                                ctx->cJ.as<float>(), s, cJz));
        }
        CK(launch_exact_like(c, gv, th, gi, m, ctx->cJ.as<float>(), ctx->rowinfo.as<float>(), mo, sg,
                             mk, mag_out ? mag_out + r0 * c.n_band : nullptr,
                             ll_out ? ll_out + r0 : nullptr, ctx->gbar.as<float>(), nf, s, cJz, rowz,
                             ll64_out ? ll64_out + r0 : nullptr));
        if (grad_out) {
            if (tc) {
                if (tf)
                    CK(launch_exact_vgen(c, grid, gv, th, gi, m, ctx->gbar.as<float>(), ctx->V.as<float>(),
                                         nullptr, s, ctx->Vlo.as<float>()));
                else
                    CK(launch_exact_vgen(c, grid, gv, th, gi, m, ctx->gbar.as<float>(), nullptr,
                                         ctx->V.as<uint16_t>(), s));
                TcMaps tm;
                const bool ok = tf ? (make_tmap_f32(&tm.a[0], ctx->V.p, c.lam_pad, m, c.lam_pad, 128) &&
                                      make_tmap_f32(&tm.a[1], ctx->Vlo.p, c.lam_pad, m, c.lam_pad, 128) &&
                                      make_tmap_f32(&tm.b[0], ctx->ssp_hi.p, c.lam_pad, c.K, c.lam_pad, 224) &&
                                      make_tmap_f32(&tm.b[1], ctx->ssp_lo.p, c.lam_pad, c.K, c.lam_pad, 224))
                                   : (make_tmap_bf16(&tm.a[0], ctx->V.p, c.lam_pad, m, c.lam_pad, 128) &&
                                      make_tmap_bf16(&tm.b[0], ctx->ssp_bf.p, c.lam_pad, c.K, c.lam_pad, 224));
                if (!ok) return fail(SPS_E_CUDA, "tensor map encoding failed");
                if (!tf) tm.a[1] = tm.a[0], tm.b[1] = tm.b[0];
                CK(launch_adj_tc(tm, tf, c, grid, m, ctx->Wbar.as<float>(), terr, s));
            } else {
                CK(launch_exact_vgen(c, grid, gv, th, gi, m, ctx->gbar.as<float>(), ctx->V.as<float>(),
                                     nullptr, s));
                CK(launch_exact_adj(c, grid, m, bf16, ctx->V.as<float>(), ctx->Wbar.as<float>(), s));
            }
            CK(launch_exact_grad(c, gv, th, gi, m, ctx->rowinfo.as<float>(), ctx->Wbar.as<float>(),
                                 grad_out + r0 * NG, s, rowz, keep));
        }
    }
    return SPS_OK;
}

static sps_status finish_call(sps_ctx* ctx, Stager& st, cudaStream_t s) {
    int fl[2] = {0, 0};
    CK(st.finish());
    CK(cudaMemcpyAsync(fl, ctx->nonfinite.p, sizeof(fl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (fl[1]) return fail(SPS_E_TIMEOUT, "a tensor-core pipeline wait timed out");
    if (fl[0]) return fail(SPS_E_NONFINITE, "some rows are NaN (non-finite inputs or results)");
    return SPS_OK;
}

sps_status sps_photometry(sps_ctx* ctx, const float* theta, const int32_t* gal_idx, int64_t n,
                          sps_mode mode, sps_prec prec, float* mag_out, void* stream) {
    sps_status st0 = check_rows(ctx, theta, gal_idx, n);
    if (st0 != SPS_OK) return st0;
    if (mode != SPS_EXACT && mode != SPS_APPROX) return fail(SPS_E_INVALID_ARG, "bad mode");
    if (prec != SPS_FP32 && prec != SPS_BF16 && prec != SPS_TF32X3) return fail(SPS_E_INVALID_ARG, "bad precision");
    if (mode == SPS_APPROX && prec != SPS_FP32) return fail(SPS_E_UNSUPPORTED, "approximate path is FP32");
    if (mode == SPS_APPROX && !ctx->has_approx) return fail(SPS_E_STATE, "galaxy set built without approx tables");
    if (n > 0 && !mag_out) return fail(SPS_E_INVALID_ARG, "mag_out is NULL");
    if (n == 0) return SPS_OK;
    DeviceGuard dg(ctx->device);
    CK(dg.err);
    cudaStream_t s = (cudaStream_t)stream;
    Stager st{ctx, s};
    const float* th = st.in(theta, (size_t)n * SPS_NPARAM);
    const int32_t* gi = st.in(gal_idx, (size_t)n);
    float* mo = st.out(mag_out, (size_t)n * ctx->c.n_band);
    if (sps_status r = st.check(); r != SPS_OK) return r;
    CK(cudaMemsetAsync(ctx->nonfinite.p, 0, 2 * sizeof(int), s));
    if (mode == SPS_APPROX && ctx->c.n_met <= 12 && !ctx->c.mdf_age && !std::getenv("SPS_LIKE_ROWS")) {
        // forward-only team evaluation, one row per warp
        CK(launch_phot_team(ctx->c, ctx->gal(), th, gi, n, mo, ctx->nonfinite.as<int>(), s));
    } else if (mode == SPS_APPROX) {
        CK(launch_approx_rows(ctx->c, ctx->gal(), th, 0, gi, n, nullptr, nullptr, nullptr, mo, nullptr,
                              nullptr, nullptr, ctx->nonfinite.as<int>(), s));
    } else {
        sps_status r = run_exact(ctx, th, gi, n, nullptr, nullptr, nullptr, prec, mo,
                                 nullptr, nullptr, s);
        if (r != SPS_OK) return r;
    }
    return finish_call(ctx, st, s);
}

sps_status sps_loglike_grad(sps_ctx* ctx, const float* theta, const int32_t* gal_idx, int64_t n,
                            const float* mag_obs, const float* sigma, const uint32_t* mask,
                            sps_mode mode, sps_prec prec, float* loglike_out, float* grad_out,
                            void* stream) {
    sps_status st0 = check_rows(ctx, theta, gal_idx, n);
    if (st0 != SPS_OK) return st0;
    if (mode != SPS_EXACT && mode != SPS_APPROX) return fail(SPS_E_INVALID_ARG, "bad mode");
    if (prec != SPS_FP32 && prec != SPS_BF16 && prec != SPS_TF32X3) return fail(SPS_E_INVALID_ARG, "bad precision");
    if (mode == SPS_APPROX && prec != SPS_FP32) return fail(SPS_E_UNSUPPORTED, "approximate path is FP32");
    if (mode == SPS_APPROX && !ctx->has_approx) return fail(SPS_E_STATE, "galaxy set built without approx tables");
    if (n > 0 && (!mag_obs || !sigma || !mask || !loglike_out))
        return fail(SPS_E_INVALID_ARG, "null data or output pointer");
    if (n == 0) return SPS_OK;
    DeviceGuard dg(ctx->device);
    CK(dg.err);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t GB = (size_t)ctx->n_gal * ctx->c.n_band;
    Stager st{ctx, s};
    const float* th = st.in(theta, (size_t)n * SPS_NPARAM);
    const int32_t* gi = st.in(gal_idx, (size_t)n);
    const float* mo = st.in(mag_obs, GB);
    const float* sg = st.in(sigma, GB);
    const uint32_t* mk = st.in(mask, (size_t)ctx->n_gal);
    float* llo = st.out(loglike_out, (size_t)n);
    float* gro = st.out(grad_out, (size_t)n * SPS_NPARAM);
    if (sps_status r = st.check(); r != SPS_OK) return r;
    CK(cudaMemsetAsync(ctx->nonfinite.p, 0, 2 * sizeof(int), s));
    if (mode == SPS_APPROX && ctx->c.n_met <= 12 && !std::getenv("SPS_LIKE_ROWS")) {
        // the team evaluation, one row per warp
        CK(launch_like_team(ctx->c, ctx->gal(), th, gi, n, mo, sg, mk, llo, gro, ctx->nonfinite.as<int>(), s));
    } else if (mode == SPS_APPROX) {
        CK(launch_approx_rows(ctx->c, ctx->gal(), th, 0, gi, n, mo, sg, mk, nullptr, llo, gro, nullptr,
                              ctx->nonfinite.as<int>(), s));
    } else {
        sps_status r = run_exact(ctx, th, gi, n, mo, sg, mk, prec, nullptr, llo, gro, s);
        if (r != SPS_OK) return r;
    }
    return finish_call(ctx, st, s);
}

sps_status sps_loglike_grad_z(sps_ctx* ctx, const float* theta, const int32_t* gal_idx, int64_t n,
                              const float* mag_obs, const float* sigma, const uint32_t* mask,
                              sps_mode mode, sps_prec prec, float* loglike_out, float* grad_out,
                              void* stream) {
    sps_status st0 = check_rows(ctx, theta, gal_idx, n);
    if (st0 != SPS_OK) return st0;
    if (mode != SPS_EXACT && mode != SPS_APPROX) return fail(SPS_E_INVALID_ARG, "bad mode");
    if (prec != SPS_FP32 && prec != SPS_BF16 && prec != SPS_TF32X3) return fail(SPS_E_INVALID_ARG, "bad precision");
    if (mode == SPS_APPROX && prec != SPS_FP32) return fail(SPS_E_UNSUPPORTED, "approximate path is FP32");
    if (mode == SPS_APPROX && !ctx->has_approx) return fail(SPS_E_STATE, "galaxy set built without approx tables");
    for (int b = 0; b < ctx->c.n_band; ++b)
        if (ctx->c.band_kind[b] == SPS_BAND_TOPHAT)
            return fail(SPS_E_UNSUPPORTED, "the redshift derivative needs bands with a continuous "
                                           "transmission (Gaussian or tabulated); band " + std::to_string(b) +
                                           " is a top-hat");
    if (n > 0 && (!mag_obs || !sigma || !mask || !loglike_out || !grad_out))
        return fail(SPS_E_INVALID_ARG, "null data or output pointer");
    if (n == 0) return SPS_OK;
    DeviceGuard dg(ctx->device);
    CK(dg.err);
    cudaStream_t s = (cudaStream_t)stream;
    const Consts& c = ctx->c;
    if (mode == SPS_APPROX && !ctx->has_dcssp) {          // d c_SSP / dz, once per galaxy set
        cudaError_t e = ctx->gdcssp.reserve((size_t)ctx->n_gal * c.n_band * c.K * sizeof(float));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SPS_E_NOMEM, "the d c_SSP / dz table does not fit in device memory");
        }
        CK(launch_cssp(c, ctx->grid(), ctx->gal(), ctx->bp0.as<double>(), ctx->bp1.as<double>(),
                       ctx->gdcssp.as<float>(), s, 1));
        ctx->has_dcssp = true;
    }
    const size_t GB = (size_t)ctx->n_gal * c.n_band;
    Stager st{ctx, s};
    const float* th = st.in(theta, (size_t)n * SPS_NPARAM);
    const int32_t* gi = st.in(gal_idx, (size_t)n);
    const float* mo = st.in(mag_obs, GB);
    const float* sg = st.in(sigma, GB);
    const uint32_t* mk = st.in(mask, (size_t)ctx->n_gal);
    float* llo = st.out(loglike_out, (size_t)n);
    float* gro = st.out(grad_out, (size_t)n * (SPS_NPARAM + 1));
    if (sps_status r = st.check(); r != SPS_OK) return r;
    CK(cudaMemsetAsync(ctx->nonfinite.p, 0, 2 * sizeof(int), s));
    if (mode == SPS_APPROX) {
        CK(launch_approx_rows_z(c, ctx->gal(), th, gi, n, mo, sg, mk, llo, gro, ctx->nonfinite.as<int>(), s));
    } else {
        sps_status r = run_exact(ctx, th, gi, n, mo, sg, mk, prec, nullptr, llo, gro, s, true);
        if (r != SPS_OK) return r;
    }
    return finish_call(ctx, st, s);
}

sps_status sps_loglike_grad_forward_mode(sps_ctx* ctx, const float* theta, const int32_t* gal_idx,
                                         int64_t n, const float* mag_obs, const float* sigma,
                                         const uint32_t* mask, float* loglike_out, float* grad_out,
                                         void* stream) {
    sps_status st0 = check_rows(ctx, theta, gal_idx, n);
    if (st0 != SPS_OK) return st0;
    if (!ctx->has_approx) return fail(SPS_E_STATE, "galaxy set built without approx tables");
    if (ctx->c.mdf_age) return fail(SPS_E_UNSUPPORTED, "the forward-mode baseline supports the separable model only");
    if (n > 0 && (!mag_obs || !sigma || !mask || !loglike_out))
        return fail(SPS_E_INVALID_ARG, "null data or output pointer");
    if (n == 0) return SPS_OK;
    DeviceGuard dg(ctx->device);
    CK(dg.err);
    cudaStream_t s = (cudaStream_t)stream;
    const Consts& c = ctx->c;
    const size_t GB = (size_t)ctx->n_gal * c.n_band;
    Stager st{ctx, s};
    const float* th = st.in(theta, (size_t)n * SPS_NPARAM);
    const int32_t* gi = st.in(gal_idx, (size_t)n);
    const float* mo = st.in(mag_obs, GB);
    const float* sg = st.in(sigma, GB);
    const uint32_t* mk = st.in(mask, (size_t)ctx->n_gal);
    float* llo = st.out(loglike_out, (size_t)n);
    float* gro = st.out(grad_out, (size_t)n * SPS_NPARAM);
    if (sps_status r = st.check(); r != SPS_OK) return r;
    CK(cudaMemsetAsync(ctx->nonfinite.p, 0, 2 * sizeof(int), s));
    const int64_t chunk = 32768;
    const int64_t rows = std::min<int64_t>(n, chunk);
    CK(ctx->plainT.reserve((size_t)rows * 9 * c.K * sizeof(float)));
    CK(ctx->plainC.reserve((size_t)rows * c.n_band * 9 * sizeof(float)));
    const Galaxies gal = ctx->gal();
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t m = std::min(chunk, n - r0);
        Galaxies gv = gal;
        const float* mo2 = mo;
        const float* sg2 = sg;
        const uint32_t* mk2 = mk;
        if (!gi) {
            mo2 += r0 * c.n_band; sg2 += r0 * c.n_band; mk2 += r0;
            gv.z += r0; gv.lnT += r0; gv.lT10 += r0; gv.bins += r0 * c.n_age;
            gv.zp += r0 * c.n_band; gv.support += r0 * c.n_band; gv.gauss += r0 * c.n_band;
            gv.dust_eff += r0 * c.n_band; gv.cssp += r0 * c.n_band * c.K; gv.n = m;
        }
        CK(launch_plain(c, gv, th + r0 * SPS_NPARAM, gi ? gi + r0 : nullptr, m, mo2, sg2, mk2,
                        llo + r0, gro ? gro + r0 * SPS_NPARAM : nullptr, ctx->plainT.as<float>(),
                        ctx->plainC.as<float>(), s));
    }
    return finish_call(ctx, st, s);
}

sps_status sps_leapfrog(sps_ctx* ctx, const float* x0, const float* p0, const float* eps,
                        const int32_t* L, const int32_t* gal_idx, int64_t n, const float* mag_obs,
                        const float* sigma, const uint32_t* mask, float* x_out, float* p_out,
                        double* logp_out, void* stream) {
    sps_status st0 = check_rows(ctx, x0, gal_idx, n);
    if (st0 != SPS_OK) return st0;
    if (!ctx->has_approx) return fail(SPS_E_STATE, "galaxy set built without approx tables");
    if (n > 0 && (!p0 || !eps || !L || !mag_obs || !sigma || !mask || !x_out || !p_out || !logp_out))
        return fail(SPS_E_INVALID_ARG, "null argument");
    if (n == 0) return SPS_OK;
    if (pointer_location(L, ctx->device) == 0)
        for (int64_t i = 0; i < n; ++i)
            if (L[i] < 0 || L[i] > 100000) return fail(SPS_E_SHAPE, "L out of range");
    DeviceGuard dg(ctx->device);
    CK(dg.err);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t GB = (size_t)ctx->n_gal * ctx->c.n_band;
    Stager st{ctx, s};
    const float* x = st.in(x0, (size_t)n * SPS_NPARAM);
    const float* p = st.in(p0, (size_t)n * SPS_NPARAM);
    const float* e = st.in(eps, (size_t)n);
    const int32_t* l = st.in(L, (size_t)n);
    const int32_t* gi = st.in(gal_idx, (size_t)n);
    const float* mo = st.in(mag_obs, GB);
    const float* sg = st.in(sigma, GB);
    const uint32_t* mk = st.in(mask, (size_t)ctx->n_gal);
    float* xo = st.out(x_out, (size_t)n * SPS_NPARAM);
    float* po = st.out(p_out, (size_t)n * SPS_NPARAM);
    double* lo = st.out(logp_out, (size_t)n);
    if (sps_status r = st.check(); r != SPS_OK) return r;
    CK(launch_leapfrog(ctx->c, ctx->gal(), x, p, e, l, gi, n, mo, sg, mk, xo, po, lo, s));
    CK(st.finish());
    return SPS_OK;
}

sps_status sps_philox(sps_ctx* ctx, const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out,
                      void* stream) {
    if (!ctx || (n > 0 && (!ctr || !out))) return fail(SPS_E_INVALID_ARG, "null argument");
    if (n <= 0) return SPS_OK;
    DeviceGuard dg(ctx->device);
    CK(dg.err);
    cudaStream_t s = (cudaStream_t)stream;
    Stager st{ctx, s};
    const uint32_t* c = st.in(ctr, (size_t)n * 4);
    uint32_t* o = st.out(out, (size_t)n * 4);
    if (sps_status r = st.check(); r != SPS_OK) return r;
    CK(launch_philox(c, n, key, o, s));
    CK(st.finish());
    return SPS_OK;
}

sps_status sps_weights(sps_ctx* ctx, const float* theta, const int32_t* gal_idx, int64_t n,
                       float* W_out, double* mstar_out, void* stream) {
    sps_status st0 = check_rows(ctx, theta, gal_idx, n);
    if (st0 != SPS_OK) return st0;
    if (n == 0) return SPS_OK;
    DeviceGuard dg(ctx->device);
    CK(dg.err);
    cudaStream_t s = (cudaStream_t)stream;
    Stager st{ctx, s};
    const float* th = st.in(theta, (size_t)n * SPS_NPARAM);
    const int32_t* gi = st.in(gal_idx, (size_t)n);
    float* w = st.out(W_out, (size_t)n * ctx->c.K);
    double* m = st.out(mstar_out, (size_t)n);
    if (sps_status r = st.check(); r != SPS_OK) return r;
    CK(launch_weights_rows(ctx->c, ctx->gal(), th, gi, n, w, m, s));
    CK(st.finish());
    return SPS_OK;
}

sps_status sps_get_info(const sps_ctx* ctx, sps_info* out) {
    if (!ctx || !out) return fail(SPS_E_INVALID_ARG, "null argument");
    out->n_age = ctx->c.n_age;
    out->n_met = ctx->c.n_met;
    out->n_lam = ctx->c.n_lam;
    out->n_band = ctx->c.n_band;
    out->k_pad = ctx->c.k_pad;
    out->n_gal = ctx->n_gal;
    out->has_approx = ctx->has_approx ? 1 : 0;
    out->device = ctx->device;
    out->sfh_gl_order = ctx->c.gl_order;
    out->max_panels = kMaxPanels;
    out->hmc_launches = ctx->hmc_launches;
    return SPS_OK;
}

sps_status sps_gl_rule(const sps_ctx* ctx, double* nodes, double* weights) {
    if (!ctx || !nodes || !weights) return fail(SPS_E_INVALID_ARG, "null argument");
    for (int i = 0; i < ctx->c.gl_order; ++i) {
        nodes[i] = ctx->gl_x[i];
        weights[i] = ctx->gl_w[i];
    }
    return SPS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- HMC
namespace {

struct HmcLaunch {
    int warps, blocks;
    size_t table_bytes;
};

}  // namespace

namespace sps {
// exact_tc.cu: the tensor-core pipeline's bounded wait on a barrier completed or not
cudaError_t launch_wait_probe(int ready, uint32_t limit, int* err, cudaStream_t s);
}  // namespace sps

extern "C" sps_status sps_wait_probe(sps_ctx* ctx, int32_t ready, uint32_t spin_limit, void* stream) {
    if (!ctx) return fail(SPS_E_INVALID_ARG, "null context");
    if (spin_limit < 1 || spin_limit > (1u << 26)) return fail(SPS_E_INVALID_ARG, "spin_limit in [1, 2^26]");
    DeviceGuard dg(ctx->device);
    CK(dg.err);
    cudaStream_t s = (cudaStream_t)stream;
    int fl[2] = {0, 0};
    CK(cudaMemsetAsync(ctx->nonfinite.p, 0, 2 * sizeof(int), s));
    CK(launch_wait_probe(ready != 0, spin_limit, ctx->nonfinite.as<int>() + 1, s));
    CK(cudaMemcpyAsync(fl, ctx->nonfinite.p, sizeof(fl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (fl[1]) return fail(SPS_E_TIMEOUT, "the probed wait timed out");
    return SPS_OK;
}

// HMC on the exact photometry (Eq. photo_integral_exact): one gradient
// evaluation of every chain per round through the exact path (the tensor-core
// contractions for BF16 and 3xTF32), then one trajectory-asynchronous leapfrog
// step of every chain (hmc_plain.cu: k_async_step), for as many rounds as the
// longest chain's leapfrog steps.  Same sampler and draws as sps_hmc_run's
// HMC with the identity metric.
static sps_status hmc_exact(sps_ctx* ctx, const sps_hmc_config* cfg, const float* theta0_unb,
                            const float* mag_obs, const float* sigma, const uint32_t* mask,
                            float* samples_out, sps_hmc_stats* stats, cudaStream_t s) {
    if (cfg->sampler != SPS_HMC) return fail(SPS_E_UNSUPPORTED, "the exact-path sampler runs HMC");
    if (cfg->adapt_mass != 0) return fail(SPS_E_UNSUPPORTED, "the exact-path sampler uses the identity metric");
    if (cfg->prec != SPS_FP32 && cfg->prec != SPS_BF16 && cfg->prec != SPS_TF32X3)
        return fail(SPS_E_INVALID_ARG, "bad precision");
    if (cfg->L_min < 1 || cfg->L_max < cfg->L_min || cfg->L_max > 4096) return fail(SPS_E_SHAPE, "L range");
    const int64_t G = ctx->n_gal;
    const int C = cfg->chains_per_gal;
    const int64_t NC = G * C;
    const Consts& c = ctx->c;
    const size_t GB = (size_t)G * c.n_band;
    Stager st{ctx, s};
    const float* x0 = st.in(theta0_unb, (size_t)NC * SPS_NPARAM);
    const float* mo = st.in(mag_obs, GB);
    const float* sg = st.in(sigma, GB);
    const uint32_t* mk = st.in(mask, (size_t)G);
    float* so = st.out(samples_out, (size_t)NC * cfg->n_samp * SPS_NPARAM);
    float* acc = stats ? st.out(stats->accept_prob, (size_t)NC) : nullptr;
    float* epo = stats ? st.out(stats->step_size, (size_t)NC) : nullptr;
    int32_t* dv = stats ? st.out(stats->divergences, (size_t)NC) : nullptr;
    int64_t* nev = stats ? st.out(stats->grad_evals, (size_t)NC) : nullptr;
    int32_t* sto = stats ? st.out(stats->status, (size_t)NC) : nullptr;
    if (sps_status r = st.check(); r != SPS_OK) return r;
    HmcParams hp{C, cfg->n_warm, cfg->n_samp, cfg->L_min, cfg->L_max, cfg->target_accept, cfg->eps0,
                 cfg->seed, 0, 1};
    CK(ctx->pst.reserve(sizeof(PlainChain) * (size_t)NC));
    CK(ctx->pth.reserve(sizeof(float) * SPS_NPARAM * (size_t)NC));
    CK(ctx->pll.reserve(sizeof(double) * (size_t)NC));
    CK(ctx->pgr.reserve(sizeof(float) * SPS_NPARAM * (size_t)NC));
    CK(ctx->pgi.reserve(sizeof(int32_t) * (size_t)NC));
    CK(ctx->rowz.reserve(sizeof(float) * (size_t)std::max<int64_t>(NC, 2)));   // FP32 log L (unused)
    PlainChain* pst = ctx->pst.as<PlainChain>();
    float* th = ctx->pth.as<float>();
    double* ll = ctx->pll.as<double>();
    float* gr = ctx->pgr.as<float>();
    int32_t* gi = ctx->pgi.as<int32_t>();
    float* llf = ctx->rowz.as<float>();
    const sps_prec prec = (sps_prec)cfg->prec;
    cudaStream_t gs = s;                  // the stream the gradient is enqueued on
    auto gradient = [&]() -> sps_status {
        return run_exact(ctx, th, gi, NC, mo, sg, mk, prec, nullptr, llf, gr, gs, false, ll);
    };
    CK(cudaMemsetAsync(ctx->nonfinite.p, 0, 2 * sizeof(int), s));
    CK(plain_hmc_init(c, NC, C, x0, hp.eps0, pst, th, gi, s));
    if (sps_status r = gradient(); r != SPS_OK) return r;
    CK(plain_hmc_absorb(c, NC, pst, ll, gr, s));
    CK(plain_hmc_start(c, hp, NC, pst, th, s));
    int rounds = 0;
    int* rbuf = ctx->nonfinite.as<int>() + 2;
    CK(async_hmc_rounds(hp, NC, rbuf, s));
    CK(cudaMemcpyAsync(&rounds, rbuf, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // A round (the exact log L + gradient of every chain, then one leapfrog
    // step each) is the same sequence of launches every time: captured once
    // as a CUDA graph (on a private stream; the buffers it uses were reserved
    // by the first gradient above) and replayed, so the host encodes tensor
    // maps and issues launches once per call instead of once per round.
    // SPS_EXACT_GRAPH=0 enqueues every round directly.
    const char* gv = std::getenv("SPS_EXACT_GRAPH");
    if (rounds > 1 && !(gv && gv[0] == '0')) {
        cudaStream_t cs;
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t gr0 = nullptr;
        cudaGraphExec_t gx = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        sps_status rs = SPS_OK;
        if (e == cudaSuccess) {
            gs = cs;
            rs = gradient();
            if (rs == SPS_OK) e = async_hmc_step(c, hp, NC, pst, ll, gr, th, so, cs);
            gs = s;
            const cudaError_t e2 = cudaStreamEndCapture(cs, &gr0);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess && rs == SPS_OK) e = cudaGraphInstantiate(&gx, gr0, 0);
        if (gr0) cudaGraphDestroy(gr0);
        cudaStreamDestroy(cs);
        if (rs != SPS_OK) {
            if (gx) cudaGraphExecDestroy(gx);
            return rs;
        }
        if (e != cudaSuccess) {
            if (gx) cudaGraphExecDestroy(gx);
            return cuda_fail(e, "exact round capture");
        }
        for (int r = 0; r < rounds && e == cudaSuccess; ++r) e = cudaGraphLaunch(gx, s);
        cudaGraphExecDestroy(gx);
        if (e != cudaSuccess) return cuda_fail(e, "exact round launch");
    } else {
        for (int r = 0; r < rounds; ++r) {
            if (sps_status e = gradient(); e != SPS_OK) return e;
            CK(async_hmc_step(c, hp, NC, pst, ll, gr, th, so, s));
        }
    }
    CK(plain_hmc_stats(hp, NC, pst, acc, epo, dv, nev, sto, s));
    int fl[2] = {0, 0};
    CK(st.finish());
    CK(cudaMemcpyAsync(fl, ctx->nonfinite.p, sizeof(fl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (fl[1]) return fail(SPS_E_TIMEOUT, "a tensor-core pipeline wait timed out");
    return SPS_OK;
}

extern "C" sps_status sps_hmc_run(sps_ctx* ctx, const sps_hmc_config* cfg, const float* theta0_unb,
                                  const float* mag_obs, const float* sigma, const uint32_t* mask,
                                  float* samples_out, sps_hmc_stats* stats, void* stream) {
    if (!ctx || !cfg) return fail(SPS_E_INVALID_ARG, "null argument");
    if (ctx->n_gal <= 0) return fail(SPS_E_STATE, "no galaxy set");
    if (cfg->mode != SPS_APPROX && cfg->mode != SPS_EXACT) return fail(SPS_E_INVALID_ARG, "bad mode");
    if (cfg->mode == SPS_APPROX && !ctx->has_approx) return fail(SPS_E_STATE, "galaxy set built without approx tables");
    if (cfg->chains_per_gal < 1 || cfg->chains_per_gal > 64) return fail(SPS_E_SHAPE, "chains_per_gal in [1, 64]");
    if (cfg->n_warm < 0 || cfg->n_samp < 0 || cfg->n_warm + cfg->n_samp < 1)
        return fail(SPS_E_SHAPE, "iteration counts");
    if (cfg->mode == SPS_EXACT) {
        if (!(cfg->eps0 > 0) || !(cfg->target_accept > 0 && cfg->target_accept < 1))
            return fail(SPS_E_INVALID_ARG, "eps0 / target_accept");
        if (!theta0_unb || !mag_obs || !sigma || !mask) return fail(SPS_E_INVALID_ARG, "null input");
        if ((int64_t)ctx->n_gal * cfg->chains_per_gal > ((int64_t)1 << 31)) return fail(SPS_E_SHAPE, "too many chains");
        DeviceGuard dg(ctx->device);
        CK(dg.err);
        return hmc_exact(ctx, cfg, theta0_unb, mag_obs, sigma, mask, samples_out, stats, (cudaStream_t)stream);
    }
    const bool nuts = cfg->sampler == SPS_NUTS;
    if (cfg->sampler != SPS_HMC && !nuts) return fail(SPS_E_INVALID_ARG, "sampler");
    if (!nuts && (cfg->L_min < 1 || cfg->L_max < cfg->L_min || cfg->L_max > 4096))
        return fail(SPS_E_SHAPE, "L range");
    if (nuts && (cfg->max_depth < 1 || cfg->max_depth > kNutsMaxDepth)) return fail(SPS_E_SHAPE, "max_depth in [1, 10]");
    if (nuts && cfg->adapt_mass != 0) return fail(SPS_E_UNSUPPORTED, "NUTS runs with the identity metric");
    if (!(cfg->eps0 > 0) || !(cfg->target_accept > 0 && cfg->target_accept < 1))
        return fail(SPS_E_INVALID_ARG, "eps0 / target_accept");
    if (!theta0_unb || !mag_obs || !sigma || !mask) return fail(SPS_E_INVALID_ARG, "null input");
    const int64_t G = ctx->n_gal;
    const int C = cfg->chains_per_gal;
    const int64_t NC = G * C;
    if (NC > ((int64_t)1 << 31)) return fail(SPS_E_SHAPE, "too many chains");
    DeviceGuard dg(ctx->device);
    CK(dg.err);
    cudaStream_t s = (cudaStream_t)stream;
    const Consts& c = ctx->c;
    const size_t GB = (size_t)G * c.n_band;
    // maximum observed band count decides the shared table size
    std::vector<uint32_t> mh((size_t)G);
    if (pointer_location(mask, ctx->device) != 0) CK(cudaMemcpy(mh.data(), mask, G * 4, cudaMemcpyDeviceToHost));
    else std::memcpy(mh.data(), mask, G * 4);
    const uint32_t all = (c.n_band >= 32) ? 0xffffffffu : ((1u << c.n_band) - 1u);
    int nb_max = 0;
    std::vector<int32_t> order((size_t)G);
    std::vector<int> nbs((size_t)G);
    for (int64_t g = 0; g < G; ++g) {
        nbs[g] = __builtin_popcount(mh[g] & all);
        nb_max = std::max(nb_max, nbs[g]);
        order[g] = (int32_t)g;
    }
    // longest work first (more observed bands = more work per gradient)
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return nbs[a] > nbs[b]; });
    Stager st{ctx, s};
    const float* x0 = st.in(theta0_unb, (size_t)NC * SPS_NPARAM);
    const float* mo = st.in(mag_obs, GB);
    const float* sg = st.in(sigma, GB);
    const uint32_t* mk = st.in(mask, (size_t)G);
    const int32_t* ord = st.in(order.data(), (size_t)G);
    float* so = st.out(samples_out, (size_t)NC * cfg->n_samp * SPS_NPARAM);
    float* acc = stats ? st.out(stats->accept_prob, (size_t)NC) : nullptr;
    float* epo = stats ? st.out(stats->step_size, (size_t)NC) : nullptr;
    int32_t* dv = stats ? st.out(stats->divergences, (size_t)NC) : nullptr;
    int64_t* nev = stats ? st.out(stats->grad_evals, (size_t)NC) : nullptr;
    int32_t* sto = stats ? st.out(stats->status, (size_t)NC) : nullptr;
    if (sps_status r = st.check(); r != SPS_OK) return r;

    HmcParams hp{C, cfg->n_warm, cfg->n_samp, cfg->L_min, cfg->L_max, cfg->target_accept, cfg->eps0,
                 cfg->seed, cfg->adapt_mass < 0 ? 0 : (cfg->adapt_mass > 2 ? 2 : cfg->adapt_mass), 1};
    if (const char* v = std::getenv("SPS_HMC_SYNC")) hp.sync_every = std::max(1, std::atoi(v));
    if (nuts) {
        hp.L_min = hp.L_max = 1;
        hp.max_depth = cfg->max_depth;
        CK(ctx->hmcn.reserve(sizeof(NutsChain) * (size_t)std::max<int64_t>(NC, 1)));
        hp.nuts = ctx->hmcn.as<NutsChain>();
    }
    if (c.n_met > 12) return fail(SPS_E_UNSUPPORTED, "HMC kernel holds at most 12 metallicity bins in registers");
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, ctx->device));
    const int sms = prop.multiProcessorCount;
    CK(ctx->hmcm.reserve(sizeof(ChainMetric) * (size_t)std::max<int64_t>(NC, 1)));
    ChainMetric* cmet = ctx->hmcm.as<ChainMetric>();
    // launch shapes: chains of a galaxy per warp (cpw) x warps per block; the
    // grid is persistent (occupancy x SMs) and pulls (galaxy, chain group)
    // items from the queue
    // first candidate = default; another replaces it only if >3% faster in the probe
    // an age-dependent MDF runs the one-chain-per-warp variant with the per-age q matrix
    const bool rows = ctx->c.mdf_age != 0;
    std::vector<std::pair<int, int>> cands = {{1, 8}, {1, 16}};
    if (rows) {
        cands = {{1, 4}, {1, 2}, {1, 8}};
    } else if (nuts) {
        // NUTS: the 8-iteration probe from the start points does not rank the
        // shapes reliably (tree depths change over the warm-up); one chain per
        // warp measured best on full runs, two per warp within 1%
        cands = {{1, 8}};
        if (C >= 2) cands.push_back({2, 8});
    } else {
        if (C >= 2) cands.insert(cands.begin(), {{2, 4}, {2, 8}, {2, 16}});
        if (C >= 4) cands.push_back({4, 8});
    }
    const int cpw0 = cands[0].first;
    auto blocks_for = [&](int cpw, int warps, int& blocks) -> cudaError_t {
        int per_sm = 0;
        cudaError_t e = hmc_team_occupancy(cpw, rows, nuts, warps, &per_sm);
        if (e != cudaSuccess) return e;
        blocks = std::max(1, per_sm) * sms;
        return cudaSuccess;
    };
    const std::string key = std::to_string(G) + ":" + std::to_string(C) + ":" + std::to_string(nb_max) +
                            (nuts ? ":nuts" : "") + (rows ? ":rows" : "");
    int cpw = cpw0, warps = cands[0].second, blocks = sms;
    auto it = ctx->tuned.find(key);
    const char* force = std::getenv("SPS_HMC_SHAPE");   // "cpw,warps": fixed launch shape
    int fc = 0, fw = 0;
    if (force && std::sscanf(force, "%d,%d", &fc, &fw) == 2 && (fc == 1 || (!rows && (fc == 2 || fc == 4))) &&
        fc <= std::max(C, 1) && fw >= 1 && fw <= 16) {
        cpw = fc;
        warps = fw;
        CK(blocks_for(cpw, warps, blocks));
    } else if (it != ctx->tuned.end()) {
        cpw = it->second.first / 100;
        warps = it->second.first % 100;
        blocks = it->second.second;
    } else if (cfg->autotune && G >= 2 * sms) {
        // time each candidate on a short run over a slice of the galaxies
        float best = 1e30f;
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        HmcParams tp = hp;
        tp.n_warm = 8;
        tp.n_samp = 0;
        Galaxies gsub = ctx->gal();
        for (auto cw : cands) {
            int b = 0;
            CK(blocks_for(cw.first, cw.second, b));
            const int groups = (C + cw.first - 1) / cw.first;
            gsub.n = std::min<int64_t>(G, ((int64_t)b * cw.second * 2 + groups - 1) / groups);
            CK(cudaMemsetAsync(ctx->queue.p, 0, sizeof(int), s));
            CK(cudaEventRecord(e0, s));
            CK(launch_hmc_team(cw.first, rows, c, gsub, tp, x0, mo, sg, mk, ord, nullptr, nullptr, nullptr,
                               nullptr, nullptr, nullptr, ctx->queue.as<int>(), cmet, b, cw.second, s));
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            const float per = ms / (float)(gsub.n * C);
            if (cw == cands[0] ? per < best : per < 0.97f * best) {
                best = per;
                cpw = cw.first;
                warps = cw.second;
                blocks = b;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ctx->tuned[key] = {cpw * 100 + warps, blocks};
    } else {
        CK(blocks_for(cpw, warps, blocks));
    }

    // When the last wave of two-chain teams would fill under 3/4 of the
    // resident warps, its chains run as one-chain teams in a second launch
    // (HMC, separable model, an even chain count): the same chains and draws,
    // spread over more warps. SPS_HMC_TAIL=0 keeps one launch.
    int64_t main_end = -1;      // two-chain items of the first launch (< 0: all)
    int blocks1 = 0;
    {
        const int64_t slots = (int64_t)blocks * warps;
        const int64_t items = G * (int64_t)((C + cpw - 1) / cpw);
        const char* tv = std::getenv("SPS_HMC_TAIL");
        if (!nuts && !rows && cpw == 2 && C % 2 == 0 && !(tv && tv[0] == '0') && items > slots &&
            items % slots != 0 && 4 * (items % slots) < 3 * slots) {
            main_end = items / slots * slots;
            CK(blocks_for(1, warps, blocks1));
            if (!ctx->side) {
                CK(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
                CK(cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming));
                CK(cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming));
            }
        }
    }
    // The tail launch goes on a side stream forked after the queue resets, so
    // its blocks take SMs as the main launch's blocks retire; the join makes
    // the call's stream wait for both.  The two launches pull from separate
    // queue counters and touch disjoint chains.
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(ctx->queue.p, 0, 2 * sizeof(int), s);
        if (e != cudaSuccess) return e;
        HmcParams h1 = hp;
        h1.item_end = main_end;
        if (main_end >= 0) {
            if ((e = cudaEventRecord(ctx->fork, s)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(ctx->side, ctx->fork, 0)) != cudaSuccess) return e;
        }
        e = launch_hmc_team(cpw, rows, c, ctx->gal(), h1, x0, mo, sg, mk, ord, so, acc, epo, dv, nev, sto,
                            ctx->queue.as<int>(), cmet, blocks, warps, s);
        if (e != cudaSuccess || main_end < 0) return e;
        HmcParams h2 = hp;
        h2.item0 = 2 * main_end;      // one-chain items: two per two-chain item
        h2.item_end = G * (int64_t)C;
        e = launch_hmc_team(1, rows, c, ctx->gal(), h2, x0, mo, sg, mk, ord, so, acc, epo, dv, nev, sto,
                            ctx->queue.as<int>() + 1, cmet, blocks1, warps, ctx->side);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventRecord(ctx->join, ctx->side)) != cudaSuccess) return e;
        return cudaStreamWaitEvent(s, ctx->join, 0);
    };
    ctx->hmc_launches = main_end < 0 ? 1 : 2;
    if (cfg->use_graph) {
        char kb[512];
        std::snprintf(kb, sizeof(kb), "%p%p%p%p%p%p%p%p%p%p%p%lld%d%d%d%d%d%d%d%llu%g%g", (const void*)x0,
                      (const void*)mo, (const void*)sg, (const void*)mk, (const void*)ord, (void*)so,
                      (void*)acc, (void*)epo, (void*)dv, (void*)nev, (void*)sto, (long long)G, C,
                      hp.n_warm, hp.n_samp, hp.L_min, hp.L_max, warps, hp.adapt_mass, (unsigned long long)hp.seed,
                      (double)hp.eps0, (double)hp.target_accept);
        char kc[64];
        std::snprintf(kc, sizeof(kc), "%p%p%d", (void*)cmet, (void*)hp.nuts, hp.max_depth);
        std::string gk = std::string(kb) + ":" + std::to_string(blocks) + ":" + std::to_string(cpw) + kc + ":" +
                         std::to_string(hp.sync_every) + ":" + std::to_string(main_end) + ":" +
                         std::to_string(blocks1);
        if (!ctx->graph || gk != ctx->graph_key) {
            if (ctx->graph) {
                cudaGraphExecDestroy(ctx->graph);
                ctx->graph = nullptr;
            }
            cudaStream_t cs;
            CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t gr;
            CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            cudaStream_t saved = s;
            s = cs;
            cudaError_t e = enqueue();
            s = saved;
            cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) return cuda_fail(e, "capture");
            if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
            CK(cudaGraphInstantiate(&ctx->graph, gr, 0));
            cudaGraphDestroy(gr);
            ctx->graph_key = gk;
        }
        CK(cudaGraphLaunch(ctx->graph, s));
    } else {
        CK(enqueue());
    }
    CK(st.finish());
    return SPS_OK;
}

extern "C" sps_status sps_hmc_run_forward_mode(sps_ctx* ctx, const sps_hmc_config* cfg,
                                               const float* theta0_unb, const float* mag_obs,
                                               const float* sigma, const uint32_t* mask,
                                               float* samples_out, sps_hmc_stats* stats, void* stream) {
    if (!ctx || !cfg) return fail(SPS_E_INVALID_ARG, "null argument");
    if (ctx->n_gal <= 0) return fail(SPS_E_STATE, "no galaxy set");
    if (cfg->mode != SPS_APPROX) return fail(SPS_E_UNSUPPORTED, "HMC runs on the approximate path");
    if (!ctx->has_approx) return fail(SPS_E_STATE, "galaxy set built without approx tables");
    if (cfg->adapt_mass != 0) return fail(SPS_E_UNSUPPORTED, "the plain sampler uses the identity metric");
    if (cfg->sampler != SPS_HMC) return fail(SPS_E_UNSUPPORTED, "the plain sampler runs HMC");
    if (ctx->c.mdf_age) return fail(SPS_E_UNSUPPORTED, "the plain sampler supports the separable model only");
    if (cfg->chains_per_gal < 1 || cfg->chains_per_gal > 64) return fail(SPS_E_SHAPE, "chains_per_gal in [1, 64]");
    if (cfg->n_warm < 0 || cfg->n_samp < 0 || cfg->n_warm + cfg->n_samp < 1)
        return fail(SPS_E_SHAPE, "iteration counts");
    if (cfg->L_min < 1 || cfg->L_max < cfg->L_min || cfg->L_max > 4096) return fail(SPS_E_SHAPE, "L range");
    if (!(cfg->eps0 > 0) || !(cfg->target_accept > 0 && cfg->target_accept < 1))
        return fail(SPS_E_INVALID_ARG, "eps0 / target_accept");
    if (!theta0_unb || !mag_obs || !sigma || !mask) return fail(SPS_E_INVALID_ARG, "null input");
    const int64_t G = ctx->n_gal;
    const int C = cfg->chains_per_gal;
    const int64_t NC = G * C;
    if (NC > ((int64_t)1 << 31)) return fail(SPS_E_SHAPE, "too many chains");
    DeviceGuard dg(ctx->device);
    CK(dg.err);
    cudaStream_t s = (cudaStream_t)stream;
    const Consts& c = ctx->c;
    const size_t GB = (size_t)G * c.n_band;
    Stager st{ctx, s};
    const float* x0 = st.in(theta0_unb, (size_t)NC * SPS_NPARAM);
    const float* mo = st.in(mag_obs, GB);
    const float* sg = st.in(sigma, GB);
    const uint32_t* mk = st.in(mask, (size_t)G);
    float* so = st.out(samples_out, (size_t)NC * cfg->n_samp * SPS_NPARAM);
    float* acc = stats ? st.out(stats->accept_prob, (size_t)NC) : nullptr;
    float* epo = stats ? st.out(stats->step_size, (size_t)NC) : nullptr;
    int32_t* dv = stats ? st.out(stats->divergences, (size_t)NC) : nullptr;
    int64_t* nev = stats ? st.out(stats->grad_evals, (size_t)NC) : nullptr;
    int32_t* sto = stats ? st.out(stats->status, (size_t)NC) : nullptr;
    if (sps_status r = st.check(); r != SPS_OK) return r;
    HmcParams hp{C, cfg->n_warm, cfg->n_samp, cfg->L_min, cfg->L_max, cfg->target_accept, cfg->eps0,
                 cfg->seed, 0, 1};
    // state, theta, FP64 log L, gradient, chain -> galaxy, forward-mode scratch
    const int64_t chunk = std::min<int64_t>(NC, 32768);
    CK(ctx->pst.reserve(sizeof(PlainChain) * (size_t)NC));
    CK(ctx->pth.reserve(sizeof(float) * SPS_NPARAM * (size_t)NC));
    CK(ctx->pll.reserve(sizeof(double) * (size_t)NC));
    CK(ctx->pgr.reserve(sizeof(float) * SPS_NPARAM * (size_t)NC));
    CK(ctx->pgi.reserve(sizeof(int32_t) * (size_t)NC));
    CK(ctx->plainT.reserve((size_t)chunk * 9 * c.K * sizeof(float)));
    CK(ctx->plainC.reserve((size_t)chunk * c.n_band * 9 * sizeof(float)));
    PlainChain* pst = ctx->pst.as<PlainChain>();
    float* th = ctx->pth.as<float>();
    double* ll = ctx->pll.as<double>();
    float* gr = ctx->pgr.as<float>();
    int32_t* gi = ctx->pgi.as<int32_t>();
    const Galaxies gal = ctx->gal();
    auto gradient = [&](cudaStream_t q) -> cudaError_t {
        for (int64_t r0 = 0; r0 < NC; r0 += chunk) {
            const int64_t m = std::min(chunk, NC - r0);
            cudaError_t e = launch_plain(c, gal, th + r0 * SPS_NPARAM, gi + r0, m, mo, sg, mk, nullptr,
                                         gr + r0 * SPS_NPARAM, ctx->plainT.as<float>(),
                                         ctx->plainC.as<float>(), q, ll + r0);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    // one iteration: start every trajectory, then L_max rounds of gradient + step
    auto iteration = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t e = plain_hmc_start(c, hp, NC, pst, th, q);
        for (int r = 0; r < hp.L_max && e == cudaSuccess; ++r) {
            e = gradient(q);
            if (e == cudaSuccess) e = plain_hmc_step(c, hp, NC, pst, ll, gr, th, so, q);
        }
        return e;
    };
    CK(plain_hmc_init(c, NC, C, x0, hp.eps0, pst, th, gi, s));
    CK(gradient(s));
    CK(plain_hmc_absorb(c, NC, pst, ll, gr, s));
    const int n_it = hp.n_warm + hp.n_samp;
    if (cfg->use_graph) {
        cudaStream_t cs;
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t gr_it;
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = iteration(cs);
            cudaError_t e2 = cudaStreamEndCapture(cs, &gr_it);
            e = (e1 != cudaSuccess) ? e1 : e2;
            if (e == cudaSuccess) {
                e = cudaGraphInstantiate(&ex, gr_it, 0);
                cudaGraphDestroy(gr_it);
            }
        }
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return cuda_fail(e, "plain HMC capture");
        for (int it = 0; it < n_it && e == cudaSuccess; ++it) e = cudaGraphLaunch(ex, s);
        cudaGraphExecDestroy(ex);
        if (e != cudaSuccess) return cuda_fail(e, "plain HMC launch");
    } else {
        for (int it = 0; it < n_it; ++it) CK(iteration(s));
    }
    CK(plain_hmc_stats(hp, NC, pst, acc, epo, dv, nev, sto, s));
    CK(st.finish());
    return SPS_OK;
}
