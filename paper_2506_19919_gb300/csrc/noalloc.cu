// Exact FP32 photometry without any device allocation.
//
// Some callers cannot call cudaMalloc once they are running: services that
// reserve a fixed device-memory budget at start-up and must not grow it,
// hosts whose own allocator owns the device memory and forbids allocations
// behind its back, and latency-critical loops where cudaMalloc / cudaFree
// would synchronise the device or fail on a fragmented or fully reserved
// heap.  sps_photometry() grows context-owned scratch buffers on demand;
// this entry point instead places its scratch (the SSP weights W and the
// per-band reduction A of the exact path) in a file-scope __device__ array of
// fixed size that is part of the loaded module, so a call allocates nothing.
//
// The array lives on every GPU that loads the library until the process
// exits.  Host code reaches it only through cudaGetSymbolAddress: the array's
// name in host code is a host-side stand-in, not a device address.  The
// address is looked up once per device (again if the device's context was
// reset in between), the first time this entry point runs with that device
// current; that first call should therefore come before any stream capture.
// The caller's current device is restored before the call returns.  All
// calls share the array and leave their contents in it;
// every element a call reads is written earlier in the same call (weights
// including their zero padding, then the reduction), so nothing needs
// clearing.  Calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "ctx.h"
#include "sps_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB on every device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// per device: the scratch address and the ID of the context it belongs to
struct ScratchAddr {
    void* ptr = nullptr;
    unsigned long long ctx_id = 0;
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

sps_status fail(sps_status s, const std::string& msg) {
    sps::set_last_error(("sps_photometry_exact_noalloc: " + msg).c_str());
    return s;
}

sps_status cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();
    return fail(SPS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The unique ID of the current device's context (driver entry points
// cuCtxGetCurrent / cuCtxGetId, reached through the runtime); 0 if unknown.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(p);
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

}  // namespace

extern "C" sps_status sps_photometry_exact_noalloc(sps_ctx* ctx, const float* theta,
                                                   const int32_t* gal_idx, int64_t n,
                                                   float* mag_out, void* stream) {
    if (!ctx) return fail(SPS_E_INVALID_ARG, "null context");
    if (ctx->n_gal <= 0) return fail(SPS_E_STATE, "no galaxy set: call sps_set_galaxies first");
    if (n < 0) return fail(SPS_E_SHAPE, "negative row count");
    if (n == 0) return SPS_OK;
    if (!theta || !mag_out) return fail(SPS_E_INVALID_ARG, "theta or mag_out is NULL");
    if (!gal_idx && n != ctx->n_gal)
        return fail(SPS_E_SHAPE, "gal_idx is NULL but n differs from the galaxy count");
    const sps::Consts& c = ctx->c;
    // rows that fit: each row takes 4 * k_pad bytes of weights and 16 * n_band
    // of band reductions (plus at most 255 bytes of alignment per part)
    const size_t per_row = (size_t)c.k_pad * sizeof(float) + (size_t)c.n_band * 4 * sizeof(float);
    if ((uint64_t)n > (kScratchBytes - 512) / per_row)
        return fail(SPS_E_SHAPE, "n = " + std::to_string(n) + " rows need more than the 32 MiB static "
                    "scratch (at most " + std::to_string((kScratchBytes - 512) / per_row) +
                    " rows on this grid); call it on fewer rows at a time");
    const size_t w_bytes = align256((size_t)n * c.k_pad * sizeof(float));
    const size_t a_bytes = align256((size_t)n * c.n_band * 4 * sizeof(float));
    if (w_bytes + a_bytes > kScratchBytes) return fail(SPS_E_SHAPE, "scratch size");
    // staging a host array would need a device buffer: device pointers only,
    // and in the memory of the context's own device
    const int lt = sps::pointer_location(theta, ctx->device);
    const int lm = sps::pointer_location(mag_out, ctx->device);
    const int lg = gal_idx ? sps::pointer_location(gal_idx, ctx->device) : 1;
    if (lt < 0 || lm < 0 || lg < 0)
        return fail(SPS_E_INVALID_ARG, "theta, gal_idx and mag_out must live on the context's device");
    if (lt == 0 || lm == 0 || lg == 0)
        return fail(SPS_E_INVALID_ARG, "theta, gal_idx and mag_out must be device pointers (host "
                    "arrays would need staging allocations)");
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return fail(SPS_E_UNSUPPORTED, "device ordinal beyond the scratch address table");
    sps::DeviceGuard dg(ctx->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        ScratchAddr& a = g_scratch_addr[ctx->device];
        const unsigned long long id = current_context_id();
        if (!a.ptr || id == 0 || id != a.ctx_id) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) {
                a = ScratchAddr{};
                return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
            }
            a.ptr = p;
            a.ctx_id = id;
        }
        base = a.ptr;
    }
    float* W = static_cast<float*>(base);
    float* A = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + w_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    const sps::Grid grid = ctx->grid();
    const sps::Galaxies gal = ctx->gal();
    int* nf = ctx->nonfinite.as<int>();
    cudaError_t e;
    if ((e = cudaMemsetAsync(nf, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if ((e = sps::launch_exact_weights(c, grid, gal, theta, gal_idx, n, 0, W, nullptr, s)) != cudaSuccess)
        return cuda_fail(e, "weights launch");
    if ((e = sps::launch_exact_fwd(c, grid, gal, theta, gal_idx, n, 0, W, nullptr, A, s)) != cudaSuccess)
        return cuda_fail(e, "contraction launch");
    if ((e = sps::launch_exact_like(c, gal, theta, gal_idx, n, A, nullptr, nullptr, nullptr, nullptr,
                                    mag_out, nullptr, nullptr, nf, s)) != cudaSuccess)
        return cuda_fail(e, "magnitude launch");
    int flag = 0;
    if ((e = cudaMemcpyAsync(&flag, nf, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (flag) return fail(SPS_E_NONFINITE, "some rows are NaN (non-finite inputs or results)");
    return SPS_OK;
}
