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
// address is looked up once per device, the first time this entry point runs
// with that device current; that first call should therefore come before any
// stream capture.  All calls share the array and leave their contents in it;
// every element a call reads is written earlier in the same call (weights
// including their zero padding, then the reduction), so nothing needs
// clearing.  Calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "ctx.h"
#include "sps_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB on every device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

bool device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" sps_status sps_photometry_exact_noalloc(sps_ctx* ctx, const float* theta,
                                                   const int32_t* gal_idx, int64_t n,
                                                   float* mag_out, void* stream) {
    if (!ctx) return SPS_E_INVALID_ARG;
    if (ctx->n_gal <= 0) return SPS_E_STATE;
    if (n < 0) return SPS_E_SHAPE;
    if (n == 0) return SPS_OK;
    if (!theta || !mag_out) return SPS_E_INVALID_ARG;
    if (!gal_idx && n != ctx->n_gal) return SPS_E_SHAPE;
    const sps::Consts& c = ctx->c;
    const size_t w_bytes = align256((size_t)n * c.k_pad * sizeof(float));
    const size_t a_bytes = align256((size_t)n * c.n_band * 4 * sizeof(float));
    if (w_bytes + a_bytes > kScratchBytes) {
        sps::set_last_error("sps_photometry_exact_noalloc: n rows need more than the 32 MiB "
                            "static scratch (4 * k_pad + 16 * n_band bytes per row); call it on "
                            "fewer rows at a time");
        return SPS_E_SHAPE;
    }
    // staging a host array would need a device buffer: device pointers only
    if (!device_ptr(theta) || !device_ptr(mag_out) || (gal_idx && !device_ptr(gal_idx))) {
        sps::set_last_error("sps_photometry_exact_noalloc: theta, gal_idx and mag_out must be "
                            "device pointers (host arrays would need staging allocations)");
        return SPS_E_INVALID_ARG;
    }
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return SPS_E_UNSUPPORTED;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return SPS_E_CUDA;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_ptr[ctx->device]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                sps::set_last_error("sps_photometry_exact_noalloc: cudaGetSymbolAddress failed");
                return SPS_E_CUDA;
            }
            g_scratch_ptr[ctx->device] = p;
        }
        base = g_scratch_ptr[ctx->device];
    }
    float* W = static_cast<float*>(base);
    float* A = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + w_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    const sps::Grid grid = ctx->grid();
    const sps::Galaxies gal = ctx->gal();
    int* nf = ctx->nonfinite.as<int>();
    if (cudaMemsetAsync(nf, 0, sizeof(int), s) != cudaSuccess) return SPS_E_CUDA;
    if (sps::launch_exact_weights(c, grid, gal, theta, gal_idx, n, 0, W, nullptr, s) != cudaSuccess ||
        sps::launch_exact_fwd(c, grid, gal, theta, gal_idx, n, 0, W, nullptr, A, s) != cudaSuccess ||
        sps::launch_exact_like(c, gal, theta, gal_idx, n, A, nullptr, nullptr, nullptr, nullptr,
                               mag_out, nullptr, nullptr, nf, s) != cudaSuccess)
        return SPS_E_CUDA;
    int flag = 0;
    if (cudaMemcpyAsync(&flag, nf, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SPS_E_CUDA;
    return flag ? SPS_E_NONFINITE : SPS_OK;
}
