// Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11)
// and the HMC draws built on it.  Counter layout per chain and iteration:
// (iteration, block, chain, 0), key = 64-bit seed; blocks 0-2 -> 12 uniforms
// -> 6 Box-Muller pairs (momenta), block 3 -> word 0: accept uniform,
// word 1: trajectory length L = L_min + (word * n) >> 32, n = L_max - L_min + 1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sps {

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// (word + 1/2) 2^-32, in (0, 1), exact in FP64.
__device__ __forceinline__ double u01_d(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }
// The same in FP32, rounded; in (0, 1].
__device__ __forceinline__ float u01_f(uint32_t w) { return fmaf((float)w, 2.3283064e-10f, 1.1641532e-10f); }

}  // namespace sps
