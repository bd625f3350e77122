// Tabulated filter transmission (SPS_BAND_TABLE): the linear interpolant of
// samples T[0..n-1] taken at l = start + m * step (observed frame), zero
// outside the samples.  u = (l_obs - start) / step is the sample coordinate.
#pragma once

#include <cuda_runtime.h>

namespace sps {

// FP64, for the once-per-galaxy set-up (zero points, lambda_eff, c_SSP).
__device__ __forceinline__ double tab_T64(const double* __restrict__ T, int n, double u) {
    if (!(u >= 0.0 && u <= (double)(n - 1))) return 0.0;
    const int m = min((int)u, n - 2);
    const double f = u - (double)m;
    return T[m] + f * (T[m + 1] - T[m]);
}

// dT/du of the interpolant (the slope of the segment holding u; zero outside
// the samples), FP64, for the redshift derivatives of the set-up.
__device__ __forceinline__ double tab_dT64(const double* __restrict__ T, int n, double u) {
    if (!(u >= 0.0 && u <= (double)(n - 1))) return 0.0;
    const int m = min((int)u, n - 2);
    return T[m + 1] - T[m];
}

// FP32, for the exact-path epilogues.
__device__ __forceinline__ float tab_T32(const float* __restrict__ T, int n, float u) {
    if (!(u >= 0.0f && u <= (float)(n - 1))) return 0.0f;
    const int m = min((int)u, n - 2);
    const float t0 = __ldg(T + m);
    return fmaf(u - (float)m, __ldg(T + m + 1) - t0, t0);
}

// dT/du of the interpolant, FP32 (the exact-path epilogues' redshift terms).
__device__ __forceinline__ float tab_dT32(const float* __restrict__ T, int n, float u) {
    if (!(u >= 0.0f && u <= (float)(n - 1))) return 0.0f;
    const int m = min((int)u, n - 2);
    return __ldg(T + m + 1) - __ldg(T + m);
}

}  // namespace sps
