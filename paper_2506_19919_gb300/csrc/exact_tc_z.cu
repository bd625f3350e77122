// The tensor-core forward contraction of the exact path with the redshift
// derivative of the band weights accumulated in its epilogue (the z column of
// sps_loglike_grad_z).  A translation unit of its own so that these
// instantiations compile in parallel with exact_tc.cu.
#include "exact_tc.cuh"

namespace sps {

cudaError_t launch_fwd_tc_z(const TcMaps& tm, bool tf, const Consts& c, const Grid& grid, const Galaxies& g,
                            const float* theta, const int32_t* gal_idx, const int32_t* perm, int64_t n,
                            float* cJ, int* err, cudaStream_t s, float* cJz) {
    return fwd_tc_launch<true>(tm, tf, c, grid, g, theta, gal_idx, perm, n, cJ, err, s, cJz);
}

}  // namespace sps
