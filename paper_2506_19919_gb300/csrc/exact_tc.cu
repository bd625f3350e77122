// Tensor-core (tcgen05) contractions of the exact path (Eq. photo_integral_exact)
// for sm_103a, FP32 accumulation in TMEM, with either
//   BF16 operands (kind::f16) with per-age-row power-of-two scaling, or
//   FP32 operands as 3xTF32 (kind::tf32): x = x_hi + x_lo with x_hi the TF32
//   rounding of x, and A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped
//   A_lo B_lo term is ~2^-22 relative), which keeps FP32-level accuracy.
//
// Forward: S[r][n] = sum_k W[r][k] L[k][n] for a 128-row tile and 256-wide
// wavelength tiles, with the dust x filter reduction over n fused into the
// epilogue (the SED never reaches HBM).  Adjoint: Wbar[r][k] = sum_n v[r][n]
// L[k][n] for 128 x 224 tiles.
//
// Block of 6 warps, one block per SM: warp 0 issues TMA loads of A and B
// k-blocks (128-byte rows, 128-byte swizzle) into a ring of stages; one lane
// of warp 1 issues tcgen05.mma into one of two TMEM accumulators and commits
// to mbarriers; warps 2-5 drain the other accumulator with tcgen05.ld.  Every
// wait is bounded: a timeout sets the block's abort flag and the global error
// word, the roles unwind, in-flight copies are waited for (bounded) and TMEM
// is released.
#include <algorithm>
#include <cstdlib>

#include "exact_tc.cuh"

namespace sps {

namespace {

// ---------------------------------------------------------------- wait probe
// Exercises the pipeline's bounded wait: warp 0 waits on an mbarrier that
// warp 1 arrives on when `ready`; otherwise nothing completes it, the wait
// gives up after `limit` polls, sets the abort flag and raises error bit 2,
// and the kernel returns normally.
__global__ void __launch_bounds__(64) k_wait_probe(int ready, uint32_t limit, int* err) {
    __shared__ Ctl ctl;
    if (threadIdx.x == 0) {
        tc::mbar_init(&ctl.drain, 1);
        ctl.abort = 0;
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 32 && ready) tc::mbar_arrive(&ctl.drain);
    if (threadIdx.x == 0) wait_or_abort(&ctl.drain, 0u, &ctl, err, limit);
    __syncthreads();
}

// ---------------------------------------------------------------- adjoint
template <bool TF>
__global__ void __launch_bounds__(kThreadsTC, 1)
k_adj_tc(const __grid_constant__ TcMaps tm, const __grid_constant__ Consts c, const Grid grid, int64_t n,
         float* __restrict__ Wbar, int* err, int tpc) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int ST = TF ? 2 : kAdjStages;
    using R = Ring<kAdjBN, ST, TF>;
    Ctl* ctl;
    uint8_t* ring = carve<kAdjBN, ST, TF>(smem_raw, ctl);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // a block takes tpc of the row block's n tiles; the groups of a row block
    // are adjacent in launch order, so they run together and read its V rows
    // from L2 after the first has brought them in
    const int n_tiles_all = (c.K + kAdjBN - 1) / kAdjBN;
    const int groups = (n_tiles_all + tpc - 1) / tpc;
    const int m0 = (int)(blockIdx.x / groups) * kTM;
    const int nt0 = (int)(blockIdx.x % groups) * tpc;
    const int n_tiles = min(tpc, n_tiles_all - nt0);
    const int n_kb = (c.lam_pad + R::kBK - 1) / R::kBK;   // the last block reads zero fill
    const int kchunk = n_kb;                                // one accumulation per tile
    const int n_kc = (n_kb + kchunk - 1) / kchunk;
    tc_setup<ST>(ctl, warp);
    if (warp == 0) {
        if (lane == 0) tc_produce<kAdjBN, ST, TF>(ctl, ring, tm.a, tm.b, m0, n_tiles, n_kb, err, kchunk, nt0);
    } else if (warp == 1) {
        if (lane == 0) tc_mma<kAdjBN, ST, TF>(ctl, ring, n_tiles, n_kb, err, kchunk);
    } else {
        const int q = warp & 3;
        const int64_t row = (int64_t)m0 + 32 * q + lane;
        const bool live = row < n;
        for (int item = 0; item < n_tiles * n_kc; ++item) {
            const int buf = item & 1;
            const uint32_t use = (uint32_t)(item >> 1);
            const int nt = item / n_kc, kc = item - nt * n_kc;
            if (!warp_wait(&ctl->tfull[buf], use & 1u, ctl, err)) break;
            tc::tc_fence_after();
            for (int cc = 0; cc < kAdjBN / 32; ++cc) {
                float S[32];
                tc::tmem_ld32(ctl->tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * kAdjBN + cc * 32), S);
                const int k0 = (nt0 + nt) * kAdjBN + cc * 32;
                if (live) {
                    // 16-byte stores (k_pad is a multiple of 64, k0 of 32): a lane
                    // owns one row, so each store covers half a sector, not an eighth
                    float* orow = Wbar + row * c.k_pad;
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const int k = k0 + j;
                        float v[4];
                        float cs[4] = {1.0f, 1.0f, 1.0f, 1.0f};
                        if (!TF) {
                            const float4 c4 = __ldg(reinterpret_cast<const float4*>(grid.col_scale + k));
                            cs[0] = c4.x; cs[1] = c4.y; cs[2] = c4.z; cs[3] = c4.w;
                        }
#pragma unroll
                        for (int t = 0; t < 4; ++t) v[t] = TF ? S[j + t] : S[j + t] * cs[t];
                        if (k + 3 < c.K) {
                            float4* o = reinterpret_cast<float4*>(orow + k);
                            if (kc == 0) {
                                *o = make_float4(v[0], v[1], v[2], v[3]);
                            } else {
                                float4 p = *o;
                                *o = make_float4(p.x + v[0], p.y + v[1], p.z + v[2], p.w + v[3]);
                            }
                        } else {
#pragma unroll
                            for (int t = 0; t < 4; ++t)
                                if (k + t < c.K) {
                                    if (kc == 0) orow[k + t] = v[t];
                                    else orow[k + t] += v[t];
                                }
                        }
                    }
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&ctl->tempty[buf]);
        }
    }
    tc_teardown<ST>(ctl, warp);
}

}  // namespace

size_t tc_fwd_smem(bool tf) {
    return (tf ? Ring<kFwdBNtf, kFwdStagesTf, true>::kBytes : Ring<kFwdBN, kFwdStages, false>::kBytes) + 256 +
           kFwdConstBytes + 1024;
}
size_t tc_adj_smem(bool tf) {
    return (tf ? Ring<kAdjBN, 2, true>::kBytes : Ring<kAdjBN, kAdjStages, false>::kBytes) + sizeof(Ctl) + 1024;
}

cudaError_t launch_fwd_tc(const TcMaps& tm, bool tf, const Consts& c, const Grid& grid, const Galaxies& g,
                          const float* theta, const int32_t* gal_idx, const int32_t* perm, int64_t n, float* cJ,
                          int* err, cudaStream_t s, float* cJz) {
    if (cJz) return launch_fwd_tc_z(tm, tf, c, grid, g, theta, gal_idx, perm, n, cJ, err, s, cJz);
    return fwd_tc_launch<false>(tm, tf, c, grid, g, theta, gal_idx, perm, n, cJ, err, s, nullptr);
}

cudaError_t launch_adj_tc(const TcMaps& tm, bool tf, const Consts& c, const Grid& grid, int64_t n, float* Wbar,
                          int* err, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    // n tiles per block (SPS_ADJ_TPC overrides; tuning only): 3 keeps the
    // TMEM double buffer busy while the row block's 2 blocks share V in L2
    // (measured 2-7% faster than one block streaming V for all 6 tiles)
    const int n_tiles_all = (c.K + kAdjBN - 1) / kAdjBN;
    int tpc = 3;
    if (const char* v = std::getenv("SPS_ADJ_TPC")) tpc = std::atoi(v);
    tpc = std::max(1, std::min(tpc, n_tiles_all));
    const int groups = (n_tiles_all + tpc - 1) / tpc;
    const unsigned blocks = (unsigned)(((n + kTM - 1) / kTM) * groups);
    const size_t smem = tc_adj_smem(tf);
    cudaError_t e;
    if (tf) {
        e = cudaFuncSetAttribute(k_adj_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_adj_tc<true><<<blocks, kThreadsTC, smem, s>>>(tm, c, grid, n, Wbar, err, tpc);
    } else {
        e = cudaFuncSetAttribute(k_adj_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_adj_tc<false><<<blocks, kThreadsTC, smem, s>>>(tm, c, grid, n, Wbar, err, tpc);
    }
    return cudaGetLastError();
}

cudaError_t launch_wait_probe(int ready, uint32_t limit, int* err, cudaStream_t s) {
    k_wait_probe<<<1, 64, 0, s>>>(ready, limit, err);
    return cudaGetLastError();
}

}  // namespace sps
