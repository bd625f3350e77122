// Library context (internal): device tables, the current galaxy set and
// scratch buffers.  Shared by the C-ABI translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "sps_internal.h"

namespace sps {

// Makes `dev` the current device for the guard's lifetime and gives the
// caller's current device back on destruction, so an entry point never
// leaves a different device current behind.
struct DeviceGuard {
    int prev = -1;
    int dev;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int d) : dev(d) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Grow-only device buffer.
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t bytes) {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess) cap = bytes;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <typename T>
    T* as() const { return reinterpret_cast<T*>(p); }
};

}  // namespace sps

struct sps_ctx {
    using DevBuf = sps::DevBuf;
    using Consts = sps::Consts;
    using Grid = sps::Grid;
    using Galaxies = sps::Galaxies;
    int device = 0;
    Consts c{};
    double h0 = 70.0, om = 0.3;
    double gl_x[sps::kMaxGL], gl_w[sps::kMaxGL];
    std::vector<double> band_p0, band_p1;
    // tables
    DevBuf lam64, lam32, lamc, lamq, ssp, ssp_t, ssp_bf, ssp_t_bf, row_scale, col_scale, age_edges, bp0, bp1;
    DevBuf ssp_hi, ssp_lo, ssp_t_hi, ssp_t_lo;   // 3xTF32 halves of the FP32 tables
    DevBuf tabT, tabT64;                         // tabulated transmission samples
    // galaxies
    int64_t n_gal = 0;
    bool has_approx = false;
    DevBuf gz, glnT, glT10, gbins, gzp, gsup, ggauss, gcssp, gdust;
    DevBuf gdtdz, gdzp, gddust;       // redshift derivatives of the per-galaxy set-up
    DevBuf gdcssp;                    // d c_SSP / dz, built on the first request
    bool has_dcssp = false;
    DevBuf cJz, rowz;                 // exact path: the z accumulators and explicit z term
    // scratch
    DevBuf nonfinite, queue, err;
    DevBuf W, V, Wbar, cJ, gbar, rowinfo, tcerr, plainT, plainC, hmcm;
    DevBuf pst, pth, pll, pgr, pgi;   // plain lock-step HMC state and gradient buffers
    DevBuf hmcn;                      // NUTS tree state per chain
    DevBuf zperm;                     // redshift order of the rows of a tensor-core chunk
    DevBuf Wlo, Vlo;                  // low TF32 halves of W and v (3xTF32 exact path)
    DevBuf keep;                      // exact path: weight arrays per row, kept for the gradient
    int hmc_launches = 0;             // team-kernel launches of the last approximate-path HMC run
    cudaStream_t side = nullptr;      // HMC: the one-chain tail launch runs beside the main one
    cudaEvent_t fork = nullptr, join = nullptr;
    bool use_tc = true;   // tcgen05 contraction for BF16 operands
    DevBuf stage[12];
    // HMC graph cache
    cudaGraphExec_t graph = nullptr;
    std::string graph_key;
    std::map<std::string, std::pair<int, int>> tuned;  // key -> (warps, blocks)

    Grid grid() const {
        Grid g;
        g.lam = lam32.as<float>();
        g.lamc = lamc.as<float4>();
        g.lamq = lamq.as<float2>();
        g.lam64 = lam64.as<double>();
        g.ssp = ssp.as<float>();
        g.ssp_t = ssp_t.as<float>();
        g.ssp_bf = ssp_bf.as<uint16_t>();
        g.ssp_t_bf = ssp_t_bf.as<uint16_t>();
        g.row_scale = row_scale.as<float>();
        g.col_scale = col_scale.as<float>();
        g.band_T = tabT.as<float>();
        g.band_T64 = tabT64.as<double>();
        return g;
    }
    Galaxies gal() const {
        Galaxies g;
        g.n = n_gal;
        g.z = gz.as<float>();
        g.lnT = glnT.as<float>();
        g.lT10 = glT10.as<float>();
        g.bins = gbins.as<float2>();
        g.zp = gzp.as<double>();
        g.support = gsup.as<int2>();
        g.gauss = ggauss.as<float2>();
        g.cssp = has_approx ? gcssp.as<float>() : nullptr;
        g.dust_eff = gdust.as<float4>();
        g.dtdz = gdtdz.as<float>();
        g.dzp = gdzp.as<float>();
        g.ddust = gddust.as<float4>();
        g.dcssp = has_dcssp ? gdcssp.as<float>() : nullptr;
        return g;
    }
    ~sps_ctx() {
        sps::DeviceGuard dg(device);
        if (graph) cudaGraphExecDestroy(graph);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (side) cudaStreamDestroy(side);
        DevBuf* all[] = {&lam64, &lam32, &lamc, &lamq, &ssp, &ssp_t, &ssp_bf, &ssp_t_bf, &row_scale, &col_scale,
                         &age_edges, &bp0, &bp1, &gz, &glnT, &glT10, &gbins, &gzp, &gsup, &ggauss,
                         &gcssp, &gdust, &gdtdz, &gdzp, &gddust, &gdcssp, &cJz, &rowz, &nonfinite, &queue, &err, &W, &V, &Wbar, &cJ, &gbar,
                         &rowinfo, &tcerr, &plainT, &plainC, &hmcm, &pst, &pth, &pll, &pgr,
                         &pgi, &hmcn, &zperm, &ssp_hi, &ssp_lo, &ssp_t_hi, &ssp_t_lo, &Wlo, &Vlo, &keep, &tabT, &tabT64};
        for (DevBuf* b : all) b->release();
        for (auto& b : stage) b.release();
    }
};

