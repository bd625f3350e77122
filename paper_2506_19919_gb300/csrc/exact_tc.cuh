// Shared pieces of the tensor-core (tcgen05) exact-path kernels: tile
// constants, the TMA / MMA / TMEM pipeline roles with bounded waits, and the
// forward contraction with its fused dust x filter epilogue (k_fwd_tc).
// Included by exact_tc.cu and exact_tc_z.cu, which instantiate it (each
// translation unit gets its own copy of these internal definitions).
#pragma once

#include <cuda.h>

#include <type_traits>

#include "band_tab.cuh"
#include "sps_device.cuh"
#include "tc_ptx.cuh"

namespace sps {

namespace {

constexpr int kTM = 128;       // rows per tile (MMA M)
constexpr int kRowBytes = 128; // one k-block row: 64 BF16 or 32 FP32 (128-byte swizzle)
constexpr int kThreadsTC = 192;   // adjoint: TMA warp, MMA warp, 4 epilogue warps
constexpr int kFwdGroupBands = 8; // forward: bands per epilogue warp
constexpr int kFwdMaxEpiWarps = 16;
constexpr int kFwdBN = 256;
constexpr int kFwdStages = 4;    // BF16 ring depth
// 3xTF32 forward: 128-column tiles, each with two TMEM accumulators (the
// hi x hi product, and the hi x lo + lo x hi corrections, added in FP32 in the
// epilogue), so that the large accumulator takes a third of the additions:
// the tensor core's FP32 accumulation loses a fraction of an ulp per addition
// in one direction, which over 3 x 168 additions left fluxes ~1.5e-5 low
constexpr int kFwdBNtf = 128;
constexpr int kFwdStagesTf = 3;  // four 16 KB tiles per stage
constexpr int kAdjBN = 224;      // K = 1344 = 6 x 224: each 128-row block streams V six times
constexpr int kAdjStages = 5;    // BF16 ring depth (TF32: 2)
constexpr uint32_t kTmemCols = 512;
// Forward epilogue: per warp, the wavelength constants (lamc, lam) of the
// 32-column chunk being processed, staged in shared memory after the control
// block (the next chunk's are loaded into registers meanwhile).
constexpr int kFwdConstBytes = kFwdMaxEpiWarps * 32 * (16 + 4);

// Ring of STAGES stages; a stage holds an A tile (kTM rows) and a B tile (BN
// rows) of one k-block, twice (hi and lo parts) for 3xTF32.
template <int BN, int STAGES, bool TF>
struct Ring {
    static constexpr int kBK = TF ? 32 : 64;          // k per block row
    static constexpr int kParts = TF ? 2 : 1;
    static constexpr int kA = kTM * kRowBytes;
    static constexpr int kB = BN * kRowBytes;
    static constexpr int kStage = kParts * (kA + kB);
    static constexpr int kBytes = STAGES * kStage;
};

struct Ctl {
    uint64_t full[8], empty[8];
    uint64_t tfull[2], tempty[2];
    uint64_t drain;
    uint32_t tmem_base;
    volatile int abort;
    int issued;
};

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, Ctl* ctl, int* err,
                                              uint32_t limit = tc::kSpinLimit);

// Warp-uniform wait: lane 0 polls, the outcome is broadcast.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, Ctl* ctl, int* err) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = wait_or_abort(bar, parity, ctl, err) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, Ctl* ctl, int* err,
                                              uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 1023) == 1023 && ctl->abort) return false;
    }
    ctl->abort = 1;
    atomicOr(err, 2);
    return false;
}

// Shared prologue: barriers and TMEM allocation.  Returns the ring base.
template <int STAGES>
__device__ __forceinline__ void tc_setup(Ctl* ctl, int warp, int epi_threads = 4 * 32) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&ctl->full[s], 1);
            tc::mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&ctl->tfull[b], 1);
            tc::mbar_init(&ctl->tempty[b], epi_threads);
        }
        tc::mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        ctl->issued = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&ctl->tmem_base, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
}

// Producer (one lane): k-blocks of A (rows m0..) and B (rows of the n tile).
// Stage layout: A_hi, B_hi, then (3xTF32) A_lo, B_lo.  tA[1], tB[1] are the
// lo-part maps (unused for BF16).
// Work items: (output tile nt, k chunk kc) for nt < n_tiles, kc < ceil(n_kb / kchunk);
// an item accumulates k-blocks [kc kchunk, min((kc + 1) kchunk, n_kb)) from zero.
template <int BN, int STAGES, bool TF>
__device__ __forceinline__ void tc_produce(Ctl* ctl, uint8_t* ring, const CUtensorMap* tA,
                                           const CUtensorMap* tB, int m0, int n_tiles, int n_kb,
                                           int* err, int kchunk, int nt0 = 0) {
    using R = Ring<BN, STAGES, TF>;
    int it = 0;
    const int n_items = n_tiles * ((n_kb + kchunk - 1) / kchunk);
    const int n_kc = (n_kb + kchunk - 1) / kchunk;
    for (int item = 0; item < n_items && !ctl->abort; ++item) {
        const int nt = item / n_kc, kc = item - nt * n_kc;
        const int kb_end = min((kc + 1) * kchunk, n_kb);
        for (int kb = kc * kchunk; kb < kb_end; ++kb, ++it) {
            const int s = it % STAGES;
            const uint32_t round = (uint32_t)(it / STAGES);
            if (!wait_or_abort(&ctl->empty[s], (round & 1u) ^ 1u, ctl, err)) return;
            uint8_t* a = ring + s * R::kStage;
            uint8_t* b = a + R::kA;
            tc::mbar_expect_tx(&ctl->full[s], R::kStage);
            tc::tma_load_2d(a, &tA[0], kb * R::kBK, m0, &ctl->full[s]);
            tc::tma_load_2d(b, &tB[0], kb * R::kBK, (nt0 + nt) * BN, &ctl->full[s]);
            if (TF) {
                tc::tma_load_2d(b + R::kB, &tA[1], kb * R::kBK, m0, &ctl->full[s]);
                tc::tma_load_2d(b + R::kB + R::kA, &tB[1], kb * R::kBK, (nt0 + nt) * BN, &ctl->full[s]);
            }
            ctl->issued = it + 1;
        }
    }
}

// MMA issuer (one lane).  SPLIT (3xTF32): per buffer two accumulators of
// BN columns, the hi x hi product in the first, the two correction products
// in the second.
template <int BN, int STAGES, bool TF, bool SPLIT = false>
__device__ __forceinline__ void tc_mma(Ctl* ctl, uint8_t* ring, int n_tiles, int n_kb, int* err,
                                       int kchunk) {
    using R = Ring<BN, STAGES, TF>;
    constexpr uint32_t idesc = TF ? tc::idesc_tf32(kTM, BN) : tc::idesc_bf16(kTM, BN);
    int it = 0;
    const int n_kc = (n_kb + kchunk - 1) / kchunk;
    const int n_items = n_tiles * n_kc;
    for (int item = 0; item < n_items; ++item) {
        const int buf = item & 1;
        const uint32_t use = (uint32_t)(item >> 1);
        const int kc = item % n_kc;
        const int kb0 = kc * kchunk, kb_end = min(kb0 + kchunk, n_kb);
        if (!wait_or_abort(&ctl->tempty[buf], (use & 1u) ^ 1u, ctl, err)) break;
        tc::tc_fence_after();
        const uint32_t d = ctl->tmem_base + (uint32_t)(buf * (SPLIT ? 2 * BN : BN));
        const uint32_t dc = SPLIT ? d + (uint32_t)BN : d;        // corrections
        bool ok = true;
        for (int kb = kb0; kb < kb_end; ++kb, ++it) {
            const int s = it % STAGES;
            const uint32_t round = (uint32_t)(it / STAGES);
            if (!wait_or_abort(&ctl->full[s], round & 1u, ctl, err)) {
                ok = false;
                break;
            }
            tc::tc_fence_after();
            uint8_t* a = ring + s * R::kStage;
            uint8_t* b = a + R::kA;
            const uint64_t da = tc::sw128_desc(a), db = tc::sw128_desc(b);
            if (TF) {
                const uint64_t dal = tc::sw128_desc(b + R::kB), dbl = tc::sw128_desc(b + R::kB + R::kA);
                // four k-steps of 8 FP32 (32 bytes) per 128-byte row
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool acc = ((kb - kb0) | k) != 0;
                    tc::mma_tf32(dc, da + 2 * k, dbl + 2 * k, idesc, acc);                 // hi lo
                    tc::mma_tf32(dc, dal + 2 * k, db + 2 * k, idesc, 1);                   // lo hi
                    tc::mma_tf32(d, da + 2 * k, db + 2 * k, idesc, SPLIT ? acc : true);   // hi hi
                }
            } else {
                // four k-steps of 16 BF16 (32 bytes) per 128-byte row
#pragma unroll
                for (int k = 0; k < 4; ++k) tc::mma_bf16(d, da + 2 * k, db + 2 * k, idesc, ((kb - kb0) | k) != 0);
            }
            tc::mma_commit(&ctl->empty[s]);
        }
        if (!ok) break;
        tc::mma_commit(&ctl->tfull[buf]);
    }
    // all issued MMAs complete before TMEM is released
    tc::mma_commit(&ctl->drain);
    for (uint32_t i = 0; i < tc::kSpinLimit; ++i)
        if (tc::mbar_try_wait(&ctl->drain, 0)) break;
}

// Teardown: wait (bounded) for the producer's copies still in flight, then
// free TMEM from the allocating warp.
template <int STAGES>
__device__ __forceinline__ void tc_teardown(Ctl* ctl, int warp) {
    __syncwarp();
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int issued = ctl->issued;
        for (int it = max(0, issued - STAGES); it < issued; ++it) {
            const int s = it % STAGES;
            const uint32_t round = (uint32_t)(it / STAGES);
            for (uint32_t i = 0; i < tc::kSpinLimit; ++i)
                if (tc::mbar_try_wait(&ctl->full[s], round & 1u)) break;
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(ctl->tmem_base, kTmemCols);
    }
}

static_assert(sizeof(Ctl) <= 256, "control block must fit before the staging area");

template <int BN, int STAGES, bool TF>
__device__ __forceinline__ uint8_t* carve(unsigned char* raw, Ctl*& ctl) {
    uintptr_t p = reinterpret_cast<uintptr_t>(raw);
    p = (p + 1023) & ~uintptr_t(1023);
    uint8_t* ring = reinterpret_cast<uint8_t*>(p);
    ctl = reinterpret_cast<Ctl*>(ring + Ring<BN, STAGES, TF>::kBytes);
    return ring;
}

// ---------------------------------------------------------------- forward
// Epilogue layout: 4 x n_groups x n_halves warps.  A warp reads the TMEM lane
// quarter q = (warp id mod 4) (32 rows) of each tile, for the bands of its group (<= 8, held in
// registers) and, when one group covers all bands, for one half of the tile's
// columns.  Rows arrive sorted by redshift (perm), so the 32 rows of a warp see
// nearly the same band supports: a band is visited in a 32-column chunk only if
// it overlaps the chunk in some lane.
// KZ also accumulates the redshift derivative of the band weights,
// wb' = q_n T'((1+z) l_n), into cJz[row][b][2] = sum_n wb' S (1, E).
template <int MAXT, bool TF, bool KZ = false>
__global__ void __launch_bounds__(MAXT, 1)
k_fwd_tc(const __grid_constant__ TcMaps tm, const __grid_constant__ Consts c, const Grid grid, const Galaxies g,
         const float* __restrict__ theta, const int32_t* __restrict__ gal_idx,
         const int32_t* __restrict__ perm, int64_t n, int n_halves, float* __restrict__ cJ, int* err,
         float* __restrict__ cJz) {
    constexpr int NB = kFwdGroupBands;
    extern __shared__ unsigned char smem_raw[];
    Ctl* ctl;
    constexpr int BN = TF ? kFwdBNtf : kFwdBN;
    constexpr int ST = TF ? kFwdStagesTf : kFwdStages;
    constexpr int ACC = TF ? 2 * BN : BN;          // TMEM columns per buffer
    using R = Ring<BN, ST, TF>;
    uint8_t* ring = carve<BN, ST, TF>(smem_raw, ctl);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kTM;
    const int n_tiles = (c.n_lam + BN - 1) / BN;
    const int n_kb = (c.k_pad + R::kBK - 1) / R::kBK;
    const int epi_threads = (int)blockDim.x - 64;
    tc_setup<ST>(ctl, warp, epi_threads);
    if (warp == 0) {
        if (lane == 0) tc_produce<BN, ST, TF>(ctl, ring, tm.a, tm.b, m0, n_tiles, n_kb, err, n_kb);
    } else if (warp == 1) {
        if (lane == 0) tc_mma<BN, ST, TF, TF>(ctl, ring, n_tiles, n_kb, err, n_kb);
    } else {
        const int e = warp - 2;
        const int q = warp & 3;                    // TMEM lane quarter this warp may access (warp id mod 4)
        const int half = (e >> 2) % n_halves;      // column half (one group only)
        const int B = c.n_band;
        // the bands split evenly over the groups (12 bands: 6 + 6, not 8 + 4);
        // this warp's bands are [b0, b_end)
        const int n_groups = (B + NB - 1) / NB;
        const int bpg = (B + n_groups - 1) / n_groups;
        const int b0 = ((e >> 2) / n_halves) * bpg;
        const int b_end = min(b0 + bpg, B);
        const int ncol = BN / n_halves;
        const int rl = 32 * q + lane;
        const int64_t pos = (int64_t)m0 + rl;
        const bool live = pos < n;
        const int64_t row = live ? (perm ? (int64_t)perm[pos] : pos) : 0;
        int64_t gi = live ? (gal_idx ? (int64_t)gal_idx[row] : row) : 0;
        const bool valid = live && gi >= 0 && gi < g.n;
        if (!valid) gi = 0;
        float cA = 0.f, dl = 0.f, eb = 0.f;
        if (valid) {
            const float* t = theta + row * SPS_NPARAM;
            cA = -0.4f * kLog2_10f * t[9] * (1.0f / 4.05f);
            dl = t[10];
            eb = fmaxf(0.85f - 1.9f * dl, 0.0f);
        }
        const float dl2 = dl * 1.4426950408889634f;     // delta log2(e)
        const float nd19 = eb > 0.0f ? -1.9f : 0.0f;    // d E_b / d delta
        uint32_t sxy[NB];                          // support [lo, hi): lo | hi << 16
        float gc[NB], gs[NB];
        float acc[NB][4];
        float accz[KZ ? NB : 1][2];                // KZ: sum wb' S (1, E)
        const float iopz = (KZ && valid) ? 1.0f / (1.0f + g.z[gi]) : 0.0f;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int b = b0 + k;
            int2 sp = make_int2(0, 0);
            float2 ga = make_float2(0.f, 0.f);
            if (b < b_end && valid) {
                sp = g.support[gi * B + b];
                ga = g.gauss[gi * B + b];
            }
            sxy[k] = (uint32_t)sp.x | ((uint32_t)sp.y << 16);
            gc[k] = ga.x;
            gs[k] = (b < b_end && c.band_kind[b] != 0) ? ga.y : 0.0f;   // 0 top-hat, > 0 Gaussian, < 0 table
            acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.0f;
            if (KZ) accz[k][0] = accz[k][1] = 0.0f;
        }
        // warp-wide hull of each band's support (lanes without the band excluded):
        // a group is visited for a band if the hull reaches it
        int hlo[NB], hhi[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int lo = (int)(sxy[k] & 0xffffu), hi = (int)(sxy[k] >> 16);
            hlo[k] = (int)__reduce_min_sync(0xffffffffu, (unsigned)(lo < hi ? lo : 0xffff));
            hhi[k] = (int)__reduce_max_sync(0xffffffffu, (unsigned)(lo < hi ? hi : 0));
        }
        bool has_tab = false;                      // a tabulated band in this warp's group
#pragma unroll
        for (int k = 0; k < NB; ++k) has_tab = has_tab || (b0 + k < b_end && c.band_kind[b0 + k] == 2);
        // this warp's staging of the chunk constants (lane j: column nb0 + j,
        // clamped to the grid), and the registers holding the next chunk's
        float4* cst4 = reinterpret_cast<float4*>(reinterpret_cast<uint8_t*>(ctl) + 256) + 32 * e;
        float* cstl = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(ctl) + 256 + kFwdMaxEpiWarps * 32 * 16) +
                      32 * e;
        float4 pL4;
        float pl;
        {
            const int nn = min(half * ncol + lane, c.n_lam - 1);
            pL4 = __ldg(grid.lamc + nn);
            pl = __ldg(grid.lam + nn);
        }
        for (int nt = 0; nt < n_tiles; ++nt) {
            const int buf = nt & 1;
            const uint32_t use = (uint32_t)(nt >> 1);
            if (!warp_wait(&ctl->tfull[buf], use & 1u, ctl, err)) break;
            tc::tc_fence_after();
            const int col0 = nt * BN + half * ncol;
            const int col_end = min(col0 + ncol, c.n_lam);
            for (int cc = 0; cc < ncol / 32; ++cc) {
                const int nb0 = col0 + cc * 32;
                if (nb0 >= c.n_lam) break;                 // warp-uniform
                // publish this chunk's constants, then load the next chunk's
                // (the next one processed: in this tile, else the next tile's first)
                __syncwarp();
                cst4[lane] = pL4;
                cstl[lane] = pl;
                __syncwarp();
                {
                    const int nx = (nb0 + 32 < col_end) ? nb0 + 32 : (nt + 1) * BN + half * ncol;
                    const int nn = min(nx + lane, c.n_lam - 1);
                    pL4 = __ldg(grid.lamc + nn);
                    pl = __ldg(grid.lam + nn);
                }
                const uint32_t taddr = ctl->tmem_base + ((uint32_t)(32 * q) << 16) +
                                       (uint32_t)(buf * ACC + half * ncol + cc * 32);
                // 32 columns x this warp's bands, in groups of CG columns: the
                // band-independent terms of a column (S q / lambda and its
                // products with E = 10^-0.4A, E base and E dterm, which give c
                // and the A_V and delta factors) are formed once per group, then
                // each band whose support some lane reaches in the group adds
                // its weights over the group's columns (independent columns, so
                // the band loop keeps its ILP).  Columns past the grid carry
                // S = 0 (zero-filled table rows).  The tabulated-curve form is a
                // separate copy, run only by groups holding a tabulated band, so
                // that the Gaussian / top-hat loop keeps its instruction footprint.
                auto columns = [&](auto tab_tag) {
                    constexpr bool kTab = decltype(tab_tag)::value;
                    constexpr int CG = 8;                  // = the TMEM load width below
                    // group h + 1's TMEM words are loaded while group h is computed
                    uint32_t rn[CG], rc[CG];
                    tc::tmem_ld8_issue(taddr, rn);
                    if (TF) tc::tmem_ld8_issue(taddr + (uint32_t)BN, rc);
#pragma unroll
                    for (int h = 0; h < 32 / CG; ++h) {
                        const int g0 = nb0 + h * CG;
                        tc::tmem_ld8_wait(rn);
                        if (TF) tc::tmem_ld8_wait(rc);
                        float S[CG];
#pragma unroll
                        for (int jj = 0; jj < CG; ++jj)     // + the corrections, FP32 round to nearest
                            S[jj] = TF ? __uint_as_float(rn[jj]) + __uint_as_float(rc[jj]) : __uint_as_float(rn[jj]);
                        if (h + 1 < 32 / CG) {
                            tc::tmem_ld8_issue(taddr + (uint32_t)((h + 1) * CG), rn);
                            if (TF) tc::tmem_ld8_issue(taddr + (uint32_t)(BN + (h + 1) * CG), rc);
                        }
                        uint32_t act = 0;                          // warp-uniform
#pragma unroll
                        for (int k = 0; k < NB; ++k) {
                            if (hlo[k] < g0 + CG && hhi[k] > g0) act |= 1u << k;
                        }
                        if (act == 0u) continue;
                        float s0[CG], sE[CG], sEb[CG], sEd[CG], lm[CG];
#pragma unroll
                        for (int jj = 0; jj < CG; ++jj) {
                            const float4 L4 = cst4[h * CG + jj];
                            lm[jj] = cstl[h * CG + jj];
                            const float ypw = L4.y * exp2f(dl2 * L4.z);      // k0 (l / l_V)^delta
                            const float base = fmaf(eb, L4.w, ypw);
                            const float E = exp2f(cA * base);
                            const float dterm = fmaf(ypw, L4.z, nd19 * L4.w);
                            s0[jj] = S[jj] * L4.x;
                            sE[jj] = s0[jj] * E;
                            sEb[jj] = sE[jj] * base;
                            sEd[jj] = sE[jj] * dterm;
                        }
#pragma unroll
                        for (int k = 0; k < NB; ++k) {
                            if (!((act >> k) & 1u)) continue;
                            const int lo = (int)(sxy[k] & 0xffffu), hi = (int)(sxy[k] >> 16);
                            if constexpr (!KZ && !kTab) {
                                // Gaussian / top-hat band weights of column pairs, packed
                                // FP32x2; a column outside the support adds S x 0
                                float2 p0 = make_float2(0.f, 0.f), p1 = p0, p2 = p0, p3 = p0;
                                // e^{-u^2 / 2} = 2^{-v^2}, v = u sqrt(log2(e) / 2)
                                const float gsv = gs[k] * 0.84932180028801904f;
                                const float2 ngc = make_float2(-gc[k], -gc[k]), gs2 = make_float2(gsv, gsv);
                                const bool gauss = gs[k] != 0.0f;
#pragma unroll
                                for (int jj = 0; jj < CG; jj += 2) {
                                    const int nn = g0 + jj;
                                    const bool i0 = nn >= lo && nn < hi, i1 = nn + 1 >= lo && nn + 1 < hi;
                                    float2 w = make_float2(i0 ? 1.0f : 0.0f, i1 ? 1.0f : 0.0f);
                                    if (gauss) {
                                        const float2 u = __fmul2_rn(__fadd2_rn(make_float2(lm[jj], lm[jj + 1]), ngc), gs2);
                                        const float2 t = __fmul2_rn(u, u);
                                        w = make_float2(i0 ? exp2f(-t.x) : 0.0f, i1 ? exp2f(-t.y) : 0.0f);
                                    }
                                    p0 = __ffma2_rn(make_float2(s0[jj], s0[jj + 1]), w, p0);
                                    p1 = __ffma2_rn(make_float2(sE[jj], sE[jj + 1]), w, p1);
                                    p2 = __ffma2_rn(make_float2(sEb[jj], sEb[jj + 1]), w, p2);
                                    p3 = __ffma2_rn(make_float2(sEd[jj], sEd[jj + 1]), w, p3);
                                }
                                acc[k][0] += p0.x + p0.y;
                                acc[k][1] += p1.x + p1.y;
                                acc[k][2] += p2.x + p2.y;
                                acc[k][3] += p3.x + p3.y;
                                continue;
                            }
                            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, z0 = 0.f, z1 = 0.f;
#pragma unroll
                            for (int jj = 0; jj < CG; ++jj) {
                                const int nn = g0 + jj;
                                if (nn >= lo && nn < hi) {
                                    float w = 1.0f;
                                    float wz = 0.0f;               // KZ: lambda T'
                                    if (kTab && gs[k] < 0.0f) {
                                        const int b = b0 + k;
                                        const float ut = (lm[jj] - gc[k]) * -gs[k];
                                        w = tab_T32(grid.band_T + c.tab_off[b], c.tab_n[b], ut);
                                        if (KZ)     // T' = dT/du / step, 1/step = -gs/(1+z)
                                            wz = lm[jj] * tab_dT32(grid.band_T + c.tab_off[b], c.tab_n[b], ut) *
                                                 (-gs[k] * iopz);
                                    } else if (gs[k] != 0.0f) {
                                        const float u = (lm[jj] - gc[k]) * gs[k];
                                        w = __expf(-0.5f * u * u);
                                        if (KZ) wz = -w * lm[jj] * u * (gs[k] * iopz);   // T' = -u T / s
                                    }
                                    a0 = fmaf(s0[jj], w, a0);
                                    a1 = fmaf(sE[jj], w, a1);
                                    a2 = fmaf(sEb[jj], w, a2);
                                    a3 = fmaf(sEd[jj], w, a3);
                                    if (KZ) {
                                        z0 = fmaf(s0[jj], wz, z0);
                                        z1 = fmaf(sE[jj], wz, z1);
                                    }
                                }
                            }
                            acc[k][0] += a0;
                            acc[k][1] += a1;
                            acc[k][2] += a2;
                            acc[k][3] += a3;
                            if (KZ) {
                                accz[k][0] += z0;
                                accz[k][1] += z1;
                            }
                        }
                    }
                };
                if (has_tab)
                    columns(std::true_type{});
                else
                    columns(std::false_type{});
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&ctl->tempty[buf]);
        }
        // cJ is zeroed before the launch; a (row, band) gets one addend per
        // column half, so the sum does not depend on their order
        if (valid && !ctl->abort) {
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (b0 + k < b_end) {
                    float* o = cJ + (row * B + b0 + k) * 4;
                    atomicAdd(o + 0, acc[k][0]);
                    atomicAdd(o + 1, acc[k][1]);
                    atomicAdd(o + 2, acc[k][2]);
                    atomicAdd(o + 3, acc[k][3]);
                    if (KZ) {
                        float* oz = cJz + (row * B + b0 + k) * 2;
                        atomicAdd(oz + 0, accz[k][0]);
                        atomicAdd(oz + 1, accz[k][1]);
                    }
                }
        }
    }
    tc_teardown<ST>(ctl, warp);
}

// Launch of k_fwd_tc for the band count (epilogue warps: 8 bands per group,
// one group and two column halves, or up to four groups); KZ selects the
// variant that also accumulates the redshift derivative into cJz.
template <bool KZ>
cudaError_t fwd_tc_launch(const TcMaps& tm, bool tf, const Consts& c, const Grid& grid, const Galaxies& g,
                          const float* theta, const int32_t* gal_idx, const int32_t* perm, int64_t n, float* cJ,
                          int* err, cudaStream_t s, float* cJz) {
    if (n <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + kTM - 1) / kTM);
    const size_t smem = tc_fwd_smem(tf);
    const int groups = (c.n_band + kFwdGroupBands - 1) / kFwdGroupBands;   // <= 4 (B <= 32)
    const int halves = groups == 1 ? 2 : 1;
    const int threads = 64 + 32 * 4 * groups * halves;
    cudaError_t e = cudaMemsetAsync(cJ, 0, (size_t)n * c.n_band * 4 * sizeof(float), s);
    if (e != cudaSuccess) return e;
    if (cJz) {
        e = cudaMemsetAsync(cJz, 0, (size_t)n * c.n_band * 2 * sizeof(float), s);
        if (e != cudaSuccess) return e;
    }
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r != cudaSuccess) return r;
        kern<<<blocks, threads, smem, s>>>(tm, c, grid, g, theta, gal_idx, perm, n, halves, cJ, err, cJz);
        return cudaSuccess;
    };
    constexpr int T8 = 64 + 32 * 8, T12 = 64 + 32 * 12, T16 = 64 + 32 * kFwdMaxEpiWarps;
    if (threads <= T8) e = tf ? go(k_fwd_tc<T8, true, KZ>) : go(k_fwd_tc<T8, false, KZ>);         // <= 16 bands
    else if (threads <= T12) e = tf ? go(k_fwd_tc<T12, true, KZ>) : go(k_fwd_tc<T12, false, KZ>); // <= 24 bands
    else e = tf ? go(k_fwd_tc<T16, true, KZ>) : go(k_fwd_tc<T16, false, KZ>);                     // <= 32 bands
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

}  // namespace sps
