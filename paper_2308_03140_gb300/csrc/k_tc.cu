// 5th-generation tensor-core GEMM (tcgen05, sm_103a) for the mixed-precision
// Newton-Schulz iteration behind Eqs. (diagonalization), (mbd-energy):
//
//   C = alpha * sum_p A_p B_p^T + beta * D      (FP32 accumulate in tensor memory)
//
// with K-major operands (rows of A and of B run along K).  Three operand kinds:
//   TF32   one product, operands stored as FP32 (kind::tf32 uses their top 19 bits);
//   BF16x3 three products A_hi B_hi + A_hi B_lo + A_lo B_hi, operands stored as bf16
//          hi/lo pairs (X = X_hi + X_lo), about 16 significant bits per product;
//   TF32x3 the same three products with TF32 hi and TF32-rounded remainder parts.
// Three forms of the kernel share the operand staging, the chunked accumulation and the
// epilogue: the wide form (the default: 128 x 256 tiles, 12 warps per CTA, its work items
// read from a host-computed table; "wide form" below), the 128 x 128 form described in this
// paragraph, and the CTA-pair form (256 x 128 tiles on two CTAs, cta_group::2; "CTA-pair
// form" below); tc_gemm picks one by MBDGB_TC_FORM.
// Each is persistent: one CTA (6 warps in the 128 x 128 form) per SM loops over output tiles
// (and the items of a batched product), its stage and chunk counters running on across tiles
// so that the next tile's loads and MMAs overlap the last tile's epilogue.  Operand tiles of
// 128 rows x 128 bytes are staged in shared memory by TMA (128-byte swizzle) through an
// mbarrier ring;
// warp 4 issues the TMA loads, warp 5 issues tcgen05.mma.  K is split into chunks of
// `chunk_stages` stages, each accumulated afresh in one of kBufs 128-column TMEM buffers;
// warps 0-3 (one tile row per thread) read each finished chunk back (tcgen05.ld 32x32b)
// and add it to FP32 registers with round-to-nearest while the next chunk accumulates.
// The tensor core's own accumulation truncates: its bias grows with the number of terms
// per accumulator, and in the Newton-Schulz iteration it breaks the coupling Y = Y0 Z.
// Epilogue: alpha/beta, FP32 and/or split outputs, optional transposed copies, mirrored
// writes of upper tiles (symmetric products), optional FP64 accumulation output and
// optional sum of (I - C)^2.
//
// Every wait is bounded (clock64 budget); on a timeout the kernel raises the error
// flag, stops issuing work, waits (bounded) for its own TMA copies and MMAs, frees its
// tensor memory and returns.
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "internal.h"
#include "tc_ops.cuh"
#include "tc_tiles.cuh"

namespace mbdgb {
namespace {

using namespace tcops;

constexpr int TM = 128, TN = 128;
constexpr int KB = 128;                         // bytes of K per stage per row (one swizzle atom)
constexpr int TILE_BYTES = TM * KB;             // 16 KB
// Tensor-memory accumulation buffers of TN columns each (all 512 columns of the SM): chunk c
// accumulates in buffer c % kBufs, so the MMAs run up to kBufs - 1 chunks ahead of the
// epilogue warps that drain them.
constexpr int kBufs = 4;

// Instruction descriptor: FP32 accumulator, A/B format fmt (1 = bf16, 2 = tf32), both
// K-major, N = TN, M = TM.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(TN >> 3) << 17) |
           (static_cast<uint32_t>(TM >> 4) << 24);
}
template <bool TF32>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    if (TF32)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(a), "l"(b), "r"(idesc(2)), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(a), "l"(b), "r"(idesc(1)), "r"(acc));
}
// Element j of a packed split row (bf16 pairs for KIND 1, 32-bit words for KIND 2).
template <int KIND>
__device__ __forceinline__ void store_part(void *base, long long off, const uint32_t *w, int j) {
    if (KIND == 2)
        static_cast<uint32_t *>(base)[off] = w[j];
    else
        static_cast<unsigned short *>(base)[off] = static_cast<unsigned short>(w[j >> 1] >> (16 * (j & 1)));
}

// Batch item and tile of work item w (items ordered batch item by batch item; tiles in the
// grouped order of tc_tiles.cuh, so that the CTAs resident at one time share operand panels in
// L2).
__device__ __forceinline__ void item_tile(int w, int tiles, int mode, int tiles_m, int tiles_n, int &bz, int &tm,
                                          int &tn) {
    bz = w / tiles;
    tctiles::grouped_tile(w - bz * tiles, mode, tiles_m, tiles_n, tm, tn);
}

template <int KIND>   // 0: TF32 single product; 1: BF16x3; 2: TF32x3
struct TcCfg {
    static constexpr int PAIRS = KIND == 0 ? 1 : 3;
    static constexpr int TILES = KIND == 0 ? 2 : 4;
    static constexpr int STAGES = KIND == 0 ? 4 : 3;
    static constexpr int STAGE_BYTES = TILES * TILE_BYTES;
    static constexpr int ELEM = KIND == 1 ? 2 : 4;
    static constexpr bool TF32 = KIND != 1;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 512;
};

// Epilogue of one 128 x 128 tile for the thread owning row m: alpha/beta with D, the
// optional outputs (FP32, split parts, FP64 accumulation, transposes, mirrored writes of the
// symmetric products) and the residual sum.  Warp-uniform: every lane of a warp handles a row
// of the same tile.
template <int KIND>
__device__ __forceinline__ void tile_epilogue(const TcArgs &g, const float (&acc)[TN], long long m, int tm, int tn,
                                              const float *Dp, float *Cp, int lane) {
    using Cfg = TcCfg<KIND>;
    const bool mirror = (g.mode == 2) && (tm != tn);
    const bool diag = (g.mode == 2) && (tm == tn);
    double rs = 0.0;
#pragma unroll
    for (int c0 = 0; c0 < TN; c0 += 16) {
        const long long n0 = static_cast<long long>(tn) * TN + c0;
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = g.alpha * acc[c0 + j];
        if (g.beta != 0.f) {   // this row of D was prefetched into L2 during the last chunks
            const float4 *dp = reinterpret_cast<const float4 *>(Dp + m * g.ld + n0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 d = dp[q];
                v[4 * q] += g.beta * d.x;
                v[4 * q + 1] += g.beta * d.y;
                v[4 * q + 2] += g.beta * d.z;
                v[4 * q + 3] += g.beta * d.w;
            }
        }
        if (g.resid && m < g.nvalid) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (n0 + j < g.nvalid) {
                    const double e = (m == n0 + j ? 1.0 : 0.0) - static_cast<double>(v[j]);
                    rs += e * e;
                }
        }
        if (g.C64) {   // FP64 accumulation output (caller splits K: C64 += result)
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if (diag && n0 + j < m) continue;
                g.C64[m * g.ld + n0 + j] += static_cast<double>(v[j]);
                if ((mirror || diag) && n0 + j != m) g.C64[(n0 + j) * g.ld + m] += static_cast<double>(v[j]);
            }
        }
        // split of the result into the next product's operand parts: bf16 pairs
        // packed two per word (BF16x3), or TF32 hi and TF32 remainder (TF32x3),
        // each rounded to nearest
        uint32_t hw[KIND == 2 ? 16 : 8], lw[KIND == 2 ? 16 : 8];
        if (g.Ch || g.CTh) {
            if (KIND == 2) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    uint32_t h, l;
                    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(v[j]));
                    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(l) : "f"(v[j] - __uint_as_float(h)));
                    hw[j] = h;
                    lw[j] = l;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * q]), h1 = __float2bfloat16_rn(v[2 * q + 1]);
                    const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * q] - __bfloat162float(h0));
                    const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * q + 1] - __bfloat162float(h1));
                    hw[q] = static_cast<uint32_t>(__bfloat16_as_ushort(h0)) |
                            (static_cast<uint32_t>(__bfloat16_as_ushort(h1)) << 16);
                    lw[q] = static_cast<uint32_t>(__bfloat16_as_ushort(l0)) |
                            (static_cast<uint32_t>(__bfloat16_as_ushort(l1)) << 16);
                }
            }
        }
        // Symmetric products (mode 2): upper tiles are mirrored into the lower half;
        // diagonal tiles keep their upper triangle and mirror it, so the result is
        // exactly symmetric whatever order the tensor cores summed in.
        if (!diag) {
            if (Cp) {
                float4 *cp = reinterpret_cast<float4 *>(Cp + m * g.ld + n0);
#pragma unroll
                for (int q = 0; q < 4; ++q) cp[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
            if (g.Ch) {
                constexpr int NV = KIND == 2 ? 4 : 2;   // uint4 vectors per 16 elements
                uint4 *hp = reinterpret_cast<uint4 *>(static_cast<char *>(g.Ch) + (m * g.ld + n0) * Cfg::ELEM);
                uint4 *lp = reinterpret_cast<uint4 *>(static_cast<char *>(g.Cl) + (m * g.ld + n0) * Cfg::ELEM);
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    hp[q] = make_uint4(hw[4 * q], hw[4 * q + 1], hw[4 * q + 2], hw[4 * q + 3]);
                    lp[q] = make_uint4(lw[4 * q], lw[4 * q + 1], lw[4 * q + 2], lw[4 * q + 3]);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if (n0 + j < m) continue;
                const long long off = m * g.ld + n0 + j;
                if (Cp) Cp[off] = v[j];
                if (g.Ch) {
                    store_part<KIND>(g.Ch, off, hw, j);
                    store_part<KIND>(g.Cl, off, lw, j);
                }
            }
        }
        // transposed copies (coalesced across the warp: consecutive rows m).  For a
        // mirrored tile of a symmetric product the transpose goes into C itself.
        const bool into_c = mirror || diag;
        float *Tf = into_c ? Cp : g.CT;
        void *Th = into_c ? g.Ch : g.CTh, *Tl = into_c ? g.Cl : g.CTl;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (diag && n0 + j <= m) continue;
            const long long off = (n0 + j) * g.ld + m;
            if (Tf) Tf[off] = v[j];
            if (Th) {
                store_part<KIND>(Th, off, hw, j);
                store_part<KIND>(Tl, off, lw, j);
            }
        }
    }
    if (g.resid) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
        if (lane == 0 && rs != 0.0) atomicAdd(g.resid, rs);
    }
}

template <int KIND>
__global__ void __launch_bounds__(192, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
              const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1, TcArgs g,
              int tiles_n) {
    using Cfg = TcCfg<KIND>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + Cfg::STAGES * Cfg::STAGE_BYTES);
    uint64_t *empty = full + Cfg::STAGES;
    uint64_t *cfull = empty + Cfg::STAGES;   // [kBufs] accumulator buffer holds a finished chunk
    uint64_t *cfree = cfull + kBufs;         // [kBufs] epilogue has drained the buffer
    uint64_t *done = cfree + kBufs;          // every MMA issued has completed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    // Persistent CTAs: work item w = (batch item, tile) runs over blockIdx.x, blockIdx.x +
    // gridDim.x, ...; stage and chunk counters run on across items, so the producer and the
    // MMA issuer start the next tile while the epilogue warps store the last one.
    const int tiles_m = g.M / TM;
    const int tiles = tctiles::tile_count(g.mode, tiles_m, tiles_n);
    const int items = tiles * g.batch;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < kBufs; ++b) {
            mbar_init(&cfull[b], 1);
            mbar_init(&cfree[b], 4);   // one arrival per epilogue warp
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                     "r"(kBufs * TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nk = static_cast<int>((static_cast<long long>(g.K) * Cfg::ELEM) / KB);
    const int cs = (g.chunk_stages > 0 && g.chunk_stages < nk) ? g.chunk_stages : nk;   // stages per chunk
    const int nchunks = (nk + cs - 1) / cs;
    constexpr int KELEM = KB / Cfg::ELEM;   // elements of K per stage

    if (warp == 4) {
        // ---- TMA producer (one thread) ----
        if (lane == 0) {
            int issued = 0, kg = 0;   // kg: stages issued by this CTA so far
            for (int w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
                int bz, tm, tn;
                item_tile(w, tiles, g.mode, tiles_m, tiles_n, bz, tm, tn);
                const int ya = bz * g.M + tm * TM, yb = bz * g.N + tn * TN;
                for (int kt = 0; kt < nk && !*abort_flag; ++kt, ++kg) {
                    const int s = kg % Cfg::STAGES;
                    const uint32_t ph = (kg / Cfg::STAGES) & 1;
                    if (kg >= Cfg::STAGES && !mbar_wait(&empty[s], ph ^ 1, g.err)) {
                        *abort_flag = 1;
                        break;
                    }
                    uint8_t *st = smem + s * Cfg::STAGE_BYTES;
                    mbar_expect_tx(&full[s], Cfg::STAGE_BYTES);
                    const int kx = kt * KELEM;
                    tma_load_2d(st, &mA0, kx, ya, &full[s]);
                    tma_load_2d(st + TILE_BYTES, &mB0, kx, yb, &full[s]);
                    if (Cfg::TILES == 4) {
                        tma_load_2d(st + 2 * TILE_BYTES, &mA1, kx, ya, &full[s]);
                        tma_load_2d(st + 3 * TILE_BYTES, &mB1, kx, yb, &full[s]);
                    }
                    issued = kg + 1;
                }
            }
            if (*abort_flag) {   // let this CTA's copies land before shared memory is released
                for (int k = (issued > Cfg::STAGES ? issued - Cfg::STAGES : 0); k < issued; ++k)
                    mbar_wait(&full[k % Cfg::STAGES], (k / Cfg::STAGES) & 1, g.err);
            }
        }
    } else if (warp == 5) {
        // ---- MMA issuer (one thread): chunk c accumulates afresh into buffer c % kBufs ----
        if (lane == 0) {
            int kg = 0, cg = 0;   // stages consumed and chunks begun by this CTA before the current item
            for (int w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x, cg += nchunks) {
                for (int kt = 0; kt < nk && !*abort_flag; ++kt, ++kg) {
                    const int c = cg + kt / cs, buf = c % kBufs;
                    if (kt % cs == 0 && c >= kBufs && !mbar_wait(&cfree[buf], ((c / kBufs) - 1) & 1, g.err)) {
                        *abort_flag = 1;
                        break;
                    }
                    const int s = kg % Cfg::STAGES;
                    if (!mbar_wait(&full[s], (kg / Cfg::STAGES) & 1, g.err)) {
                        *abort_flag = 1;
                        break;
                    }
                    fence_after();
                    const uint32_t base = su32(smem + s * Cfg::STAGE_BYTES);
                    const uint32_t dt = tmem + static_cast<uint32_t>(buf * TN);
#pragma unroll
                    for (int k = 0; k < KB / 32; ++k) {   // 32 bytes of K per instruction
                        const uint64_t a0 = sdesc(base + k * 32), b0 = sdesc(base + TILE_BYTES + k * 32);
                        mma<Cfg::TF32>(dt, a0, b0, (kt % cs != 0 || k != 0) ? 1u : 0u);
                        if (Cfg::PAIRS == 3) {
                            const uint64_t a1 = sdesc(base + 2 * TILE_BYTES + k * 32);
                            const uint64_t b1 = sdesc(base + 3 * TILE_BYTES + k * 32);
                            mma<Cfg::TF32>(dt, a0, b1, 1u);
                            mma<Cfg::TF32>(dt, a1, b0, 1u);
                        }
                    }
                    mma_commit(&empty[s]);                              // stage free once read
                    if (kt % cs == cs - 1 || kt == nk - 1) mma_commit(&cfull[buf]);   // chunk finished
                }
            }
            mma_commit(done);
        }
    } else {
        // ---- epilogue warps 0-3: thread = row of the tile; chunk sums added in FP32 with
        // round-to-nearest (the tensor core's own accumulation truncates) ----
        bool ok = true;
        int cg = 0;   // chunks of earlier items
        for (int w = blockIdx.x; w < items && ok; w += gridDim.x, cg += nchunks) {
            int bz, tm, tn;
            item_tile(w, tiles, g.mode, tiles_m, tiles_n, bz, tm, tn);
            const float *Dp = g.D ? g.D + bz * g.sC : nullptr;
            float *Cp = g.C ? g.C + bz * g.sC : nullptr;
            float acc[TN];
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[j] = 0.f;
            const int row = warp * 32 + lane;
            const long long m = static_cast<long long>(tm) * TM + row;
            for (int c = 0; c < nchunks; ++c) {
                const int buf = (cg + c) % kBufs;
                if (c == max(0, nchunks - 2) && g.beta != 0.f) {   // this row of D into L2 ahead of the epilogue
                    const float *drow = Dp + m * g.ld + static_cast<long long>(tn) * TN;
#pragma unroll
                    for (int q = 0; q < TN / 32; ++q) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(drow + 32 * q));
                }
                ok = mbar_wait(&cfull[buf], ((cg + c) / kBufs) & 1, g.err) && !*abort_flag;
                ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t tb = tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(buf * TN);
#pragma unroll
                for (int q = 0; q < TN / 32; ++q) {
                    uint32_t r[32];
                    tmem_ld32(tb + q * 32, r);
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc[q * 32 + j] += __uint_as_float(r[j]);
                }
                fence_before();
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(&cfree[buf])) : "memory");
            }
            if (ok) tile_epilogue<KIND>(g, acc, m, tm, tn, Dp, Cp, lane);
        }   // work items
    }
    __syncwarp();
    fence_before();
    __syncthreads();
    if (warp == 0) {
        // every MMA this CTA issued must have completed before its tensor memory is freed
        if (lane == 0) mbar_wait(done, 0, g.err);
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kBufs * TN));
    }
}

// ---- wide form: 128 x 256 tiles -------------------------------------------------------------
// One CTA per SM computes 128 x 256 tiles (tile row tm, tile columns 2 TPn and 2 TPn + 1;
// tc_tiles.cuh): each K stage holds 128 rows of A and 256 of B (96 KB for the split kinds, two
// stages), and one tcgen05.mma with N = 256 does the work of two 128 x 128 ones, so every
// barrier handshake and TMA box of the ring feeds twice the MMA work.  Each chunk accumulates
// in one of two 256-column TMEM buffers; eight epilogue warps drain them, warp w taking the
// TMEM lane quarter w % 4 and the column half w / 4 (128 sums per thread), and store each half
// as a 128 x 128 tile.  Warp 8 issues the TMA loads, warp 9 the MMAs; warps 10 and 11 complete
// the third warpgroup.  Registers: the launch gives 168 per thread (384 x 168 = 64512, three
// warps on each SM sub-partition); the epilogue warpgroups raise theirs to EPI_REGS and the
// third lowers its to 504 - 2 EPI_REGS, so the sum stays the launch's.
constexpr int TNW = 256;
constexpr int kWideBufs = 2;
#ifndef EPI_REGS_OVERRIDE
constexpr int EPI_REGS = 240;
#else
constexpr int EPI_REGS = EPI_REGS_OVERRIDE;
#endif
static_assert(EPI_REGS % 8 == 0 && 2 * EPI_REGS + (504 - 2 * EPI_REGS) == 504 && 504 - 2 * EPI_REGS >= 24,
              "register shares of the wide GEMM must add up to the launch's 168 per thread");
template <int KIND>
struct TcCfgW {
    static constexpr int PAIRS = KIND == 0 ? 1 : 3;
    static constexpr int B_BYTES = TNW * KB;   // 32 KB
    static constexpr int OFF_B0 = TILE_BYTES, OFF_A1 = TILE_BYTES + B_BYTES, OFF_B1 = 2 * TILE_BYTES + B_BYTES;
    static constexpr int STAGE_BYTES = (KIND == 0 ? 1 : 2) * (TILE_BYTES + B_BYTES);
    static constexpr int STAGES = KIND == 0 ? 4 : 2;
    static constexpr int ELEM = KIND == 1 ? 2 : 4;
    static constexpr bool TF32 = KIND != 1;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 512;
};
__host__ __device__ constexpr uint32_t idescw(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(TNW >> 3) << 17) |
           (static_cast<uint32_t>(TM >> 4) << 24);
}
template <bool TF32>
__device__ __forceinline__ void mmaw(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    if (TF32)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(a), "l"(b), "r"(idescw(2)), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(a), "l"(b), "r"(idescw(1)), "r"(acc));
}

template <int KIND>
__global__ void __launch_bounds__(384, 1)
    k_tc_gemm_w(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1, TcArgs g,
                int tiles_n, const int2 *tile_of) {
    using Cfg = TcCfgW<KIND>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + Cfg::STAGES * Cfg::STAGE_BYTES);
    uint64_t *empty = full + Cfg::STAGES;
    uint64_t *cfull = empty + Cfg::STAGES;
    uint64_t *cfree = cfull + kWideBufs;
    uint64_t *done = cfree + kWideBufs;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tiles_m = g.M / TM;
    const int wtiles = tctiles::wide_tile_count(g.mode, tiles_m, tiles_n);
    const int items = wtiles * g.batch;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < kWideBufs; ++b) {
            mbar_init(&cfull[b], 1);
            mbar_init(&cfree[b], 8);   // one arrival per epilogue warp
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                     "r"(kWideBufs * TNW));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nk = static_cast<int>((static_cast<long long>(g.K) * Cfg::ELEM) / KB);
    const int cs = (g.chunk_stages > 0 && g.chunk_stages < nk) ? g.chunk_stages : nk;
    const int nchunks = (nk + cs - 1) / cs;
    constexpr int KELEM = KB / Cfg::ELEM;

    if (warp >= 8) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(504 - 2 * EPI_REGS));
        if (warp == 8 && lane == 0) {
            // ---- TMA producer ----
            int issued = 0, kg = 0;
            for (int w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
                const int bz = w / wtiles;
                int tm, TPn;
                {
                    const int2 c = tile_of[w - bz * wtiles];   // (tm, TPn) of the item, tabulated on the host
                    tm = c.x;
                    TPn = c.y;
                }
                const int ya = bz * g.M + tm * TM, yb = bz * g.N + TPn * TNW;
                for (int kt = 0; kt < nk && !*abort_flag; ++kt, ++kg) {
                    const int s = kg % Cfg::STAGES;
                    const uint32_t ph = (kg / Cfg::STAGES) & 1;
                    if (kg >= Cfg::STAGES && !mbar_wait(&empty[s], ph ^ 1, g.err)) {
                        *abort_flag = 1;
                        break;
                    }
                    uint8_t *st = smem + s * Cfg::STAGE_BYTES;
                    mbar_expect_tx(&full[s], Cfg::STAGE_BYTES);
                    const int kx = kt * KELEM;
                    tma_load_2d(st, &mA0, kx, ya, &full[s]);
                    tma_load_2d(st + Cfg::OFF_B0, &mB0, kx, yb, &full[s]);
                    if (KIND != 0) {
                        tma_load_2d(st + Cfg::OFF_A1, &mA1, kx, ya, &full[s]);
                        tma_load_2d(st + Cfg::OFF_B1, &mB1, kx, yb, &full[s]);
                    }
                    issued = kg + 1;
                }
            }
            if (*abort_flag) {   // let this CTA's copies land before shared memory is released
                for (int k = (issued > Cfg::STAGES ? issued - Cfg::STAGES : 0); k < issued; ++k)
                    mbar_wait(&full[k % Cfg::STAGES], (k / Cfg::STAGES) & 1, g.err);
            }
        } else if (warp == 9 && lane == 0) {
            // ---- MMA issuer: chunk c accumulates afresh into buffer c % kWideBufs ----
            int kg = 0, cg = 0;
            for (int w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x, cg += nchunks) {
                for (int kt = 0; kt < nk && !*abort_flag; ++kt, ++kg) {
                    const int c = cg + kt / cs, buf = c % kWideBufs;
                    if (kt % cs == 0 && c >= kWideBufs &&
                        !mbar_wait(&cfree[buf], ((c / kWideBufs) - 1) & 1, g.err)) {
                        *abort_flag = 1;
                        break;
                    }
                    const int s = kg % Cfg::STAGES;
                    if (!mbar_wait(&full[s], (kg / Cfg::STAGES) & 1, g.err)) {
                        *abort_flag = 1;
                        break;
                    }
                    fence_after();
                    const uint32_t base = su32(smem + s * Cfg::STAGE_BYTES);
                    const uint32_t dt = tmem + static_cast<uint32_t>(buf * TNW);
#pragma unroll
                    for (int k = 0; k < KB / 32; ++k) {
                        const uint64_t a0 = sdesc(base + k * 32), b0 = sdesc(base + Cfg::OFF_B0 + k * 32);
                        mmaw<Cfg::TF32>(dt, a0, b0, (kt % cs != 0 || k != 0) ? 1u : 0u);
                        if (Cfg::PAIRS == 3) {
                            const uint64_t a1 = sdesc(base + Cfg::OFF_A1 + k * 32);
                            const uint64_t b1 = sdesc(base + Cfg::OFF_B1 + k * 32);
                            mmaw<Cfg::TF32>(dt, a0, b1, 1u);
                            mmaw<Cfg::TF32>(dt, a1, b0, 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                    if (kt % cs == cs - 1 || kt == nk - 1) mma_commit(&cfull[buf]);
                }
            }
            mma_commit(done);
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(EPI_REGS));
        // ---- epilogue warps 0-7: lane quarter q, column half h; thread = row of the tile ----
        const int q = warp & 3, h = warp >> 2;
        bool ok = true;
        int cg = 0;
        for (int w = blockIdx.x; w < items && ok; w += gridDim.x, cg += nchunks) {
            const int bz = w / wtiles;
            int tm, TPn;
            {
                    const int2 c = tile_of[w - bz * wtiles];   // (tm, TPn) of the item, tabulated on the host
                    tm = c.x;
                    TPn = c.y;
                }
            const int tn = 2 * TPn + h;
            const bool write = tctiles::wide_half_valid(g.mode, tiles_n, tm, TPn, h);
            const float *Dp = g.D ? g.D + bz * g.sC : nullptr;
            float *Cp = g.C ? g.C + bz * g.sC : nullptr;
            float acc[TN];
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[j] = 0.f;
            const int row = q * 32 + lane;
            const long long m = static_cast<long long>(tm) * TM + row;
            for (int c = 0; c < nchunks; ++c) {
                const int buf = (cg + c) % kWideBufs;
                if (write && c == max(0, nchunks - 2) && g.beta != 0.f) {
                    const float *drow = Dp + m * g.ld + static_cast<long long>(tn) * TN;
#pragma unroll
                    for (int qq = 0; qq < TN / 32; ++qq) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(drow + 32 * qq));
                }
                ok = mbar_wait(&cfull[buf], ((cg + c) / kWideBufs) & 1, g.err) && !*abort_flag;
                ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t tb = tmem + (static_cast<uint32_t>(q * 32) << 16) +
                                    static_cast<uint32_t>(buf * TNW + h * TN);
#pragma unroll
                for (int qq = 0; qq < TN / 32; ++qq) {
                    uint32_t r[32];
                    tmem_ld32(tb + qq * 32, r);
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc[qq * 32 + j] += __uint_as_float(r[j]);
                }
                fence_before();
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(&cfree[buf])) : "memory");
            }
            if (ok && write) tile_epilogue<KIND>(g, acc, m, tm, tn, Dp, Cp, lane);
        }
    }
    __syncwarp();
    fence_before();
    __syncthreads();
    if (warp == 0) {
        if (lane == 0) mbar_wait(done, 0, g.err);
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kWideBufs * TNW));
    }
}

// ---- CTA-pair form (tcgen05 cta_group::2) ----------------------------------------------
// A cluster of two CTAs computes a pair tile of 256 x 128 (tile rows 2 TP and 2 TP + 1 of
// tile column tn, tc_tiles.cuh): CTA r stages A rows [256 TP + 128 r, +128) and B rows
// [128 tn + 64 r, +64) of every K stage in its own shared memory (TMA, 128-byte swizzle); the
// even CTA issues tcgen05.mma.cta_group::2 with M = 256, N = 128, which takes the A halves and
// the B halves of both CTAs and accumulates rows 128 r .. 128 r + 127 of the pair tile in
// CTA r's tensor memory.  A CTA then stages 48 KB of operands per K stage (split kinds) for
// the MMA work that 64 KB feeds in the single-CTA form, and four stages fit where three do.
// Barriers in each CTA's shared memory:
//   full[s]   (even CTA) the bytes of stage s of both CTAs landed: the even CTA's producer
//             expects both CTAs' bytes, and the odd CTA's loads count their bytes on the even
//             CTA's barrier (cta_group::2 form of the TMA load);
//   empty[s]  the MMAs reading stage s completed (the even CTA commits to both CTAs);
//   cfull[b]  a chunk finished in tensor-memory buffer b (committed to both);
//   cfree[b]  (even CTA) the eight epilogue warps of the pair drained buffer b;
//   done      every MMA issued completed (committed to both).
// Every wait is bounded as in the single-CTA form; on a timeout the CTA raises the error
// flag and stops, and its peer's waits run out in turn.  Both CTAs leave through a cluster
// barrier, so neither exits while the other can still signal its shared memory.
template <int KIND>
struct TcCfg2 {
    static constexpr int PAIRS = KIND == 0 ? 1 : 3;
    static constexpr int B_BYTES = TILE_BYTES / 2;   // 64 rows x 128 bytes
    static constexpr int OFF_B0 = TILE_BYTES, OFF_A1 = TILE_BYTES + B_BYTES, OFF_B1 = 2 * TILE_BYTES + B_BYTES;
    static constexpr int STAGE_BYTES = (KIND == 0 ? 1 : 2) * (TILE_BYTES + B_BYTES);
    static constexpr int STAGES = KIND == 0 ? 8 : 4;
    static constexpr int ELEM = KIND == 1 ? 2 : 4;
    static constexpr bool TF32 = KIND != 1;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 512;
};

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
// Address in the shared::cluster window of the same shared-memory object in CTA `rank`.
__device__ __forceinline__ uint32_t peer_addr(uint32_t local, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(a) : "r"(local), "r"(rank));
    return a;
}
__device__ __forceinline__ void remote_arrive(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];\n" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_cl(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait (cluster-scope acquire: arrivals may come from the peer CTA).
__device__ __forceinline__ bool mbar_wait_cl(uint64_t *b, uint32_t parity, int *err) {
    const long long t0 = clock64();
    while (!mbar_try_cl(b, parity)) {
        if (clock64() - t0 > kSpinCycles) {
            atomicOr(err, ST_TC_TIMEOUT);
            return false;
        }
    }
    return true;
}
// TMA load into this CTA's shared memory whose completion is counted on an mbarrier of either
// CTA of the pair (shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            su32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// Instruction descriptor of the pair MMA: M = 256 (two CTAs), N = TN.
__host__ __device__ constexpr uint32_t idesc2(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(TN >> 3) << 17) | (static_cast<uint32_t>(256 >> 4) << 24);
}
template <bool TF32>
__device__ __forceinline__ void mma2(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    if (TF32)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(a), "l"(b), "r"(idesc2(2)), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(a), "l"(b), "r"(idesc2(1)), "r"(acc));
}
// Arrival on an mbarrier (own or peer, shared::cluster address) once every prior MMA of this
// thread has completed.
__device__ __forceinline__ void commit2(uint32_t cluster_addr) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(cluster_addr)
                 : "memory");
}

template <int KIND>
__global__ void __launch_bounds__(192, 1)
    k_tc_gemm2(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
               const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1, TcArgs g,
               int tiles_n) {
    using Cfg = TcCfg2<KIND>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + Cfg::STAGES * Cfg::STAGE_BYTES);
    uint64_t *empty = full + Cfg::STAGES;
    uint64_t *cfull = empty + Cfg::STAGES;
    uint64_t *cfree = cfull + kBufs;
    uint64_t *done = cfree + kBufs;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const uint32_t rank = cluster_rank();
    const bool lead = rank == 0;
    const int cl = static_cast<int>(blockIdx.x >> 1), ncl = static_cast<int>(gridDim.x >> 1);
    const int tiles_m = g.M / TM;
    const int ptiles = tctiles::pair_tile_count(g.mode, tiles_m, tiles_n);
    const int items = ptiles * g.batch;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < kBufs; ++b) {
            mbar_init(&cfull[b], 1);
            mbar_init(&cfree[b], 8);   // four epilogue warps in each CTA of the pair
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 0) {   // both CTAs of the pair allocate, at the same tensor-memory address
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                     "r"(kBufs * TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;\n");
    }
    fence_before();
    __syncthreads();
    cluster_sync();   // both CTAs' barriers exist before either signals the other
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nk = static_cast<int>((static_cast<long long>(g.K) * Cfg::ELEM) / KB);
    const int cs = (g.chunk_stages > 0 && g.chunk_stages < nk) ? g.chunk_stages : nk;
    const int nchunks = (nk + cs - 1) / cs;
    constexpr int KELEM = KB / Cfg::ELEM;

    if (warp == 4) {
        // ---- TMA producer of this CTA's halves (one thread); every stage's bytes are counted on
        // the even CTA's full[s] ----
        if (lane == 0) {
            int issued = 0, kg = 0;
            const uint32_t full_pair = peer_addr(su32(&full[0]), 0);
            for (int w = cl; w < items && !*abort_flag; w += ncl) {
                const int bz = w / ptiles;
                int TP, tn;
                tctiles::pair_tile(w - bz * ptiles, g.mode, tiles_m, tiles_n, TP, tn);
                const int ya = bz * g.M + (2 * TP + static_cast<int>(rank)) * TM;
                const int yb = bz * g.N + tn * TN + static_cast<int>(rank) * (TN / 2);
                for (int kt = 0; kt < nk && !*abort_flag; ++kt, ++kg) {
                    const int s = kg % Cfg::STAGES;
                    const uint32_t ph = (kg / Cfg::STAGES) & 1;
                    if (kg >= Cfg::STAGES && !mbar_wait_cl(&empty[s], ph ^ 1, g.err)) {
                        *abort_flag = 1;
                        break;
                    }
                    uint8_t *st = smem + s * Cfg::STAGE_BYTES;
                    if (lead) mbar_expect_tx(&full[s], 2 * Cfg::STAGE_BYTES);   // both CTAs' bytes
                    const uint32_t fb = full_pair + static_cast<uint32_t>(s) * 8u;
                    const int kx = kt * KELEM;
                    tma_load_2d_pair(st, &mA0, kx, ya, fb);
                    tma_load_2d_pair(st + Cfg::OFF_B0, &mB0, kx, yb, fb);
                    if (KIND != 0) {
                        tma_load_2d_pair(st + Cfg::OFF_A1, &mA1, kx, ya, fb);
                        tma_load_2d_pair(st + Cfg::OFF_B1, &mB1, kx, yb, fb);
                    }
                    issued = kg + 1;
                }
            }
            if (*abort_flag) {
                // let the copies land before shared memory is released: the even CTA waits for
                // the stages it expected (they count both CTAs' bytes); the odd CTA, which cannot
                // observe the even CTA's barriers, gives its last copies a bounded time to land
                if (lead) {
                    for (int k = (issued > Cfg::STAGES ? issued - Cfg::STAGES : 0); k < issued; ++k)
                        mbar_wait(&full[k % Cfg::STAGES], (k / Cfg::STAGES) & 1, g.err, kSpinCycles / 8);
                } else {
                    const long long t0 = clock64();
                    while (clock64() - t0 < 2000000LL) {
                    }
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0 && lead) {
            // ---- MMA issuer of the pair (even CTA) ----
            const uint32_t peer = 1;
            int kg = 0, cg = 0;
            for (int w = cl; w < items && !*abort_flag; w += ncl, cg += nchunks) {
                for (int kt = 0; kt < nk && !*abort_flag; ++kt, ++kg) {
                    const int c = cg + kt / cs, buf = c % kBufs;
                    if (kt % cs == 0 && c >= kBufs && !mbar_wait_cl(&cfree[buf], ((c / kBufs) - 1) & 1, g.err)) {
                        *abort_flag = 1;
                        break;
                    }
                    const int s = kg % Cfg::STAGES;
                    if (!mbar_wait_cl(&full[s], (kg / Cfg::STAGES) & 1, g.err)) {
                        *abort_flag = 1;
                        break;
                    }
                    fence_after();
                    const uint32_t base = su32(smem + s * Cfg::STAGE_BYTES);
                    const uint32_t dt = tmem + static_cast<uint32_t>(buf * TN);
#pragma unroll
                    for (int k = 0; k < KB / 32; ++k) {
                        const uint64_t a0 = sdesc(base + k * 32), b0 = sdesc(base + Cfg::OFF_B0 + k * 32);
                        mma2<Cfg::TF32>(dt, a0, b0, (kt % cs != 0 || k != 0) ? 1u : 0u);
                        if (Cfg::PAIRS == 3) {
                            const uint64_t a1 = sdesc(base + Cfg::OFF_A1 + k * 32);
                            const uint64_t b1 = sdesc(base + Cfg::OFF_B1 + k * 32);
                            mma2<Cfg::TF32>(dt, a0, b1, 1u);
                            mma2<Cfg::TF32>(dt, a1, b0, 1u);
                        }
                    }
                    commit2(su32(&empty[s]));
                    commit2(peer_addr(su32(&empty[s]), peer));
                    if (kt % cs == cs - 1 || kt == nk - 1) {
                        commit2(su32(&cfull[buf]));
                        commit2(peer_addr(su32(&cfull[buf]), peer));
                    }
                }
            }
            commit2(su32(done));
            commit2(peer_addr(su32(done), peer));
        }
    } else {
        // ---- epilogue warps 0-3 of each CTA: thread = row of this CTA's tile ----
        bool ok = true;
        int cg = 0;
        const uint32_t cfree_pair = lead ? su32(&cfree[0]) : peer_addr(su32(&cfree[0]), 0);
        for (int w = cl; w < items && ok; w += ncl, cg += nchunks) {
            const int bz = w / ptiles;
            int TP, tn;
            tctiles::pair_tile(w - bz * ptiles, g.mode, tiles_m, tiles_n, TP, tn);
            const int tm = 2 * TP + static_cast<int>(rank);
            const bool write = tctiles::pair_tile_valid(g.mode, tiles_m, TP, tn, static_cast<int>(rank));
            const float *Dp = g.D ? g.D + bz * g.sC : nullptr;
            float *Cp = g.C ? g.C + bz * g.sC : nullptr;
            float acc[TN];
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[j] = 0.f;
            const int row = warp * 32 + lane;
            const long long m = static_cast<long long>(tm) * TM + row;
            for (int c = 0; c < nchunks; ++c) {
                const int buf = (cg + c) % kBufs;
                if (write && c == max(0, nchunks - 2) && g.beta != 0.f) {
                    const float *drow = Dp + m * g.ld + static_cast<long long>(tn) * TN;
#pragma unroll
                    for (int q = 0; q < TN / 32; ++q) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(drow + 32 * q));
                }
                ok = mbar_wait_cl(&cfull[buf], ((cg + c) / kBufs) & 1, g.err) && !*abort_flag;
                ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t tb = tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(buf * TN);
#pragma unroll
                for (int q = 0; q < TN / 32; ++q) {
                    uint32_t r[32];
                    tmem_ld32(tb + q * 32, r);
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc[q * 32 + j] += __uint_as_float(r[j]);
                }
                fence_before();
                __syncwarp();
                if (lane == 0) remote_arrive(cfree_pair + static_cast<uint32_t>(buf) * 8u);
            }
            if (ok && write) tile_epilogue<KIND>(g, acc, m, tm, tn, Dp, Cp, lane);
        }
    }
    __syncwarp();
    fence_before();
    __syncthreads();
    if (warp == 0) {
        // every MMA of the pair must have completed before this CTA's tensor memory is freed
        if (lane == 0) mbar_wait_cl(done, 0, g.err);
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kBufs * TN));
    }
    __syncthreads();
    cluster_sync();   // the peer no longer signals this CTA's shared memory
}

// The GEMM's bounded wait on a barrier that nothing arrives at: it gives up after `budget`
// cycles and raises ST_TC_TIMEOUT, as a GEMM wait does.  One thread; nothing in flight.
__global__ void k_wait_probe(long long budget, int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        mbar_wait(&bar, 0, err, budget);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map of a row-major rows x cols matrix (row pitch ld elements), box of 128 rows
// by 128 bytes, 128-byte swizzle.
bool make_map(CUtensorMap *m, const void *base, int kind, long long rows, long long cols, long long ld,
              int box_rows = TM) {
    auto fn = encode_fn();
    if (!fn || !base) return false;
    const int elem = kind == 1 ? 2 : 4;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld * elem)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(KB / elem), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t es[2] = {1, 1};
    return fn(m, kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
              const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KIND>
cudaError_t launch_tc(const TcOperands &op, const TcArgs &g, cudaStream_t s) {
    using Cfg = TcCfg<KIND>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap a0, a1, b0, b1;
    const long long lda = op.lda, ldb = op.ldb;
    const long long rows_a = static_cast<long long>(g.batch) * g.M, rows_b = static_cast<long long>(g.batch) * g.N;
    if (!make_map(&a0, op.A0, KIND, rows_a, g.K, lda) || !make_map(&b0, op.B0, KIND, rows_b, g.K, ldb))
        return cudaErrorInvalidValue;
    if (KIND != 0) {
        if (!make_map(&a1, op.A1, KIND, rows_a, g.K, lda) || !make_map(&b1, op.B1, KIND, rows_b, g.K, ldb))
            return cudaErrorInvalidValue;
    } else {
        a1 = a0;
        b1 = b0;
    }
    const int tmt = g.M / TM, tnt = g.N / TN;
    const long long items = static_cast<long long>(g.mode == 0 ? tmt * tnt : tmt * (tmt + 1) / 2) * g.batch;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = static_cast<int>(std::min<long long>(items, sms));   // one resident CTA per SM
    count_launches(1);
    k_tc_gemm<KIND><<<grid, 192, Cfg::SMEM, s>>>(a0, a1, b0, b1, g, tnt);
    return cudaGetLastError();
}

// (tm, TPn) of every wide-tile work item of (mode, tiles_m, tiles_n), computed on the host by
// the decomposition of tc_tiles.cuh and kept on the device for the life of the process (one
// table per shape and device): the kernel's threads then look their tile up instead of walking
// the super-tiles, which costs the single producer thread thousands of cycles per tile.
cudaError_t wide_tile_table(int dev, int mode, int tiles_m, int tiles_n, const int2 **out) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int>, int2 *> cache;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, mode, tiles_m, tiles_n);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    const int n = tctiles::wide_tile_count(mode, tiles_m, tiles_n);
    std::vector<int2> h(static_cast<size_t>(n));
    for (int b = 0; b < n; ++b) tctiles::wide_tile(b, mode, tiles_m, tiles_n, h[b].x, h[b].y);
    int2 *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int2) * std::max(n, 1));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(d, h.data(), sizeof(int2) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return e;
    }
    cache[key] = d;
    *out = d;
    return cudaSuccess;
}

template <int KIND>
cudaError_t launch_tcw(const TcOperands &op, const TcArgs &g, cudaStream_t s) {
    using Cfg = TcCfgW<KIND>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_gemm_w<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap a0, a1, b0, b1;
    const long long lda = op.lda, ldb = op.ldb;
    const long long rows_a = static_cast<long long>(g.batch) * g.M, rows_b = static_cast<long long>(g.batch) * g.N;
    if (!make_map(&a0, op.A0, KIND, rows_a, g.K, lda, TM) || !make_map(&b0, op.B0, KIND, rows_b, g.K, ldb, TNW))
        return cudaErrorInvalidValue;
    if (KIND != 0) {
        if (!make_map(&a1, op.A1, KIND, rows_a, g.K, lda, TM) || !make_map(&b1, op.B1, KIND, rows_b, g.K, ldb, TNW))
            return cudaErrorInvalidValue;
    } else {
        a1 = a0;
        b1 = b0;
    }
    const int tmt = g.M / TM, tnt = g.N / TN;
    const long long items = static_cast<long long>(tctiles::wide_tile_count(g.mode, tmt, tnt)) * g.batch;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = static_cast<int>(std::min<long long>(items, sms));
    const int2 *table = nullptr;
    e = wide_tile_table(dev, g.mode, tmt, tnt, &table);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_tc_gemm_w<KIND><<<grid, 384, Cfg::SMEM, s>>>(a0, a1, b0, b1, g, tnt, table);
    return cudaGetLastError();
}

// CTA-pair launch: clusters of two CTAs, one pair per two SMs, as many pairs as fit at once
// (persistent), each looping over pair tiles.
template <int KIND>
cudaError_t launch_tc2(const TcOperands &op, const TcArgs &g, cudaStream_t s) {
    using Cfg = TcCfg2<KIND>;
    static int max_clusters = 0;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attrs[1];
    attrs[0].id = cudaLaunchAttributeClusterDimension;
    attrs[0].val.clusterDim.x = 2;
    attrs[0].val.clusterDim.y = 1;
    attrs[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = Cfg::SMEM;
    cfg.stream = s;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    if (!max_clusters) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_gemm2<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        cfg.gridDim = dim3(static_cast<unsigned>(sms & ~1), 1, 1);
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k_tc_gemm2<KIND>, &cfg);
        if (e != cudaSuccess) return e;
        if (n < 1) return cudaErrorInvalidConfiguration;
        max_clusters = n;
    }
    CUtensorMap a0, a1, b0, b1;
    const long long lda = op.lda, ldb = op.ldb;
    const long long rows_a = static_cast<long long>(g.batch) * g.M, rows_b = static_cast<long long>(g.batch) * g.N;
    if (!make_map(&a0, op.A0, KIND, rows_a, g.K, lda, TM) || !make_map(&b0, op.B0, KIND, rows_b, g.K, ldb, TN / 2))
        return cudaErrorInvalidValue;
    if (KIND != 0) {
        if (!make_map(&a1, op.A1, KIND, rows_a, g.K, lda, TM) || !make_map(&b1, op.B1, KIND, rows_b, g.K, ldb, TN / 2))
            return cudaErrorInvalidValue;
    } else {
        a1 = a0;
        b1 = b0;
    }
    const int tmt = g.M / TM, tnt = g.N / TN;
    const long long items = static_cast<long long>(tctiles::pair_tile_count(g.mode, tmt, tnt)) * g.batch;
    const int clusters = static_cast<int>(std::min<long long>(items, max_clusters));
    cfg.gridDim = dim3(static_cast<unsigned>(2 * clusters), 1, 1);
    count_launches(1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_tc_gemm2<KIND>, a0, a1, b0, b1, g, tnt);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Form of the GEMM: MBDGB_TC_FORM in the environment selects "wide" (128 x 256 tiles),
// "single" (128 x 128 tiles, one CTA) or "pair" (256 x 128 tiles on a CTA pair); the default is
// the wide form.
int tc_form() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("MBDGB_TC_FORM");
        const std::string f = e ? std::string(e) : std::string();
        v = f == "pair" ? 2 : (f == "single" ? 1 : 0);
    }
    return v;
}

}  // namespace

cudaError_t tc_wait_probe(long long budget, int *err, cudaStream_t s) {
    if (budget < 1 || budget > (1LL << 32) || !err) return cudaErrorInvalidValue;
    count_launches(1);
    k_wait_probe<<<1, 32, 0, s>>>(budget, err);
    return cudaGetLastError();
}

cudaError_t tc_gemm(int kind, const TcOperands &op, const TcArgs &g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.M % TM || g.N % TN || g.K % 64 || g.mode < 0 || g.mode > 2 ||
        (g.mode != 0 && (g.M != g.N || g.CT || g.CTh || g.resid)) || ((g.CT || g.CTh) && g.M != g.N) ||
        g.ld % 8 || op.lda % 8 || op.ldb % 8 ||
        !g.err || (g.beta != 0.f && !g.D) || (g.Ch && !g.Cl) || (g.CTh && !g.CTl) || kind < 0 || kind > 2 ||
        (kind != 0 && (!op.A1 || !op.B1)) || (kind == 0 && (g.Ch || g.CTh)) || g.batch < 1 || g.batch > 65535 ||
        (g.batch > 1 && (g.Ch || g.CT || g.CTh || g.C64 || g.resid || g.sC < static_cast<long long>(g.M) * g.ld)))
        return cudaErrorInvalidValue;
    const int form = tc_form();
    if (form == 0) {
        if (kind == 0) return launch_tcw<0>(op, g, s);
        if (kind == 1) return launch_tcw<1>(op, g, s);
        return launch_tcw<2>(op, g, s);
    }
    if (form == 2) {
        if (kind == 0) return launch_tc2<0>(op, g, s);
        if (kind == 1) return launch_tc2<1>(op, g, s);
        return launch_tc2<2>(op, g, s);
    }
    if (kind == 0) return launch_tc<0>(op, g, s);
    if (kind == 1) return launch_tc<1>(op, g, s);
    return launch_tc<2>(op, g, s);
}

}  // namespace mbdgb

// ---- conversions and the variational energy of the mixed-precision path ----------
namespace mbdgb {
namespace {

// Split v into the hi/lo operand pair of a split mode: kind 1 bf16 (hi, lo), kind 2
// TF32-rounded hi and FP32 remainder; element e of the arrays H, L.
__device__ __forceinline__ void split_store(int kind, float v, void *H, void *L, long long e) {
    if (kind == 1) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        static_cast<__nv_bfloat16 *>(H)[e] = h;
        static_cast<__nv_bfloat16 *>(L)[e] = __float2bfloat16_rn(v - __bfloat162float(h));
    } else {
        uint32_t h, l;
        asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(v));
        asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(l) : "f"(v - __uint_as_float(h)));
        static_cast<uint32_t *>(H)[e] = h;
        static_cast<uint32_t *>(L)[e] = l;
    }
}

// TF32x3 parts of scale * Q for an FP64 Q: hi = tf32(q), lo = tf32(q - hi), both rounded
// to nearest, the remainder taken in FP64.
__global__ void k_split_tf32_f64(const double *Q, long long total, long long ld, double scale, int zero_diag,
                                 uint32_t *H, uint32_t *L) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double q = (zero_diag && e / ld == e % ld) ? 0.0 : scale * Q[e];
        uint32_t h, l;
        asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(static_cast<float>(q)));
        asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(l) : "f"(static_cast<float>(q - static_cast<double>(__uint_as_float(h)))));
        H[e] = h;
        L[e] = l;
    }
}

// TF32x3 parts of scale * A^T for an FP64 A (32x32 tiles through shared memory).
__global__ void k_split_tf32_f64_t(const double *A, long long ld, double scale, uint32_t *H, uint32_t *L) {
    __shared__ double t[32][33];
    const long long r0 = static_cast<long long>(blockIdx.y) * 32, c0 = static_cast<long long>(blockIdx.x) * 32;
    for (int k = threadIdx.y; k < 32; k += 8) t[k][threadIdx.x] = A[(r0 + k) * ld + c0 + threadIdx.x];
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const double q = scale * t[threadIdx.x][k];
        uint32_t h, l;
        asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(static_cast<float>(q)));
        asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(l) : "f"(static_cast<float>(q - static_cast<double>(__uint_as_float(h)))));
        const long long o = (c0 + k) * ld + r0 + threadIdx.x;
        H[o] = h;
        L[o] = l;
    }
}

// TF32x3 parts of an FP32 matrix (optionally with its diagonal set to zero).
__global__ void k_split_tf32_f32(const float *Z, long long total, long long ld, int zero_diag, uint32_t *H,
                                 uint32_t *L) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        split_store(2, (zero_diag && e / ld == e % ld) ? 0.f : Z[e], H, L, e);
}

// TF32x3 parts of a rows x cols panel of each matrix of a batch (A points at the panel's
// first element, row pitch ld, matrices mstride apart) into H, L stacked as
// [batch][rows][cols].
__global__ void k_split_panel_tf32(const float *A, long long ld, long long mstride, long long rows, int cols,
                                   long long total, uint32_t *H, uint32_t *L) {
    const long long per = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long b = e / per, r = e - b * per, i = r / cols, c = r - i * cols;
        split_store(2, A[b * mstride + i * ld + c], H, L, e);
    }
}

// tq[i] = sqrt_s (3 Tr V_ii - Tr (V W)_ii) / 2 over the 3x3 diagonal block of atom i; one
// warp per atom, (V W)_pp = sum_k V[p][k] W[k][p] with the rows of V read coalesced.
__global__ void __launch_bounds__(128) k_block_trace_sqrt(const double *V, const double *W, long long ld, int N,
                                                         double sqrt_s, double *tq) {
    const int i = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= N) return;
    double acc = 0.0;
    for (int x = 0; x < 3; ++x) {
        const long long p = 3LL * i + x;
        const double *vp = V + p * ld;
        for (long long k = lane; k < ld; k += 32) acc += vp[k] * W[k * ld + p];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const long long p = 3LL * i;
        const double trv = V[p * ld + p] + V[(p + 1) * ld + p + 1] + V[(p + 2) * ld + p + 2];
        tq[i] = sqrt_s * 0.5 * (3.0 * trv - acc);
    }
}

// Out[p][q] = scale * A[p][p] * B[p][q] (row scaling by a diagonal, FP64).
template <typename TA, typename TB>
__global__ void k_diag_scale_rows(const TA *A, const TB *B, long long ld, double scale, double *Out) {
    const long long total = ld * ld;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long p = e / ld;
        Out[e] = scale * static_cast<double>(A[p * ld + p]) * static_cast<double>(B[e]);
    }
}

// Y = scale * Q (FP64 -> FP32, plus bf16 hi/lo when Yh is given); Z = I likewise.
__global__ void k_mixed_init(int kind, const double *Q, long long total, long long ld, double scale, float *Yf,
                             void *Yh, void *Yl, float *Zf, void *Zh, void *Zl) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float y = static_cast<float>(scale * Q[e]);
        const float z = (e / ld == e % ld) ? 1.f : 0.f;
        Yf[e] = y;
        Zf[e] = z;
        if (Yh) {
            split_store(kind, y, Yh, Yl, e);
            split_store(kind, z, Zh, Zl, e);
        }
    }
}

// Z = a I + b P (first scaled Newton-Schulz step, where P = Y0).
__global__ void k_mixed_axpby_identity(int kind, const float *P, long long total, long long ld, float a, float b,
                                       float *Zf, void *Zh, void *Zl) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float z = ((e / ld == e % ld) ? a : 0.f) + b * P[e];
        Zf[e] = z;
        if (Zh) split_store(kind, z, Zh, Zl, e);
    }
}

// Zd = scale * Zf (FP32 -> FP64).
__global__ void k_to_f64(const float *Zf, long long total, double scale, double *Zd) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        Zd[e] = scale * static_cast<double>(Zf[e]);
}

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Per-block compensated partial sums of Tr V (diagonal of the leading n x n block) and
// of sum_pq V_pq W_pq; out[2 * block + {0,1}].
__global__ void __launch_bounds__(256) k_trace_dot_partials(const double *V, const double *W, long long ld, int n,
                                                            double *out) {
    double s0 = 0.0, c0 = 0.0, s1 = 0.0, c1 = 0.0;
    const long long total = static_cast<long long>(n) * n;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < total; e += static_cast<long long>(gridDim.x) * 256) {
        const long long i = e / n, j = e % n;
        const double v = V[i * ld + j];
        double t, r;
        two_sum(s1, v * W[i * ld + j], t, r);
        s1 = t; c1 += r;
        if (i == j) {
            two_sum(s0, v, t, r);
            s0 = t; c0 += r;
        }
    }
    __shared__ double sh[4][256];
    sh[0][threadIdx.x] = s0; sh[1][threadIdx.x] = c0; sh[2][threadIdx.x] = s1; sh[3][threadIdx.x] = c1;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, ac = 0.0, b = 0.0, bc = 0.0;
        for (int k = 0; k < 256; ++k) {
            double t, r;
            two_sum(a, sh[0][k], t, r); a = t; ac += r + sh[1][k];
            two_sum(b, sh[2][k], t, r); b = t; bc += r + sh[3][k];
        }
        out[2 * blockIdx.x] = a + ac;
        out[2 * blockIdx.x + 1] = b + bc;
    }
}

// Per-block compensated partials over the leading n x n block of T1 = sum (scale Q) o Z
// (FP64 x FP32, i.e. Tr(scale Q Z) for symmetric Z), T2 = sum V o W (FP32 x FP32) and
// R = sum (delta - W)^2; out[3 * block + {0,1,2}].
__global__ void __launch_bounds__(256) k_correction_partials(const double *Q, double scale, const float *Z,
                                                             const double *V, const double *W, long long ld, int n,
                                                             double *out) {
    double s0 = 0.0, c0 = 0.0, s1 = 0.0, c1 = 0.0, r2 = 0.0;
    const long long total = static_cast<long long>(n) * n;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < total; e += static_cast<long long>(gridDim.x) * 256) {
        const long long i = e / n, j = e % n, o = i * ld + j;
        double t, r;
        two_sum(s0, scale * Q[o] * static_cast<double>(Z[o]), t, r);
        s0 = t; c0 += r;
        const double w = W[o];
        two_sum(s1, V[o] * w, t, r);
        s1 = t; c1 += r;
        const double d = (i == j ? 1.0 : 0.0) - w;
        r2 += d * d;
    }
    __shared__ double sh[5][256];
    sh[0][threadIdx.x] = s0; sh[1][threadIdx.x] = c0; sh[2][threadIdx.x] = s1; sh[3][threadIdx.x] = c1;
    sh[4][threadIdx.x] = r2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, ac = 0.0, b = 0.0, bc = 0.0, rr = 0.0;
        for (int k = 0; k < 256; ++k) {
            double t, r;
            two_sum(a, sh[0][k], t, r); a = t; ac += r + sh[1][k];
            two_sum(b, sh[2][k], t, r); b = t; bc += r + sh[3][k];
            rr += sh[4][k];
        }
        out[3 * blockIdx.x] = a + ac;
        out[3 * blockIdx.x + 1] = b + bc;
        out[3 * blockIdx.x + 2] = rr;
    }
}

// E = (sqrt(s)/4)(3 T1 - T2) - 3/2 sum omega_bar; resid = sqrt(R).
__global__ void k_energy_correction(const double *part, int nblocks, double sqrt_s, const double *ombar, int N,
                                    double *out, double *resid) {
    if (threadIdx.x != 0) return;
    double a = 0.0, ac = 0.0, b = 0.0, bc = 0.0, w = 0.0, wc = 0.0, rr = 0.0;
    for (int k = 0; k < nblocks; ++k) {
        double t, r;
        two_sum(a, part[3 * k], t, r); a = t; ac += r;
        two_sum(b, part[3 * k + 1], t, r); b = t; bc += r;
        rr += part[3 * k + 2];
    }
    for (int i = 0; i < N; ++i) {
        double t, r;
        two_sum(w, ombar[i], t, r); w = t; wc += r;
    }
    out[0] = 0.25 * sqrt_s * (3.0 * (a + ac) - (b + bc)) - 1.5 * (w + wc);
    resid[0] = sqrt(rr);
}

// E = 1/2 * (1/2)(3 Tr V - sum V o W) - 3/2 sum omega_bar, from the partials (one CTA).
__global__ void k_energy_variational(const double *part, int nblocks, const double *ombar, int N, double *out) {
    if (threadIdx.x != 0) return;
    double a = 0.0, ac = 0.0, b = 0.0, bc = 0.0, w = 0.0, wc = 0.0;
    for (int k = 0; k < nblocks; ++k) {
        double t, r;
        two_sum(a, part[2 * k], t, r); a = t; ac += r;
        two_sum(b, part[2 * k + 1], t, r); b = t; bc += r;
    }
    for (int i = 0; i < N; ++i) {
        double t, r;
        two_sum(w, ombar[i], t, r); w = t; wc += r;
    }
    const double trv = a + ac, vw = b + bc, sw = w + wc;
    out[0] = 0.25 * (3.0 * trv - vw) - 1.5 * sw;
}

inline int grid_for(long long total) { return static_cast<int>(std::min<long long>((total + 255) / 256, 152 * 16)); }

}  // namespace

void mixed_init(int kind, const double *Q, long long ld, double scale, float *Yf, void *Yh, void *Yl, float *Zf,
                void *Zh, void *Zl, cudaStream_t s) {
    count_launches(1);
    k_mixed_init<<<grid_for(ld * ld), 256, 0, s>>>(kind, Q, ld * ld, ld, scale, Yf, Yh, Yl, Zf, Zh, Zl);
}

void mixed_axpby_identity(int kind, const float *P, long long ld, float a, float b, float *Zf, void *Zh, void *Zl,
                          cudaStream_t s) {
    count_launches(1);
    k_mixed_axpby_identity<<<grid_for(ld * ld), 256, 0, s>>>(kind, P, ld * ld, ld, a, b, Zf, Zh, Zl);
}

void to_f64(const float *Zf, long long ld, double scale, double *Zd, cudaStream_t s) {
    count_launches(1);
    k_to_f64<<<grid_for(ld * ld), 256, 0, s>>>(Zf, ld * ld, scale, Zd);
}

void split_tf32_f64(const double *Q, long long ld, double scale, int zero_diag, void *H, void *L, cudaStream_t s) {
    count_launches(1);
    k_split_tf32_f64<<<grid_for(ld * ld), 256, 0, s>>>(Q, ld * ld, ld, scale, zero_diag, static_cast<uint32_t *>(H),
                                                       static_cast<uint32_t *>(L));
}

void diag_scale_rows_f64(const double *A, const float *B, long long ld, double scale, double *Out, cudaStream_t s) {
    count_launches(1);
    k_diag_scale_rows<double, float><<<grid_for(ld * ld), 256, 0, s>>>(A, B, ld, scale, Out);
}

void diag_scale_rows_f32(const float *A, const double *B, long long ld, double *Out, cudaStream_t s) {
    count_launches(1);
    k_diag_scale_rows<float, double><<<grid_for(ld * ld), 256, 0, s>>>(A, B, ld, 1.0, Out);
}

void split_tf32_f64_t(const double *A, long long ld, double scale, void *H, void *L, cudaStream_t s) {
    count_launches(1);
    k_split_tf32_f64_t<<<dim3(static_cast<unsigned>(ld / 32), static_cast<unsigned>(ld / 32)), dim3(32, 8), 0, s>>>(
        A, ld, scale, static_cast<uint32_t *>(H), static_cast<uint32_t *>(L));
}

void split_tf32_f32(const float *Z, long long ld, int zero_diag, void *H, void *L, cudaStream_t s) {
    count_launches(1);
    k_split_tf32_f32<<<grid_for(ld * ld), 256, 0, s>>>(Z, ld * ld, ld, zero_diag, static_cast<uint32_t *>(H),
                                                       static_cast<uint32_t *>(L));
}

void block_trace_sqrt(const double *V, const double *W, long long ld, int N, double sqrt_s, double *tq,
                      cudaStream_t s) {
    count_launches(1);
    k_block_trace_sqrt<<<(N + 3) / 4, 128, 0, s>>>(V, W, ld, N, sqrt_s, tq);
}

void split_panel_tf32(const float *A, long long ld, long long mstride, int batch, long long rows, int cols,
                      uint32_t *H, uint32_t *L, cudaStream_t s) {
    const long long total = static_cast<long long>(batch) * rows * cols;
    count_launches(1);
    k_split_panel_tf32<<<grid_for(total), 256, 0, s>>>(A, ld, mstride, rows, cols, total, H, L);
}

void energy_correction(const double *Q, double scale, const float *Z, const double *V, const double *W, long long ld,
                       int n, double sqrt_s, const double *ombar, int N, double *work, double *out, double *resid,
                       cudaStream_t s) {
    const int nb = 304;   // work: 3 * nb doubles
    count_launches(2);
    k_correction_partials<<<nb, 256, 0, s>>>(Q, scale, Z, V, W, ld, n, work);
    k_energy_correction<<<1, 32, 0, s>>>(work, nb, sqrt_s, ombar, N, out, resid);
}

void energy_variational(const double *V, const double *W, long long ld, int n, const double *ombar, int N,
                        double *work, double *out, cudaStream_t s) {
    const int nb = 304;   // work: 2 * nb doubles
    count_launches(2);
    k_trace_dot_partials<<<nb, 256, 0, s>>>(V, W, ld, n, work);
    k_energy_variational<<<1, 32, 0, s>>>(work, nb, ombar, N, out);
}

}  // namespace mbdgb
