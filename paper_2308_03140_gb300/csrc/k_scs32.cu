// Mixed-precision screening solves for Eq. (scs): the matrices A(u) = alpha(u)^{-1} +
// T^scs (one per frequency point, Sec. 2.3) are factorised in FP32, blocked in panels of
// kScsPanel columns, each panel in sub-panels of kScsSub columns: 64-wide right-looking
// steps inside a sub-panel on the CUDA cores (SIMT FFMA), the panel's columns right of each
// sub-panel and the trailing matrix after each panel updated on the tensor cores (TF32x3
// parts, k_tc.cu).  A X = B is then solved by iterative refinement:
// X <- X + A32^{-1} (B - A X), with the residual formed from the FP64 matrix.  For the
// moderately conditioned screening matrices (cond ~ 1e1 - 2e3) the FP32 solution is within a
// few 1e-7 and each step gains six digits or more.
//
// Layout as in k_dense.cu: batch of row-major ld x ld matrices, ld a multiple of 64,
// right-hand sides [batch][ld][3].
#include "internal.h"

namespace mbdgb {
namespace {

constexpr int T64 = 64;

__device__ __forceinline__ double warp_sumd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// C = alpha A B^T + beta C on 64x64 tiles, FP32 SIMT: 256 threads, 4x4 outputs each.
// mode 0 all tiles, mode 1 lower tiles only (square).  Batched by blockIdx.z.
__global__ void __launch_bounds__(256) k_sgemm_nt(const float *A, const float *B, float *C, long long lda,
                                                  long long ldb, long long ldc, long long sA, long long sB,
                                                  long long sC, int K, float alpha, float beta, int mode,
                                                  int tiles_n) {
    int tm, tn;
    if (mode == 0) {
        tm = blockIdx.x / tiles_n;
        tn = blockIdx.x % tiles_n;
    } else {
        int x = static_cast<int>((sqrt(8.0 * blockIdx.x + 1.0) - 1.0) * 0.5);
        while ((x + 1) * (x + 2) / 2 <= static_cast<int>(blockIdx.x)) ++x;
        while (x * (x + 1) / 2 > static_cast<int>(blockIdx.x)) --x;
        tm = x;
        tn = blockIdx.x - x * (x + 1) / 2;
    }
    const long long b = blockIdx.z;
    const float *Ab = A + b * sA + static_cast<long long>(tm) * T64 * lda;
    const float *Bb = B + b * sB + static_cast<long long>(tn) * T64 * ldb;
    __shared__ float As[16][T64 + 4], Bs[16][T64 + 4];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    float acc[4][4] = {};
    const int lr = t >> 2, lk = (t & 3) * 4;   // loader: row 0..63, k offset 0,4,8,12
    for (int k0 = 0; k0 < K; k0 += 16) {
        const float4 a = *reinterpret_cast<const float4 *>(Ab + static_cast<long long>(lr) * lda + k0 + lk);
        const float4 c = *reinterpret_cast<const float4 *>(Bb + static_cast<long long>(lr) * ldb + k0 + lk);
        As[lk][lr] = a.x; As[lk + 1][lr] = a.y; As[lk + 2][lr] = a.z; As[lk + 3][lr] = a.w;
        Bs[lk][lr] = c.x; Bs[lk + 1][lr] = c.y; Bs[lk + 2][lr] = c.z; Bs[lk + 3][lr] = c.w;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float4 av = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
        }
        __syncthreads();
    }
    float *Cb = C + b * sC;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long m = static_cast<long long>(tm) * T64 + ty * 4 + i;
        float4 *cp = reinterpret_cast<float4 *>(Cb + m * ldc + static_cast<long long>(tn) * T64 + tx * 4);
        float4 cv = beta != 0.f ? *cp : make_float4(0.f, 0.f, 0.f, 0.f);
        cv.x = alpha * acc[i][0] + beta * cv.x;
        cv.y = alpha * acc[i][1] + beta * cv.y;
        cv.z = alpha * acc[i][2] + beta * cv.z;
        cv.w = alpha * acc[i][3] + beta * cv.w;
        *cp = cv;
    }
}

// FP32 Cholesky of a 64x64 diagonal block plus the inverse of its factor, one CTA per
// matrix.  The factorisation is blocked by 16: warp 0 factors each 16x16 diagonal block
// (warp-synchronous, one lane per row), one thread per row solves the rows below it, and
// all threads apply the 16-term trailing update (3 block barriers per 16 columns).  The
// inverse is blocked by 16 as well: the diagonal blocks by forward substitution in
// registers, the blocks below them by two small block products per block row.
__global__ void __launch_bounds__(256) k_spotrf_diag(float *A, long long ld, long long mstride, float *dinv,
                                                     long long dstride, int *status) {
    __shared__ float S[64][65];
    __shared__ float V[64][65];
    __shared__ float Tp[3][16][17];
    __shared__ int bad;
    float *Ab = A + static_cast<long long>(blockIdx.x) * mstride;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) bad = 0;
    for (int e = t; e < 4096; e += 256) {
        const int r = e >> 6, c = e & 63;
        S[r][c] = (c <= r) ? Ab[r * ld + c] : 0.f;
    }
    __syncthreads();
    for (int j0 = 0; j0 < 64; j0 += 16) {
        if (warp == 0) {   // 16x16 diagonal block, lane = row j0 + lane
            for (int j = 0; j < 16; ++j) {
                const int jj = j0 + j;
                float d = S[jj][jj];
                if (!(d > 0.f)) {
                    if (lane == 0) bad = 1;
                    d = 1.f;
                }
                d = sqrtf(d);
                __syncwarp();
                if (lane == 0) S[jj][jj] = d;
                if (lane > j && lane < 16) S[j0 + lane][jj] /= d;
                __syncwarp();
                if (lane > j && lane < 16) {
                    const int i = j0 + lane;
                    const float lij = S[i][jj];
                    for (int k = jj + 1; k <= i; ++k) S[i][k] -= lij * S[k][jj];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int i = j0 + 16 + t; i < 64; i += 256) {   // rows below: L21 = A21 L11^{-T}
            for (int c = 0; c < 16; ++c) {
                float v = S[i][j0 + c];
                for (int k = 0; k < c; ++k) v -= S[i][j0 + k] * S[j0 + c][j0 + k];
                S[i][j0 + c] = v / S[j0 + c][j0 + c];
            }
        }
        __syncthreads();
        const int r0 = j0 + 16;   // trailing lower triangle [r0, 64)^2 -= L21 L21^T
        if (r0 < 64) {
            const int ty = t >> 4, tx = t & 15;
            for (int i = r0 + ty; i < 64; i += 16)
                for (int k = r0 + tx; k <= i; k += 16) {
                    float v = S[i][k];
#pragma unroll
                    for (int c = 0; c < 16; ++c) v -= S[i][j0 + c] * S[k][j0 + c];
                    S[i][k] = v;
                }
        }
        __syncthreads();
    }
    // V = L^{-1} by 16x16 blocks.  Diagonal blocks: warp w < 4 inverts block w, lane c < 16
    // holding column c in registers (forward substitution).  Block rows I = 1..3 then follow
    // from V_IJ = -V_II sum_{K=J}^{I-1} L_IK V_KJ (J < I), every element in parallel.
    if (warp < 4 && lane < 16) {
        const int b0 = 16 * warp, c = lane;
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            float sum = (i == c) ? 1.f : 0.f;
#pragma unroll
            for (int k = 0; k < i; ++k)
                if (k >= c) sum -= S[b0 + i][b0 + k] * v[k];
            v[i] = (i >= c) ? sum / S[b0 + i][b0 + i] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) V[b0 + i][b0 + c] = v[i];
    }
    __syncthreads();
    for (int I = 1; I < 4; ++I) {
        for (int e = t; e < I * 256; e += 256) {   // Tp[J] = sum_K L_IK V_KJ
            const int J = e >> 8, r = (e >> 4) & 15, cc = e & 15;
            const int i = 16 * I + r, j = 16 * J + cc;
            float sum = 0.f;
            for (int k = 16 * J; k < 16 * I; ++k) sum += S[i][k] * V[k][j];
            Tp[J][r][cc] = sum;
        }
        __syncthreads();
        for (int e = t; e < I * 256; e += 256) {   // V_IJ = -V_II Tp[J]
            const int J = e >> 8, r = (e >> 4) & 15, cc = e & 15;
            float sum = 0.f;
            for (int k = 0; k <= r; ++k) sum += V[16 * I + r][16 * I + k] * Tp[J][k][cc];
            V[16 * I + r][16 * J + cc] = -sum;
        }
        __syncthreads();
    }
    float *Db = dinv + static_cast<long long>(blockIdx.x) * dstride;
    for (int e = t; e < 4096; e += 256) {
        const int r = e >> 6, c = e & 63;
        if (c <= r) Ab[r * ld + c] = S[r][c];
        Db[e] = (c > r) ? 0.f : V[r][c];
    }
    if (t == 0 && bad) atomicOr(status, ST_SCS_NOT_PD);
}

// B32 = (float) A64, whole batch.
__global__ void k_to_f32(const double *A, long long total, float *B) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        B[e] = static_cast<float>(A[e]);
}

// R = B - A X (FP64, A full row-major, 3 RHS); r32 = (float) R.  A CTA of 8 warps owns 32
// consecutive rows (4 per warp) and stages X in chunks of 1024 rows in shared memory, so X is
// read from L2 once per 32 rows while A streams from HBM once; the column loop is unrolled so
// that each lane keeps 16 loads of A in flight.
constexpr int kResRows = 4, kResChunk = 1024;
__global__ void __launch_bounds__(256) k_residual3(const double *A, long long ld, long long mstride, const double *Bv,
                                                   const double *X, long long xstride, float *r32, int n) {
    __shared__ double xs[kResChunk * 3];
    const int b = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long row0 = blockIdx.x * 32LL + warp * kResRows;
    const double *Ab = A + b * mstride;
    const double *x = X + b * xstride;
    double acc[kResRows][3];
#pragma unroll
    for (int r = 0; r < kResRows; ++r) acc[r][0] = acc[r][1] = acc[r][2] = 0.0;
    for (int c0 = 0; c0 < n; c0 += kResChunk) {
        const int m = min(kResChunk, n - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < 3 * m; e += 256) xs[e] = x[3LL * c0 + e];
        __syncthreads();
#pragma unroll 4
        for (int c = lane; c < m; c += 32) {
            const double x0 = xs[3 * c], x1 = xs[3 * c + 1], x2 = xs[3 * c + 2];
#pragma unroll
            for (int r = 0; r < kResRows; ++r) {
                const long long row = row0 + r;
                if (row < n) {
                    const double v = Ab[row * ld + c0 + c];
                    acc[r][0] += v * x0;
                    acc[r][1] += v * x1;
                    acc[r][2] += v * x2;
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kResRows; ++r) {
        const double s0 = warp_sumd(acc[r][0]), s1 = warp_sumd(acc[r][1]), s2 = warp_sumd(acc[r][2]);
        const long long row = row0 + r;
        if (lane == 0 && row < ld) {
            const double *bb = Bv + b * xstride + 3 * row;
            float *rr = r32 + b * xstride + 3 * row;
            rr[0] = static_cast<float>(bb[0] - (row < n ? s0 : 0.0));
            rr[1] = static_cast<float>(bb[1] - (row < n ? s1 : 0.0));
            rr[2] = static_cast<float>(bb[2] - (row < n ? s2 : 0.0));
        }
    }
}

// X64 (+)= (double) X32 over [batch][ld][3].
__global__ void k_accumulate(double *X, const float *dx, long long total, int overwrite) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        X[e] = (overwrite ? 0.0 : X[e]) + static_cast<double>(dx[e]);
}

__global__ void k_rhs_to_f32(const double *B, long long total, float *b32) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        b32[e] = static_cast<float>(B[e]);
}

inline int gridn(long long total) { return static_cast<int>(std::min<long long>((total + 255) / 256, 152 * 16)); }

void sgemm_nt(const float *A, const float *B, float *C, long long lda, long long ldb, long long ldc, long long sA,
              long long sB, long long sC, int M, int N, int K, int batch, float alpha, float beta, int mode,
              cudaStream_t s) {
    const int tm = M / T64, tn = N / T64;
    const dim3 grid(mode == 0 ? tm * tn : tm * (tm + 1) / 2, 1, batch);
    count_launches(1);
    k_sgemm_nt<<<grid, 256, 0, s>>>(A, B, C, lda, ldb, ldc, sA, sB, sC, K, alpha, beta, mode, tn);
}

void chol_solve3_f32(const float *L, long long ld, long long mstride, int batch, const float *dinv, float *X,
                     float *W, long long xstride, cudaStream_t s) {
    trsv_blocked<float>(L, ld, mstride, batch, dinv, X, W, xstride, s);
}

}  // namespace

cudaError_t cholesky_f32_from_f64(const double *A64, float *A32, long long ld, int batch, float *dinv,
                                  uint32_t *panel, int *status, cudaStream_t s) {
    const long long mstride = ld * ld, dstride = (ld / T64) * 4096;
    count_launches(1);
    k_to_f32<<<gridn(mstride * batch), 256, 0, s>>>(A64, mstride * batch, A32);
    constexpr int kPanel = kScsPanel;
    const int first = static_cast<int>(ld % kPanel) ? static_cast<int>(ld % kPanel) : kPanel;
    for (long long p0 = 0; p0 < ld;) {
        const int pw = p0 == 0 ? first : kPanel;   // panel columns [p0, p0 + pw)
        for (long long s0 = p0; s0 < p0 + pw; s0 += kScsSub) {
            const long long s1 = std::min<long long>(s0 + kScsSub, p0 + pw);   // sub-panel columns [s0, s1)
            // right-looking 64-wide steps restricted to the sub-panel's columns
            for (long long k0 = s0; k0 < s1; k0 += T64) {
                const int k = static_cast<int>(k0 / T64);
                count_launches(1);
                k_spotrf_diag<<<batch, 256, 0, s>>>(A32 + k0 * ld + k0, ld, mstride, dinv + k * 4096LL, dstride,
                                                    status);
                const int rem = static_cast<int>(ld - k0 - T64);   // rows below the diagonal block
                if (rem <= 0) continue;
                float *A21 = A32 + (k0 + T64) * ld + k0;
                sgemm_nt(A21, dinv + k * 4096LL, A21, ld, 64, ld, mstride, dstride, mstride, rem, 64, 64, batch, 1.f,
                         0.f, 0, s);
                const int w = static_cast<int>(s1 - k0 - T64);   // sub-panel columns right of the block
                if (w > 0)
                    sgemm_nt(A21, A21, A21 + T64, ld, ld, ld, mstride, mstride, mstride, rem, w, 64, batch, -1.f, 1.f,
                             0, s);
            }
            // the panel's columns right of the sub-panel, A[s1:, s1:p0+pw) -= L[s1:, s0:s1) L[s1:p0+pw, s0:s1)^T,
            // on the tensor cores (TF32x3 parts; every tile of the block, whose part above the
            // diagonal the factorisation does not read)
            const int wr = static_cast<int>(p0 + pw - s1);
            if (wr > 0) {
                const long long r1 = ld - s1;
                const int sw = static_cast<int>(s1 - s0);
                uint32_t *HA = panel, *LA = panel + static_cast<long long>(batch) * r1 * sw;
                uint32_t *HB = LA + static_cast<long long>(batch) * r1 * sw, *LB = HB + static_cast<long long>(batch) * wr * sw;
                split_panel_tf32(A32 + s1 * ld + s0, ld, mstride, batch, r1, sw, HA, LA, s);
                split_panel_tf32(A32 + s1 * ld + s0, ld, mstride, batch, wr, sw, HB, LB, s);
                float *C = A32 + s1 * ld + s1;
                TcOperands op{HA, LA, HB, LB, sw, sw};
                TcArgs g{static_cast<int>(r1), wr, sw, -1.f, 1.f, C, ld, C, nullptr, nullptr, nullptr, nullptr, nullptr,
                         nullptr, 0, 0, status};
                g.chunk_stages = 8;
                g.batch = batch;
                g.sC = mstride;
                const cudaError_t e = tc_gemm(2, op, g, s);
                if (e != cudaSuccess) return e;
            }
        }
        const long long t0 = p0 + pw, rem = ld - t0;   // trailing matrix [t0, ld)^2
        if (rem > 0) {
            // A22 -= L21 L21^T with L21 = A[t0:, p0:t0] as TF32x3 parts on the tensor cores;
            // only the tiles of the lower triangle of A22 (the part the factorisation reads)
            uint32_t *H = panel, *L = panel + static_cast<long long>(batch) * rem * pw;
            split_panel_tf32(A32 + t0 * ld + p0, ld, mstride, batch, rem, pw, H, L, s);
            float *A22 = A32 + t0 * ld + t0;
            TcOperands op{H, L, H, L, pw, pw};
            TcArgs g{static_cast<int>(rem), static_cast<int>(rem), pw, -1.f, 1.f, A22, ld, A22, nullptr, nullptr,
                     nullptr, nullptr, nullptr, nullptr, 0, 1, status};
            g.chunk_stages = 8;   // 256 TF32 products per TMEM sum: the refinement absorbs the truncation
            g.batch = batch;
            g.sC = mstride;
            const cudaError_t e = tc_gemm(2, op, g, s);
            if (e != cudaSuccess) return e;
        }
        p0 += pw;
    }
    return cudaGetLastError();
}

void refine_solve3(const double *A64, const float *L32, const float *dinv, long long ld, int n, int batch,
                   const double *B, double *X, float *work, int steps, cudaStream_t s) {
    const long long xs = 3 * ld, total = xs * batch;
    float *work2 = work + total;   // intermediate of the triangular solves
    count_launches(1);
    k_rhs_to_f32<<<gridn(total), 256, 0, s>>>(B, total, work);
    chol_solve3_f32(L32, ld, ld * ld, batch, dinv, work, work2, xs, s);
    count_launches(1);
    k_accumulate<<<gridn(total), 256, 0, s>>>(X, work, total, 1);
    for (int it = 0; it < steps; ++it) {
        count_launches(1);
        k_residual3<<<dim3(static_cast<unsigned>((ld + 31) / 32), batch), 256, 0, s>>>(A64, ld, ld * ld, B, X, xs,
                                                                                      work, n);
        chol_solve3_f32(L32, ld, ld * ld, batch, dinv, work, work2, xs, s);
        count_launches(1);
        k_accumulate<<<gridn(total), 256, 0, s>>>(X, work, total, 0);
    }
}

}  // namespace mbdgb
