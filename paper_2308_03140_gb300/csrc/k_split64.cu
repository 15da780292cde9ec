// FP64-accurate GEMM on the tcgen05 TF32 tensor path by error-free splitting (sm_103a):
//
//   C = alpha A op(B) + beta D,   A M x K, op(B) K x N, all FP64,
//
// with the operands cut into split64::kSlices slices of kSliceBits bits each (split64.cuh:
// A by rows, op(B) by columns, each row or column scaled by a power of two), the slice
// products of weight p + q <= kSlices taken by k_tc_gemm (kind 0, TF32 operands that hold
// the slices exactly) over K in pieces of at most kSplitChunk, where every partial sum is
// exact in FP32, and each piece added into C in FP64 by the GEMM's FP64 output.
//
//  k_row_exponents   per row of a row-major matrix: the exponent that scales it below 1
//  k_col_exponents   the same per column
//  k_row_slices      slices of the rows of A (or of B^T given as N x K): S[p][r][c]
//  k_col_slices      slices of B^T from B (K x N) through 32 x 32 shared-memory tiles
//  k_axpby64         C = alpha C + beta D (the final scaling)
//
// Per product: 53 slice products x ceil(K/1024) launches of an M x N x <=1024 TF32 GEMM,
// and (M + N) K x 9 FP32 slices of workspace.
#include <algorithm>

#include "split64.cuh"

namespace mbdgb {
namespace {

using split64::kSlices;
using split64::kSliceBits;

__global__ void k_row_exponents(const double *A, long long lda, int rows, int cols, int *e) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= rows) return;
    double m = 0.0;
    for (int c = lane; c < cols; c += 32) m = fmax(m, fabs(A[r * lda + c]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) e[r] = split64::scale_exponent(m);
}

__global__ void k_col_exponents(const double *B, long long ldb, int rows, int cols, int *e) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double m = 0.0;
    for (int r = 0; r < rows; ++r) m = fmax(m, fabs(B[r * ldb + c]));
    e[c] = split64::scale_exponent(m);
}

// S[p][r][c] (slice stride rows * cols, row pitch cols) for a row-major rows x cols source.
__global__ void k_row_slices(const double *A, long long lda, int rows, int cols, const int *e, float *S) {
    const long long total = static_cast<long long>(rows) * cols, stride = total;
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long r = t / cols, c = t - r * cols;
        float sl[kSlices];
        split64::slice(A[r * lda + c], e[r], sl);
#pragma unroll
        for (int p = 0; p < kSlices; ++p) S[p * stride + t] = sl[p];
    }
}

// Slices of B^T (N x K, row pitch K) from B (K x N, pitch ldb) with column exponents f:
// 32 x 32 tiles read along rows of B and written along rows of B^T.
__global__ void k_col_slices(const double *B, long long ldb, int K, int N, const int *f, float *S) {
    __shared__ double t[32][33];
    const int k0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int kk = k0 + k, jj = j0 + threadIdx.x;
        t[k][threadIdx.x] = (kk < K && jj < N) ? B[static_cast<long long>(kk) * ldb + jj] : 0.0;
    }
    __syncthreads();
    const long long stride = static_cast<long long>(N) * K;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int jj = j0 + j, kk = k0 + threadIdx.x;
        if (jj >= N || kk >= K) continue;
        float sl[kSlices];
        split64::slice(t[threadIdx.x][j], f[jj], sl);
        const long long o = static_cast<long long>(jj) * K + kk;
#pragma unroll
        for (int p = 0; p < kSlices; ++p) S[p * stride + o] = sl[p];
    }
}

__global__ void k_axpby64(double *C, long long ldc, int M, int N, double alpha, double beta, const double *D,
                          long long ldd) {
    const long long total = static_cast<long long>(M) * N;
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long r = t / N, c = t - r * N;
        const double d = beta != 0.0 ? beta * D[r * ldd + c] : 0.0;
        C[r * ldc + c] = alpha * C[r * ldc + c] + d;
    }
}

inline int cdiv(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }
inline int grid_for(long long n) { return static_cast<int>(std::min<long long>(cdiv(n, 256), 152LL * 16)); }

}  // namespace

size_t gemm_f64_split_work_bytes(int M, int N, int K) {
    return sizeof(float) * static_cast<size_t>(kSlices) * (static_cast<size_t>(M) + N) * K +
           sizeof(int) * (static_cast<size_t>(M) + N);
}

cudaError_t gemm_f64_split(int trans_b, int mode, int M, int N, int K, double alpha, const double *A, long long lda,
                           const double *B, long long ldb, double beta, const double *D, long long ldd, double *C,
                           long long ldc, void *work, int *err, cudaStream_t s) {
    if ((mode != 0 && mode != 2) || (mode == 2 && M != N)) return cudaErrorInvalidValue;
    float *SA = static_cast<float *>(work);
    float *SB = SA + static_cast<size_t>(kSlices) * M * K;
    int *eA = reinterpret_cast<int *>(SB + static_cast<size_t>(kSlices) * N * K);
    int *eB = eA + M;
    cudaError_t e = cudaSuccess;
    // C prepared for accumulation: zero, or beta/alpha D when D is C itself
    if (alpha == 0.0) {
        count_launches(1);
        k_axpby64<<<grid_for(static_cast<long long>(M) * N), 256, 0, s>>>(C, ldc, M, N, 0.0, beta, D, ldd);
        return cudaGetLastError();
    }
    const bool in_place = beta != 0.0 && D == C;
    if (in_place) {
        count_launches(1);
        k_axpby64<<<grid_for(static_cast<long long>(M) * N), 256, 0, s>>>(C, ldc, M, N, beta / alpha, 0.0, nullptr, 0);
    } else {
        e = cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * N, M, s);
        if (e != cudaSuccess) return e;
    }
    count_launches(4);
    k_row_exponents<<<cdiv(M, 8), 256, 0, s>>>(A, lda, M, K, eA);
    k_row_slices<<<grid_for(static_cast<long long>(M) * K), 256, 0, s>>>(A, lda, M, K, eA, SA);
    if (trans_b) {   // op(B) = B^T with B N x K: its rows are the columns of op(B)
        k_row_exponents<<<cdiv(N, 8), 256, 0, s>>>(B, ldb, N, K, eB);
        k_row_slices<<<grid_for(static_cast<long long>(N) * K), 256, 0, s>>>(B, ldb, N, K, eB, SB);
    } else {
        k_col_exponents<<<cdiv(N, 128), 128, 0, s>>>(B, ldb, K, N, eB);
        k_col_slices<<<dim3(cdiv(N, 32), cdiv(K, 32)), dim3(32, 8), 0, s>>>(B, ldb, K, N, eB, SB);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t sa = static_cast<size_t>(M) * K, sb = static_cast<size_t>(N) * K;
    for (int p = 0; p < kSlices; ++p)
        for (int q = 0; q < kSlices && p + q <= kSlices; ++q)
            for (int k0 = 0; k0 < K; k0 += split64::kSplitChunk) {
                const int kc = std::min(split64::kSplitChunk, K - k0);
                TcOperands op{SA + p * sa + k0, nullptr, SB + q * sb + k0, nullptr, K, K};
                TcArgs g{M, N, kc, 1.f, 0.f, nullptr, ldc, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                         nullptr, 0, mode, err};
                g.C64 = C;
                e = tc_gemm(0, op, g, s);
                if (e != cudaSuccess) return e;
            }
    if (in_place || alpha != 1.0 || beta != 0.0) {
        count_launches(1);
        k_axpby64<<<grid_for(static_cast<long long>(M) * N), 256, 0, s>>>(C, ldc, M, N, alpha, in_place ? 0.0 : beta,
                                                                          D, ldd);
    }
    return cudaGetLastError();
}

}  // namespace mbdgb
