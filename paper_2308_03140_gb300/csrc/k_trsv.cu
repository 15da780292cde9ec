// Batched triangular solves with 3 right-hand sides for the screening systems of
// Eq. (scs): L y = b, then L^T x = y, with L from the blocked Cholesky factorisations
// (FP64 or FP32) and the inverses of its 64x64 diagonal blocks.
//
// Block-column form, one launch per diagonal block I and direction: every CTA first
// solves the 64x3 diagonal-block system from the already final right-hand side rows
// of block I (a 64x64 triangular product with the stored inverse), then subtracts the
// block's contribution from its own slice of the rows still to be solved.  Launches on
// one stream serialise the blocks; within a launch the work spreads over
// (remaining rows / 64) CTAs per matrix, with coalesced reads of L.
//
// Forward:  y_I = D_I^{-1} b_I;  b_J -= L_JI y_I  (J > I; CTA slice = 64 rows of L, four
//           threads per row),
//           b (the caller's array) is the running right-hand side, y goes to work.
// Backward: x_I = D_I^{-T} y_I;  y_J -= L_IJ^T x_I (J < I; CTA slice = 64 columns),
//           work is the running right-hand side, x goes to the caller's array.
// No launch both reads and writes one block of one array: block I is read, blocks
// J != I of the same array updated, and block I of the other array written.
#include "internal.h"

namespace mbdgb {
namespace {

// x (64x3, shared) = D^{-1} b_I (forward) or D^{-T} b_I (backward).  The 64x64 inverse is
// first staged into shared memory with coalesced loads (all in flight at once), so the
// triangular products read on-chip memory instead of chaining 64 dependent global loads.
template <typename T, bool BWD>
__device__ void diag_solve(const T *Di, const T *bI, T (*D)[65], T (*s)[3], T (*x)[3]) {
    const int t = threadIdx.x;
    for (int e = t; e < 64 * 64; e += blockDim.x) D[e >> 6][e & 63] = Di[e];
    if (t < 192) s[t / 3][t % 3] = bI[t];
    __syncthreads();
    if (t < 192) {
        const int r = t / 3, c = t % 3;
        T v = 0;
        if (!BWD)
            for (int k = 0; k <= r; ++k) v += D[r][k] * s[k][c];
        else
            for (int k = r; k < 64; ++k) v += D[k][r] * s[k][c];
        x[r][c] = v;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_trsv_fwd_block(const T *L, long long ld, long long mstride, const T *dinv,
                                                        long long dstride, T *X, T *W, long long xstride, int I) {
    const long long b = blockIdx.y;
    const T *Lb = L + b * mstride;
    T *Xb = X + b * xstride, *Wb = W + b * xstride;
    __shared__ T D[64][65], s[64][3], x[64][3];
    const long long I0 = static_cast<long long>(I) * 64;
    diag_solve<T, false>(dinv + b * dstride + static_cast<long long>(I) * 4096, Xb + 3 * I0, D, s, x);
    // rows of this CTA: 64 rows starting after block I; four threads per row, each taking
    // 16 consecutive columns of the block, combined by two shuffles
    const long long r0 = I0 + 64 + static_cast<long long>(blockIdx.x) * 64;
    if (r0 < ld) {
        const int rr = threadIdx.x >> 2, q = threadIdx.x & 3;
        const T *Lq = Lb + (r0 + rr) * ld + I0 + 16 * q;
        T l[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) l[c] = Lq[c];
        T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            a0 += l[c] * x[16 * q + c][0];
            a1 += l[c] * x[16 * q + c][1];
            a2 += l[c] * x[16 * q + c][2];
        }
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (q == 0) {
            T *xq = Xb + 3 * (r0 + rr);
            xq[0] -= a0;
            xq[1] -= a1;
            xq[2] -= a2;
        }
    }
    // every CTA computed the same y_I; CTA 0 stores it
    if (blockIdx.x == 0 && threadIdx.x < 192) Wb[3 * I0 + threadIdx.x] = x[threadIdx.x / 3][threadIdx.x % 3];
}

template <typename T>
__global__ void __launch_bounds__(256) k_trsv_bwd_block(const T *L, long long ld, long long mstride, const T *dinv,
                                                        long long dstride, T *X, T *W, long long xstride, int I) {
    const long long b = blockIdx.y;
    const T *Lb = L + b * mstride;
    T *Xb = X + b * xstride, *Wb = W + b * xstride;
    __shared__ T D[64][65], s[64][3], x[64][3];
    __shared__ T part[4][64][3];
    const long long I0 = static_cast<long long>(I) * 64;
    diag_solve<T, true>(dinv + b * dstride + static_cast<long long>(I) * 4096, Wb + 3 * I0, D, s, x);
    // columns of this CTA: 64 columns j < I0
    const long long c0 = static_cast<long long>(blockIdx.x) * 64;
    const int t = threadIdx.x, col = t & 63, grp = t >> 6;
    if (c0 < I0) {
        T l[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) l[k] = Lb[(I0 + grp + 4 * k) * ld + c0 + col];   // rows of block I
        T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int i = grp + 4 * k;
            a0 += l[k] * x[i][0];
            a1 += l[k] * x[i][1];
            a2 += l[k] * x[i][2];
        }
        part[grp][col][0] = a0; part[grp][col][1] = a1; part[grp][col][2] = a2;
    }
    __syncthreads();
    if (c0 < I0 && t < 192) {
        const int cc = t / 3, k = t % 3;
        Wb[3 * (c0 + cc) + k] -= part[0][cc][k] + part[1][cc][k] + part[2][cc][k] + part[3][cc][k];
    }
    if (blockIdx.x == 0 && t < 192) Xb[3 * I0 + t] = x[t / 3][t % 3];
}

}  // namespace

template <typename T>
void trsv_blocked(const T *L, long long ld, long long mstride, int batch, const T *dinv, T *X, T *W, long long xstride,
                  cudaStream_t s) {
    const int nb = static_cast<int>(ld / 64);
    const long long dstride = static_cast<long long>(nb) * 4096;
    for (int I = 0; I < nb; ++I) {
        const int rows = nb - 1 - I;   // 64-row slices below block I
        count_launches(1);
        k_trsv_fwd_block<T><<<dim3(rows > 0 ? rows : 1, batch), 256, 0, s>>>(L, ld, mstride, dinv, dstride, X, W,
                                                                           xstride, I);
    }
    for (int I = nb - 1; I >= 0; --I) {
        const int cols = I;            // 64-column slices left of block I
        count_launches(1);
        k_trsv_bwd_block<T><<<dim3(cols > 0 ? cols : 1, batch), 256, 0, s>>>(L, ld, mstride, dinv, dstride, X, W,
                                                                           xstride, I);
    }
}

template void trsv_blocked<double>(const double *, long long, long long, int, const double *, double *, double *,
                                   long long, cudaStream_t);
template void trsv_blocked<float>(const float *, long long, long long, int, const float *, float *, float *,
                                  long long, cudaStream_t);

}  // namespace mbdgb
