// Dense FP64 kernels for sm_103a: a 64x64-tile GEMM on the FP64 tensor path
// (mma.sync m8n8k4 f64), batched right-looking blocked Cholesky, batched triangular
// solves with three right-hand sides, and small matrix utilities.
//
// These carry the cubic stages of the method: the screening solves of Eq. (scs) (one
// factorisation per frequency point, Sec. 2.3) and the coupled Newton-Schulz iteration
// for Q^{1/2} and Q^{-1/2} behind Eqs. (diagonalization), (mbd-energy), (mbd-gradient).
#include <type_traits>

#include "internal.h"

namespace mbdgb {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, PK = BK + 4;  // smem row stride 20 doubles: conflict-free fragments
constexpr int PN = BN + 8;                             // NN operand row stride 72 doubles
static_assert(BK * PN <= BN * PK, "NN tile must fit the NT tile's storage");

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// D(8x8) += A(8x4, row) * B(4x8, col), FP64.  Fragments: a = A[lane/4][lane%4],
// b = B[lane%4][lane/4], {c0,c1} = C[lane/4][2(lane%4) + {0,1}].
__device__ __forceinline__ void dmma(double &c0, double &c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

// Triangular enumeration of tile pairs: bid -> (r, c), c <= r.
__device__ __forceinline__ void tri_index(int bid, int &r, int &c) {
    int x = static_cast<int>((sqrt(8.0 * bid + 1.0) - 1.0) * 0.5);
    while ((x + 1) * (x + 2) / 2 <= bid) ++x;
    while (x * (x + 1) / 2 > bid) --x;
    r = x;
    c = bid - x * (x + 1) / 2;
}

// TB: B is N x K (C = A B^T) when true, K x N (C = A B) when false.
template <bool TB>
__device__ __forceinline__ void gemm_tile(const GemmArgs &g, int tiles_n) {
    int tm, tn;
    if (g.mode == 0) {
        tm = blockIdx.x / tiles_n;
        tn = blockIdx.x % tiles_n;
    } else {
        int r, c;
        tri_index(blockIdx.x, r, c);
        if (g.mode == 1) { tm = r; tn = c; } else { tm = c; tn = r; }
    }
    const long long b = blockIdx.z;
    const double *A = g.A + b * g.sA + static_cast<long long>(tm) * BM * g.lda;
    const double *B = g.B + b * g.sB + (TB ? static_cast<long long>(tn) * BN * g.ldb
                                            : static_cast<long long>(tn) * BN);
    __shared__ __align__(16) double As[2][BM][PK];
    // NT: Bs[n][k] (row stride 20); NN: Bs[k][n] viewed with row stride 72 (also
    // conflict-free for the fragment pattern).  Same 40 KB either way.
    __shared__ __align__(16) double Bs_raw[2][BN * PK];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int fr = lane >> 2, fc = lane & 3;
    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    const int nk = g.K / BK;
    auto load = [&](int stage, int kt) {
        const int k0 = kt * BK;
#pragma unroll
        for (int i = 0; i < 4; ++i) {   // 64 rows x 8 chunks of 16 B per operand
            const int ch = tid + i * 128, row = ch >> 3, col = (ch & 7) * 2;
            cp_async16(&As[stage][row][col], A + static_cast<long long>(row) * g.lda + k0 + col);
            if (TB) {
                cp_async16(&Bs_raw[stage][row * PK + col], B + static_cast<long long>(row) * g.ldb + k0 + col);
            } else {   // 16 rows (k) x 32 chunks of 16 B
                const int kr = ch >> 5, nc = (ch & 31) * 2;
                cp_async16(&Bs_raw[stage][kr * PN + nc], B + static_cast<long long>(k0 + kr) * g.ldb + nc);
            }
        }
        cp_async_commit();
    };
    load(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < nk) {
            load(st ^ 1, kt + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 4) {
            double af[4], bf[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) af[i] = As[st][wm + i * 8 + fr][kk + fc];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                bf[j] = TB ? Bs_raw[st][(wn + j * 8 + fr) * PK + kk + fc]
                           : Bs_raw[st][(kk + fc) * PN + wn + j * 8 + fr];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) dmma(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
        }
        __syncthreads();
    }
    double *C = g.C + b * g.sC;
    const double *D = g.D ? g.D + b * g.sD : nullptr;
    // modes 2 and 3: upper tiles, mirrored into the lower half (mode 3 with a sign change,
    // for antisymmetric results such as the imaginary part of a Hermitian product)
    const bool mirror = (g.mode >= 2) && (tm != tn);
    const double msign = g.mode == 3 ? -1.0 : 1.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long m = static_cast<long long>(tm) * BM + wm + i * 8 + fr;
            const long long n = static_cast<long long>(tn) * BN + wn + j * 8 + 2 * fc;
            double v0 = g.alpha * acc[i][j][0], v1 = g.alpha * acc[i][j][1];
            if (g.beta != 0.0) {
                const double2 d = *reinterpret_cast<const double2 *>(D + m * g.ldd + n);
                v0 += g.beta * d.x;
                v1 += g.beta * d.y;
            }
            *reinterpret_cast<double2 *>(C + m * g.ldc + n) = make_double2(v0, v1);
            if (mirror) {
                C[n * g.ldc + m] = msign * v0;
                C[(n + 1) * g.ldc + m] = msign * v1;
            }
        }
}

__global__ void __launch_bounds__(128) k_gemm_nt(GemmArgs g, int tiles_n) { gemm_tile<true>(g, tiles_n); }
__global__ void __launch_bounds__(128) k_gemm_nn(GemmArgs g, int tiles_n) { gemm_tile<false>(g, tiles_n); }

// Unblocked Cholesky of the 64x64 diagonal block (lower part read), in shared memory,
// followed by the inverse of the triangular factor.  L^{-1} (lower) is kept in the
// strict upper triangle of S, transposed (L^{-1}[i][c] at S[c][i], i > c), with its
// diagonal in dg, so the kernel needs 33 KB of shared memory.
__global__ void __launch_bounds__(256) k_potrf_diag(double *A, long long ld, long long mstride,
                                                    double *dinv, long long dstride, int *status) {
    __shared__ double S[64][65];
    __shared__ double dg[64];
    __shared__ int bad;
    double *Ab = A + static_cast<long long>(blockIdx.x) * mstride;
    const int t = threadIdx.x;
    if (t == 0) bad = 0;
    for (int e = t; e < 4096; e += 256) {
        const int r = e >> 6, c = e & 63;
        S[r][c] = (c <= r) ? Ab[r * ld + c] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < 64; ++j) {
        if (t == 0) {
            double d = S[j][j];
            if (!(d > 0.0)) { bad = 1; d = 1.0; }
            S[j][j] = sqrt(d);
        }
        __syncthreads();
        const double djj = S[j][j];
        for (int i = j + 1 + t; i < 64; i += 256) S[i][j] /= djj;
        __syncthreads();
        const int m = 63 - j;
        for (int e = t; e < m * m; e += 256) {
            const int i = j + 1 + e / m, k = j + 1 + e % m;
            if (k <= i) S[i][k] -= S[i][j] * S[k][j];
        }
        __syncthreads();
    }
    if (t < 64) {   // column c of L^{-1} by forward substitution (thread c owns row c of S's upper part)
        const int c = t;
        for (int i = c; i < 64; ++i) {
            double acc = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) acc -= S[i][k] * (k == c ? dg[c] : S[c][k]);
            const double v = acc / S[i][i];
            if (i == c) dg[c] = v; else S[c][i] = v;
        }
    }
    __syncthreads();
    double *Db = dinv + static_cast<long long>(blockIdx.x) * dstride;
    for (int e = t; e < 4096; e += 256) {
        const int r = e >> 6, c = e & 63;
        if (c <= r) Ab[r * ld + c] = S[r][c];
        Db[e] = (c > r) ? 0.0 : (c == r ? dg[r] : S[c][r]);
    }
    if (t == 0 && bad) atomicOr(status, ST_SCS_NOT_PD);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void k_frob_dev_identity(const double *P, long long ld, int n, double *out) {
    double acc = 0.0;
    const long long total = static_cast<long long>(n) * n;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / n, j = e % n;
        const double d = (i == j ? 1.0 : 0.0) - P[i * ld + j];
        acc += d * d;
    }
    acc = warp_sum(acc);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) atomicAdd(out, v);
    }
}

__global__ void k_scale(double *Y, long long total, double scale) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        Y[e] *= scale;
}

__global__ void k_identity(double *Z, long long ld) {
    const long long total = ld * ld;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        Z[e] = (e / ld == e % ld) ? 1.0 : 0.0;
}

// Positive doubles order like their bit patterns, so atomicMax on the bits is a max.
__global__ void k_max_abs_rowsum(const double *Q, long long ld, int n, unsigned long long *out) {
    const int row = blockIdx.x;
    double acc = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) acc += fabs(Q[static_cast<long long>(row) * ld + j]);
    acc = warp_sum(acc);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(v)));
    }
}

// ---- Lanczos estimates of the extreme eigenvalues of a symmetric matrix ----
// y = A x for an ld x ld row-major A: one warp per row, coalesced row reads.  T = double,
// or float for an FP32 copy of A with an FP32 copy of x (products and row sums in FP32).
template <typename T>
__global__ void k_gemv(const T *A, long long ld, const T *x, double *y) {
    const long long row = blockIdx.x * static_cast<long long>(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= ld) return;
    const T *a = A + row * ld;
    T acc = 0;
    for (long long c = lane; c < ld; c += 32) acc += a[c] * x[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[row] = static_cast<double>(acc);
}

__global__ void k_f64_to_f32(const double *A, long long total, float *B) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        B[e] = static_cast<float>(A[e]);
}

__device__ double block_sum1024(double v, double *sh) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = (threadIdx.x < 32) ? sh[threadIdx.x] : 0.0;
    if (threadIdx.x < 32) t = warp_sum(t);
    __syncthreads();
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

// v = a fixed pseudo-random unit vector, vprev = 0; v32 (if given) = (float) v.
__global__ void __launch_bounds__(1024) k_lanczos_init(double *v, double *vprev, float *v32, long long ld) {
    __shared__ double sh[32];
    double ss = 0.0;
    for (long long p = threadIdx.x; p < ld; p += 1024) {
        const double x = sin(0.7548776662 * static_cast<double>(p) + 0.5698402910) + 0.25;
        v[p] = x;
        vprev[p] = 0.0;
        ss += x * x;
    }
    const double nrm = sqrt(block_sum1024(ss, sh));
    for (long long p = threadIdx.x; p < ld; p += 1024) {
        v[p] /= nrm;
        if (v32) v32[p] = static_cast<float>(v[p]);
    }
}

// One Lanczos step after w = A v: alpha = w.v; w -= alpha v + beta_prev vprev;
// beta = |w|; vprev = v; v = w / beta (and v32 = (float) v if given).  coef[2j] = alpha,
// coef[2j+1] = beta.
__global__ void __launch_bounds__(1024) k_lanczos_update(double *w, double *v, double *vprev, float *v32, long long ld,
                                                         double *coef, int j) {
    __shared__ double sh[32];
    double d = 0.0;
    for (long long p = threadIdx.x; p < ld; p += 1024) d += w[p] * v[p];
    const double alpha = block_sum1024(d, sh);
    const double bprev = j > 0 ? coef[2 * j - 1] : 0.0;
    double ss = 0.0;
    for (long long p = threadIdx.x; p < ld; p += 1024) {
        const double x = w[p] - alpha * v[p] - bprev * vprev[p];
        w[p] = x;
        ss += x * x;
    }
    const double beta = sqrt(block_sum1024(ss, sh));
    const double inv = beta > 1e-300 ? 1.0 / beta : 0.0;
    for (long long p = threadIdx.x; p < ld; p += 1024) {
        vprev[p] = v[p];
        v[p] = w[p] * inv;
        if (v32) v32[p] = static_cast<float>(v[p]);
    }
    if (threadIdx.x == 0) {
        coef[2 * j] = alpha;
        coef[2 * j + 1] = beta;
    }
}

}  // namespace

// work: 3 ld doubles (v, vprev, w), then for T = float ld floats (the FP32 copy of v).
template <typename T>
void lanczos_run(const T *A, long long ld, int steps, double *work, double *coef, cudaStream_t s) {
    double *v = work, *vprev = work + ld, *w = work + 2 * ld;
    float *v32 = std::is_same<T, float>::value ? reinterpret_cast<float *>(work + 3 * ld) : nullptr;
    const T *x = std::is_same<T, float>::value ? reinterpret_cast<const T *>(v32) : reinterpret_cast<const T *>(v);
    count_launches(1);
    k_lanczos_init<<<1, 1024, 0, s>>>(v, vprev, v32, ld);
    for (int j = 0; j < steps; ++j) {
        count_launches(2);
        k_gemv<T><<<static_cast<int>((ld + 7) / 8), 256, 0, s>>>(A, ld, x, w);
        k_lanczos_update<<<1, 1024, 0, s>>>(w, v, vprev, v32, ld, coef, j);
    }
}

void lanczos_coefficients(const double *A, long long ld, int steps, double *work, double *coef, cudaStream_t s) {
    lanczos_run<double>(A, ld, steps, work, coef, s);
}

void lanczos_coefficients_f32(const double *A, float *A32, long long ld, int steps, double *work, double *coef,
                              cudaStream_t s) {
    count_launches(1);
    k_f64_to_f32<<<static_cast<int>(std::min<long long>((ld * ld + 255) / 256, 152 * 16)), 256, 0, s>>>(A, ld * ld,
                                                                                                      A32);
    lanczos_run<float>(A32, ld, steps, work, coef, s);
}

void gemm_f64(const GemmArgs &g, cudaStream_t s) {
    const int tm = g.M / BM, tn = g.N / BN;
    dim3 grid;
    if (g.mode == 0) grid = dim3(tm * tn, 1, g.batch);
    else grid = dim3(tm * (tm + 1) / 2, 1, g.batch);   // square M == N for triangular modes
    if (g.trans_b) {
        count_launches(1);
        k_gemm_nt<<<grid, 128, 0, s>>>(g, tn);
    }
    else {
        count_launches(1);
        k_gemm_nn<<<grid, 128, 0, s>>>(g, tn);
    }
}

__global__ void k_axpby_identity(double *Z, const double *P, long long ld, double a, double b) {
    const long long total = ld * ld;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        Z[e] = (e / ld == e % ld ? a : 0.0) + b * P[e];
}

void axpby_identity(double *Z, const double *P, long long ld, double a, double b, cudaStream_t s) {
    count_launches(1);
    k_axpby_identity<<<1216, 256, 0, s>>>(Z, P, ld, a, b);
}

void cholesky_f64(double *A, long long ld, long long mstride, int batch, double *dinv, int *status,
                  cudaStream_t s) {
    const int nb = static_cast<int>(ld / kTile);
    for (int k = 0; k < nb; ++k) {
        const long long k0 = static_cast<long long>(k) * kTile;
        count_launches(1);
        k_potrf_diag<<<batch, 256, 0, s>>>(A + k0 * ld + k0, ld, mstride, dinv + k * 4096LL,
                                           static_cast<long long>(nb) * 4096, status);
        const int rem = static_cast<int>(ld - k0 - kTile);
        if (rem <= 0) continue;
        double *A21 = A + (k0 + kTile) * ld + k0;
        double *A22 = A + (k0 + kTile) * ld + k0 + kTile;
        GemmArgs t{A21, dinv + k * 4096LL, nullptr, A21, ld, 64, 0, ld,
                   mstride, static_cast<long long>(nb) * 4096, 0, mstride,
                   rem, 64, 64, batch, 1.0, 0.0, 0, 1};
        gemm_f64(t, s);
        GemmArgs y{A21, A21, A22, A22, ld, ld, ld, ld, mstride, mstride, mstride, mstride,
                   rem, rem, 64, batch, -1.0, 1.0, 1, 1};
        gemm_f64(y, s);
    }
}

void chol_solve3_f64(const double *L, long long ld, long long mstride, int batch, const double *dinv,
                     double *X, double *work, long long xstride, cudaStream_t s) {
    trsv_blocked<double>(L, ld, mstride, batch, dinv, X, work, xstride, s);
}

void frob_dev_identity(const double *P, long long ld, int n, double *out, cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(double), s);
    count_launches(1);
    k_frob_dev_identity<<<608, 256, 0, s>>>(P, ld, n, out);
}

void scale_matrix(double *Y, long long ld, double scale, cudaStream_t s) {
    count_launches(1);
    k_scale<<<1216, 256, 0, s>>>(Y, ld * ld, scale);
}

void set_identity(double *Z, long long ld, cudaStream_t s) {
    count_launches(1);
    k_identity<<<1216, 256, 0, s>>>(Z, ld);
}

void max_abs_rowsum(const double *Q, long long ld, int n, double *out, cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(double), s);
    count_launches(1);
    k_max_abs_rowsum<<<n, 256, 0, s>>>(Q, ld, n, reinterpret_cast<unsigned long long *>(out));
}

}  // namespace mbdgb
