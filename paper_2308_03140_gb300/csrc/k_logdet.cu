// MBD energy by the imaginary-frequency log formula, Eq. (log-formula), and its many-body
// orders, Eq. (rpa), for the (screened) oscillators of an evaluation:
//
//   E     = 1/(2 pi) sum_k w_k ln det(I + A_k),  A_k = alpha(u_k)^{1/2} T^lr alpha(u_k)^{1/2},
//   E^(m) = -1/(2 pi) sum_k w_k (-1)^m/m Tr A_k^m,
//
// alpha_i(u) = alpha_bar0_i / (1 + u^2/omega_bar_i^2), T^lr_ij = g_ij T(R_j - R_i) as in Q
// (zero diagonal blocks), on the frequency nodes u_k > 0 of the screening grid.  ln det
// comes from FP64 Cholesky factors (2 sum ln L_ii); Tr A^2 = |A|_F^2, Tr A^3 = <A^2, A>,
// Tr A^4 = |A^2|_F^2.
//
// Layout: nf matrices of ld x ld doubles, mstride apart; rows and columns >= 3N are zero in
// A and identity in I + A (they add ln 1 = 0).
#include "pair_math.cuh"

namespace mbdgb {
namespace {

using pairs::fermi;

// Thread (i, j), j <= i: block (i, j) of every A_k and its mirror (j, i).
__global__ void k_build_lr_freq(AtomBufs b, double beta, double a, double *A, long long ld, long long mstride,
                                int nf, int *status) {
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    if (i >= b.N || j > i) return;
    if (i == j) return;   // zero diagonal blocks (the batch is cleared first)
    const double r[3] = {b.R[3 * j] - b.R[3 * i], b.R[3 * j + 1] - b.R[3 * i + 1], b.R[3 * j + 2] - b.R[3 * i + 2]};
    const double rho2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], rho = sqrt(rho2);
    if (!(rho > 1e-8)) atomicOr(status, ST_INPUT);
    const double g = fermi(rho, b.rbar[i] + b.rbar[j], beta, a).f;
    const double ir3 = 1.0 / (rho2 * rho), ir5 = ir3 / rho2;
    double T[9];
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) T[3 * x + y] = g * ((x == y ? ir3 : 0.0) - 3.0 * r[x] * r[y] * ir5);
    const double wi = b.ombar[i], wj = b.ombar[j];
    for (int k = 0; k < nf; ++k) {
        const double u = b.u[k + 1];
        const double ai = b.abar0[i] / (1.0 + u * u / (wi * wi)), aj = b.abar0[j] / (1.0 + u * u / (wj * wj));
        const double pre = sqrt(ai * aj);
        double *Ak = A + k * mstride;
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) {
                Ak[(3LL * i + x) * ld + 3 * j + y] = pre * T[3 * x + y];
                Ak[(3LL * j + x) * ld + 3 * i + y] = pre * T[3 * y + x];
            }
    }
}

// out[b] += sum_e X[b][e] * Y[b][e] over `per` elements (X == Y: sum of squares); FP64
// block sums combined by atomics.
__global__ void __launch_bounds__(256) k_batch_dot(const double *X, const double *Y, long long per,
                                                   long long stride, double *out) {
    __shared__ double sh[8];
    const double *x = X + blockIdx.y * stride, *y = Y + blockIdx.y * stride;
    double acc = 0.0;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < per; e += 256LL * gridDim.x) acc += x[e] * y[e];
    acc = pairs::warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        atomicAdd(out + blockIdx.y, t);
    }
}

// Diagonal of every matrix += 1 (I + A).
__global__ void k_add_identity_batch(double *A, long long ld, long long mstride) {
    double *Ab = A + blockIdx.y * mstride;
    for (long long p = blockIdx.x * 256LL + threadIdx.x; p < ld; p += 256LL * gridDim.x) Ab[p * ld + p] += 1.0;
}

// out[b] = sum_p ln L_pp of the Cholesky factor of matrix b (one CTA per matrix).
__global__ void __launch_bounds__(256) k_logdiag_batch(const double *L, long long ld, long long mstride, double *out,
                                                       int *status) {
    __shared__ double sh[8];
    const double *Lb = L + blockIdx.x * mstride;
    double acc = 0.0;
    for (long long p = threadIdx.x; p < ld; p += 256) {
        const double d = Lb[p * ld + p];
        if (!(d > 0.0)) atomicOr(status, ST_SCS_NOT_PD);
        acc += log(d);
    }
    acc = pairs::warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        out[blockIdx.x] = t;
    }
}

inline int cdiv(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

}  // namespace

cudaError_t build_lr_freq(const AtomBufs &b, double beta, double a, double *A, long long ld, long long mstride,
                          int nf, int *status, cudaStream_t s) {
    const cudaError_t e = cudaMemsetAsync(A, 0, sizeof(double) * mstride * nf, s);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_build_lr_freq<<<dim3(cdiv(b.N, 32), cdiv(b.N, 8)), dim3(32, 8), 0, s>>>(b, beta, a, A, ld, mstride, nf, status);
    return cudaGetLastError();
}

cudaError_t batch_dot(const double *X, const double *Y, long long per, long long stride, int batch, double *out,
                      cudaStream_t s) {
    const cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * batch, s);
    if (e != cudaSuccess) return e;
    const int blocks = static_cast<int>(std::min<long long>(cdiv(per, 256), 1216));
    count_launches(1);
    k_batch_dot<<<dim3(blocks, batch), 256, 0, s>>>(X, Y, per, stride, out);
    return cudaGetLastError();
}

void add_identity_batch(double *A, long long ld, long long mstride, int batch, cudaStream_t s) {
    count_launches(1);
    k_add_identity_batch<<<dim3(cdiv(ld, 256), batch), 256, 0, s>>>(A, ld, mstride);
}

void logdiag_batch(const double *L, long long ld, long long mstride, int batch, double *out, int *status,
                   cudaStream_t s) {
    count_launches(1);
    k_logdiag_batch<<<batch, 256, 0, s>>>(L, ld, mstride, out, status);
}

}  // namespace mbdgb
