/*
 * mbd_gb300_kernels.h -- kernel-level C ABI of libmbdgb: the dense FP64 building blocks
 * behind the screening solves of Eq. (scs) (one Cholesky factorisation per frequency
 * point, Sec. 2.3) and the coupled Newton-Schulz iteration for Q^{1/2}, Q^{-1/2}
 * (Eqs. diagonalization, mbd-energy, mbd-gradient).  They stand where the paper's
 * implementation calls LAPACK/ScaLAPACK (Sec. 3.1).
 *
 * All matrix pointers are DEVICE pointers (FP64, row-major) on the current CUDA device;
 * `stream` is a cudaStream_t (NULL: legacy default stream).  Calls are asynchronous on
 * that stream; errors of the launch itself are returned (MBD_ERR_CUDA), numerical
 * failures are written to the device status word.  Dimensions must be positive
 * multiples of 64 (MBD_ERR_INPUT otherwise).  Buffers belong to the caller.
 */
#ifndef MBD_GB300_KERNELS_H
#define MBD_GB300_KERNELS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* C = alpha * A * op(B) + beta * D on the FP64 tensor path (mma.sync m8n8k4 f64).
 * A is M x K (lda).  trans_b = 1: op(B) = B^T with B N x K; trans_b = 0: op(B) = B
 * with B K x N (ldb).  C and D are M x N (ldc, ldd).  D may be NULL when beta == 0 and
 * may alias C.  mode 0 computes every 64x64 tile; mode 1 only tiles on or below the
 * diagonal (M == N); mode 2 only tiles on or above it and mirrors them into the lower
 * half (M == N, for products that are symmetric); mode 3 as mode 2 with the mirrored
 * entries negated (antisymmetric results).  Leading dimensions must be even
 * (16-byte aligned rows).  The matrices must not overlap C except D == C. */
int mbdk_gemm_f64(void *stream, int trans_b, int mode, int M, int N, int K, double alpha,
                  const double *A, long long lda, const double *B, long long ldb, double beta,
                  const double *D, long long ldd, double *C, long long ldc);

/* In-place lower Cholesky factorisation of `batch` matrices of order ld (consecutive,
 * stride ld*ld).  Reads the lower triangle only.  dinv receives the inverses of the
 * 64x64 diagonal blocks of each factor: batch * (ld/64) * 4096 doubles.  status (device
 * int) gets bit 2 set on a non-positive pivot; it is not cleared by the call. */
int mbdk_cholesky_f64(void *stream, double *A, long long ld, int batch, double *dinv, int *status);

/* Solves A X = B in place for 3 right-hand sides per matrix, X [batch][ld][3], with the
 * factors and diagonal-block inverses from mbdk_cholesky_f64.  work: caller-owned
 * device buffer of the same size as X (the intermediate L^{-1} B), not aliasing X. */
int mbdk_chol_solve3_f64(void *stream, const double *L, long long ld, int batch, const double *dinv,
                         double *X, double *work);

/* C = alpha * sum_p A_p B_p^T + beta * D on the 5th-generation tensor cores (tcgen05,
 * TMA-staged operands, FP32 accumulation in tensor memory) -- the products of the
 * mixed-precision Newton-Schulz iteration.  kind 0 (TF32): A0 = A and B0 = B are FP32,
 * A1/B1 ignored.  kind 1 (BF16x3): A0/A1 = bf16 hi/lo parts of A (A = A0 + A1), likewise
 * B; the three products A0 B0 + A0 B1 + A1 B0 are accumulated.  kind 2 (TF32x3): as kind
 * 1 with 32-bit parts (A0 = TF32-rounded A, A1 = FP32 remainder).  A is M x K (lda), B is
 * N x K (ldb); D (FP32, may be NULL when beta == 0), C (FP32, may be NULL), C_hi/C_lo
 * (split of the result in the kind's part format, kinds 1 and 2, may be NULL) and CT (FP32 transpose of the result, mode 0
 * and M == N only, may be NULL) share the leading dimension ldc.  M and N multiples of 128, K of 64,
 * leading dimensions multiples of 8.  mode 0: all tiles; mode 1: tiles on or below the
 * diagonal only, not mirrored (M == N); mode 2: upper tiles mirrored (M == N, symmetric
 * results).  chunk_stages: K stages (32 TF32 / 64 bf16 elements) per
 * tensor-memory accumulation, partial sums added in FP32 with round-to-nearest (0: all of
 * K in one accumulation).  err (device int) gets bit 8 set if a wait timed out. */
int mbdk_gemm_tc(void *stream, int kind, int mode, int M, int N, int K, float alpha, const void *A0,
                 const void *A1, long long lda, const void *B0, const void *B1, long long ldb, float beta,
                 const float *D, float *C, void *C_hi, void *C_lo, float *CT, long long ldc, int chunk_stages,
                 int *err);

/* Runs the tensor-core GEMM's bounded wait (the budget every wait of mbdk_gemm_tc and of the
 * mixed-precision evaluation has, about 2 s there) on an mbarrier that nothing arrives at,
 * with a budget of spin_cycles SM clock cycles (1 .. 2^32): the wait gives up and sets bit 8
 * (the timeout bit) in the device int *err, which the caller reads after synchronising.  It
 * tests the timeout path without a fault or a hang.  MBD_ERR_INPUT for a budget out of range
 * or a NULL err. */
int mbdk_tc_wait_check(void *stream, long long spin_cycles, int *err);

/* C = alpha * A * op(B) + beta * D, FP64-accurate, on the TF32 tensor path by error-free
 * splitting (the paper has none: its FP64 products run on CPUs; this serves GB300, whose FP64
 * rate is a small fraction of its tensor rate).  A is M x K (lda); trans_b = 1: op(B) = B^T
 * with B N x K; trans_b = 0: op(B) = B with B K x N (ldb); C and D are M x N (ldc, ldd), D
 * may be NULL when beta == 0 and may be C itself.  Each row of A and each column of op(B) is
 * scaled by a power of two and cut into 9 slices of 6 bits, stored exactly as FP32; the 53
 * slice products of weight p + q <= 9 run as TF32 tensor-core GEMMs over K in pieces of at
 * most 1024, where every partial sum is an integer below 2^22 times a power of two and so
 * exact in FP32, and each piece is added into C in FP64.  The result carries the rounding
 * of those FP64 additions and a truncation below 2^-54 of each operand row or column's
 * largest entry (as an FP64 product's own rounding); rows and columns whose largest
 * entries' product is below 2^-60 lose low slices to FP32 underflow.  M and N multiples of
 * 128, K of 64, ldc of 8.  work: device buffer of mbdk_gemm_f64_split_work_bytes(M, N, K)
 * bytes (9 (M + N) K floats and M + N ints).  err as in mbdk_gemm_tc. */
size_t mbdk_gemm_f64_split_work_bytes(int M, int N, int K);
int mbdk_gemm_f64_split(void *stream, int trans_b, int M, int N, int K, double alpha, const double *A,
                        long long lda, const double *B, long long ldb, double beta, const double *D, long long ldd,
                        double *C, long long ldc, void *work, int *err);

/* Allocation-free factor-and-solve (the paper has no counterpart; this serves callers
 * that cannot let a library allocate device memory -- codes that give the whole GPU to
 * their own memory pool, or that must not incur the device-wide synchronisation
 * cudaMalloc/cudaFree can cause inside a time step).
 *
 * Same result as mbdk_cholesky_f64 followed by mbdk_chol_solve3_f64 on the same
 * stream: A [batch][ld][ld] is overwritten by its lower Cholesky factors and X
 * [batch][ld][3] by the solutions of A X = B.  The diagonal-block inverses that those
 * calls keep in the caller's dinv and work buffers live instead in one static 16 MiB
 * device array inside the library (2^21 doubles), so the call allocates nothing and
 * calls no allocating routine.  Limit: batch * ((ld/64) * 4096 + 3 * ld) <= 2^21; larger
 * requests return MBD_ERR_SCRATCH_LIMIT before any work is launched.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current, so
 * make that first call before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset of that device the library must be unloaded and loaded
 * again before the next call.  All calls on a device share the
 * array and it keeps the last call's contents; calls whose work overlaps on the GPU
 * race on it and must be serialised by the caller.  status as in mbdk_cholesky_f64. */
#define MBD_ERR_SCRATCH_LIMIT 9
int mbdk_cholesky_solve3_f64_noalloc(void *stream, double *A, long long ld, int batch, double *X,
                                     int *status);

/* ---- Learned screening model -------------------------------------------------------
 * The paper has no learned part.  This per-atom model stands in for the screening solves
 * of Eqs. (scs) and (contraction) (Sec. 2.3): features of the local geometry -> MLP ->
 * y_k = log(alpha_bar(u_k) / alpha(u_k)) at the 16 grid points (u_0 = 0 and the 15 nodes).
 * All pointers are device pointers; every call enqueues on `stream` (a cudaStream_t) and
 * returns MBD_OK, MBD_ERR_INPUT for bad sizes or null pointers, or MBD_ERR_CUDA.
 *
 * Features (MBD_LEARNED_FEATURES per atom, FP32): for every other atom j of the same system
 * at distance d < 24 bohr, alpha0_j fc(d) exp(-(d - mu_m)^2 / (2 w^2)) summed over j, for
 * m = 0..63, mu_m = (m + 1/2) w, w = 0.375 bohr (4 radial shells of 6 bohr x 16 Gaussians),
 * fc(d) = (1 + cos(pi d / 24)) / 2, alpha0_j TS-scaled (Eq. ts-scaling); then the atom's own
 * TS-scaled alpha0, omega, R_vdW and its volume ratio; then the static screening moments
 * (the terms of the Dyson series of Eq. scs at u = 0): with B_ij = (1 - f_ij) T^GG_ij
 * (Eqs. scs-sr-dipole, tgg, mayer, fermi-damping; beta 0.83, a 6) and
 * M_i = sum_{j, d<24} alpha0_j B_ij: m1 = Tr M_i / 3, m2 = Tr(sum_j alpha0_j B_ij M_j) / 3,
 * m3 = Tr(M_i M_i) / 3, alpha0_i m1, alpha0_i^2 m2, alpha0_i^2 m3; then the terms of the
 * Dyson series of Eq. scs at the 16 grid points u_k (u_0 = 0 and the 15 nodes of Eq.
 * casimir-polder, Sec. 3.3): with alpha_j(u) of Eq. dyn-pol and B_ij(u) = (1 - f_ij) T^GG_ij
 * at the widths of alpha(u) (Eq. mayer), H^(0)_i = I and H^(q)_i = sum_{j != i} alpha_j(u)
 * B_ij(u) H^(q-1)_j over all atoms of the system, feature 74 + 3 k + q - 1 is
 * Tr H^(q)_i(u_k) / 3 for q = 1, 2, 3 (pair arithmetic in FP32, sums over partners in FP64).
 * Network: MLP 122 -> 128 -> 128 -> 16 on standardised features (x - mean) / std, SiLU
 * activations, FP16 weights and biases, FP32 accumulation.  One ensemble member's
 * parameters are MBD_LEARNED_PARAMS halves: W1 [122][128], b1 [128], W2 [128][128], b2 [128],
 * W3 [128][16], b3 [16] (W[in][out], row-major); members are stored one after another. */
#define MBD_LEARNED_FEATURES 122
#define MBD_LEARNED_OUTPUTS 16
#define MBD_LEARNED_PARAMS 34320
#define MBD_LEARNED_WORK 144   /* FP64 words of mbdk_scs_features scratch per atom */

/* Features of n_atoms atoms of n_systems systems stored one after another: system s holds
 * atoms offsets[s] .. offsets[s+1]-1 (offsets [n_systems + 1], offsets[0] = 0,
 * offsets[n_systems] = n_atoms).  coords [n_atoms][3] (bohr) and the free-atom parameters
 * [n_atoms] each as in mbd_set_free_atom_params (FP64); X [n_atoms][122] (FP32); work
 * [n_atoms][MBD_LEARNED_WORK] FP64 words of scratch (the moments M_i and the Dyson terms). */
int mbdk_scs_features(void *stream, int n_atoms, int n_systems, const int *offsets, const double *coords,
                      const double *alpha0_ref, const double *c6_ref, const double *rvdw_ref,
                      const double *volume_ratio, float *X, double *work);

/* Forward pass of n_members members on n_atoms rows of raw features X [n_atoms][122]:
 * Y [n_members][n_atoms][16]; mean, std [122]; params_fp16 [n_members][MBD_LEARNED_PARAMS].
 * zcache (optional, [n_members][2][n_atoms][128] FP32) keeps the pre-activations of both
 * hidden layers for mbdk_mlp_backward. */
int mbdk_mlp_forward(void *stream, int n_atoms, int n_members, const float *X, const float *mean,
                     const float *std, const void *params_fp16, float *Y, float *zcache);

/* Backward pass of sum(dY * Y) after mbdk_mlp_forward with a zcache, dY [n_members][n_atoms]
 * [16]: dX (optional) [n_members][n_atoms][122] receives the gradient with respect to the raw
 * features; grad (optional) [n_members][MBD_LEARNED_PARAMS] FP32 is ACCUMULATED with the
 * gradient with respect to the parameters (clear it first for a fresh gradient).  Without grad
 * the products run on the tensor cores (TF32 hi/lo parts against the exact FP16 weights, as
 * the forward), with grad in FP32 on the CUDA cores. */
int mbdk_mlp_backward(void *stream, int n_atoms, int n_members, const float *X, const float *mean,
                      const float *std, const void *params_fp16, const float *zcache, const float *dY,
                      float *dX, float *grad);

/* Mean squared error of y against t (n entries): dy = 2 (y - t) / n and, if loss is not
 * NULL, *loss = mean((y - t)^2) (FP64). */
int mbdk_mse_grad(void *stream, long long n, const float *y, const float *t, float *dy, double *loss);

/* One Adam step (b1 0.9, b2 0.999, eps 1e-8; step counts from 1) on n FP32 parameters with
 * moments m, v (updated in place); params_fp16 (optional) receives the updated parameters
 * rounded to FP16 (to nearest). */
int mbdk_adam_step(void *stream, long long n, float *params, const float *grad, float *m, float *v, int step,
                   float lr, void *params_fp16);

/* Training targets of the model: Y [n_atoms][16] (FP32) = log(alpha_bar[k][i] /
 * alpha_free[k][i]) from the screened and free polarizabilities [16][n_atoms] (FP64) of one
 * system at the 16 grid points. */
int mbdk_learned_targets(void *stream, int n_atoms, const double *alpha_bar, const double *alpha_free, float *Y);

/* dst[r][c] = src[idx[r]][c] for r < rows, c < width (FP32). */
int mbdk_gather_rows(void *stream, long long rows, int width, const int *idx, const float *src, float *dst);

#ifdef __cplusplus
}
#endif

#endif /* MBD_GB300_KERNELS_H */
