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

#ifdef __cplusplus
extern "C" {
#endif

/* C = alpha * A * op(B) + beta * D on the FP64 tensor path (mma.sync m8n8k4 f64).
 * A is M x K (lda).  trans_b = 1: op(B) = B^T with B N x K; trans_b = 0: op(B) = B
 * with B K x N (ldb).  C and D are M x N (ldc, ldd).  D may be NULL when beta == 0 and
 * may alias C.  mode 0 computes every 64x64 tile; mode 1 only tiles on or below the
 * diagonal (M == N); mode 2 only tiles on or above it and mirrors them into the lower
 * half (M == N, for products that are symmetric).  Leading dimensions must be even
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
 * leading dimensions multiples of 8.  mode 0: all tiles; mode 2: upper tiles mirrored
 * (M == N, symmetric results).  chunk_stages: K stages (32 TF32 / 64 bf16 elements) per
 * tensor-memory accumulation, partial sums added in FP32 with round-to-nearest (0: all of
 * K in one accumulation).  err (device int) gets bit 8 set if a wait timed out. */
int mbdk_gemm_tc(void *stream, int kind, int mode, int M, int N, int K, float alpha, const void *A0,
                 const void *A1, long long lda, const void *B0, const void *B1, long long ldb, float beta,
                 const float *D, float *C, void *C_hi, void *C_lo, float *CT, long long ldc, int chunk_stages,
                 int *err);

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
 * make that first call before any stream capture.  All calls on a device share the
 * array and it keeps the last call's contents; calls whose work overlaps on the GPU
 * race on it and must be serialised by the caller.  status as in mbdk_cholesky_f64. */
#define MBD_ERR_SCRATCH_LIMIT 9
int mbdk_cholesky_solve3_f64_noalloc(void *stream, double *A, long long ld, int batch, double *X,
                                     int *status);

#ifdef __cplusplus
}
#endif

#endif /* MBD_GB300_KERNELS_H */
