// Internal declarations of the sm_103a kernels of libmbdgb.  Not part of the C ABI.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace mbdgb {

constexpr int kTile = 64;          // dense tile edge; leading dimensions are multiples of it
constexpr int kMaxFreq = 64;       // upper bound on n_freq + 1

// Process-wide count of kernel launches made by this library (for profiles).
void count_launches(int k);
long long launch_count();

// Bits of the device status word.
enum : int {
    ST_INPUT = 1,          // NaN input or coincident atoms
    ST_SCS_NOT_PD = 2,     // non-positive pivot in the SCS Cholesky factorisation
    ST_NEG_ALPHA = 4,      // screened alpha0 or C6 not positive
    ST_TC_TIMEOUT = 8,     // a tensor-core GEMM wait ran out of its budget
};

// ---- tcgen05 GEMM (k_tc.cu) ------------------------------------------------------
// C = alpha sum_p A_p B_p^T + beta D on 128x128 tiles.  kind 0: TF32, operands FP32
// (A0, B0); kind 1: BF16x3, operands bf16 hi/lo pairs (A0 = A_hi, A1 = A_lo, same for
// B); kind 2: TF32x3, operands TF32-rounded hi and FP32 remainder lo (32-bit each).  A is M x K, B is N x K (row pitch lda, ldb elements); C, D, transposes share ld.
// mode 0: all tiles; mode 1: tiles on or below the diagonal only, not mirrored (square; for
// updates of which only the lower triangle is read); mode 2: upper tiles mirrored (symmetric
// products).  Optional
// outputs: C (FP32), Ch/Cl (bf16 hi/lo), CT/CTh/CTl (transposes, mode 0 only), and
// resid += sum over the leading nvalid x nvalid block of (delta - C)^2 (mode 0 only).
// Timeouts set ST_TC_TIMEOUT in *err.
struct TcOperands {
    const void *A0, *A1, *B0, *B1;
    long long lda, ldb;
};
struct TcArgs {
    int M, N, K;
    float alpha, beta;
    const float *D;
    long long ld;
    float *C;
    void *Ch, *Cl;       // split outputs: bf16 (kind 1) or 32-bit (kind 2)
    float *CT;
    void *CTh, *CTl;
    double *resid;
    long long nvalid;
    int mode;
    int *err;
    double *C64 = nullptr;   // optional FP64 output accumulated in place: C64 += result
    int chunk_stages = 0;    // K stages per TMEM accumulation (0: all of K in one)
    // Batch of independent products (blockIdx.y): A and B stacked as [batch][M][lda] and
    // [batch][N][ldb]; D and C of item b at D + b sC, C + b sC.  batch > 1 allows no other
    // output than C.
    int batch = 1;
    long long sC = 0;
};
cudaError_t tc_gemm(int kind, const TcOperands &op, const TcArgs &g, cudaStream_t s);
// The GEMM's bounded mbarrier wait on a barrier nothing arrives at, with a budget of `budget`
// clock cycles: sets ST_TC_TIMEOUT in *err when it gives up.
cudaError_t tc_wait_probe(long long budget, int *err, cudaStream_t s);
// FP64-accurate C = alpha A op(B) + beta D (k_split64.cu): the operands cut into exact TF32
// slices (split64.cuh), the slice products on the tensor cores (tc_gemm kind 0) over K in
// exact pieces, summed into C in FP64.  trans_b: op(B) = B^T with B N x K, else B is K x N.
// M, N multiples of 128, K of 64, ldc of 8; D may be C; work: gemm_f64_split_work_bytes.
// mode 0: every tile; mode 2 (M == N): upper tiles mirrored, for symmetric products.
size_t gemm_f64_split_work_bytes(int M, int N, int K);
cudaError_t gemm_f64_split(int trans_b, int mode, int M, int N, int K, double alpha, const double *A, long long lda,
                           const double *B, long long ldb, double beta, const double *D, long long ldd, double *C,
                           long long ldc, void *work, int *err, cudaStream_t s);
// Mixed-precision helpers: Y = scale Q (FP32 and, if Yh, bf16 hi/lo) and Z = I;
// Z = a I + b P; Zd = scale Zf in FP64; and the variational energy
// E = (1/4)(3 Tr V - sum V o W) - 3/2 sum omega (work: 608 doubles).
void mixed_init(int kind, const double *Q, long long ld, double scale, float *Yf, void *Yh, void *Yl, float *Zf,
                void *Zh, void *Zl, cudaStream_t s);
void mixed_axpby_identity(int kind, const float *P, long long ld, float a, float b, float *Zf, void *Zh, void *Zl,
                          cudaStream_t s);
void to_f64(const float *Zf, long long ld, double scale, double *Zd, cudaStream_t s);
// TF32x3 operand parts (32-bit hi, lo) of scale * Q (FP64) and of an FP32 matrix, with
// the diagonal optionally set to zero; Out = scale diag(A) B in FP64.
void split_tf32_f64(const double *Q, long long ld, double scale, int zero_diag, void *H, void *L, cudaStream_t s);
void split_tf32_f32(const float *Z, long long ld, int zero_diag, void *H, void *L, cudaStream_t s);
// TF32x3 parts (hi = tf32(a), lo = tf32(a - hi)) of a rows x cols panel of each FP32 matrix
// of a batch (A at the panel's first element, row pitch ld, matrices mstride apart) into H
// and L, each stacked [batch][rows][cols].
void split_panel_tf32(const float *A, long long ld, long long mstride, int batch, long long rows, int cols,
                      uint32_t *H, uint32_t *L, cudaStream_t s);
void diag_scale_rows_f64(const double *A, const float *B, long long ld, double scale, double *Out, cudaStream_t s);
void diag_scale_rows_f32(const float *A, const double *B, long long ld, double *Out, cudaStream_t s);
void split_tf32_f64_t(const double *A, long long ld, double scale, void *H, void *L, cudaStream_t s);   // of A^T
// Energy of the mixed modes from T1 = Tr(scale Q Z) (FP64 dot), T2 = sum V o W:
// E = (sqrt_s/4)(3 T1 - T2) - 3/2 sum omega; resid = |I - W|_F (work: 912 doubles).
void energy_correction(const double *Q, double scale, const float *Z, const double *V, const double *W, long long ld,
                       int n, double sqrt_s, const double *ombar, int N, double *work, double *out, double *resid,
                       cudaStream_t s);
void energy_variational(const double *V, const double *W, long long ld, int n, const double *ombar, int N,
                        double *work, double *out, cudaStream_t s);

// ---- dense FP64 (k_dense.cu) ----------------------------------------------------
// C[b] = alpha * A[b] op(B[b]) + beta * D[b] on 64x64 tiles, FP64 DMMA (mma.sync m8n8k4).
// A is M x K; op(B) = B^T with B N x K (trans_b = 1) or B with B K x N (trans_b = 0);
// C and D are M x N; all row-major with leading dimensions.  M, N, K are multiples of
// 64.  mode: 0 every tile; 1 lower tiles (tile row >= tile col) only; 2 upper tiles
// only, each also written transposed into the lower half (for products known to be
// symmetric).  D may alias C (each element is read before it is written).
struct GemmArgs {
    const double *A, *B, *D;
    double *C;
    long long lda, ldb, ldd, ldc;
    long long sA, sB, sD, sC;   // batch strides (elements)
    int M, N, K, batch;
    double alpha, beta;
    int mode;
    int trans_b;
};
void gemm_f64(const GemmArgs &g, cudaStream_t s);
// Z = a I + b P (ld x ld).
void axpby_identity(double *Z, const double *P, long long ld, double a, double b, cudaStream_t s);

// Batched right-looking blocked Cholesky (lower) of `batch` ld x ld matrices (stride
// mstride), in place.  Diagonal-block inverses L_kk^{-1} (64x64 each, nb per matrix)
// are written to dinv[b][k].  Sets ST_SCS_NOT_PD on a non-positive pivot.
void cholesky_f64(double *A, long long ld, long long mstride, int batch, double *dinv,
                  int *status, cudaStream_t s);

// Batched triangular solves with 3 right-hand sides, in place on X [b][ld][3]:
// forward L y = x, then backward L^T z = y (L from cholesky_f64).  work: same shape
// as X (the intermediate y).
void chol_solve3_f64(const double *L, long long ld, long long mstride, int batch,
                     const double *dinv, double *X, double *work, long long xstride, cudaStream_t s);
// Block-column triangular solves (k_trsv.cu), T = double or float: X <- L^-T L^-1 X.
template <typename T>
void trsv_blocked(const T *L, long long ld, long long mstride, int batch, const T *dinv, T *X, T *W, long long xstride,
                  cudaStream_t s);

// Mixed-precision screening solves (k_scs32.cu): FP32 copy of the batch, FP32 blocked
// Cholesky with FP32 diagonal-block inverses; then X = A^{-1} B by FP32 solves and
// `steps` iterative-refinement steps with residuals from the FP64 matrix (full, both
// triangles; rows >= n are padding).  work: 2 * batch * 3 ld floats.
// The factorisation is blocked in panels of kScsPanel columns (the first panel takes
// ld mod kScsPanel when that is not 0, so every trailing matrix is a multiple of 128): inside a panel 64-wide
// steps on the SIMT cores over sub-panels of kScsSub columns, the rest of the panel updated
// after each sub-panel on the tensor cores, and the trailing update A22 -= L21 L21^T on the
// tensor cores (TF32x3, k_tc_gemm, tiles of the lower triangle only).  panel: scratch of
// 2 * batch * ld * kScsPanel 32-bit words.  Only the lower triangle of A32 is read; tiles
// that cross the diagonal are written whole.  Tensor-core timeouts set ST_TC_TIMEOUT in
// *status; a launch error is returned.
constexpr int kScsPanel = 1024;
// Inside a panel, sub-panels of kScsSub columns are factorised by the 64-wide steps and the
// panel's columns right of each are updated on the tensor cores (a product of K = kScsSub).
constexpr int kScsSub = 256;
cudaError_t cholesky_f32_from_f64(const double *A64, float *A32, long long ld, int batch, float *dinv,
                                  uint32_t *panel, int *status, cudaStream_t s);
void refine_solve3(const double *A64, const float *L32, const float *dinv, long long ld, int n, int batch,
                   const double *B, double *X, float *work, int steps, cudaStream_t s);

// Sum of squares of (I - P) over the leading n x n block, written to out[0].
void frob_dev_identity(const double *P, long long ld, int n, double *out, cudaStream_t s);
// Y = Y * scale over the full ld x ld matrix.
void scale_matrix(double *Y, long long ld, double scale, cudaStream_t s);
// Z = I (ld x ld).
void set_identity(double *Z, long long ld, cudaStream_t s);
// Lanczos tridiagonal coefficients of a symmetric ld x ld matrix from a fixed start
// vector: coef[2j] = alpha_j, coef[2j+1] = beta_j, j < steps.  work: 3 ld doubles.
void lanczos_coefficients(const double *A, long long ld, int steps, double *work, double *coef,
                          cudaStream_t s);
// As lanczos_coefficients, with the matrix-vector products in FP32 on an FP32 copy of A
// written to A32 (ld x ld floats) and an FP32 copy of the Lanczos vector; the recurrence
// (alpha, beta, orthogonalisation) stays FP64.  work: 3 ld doubles + ld floats.
void lanczos_coefficients_f32(const double *A, float *A32, long long ld, int steps, double *work, double *coef,
                              cudaStream_t s);
// Maximum absolute row sum over rows 0..n-1 (Gershgorin bound), written to out[0].
void max_abs_rowsum(const double *Q, long long ld, int n, double *out, cudaStream_t s);

// ---- per-atom and pair kernels (k_atoms.cu, k_pairs.cu) -----------------------
struct AtomBufs {
    int N, nf1;                 // atoms, frequency points (u_0 = 0 included)
    const double *R;            // [N][3]
    const double *a0ref, *c6ref, *rref, *ratio;
    double *a0, *om, *rv;       // TS-scaled
    double *al_u, *sig_u;       // [nf1][N]
    double *abar;               // [nf1][N] screened alpha(iu)
    double *abar0, *c6bar, *ombar, *rbar;
    const double *u, *wu;       // [nf1] grid (device)
};

void prepare_atoms(const AtomBufs &b, int *status, cudaStream_t s);
void build_scs(const AtomBufs &b, double beta, double a, double *M, long long ld,
               long long mstride, int *status, cudaStream_t s);
// Rows and columns n..ld-1 of nf1 matrices: identity on the diagonal, zero couplings.
void pad_identity(double *M, long long ld, int n, int nf1, long long mstride, cudaStream_t s);
void init_rhs_identity(double *X, long long ld, int n, int nf1, long long xstride, cudaStream_t s);
void contract_screen(const AtomBufs &b, const double *X, long long ld, long long xstride,
                     int *status, cudaStream_t s);
// Eqs. (casimir-polder), (scale-rvdw-scs) from alpha_bar(u) already in b.abar.
void screened_params(const AtomBufs &b, int *status, cudaStream_t s);
void build_q(const AtomBufs &b, double beta, double a, double *Q, long long ld, int *status,
             cudaStream_t s);
void energy_trace(const double *Y, long long ld, int n, const double *ombar, int N,
                  double sqrt_s, double *out, cudaStream_t s);

// MBD gradient pass (Eq. mbd-gradient): reads Z (Q^{-1/2} = zscale * Z) once.
// Per atom: g_ombar (incl. the diagonal block and -3/2), g_abar0, g_rbar, gR [N][3].
struct MbdGradOut { double *g_ombar, *g_abar0, *g_rbar, *gR; };
// tq: per-atom Tr (Q^{1/2})_ii for dE/d omega_bar (second order in the error of Z), or NULL to
// take it from Z itself.
void mbd_grad_pass(const AtomBufs &b, double beta, double a, const double *Z, long long ld,
                   double zscale, const MbdGradOut &o, cudaStream_t s, const double *tq = nullptr);
// tq_i = sqrt_s Tr(X_ii), X = (3 V - V W)/2, for V = (Q/s) Z and W = Z V in FP64 with
// Z ~ (Q/s)^{-1/2}: Tr X_ii is second order in the error of Z (X ~ (Q/s)^{1/2}).
void block_trace_sqrt(const double *V, const double *W, long long ld, int N, double sqrt_s, double *tq,
                      cudaStream_t s);

// Chain through Eqs. (casimir-polder), (scale-rvdw-scs): h[k][i] = dE/d abar_i(u_k),
// and the direct parts of dE/d alpha0, dE/d R_vdW (g_a0, g_rv, overwritten).  Also
// writes the adjoint right-hand sides H[k][p][c] = h[k][p/3] delta_{p%3,c}.
void chain_screen(const AtomBufs &b, const MbdGradOut &o, double *h, double *g_a0,
                  double *g_rv, double *H, long long ld, long long xstride, cudaStream_t s);

// SCS adjoint pair pass: with X = M^{-1} E and V = M^{-1} H per frequency, adds
// -1/3 sum dM_pq (V X^T)_pq to dE/d alpha0, dE/d omega, dE/d R_vdW (g_a0, g_om, g_rv)
// and dE/dR (gR, accumulated).  With work32 (2 nf1 (xstride + N) floats) the per-pair
// arithmetic runs in single precision on FP32 copies of X, V, sigma(iu) and alpha(iu) (sums
// FP64), for the reduced-precision modes; with work32 = NULL, in FP64.
void scs_grad_pass(const AtomBufs &b, double beta, double a, const double *X, const double *V,
                   long long xstride, double *g_a0, double *g_om, double *g_rv, double *gR, float *work32,
                   cudaStream_t s);

// MBD-NL (Sec. 2.7, Eqs. mbd-nl-scaling, mbd-nl-rvdw): the oscillators from the inputs
// alpha0_ref, C6_ref, ra (in rref) and rw (in ratio), written to abar0, ombar, rbar, c6bar,
// abar (and a0, om, rv); ST_INPUT on non-positive or non-finite inputs.
void nl_params(const AtomBufs &b, int *status, cudaStream_t s);
// MBD-NL chain from the pair pass outputs to dE/d(alpha0_ref, C6_ref, ra, rw) [4][N], times
// *scale (device) if given.
void nl_chain(const AtomBufs &b, const MbdGradOut &o, const double *scale, double *gp, cudaStream_t s);

// Log-formula energy route (k_logdet.cu), Eqs. (log-formula), (rpa).  build_lr_freq: the nf
// matrices A_k = alpha(u_k)^{1/2} T^lr alpha(u_k)^{1/2} of the oscillators abar0, ombar, rbar
// on the nodes u_1..u_nf (b.u), ld x ld each, mstride apart, zero outside the 3N x 3N
// block and on the diagonal blocks.  batch_dot: out[b] = <X_b, Y_b> over `per` elements.
// add_identity_batch: A_b += I.  logdiag_batch: out[b] = sum_p ln L_b,pp (ST_SCS_NOT_PD on a
// non-positive diagonal).
cudaError_t build_lr_freq(const AtomBufs &b, double beta, double a, double *A, long long ld, long long mstride,
                          int nf, int *status, cudaStream_t s);
cudaError_t batch_dot(const double *X, const double *Y, long long per, long long stride, int batch, double *out,
                      cudaStream_t s);
void add_identity_batch(double *A, long long ld, long long mstride, int batch, cudaStream_t s);
void logdiag_batch(const double *L, long long ld, long long mstride, int batch, double *out, int *status,
                   cudaStream_t s);

// TS pairwise dispersion (Eqs. pairwise, ts-scaling, fermi-damping with steepness 20 and
// s_R = s_r) of the TS-scaled oscillators b.a0, b.om, b.rv (prepare_atoms): per-atom energy
// eatom [N] (E = sum), dE/dR [N][3] and dE/d(a0, om, rv) of the scaled oscillators [N] each.
void ts_pairs(const AtomBufs &b, double s_r, double *eatom, double *gR, double *ga0, double *gom, double *grv,
              cudaStream_t s);

// TS-scaling chain to [4][N] parameter gradients, times *scale (device) if given.
void ts_chain(const AtomBufs &b, const double *g_a0, const double *g_om, const double *g_rv,
              const double *scale, double *gp, cudaStream_t s);
// y = (*scale) x (scale device pointer, NULL for 1).
void scale_copy(const double *x, int n, const double *scale, double *y, cudaStream_t s);

// ---- periodic systems (k_periodic.cu) --------------------------------------------
// Cell: rows of A are the lattice vectors; Ainv = A^{-1}; rows of B are the reciprocal
// vectors (a_c . b_d = 2 pi delta_cd); vol = |det A|.  Ewald split gamma, real-space
// cutoff rc (also the cutoff of the damped and screening lattice sums), reciprocal
// cutoff kc.
struct CellGeom {
    double A[9], Ainv[9], B[9];
    double vol, gamma, rc, kc;
};
// Bloch vectors and reciprocal lattice: kq [nk][3] (Cartesian q), G [nG][3] (every G
// with |G + q| < kc for some q), glist [nk][maxG] indices into G of the vectors with
// 0 < |G + q_k| < kc (gcount[k] of them), S [nG][N] structure factors e^{i G.R_i}.
struct PeriodicBufs {
    CellGeom cell;
    int nk, nG, maxG;
    const double *kq, *G;
    const int *glist, *gcount;
    double2 *S;
};
// Complex matrices are planar: matrix k has its real part at base + k * 2 ld^2 and its
// imaginary part ld^2 further on.
void structure_factors(const AtomBufs &b, const PeriodicBufs &p, cudaStream_t s);
// Gamma-point screening matrices: alpha^{-1} + sum over lattice images of (1 - f) T^GG.
void build_scs_periodic(const AtomBufs &b, const CellGeom &c, double beta, double a, double *M, long long ld,
                        long long mstride, int *status, cudaStream_t s);
// Q(q_k) for every Bloch vector: diag(omega^2) + c_i c_j T^lr(q), T^lr = Ewald[T] minus the
// damped-away part, both triangles; rows >= n padded with omega_0^2 on the diagonal.
void build_q_periodic(const AtomBufs &b, const PeriodicBufs &p, double beta, double a, double *Q, long long ld,
                      int n, int *status, cudaStream_t s);
// Batched complex helpers (nk planar matrices of order ld).
void cscale(double *Y, long long ld, int nk, double scale, cudaStream_t s);
void cset_identity(double *Z, long long ld, int nk, cudaStream_t s);
void caxpby_identity(double *Z, const double *P, long long ld, int nk, double a, double b, cudaStream_t s);
void cfrob_dev_identity(const double *P, long long ld, int n, int nk, double *out, cudaStream_t s);
void cmax_abs_rowsum(const double *Q, long long ld, int nk, double *out, cudaStream_t s);
// C = alpha A B + beta D for nk planar complex matrices (4 real FP64 GEMMs; D may be C).
// herm: the result is Hermitian (as Y Z Y, Z Y Z for Hermitian Y, Z): upper tiles only,
// mirrored (real part symmetric, imaginary part antisymmetric).
void cgemm_f64(const double *A, const double *B, const double *D, double *C, long long ld, int nk, double alpha,
               double beta, bool herm, cudaStream_t s);
// Lanczos coefficients of every Q_k: coef[k][2j] = alpha_j, coef[k][2j+1] = beta_j.
// work: 3 nk 2 ld doubles.
void clanczos_coefficients(const double *Q, long long ld, int nk, int steps, double *work, double *coef,
                           cudaStream_t s);
// Mixed modes on a cell: the real symmetric embedding M = [[Re, -Im], [Im, Re]] of planar slot k
// of Q (order 2n in an lde x lde matrix, padded), the planar slot k of Z from the embedded
// Ze ~ M^{-1/2}, and E = 1/(2 nk) sum_k ek[k] - 3/4 sum omega_bar from the embedded energies.
void embed_hermitian(const double *Q, long long ld, int n, int k, double *M, long long lde, cudaStream_t s);
void extract_hermitian(const double *Ze, long long lde, int n, double *Z, long long ld, int k, cudaStream_t s);
void periodic_mixed_energy(const double *ek, int nk, const double *ombar, int N, double *out, cudaStream_t s);
// E = sqrt_s/(2 nk) sum_k Re Tr Y_k - 3/2 sum omega_bar (compensated).
void energy_trace_periodic(const double *Y, long long ld, int n, int nk, const double *ombar, int N,
                           double sqrt_s, double *out, cudaStream_t s);
// MBD gradient of the periodic energy from Z_k (Q(q_k)^{-1/2} = zscale Z_k): per atom
// g_ombar, g_abar0, g_rbar, gR (o), and dE/dA accumulated into gA [9].  work: 2N doubles.
// tq: (1/nk) sum_q Re Tr (Q(q)^{1/2})_ii per atom for dE/d omega_bar (second order in the error of
// Z), or NULL to take it from Z.
// f32_recip: the reciprocal-space sum in FP32 (chunk sums added in FP64), for the mixed
// modes, whose Z ~ Q^{-1/2} is accurate to far less than FP32 rounding.
void periodic_mbd_grad(const AtomBufs &b, const PeriodicBufs &p, double beta, double a, const double *Z,
                       long long ld, double zscale, const MbdGradOut &o, double *work, double *gA, cudaStream_t s,
                       const double *tq = nullptr, bool f32_recip = false);
// out[i] = (1/rows) sum_r x[r][i] for a rows x N array (compensated).
void mean_rows(const double *x, int rows, int N, double *out, cudaStream_t s);
// SCS adjoint pair pass over lattice images (as scs_grad_pass), with the lattice part
// accumulated into gA [9].  gA_part: N x 9 doubles of workspace.
void scs_grad_periodic(const AtomBufs &b, const CellGeom &c, double beta, double a, const double *X,
                       const double *V, long long xstride, double *g_a0, double *g_om, double *g_rv, double *gR,
                       double *gA_part, double *gA, cudaStream_t s);

// Periodic TS dispersion (k_ts_periodic.cu; the sum of Eq. ts-ewald minus the damped-away
// part) of the TS-scaled oscillators, from the structure factors p.S of the current
// coordinates: per-atom energy eatom [N], dE/dR [N][3], dE/d(a0, om, rv) [N] each and the
// lattice gradient gA [9] (gA_part: 9N doubles of workspace; tab: 2 nG doubles).
void ts_periodic(const AtomBufs &b, const PeriodicBufs &p, double s_r, double *tab, double *eatom, double *gR,
                 double *ga0, double *gom, double *grv, double *gA_part, double *gA, int *status, cudaStream_t s);

// ---- learned screening model (k_learned.cu) ---------------------------------------
// FP64 words per atom of the features' work (scs_features: static moments, then the FP32
// state of the Dyson block) and of the learned forces' work (learned_forces).
constexpr int kLearnedWork = 144;
constexpr int kLearnedAdjointWork = 243;
int learned_param_count();
void scs_features(int n_atoms, int n_sys, const int *offsets, const double *R, const double *a0ref,
                  const double *c6ref, const double *rref, const double *ratio, float *X, double *work,
                  cudaStream_t s);
// MLP forward on the tensor cores; err (optional, device int) receives ST_TC_TIMEOUT if a wait
// runs out (the outputs are then NaN).  packed (optional): the weights in the kernels' shared-
// memory layout, kLearnedPackedFloats per member, from mlp_pack (else the kernels convert
// the FP16 parameters themselves).
constexpr long long kLearnedPackedFloats = 6LL * 128 * 128;
cudaError_t mlp_pack(int members, const void *params16, float *packed, cudaStream_t s);
cudaError_t mlp_forward(int B, int members, const float *X, const float *mean, const float *stdv,
                        const void *params16, float *Y, float *zcache, cudaStream_t s, int *err = nullptr,
                        const float *packed = nullptr);
cudaError_t mlp_backward(int B, int members, const float *X, const float *mean, const float *stdv,
                         const void *params16, const float *zcache, const float *dY, float *dX, float *grad,
                         cudaStream_t s, const float *packed = nullptr);
void mse_grad(long long n, const float *y, const float *t, float *dy, double *loss, cudaStream_t s);
void adam_step(long long n, float *p, const float *g, float *m, float *v, int step, float lr, void *p16,
               cudaStream_t s);
void gather_rows(long long rows, int width, const int *idx, const float *src, float *dst, cudaStream_t s);
// alpha_bar[k][i] = alpha_i(u_k) exp(mean over members of Y[m][i][k]) and the member spread
// spread[k][i] (population standard deviation of alpha_i(u_k) exp(Y[m][i][k])).
void learned_alpha(int N, int members, int nf1, const double *al_u, const float *Y, double *abar, double *spread,
                   cudaStream_t s);
// Learned path gradients: dY[m][i][k] = h[k][i] alpha_bar[k][i] / members (member outputs'
// upstream gradient); gR[i] += dE/dR_i through the features of one system (offsets [0, N]),
// from dX [members][N][122] (mlp_backward), the work [N][kLearnedWork] that scs_features
// filled and workspace adjoint [N][kLearnedAdjointWork].
void learned_dy(int N, int members, int nf1, const double *h, const double *abar, float *dY, cudaStream_t s);
void learned_forces(int N, const int *offsets, const double *R, const double *a0ref, const double *rref,
                    const double *ratio, double *work, const float *dX, int members, double *adjoint, double *gR,
                    cudaStream_t s);
// out[0] = scale std_m(D_m) / N, D_m = sum_{k,i} h[k][i] alpha_i(u_k) (e^{Y[m][i][k]} - its mean over
// the members): the energy-error estimate per atom from the members' first-order energies.
void learned_estimate(int N, int nf1, int members, double scale, const double *h, const double *al_u,
                      const float *Y, double *out, cudaStream_t s);

}  // namespace mbdgb
