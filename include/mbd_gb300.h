/*
 * mbd_gb300.h -- C ABI of the GB300 (sm_103a) MBD@rsSCS library (libmbdgb.so).
 *
 * The library evaluates the many-body-dispersion energy of the MBD@rsSCS method and its
 * analytic gradients (arXiv 2308.03140):
 *   - TS volume scaling of free-atom parameters, Eq. (ts-scaling), Sec. 2.7;
 *   - range-separated self-consistent screening on an imaginary-frequency grid,
 *     Eqs. (scs), (contraction), (casimir-polder), (dyn-pol), (tgg), (mayer),
 *     (scs-sr-dipole), (scale-rvdw-scs), Secs. 2.3 and 2.7, grid of Sec. 3.3;
 *   - the coupled-oscillator matrix Q, Eq. (q-matrix), and the energy, Eq. (mbd-energy),
 *     through Q^{1/2} and Q^{-1/2} from coupled Newton-Schulz iterations;
 *   - gradients, Eq. (mbd-gradient) and the SCS derivative of Eq. (scs-gradient) in
 *     adjoint form, with respect to coordinates and the free-atom parameters.
 * The calls follow the paper's statement of the problem and its Fortran API (Sec. 3.1,
 * Listing fortran-api): a plain input set, an opaque handle, an evaluate call and an
 * exception query.
 *
 * Units: Hartree atomic units (bohr, Hartree).  Arrays are row-major and owned by the
 * caller; the library never keeps a caller pointer after a call returns.  The context
 * owns its device workspace, allocated by mbd_set_geometry.  A context is not
 * thread-safe: one call at a time per context.
 *
 * Every call returns MBD_OK (0) or an MBD_ERR_* code; the code, the name of the
 * failing stage and a message are kept in the context for mbd_get_exception (the
 * get_exception protocol of Sec. 3.1).  Outputs are written only on success.
 */
#ifndef MBD_GB300_H
#define MBD_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define MBD_OK 0
#define MBD_ERR_INPUT 1           /* invalid argument, NaN input, overlapping atoms   */
#define MBD_ERR_NEG_EIGENVALUE 2  /* Q not positive definite: polarization catastrophe, Sec. 2.1 */
#define MBD_ERR_SCS_NEG_ALPHA 3   /* screened static polarizability or C6 <= 0       */
#define MBD_ERR_SCS_NOT_PD 4      /* SCS matrix alpha^-1 + T^scs not positive definite */
#define MBD_ERR_NOT_CONVERGED 5   /* Newton-Schulz iteration cap reached             */
#define MBD_ERR_CUDA 6            /* CUDA runtime error                              */
#define MBD_ERR_STATE 7           /* call order (geometry/parameters not set)        */
#define MBD_ERR_UNSUPPORTED 8     /* option not supported for this system or mode    */

/* Arithmetic of the matrix function Q^{+-1/2}.  The mixed modes run the Newton-Schulz
 * iterations on the 5th-generation tensor cores with FP32 accumulation, then one FP64
 * correction: with Z ~ Q^{-1/2}, V = Q Z and W = Z V (FP64), Tr Q^{1/2} is taken as
 * (3 Tr V - sum V o W)/2, whose error is second order in the error of Z; the energy
 * subtraction and all sums stay in FP64 with compensation.  Gradients use Z.  In the same
 * modes the screening matrices are factored in FP32 (tensor-core TF32x3 updates) and each
 * solution is refined once against the FP64 matrix. */
#define MBD_PREC_FP64 0           /* plain FP64 throughout                           */
#define MBD_PREC_TF32 1           /* TF32 tensor-core products, FP64 correction      */
#define MBD_PREC_BF16X3 2         /* bf16 hi/lo split products (3 per GEMM), FP64 correction */
#define MBD_PREC_TF32X3 3         /* TF32 hi/lo split products (3 per GEMM), FP64 correction */
#define MBD_PREC_FP64_SPLIT 4     /* as FP64, the Newton-Schulz products FP64-accurate on the TF32
                                     tensor cores by error-free splitting (finite systems) */

typedef struct mbd_ctx mbd_ctx;

/* Options.  Defaults (mbd_default_options): n_freq 15 (Sec. 3.3), beta 0.83, a 6
 * (Sec. 2.7), precision FP64, ns_tol 1e-8 (Frobenius norm of I - Z Y at which one
 * final Newton-Schulz step is taken; periodic systems: of all Bloch vectors' matrices
 * together), ns_max_iter 100, tc_chunk_stages 0 (per kind), ewald_gamma, real_cutoff and
 * recip_cutoff 0 (automatic, see below), learned_max_error 1e-6, mixed_max_error 1e-7,
 * learned_estimate_scale 1. */
typedef struct {
    int n_freq;          /* Gauss-Legendre points of the Casimir-Polder integral     */
    double beta;         /* damping scale s_R of the Fermi function, Eq. (fermi-damping) */
    double a;            /* damping steepness                                          */
    int precision;       /* MBD_PREC_* (default FP64)                                  */
    double ns_tol;
    int ns_max_iter;
    int tc_chunk_stages; /* mixed modes: K stages (32 TF32 or 64 bf16 elements each) per
                            tensor-memory accumulation; the partial sums are added in FP32
                            with round-to-nearest (0, the default: 8 for BF16x3, 2 for TF32
                            and TF32x3)                                                   */
    /* Periodic systems (Sec. 2.2, Ewald summation of the dipole tensor).  <= 0 selects:
     * real_cutoff = 6/ewald_gamma; ewald_gamma = 6/real_cutoff when only the cutoff is
     * given, else 2.5/Omega^(1/3); recip_cutoff = 10 ewald_gamma.  real_cutoff (bohr) also
     * bounds the lattice sums of the damped tensors (screening and the damped-away part of
     * T^lr), where (1 - f) decays exponentially.                                         */
    double ewald_gamma;   /* Ewald splitting parameter (1/bohr)                          */
    double real_cutoff;   /* real-space cutoff (bohr)                                    */
    double recip_cutoff;  /* reciprocal-space cutoff on |G + q| (1/bohr)                 */
    /* Screening: MBD_SCS_PLAIN (the Dyson solves of Eq. (scs)) or MBD_SCS_LEARNED (the model
     * set by mbd_set_scs_model predicts alpha_bar(iu); when its estimated energy error per
     * atom exceeds learned_max_error (Ha, default 1e-6) the evaluation is redone with plain
     * screening; the model's features and outputs use the 15-point grid, so learned mode
     * needs n_freq = 15).  The learned model is not part of the paper.
     * MBD_SCS_NL selects MBD-NL (Sec. 2.7, paragraph MBD-NL): no screening; the oscillators
     * are set directly by Eq. (mbd-nl-scaling), alpha0_i = alpha0_ref,i ra_i and
     * omega_i = omega_ref,i rw_i with omega_ref = 4 c6_ref / (3 alpha0_ref^2), and the damping
     * radii by Eq. (mbd-nl-rvdw), R_i = 5/2 alpha0_ref,i^(1/7) ra_i^(1/3), where
     * ra = alpha0_df/alpha0_df,ref and rw = omega_df/omega_df,ref are the ratios of a density
     * polarizability functional for the atom in the system and the free atom.  In this mode
     * the third and fourth per-atom arrays of mbd_set_free_atom_params, mbd_evaluate_dev and
     * mbd_backward_dev are ra and rw (in place of rvdw_ref and the volume ratio), and
     * grad_params holds dE/d(alpha0_ref, c6_ref, ra, rw).  Finite and periodic systems.    */
    int scs_mode;
    double learned_max_error;
    /* BF16x3 and TF32x3: largest accepted estimate of the energy error per atom (Ha) left by
     * the tensor-core Z ~ Q^{-1/2} after the FP64 correction, (3/16) sqrt(s) r^2 / N with
     * r = |Z Q Z - I|_F (the correction's error is second order in that of Z; default 1e-7).
     * Above it the evaluation fails with MBD_ERR_NOT_CONVERGED (for instance a Q so badly
     * conditioned that the reduced-precision iteration cannot resolve it; the FP64 path can). */
    double mixed_max_error;
    /* MBD_SCS_LEARNED: factor on the ensemble's error estimate (mbd_set_scs_model), fitted
     * with the model on held-out clusters so that the scaled estimate bounds the true error of
     * most of them (default 1, the unscaled estimate; must be positive).                 */
    double learned_estimate_scale;
} mbd_options;

#define MBD_SCS_PLAIN 0
#define MBD_SCS_LEARNED 1
#define MBD_SCS_NL 2

/* Fills *opt with the defaults above.  Returns MBD_ERR_INPUT if opt is NULL. */
int mbd_default_options(mbd_options *opt);

/* Creates a context on CUDA device `cuda_device` with options *opt (NULL: defaults).
 * *out receives the handle.  Allocates no device memory yet. */
int mbd_create(mbd_ctx **out, int cuda_device, const mbd_options *opt);

/* Frees the context and all device memory it owns.  NULL is accepted. */
int mbd_destroy(mbd_ctx *ctx);

/* Sets the system: n_atoms atoms at coords [n_atoms][3] (bohr, host memory), and for a
 * periodic system the lattice [3][3] (rows are the lattice vectors, bohr) and the
 * Monkhorst-Pack grid k_grid [3] (k-points (2m - n_c - 1)/(2 n_c) in fractional
 * reciprocal coordinates, m = 1..n_c, Sec. 2.2); lattice and k_grid are both NULL for a
 * finite system.  Allocates the device workspace for that size.  Periodic systems run in
 * FP64 or in the tensor-core modes (TF32, BF16X3, TF32X3: each Q(q) through its real
 * symmetric embedding); MBD_PREC_FP64_SPLIT returns MBD_ERR_UNSUPPORTED here for them, and
 * learned screening returns it at evaluation. */
int mbd_set_geometry(mbd_ctx *ctx, int n_atoms, const double *coords, const double *lattice,
                     const int *k_grid);

/* Free-atom parameters, host arrays of n_atoms each: alpha0_ref (bohr^3), c6_ref
 * (Ha bohr^6), rvdw_ref (bohr) and the volume ratio V/V_ref of Eq. (ts-scaling), as in
 * update_vdw_params_from_ratios of the Fortran API. */
int mbd_set_free_atom_params(mbd_ctx *ctx, const double *alpha0_ref, const double *c6_ref,
                             const double *rvdw_ref, const double *volume_ratio);

/* Evaluates the energy (Ha) with host-memory inputs set above and host-memory outputs.
 * grad_coords [n_atoms][3] (Ha/bohr), grad_params [4][n_atoms] (dE/d alpha0_ref,
 * dE/d c6_ref, dE/d rvdw_ref, dE/d ratio) and alpha_scs [n_atoms] (screened static
 * polarizability) may each be NULL; gradients are computed only if one of grad_coords
 * or grad_params is given.  grad_lattice [3][3] (dE/dA_cd for lattice vector c, component d,
 * with the Cartesian atom positions held fixed) is for periodic systems only. */
int mbd_evaluate(mbd_ctx *ctx, double *energy, double *grad_coords, double *grad_lattice,
                 double *grad_params, double *alpha_scs);

/* Device-memory variant for callers that keep tensors on the GPU (the PyTorch binding).
 * All pointers are device pointers on the context's device: coords [n_atoms][3],
 * the four parameter arrays [n_atoms] each, energy [1], grad_coords [n_atoms][3] or
 * NULL, grad_params [4][n_atoms] or NULL, alpha_scs [n_atoms] or NULL.  `stream` is a
 * cudaStream_t (NULL: the legacy default stream); the call enqueues its work there and
 * returns after that stream has finished it.  n_atoms must equal the size given to
 * mbd_set_geometry. */
int mbd_evaluate_dev(mbd_ctx *ctx, void *stream, int n_atoms, const double *coords,
                     const double *alpha0_ref, const double *c6_ref, const double *rvdw_ref,
                     const double *volume_ratio, double *energy, double *grad_coords,
                     double *grad_params, double *alpha_scs);

/* Number of successful evaluations (mbd_evaluate, mbd_evaluate_dev) of the context so far;
 * after an evaluation it is that evaluation's number, which mbd_backward_dev checks.
 * MBD_ERR_INPUT if ctx or count is NULL. */
int mbd_get_evaluation_count(const mbd_ctx *ctx, long long *count);

/* Hand-written backward of the last evaluation (the analytic gradient of Sec. 2.4 as a
 * reverse-mode pass): from the device state the last mbd_evaluate or mbd_evaluate_dev
 * left in the context (screening factors, M^{-1} 1 and Q^{-1/2}), computes
 * grad_energy[0] * dE/dX for coordinates (grad_coords [n_atoms][3]) and free-atom
 * parameters (grad_params [4][n_atoms]); either may be NULL.  All pointers are device
 * pointers; grad_energy may be NULL (factor 1).  `evaluation` is the number
 * (mbd_get_evaluation_count, read right after the forward call) of the evaluation to
 * differentiate: MBD_ERR_STATE if the context's last evaluation is another one, whose state
 * has replaced it (0 skips the check).  The inputs must be the ones of that evaluation (same
 * values; they are read again).  MBD_ERR_STATE if no evaluation has succeeded since the
 * context was created or its geometry last reallocated. */
int mbd_backward_dev(mbd_ctx *ctx, void *stream, long long evaluation, int n_atoms, const double *coords,
                     const double *alpha0_ref, const double *c6_ref, const double *rvdw_ref,
                     const double *volume_ratio, const double *grad_energy, double *grad_coords,
                     double *grad_params);

/* Learned screening model for MBD_SCS_LEARNED (host arrays, copied): n_members ensemble
 * members of MBD_LEARNED_PARAMS FP16 values each (layout in include/mbd_gb300_kernels.h),
 * feature mean and std [MBD_LEARNED_FEATURES = 122] (FP32).  The prediction is the members' mean of
 * y = log(alpha_bar/alpha); the spread of the members' first-order energies gives the
 * energy-error estimate c std_m( sum_{i,u} dE/d alpha_bar_i(u) (alpha_bar_m,i(u) - mean over
 * members) ) / N, alpha_bar_m = alpha exp(y_m), c = learned_estimate_scale.  Finite systems only; energies and coordinate
 * gradients (through the network and the features); a request for parameter gradients in
 * learned mode returns MBD_ERR_UNSUPPORTED. */
int mbd_set_scs_model(mbd_ctx *ctx, int n_members, const void *params_fp16, const float *mean, const float *std);

/* Outcome of the last learned-mode evaluation: the estimated energy error per atom (Ha) and
 * whether the evaluation fell back to plain screening (1) or kept the model's result (0). */
int mbd_get_learned_stats(mbd_ctx *ctx, double *estimated_error, int *fell_back);

/* Screening only (Secs. 2.3 and 2.7: Eqs. ts-scaling, scs, contraction, casimir-polder,
 * scale-rvdw-scs) with plain Dyson solves, for the geometry and parameters set above: host
 * outputs alpha_iu [n_freq+1][n_atoms] (screened), alpha_free_iu [n_freq+1][n_atoms] (the
 * unscreened alpha_i(iu) of Eq. dyn-pol), c6, omega, rvdw [n_atoms]; any may be NULL.
 * Finite and periodic (Gamma-point) systems; MBD_ERR_UNSUPPORTED in MBD-NL mode, which
 * has no screening step. */
int mbd_screen(mbd_ctx *ctx, double *alpha_iu, double *alpha_free_iu, double *c6, double *omega, double *rvdw);

/* Lattice gradient [3][3] (host) of the last gradient evaluation of a periodic system
 * (mbd_evaluate with gradients, mbd_evaluate_dev with gradients, or mbd_backward_dev,
 * scaled like its other outputs).  MBD_ERR_STATE if there is none. */
int mbd_get_lattice_gradient(mbd_ctx *ctx, double *grad_lattice);

/* Screening detail of the last successful evaluation, host arrays: alpha_iu
 * [n_freq+1][n_atoms] (row 0 is u = 0), c6 [n_atoms], omega [n_atoms] (screened
 * frequencies), rvdw [n_atoms] (screened damping radii).  Any may be NULL.  In MBD-NL mode
 * these are the oscillators of Eqs. (mbd-nl-scaling), (mbd-nl-rvdw): alpha_iu =
 * alpha0 / (1 + u^2/omega^2), c6 = 3/4 alpha0^2 omega, omega, and the damping radii. */
int mbd_get_scs_detail(mbd_ctx *ctx, double *alpha_iu, double *c6, double *omega, double *rvdw);

/* MBD energy by the imaginary-frequency log formula, Eq. (log-formula), and its many-body
 * orders, Eq. (rpa) -- a second route to the energy, for cross-checks and for the analysis
 * of many-body contributions.  For the oscillators of the last successful evaluation
 * (screened alpha_bar0, omega_bar and damping radii R_bar, or those of MBD-NL) and the
 * coordinates set by mbd_set_geometry: *energy = 1/(2 pi) sum_k w_k ln det(I + A_k) with
 * A_k = alpha(u_k)^(1/2) T^lr alpha(u_k)^(1/2), alpha_i(u) = alpha_bar0_i/(1 + u^2/omega_bar_i^2)
 * and T^lr of Eq. (mbd-lr-dipole), over the n_freq Gauss-Legendre nodes u_k > 0 of the
 * screening grid (Sec. 3.3) with their weights; orders[m - 2] = E^(m) =
 * -1/(2 pi) sum_k w_k (-1)^m/m Tr A_k^m for m = 2..max_order (max_order 1..4; orders may be
 * NULL when max_order is 1).  FP64 throughout (Cholesky factors of I + A_k; orders 3 and 4
 * cost one n x n x n product per node).  Finite systems only.  The call reuses the screening
 * buffers, so mbd_backward_dev needs a new evaluation afterwards.  MBD_ERR_STATE without a
 * prior evaluation; MBD_ERR_SCS_NOT_PD if some I + A_k is not positive definite (dipole
 * collapse). */
int mbd_log_energy(mbd_ctx *ctx, int max_order, double *energy, double *orders);

/* TS pairwise dispersion (Secs. 2.6 and 2.7: Eq. pairwise with the oscillators of Eq.
 * ts-scaling and the damping of Eq. fermi-damping with steepness 20 and s_R = s_r, which
 * depends on the short-range model) for the geometry and free-atom parameters set above:
 * E = -1/2 sum_{i != j} C6_ij f_ij / R_ij^6, C6_ij = 3/2 alpha0_i alpha0_j / (1/omega_i + 1/omega_j).
 * For a cell (mbd_set_geometry with a lattice; the k-grid is not used) E is per cell and the
 * sum runs over j in the cell and all lattice images: the Ewald sum of 1/R^6 of Eq. ts-ewald
 * (gamma, real_cutoff, recip_cutoff of the options, the G = 0 term included, self term
 * -gamma^6/6) minus the real-space sum of (1 - f)/R^6 within real_cutoff.
 * Host outputs: *energy (Ha), grad_coords [n_atoms][3], grad_lattice [3][3] (dE/dA with A's
 * rows the lattice vectors and the Cartesian coordinates held fixed; cells only, else
 * MBD_ERR_UNSUPPORTED) and grad_params [4][n_atoms] (dE/d alpha0_ref, c6_ref, rvdw_ref,
 * volume ratio); any gradient may be NULL.  FP64.  MBD_ERR_UNSUPPORTED in MBD-NL mode;
 * MBD_ERR_INPUT for non-positive parameters or coincident atoms.  The call reuses gradient
 * scratch, so mbd_backward_dev needs a new evaluation afterwards. */
int mbd_ts_energy(mbd_ctx *ctx, double s_r, double *energy, double *grad_coords, double *grad_lattice,
                  double *grad_params);

/* Statistics of the last evaluation: Newton-Schulz iterations, the scale s of
 * Y0 = Q/s, the final Frobenius norm of I - Z Y, and (mixed modes) the Frobenius norm of
 * Z Q Z - I in FP64 for the Z ~ Q^{-1/2} used (0 in FP64 mode).  Any may be NULL. */
int mbd_get_stats(mbd_ctx *ctx, int *ns_iterations, double *ns_scale, double *ns_residual,
                  double *correction_residual);

/* Device-time profile of the last evaluation, gathered with CUDA events on the stream
 * the work was launched on when profiling is enabled (mbd_set_profiling).  Times in
 * milliseconds; flops are the algorithmic counts of the listed kernels (2 m n k for a
 * full product, n^2 (n + 1) for a product whose symmetric result is formed from one
 * triangle, n^3/3 per Cholesky factorisation). */
typedef struct {
    int launches;            /* CUDA kernels launched by the evaluation                  */
    int gemm_launches;       /* FP64 tensor-path GEMM launches of the Newton-Schulz stage */
    double gemm_ms;          /* summed device time of those launches                      */
    double gemm_flops;       /* their summed algorithmic flops                            */
    double screening_ms;     /* build + factorise + solve, all frequency points           */
    double screening_flops;  /* (n_freq + 1) n^3 / 3                                      */
    double newton_schulz_ms; /* Q build, scale, iterations, energy                        */
    double gradient_ms;      /* all gradient passes and adjoint solves                    */
    double total_ms;
    int tc_launches;         /* tensor-core (tcgen05) GEMM launches, mixed modes           */
    double tc_ms;            /* their summed device time                                  */
    double tc_flops;         /* their algorithmic flops (one product each)                */
    double correction_ms;    /* FP64 correction of the mixed modes                        */
} mbd_profile;

/* Enables (1) or disables (0) event timing of the following evaluations. */
int mbd_set_profiling(mbd_ctx *ctx, int enable);

/* Profile of the last evaluation; all zero if profiling was off. */
int mbd_get_profile(mbd_ctx *ctx, mbd_profile *out);

/* Last error of this context: code, the stage that failed (origin) and a message,
 * each string truncated to len bytes including the terminator.  ctx may not be NULL. */
int mbd_get_exception(const mbd_ctx *ctx, int *code, char *origin, char *msg, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* MBD_GB300_H */
