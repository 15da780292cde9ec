/*
 * mbd_oracle.c -- plain, slow FP64 CPU oracle for MBD@rsSCS (arXiv 2308.03140).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file: it is
 * loaded by the tests, by the package's smoke check and by the benchmark's CPU-baseline
 * leg.  It shares no code, header, table or constant generator with the CUDA path.
 *
 * Every routine follows the paper's equations in the paper's order, with explicit
 * loops: explicit dipole sums, cyclic Jacobi eigendecomposition, Gauss-Jordan
 * inversion with partial pivoting, Neumaier-compensated sums.  Hartree atomic units.
 *
 * Readings of the paper taken here (each one is listed with its reason in the design
 * notes of the repository):
 *   R1  Dipole tensor: the explicit form (delta r^2 - 3 r r)/r^5 of Eq. (dipole), i.e.
 *       T = -grad grad (1/r).  T^GG and T^erfc are taken with the same sign convention.
 *   R2  T^erfc numerator: (-r_a r_b C + delta r^2 B)/r^5 (the -grad grad of erfc(g r)/r);
 *       the printed -3 r_a r_b C fails the gamma -> 0 limit.
 *   R5  T^lr = g(Rbar) T (the approximate form of Eq. mbd-lr-dipole).
 *   R7  Screening is evaluated at u = 0 plus the 15 mapped Gauss-Legendre nodes;
 *       C6bar uses only the weighted nodes.
 *   R8  Gradient: dE = 1/4 Tr(Q^{-1/2} dQ) - 3/2 sum d(omega_bar).
 *   R9  SCS damping uses the TS-scaled R_vdW; the MBD damping uses Rbar.  Both a=6,
 *       s_R = beta.
 *   R11 The -3/2 sum(omega) term uses the screened omega_bar.
 *
 * Parity status of each function is recorded in its comment ("pinned by ...").
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "mbd_oracle_internal.h"

/* ------------------------------------------------------------------------- */
/* Compensated summation (Neumaier).                                         */
/* ------------------------------------------------------------------------- */
void ksum_add(orc_sum *k, double x) {
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x; else k->c += (x - t) + k->s;
    k->s = t;
}
double ksum_get(const orc_sum *k) { return k->s + k->c; }

/* ------------------------------------------------------------------------- */
/* Imaginary-frequency grid (Sec. 3.3): Gauss-Legendre on [-1,1] mapped by    */
/* x -> 0.6 (1+x)/(1-x).  Pinned by numpy's leggauss and by the closed-form  */
/* Casimir-Polder integral of a single oscillator.                           */
/* ------------------------------------------------------------------------- */
int orc_gauss_legendre(int n, double *x, double *w) {
    if (n < 1) return ORC_ERR_INPUT;
    for (int i = 0; i < n; ++i) {
        /* Newton on P_n, started from the Tricomi-like guess for the i-th root */
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < n; ++k) {           /* (k+1) P_{k+1} = (2k+1) z P_k - k P_{k-1} */
                double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1; p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);   /* P_n' from P_n, P_{n-1} */
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the converged root */
        double p0 = 1.0, p1 = z;
        for (int k = 1; k < n; ++k) {
            double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
            p0 = p1; p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[n - 1 - i] = z;                            /* ascending order */
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return ORC_OK;
}

/* u[0] = 0 with weight 0 (the static point, reading R7); u[k], k = 1..n_freq, the
 * mapped nodes with weights w_k * dU/dx = w_k * 1.2/(1-x_k)^2. */
int orc_freq_grid(int n_freq, double *u, double *wu) {
    double *x = (double *)malloc(sizeof(double) * n_freq);
    double *w = (double *)malloc(sizeof(double) * n_freq);
    int rc = orc_gauss_legendre(n_freq, x, w);
    u[0] = 0.0; wu[0] = 0.0;
    for (int k = 0; k < n_freq; ++k) {
        u[k + 1] = 0.6 * (1.0 + x[k]) / (1.0 - x[k]);
        wu[k + 1] = w[k] * 1.2 / ((1.0 - x[k]) * (1.0 - x[k]));
    }
    free(x); free(w);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Dipole tensors.  Each is written as T_ab = A(r) delta_ab + Bf(r) r_a r_b.  */
/* ------------------------------------------------------------------------- */

/* Bare dipole tensor, Eq. (dipole) explicit form (reading R1).
 * Pinned by central differences of -grad grad (1/r). */
void orc_T_bare(const double *r, double *T) {
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], rr = sqrt(r2);
    double r5 = r2 * r2 * rr;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            T[3 * a + b] = ((a == b ? r2 : 0.0) - 3.0 * r[a] * r[b]) / r5;
}

/* Gaussian-Gaussian dipole tensor, Eq. (tgg), with s = sqrt(sigma_i^2 + sigma_j^2):
 *   T^GG = (erf z - Theta) T + 2 z^2 Theta r r / r^5,  Theta = 2z/sqrt(pi) exp(-z^2), z = r/s.
 * Pinned by: T^GG -> T as s -> 0; central differences of -grad grad (erf(r/s)/r);
 * T^GG = T - T^erfc(gamma = 1/s). */
void orc_T_gg(const double *r, double s, double *T) {
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], rr = sqrt(r2);
    double r5 = r2 * r2 * rr, z = rr / s;
    double th = 2.0 * z / sqrt(ORC_PI) * exp(-z * z);
    double f1 = erf(z) - th, f2 = 2.0 * z * z * th;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double t = ((a == b ? r2 : 0.0) - 3.0 * r[a] * r[b]) / r5;
            T[3 * a + b] = f1 * t + f2 * r[a] * r[b] / r5;
        }
}

/* Short-range (erfc-screened) dipole tensor, Eq. (terfc) with the numerator read as
 * (-r_a r_b C + delta r^2 B) (reading R2).  Pinned by T^erfc -> T as gamma -> 0 and
 * central differences of -grad grad (erfc(gamma r)/r). */
void orc_T_erfc(const double *r, double gamma, double *T) {
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], rr = sqrt(r2);
    double r5 = r2 * r2 * rr, x = gamma * rr;
    double e = 2.0 * x / sqrt(ORC_PI) * exp(-x * x);
    double B = erfc(x) + e;
    double C = 3.0 * erfc(x) + e * (3.0 + 2.0 * x * x);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            T[3 * a + b] = (-r[a] * r[b] * C + (a == b ? r2 * B : 0.0)) / r5;
}

/* Fermi damping, Eq. (fermi-damping): f = 1/(1 + exp(-a (R/(s_R (Ri+Rj)) - 1))). */
double orc_fermi(double rho, double rsum, double sr, double a) {
    return 1.0 / (1.0 + exp(-a * (rho / (sr * rsum) - 1.0)));
}

/* Radial coefficients of T^GG and their derivatives, used by the gradients.
 * T^GG_ab = A delta_ab + Bf r_a r_b with A = F1/r^3, Bf = (F2 - 3 F1)/r^5,
 * F1 = erf z - Theta, F2 = 2 z^2 Theta.  dF1/dz = 2 z Theta, d(F2-3F1)/dz = -4 z^3 Theta.
 * Outputs A, Bf, dA/dr, dBf/dr, dA/ds, dBf/ds.  Pinned by central differences of the
 * tensor with respect to r and s. */
static void tgg_radial(double rr, double s, double *A, double *Bf, double *dA, double *dBf,
                       double *dAs, double *dBfs) {
    double z = rr / s, th = 2.0 * z / sqrt(ORC_PI) * exp(-z * z);
    double F1 = erf(z) - th, G = 2.0 * z * z * th - 3.0 * F1;
    double r3 = rr * rr * rr, r5 = r3 * rr * rr;
    *A = F1 / r3;
    *Bf = G / r5;
    *dA = 2.0 * z * th / (s * r3) - 3.0 * F1 / (r3 * rr);
    *dBf = -4.0 * z * z * z * th / (s * r5) - 5.0 * G / (r5 * rr);
    *dAs = -2.0 * z * z * th / (s * r3);
    *dBfs = 4.0 * z * z * z * z * th / (s * r5);
}

/* dT_ab/dr_c for a tensor A delta_ab + Bf r_a r_b with radial derivatives dA, dBf. */
void radial_tensor_deriv(const double *r, double rr, double A, double Bf, double dA,
                                double dBf, double *dT /* [3][3][3]: c, a, b */) {
    (void)A;
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                dT[9 * c + 3 * a + b] = (a == b ? dA * r[c] / rr : 0.0)
                                      + dBf * r[c] / rr * r[a] * r[b]
                                      + Bf * ((a == c ? r[b] : 0.0) + (b == c ? r[a] : 0.0));
}

/* Exposed for the derivative pins: dT^GG/dr_c and dT^GG/ds. */
void orc_T_gg_deriv(const double *r, double s, double *dT_dr /*27*/, double *dT_ds /*9*/) {
    double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double A, Bf, dA, dBf, dAs, dBfs;
    tgg_radial(rr, s, &A, &Bf, &dA, &dBf, &dAs, &dBfs);
    radial_tensor_deriv(r, rr, A, Bf, dA, dBf, dT_dr);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) dT_ds[3 * a + b] = (a == b ? dAs : 0.0) + dBfs * r[a] * r[b];
}

/* ------------------------------------------------------------------------- */
/* Dense linear algebra.                                                      */
/* ------------------------------------------------------------------------- */

/* Gauss-Jordan inversion with partial pivoting.  Pinned by numpy.linalg.inv and
 * by A A^{-1} = I. */
int orc_gauss_jordan_inverse(int n, const double *A, double *Ainv) {
    int m = 2 * n;
    double *W = (double *)malloc(sizeof(double) * (size_t)n * m);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j)
            W[(size_t)i * m + j] = j < n ? A[(size_t)i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (fabs(W[(size_t)i * m + col]) > fabs(W[(size_t)piv * m + col])) piv = i;
        if (W[(size_t)piv * m + col] == 0.0) { free(W); return ORC_ERR_SINGULAR; }
        if (piv != col)
            for (int j = 0; j < m; ++j) {
                double t = W[(size_t)col * m + j];
                W[(size_t)col * m + j] = W[(size_t)piv * m + j];
                W[(size_t)piv * m + j] = t;
            }
        double d = W[(size_t)col * m + col];
        for (int j = 0; j < m; ++j) W[(size_t)col * m + j] /= d;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) {
            if (i == col) continue;
            double f = W[(size_t)i * m + col];
            if (f == 0.0) continue;
            for (int j = 0; j < m; ++j) W[(size_t)i * m + j] -= f * W[(size_t)col * m + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[(size_t)i * n + j] = W[(size_t)i * m + n + j];
    free(W);
    return ORC_OK;
}

/* Cyclic Jacobi eigendecomposition of a real symmetric matrix: A = V diag(lam) V^T,
 * eigenvectors in the columns of V.  Sweeps until the off-diagonal Frobenius norm is
 * below 1e-15 of the full norm.  Pinned by numpy.linalg.eigh and A V = V diag(lam). */
int orc_jacobi_eigh(int n, const double *Ain, double *lam, double *V) {
    double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
    memcpy(A, Ain, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = (i == j);
    double fro = 0.0;
    for (size_t k = 0; k < (size_t)n * n; ++k) fro += A[k] * A[k];
    int rc = ORC_ERR_NOT_CONVERGED;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += 2.0 * A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off <= 1e-30 * fro) { rc = ORC_OK; break; }
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {          /* columns p, q */
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {          /* rows p, q */
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                A[(size_t)p * n + q] = 0.0; A[(size_t)q * n + p] = 0.0;
                for (int k = 0; k < n; ++k) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
    free(A);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Method steps.                                                              */
/* ------------------------------------------------------------------------- */

/* TS volume scaling, Eq. (ts-scaling): alpha0 = alpha0_ref v, omega = 4 C6_ref /
 * (3 alpha0_ref^2) (independent of v), R_vdW = R_ref v^(1/3). */
void orc_ts_scaling(int N, const double *a0ref, const double *c6ref, const double *rref,
                    const double *ratio, double *a0, double *om, double *rv) {
    for (int i = 0; i < N; ++i) {
        a0[i] = a0ref[i] * ratio[i];
        om[i] = 4.0 * c6ref[i] / (3.0 * a0ref[i] * a0ref[i]);
        rv[i] = rref[i] * cbrt(ratio[i]);
    }
}

/* Dynamic polarizability, Eq. (dyn-pol), and Mayer width, Eq. (mayer). */
double alpha_iu(double a0, double om, double u) { return a0 / (1.0 + u * u / (om * om)); }
double mayer_sigma(double al) { return cbrt(sqrt(2.0 / ORC_PI) * al / 3.0); }

/* SCS matrix at one frequency, Eq. (scs) with Eq. (scs-sr-dipole):
 * M = diag(1/alpha_i) x I3 + (1 - f_ij) T^GG_ij for i != j, row-major n x n, n = 3N. */
void orc_scs_matrix(int N, const double *R, const double *al, const double *rv, double beta,
                    double a, double *M) {
    int n = 3 * N;
    memset(M, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < N; ++i) {
        for (int c = 0; c < 3; ++c) M[(size_t)(3 * i + c) * n + 3 * i + c] = 1.0 / al[i];
        double si = mayer_sigma(al[i]);
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            double r[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
            double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            double sj = mayer_sigma(al[j]);
            double T[9];
            orc_T_gg(r, sqrt(si * si + sj * sj), T);
            double f = orc_fermi(rr, rv[i] + rv[j], beta, a);
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y)
                    M[(size_t)(3 * i + x) * n + 3 * j + y] = (1.0 - f) * T[3 * x + y];
        }
    }
}

/* Contraction, Eq. (contraction): alpha_bar_i = 1/3 sum_a sum_j Abar[ia, ja]. */
static double contract_atom(int N, const double *Ab, int i) {
    int n = 3 * N;
    orc_sum s = {0, 0};
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < N; ++j) ksum_add(&s, Ab[(size_t)(3 * i + a) * n + 3 * j + a]);
    return ksum_get(&s) / 3.0;
}

/* Screening at every grid point: alpha_bar[k*N + i] for k = 0..n_freq (u[0] = 0).
 * Optionally keeps the full inverse Abar[k] (n x n each) for the gradients.
 * Pinned by the two-atom closed form and by isolated atoms (alpha_bar = alpha). */
int orc_scs(int N, const double *R, const double *a0, const double *om, const double *rv,
            double beta, double a, int n_freq, const double *u, double *alpha_bar,
            double *Abar_keep) {
    int n = 3 * N, rc = ORC_OK;
    for (int k = 0; k <= n_freq; ++k) {
        double *al = (double *)malloc(sizeof(double) * N);
        double *M = (double *)malloc(sizeof(double) * (size_t)n * n);
        double *Ai = Abar_keep ? Abar_keep + (size_t)k * n * n
                               : (double *)malloc(sizeof(double) * (size_t)n * n);
        for (int i = 0; i < N; ++i) al[i] = alpha_iu(a0[i], om[i], u[k]);
        orc_scs_matrix(N, R, al, rv, beta, a, M);
        int r2 = orc_gauss_jordan_inverse(n, M, Ai);
        if (r2) rc = r2;
        for (int i = 0; i < N; ++i) alpha_bar[(size_t)k * N + i] = contract_atom(N, Ai, i);
        if (!Abar_keep) free(Ai);
        free(M); free(al);
    }
    return rc;
}

/* Screened oscillator parameters, Eqs. (casimir-polder) and (scale-rvdw-scs):
 * abar0 = alpha_bar(0); C6bar = 3/pi sum_k w_k alpha_bar(u_k)^2; omega_bar =
 * 4 C6bar / (3 abar0^2); Rbar = R_vdW (abar0/alpha0)^(1/3). */
int orc_screened_params(int N, int n_freq, const double *alpha_bar, const double *wu,
                        const double *a0, const double *rv, double *abar0, double *c6bar,
                        double *ombar, double *rbar) {
    int rc = ORC_OK;
    for (int i = 0; i < N; ++i) {
        orc_sum s = {0, 0};
        for (int k = 1; k <= n_freq; ++k) {
            double ab = alpha_bar[(size_t)k * N + i];
            ksum_add(&s, wu[k] * ab * ab);
        }
        abar0[i] = alpha_bar[i];
        c6bar[i] = 3.0 / ORC_PI * ksum_get(&s);
        if (!(abar0[i] > 0.0) || !(c6bar[i] > 0.0)) rc = ORC_ERR_SCS_NEG_ALPHA;
        ombar[i] = 4.0 * c6bar[i] / (3.0 * abar0[i] * abar0[i]);
        rbar[i] = rv[i] * cbrt(abar0[i] / a0[i]);
    }
    return rc;
}

/* Coupled-oscillator matrix, Eq. (q-matrix), finite system, with T^lr = g(Rbar) T
 * (reading R5):  Q_ij = delta_ij om_i^2 I + om_i om_j sqrt(a_i a_j) g_ij T(R_j - R_i). */
void orc_mbd_q(int N, const double *R, const double *a0, const double *om, const double *rdamp,
               double beta, double a, double *Q) {
    int n = 3 * N;
    memset(Q, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < N; ++i) {
        for (int c = 0; c < 3; ++c) Q[(size_t)(3 * i + c) * n + 3 * i + c] = om[i] * om[i];
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            double r[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
            double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            double T[9];
            orc_T_bare(r, T);
            double g = orc_fermi(rr, rdamp[i] + rdamp[j], beta, a);
            double pre = om[i] * om[j] * sqrt(a0[i] * a0[j]) * g;
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) Q[(size_t)(3 * i + x) * n + 3 * j + y] = pre * T[3 * x + y];
        }
    }
}

/* Energy from Q, Eqs. (diagonalization) and (mbd-energy):
 * E = 1/2 sum_k sqrt(lambda_k) - 3/2 sum_i om_i.  Returns ORC_ERR_NEG_EIGENVALUE when
 * Q is not positive definite (the polarization catastrophe, Sec. 2.1).  Optionally
 * returns Z = C Lambda^{-1/2} C^T (n x n) for the gradient.  Pinned by the two-oscillator
 * closed form and by the second-order (pairwise) limit, Eq. (pairwise). */
int orc_energy_from_q(int N, const double *Q, const double *om, double *E, double *Zout) {
    int n = 3 * N;
    double *lam = (double *)malloc(sizeof(double) * n);
    double *V = (double *)malloc(sizeof(double) * (size_t)n * n);
    int rc = orc_jacobi_eigh(n, Q, lam, V);
    double lmin = lam[0];
    for (int k = 1; k < n; ++k) lmin = lam[k] < lmin ? lam[k] : lmin;
    if (rc == ORC_OK && !(lmin > 0.0)) rc = ORC_ERR_NEG_EIGENVALUE;
    if (rc == ORC_OK) {
        orc_sum s = {0, 0};
        for (int k = 0; k < n; ++k) ksum_add(&s, 0.5 * sqrt(lam[k]));
        for (int i = 0; i < N; ++i) ksum_add(&s, -1.5 * om[i]);
        *E = ksum_get(&s);
        if (Zout) {
            for (int p = 0; p < n; ++p)
                for (int q = 0; q < n; ++q) {
                    double z = 0.0;
                    for (int k = 0; k < n; ++k)
                        z += V[(size_t)p * n + k] * V[(size_t)q * n + k] / sqrt(lam[k]);
                    Zout[(size_t)p * n + q] = z;
                }
        }
    }
    free(lam); free(V);
    return rc;
}

/* MBD energy of given oscillators (no screening): alpha0, omega and damping radii in.
 * Used by the closed-form pins and as the last stage of the full method. */
int orc_mbd_energy(int N, const double *R, const double *a0, const double *om,
                   const double *rdamp, double beta, double a, double *E) {
    int n = 3 * N;
    double *Q = (double *)malloc(sizeof(double) * (size_t)n * n);
    orc_mbd_q(N, R, a0, om, rdamp, beta, a, Q);
    int rc = orc_energy_from_q(N, Q, om, E, NULL);
    free(Q);
    return rc;
}

/* MBD energy by the imaginary-frequency log formula, Eq. (log-formula), and its many-body
 * orders, Eq. (rpa), for given oscillators (alpha0, omega) with damping radii rdamp:
 *   E = 1/(2 pi) int_0^inf du ln det(I + A(u)),   A(u) = alpha(u)^{1/2} T^lr alpha(u)^{1/2}
 * (the Hermitian form the paper allows under the trace), alpha_i(u) = alpha0_i/(1 + u^2/om_i^2),
 * T^lr_ij = g_ij T(R_j - R_i) as in Q (reading R5), zero diagonal blocks;
 *   E^(m) = -1/(2 pi) int du (-1)^m/m Tr A(u)^m,   m = 2..max_order -> orders[m - 2].
 * The integral runs over the n_freq Gauss-Legendre nodes u_k > 0 of Sec. 3.3 with their
 * weights.  ln det(I + A) = sum ln(1 + lambda) and Tr A^m = sum lambda^m over the
 * eigenvalues of A (Jacobi).  ORC_ERR_NEG_EIGENVALUE if I + A is not positive definite. */
int orc_mbd_log_energy(int N, const double *R, const double *a0, const double *om, const double *rdamp,
                       double beta, double a, int nf, int max_order, double *E, double *orders) {
    if (N < 1 || nf < 1 || max_order < 1) return ORC_ERR_INPUT;
    int n = 3 * N;
    double *u = malloc(sizeof(double) * (nf + 1)), *wu = malloc(sizeof(double) * (nf + 1));
    double *A = malloc(sizeof(double) * (size_t)n * n), *V = malloc(sizeof(double) * (size_t)n * n);
    double *lam = malloc(sizeof(double) * n), *al = malloc(sizeof(double) * N);
    orc_sum sE = {0, 0};
    orc_sum *so = calloc(max_order + 1, sizeof(orc_sum));
    int rc = orc_freq_grid(nf, u, wu);
    for (int k = 1; k <= nf && rc == ORC_OK; ++k) {
        for (int i = 0; i < N; ++i) al[i] = alpha_iu(a0[i], om[i], u[k]);
        memset(A, 0, sizeof(double) * (size_t)n * n);
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                if (j == i) continue;
                double r[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
                double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                double T[9];
                orc_T_bare(r, T);
                double pre = sqrt(al[i] * al[j]) * orc_fermi(rr, rdamp[i] + rdamp[j], beta, a);
                for (int x = 0; x < 3; ++x)
                    for (int y = 0; y < 3; ++y) A[(size_t)(3 * i + x) * n + 3 * j + y] = pre * T[3 * x + y];
            }
        rc = orc_jacobi_eigh(n, A, lam, V);
        for (int p = 0; p < n && rc == ORC_OK; ++p) {
            if (!(1.0 + lam[p] > 0.0)) { rc = ORC_ERR_NEG_EIGENVALUE; break; }
            ksum_add(&sE, wu[k] * log1p(lam[p]));
            double lp = lam[p];   /* lambda^m */
            for (int m = 2; m <= max_order; ++m) {
                lp *= lam[p];
                ksum_add(&so[m], wu[k] * ((m % 2 == 0) ? -lp : lp) / m);
            }
        }
    }
    if (rc == ORC_OK) {
        *E = ksum_get(&sE) / (2.0 * ORC_PI);
        for (int m = 2; m <= max_order; ++m) orders[m - 2] = ksum_get(&so[m]) / (2.0 * ORC_PI);
    }
    free(u); free(wu); free(A); free(V); free(lam); free(al); free(so);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Full MBD@rsSCS energy (finite) and its gradients.                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    int N, n, nf;
    const double *R;
    double beta, a;
    double *a0, *om, *rv;           /* TS-scaled */
    double *u, *wu;                 /* grid, nf+1 */
    double *alpha_bar;              /* (nf+1) x N */
    double *Abar;                   /* (nf+1) x n x n, full screened polarizability */
    double *abar0, *c6bar, *ombar, *rbar;
    double *Q, *Z;                  /* Z = Q^{-1/2} */
    double E;
} orc_state;

static void state_free(orc_state *S) {
    free(S->a0); free(S->om); free(S->rv); free(S->u); free(S->wu); free(S->alpha_bar);
    free(S->Abar); free(S->abar0); free(S->c6bar); free(S->ombar); free(S->rbar);
    free(S->Q); free(S->Z);
}

static int state_forward(orc_state *S, int N, const double *R, const double *a0ref,
                         const double *c6ref, const double *rref, const double *ratio,
                         double beta, double a, int nf, int keep) {
    memset(S, 0, sizeof(*S));
    S->N = N; S->n = 3 * N; S->nf = nf; S->R = R; S->beta = beta; S->a = a;
    int n = S->n;
    S->a0 = malloc(sizeof(double) * N); S->om = malloc(sizeof(double) * N);
    S->rv = malloc(sizeof(double) * N);
    S->u = malloc(sizeof(double) * (nf + 1)); S->wu = malloc(sizeof(double) * (nf + 1));
    S->alpha_bar = malloc(sizeof(double) * (size_t)(nf + 1) * N);
    S->abar0 = malloc(sizeof(double) * N); S->c6bar = malloc(sizeof(double) * N);
    S->ombar = malloc(sizeof(double) * N); S->rbar = malloc(sizeof(double) * N);
    S->Q = malloc(sizeof(double) * (size_t)n * n);
    if (keep) {
        S->Abar = malloc(sizeof(double) * (size_t)(nf + 1) * n * n);
        S->Z = malloc(sizeof(double) * (size_t)n * n);
    }
    orc_ts_scaling(N, a0ref, c6ref, rref, ratio, S->a0, S->om, S->rv);
    orc_freq_grid(nf, S->u, S->wu);
    int rc = orc_scs(N, R, S->a0, S->om, S->rv, beta, a, nf, S->u, S->alpha_bar, S->Abar);
    if (rc) return rc;
    rc = orc_screened_params(N, nf, S->alpha_bar, S->wu, S->a0, S->rv, S->abar0, S->c6bar,
                             S->ombar, S->rbar);
    if (rc) return rc;
    orc_mbd_q(N, R, S->abar0, S->ombar, S->rbar, beta, a, S->Q);
    return orc_energy_from_q(N, S->Q, S->ombar, &S->E, S->Z);
}

/* Energy only.  detail (optional): alpha_bar[(nf+1)N], c6bar[N], omega_bar[N], rbar[N]. */
int orc_mbd_rsscs_energy(int N, const double *R, const double *a0ref, const double *c6ref,
                         const double *rref, const double *ratio, double beta, double a,
                         int nf, double *E, double *detail) {
    orc_state S;
    int rc = state_forward(&S, N, R, a0ref, c6ref, rref, ratio, beta, a, nf, 0);
    if (rc == ORC_OK) *E = S.E;
    if (detail && S.alpha_bar) {
        memcpy(detail, S.alpha_bar, sizeof(double) * (size_t)(nf + 1) * N);
        memcpy(detail + (size_t)(nf + 1) * N, S.c6bar, sizeof(double) * N);
        memcpy(detail + (size_t)(nf + 2) * N, S.ombar, sizeof(double) * N);
        memcpy(detail + (size_t)(nf + 3) * N, S.rbar, sizeof(double) * N);
    }
    state_free(&S);
    return rc;
}

/* Derivative of one SCS off-diagonal block B_ij = (1-f_ij) T^GG(r, s) at frequency u,
 * with r = R_j - R_i, with respect to the elementary inputs of the pair.
 * Outputs: dB/dr_c [27], dB/dalpha_i(u) [9], dB/dalpha_j(u) [9], dB/dS [9] where
 * S = R_vdW,i + R_vdW,j. */
void scs_block_derivs(const double *r, double al_i, double al_j, double rsum,
                             double beta, double a, double *dBdr, double *dBdai,
                             double *dBdaj, double *dBdS) {
    double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double si = mayer_sigma(al_i), sj = mayer_sigma(al_j), s = sqrt(si * si + sj * sj);
    double T[9], dTdr[27], dTds[9];
    orc_T_gg(r, s, T);
    orc_T_gg_deriv(r, s, dTdr, dTds);
    double f = orc_fermi(rr, rsum, beta, a);
    double eta = rr / (beta * rsum), dfdeta = a * f * (1.0 - f);
    double dfdr = dfdeta / (beta * rsum), dfdS = -dfdeta * eta / rsum;
    /* s = sqrt(si^2 + sj^2), sigma = (sqrt(2/pi) alpha / 3)^(1/3) -> dsigma/dalpha = sigma/(3 alpha) */
    double dsdai = si / s * si / (3.0 * al_i), dsdaj = sj / s * sj / (3.0 * al_j);
    for (int k = 0; k < 9; ++k) {
        dBdai[k] = (1.0 - f) * dTds[k] * dsdai;
        dBdaj[k] = (1.0 - f) * dTds[k] * dsdaj;
        dBdS[k] = -dfdS * T[k];
    }
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 9; ++k)
            dBdr[9 * c + k] = (1.0 - f) * dTdr[9 * c + k] - dfdr * r[c] / rr * T[k];
}

/* Derivative of one MBD off-diagonal block P_ij = g_ij T(r) (without the c_i c_j
 * prefactor) with respect to r_c [27] and to S = Rbar_i + Rbar_j [9]. */
static void mbd_block_derivs(const double *r, double rsum, double beta, double a,
                             double *P, double *dPdr, double *dPdS) {
    double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double T[9], dT[27];
    orc_T_bare(r, T);
    double r3 = rr * rr * rr;
    radial_tensor_deriv(r, rr, 1.0 / r3, -3.0 / (r3 * rr * rr), -3.0 / (r3 * rr),
                        15.0 / (r3 * r3), dT);
    double g = orc_fermi(rr, rsum, beta, a);
    double eta = rr / (beta * rsum), dgdeta = a * g * (1.0 - g);
    double dgdr = dgdeta / (beta * rsum), dgdS = -dgdeta * eta / rsum;
    for (int k = 0; k < 9; ++k) { P[k] = g * T[k]; dPdS[k] = dgdS * T[k]; }
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 9; ++k) dPdr[9 * c + k] = g * dT[9 * c + k] + dgdr * r[c] / rr * T[k];
}

/* Exposed for pins: the bare-T derivative used above, dT/dr_c [27]. */
void orc_T_bare_deriv(const double *r, double *dT) {
    double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]), r3 = rr * rr * rr;
    radial_tensor_deriv(r, rr, 1.0 / r3, -3.0 / (r3 * rr * rr), -3.0 / (r3 * rr),
                        15.0 / (r3 * r3), dT);
}

/* TS-scaling chain (Eq. ts-scaling) from adjoints of (alpha0, omega, R_vdW) to the
 * adjoints of (alpha0_ref, C6_ref, R_ref, ratio), layout gp[4][N]. */
void ts_chain(int N, const double *a0ref, const double *c6ref, const double *rref,
                     const double *ratio, const double *g_a0, const double *g_om,
                     const double *g_rv, double *gp) {
    for (int i = 0; i < N; ++i) {
        double v = ratio[i];
        gp[i] = g_a0[i] * v - g_om[i] * 8.0 * c6ref[i] / (3.0 * a0ref[i] * a0ref[i] * a0ref[i]);
        gp[N + i] = g_om[i] * 4.0 / (3.0 * a0ref[i] * a0ref[i]);
        gp[2 * N + i] = g_rv[i] * cbrt(v);
        gp[3 * N + i] = g_a0[i] * a0ref[i] + g_rv[i] * rref[i] / (3.0 * cbrt(v) * cbrt(v));
    }
}

/* Forward-mode gradient, one elementary input at a time (the way the paper computes
 * gradients, Sec. 3.1), using the paper's fused SCS formula, Eq. (scs-gradient):
 * for a parameter X of atom j, with A the derivative of block-row j of the SCS matrix,
 *   d alpha_bar_i = -1/3 sum_ab ( B_{ia,jb} sum_k Abar_{ka,jb} + Abar_{jb,ia} sum_k B_{jb,ka} ),
 *   B = Abar A.
 * Reading: A is the row part of dM; the column part is A^T; the diagonal block jj
 * (which belongs to both) is halved in each so that dM = A + A^T exactly.  The
 * second term is then sum_b Abar_{ia,jb} sum_k (A Abar)_{jb,ka}.
 * MBD part, Eq. (mbd-gradient), with reading R8: dE = 1/4 sum Z_pq dQ_qp - 3/2 sum domega.
 * Cost O(N^4): tiny systems only.  Pinned by central differences of the energy. */
static int grad_forward(orc_state *S, const double *a0ref, const double *c6ref,
                        const double *rref, const double *ratio, double *gR, double *gp) {
    int N = S->N, n = S->n, nf = S->nf;
    double *g_a0 = calloc(N, sizeof(double)), *g_om = calloc(N, sizeof(double));
    double *g_rv = calloc(N, sizeof(double));
    int n_in = 6 * N;  /* R_j (3), alpha0_j, omega_j, R_vdW,j */
#pragma omp parallel for schedule(dynamic)
    for (int in = 0; in < n_in; ++in) {
        int j = in / 6, kind = in % 6;
        double *Arow = malloc(sizeof(double) * 3 * n);     /* block-row j of dM: 3 x n */
        double *dab = malloc(sizeof(double) * (size_t)(nf + 1) * N);
        double *BA = malloc(sizeof(double) * 3 * n);
        for (int k = 0; k <= nf; ++k) {
            double u = S->u[k];
            const double *Ab = S->Abar + (size_t)k * n * n;
            memset(Arow, 0, sizeof(double) * 3 * n);
            double alj = alpha_iu(S->a0[j], S->om[j], u);
            double dalj = 0.0;  /* d alpha_j(u) / dX */
            if (kind == 3) dalj = 1.0 / (1.0 + u * u / (S->om[j] * S->om[j]));
            if (kind == 4) {
                double q = 1.0 + u * u / (S->om[j] * S->om[j]);
                dalj = S->a0[j] * 2.0 * u * u / (S->om[j] * S->om[j] * S->om[j]) / (q * q);
            }
            /* diagonal block jj: d(1/alpha_j) I, halved (reading above) */
            for (int c = 0; c < 3; ++c) Arow[(size_t)c * n + 3 * j + c] = 0.5 * (-dalj / (alj * alj));
            for (int m = 0; m < N; ++m) {
                if (m == j) continue;
                double r[3] = {S->R[3 * m] - S->R[3 * j], S->R[3 * m + 1] - S->R[3 * j + 1],
                               S->R[3 * m + 2] - S->R[3 * j + 2]};
                double alm = alpha_iu(S->a0[m], S->om[m], u);
                double dBdr[27], dBda[9], dBdb[9], dBdS[9];
                scs_block_derivs(r, alj, alm, S->rv[j] + S->rv[m], S->beta, S->a, dBdr, dBda,
                                 dBdb, dBdS);
                double d[9] = {0};
                if (kind < 3) for (int t = 0; t < 9; ++t) d[t] = -dBdr[9 * kind + t];  /* dr/dR_j = -1 */
                if (kind == 3 || kind == 4) for (int t = 0; t < 9; ++t) d[t] = dBda[t] * dalj;
                if (kind == 5) for (int t = 0; t < 9; ++t) d[t] = dBdS[t];
                for (int x = 0; x < 3; ++x)
                    for (int y = 0; y < 3; ++y) Arow[(size_t)x * n + 3 * m + y] = d[3 * x + y];
            }
            /* Bp = A Abar (3 x n, rows jb);  cs[a][b] = sum_k Abar_{jb,ka};
             * rs[a][b] = sum_k Bp_{jb,ka}.  With B = Bp^T the two terms of the fused
             * formula are B_{ia,jb} cs[a][b] and Abar_{ia,jb} rs[a][b]. */
            for (int b = 0; b < 3; ++b)
                for (int q = 0; q < n; ++q) {
                    double t = 0.0;
                    for (int q2 = 0; q2 < n; ++q2) t += Arow[(size_t)b * n + q2] * Ab[(size_t)q2 * n + q];
                    BA[(size_t)b * n + q] = t;
                }
            double cs[3][3], rs[3][3];
            for (int aa = 0; aa < 3; ++aa)
                for (int b = 0; b < 3; ++b) {
                    double c1 = 0.0, c2 = 0.0;
                    for (int kk = 0; kk < N; ++kk) {
                        c1 += Ab[(size_t)(3 * j + b) * n + 3 * kk + aa];
                        c2 += BA[(size_t)b * n + 3 * kk + aa];
                    }
                    cs[aa][b] = c1; rs[aa][b] = c2;
                }
            for (int i = 0; i < N; ++i) {
                double acc = 0.0;
                for (int aa = 0; aa < 3; ++aa)
                    for (int b = 0; b < 3; ++b) {
                        int p = 3 * i + aa;
                        acc += BA[(size_t)b * n + p] * cs[aa][b] + Ab[(size_t)p * n + 3 * j + b] * rs[aa][b];
                    }
                dab[(size_t)k * N + i] = -acc / 3.0;
            }
        }
        /* chain through Eq. (casimir-polder), Eq. (scale-rvdw-scs) to dQ */
        double *dom = malloc(sizeof(double) * N), *da0b = malloc(sizeof(double) * N);
        double *drb = malloc(sizeof(double) * N);
        for (int i = 0; i < N; ++i) {
            double dc6 = 0.0;
            for (int k = 1; k <= nf; ++k)
                dc6 += 3.0 / ORC_PI * S->wu[k] * 2.0 * S->alpha_bar[(size_t)k * N + i] * dab[(size_t)k * N + i];
            double ab0 = S->abar0[i];
            da0b[i] = dab[i];
            dom[i] = 4.0 * dc6 / (3.0 * ab0 * ab0) - 8.0 * S->c6bar[i] * da0b[i] / (3.0 * ab0 * ab0 * ab0);
            double x = ab0 / S->a0[i];
            double dx = da0b[i] / S->a0[i] - (kind == 3 && i == j ? ab0 / (S->a0[i] * S->a0[i]) : 0.0);
            drb[i] = (kind == 5 && i == j ? cbrt(x) : 0.0) + S->rv[i] * dx / (3.0 * cbrt(x) * cbrt(x));
        }
        /* dE = 1/4 sum_pq Z_pq dQ_pq - 3/2 sum domega */
        orc_sum acc = {0, 0};
        for (int i = 0; i < N; ++i) {
            for (int c = 0; c < 3; ++c)
                ksum_add(&acc, 0.25 * S->Z[(size_t)(3 * i + c) * n + 3 * i + c] * 2.0 * S->ombar[i] * dom[i]);
            ksum_add(&acc, -1.5 * dom[i]);
            double ci = S->ombar[i] * sqrt(S->abar0[i]);
            double dci = dom[i] * sqrt(S->abar0[i]) + S->ombar[i] * da0b[i] / (2.0 * sqrt(S->abar0[i]));
            for (int m = 0; m < N; ++m) {
                if (m == i) continue;
                double r[3] = {S->R[3 * m] - S->R[3 * i], S->R[3 * m + 1] - S->R[3 * i + 1],
                               S->R[3 * m + 2] - S->R[3 * i + 2]};
                double cm = S->ombar[m] * sqrt(S->abar0[m]);
                double dcm = dom[m] * sqrt(S->abar0[m]) + S->ombar[m] * da0b[m] / (2.0 * sqrt(S->abar0[m]));
                double P[9], dPdr[27], dPdS[9];
                mbd_block_derivs(r, S->rbar[i] + S->rbar[m], S->beta, S->a, P, dPdr, dPdS);
                double drsum = drb[i] + drb[m];
                double dr[3] = {0, 0, 0};
                if (kind < 3) { if (m == j) dr[kind] += 1.0; if (i == j) dr[kind] -= 1.0; }
                for (int x = 0; x < 3; ++x)
                    for (int y = 0; y < 3; ++y) {
                        int t = 3 * x + y;
                        double dP = dPdS[t] * drsum + dPdr[t] * dr[0] + dPdr[9 + t] * dr[1] + dPdr[18 + t] * dr[2];
                        double dq = (dci * cm + ci * dcm) * P[t] + ci * cm * dP;
                        ksum_add(&acc, 0.25 * S->Z[(size_t)(3 * i + x) * n + 3 * m + y] * dq);
                    }
            }
        }
        double dE = ksum_get(&acc);
        if (kind < 3) gR[3 * j + kind] = dE;
        if (kind == 3) g_a0[j] = dE;
        if (kind == 4) g_om[j] = dE;
        if (kind == 5) g_rv[j] = dE;
        free(dom); free(da0b); free(drb);
        free(Arow); free(dab); free(BA);
    }
    if (gp) ts_chain(N, a0ref, c6ref, rref, ratio, g_a0, g_om, g_rv, gp);
    free(g_a0); free(g_om); free(g_rv);
    return ORC_OK;
}

/* Adjoint (reverse-mode) gradient: one backward sweep instead of one forward sweep per
 * input.  MBD part: pair sums of Z = Q^{-1/2} against dQ; chain through the
 * Casimir-Polder step to h_i(u) = dE/d alpha_bar_i(u); then per frequency
 * V = Abar H (H_{ia,c} = h_i delta_ac), X = Abar E (E_{jb,c} = delta_bc) and
 * dE = -1/3 sum_pq dM_pq (V X^T)_pq (the same Eq. (scs) derivative dAbar = -Abar dM Abar,
 * contracted from the other side).  O(N^3) after the inverses.
 * Pinned against grad_forward and central differences. */
/* MBD part of the adjoint gradient, Eq. (mbd-gradient) with reading R8: from Z = Q^{-1/2}
 * of the coupled-oscillator matrix of the oscillators (ab0, omb) with damping radii rb,
 * dE = 1/4 sum_pq Z_pq dQ_pq - 3/2 sum d omega.  Adds dE/d omega_i (g_omb), dE/d alpha0_i
 * (g_ab0), dE/d R_damp,i (g_rb) and dE/dR_i (gR, [N][3]). */
static void mbd_pair_adjoint(int N, const double *R, const double *ab0, const double *omb,
                             const double *rb, const double *Z, double beta, double a,
                             double *g_omb, double *g_ab0, double *g_rb, double *gR) {
    int n = 3 * N;
    double *g_c = calloc(N, sizeof(double));
    for (int i = 0; i < N; ++i) {
        double zd = 0.0;
        for (int c = 0; c < 3; ++c) zd += Z[(size_t)(3 * i + c) * n + 3 * i + c];
        g_omb[i] += 0.25 * zd * 2.0 * omb[i] - 1.5;
    }
    for (int i = 0; i < N; ++i) {
        double ci = omb[i] * sqrt(ab0[i]);
        for (int m = 0; m < N; ++m) {
            if (m == i) continue;
            double r[3] = {R[3 * m] - R[3 * i], R[3 * m + 1] - R[3 * i + 1], R[3 * m + 2] - R[3 * i + 2]};
            double cm = omb[m] * sqrt(ab0[m]);
            double P[9], dPdr[27], dPdS[9];
            mbd_block_derivs(r, rb[i] + rb[m], beta, a, P, dPdr, dPdS);
            double zP = 0.0, zS = 0.0, zr[3] = {0, 0, 0};
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) {
                    double z = Z[(size_t)(3 * i + x) * n + 3 * m + y];
                    int t = 3 * x + y;
                    zP += z * P[t]; zS += z * dPdS[t];
                    for (int c = 0; c < 3; ++c) zr[c] += z * dPdr[9 * c + t];
                }
            /* ordered block (i,m): 1/4 Z_{i,m} : d(c_i c_m P_im) */
            g_c[i] += 0.25 * cm * zP;
            g_c[m] += 0.25 * ci * zP;
            g_rb[i] += 0.25 * ci * cm * zS;
            g_rb[m] += 0.25 * ci * cm * zS;
            for (int c = 0; c < 3; ++c) {          /* r = R_m - R_i */
                gR[3 * m + c] += 0.25 * ci * cm * zr[c];
                gR[3 * i + c] -= 0.25 * ci * cm * zr[c];
            }
        }
    }
    for (int i = 0; i < N; ++i) {
        double sa = sqrt(ab0[i]);
        g_omb[i] += g_c[i] * sa;
        g_ab0[i] += g_c[i] * omb[i] / (2.0 * sa);
    }
    free(g_c);
}

/* MBD part of the adjoint gradient and the chain through the screened parameters,
 * Eqs. (mbd-gradient), (casimir-polder), (scale-rvdw-scs), from Z = Q^{-1/2}:
 * gR, g_a0, g_rv (written) get the MBD pair terms and the direct parts of R_bar =
 * R_vdW (abar0/alpha0)^(1/3); h[k*N + i] = dE/d alpha_bar_i(u_k) (written) for k = 0..nf. */
void orc_mbd_chain(int N, int nf, const double *R, const double *a0, const double *rv,
                   const double *alpha_bar, const double *abar0, const double *c6bar,
                   const double *ombar, const double *rbar, const double *wu, const double *Z,
                   double beta, double a, double *h, double *g_a0, double *g_rv, double *gR) {
    double *g_ombar = calloc(N, sizeof(double)), *g_ab0 = calloc(N, sizeof(double));
    double *g_rbar = calloc(N, sizeof(double));
    memset(gR, 0, sizeof(double) * 3 * N);
    mbd_pair_adjoint(N, R, abar0, ombar, rbar, Z, beta, a, g_ombar, g_ab0, g_rbar, gR);
    for (int i = 0; i < N; ++i) {
        double ab0 = abar0[i], x = ab0 / a0[i];
        double g_c6 = g_ombar[i] * 4.0 / (3.0 * ab0 * ab0);
        double gab0 = g_ab0[i] - g_ombar[i] * 8.0 * c6bar[i] / (3.0 * ab0 * ab0 * ab0)
                    + g_rbar[i] * rv[i] / (3.0 * cbrt(x) * cbrt(x) * a0[i]);
        g_a0[i] = -g_rbar[i] * rv[i] / (3.0 * cbrt(x) * cbrt(x)) * ab0 / (a0[i] * a0[i]);
        g_rv[i] = g_rbar[i] * cbrt(x);
        h[i] = gab0;
        for (int k = 1; k <= nf; ++k)
            h[(size_t)k * N + i] = g_c6 * 3.0 / ORC_PI * wu[k] * 2.0 * alpha_bar[(size_t)k * N + i];
    }
    free(g_ombar); free(g_ab0); free(g_rbar);
}

/* SCS part of the adjoint gradient, Eq. (scs-gradient) in adjoint form: per frequency u_k,
 * with X = M^{-1} E and V = M^{-1} H (n x 3 each, X[k][p][c], V[k][p][c]; H[p][c] =
 * h_k[p/3] delta_{p%3,c}), dE = -1/3 sum_pq dM_pq (V X^T)_pq, accumulated into g_a0, g_om,
 * g_rv (through alpha_i(u) of Eq. dyn-pol and the damping radii) and gR. */
void orc_scs_adjoint_pass(int N, int nf, const double *R, const double *a0, const double *om,
                          const double *rv, const double *u, double beta, double a,
                          const double *X_all, const double *V_all, double *g_a0, double *g_om,
                          double *g_rv, double *gR) {
    int n = 3 * N;
    double *gal = malloc(sizeof(double) * N);
    for (int k = 0; k <= nf; ++k) {
        const double *X = X_all + (size_t)k * 3 * n, *V = V_all + (size_t)k * 3 * n;
        double uk = u[k];
        memset(gal, 0, sizeof(double) * N);
        /* W = V X^T; gal[i] collects dE/d alpha_i(u).  Rows i run in parallel; every
         * contribution is summed by the reduction. */
#pragma omp parallel for schedule(dynamic) reduction(+ : gal[:N], g_rv[:N], gR[:3 * N])
        for (int i = 0; i < N; ++i) {
            double ali = alpha_iu(a0[i], om[i], uk);
            double wd = 0.0;
            for (int c = 0; c < 3; ++c)
                for (int cc = 0; cc < 3; ++cc) wd += V[3 * (3 * i + c) + cc] * X[3 * (3 * i + c) + cc];
            gal[i] += -1.0 / 3.0 * wd * (-1.0 / (ali * ali));   /* d(1/alpha) = -dalpha/alpha^2 */
            for (int m = 0; m < N; ++m) {
                if (m == i) continue;
                double r[3] = {R[3 * m] - R[3 * i], R[3 * m + 1] - R[3 * i + 1], R[3 * m + 2] - R[3 * i + 2]};
                double alm = alpha_iu(a0[m], om[m], uk);
                double dBdr[27], dBda[9], dBdb[9], dBdS[9];
                scs_block_derivs(r, ali, alm, rv[i] + rv[m], beta, a, dBdr, dBda, dBdb, dBdS);
                double wa = 0.0, wb = 0.0, wS = 0.0, wr[3] = {0, 0, 0};
                for (int x = 0; x < 3; ++x)
                    for (int y = 0; y < 3; ++y) {
                        double w = 0.0;
                        for (int c = 0; c < 3; ++c) w += V[3 * (3 * i + x) + c] * X[3 * (3 * m + y) + c];
                        int t = 3 * x + y;
                        wa += w * dBda[t]; wb += w * dBdb[t]; wS += w * dBdS[t];
                        for (int cc = 0; cc < 3; ++cc) wr[cc] += w * dBdr[9 * cc + t];
                    }
                /* ordered block (i,m): depends on alpha_i, alpha_m, S_im and r = R_m - R_i */
                gal[i] += -1.0 / 3.0 * wa;
                gal[m] += -1.0 / 3.0 * wb;
                g_rv[i] += -1.0 / 3.0 * wS;
                g_rv[m] += -1.0 / 3.0 * wS;
                for (int cc = 0; cc < 3; ++cc) {
                    gR[3 * m + cc] += -1.0 / 3.0 * wr[cc];
                    gR[3 * i + cc] -= -1.0 / 3.0 * wr[cc];
                }
            }
        }
        for (int i = 0; i < N; ++i) {
            double q = 1.0 + uk * uk / (om[i] * om[i]);
            g_a0[i] += gal[i] / q;
            g_om[i] += gal[i] * a0[i] * 2.0 * uk * uk / (om[i] * om[i] * om[i]) / (q * q);
        }
    }
    free(gal);
}

/* Adjoint gradient: the MBD pair pass and chain (orc_mbd_chain), X = M^{-1} E and
 * V = M^{-1} H from the full screened polarizabilities Abar = M^{-1} of the forward pass,
 * the SCS pass (orc_scs_adjoint_pass), and the chain through the TS scaling. */
static int grad_adjoint(orc_state *S, const double *a0ref, const double *c6ref,
                        const double *rref, const double *ratio, double *gR, double *gp) {
    int N = S->N, n = S->n, nf = S->nf;
    double *g_a0 = calloc(N, sizeof(double)), *g_om = calloc(N, sizeof(double));
    double *g_rv = calloc(N, sizeof(double));
    double *h = calloc((size_t)(nf + 1) * N, sizeof(double));
    orc_mbd_chain(N, nf, S->R, S->a0, S->rv, S->alpha_bar, S->abar0, S->c6bar, S->ombar, S->rbar, S->wu,
                  S->Z, S->beta, S->a, h, g_a0, g_rv, gR);
    double *X = malloc(sizeof(double) * (size_t)(nf + 1) * 3 * n);
    double *V = malloc(sizeof(double) * (size_t)(nf + 1) * 3 * n);
    for (int k = 0; k <= nf; ++k) {
        const double *Ab = S->Abar + (size_t)k * n * n;
        double *Xk = X + (size_t)k * 3 * n, *Vk = V + (size_t)k * 3 * n;
        for (int p = 0; p < n; ++p)
            for (int c = 0; c < 3; ++c) {
                double x = 0.0, v = 0.0;
                for (int jj = 0; jj < N; ++jj) {
                    x += Ab[(size_t)p * n + 3 * jj + c];
                    v += Ab[(size_t)p * n + 3 * jj + c] * h[(size_t)k * N + jj];
                }
                Xk[3 * p + c] = x; Vk[3 * p + c] = v;
            }
    }
    orc_scs_adjoint_pass(N, nf, S->R, S->a0, S->om, S->rv, S->u, S->beta, S->a, X, V, g_a0, g_om, g_rv, gR);
    if (gp) ts_chain(N, a0ref, c6ref, rref, ratio, g_a0, g_om, g_rv, gp);
    free(X); free(V); free(h);
    free(g_a0); free(g_om); free(g_rv);
    return ORC_OK;
}

/* Energy and gradients.  mode 0: forward mode with the paper's fused SCS formula;
 * mode 1: adjoint.  grad_coords [N][3], grad_params [4][N] (alpha0_ref, C6_ref, R_ref,
 * ratio).  detail as in orc_mbd_rsscs_energy. */
int orc_mbd_rsscs_gradient(int N, const double *R, const double *a0ref, const double *c6ref,
                           const double *rref, const double *ratio, double beta, double a,
                           int nf, int mode, double *E, double *grad_coords,
                           double *grad_params) {
    orc_state S;
    int rc = state_forward(&S, N, R, a0ref, c6ref, rref, ratio, beta, a, nf, 1);
    if (rc == ORC_OK) {
        *E = S.E;
        if (mode == 0) rc = grad_forward(&S, a0ref, c6ref, rref, ratio, grad_coords, grad_params);
        else rc = grad_adjoint(&S, a0ref, c6ref, rref, ratio, grad_coords, grad_params);
    }
    state_free(&S);
    return rc;
}

/* MBD-NL (Sec. 2.7, paragraph MBD-NL): no screening step.  The oscillators are set
 * directly from the free-atom reference and the ratios of a density polarizability
 * functional, Eq. (mbd-nl-scaling): alpha0_i = alpha0_ref,i ra_i, omega_i = omega_ref,i rw_i,
 * with omega_ref = 4 C6_ref / (3 alpha0_ref^2) the free atom's single-oscillator frequency
 * (reading: the relation of Eq. ts-scaling), and the damping radii of Eq. (mbd-nl-rvdw),
 * R_i = 5/2 alpha0_ref,i^{1/7} ra_i^{1/3}; then the MBD energy of Eq. (mbd-energy) with the
 * Fermi-damped T^lr of Eq. (mbd-lr-dipole).  grad_coords [N][3] and grad_params [4][N]
 * (d/d alpha0_ref, C6_ref, ra, rw) may both be NULL (energy only); params_out [3][N]
 * (alpha0, omega, R) may be NULL. */
int orc_mbd_nl(int N, const double *R, const double *a0ref, const double *c6ref, const double *ra,
               const double *rw, double beta, double a, double *E, double *grad_coords,
               double *grad_params, double *params_out) {
    for (int i = 0; i < N; ++i)
        if (!(a0ref[i] > 0.0) || !(c6ref[i] > 0.0) || !(ra[i] > 0.0) || !(rw[i] > 0.0)) return ORC_ERR_INPUT;
    int n = 3 * N;
    double *a0 = malloc(sizeof(double) * N), *om = malloc(sizeof(double) * N), *rd = malloc(sizeof(double) * N);
    for (int i = 0; i < N; ++i) {
        a0[i] = a0ref[i] * ra[i];
        om[i] = 4.0 * c6ref[i] / (3.0 * a0ref[i] * a0ref[i]) * rw[i];
        rd[i] = 2.5 * pow(a0ref[i], 1.0 / 7.0) * cbrt(ra[i]);
    }
    if (params_out)
        for (int i = 0; i < N; ++i) {
            params_out[i] = a0[i];
            params_out[N + i] = om[i];
            params_out[2 * N + i] = rd[i];
        }
    double *Q = malloc(sizeof(double) * (size_t)n * n);
    int want_grad = grad_coords != NULL || grad_params != NULL;
    double *Z = want_grad ? malloc(sizeof(double) * (size_t)n * n) : NULL;
    orc_mbd_q(N, R, a0, om, rd, beta, a, Q);
    int rc = orc_energy_from_q(N, Q, om, E, Z);
    if (rc == ORC_OK && want_grad) {
        double *g_om = calloc(N, sizeof(double)), *g_a0 = calloc(N, sizeof(double));
        double *g_rd = calloc(N, sizeof(double)), *gR = calloc((size_t)3 * N, sizeof(double));
        mbd_pair_adjoint(N, R, a0, om, rd, Z, beta, a, g_om, g_a0, g_rd, gR);
        if (grad_coords) memcpy(grad_coords, gR, sizeof(double) * 3 * N);
        if (grad_params)
            for (int i = 0; i < N; ++i) {   /* chain through Eqs. (mbd-nl-scaling), (mbd-nl-rvdw) */
                grad_params[i] = g_a0[i] * ra[i] - g_om[i] * 2.0 * om[i] / a0ref[i] + g_rd[i] * rd[i] / (7.0 * a0ref[i]);
                grad_params[N + i] = g_om[i] * om[i] / c6ref[i];
                grad_params[2 * N + i] = g_a0[i] * a0ref[i] + g_rd[i] * rd[i] / (3.0 * ra[i]);
                grad_params[3 * N + i] = g_om[i] * om[i] / rw[i];
            }
        free(g_om); free(g_a0); free(g_rd); free(gR);
    }
    free(a0); free(om); free(rd); free(Q); free(Z);
    return rc;
}
