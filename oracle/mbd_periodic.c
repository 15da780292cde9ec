/*
 * mbd_periodic.c -- plain, slow FP64 CPU oracle for periodic MBD@rsSCS (arXiv 2308.03140,
 * Sec. 2.2 "Periodic boundary conditions" and the Ewald summation of the dipole tensor).
 *
 * TEST INFRASTRUCTURE ONLY, like mbd_oracle.c: used by the tests, the package's smoke check
 * and the benchmark's CPU-baseline leg, never by the product path.  It shares no code with
 * the CUDA path.
 *
 * Cell convention: A[3c+d] is component d of lattice vector a_c (rows are lattice vectors).
 * Reciprocal vectors b_c satisfy a_c . b_d = 2 pi delta_cd, so B = 2 pi A^{-T}; the cell
 * volume is |det A|.  Bloch vectors are given by fractional coordinates kappa, q = kappa B.
 * Lattice gradients are dE/dA_cd with Cartesian atom positions and kappa held fixed.
 *
 * Readings taken here (beyond those of mbd_oracle.c):
 *   R3  Reciprocal-space phase: T(q)_ij = sum_n T(R_nij) e^{-i q.R_nij} with
 *       R_nij = R_j + R_n - R_i; Poisson summation gives the reciprocal term
 *       (4 pi/Omega) sum_{G: 0<|G+q|<k_c} k^ k^T exp(-k^2/(4 gamma^2)) e^{+i G.(R_j - R_i)},
 *       k = G + q.  The self term is -delta_ij (4 gamma^3 / (3 sqrt pi)) I.
 *   R4  Damped long-range tensor under periodic boundaries:
 *       T^lr(q) = Ewald[T](q) - sum_n (1 - g(R_nij)) T(R_nij) e^{-i q.R_nij}.
 *   R6  Periodic SCS: Gamma-point real-space lattice sum of (1 - f) T^GG up to the real-space
 *       cutoff, including i = j images with n != 0; the contraction runs over the cell's atoms.
 *   R12 k-points: Monkhorst-Pack, kappa_c = (2m - n_c - 1)/(2 n_c), m = 1..n_c.
 *
 * Complex n x n matrices are row-major arrays of (re, im) pairs.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "mbd_oracle_internal.h"

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* Cell geometry.                                                             */
/* ------------------------------------------------------------------------- */
typedef struct {
    double A[9], Ainv[9], B[9], vol;
} orc_cell;

static int cell_setup(const double *A, orc_cell *c) {
    double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6])
               + A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(fabs(det) > 0.0)) return ORC_ERR_INPUT;
    memcpy(c->A, A, sizeof(double) * 9);
    /* inverse by cofactors: Ainv[e][c] */
    double C[9] = {A[4] * A[8] - A[5] * A[7], -(A[3] * A[8] - A[5] * A[6]), A[3] * A[7] - A[4] * A[6],
                   -(A[1] * A[8] - A[2] * A[7]), A[0] * A[8] - A[2] * A[6], -(A[0] * A[7] - A[1] * A[6]),
                   A[1] * A[5] - A[2] * A[4], -(A[0] * A[5] - A[2] * A[3]), A[0] * A[4] - A[1] * A[3]};
    for (int e = 0; e < 3; ++e)
        for (int k = 0; k < 3; ++k) c->Ainv[3 * e + k] = C[3 * k + e] / det;
    for (int k = 0; k < 3; ++k)
        for (int e = 0; e < 3; ++e) c->B[3 * k + e] = 2.0 * ORC_PI * c->Ainv[3 * e + k];
    c->vol = fabs(det);
    return ORC_OK;
}

/* Exposed for pins: reciprocal vectors (rows) and volume. */
int orc_cell_reciprocal(const double *A, double *B, double *vol) {
    orc_cell c;
    int rc = cell_setup(A, &c);
    if (rc) return rc;
    memcpy(B, c.B, sizeof(double) * 9);
    *vol = c.vol;
    return ORC_OK;
}

static double norm3(const double *v) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

/* Fractional coordinate c of a Cartesian vector v: f_c = sum_e v_e Ainv[e][c]. */
static double frac(const orc_cell *c, const double *v, int k) {
    return v[0] * c->Ainv[k] + v[1] * c->Ainv[3 + k] + v[2] * c->Ainv[6 + k];
}

/* Integer ranges of lattice translations n with |x + n A| < rc possible. */
static void image_range(const orc_cell *c, const double *x, double rc, int *lo, int *hi) {
    for (int k = 0; k < 3; ++k) {
        double L = rc * norm3(c->B + 3 * k) / (2.0 * ORC_PI), d = frac(c, x, k);
        lo[k] = (int)ceil(-L - d) - 1;
        hi[k] = (int)floor(L - d) + 1;
    }
}

/* Monkhorst-Pack fractional k-points (reading R12), nk = g0 g1 g2 rows of 3. */
int orc_monkhorst_pack(const int *grid, double *kfrac) {
    int t = 0;
    for (int m0 = 1; m0 <= grid[0]; ++m0)
        for (int m1 = 1; m1 <= grid[1]; ++m1)
            for (int m2 = 1; m2 <= grid[2]; ++m2) {
                kfrac[3 * t] = (2.0 * m0 - grid[0] - 1) / (2.0 * grid[0]);
                kfrac[3 * t + 1] = (2.0 * m1 - grid[1] - 1) / (2.0 * grid[1]);
                kfrac[3 * t + 2] = (2.0 * m2 - grid[2] - 1) / (2.0 * grid[2]);
                ++t;
            }
    return t;
}

/* ------------------------------------------------------------------------- */
/* Tensors and their derivatives.                                             */
/* ------------------------------------------------------------------------- */

/* dT^erfc/dr_c [27] for T^erfc_ab = A delta_ab + Bf r_a r_b, A = B(x)/r^3,
 * Bf = -C(x)/r^5, x = gamma r, with dB/dx = -2x e, dC/dx = -4x^3 e,
 * e = 2x/sqrt(pi) exp(-x^2).  Pinned by central differences of orc_T_erfc. */
void orc_T_erfc_deriv(const double *r, double gamma, double *dT) {
    double rr = norm3(r), x = gamma * rr, r3 = rr * rr * rr, r5 = r3 * rr * rr;
    double e = 2.0 * x / sqrt(ORC_PI) * exp(-x * x);
    double Bx = erfc(x) + e, Cx = 3.0 * erfc(x) + e * (3.0 + 2.0 * x * x);
    double A = Bx / r3, Bf = -Cx / r5;
    double dA = gamma * (-2.0 * x * e) / r3 - 3.0 * Bx / (r3 * rr);
    double dBf = -gamma * (-4.0 * x * x * x * e) / r5 + 5.0 * Cx / (r5 * rr);
    radial_tensor_deriv(r, rr, A, Bf, dA, dBf, dT);
}

/* ------------------------------------------------------------------------- */
/* Long-range periodic dipole block, readings R3 and R4.                      */
/* ------------------------------------------------------------------------- */

/* T^lr(q)_ij (3x3 complex) for the separation x = R_j - R_i of one atom pair (same = 1 when
 * i = j, which removes n = 0 from the real-space sums and adds the self term), with
 * S = Rbar_i + Rbar_j the damping radius sum.  With damp = 0 the Ewald-summed bare tensor
 * alone is returned.  Optional derivatives: dx [27] (d/dx_d at index 9d + 3a + b),
 * dS [9], dA [81] (d/dA_cd at index 9(3c + d) + 3a + b).
 * Pinned by gamma-invariance, Hermiticity, T(-q) = conj T(q) and central differences. */
void orc_tlr_block(const double *Acell, const double *x, int same, const double *kappa,
                   double gamma, double rc, double kc, double S, double beta, double a, int damp,
                   double *Tout, double *dxout, double *dSout, double *dAout) {
    orc_cell c;
    cell_setup(Acell, &c);
    double q[3];
    for (int e = 0; e < 3; ++e) q[e] = kappa[0] * c.B[e] + kappa[1] * c.B[3 + e] + kappa[2] * c.B[6 + e];
    cplx T[9] = {0}, dx[27] = {0}, dS[9] = {0}, dA[81] = {0};
    const int want = dxout || dSout || dAout;
    /* real space: sum over images r = x + n A with 0 < |r| < rc */
    int lo[3], hi[3];
    image_range(&c, x, rc, lo, hi);
    for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
        for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
            for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
                int nn[3] = {n0, n1, n2};
                double r[3];
                for (int e = 0; e < 3; ++e) r[e] = x[e] + n0 * c.A[e] + n1 * c.A[3 + e] + n2 * c.A[6 + e];
                double rr = norm3(r);
                if (rr >= rc || rr < 1e-8) continue;
                double Te[9], dTe[27], Tb[9], dTb[27];
                orc_T_erfc(r, gamma, Te);
                orc_T_erfc_deriv(r, gamma, dTe);
                orc_T_bare(r, Tb);
                orc_T_bare_deriv(r, dTb);
                double g = 0.0, dgdr = 0.0, dgdS = 0.0;
                if (damp) {
                    g = orc_fermi(rr, S, beta, a);
                    double eta = rr / (beta * S), dgdeta = a * g * (1.0 - g);
                    dgdr = dgdeta / (beta * S);
                    dgdS = -dgdeta * eta / S;
                }
                /* F = T^erfc - (1 - g) T  (damp = 0: F = T^erfc) */
                double F[9], dF[27];
                for (int t = 0; t < 9; ++t) F[t] = Te[t] - (damp ? (1.0 - g) * Tb[t] : 0.0);
                for (int d = 0; d < 3; ++d)
                    for (int t = 0; t < 9; ++t)
                        dF[9 * d + t] = dTe[9 * d + t] - (damp ? (1.0 - g) * dTb[9 * d + t] - dgdr * r[d] / rr * Tb[t] : 0.0);
                double ph = -(q[0] * r[0] + q[1] * r[1] + q[2] * r[2]);
                cplx p = cos(ph) + I * sin(ph);
                double fr[3] = {frac(&c, r, 0), frac(&c, r, 1), frac(&c, r, 2)};
                for (int t = 0; t < 9; ++t) {
                    T[t] += F[t] * p;
                    if (!want) continue;
                    dS[t] += dgdS * Tb[t] * p;
                    for (int d = 0; d < 3; ++d) {
                        cplx dr = (dF[9 * d + t] - I * q[d] * F[t]) * p;   /* d(F p)/dr_d */
                        dx[9 * d + t] += dr;
                        for (int k = 0; k < 3; ++k)   /* r depends on A through n; q through B */
                            dA[9 * (3 * k + d) + t] += nn[k] * dr + I * q[d] * fr[k] * F[t] * p;
                    }
                }
            }
    /* reciprocal space: k = G + q with 0 < |k| < kc */
    int mlo[3], mhi[3];
    for (int k = 0; k < 3; ++k) {
        double L = kc * norm3(c.A + 3 * k) / (2.0 * ORC_PI);
        mlo[k] = (int)ceil(-L - kappa[k]) - 1;
        mhi[k] = (int)floor(L - kappa[k]) + 1;
    }
    double pre = 4.0 * ORC_PI / c.vol;
    double fx[3] = {frac(&c, x, 0), frac(&c, x, 1), frac(&c, x, 2)};
    for (int m0 = mlo[0]; m0 <= mhi[0]; ++m0)
        for (int m1 = mlo[1]; m1 <= mhi[1]; ++m1)
            for (int m2 = mlo[2]; m2 <= mhi[2]; ++m2) {
                double G[3], kv[3];
                for (int e = 0; e < 3; ++e) {
                    G[e] = m0 * c.B[e] + m1 * c.B[3 + e] + m2 * c.B[6 + e];
                    kv[e] = G[e] + q[e];
                }
                double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2], kk = sqrt(k2);
                if (kk >= kc || kk < 1e-12) continue;
                double E = exp(-k2 / (4.0 * gamma * gamma));
                double ph = G[0] * x[0] + G[1] * x[1] + G[2] * x[2];
                cplx p = pre * (cos(ph) + I * sin(ph));
                for (int aa = 0; aa < 3; ++aa)
                    for (int b = 0; b < 3; ++b) {
                        int t = 3 * aa + b;
                        double phi = kv[aa] * kv[b] * E / k2;
                        cplx h = phi * p;
                        T[t] += h;
                        if (!want) continue;
                        /* d phi / d k_e */
                        double dphi[3];
                        for (int e = 0; e < 3; ++e)
                            dphi[e] = ((aa == e ? kv[b] : 0.0) + (b == e ? kv[aa] : 0.0)) * E / k2
                                    - kv[aa] * kv[b] * kv[e] * E * (2.0 / (k2 * k2) + 1.0 / (2.0 * gamma * gamma * k2));
                        for (int d = 0; d < 3; ++d) {
                            dx[9 * d + t] += I * G[d] * h;
                            for (int k = 0; k < 3; ++k) {
                                double dphiA = dphi[0] * c.Ainv[k] + dphi[1] * c.Ainv[3 + k] + dphi[2] * c.Ainv[6 + k];
                                dA[9 * (3 * k + d) + t] += h * (-c.Ainv[3 * d + k] - I * G[d] * fx[k])
                                                         - kv[d] * dphiA * p;
                            }
                        }
                    }
            }
    if (same) {
        double self = 4.0 * gamma * gamma * gamma / (3.0 * sqrt(ORC_PI));
        for (int aa = 0; aa < 3; ++aa) T[4 * aa] -= self;
    }
    for (int t = 0; t < 9; ++t) { Tout[2 * t] = creal(T[t]); Tout[2 * t + 1] = cimag(T[t]); }
    if (dxout) for (int t = 0; t < 27; ++t) { dxout[2 * t] = creal(dx[t]); dxout[2 * t + 1] = cimag(dx[t]); }
    if (dSout) for (int t = 0; t < 9; ++t) { dSout[2 * t] = creal(dS[t]); dSout[2 * t + 1] = cimag(dS[t]); }
    if (dAout) for (int t = 0; t < 81; ++t) { dAout[2 * t] = creal(dA[t]); dAout[2 * t + 1] = cimag(dA[t]); }
}

/* Ewald-summed bare dipole matrix T(q) (n x n complex), Eq. (ewald) with readings R2, R3. */
int orc_ewald_T(int N, const double *R, const double *A, const double *kappa, double gamma,
                double rc, double kc, double *out) {
    int n = 3 * N;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double x[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
            double T[18];
            orc_tlr_block(A, x, i == j, kappa, gamma, rc, kc, 1.0, 1.0, 1.0, 0, T, NULL, NULL, NULL);
            for (int aa = 0; aa < 3; ++aa)
                for (int b = 0; b < 3; ++b) {
                    size_t o = 2 * ((size_t)(3 * i + aa) * n + 3 * j + b);
                    out[o] = T[2 * (3 * aa + b)];
                    out[o + 1] = T[2 * (3 * aa + b) + 1];
                }
        }
    return ORC_OK;
}

/* Periodic coupled-oscillator matrix Q(q), Eq. (q-matrix) with T^lr(q) of reading R4:
 * Q_ij = delta_ij om_i^2 I + om_i om_j sqrt(a_i a_j) T^lr(q)_ij. */
int orc_periodic_q(int N, const double *R, const double *A, const double *kappa, const double *a0,
                   const double *om, const double *rdamp, double beta, double a, double gamma,
                   double rc, double kc, double *out) {
    int n = 3 * N;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double x[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
            double T[18];
            orc_tlr_block(A, x, i == j, kappa, gamma, rc, kc, rdamp[i] + rdamp[j], beta, a, 1, T, NULL,
                          NULL, NULL);
            double pre = om[i] * om[j] * sqrt(a0[i] * a0[j]);
            for (int aa = 0; aa < 3; ++aa)
                for (int b = 0; b < 3; ++b) {
                    size_t o = 2 * ((size_t)(3 * i + aa) * n + 3 * j + b);
                    out[o] = pre * T[2 * (3 * aa + b)] + (i == j && aa == b ? om[i] * om[i] : 0.0);
                    out[o + 1] = pre * T[2 * (3 * aa + b) + 1];
                }
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Hermitian matrix functions through the real symmetric embedding            */
/* M = [[Re Q, -Im Q], [Im Q, Re Q]] (2n x 2n): every eigenvalue of Q appears  */
/* twice in M, and f(M) = [[Re f(Q), -Im f(Q)], [Im f(Q), Re f(Q)]].          */
/* ------------------------------------------------------------------------- */

/* 1/2 Tr Q^{1/2} (Eqs. diagonalization, mbd-energy) and optionally Q^{-1/2} (complex).
 * Returns ORC_ERR_NEG_EIGENVALUE when Q is not positive definite.  lam_out (optional)
 * receives the n eigenvalues of Q in ascending order.  Pinned by numpy.linalg.eigh. */
int orc_hermitian_sqrt(int n, const double *Q, double *half_tr_sqrt, double *Zout, double *lam_out) {
    int m = 2 * n;
    double *M = calloc((size_t)m * m, sizeof(double)), *lam = malloc(sizeof(double) * m);
    double *V = malloc(sizeof(double) * (size_t)m * m);
    for (int p = 0; p < n; ++p)
        for (int r = 0; r < n; ++r) {
            double re = Q[2 * ((size_t)p * n + r)], im = Q[2 * ((size_t)p * n + r) + 1];
            M[(size_t)p * m + r] = re;
            M[(size_t)(p + n) * m + r + n] = re;
            M[(size_t)p * m + r + n] = -im;
            M[(size_t)(p + n) * m + r] = im;
        }
    int rc = orc_jacobi_eigh(m, M, lam, V);
    double lmin = lam[0];
    for (int k = 1; k < m; ++k) lmin = lam[k] < lmin ? lam[k] : lmin;
    if (rc == ORC_OK && !(lmin > 0.0)) rc = ORC_ERR_NEG_EIGENVALUE;
    if (rc == ORC_OK) {
        orc_sum s = {0, 0};
        for (int k = 0; k < m; ++k) ksum_add(&s, 0.25 * sqrt(lam[k]));   /* each eigenvalue twice */
        *half_tr_sqrt = ksum_get(&s);
        if (lam_out) {
            /* ascending, every other one of the doubled list */
            double *srt = malloc(sizeof(double) * m);
            memcpy(srt, lam, sizeof(double) * m);
            for (int a1 = 1; a1 < m; ++a1) {
                double v = srt[a1];
                int b = a1 - 1;
                while (b >= 0 && srt[b] > v) { srt[b + 1] = srt[b]; --b; }
                srt[b + 1] = v;
            }
            for (int k = 0; k < n; ++k) lam_out[k] = srt[2 * k];
            free(srt);
        }
        if (Zout) {
#pragma omp parallel for schedule(dynamic)
            for (int p = 0; p < n; ++p)
                for (int r = 0; r < n; ++r) {
                    double re = 0.0, im = 0.0;
                    for (int k = 0; k < m; ++k) {
                        double w = 1.0 / sqrt(lam[k]);
                        re += V[(size_t)p * m + k] * V[(size_t)r * m + k] * w;
                        im += V[(size_t)(p + n) * m + k] * V[(size_t)r * m + k] * w;
                    }
                    Zout[2 * ((size_t)p * n + r)] = re;
                    Zout[2 * ((size_t)p * n + r) + 1] = im;
                }
        }
    }
    free(M); free(lam); free(V);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Periodic SCS, reading R6.                                                  */
/* ------------------------------------------------------------------------- */

/* Gamma-point SCS matrix at one frequency:
 * M_ij = delta_ij I / alpha_i + sum_{n: 0<|R_nij|<rc} (1 - f_ij) T^GG(R_nij, s_ij). */
int orc_periodic_scs_matrix(int N, const double *R, const double *A, const double *al,
                            const double *rv, double beta, double a, double rc, double *M) {
    orc_cell c;
    int e0 = cell_setup(A, &c);
    if (e0) return e0;
    int n = 3 * N;
    memset(M, 0, sizeof(double) * (size_t)n * n);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < N; ++i) {
        for (int t = 0; t < 3; ++t) M[(size_t)(3 * i + t) * n + 3 * i + t] = 1.0 / al[i];
        double si = mayer_sigma(al[i]);
        for (int j = 0; j < N; ++j) {
            double x[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
            double sj = mayer_sigma(al[j]), s = sqrt(si * si + sj * sj);
            int lo[3], hi[3];
            image_range(&c, x, rc, lo, hi);
            for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
                for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
                    for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
                        double r[3];
                        for (int e = 0; e < 3; ++e) r[e] = x[e] + n0 * c.A[e] + n1 * c.A[3 + e] + n2 * c.A[6 + e];
                        double rr = norm3(r);
                        if (rr >= rc || rr < 1e-8) continue;
                        double T[9];
                        orc_T_gg(r, s, T);
                        double f = orc_fermi(rr, rv[i] + rv[j], beta, a);
                        for (int xx = 0; xx < 3; ++xx)
                            for (int y = 0; y < 3; ++y) M[(size_t)(3 * i + xx) * n + 3 * j + y] += (1.0 - f) * T[3 * xx + y];
                    }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Full periodic MBD@rsSCS energy and gradients.                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    int N, n, nf, nk;
    const double *R, *A, *kappa;
    double beta, a, gamma, rc, kc;
    double *a0, *om, *rv, *u, *wu, *alpha_bar, *Abar, *abar0, *c6bar, *ombar, *rbar;
    double *Z;       /* nk x n x n complex: Q(q)^{-1/2} */
    double *Eq;      /* nk: 1/2 Tr Q(q)^{1/2} */
    double E;
} orc_pstate;

static void pstate_free(orc_pstate *S) {
    free(S->a0); free(S->om); free(S->rv); free(S->u); free(S->wu); free(S->alpha_bar);
    free(S->Abar); free(S->abar0); free(S->c6bar); free(S->ombar); free(S->rbar);
    free(S->Z); free(S->Eq);
}

static int pstate_forward(orc_pstate *S, int N, const double *R, const double *A, int nk,
                          const double *kappa, const double *a0ref, const double *c6ref,
                          const double *rref, const double *ratio, double beta, double a, int nf,
                          double gamma, double rc, double kc, int keep) {
    memset(S, 0, sizeof(*S));
    S->N = N; S->n = 3 * N; S->nf = nf; S->nk = nk; S->R = R; S->A = A; S->kappa = kappa;
    S->beta = beta; S->a = a; S->gamma = gamma; S->rc = rc; S->kc = kc;
    int n = S->n;
    S->a0 = malloc(sizeof(double) * N); S->om = malloc(sizeof(double) * N);
    S->rv = malloc(sizeof(double) * N);
    S->u = malloc(sizeof(double) * (nf + 1)); S->wu = malloc(sizeof(double) * (nf + 1));
    S->alpha_bar = malloc(sizeof(double) * (size_t)(nf + 1) * N);
    S->abar0 = malloc(sizeof(double) * N); S->c6bar = malloc(sizeof(double) * N);
    S->ombar = malloc(sizeof(double) * N); S->rbar = malloc(sizeof(double) * N);
    S->Eq = malloc(sizeof(double) * nk);
    if (keep) {
        S->Abar = malloc(sizeof(double) * (size_t)(nf + 1) * n * n);
        S->Z = malloc(sizeof(double) * 2 * (size_t)nk * n * n);
    }
    orc_ts_scaling(N, a0ref, c6ref, rref, ratio, S->a0, S->om, S->rv);
    orc_freq_grid(nf, S->u, S->wu);
    /* Gamma-point screening at every grid point */
    double *al = malloc(sizeof(double) * N), *M = malloc(sizeof(double) * (size_t)n * n);
    double *Ai = malloc(sizeof(double) * (size_t)n * n);
    int rc0 = ORC_OK;
    for (int k = 0; k <= nf && rc0 == ORC_OK; ++k) {
        for (int i = 0; i < N; ++i) al[i] = alpha_iu(S->a0[i], S->om[i], S->u[k]);
        rc0 = orc_periodic_scs_matrix(N, R, A, al, S->rv, beta, a, rc, M);
        if (!rc0) rc0 = orc_gauss_jordan_inverse(n, M, Ai);
        for (int i = 0; i < N; ++i) {   /* Eq. (contraction) over the cell's atoms */
            orc_sum s = {0, 0};
            for (int t = 0; t < 3; ++t)
                for (int j = 0; j < N; ++j) ksum_add(&s, Ai[(size_t)(3 * i + t) * n + 3 * j + t]);
            S->alpha_bar[(size_t)k * N + i] = ksum_get(&s) / 3.0;
        }
        if (keep) memcpy(S->Abar + (size_t)k * n * n, Ai, sizeof(double) * (size_t)n * n);
    }
    free(al); free(M); free(Ai);
    if (rc0) return rc0;
    rc0 = orc_screened_params(N, nf, S->alpha_bar, S->wu, S->a0, S->rv, S->abar0, S->c6bar,
                              S->ombar, S->rbar);
    if (rc0) return rc0;
    /* E = (1/nk) sum_q 1/2 Tr Q(q)^{1/2} - 3/2 sum omega_bar */
    double *Q = malloc(sizeof(double) * 2 * (size_t)n * n);
    for (int t = 0; t < nk && rc0 == ORC_OK; ++t) {
        orc_periodic_q(N, R, A, kappa + 3 * t, S->abar0, S->ombar, S->rbar, beta, a, gamma, rc, kc, Q);
        rc0 = orc_hermitian_sqrt(n, Q, &S->Eq[t], keep ? S->Z + 2 * (size_t)t * n * n : NULL, NULL);
    }
    free(Q);
    if (rc0) return rc0;
    orc_sum s = {0, 0};
    for (int t = 0; t < nk; ++t) ksum_add(&s, S->Eq[t] / nk);
    for (int i = 0; i < N; ++i) ksum_add(&s, -1.5 * S->ombar[i]);
    S->E = ksum_get(&s);
    return ORC_OK;
}

/* Periodic energy.  kappa: nk fractional Bloch vectors (rows of 3).  detail (optional):
 * alpha_bar[(nf+1)N], c6bar[N], omega_bar[N], rbar[N], E_q[nk]. */
int orc_periodic_rsscs_energy(int N, const double *R, const double *A, int nk, const double *kappa,
                              const double *a0ref, const double *c6ref, const double *rref,
                              const double *ratio, double beta, double a, int nf, double gamma,
                              double rc, double kc, double *E, double *detail) {
    orc_pstate S;
    int rc0 = pstate_forward(&S, N, R, A, nk, kappa, a0ref, c6ref, rref, ratio, beta, a, nf, gamma,
                             rc, kc, 0);
    if (rc0 == ORC_OK) *E = S.E;
    if (detail && S.alpha_bar) {
        memcpy(detail, S.alpha_bar, sizeof(double) * (size_t)(nf + 1) * N);
        memcpy(detail + (size_t)(nf + 1) * N, S.c6bar, sizeof(double) * N);
        memcpy(detail + (size_t)(nf + 2) * N, S.ombar, sizeof(double) * N);
        memcpy(detail + (size_t)(nf + 3) * N, S.rbar, sizeof(double) * N);
        memcpy(detail + (size_t)(nf + 4) * N, S.Eq, sizeof(double) * nk);
    }
    pstate_free(&S);
    return rc0;
}

/* Adjoint gradient of the periodic energy: coordinates gR [N][3], lattice gA [3][3]
 * (dE/dA_cd), free-atom parameters gp [4][N].
 * MBD part: dE = sum_q (1/nk) 1/4 Tr(Q(q)^{-1/2} dQ(q)) - 3/2 sum d omega_bar (reading R8 per
 * Bloch vector); with Z Hermitian, Tr(Z dQ) = sum_pq Re(conj(Z_pq) dQ_pq).  SCS part: the
 * finite adjoint (V = Abar H, X = Abar 1, dE = -1/3 sum dM_pq (V X^T)_pq) on the Gamma-point
 * matrices, with every image of every pair.  Pinned by central differences of the energy. */
int orc_periodic_rsscs_gradient(int N, const double *R, const double *A, int nk, const double *kappa,
                                const double *a0ref, const double *c6ref, const double *rref,
                                const double *ratio, double beta, double a, int nf, double gamma,
                                double rc, double kc, double *E, double *gR, double *gA, double *gp) {
    orc_pstate S;
    int rc0 = pstate_forward(&S, N, R, A, nk, kappa, a0ref, c6ref, rref, ratio, beta, a, nf, gamma,
                             rc, kc, 1);
    if (rc0) { pstate_free(&S); return rc0; }
    *E = S.E;
    int n = S.n;
    orc_cell cell;
    cell_setup(A, &cell);
    double *g_a0 = calloc(N, sizeof(double)), *g_om = calloc(N, sizeof(double));
    double *g_rv = calloc(N, sizeof(double)), *g_ombar = calloc(N, sizeof(double));
    double *g_ab0 = calloc(N, sizeof(double)), *g_rbar = calloc(N, sizeof(double));
    double *g_c = calloc(N, sizeof(double));
    double gAl[9] = {0};
    memset(gR, 0, sizeof(double) * 3 * N);
    /* ---- MBD part ---- */
    for (int i = 0; i < N; ++i) g_ombar[i] = -1.5;
    for (int t = 0; t < nk; ++t) {
        const double *Z = S.Z + 2 * (size_t)t * n * n;
        double w = 0.25 / nk;
        for (int i = 0; i < N; ++i) {
            double zd = 0.0;
            for (int aa = 0; aa < 3; ++aa) zd += Z[2 * ((size_t)(3 * i + aa) * n + 3 * i + aa)];
            g_ombar[i] += w * zd * 2.0 * S.ombar[i];
        }
#pragma omp parallel for schedule(dynamic) reduction(+ : gR[:3 * N], gAl[:9], g_c[:N], g_rbar[:N])
        for (int i = 0; i < N; ++i) {
            double ci = S.ombar[i] * sqrt(S.abar0[i]);
            for (int j = 0; j < N; ++j) {
                double cj = S.ombar[j] * sqrt(S.abar0[j]);
                double x[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
                double T[18], dx[54], dS[18], dA[162];
                orc_tlr_block(A, x, i == j, kappa + 3 * t, gamma, rc, kc, S.rbar[i] + S.rbar[j], beta, a, 1,
                              T, dx, dS, dA);
                /* contraction with conj(Z): Re(conj z * v) = zr vr + zi vi */
                double zT = 0.0, zS = 0.0, zx[3] = {0, 0, 0}, zA[9] = {0};
                for (int aa = 0; aa < 3; ++aa)
                    for (int b = 0; b < 3; ++b) {
                        size_t o = 2 * ((size_t)(3 * i + aa) * n + 3 * j + b);
                        double zr = Z[o], zi = Z[o + 1];
                        int tt = 3 * aa + b;
                        zT += zr * T[2 * tt] + zi * T[2 * tt + 1];
                        zS += zr * dS[2 * tt] + zi * dS[2 * tt + 1];
                        for (int d = 0; d < 3; ++d)
                            zx[d] += zr * dx[2 * (9 * d + tt)] + zi * dx[2 * (9 * d + tt) + 1];
                        for (int cd = 0; cd < 9; ++cd)
                            zA[cd] += zr * dA[2 * (9 * cd + tt)] + zi * dA[2 * (9 * cd + tt) + 1];
                    }
                g_c[i] += w * cj * zT;
                g_c[j] += w * ci * zT;
                g_rbar[i] += w * ci * cj * zS;
                g_rbar[j] += w * ci * cj * zS;
                for (int d = 0; d < 3; ++d) {   /* x = R_j - R_i */
                    gR[3 * j + d] += w * ci * cj * zx[d];
                    gR[3 * i + d] -= w * ci * cj * zx[d];
                }
                for (int cd = 0; cd < 9; ++cd) gAl[cd] += w * ci * cj * zA[cd];
            }
        }
    }
    for (int i = 0; i < N; ++i) {
        double sa = sqrt(S.abar0[i]);
        g_ombar[i] += g_c[i] * sa;
        g_ab0[i] += g_c[i] * S.ombar[i] / (2.0 * sa);
    }
    /* ---- chain through the screened parameters (Eqs. casimir-polder, scale-rvdw-scs) ---- */
    int nf1 = S.nf + 1;
    double *h = calloc((size_t)nf1 * N, sizeof(double));
    for (int i = 0; i < N; ++i) {
        double ab0 = S.abar0[i], xr = ab0 / S.a0[i];
        double g_c6 = g_ombar[i] * 4.0 / (3.0 * ab0 * ab0);
        double gab0 = g_ab0[i] - g_ombar[i] * 8.0 * S.c6bar[i] / (3.0 * ab0 * ab0 * ab0)
                    + g_rbar[i] * S.rv[i] / (3.0 * cbrt(xr) * cbrt(xr) * S.a0[i]);
        g_a0[i] += -g_rbar[i] * S.rv[i] / (3.0 * cbrt(xr) * cbrt(xr)) * ab0 / (S.a0[i] * S.a0[i]);
        g_rv[i] += g_rbar[i] * cbrt(xr);
        h[i] = gab0;
        for (int k = 1; k < nf1; ++k)
            h[(size_t)k * N + i] = g_c6 * 3.0 / ORC_PI * S.wu[k] * 2.0 * S.alpha_bar[(size_t)k * N + i];
    }
    /* ---- SCS adjoint on the Gamma-point matrices ---- */
    double *X = malloc(sizeof(double) * 3 * n), *V = malloc(sizeof(double) * 3 * n);
    for (int k = 0; k < nf1; ++k) {
        const double *Ab = S.Abar + (size_t)k * n * n;
        double u = S.u[k];
        for (int p = 0; p < n; ++p)
            for (int cc = 0; cc < 3; ++cc) {
                double xs = 0.0, vs = 0.0;
                for (int jj = 0; jj < N; ++jj) {
                    xs += Ab[(size_t)p * n + 3 * jj + cc];
                    vs += Ab[(size_t)p * n + 3 * jj + cc] * h[(size_t)k * N + jj];
                }
                X[3 * p + cc] = xs; V[3 * p + cc] = vs;
            }
        double *gal = calloc(N, sizeof(double));
        for (int i = 0; i < N; ++i) {
            double ali = alpha_iu(S.a0[i], S.om[i], u);
            double wd = 0.0;
            for (int t = 0; t < 3; ++t)
                for (int cc = 0; cc < 3; ++cc) wd += V[3 * (3 * i + t) + cc] * X[3 * (3 * i + t) + cc];
            gal[i] += -1.0 / 3.0 * wd * (-1.0 / (ali * ali));
        }
#pragma omp parallel for schedule(dynamic) reduction(+ : gR[:3 * N], gAl[:9], gal[:N], g_rv[:N])
        for (int i = 0; i < N; ++i) {
            double ali = alpha_iu(S.a0[i], S.om[i], u);
            for (int j = 0; j < N; ++j) {
                double alj = alpha_iu(S.a0[j], S.om[j], u);
                double x[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
                double wblk[9];
                for (int xx = 0; xx < 3; ++xx)
                    for (int y = 0; y < 3; ++y) {
                        double wv = 0.0;
                        for (int cc = 0; cc < 3; ++cc) wv += V[3 * (3 * i + xx) + cc] * X[3 * (3 * j + y) + cc];
                        wblk[3 * xx + y] = wv;
                    }
                int lo[3], hi[3];
                image_range(&cell, x, rc, lo, hi);
                for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
                    for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
                        for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
                            int nn[3] = {n0, n1, n2};
                            double r[3];
                            for (int e = 0; e < 3; ++e)
                                r[e] = x[e] + n0 * cell.A[e] + n1 * cell.A[3 + e] + n2 * cell.A[6 + e];
                            double rr = norm3(r);
                            if (rr >= rc || rr < 1e-8) continue;
                            double dBdr[27], dBda[9], dBdb[9], dBdS[9];
                            scs_block_derivs(r, ali, alj, S.rv[i] + S.rv[j], beta, a, dBdr, dBda, dBdb, dBdS);
                            double wa = 0.0, wb = 0.0, wS = 0.0, wr[3] = {0, 0, 0};
                            for (int tt = 0; tt < 9; ++tt) {
                                wa += wblk[tt] * dBda[tt]; wb += wblk[tt] * dBdb[tt]; wS += wblk[tt] * dBdS[tt];
                                for (int d = 0; d < 3; ++d) wr[d] += wblk[tt] * dBdr[9 * d + tt];
                            }
                            gal[i] += -1.0 / 3.0 * wa;
                            gal[j] += -1.0 / 3.0 * wb;
                            g_rv[i] += -1.0 / 3.0 * wS;
                            g_rv[j] += -1.0 / 3.0 * wS;
                            for (int d = 0; d < 3; ++d) {
                                gR[3 * j + d] += -1.0 / 3.0 * wr[d];
                                gR[3 * i + d] -= -1.0 / 3.0 * wr[d];
                                for (int c2 = 0; c2 < 3; ++c2) gAl[3 * c2 + d] += -1.0 / 3.0 * nn[c2] * wr[d];
                            }
                        }
            }
        }
        for (int i = 0; i < N; ++i) {
            double q = 1.0 + u * u / (S.om[i] * S.om[i]);
            g_a0[i] += gal[i] / q;
            g_om[i] += gal[i] * S.a0[i] * 2.0 * u * u / (S.om[i] * S.om[i] * S.om[i]) / (q * q);
        }
        free(gal);
    }
    if (gA) memcpy(gA, gAl, sizeof(double) * 9);
    if (gp) ts_chain(N, a0ref, c6ref, rref, ratio, g_a0, g_om, g_rv, gp);
    free(X); free(V); free(h);
    free(g_a0); free(g_om); free(g_rv); free(g_ombar); free(g_ab0); free(g_rbar); free(g_c);
    pstate_free(&S);
    return ORC_OK;
}
