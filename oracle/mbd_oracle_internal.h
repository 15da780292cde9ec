/*
 * mbd_oracle_internal.h -- helpers shared by the two files of the CPU oracle
 * (mbd_oracle.c: finite systems; mbd_periodic.c: periodic systems).
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: nothing in the product path
 * includes this header.
 */
#ifndef MBD_ORACLE_INTERNAL_H
#define MBD_ORACLE_INTERNAL_H

#define ORC_OK 0
#define ORC_ERR_INPUT 1
#define ORC_ERR_NEG_EIGENVALUE 2
#define ORC_ERR_SCS_NEG_ALPHA 3
#define ORC_ERR_SINGULAR 4
#define ORC_ERR_NOT_CONVERGED 5

#define ORC_PI 3.14159265358979323846264338327950288

/* Neumaier-compensated sum. */
typedef struct { double s, c; } orc_sum;
void ksum_add(orc_sum *k, double x);
double ksum_get(const orc_sum *k);

int orc_freq_grid(int n_freq, double *u, double *wu);
void orc_T_bare(const double *r, double *T);
void orc_T_gg(const double *r, double s, double *T);
void orc_T_erfc(const double *r, double gamma, double *T);
double orc_fermi(double rho, double rsum, double sr, double a);
void orc_T_bare_deriv(const double *r, double *dT);
int orc_gauss_jordan_inverse(int n, const double *A, double *Ainv);
int orc_jacobi_eigh(int n, const double *Ain, double *lam, double *V);
void orc_ts_scaling(int N, const double *a0ref, const double *c6ref, const double *rref,
                    const double *ratio, double *a0, double *om, double *rv);
int orc_screened_params(int N, int n_freq, const double *alpha_bar, const double *wu,
                        const double *a0, const double *rv, double *abar0, double *c6bar,
                        double *ombar, double *rbar);

double alpha_iu(double a0, double om, double u);
double mayer_sigma(double al);
void radial_tensor_deriv(const double *r, double rr, double A, double Bf, double dA,
                         double dBf, double *dT);
void scs_block_derivs(const double *r, double al_i, double al_j, double rsum, double beta,
                      double a, double *dBdr, double *dBdai, double *dBdaj, double *dBdS);
void ts_chain(int N, const double *a0ref, const double *c6ref, const double *rref,
              const double *ratio, const double *g_a0, const double *g_om, const double *g_rv,
              double *gp);

#endif
