// Host run of the pair kernels' radial formulas (csrc/pair_math.cuh: fermi, tgg_radial,
// bare_radial, erfc_radial and the FP32 fermi_f, tgg_radial_f) for the CPU tests.  Test
// infrastructure: built by tests/test_pair_math_host.py into tests/_build.
#include <cmath>

#include "pair_math.cuh"

using namespace mbdgb::pairs;

// out[0..2] = f, df/drho, df/dS
extern "C" void host_fermi(double rho, double S, double beta, double a, double *out) {
    const Fermi f = fermi(rho, S, beta, a);
    out[0] = f.f;
    out[1] = f.df_drho;
    out[2] = f.df_dS;
}
extern "C" void host_fermi_f(float rho, float S, float beta, float a, float *out) {
    const FermiF f = fermi_f(rho, S, beta, a);
    out[0] = f.f;
    out[1] = f.df_drho;
    out[2] = f.df_dS;
}
// out[0..5] = P, W, dP/drho, dW/drho, dP/ds, dW/ds
extern "C" void host_tgg(double rho, double s, double *out) {
    const Radial r = tgg_radial(rho, s);
    const double v[6] = {r.P, r.W, r.dP, r.dW, r.dPs, r.dWs};
    for (int k = 0; k < 6; ++k) out[k] = v[k];
}
extern "C" void host_tgg_f(float rho, float s, float *out) {
    const RadialF r = tgg_radial_f(rho, s);
    const float v[6] = {r.P, r.W, r.dP, r.dW, r.dPs, r.dWs};
    for (int k = 0; k < 6; ++k) out[k] = v[k];
}
// out[0..3] = P, W, dP/drho, dW/drho
extern "C" void host_bare(double rho, double *out) {
    const RadialT r = bare_radial(rho);
    out[0] = r.P; out[1] = r.W; out[2] = r.dP; out[3] = r.dW;
}
extern "C" void host_erfc(double rho, double gamma, double *out) {
    const RadialT r = erfc_radial(rho, gamma);
    out[0] = r.P; out[1] = r.W; out[2] = r.dP; out[3] = r.dW;
}

// The screening matrix of one frequency as k_build_scs forms it (both triangles, identity
// diagonal blocks 1/alpha): M [3N][3N] row-major, from the kernel's fermi and tgg_radial.
extern "C" void host_scs_matrix(int N, const double *R, const double *al, const double *sig, const double *rv,
                                double beta, double a, double *M) {
    const long long n = 3LL * N;
    for (long long e = 0; e < n * n; ++e) M[e] = 0.0;
    for (int i = 0; i < N; ++i) {
        for (int x = 0; x < 3; ++x) M[(3LL * i + x) * n + 3 * i + x] = 1.0 / al[i];
        for (int j = 0; j < i; ++j) {
            const double r[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
            const double rho = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            const Fermi f = fermi(rho, rv[i] + rv[j], beta, a);
            const Radial t = tgg_radial(rho, std::sqrt(sig[i] * sig[i] + sig[j] * sig[j]));
            const double sr = 1.0 - f.f;
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) {
                    const double v = sr * ((x == y ? t.P : 0.0) + t.W * r[x] * r[y]);
                    M[(3LL * i + x) * n + 3 * j + y] = v;
                    M[(3LL * j + x) * n + 3 * i + y] = v;
                }
        }
    }
}
