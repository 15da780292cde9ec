// Host run of the Newton-Schulz schedule of the library (csrc/ns_schedule.h) on the eigenvalues
// of Q: in exact arithmetic the coupled iteration acts on each eigenvalue separately
// (x = eigenvalue of P = Z Y, x' = x (c1 + c3 x)^2), so the schedule's step count and final
// residual follow from the spectrum alone.  Test infrastructure: built by
// tests/test_ns_schedule.py into tests/_build.
#include <cmath>
#include <vector>

#include "ns_schedule.h"

using namespace mbdgb;

// lam [n]: eigenvalues of Q; s = 1.05 max(lam) as the library's Lanczos-tightened scale;
// ritz_min: the smallest Lanczos Ritz value; mixed = 1: the mixed loop's stopping test with
// the floor floor_per_sqrt_n * sqrt(n), each residual evaluated as if every eigenvalue of P
// also carried an error of floor_el (the precision floor); mixed = 0: the FP64 loop (stop
// one step after r < tol).  Returns the number of steps; *resid_out: the exact residual of
// the final iterate.
extern "C" int ns_scalar_run(const double *lam, int n, double ritz_min, double fraction, int mixed, double tol,
                             double floor_per_sqrt_n, double floor_el, double *resid_out) {
    double lmax = 0.0;
    for (int k = 0; k < n; ++k) lmax = std::fmax(lmax, lam[k]);
    const double s = 1.05 * lmax;
    std::vector<double> x(lam, lam + n);
    for (double &v : x) v /= s;
    double l = ns::lower_estimate(ritz_min, s, fraction), u = 1.05, prev = 1e300;
    int it = 0;
    for (; it < 200; ++it) {
        bool last = false;
        if (it > 0) {
            double r2 = 0.0;
            for (double v : x) r2 += (1.0 - v) * (1.0 - v) + floor_el * floor_el;
            const double r = std::sqrt(r2);
            last = mixed ? ns::mixed_last(r, prev, tol, floor_per_sqrt_n * std::sqrt(static_cast<double>(n)))
                         : r < tol;
            prev = r;
        }
        const ns::Coeffs c = ns::step(l, u, last);
        for (double &v : x) v = v * (c.c1 + c.c3 * v) * (c.c1 + c.c3 * v);
        if (last) {
            ++it;
            break;
        }
    }
    double r2 = 0.0;
    for (double v : x) r2 += (1.0 - v) * (1.0 - v);
    *resid_out = std::sqrt(r2);
    return it;
}
