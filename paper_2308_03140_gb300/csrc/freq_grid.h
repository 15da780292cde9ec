// Imaginary-frequency grid of the Casimir-Polder integral (host code, shared by the MBD
// evaluation and the learned model's features).
#pragma once
#include <cmath>
#include <vector>

namespace mbdgb {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n, started from the
// asymptotic root estimate of Tricomi.  Ascending nodes.
inline void legendre_rule(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.141592653589793238462643383279502884;
    for (int k = 1; k <= n; ++k) {
        double t = std::cos(pi * (4.0 * k - 1.0) / (4.0 * n + 2.0)) *
                   (1.0 - 1.0 / (8.0 * n * n) + 1.0 / (8.0 * n * n * n));
        double deriv = 1.0;
        for (int it = 0; it < 64; ++it) {
            double pm1 = 1.0, p = t;   // P_0, P_1
            for (int m = 2; m <= n; ++m) {
                const double pn = ((2.0 * m - 1.0) * t * p - (m - 1.0) * pm1) / m;
                pm1 = p;
                p = pn;
            }
            if (n == 1) { p = t; pm1 = 1.0; }
            deriv = n * (pm1 - t * p) / (1.0 - t * t);
            const double step = p / deriv;
            t -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        {
            double pm1 = 1.0, p = t;
            for (int m = 2; m <= n; ++m) {
                const double pn = ((2.0 * m - 1.0) * t * p - (m - 1.0) * pm1) / m;
                pm1 = p;
                p = pn;
            }
            if (n == 1) { p = t; pm1 = 1.0; }
            deriv = n * (pm1 - t * p) / (1.0 - t * t);
        }
        x[n - k] = t;
        w[n - k] = 2.0 / ((1.0 - t * t) * deriv * deriv);
    }
}

// The grid of Eq. (casimir-polder) with n_freq Gauss-Legendre nodes x mapped to
// u = 0.6 (1 + x)/(1 - x), du = 1.2/(1 - x)^2 dx (Sec. 3.3): u[0] = 0 (the static point, weight
// 0) and the nodes u[1..n_freq] ascending, with their weights wu.
inline void casimir_polder_grid(int n_freq, std::vector<double> &u, std::vector<double> &wu) {
    std::vector<double> x, w;
    legendre_rule(n_freq, x, w);
    u.assign(n_freq + 1, 0.0);
    wu.assign(n_freq + 1, 0.0);
    for (int k = 0; k < n_freq; ++k) {
        u[k + 1] = 0.6 * (1.0 + x[k]) / (1.0 - x[k]);
        wu[k + 1] = w[k] * 1.2 / ((1.0 - x[k]) * (1.0 - x[k]));
    }
}

}  // namespace mbdgb
