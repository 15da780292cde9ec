// Schedule of the scaled coupled Newton-Schulz iteration (host code, shared by the finite
// FP64, mixed-precision and periodic loops, and run on the CPU by the tests).
//
// Sign-function form of the coupled iteration: with x^2 the eigenvalues of P = Z Y in
// [l^2, u^2], the step T = (al/2)(3 I - al^2 P) maps x to f(x) = (al x/2)(3 - al^2 x^2);
// al^2 = 3/(u^2 + u l + l^2) gives f(l) = f(u), so [l, u] goes onto [f(l), 1].  f stays
// positive for x < sqrt(3)/al, so any l below the true bound (and any u above it) only
// costs speed; an l above it does too, since f is increasing on (0, l] (l <= 1/al) with
// f(x)/x >= al >= 1 there, so smaller eigenvalues still grow every step.  al = 1 near
// convergence and for the last step.
#pragma once
#include <algorithm>
#include <cmath>

namespace mbdgb {
namespace ns {

struct Coeffs { double c1, c3; };   // T = c1 I + c3 P

// The step's coefficients for the current bounds (l, u) on sqrt(eig(P)), which it advances.
inline Coeffs step(double &l, double &u, bool last) {
    double al = 1.0;
    if (!last && l < 0.999) al = std::sqrt(3.0 / (u * u + u * l + l * l));
    const Coeffs c{1.5 * al, -0.5 * al * al * al};
    l = std::min(1.0, 0.5 * al * l * (3.0 - al * al * l * l));
    u = 1.0;
    return c;
}

// Estimated lower bound on sqrt(eig(Y0)), Y0 = Q/s, from the smallest Ritz value of a 48-step
// Lanczos run on Q.  That value converges slowly: it is 3-6 times the smallest eigenvalue of Q
// at 500-2000 atoms, so a fraction of it may still lie above the true bound (which costs steps
// only, see above); on those spectra a quarter of it takes one step fewer than a half.
inline double lower_estimate(double ritz_min, double s, double fraction = 0.25) {
    return std::sqrt(std::max(fraction * ritz_min / s, 1e-12));
}

// Stopping test of the mixed-precision loop after the residual r = |I - P|_F of step it > 0
// (prev: that of the step before): r below tol; a step taken from inside the quadratic basin
// (prev < 0.5) that fails to halve the residual; or a step about to be taken whose exact
// bound leaves no more than the precision floor.  For an eigenvalue x = 1 - e of P the
// plain step leaves 1 - x' = 3/4 e^2 + 1/4 e^3, so from r < 0.5 the next residual is at most
// 0.875 r^2 in exact arithmetic.
inline bool mixed_last(double r, double prev, double tol, double floor) {
    return r < tol || (prev < 0.5 && r > 0.5 * prev) || (r < 0.5 && 0.875 * r * r < floor);
}

}  // namespace ns
}  // namespace mbdgb
