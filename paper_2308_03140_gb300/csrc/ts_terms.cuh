// Terms of the periodic TS pairwise sum (Secs. 2.6 and 2.7: Eq. pairwise with the oscillators
// of Eq. ts-scaling and the damping of Eq. fermi-damping, steepness 20; the lattice sum of
// 1/R^6 by Eq. ts-ewald).  Per cell
//     E = -1/2 sum_{i,j in cell} C6_ij s_ij,
//     s_ij = sum'_n h(|R_nij|) + sum_{|G| < kc} t_G cos(G . (R_j - R_i)) - delta_ij gamma^6/6,
//     h(r) = gamma^6 phi_r(gamma r) - (1 - f(r))/r^6,   t_G = gamma^3 phi_k(|G|/gamma)/Omega,
// where R_nij = R_j + n A - R_i runs over 0 < |R_nij| < rc, the G = 0 term is kept and the
// primed sum leaves out n = 0 when i = j: the Ewald sum of 1/R^6 minus the real-space sum of
// the damped-away part (1 - f)/R^6.  Everything here is __host__ __device__ so that the pair
// kernel's arithmetic can also be run, term for term, on the host by its checks.
#pragma once
#include "internal.h"

namespace mbdgb {
namespace ts {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kSqrtPi = 1.772453850905516027298167483341145183;
constexpr double kSteep = 20.0;   // steepness of the TS damping

// phi_r(x) = (x^-6 + x^-4 + x^-2/2) e^{-x^2} and its derivative.
__host__ __device__ inline void phi_r(double x, double &v, double &d) {
    const double ix2 = 1.0 / (x * x), e = exp(-x * x);
    const double p = ix2 * ix2 * ix2 + ix2 * ix2 + 0.5 * ix2;
    v = p * e;
    d = (-(6.0 * ix2 * ix2 * ix2 + 4.0 * ix2 * ix2 + ix2) / x - 2.0 * x * p) * e;
}

// phi_k(k) = pi^{3/2}/12 ((4 - 2k^2) e^{-k^2/4} + k^3 sqrt(pi) erfc(k/2)) and its derivative
// pi^{3/2}/12 (3 k^2 sqrt(pi) erfc(k/2) - 6 k e^{-k^2/4}) (the k^3 terms cancel).
__host__ __device__ inline void phi_k(double k, double &v, double &d) {
    const double c = kPi * kSqrtPi / 12.0, e = exp(-0.25 * k * k), ec = kSqrtPi * erfc(0.5 * k);
    v = c * ((4.0 - 2.0 * k * k) * e + k * k * k * ec);
    d = c * (3.0 * k * k * ec - 6.0 * k * e);
}

// One real-space image at distance rho of a pair with radius sum S: h, dh/drho and dh/dS.
struct Image { double h, dh, dhS; };
__host__ __device__ inline Image image_term(double rho, double S, double s_r, double gamma) {
    const double eta = rho / (s_r * S);
    const double f = 1.0 / (1.0 + exp(-kSteep * (eta - 1.0)));
    const double dfe = kSteep * f * (1.0 - f);
    const double ir2 = 1.0 / (rho * rho), ir6 = ir2 * ir2 * ir2;
    double pv, pd;
    phi_r(gamma * rho, pv, pd);
    const double g3 = gamma * gamma * gamma, g6 = g3 * g3;
    Image o;
    o.h = g6 * pv - (1.0 - f) * ir6;
    o.dh = g6 * gamma * pd + dfe / (s_r * S) * ir6 + 6.0 * (1.0 - f) * ir6 / rho;
    o.dhS = -dfe * eta / S * ir6;
    return o;
}

// Per reciprocal vector: t = gamma^3 phi_k(|G|/gamma)/Omega and rp = (dt/d|G|)/|G| for
// |G| < kc (G = 0 included, with rp = 0 there since it only multiplies G), zero beyond.
struct Recip { double t, rp; };
__host__ __device__ inline Recip recip_term(double Gn, double gamma, double vol, double kc) {
    Recip o{0.0, 0.0};
    if (!(Gn < kc)) return o;
    double v, d;
    phi_k(Gn / gamma, v, d);
    o.t = gamma * gamma * gamma * v / vol;
    o.rp = Gn > 0.0 ? gamma * gamma * d / (vol * Gn) : 0.0;
    return o;
}

// Lattice translations n with |x + n A| < rc (as the periodic dipole sums bound them:
// |f_c(r)| <= |r| |b_c| / 2 pi for the fractional coordinate f_c of any r).
__host__ __device__ inline void image_range(const CellGeom &c, const double *x, int *lo, int *hi) {
    for (int k = 0; k < 3; ++k) {
        const double bn = sqrt(c.B[3 * k] * c.B[3 * k] + c.B[3 * k + 1] * c.B[3 * k + 1] + c.B[3 * k + 2] * c.B[3 * k + 2]);
        const double L = c.rc * bn / (2.0 * kPi) + 1e-9;
        const double f = x[0] * c.Ainv[k] + x[1] * c.Ainv[3 + k] + x[2] * c.Ainv[6 + k];
        lo[k] = static_cast<int>(ceil(-L - f));
        hi[k] = static_cast<int>(floor(L - f));
    }
}

// Contributions of the ordered pair (i, j), x = R_j - R_i (self: i == j), to the sums of
// atom i.  e = -1/2 C6 s_ij (E = sum over ordered pairs); s = s_ij; grv = dE/dR_vdW,i from
// both orders of the pair (-C6 sum dh/dS); gR = dE/dR_i from both orders (zero for i == j);
// gA[3 f + c] = dE/dA_fc of this ordered pair (rows of A are the lattice vectors, Cartesian
// positions fixed): the images give -1/2 C6 h'(r) n_f r_c/r, the reciprocal terms
// -1/2 C6 [-(1/2 pi) (B K)_fc - (sum_G t cos) (A^-T)_fc] with
// K_ec = sum_G rp cos G_e G_c - x_e sum_G t sin G_c (from dG = -G dA^T B / 2 pi and
// dOmega = Omega A^-T dA).  tab holds (t, rp) per G; Si, Sj point at the structure factors
// e^{i G.R} of atoms i and j for G = 0 with a stride of sstride between reciprocal vectors.
// bad is set when an image other than the self image n = 0 lies at zero distance.
struct Pair { double e, s, grv, gR[3], gA[9]; bool bad; };
__host__ __device__ inline void pair_terms(const CellGeom &c, const double *x, bool self, double c6, double S,
                                           double s_r, int nG, const double *G, const double *tab, const double2 *Si,
                                           const double2 *Sj, long long sstride, Pair &o) {
    const double g = c.gamma;
    double s = 0.0, dS = 0.0, gr[3] = {0.0, 0.0, 0.0}, ga[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    o.bad = false;
    int lo[3], hi[3];
    image_range(c, x, lo, hi);
    for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
        for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
            for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
                const int nn[3] = {n0, n1, n2};
                double r[3];
                for (int e = 0; e < 3; ++e) r[e] = x[e] + n0 * c.A[e] + n1 * c.A[3 + e] + n2 * c.A[6 + e];
                const double rho2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                if (rho2 >= c.rc * c.rc) continue;
                if (rho2 < 1e-16) {
                    if (!self || n0 || n1 || n2) o.bad = true;
                    continue;
                }
                const double rho = sqrt(rho2);
                const Image t = image_term(rho, S, s_r, g);
                s += t.h;
                dS += t.dhS;
                const double w = t.dh / rho;
                for (int e = 0; e < 3; ++e) gr[e] += w * r[e];
                for (int f = 0; f < 3; ++f)
                    for (int e = 0; e < 3; ++e) ga[3 * f + e] += nn[f] * w * r[e];
            }
    double sc = 0.0, vs[3] = {0.0, 0.0, 0.0}, M[6] = {0, 0, 0, 0, 0, 0};   // M: xx yy zz xy xz yz
    for (int q = 0; q < nG; ++q) {
        const double t = tab[2 * q], rp = tab[2 * q + 1];
        if (t == 0.0 && rp == 0.0) continue;
        const double2 a = Si[q * sstride], b = Sj[q * sstride];
        const double cs = b.x * a.x + b.y * a.y, sn = b.y * a.x - b.x * a.y;   // cos, sin of G.(R_j - R_i)
        const double Gx = G[3 * q], Gy = G[3 * q + 1], Gz = G[3 * q + 2];
        sc += t * cs;
        const double ts = t * sn, rc_ = rp * cs;
        vs[0] += ts * Gx;
        vs[1] += ts * Gy;
        vs[2] += ts * Gz;
        M[0] += rc_ * Gx * Gx;
        M[1] += rc_ * Gy * Gy;
        M[2] += rc_ * Gz * Gz;
        M[3] += rc_ * Gx * Gy;
        M[4] += rc_ * Gx * Gz;
        M[5] += rc_ * Gy * Gz;
    }
    s += sc;
    if (self) {
        const double g3 = g * g * g;
        s -= g3 * g3 / 6.0;
    }
    const double h = -0.5 * c6;
    o.e = h * s;
    o.s = s;
    o.grv = -c6 * dS;
    for (int e = 0; e < 3; ++e) o.gR[e] = self ? 0.0 : c6 * (gr[e] - vs[e]);
    const double Ms[9] = {M[0], M[3], M[4], M[3], M[1], M[5], M[4], M[5], M[2]};
    for (int f = 0; f < 3; ++f)
        for (int cc = 0; cc < 3; ++cc) {
            double bk = 0.0;   // (B K)_f,cc
            for (int e = 0; e < 3; ++e) bk += c.B[3 * f + e] * (Ms[3 * e + cc] - x[e] * vs[cc]);
            o.gA[3 * f + cc] = h * (ga[3 * f + cc] - bk / (2.0 * kPi) - sc * c.Ainv[3 * cc + f]);
        }
}

}  // namespace ts
}  // namespace mbdgb
