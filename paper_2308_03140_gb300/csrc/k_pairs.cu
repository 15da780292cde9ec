// Per-atom and pair kernels of MBD@rsSCS for sm_103a (FP64).
//
//  prepare_atoms   TS scaling, Eq. (ts-scaling); alpha(iu), Eq. (dyn-pol); Mayer width,
//                  Eq. (mayer)
//  build_scs       A = alpha^{-1} + T^scs per frequency, Eqs. (scs), (scs-sr-dipole), (tgg)
//  contract_screen Eq. (contraction) and Eqs. (casimir-polder), (scale-rvdw-scs)
//  build_q         Eq. (q-matrix) with T^lr = g(Rbar) T, Eq. (mbd-lr-dipole)
//  energy_trace    Eq. (mbd-energy) from the trace of Q^{1/2}
//  mbd_grad_pass   Eq. (mbd-gradient): 1/4 Tr(Q^{-1/2} dQ) - 3/2 sum d omega
//  chain_screen    chain rule back through Eqs. (casimir-polder), (scale-rvdw-scs)
//  scs_grad_pass   the derivative of Eq. (scs), d alpha_bar = -alpha_bar dA alpha_bar,
//                  contracted as in Eq. (scs-gradient) but from the adjoint side
//  ts_chain        chain rule back through Eq. (ts-scaling)
//
// The dipole tensors are written T_ab = P delta_ab + W r_a r_b with radial P, W.
// Pair loops keep one CTA per "row" atom and stride over partner atoms, so every
// per-atom sum is a fixed-order block reduction (deterministic, no atomics).
#include "internal.h"
#include "pair_math.cuh"

namespace mbdgb {
namespace {

using namespace pairs;

// ---- per-atom preparation ------------------------------------------------------------
__global__ void k_prepare(AtomBufs b, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    const double a0r = b.a0ref[i], c6r = b.c6ref[i], rr = b.rref[i], v = b.ratio[i];
    const double x = b.R[3 * i], y = b.R[3 * i + 1], z = b.R[3 * i + 2];
    if (!(a0r > 0.0) || !(c6r > 0.0) || !(rr > 0.0) || !(v > 0.0) || !isfinite(x) ||
        !isfinite(y) || !isfinite(z) || !isfinite(a0r * c6r * rr * v))
        atomicOr(status, ST_INPUT);
    const double a0 = a0r * v, om = 4.0 * c6r / (3.0 * a0r * a0r);
    b.a0[i] = a0;
    b.om[i] = om;
    b.rv[i] = rr * cbrt(v);
    const double cm = sqrt(2.0 / kPi) / 3.0;
    for (int k = 0; k < b.nf1; ++k) {
        const double uo = b.u[k] / om;
        const double al = a0 / (1.0 + uo * uo);
        b.al_u[k * b.N + i] = al;
        b.sig_u[k * b.N + i] = cbrt(cm * al);
    }
}

// MBD-NL oscillators (Sec. 2.7, paragraph MBD-NL): no screening.  Inputs per atom are
// alpha0_ref (a0ref), C6_ref (c6ref), ra = alpha0_df/alpha0_df,ref (in rref) and
// rw = omega_df/omega_df,ref (in ratio).  Eq. (mbd-nl-scaling): alpha0 = alpha0_ref ra,
// omega = omega_ref rw with omega_ref = 4 C6_ref / (3 alpha0_ref^2); Eq. (mbd-nl-rvdw):
// R = 5/2 alpha0_ref^(1/7) ra^(1/3).  They are written where the screened parameters go
// (abar0, ombar, rbar; c6bar = 3/4 alpha0^2 omega; abar(iu) = alpha0 / (1 + u^2/omega^2))
// and into a0, om, rv.
__global__ void k_nl_params(AtomBufs b, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    const double a0r = b.a0ref[i], c6r = b.c6ref[i], ra = b.rref[i], rw = b.ratio[i];
    const double x = b.R[3 * i], y = b.R[3 * i + 1], z = b.R[3 * i + 2];
    if (!(a0r > 0.0) || !(c6r > 0.0) || !(ra > 0.0) || !(rw > 0.0) || !isfinite(x) || !isfinite(y) ||
        !isfinite(z) || !isfinite(a0r * c6r * ra * rw))
        atomicOr(status, ST_INPUT);
    const double a0 = a0r * ra, om = 4.0 * c6r / (3.0 * a0r * a0r) * rw;
    const double rd = 2.5 * pow(a0r, 1.0 / 7.0) * cbrt(ra);
    b.a0[i] = a0;
    b.om[i] = om;
    b.rv[i] = rd;
    b.abar0[i] = a0;
    b.ombar[i] = om;
    b.rbar[i] = rd;
    b.c6bar[i] = 0.75 * a0 * a0 * om;
    for (int k = 0; k < b.nf1; ++k) {
        const double uo = b.u[k] / om;
        b.abar[k * b.N + i] = a0 / (1.0 + uo * uo);
    }
}

// dE/d(alpha0_ref, C6_ref, ra, rw) [4][N] of MBD-NL from dE/d(alpha0, omega, R) of the
// oscillators (the MBD pair pass), times *scale (device) if given.
__global__ void k_nl_chain(AtomBufs b, const double *g_ab0, const double *g_om, const double *g_rd,
                           const double *scale, double *gp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    const int N = b.N;
    const double w = scale ? scale[0] : 1.0;
    const double a0r = b.a0ref[i], c6r = b.c6ref[i], ra = b.rref[i], rw = b.ratio[i];
    const double om = b.ombar[i], rd = b.rbar[i];
    gp[i] = w * (g_ab0[i] * ra - g_om[i] * 2.0 * om / a0r + g_rd[i] * rd / (7.0 * a0r));
    gp[N + i] = w * (g_om[i] * om / c6r);
    gp[2 * N + i] = w * (g_ab0[i] * a0r + g_rd[i] * rd / (3.0 * ra));
    gp[3 * N + i] = w * (g_om[i] * om / rw);
}

// ---- screening matrices ------------------------------------------------------------
// A CTA of 32 x 8 threads takes atoms j0..j0+31 (x) against i0..i0+7 (y); thread (i, j) with
// j < i computes block (i, j) of every frequency's matrix and writes it in its rows (32
// consecutive blocks of a row per warp), then the CTA writes the mirrored blocks (j, i) --
// the blocks are symmetric 3x3 tensors, and r -> -r leaves them unchanged -- from a shared
// tile, so that those rows too are written in contiguous runs.  Thread (i, i) writes the
// diagonal block 1/alpha_i(u) I.  The factorisations read the lower triangle, the residuals
// of the refined solves the full matrix.  Rows >= n: identity (k_pad_identity).
__global__ void __launch_bounds__(256) k_build_scs(AtomBufs b, double beta, double a, double *M, long long ld,
                                                   long long mstride, int *status) {
    const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 8;
    if (j0 > i0 + 7) return;   // the whole tile lies above the diagonal
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 32 + tx;
    const int j = j0 + tx, i = i0 + ty;
    const bool pair = i < b.N && j < i, diag = i < b.N && j == i;
    __shared__ double T[24][97];
    double r[3] = {0.0, 0.0, 0.0}, rho = 1.0, sr = 0.0, far_P = 0.0, far_W = 0.0, far2 = 0.0;
    if (pair) {
        r[0] = b.R[3 * j] - b.R[3 * i];
        r[1] = b.R[3 * j + 1] - b.R[3 * i + 1];
        r[2] = b.R[3 * j + 2] - b.R[3 * i + 2];
        rho = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (!(rho > 1e-8)) atomicOr(status, ST_INPUT);
        sr = 1.0 - fermi(rho, b.rv[i] + b.rv[j], beta, a).f;
        // the bare tensor's radial parts, which T^GG equals beyond rho/s = kGaussFar (the far
        // branch of tgg_radial), once per pair for every frequency
        const double ir = 1.0 / rho, ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
        far_P = ir3;
        far_W = -3.0 * ir5;
        far2 = rho * rho / (kGaussFar * kGaussFar);   // s^2 below this: the far branch
    }
    for (int k = 0; k < b.nf1; ++k) {
        double *Mk = M + k * mstride;
        double v[9];
        if (pair) {
            const double si = b.sig_u[k * b.N + i], sj = b.sig_u[k * b.N + j];
            const double s2 = si * si + sj * sj;
            double P = far_P, W = far_W;
            if (!(s2 < far2)) {
                const Radial tg = tgg_radial(rho, sqrt(s2));
                P = tg.P;
                W = tg.W;
            }
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                double *row = Mk + (3LL * i + x) * ld + 3 * j;
#pragma unroll
                for (int y = 0; y < 3; ++y) {
                    v[3 * x + y] = sr * ((x == y ? P : 0.0) + W * r[x] * r[y]);
                    row[y] = v[3 * x + y];
                }
            }
        } else if (diag) {
            const double d = 1.0 / b.al_u[k * b.N + i];
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) Mk[(3LL * i + x) * ld + 3 * i + y] = (x == y) ? d : 0.0;
        }
        __syncthreads();   // the last frequency's mirror reads are done
        if (pair) {
#pragma unroll
            for (int x = 0; x < 3; ++x)
#pragma unroll
                for (int y = 0; y < 3; ++y) T[3 * ty + x][3 * tx + y] = v[3 * x + y];
        }
        __syncthreads();
        // mirrored blocks (j, i): 96 rows 3 j + x by 24 columns 3 i + y of this tile
        for (int e = t; e < 96 * 24; e += 256) {
            const int row = e / 24, col = e - 24 * row;
            const int jl = row / 3, x = row - 3 * jl, il = col / 3, y = col - 3 * il;
            const int jj = j0 + jl, ii = i0 + il;
            if (ii < b.N && jj < ii) Mk[(3LL * jj + x) * ld + 3 * ii + y] = T[3 * il + x][3 * jl + y];
        }
    }
}

__global__ void k_pad_identity(double *M, long long ld, int n, long long mstride) {
    // rows n..ld-1, all columns up to the row (lower part), per matrix (blockIdx.y)
    double *Mk = M + blockIdx.y * mstride;
    const long long rows = ld - n;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < rows * ld;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long r = n + e / ld, c = e % ld;
        Mk[r * ld + c] = (r == c) ? 1.0 : 0.0;
        if (c < n) Mk[c * ld + r] = 0.0;   // keep the upper half of the pad columns clean
    }
}

__global__ void k_rhs_identity(double *X, long long ld, int n, long long xstride) {
    double *Xk = X + blockIdx.y * xstride;
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < ld;
         p += static_cast<long long>(gridDim.x) * blockDim.x)
        for (int c = 0; c < 3; ++c) Xk[3 * p + c] = (p < n && (p % 3) == c) ? 1.0 : 0.0;
}

// Eqs. (casimir-polder), (scale-rvdw-scs) for atom i from its alpha_bar(u) row: C6bar,
// omega_bar, Rbar; flags a non-positive alpha_bar0 or C6bar.
__device__ __forceinline__ void screened_params_atom(const AtomBufs &b, int i, int *status) {
    double c6 = 0.0;
    for (int k = 0; k < b.nf1; ++k) {
        const double ab = b.abar[k * b.N + i];
        c6 += b.wu[k] * ab * ab;   // wu[0] = 0: the static point carries no weight
    }
    c6 *= 3.0 / kPi;
    const double ab0 = b.abar[i];
    if (!(ab0 > 0.0) || !(c6 > 0.0)) atomicOr(status, ST_NEG_ALPHA);
    b.abar0[i] = ab0;
    b.c6bar[i] = c6;
    b.ombar[i] = 4.0 * c6 / (3.0 * ab0 * ab0);
    b.rbar[i] = b.rv[i] * cbrt(ab0 / b.a0[i]);
}

// alpha_bar_i(u) = 1/3 sum_a X[3i+a][a]; then C6bar, omega_bar, Rbar per atom.
__global__ void k_contract_screen(AtomBufs b, const double *X, long long xstride, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    for (int k = 0; k < b.nf1; ++k) {
        const double *Xk = X + k * xstride;
        b.abar[k * b.N + i] = (Xk[9LL * i] + Xk[9LL * i + 4] + Xk[9LL * i + 8]) / 3.0;
    }
    screened_params_atom(b, i, status);
}

// Screened parameters from alpha_bar(u) rows already in b.abar (the learned model's path).
__global__ void k_screened_params(AtomBufs b, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < b.N) screened_params_atom(b, i, status);
}

// ---- coupled-oscillator matrix -------------------------------------------------------
__global__ void k_build_q(AtomBufs b, double beta, double a, double *Q, long long ld, int *status) {
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    if (i >= b.N || j >= b.N) return;
    double blk[9];
    if (i == j) {
        const double w2 = b.ombar[i] * b.ombar[i];
        for (int e = 0; e < 9; ++e) blk[e] = (e % 4 == 0) ? w2 : 0.0;
    } else {
        const double r[3] = {b.R[3 * j] - b.R[3 * i], b.R[3 * j + 1] - b.R[3 * i + 1],
                             b.R[3 * j + 2] - b.R[3 * i + 2]};
        const double rho2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], rho = sqrt(rho2);
        if (!(rho > 1e-8)) atomicOr(status, ST_INPUT);
        const Fermi g = fermi(rho, b.rbar[i] + b.rbar[j], beta, a);
        const double pre = b.ombar[i] * b.ombar[j] * sqrt(b.abar0[i] * b.abar0[j]) * g.f;
        const double ir3 = 1.0 / (rho2 * rho), ir5 = ir3 / rho2;
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y)
                blk[3 * x + y] = pre * ((x == y ? ir3 : 0.0) - 3.0 * r[x] * r[y] * ir5);
    }
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) Q[(3LL * i + x) * ld + 3 * j + y] = blk[3 * x + y];
}

// Pad rows/columns n..ld-1 of Q: zero couplings and the diagonal value omega_bar_0^2.
// Any diagonal entry of a symmetric matrix lies inside its spectrum, so the padded
// eigenvalue never widens [lambda_min, lambda_max] and the blocks stay decoupled.
__global__ void k_pad_q(double *Q, long long ld, int n, const double *ombar) {
    const double d = ombar[0] * ombar[0];
    const long long rows = ld - n;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < rows * ld;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long r = n + e / ld, c = e % ld;
        Q[r * ld + c] = (r == c) ? d : 0.0;
        Q[c * ld + r] = (r == c) ? d : 0.0;
    }
}

// E = 1/2 sqrt(s) Tr Y - 3/2 sum omega_bar, Neumaier-compensated, one CTA.
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__global__ void k_energy(const double *Y, long long ld, int n, const double *ombar, int N,
                         double sqrt_s, double *out) {
    double s = 0.0, c = 0.0;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        double t, e;
        two_sum(s, 0.5 * sqrt_s * Y[p * ld + p], t, e);
        s = t; c += e;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double t, e;
        two_sum(s, -1.5 * ombar[i], t, e);
        s = t; c += e;
    }
    __shared__ double ss[256], cc[256];
    ss[threadIdx.x] = s;
    cc[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, Cc = 0.0;
        for (int k = 0; k < blockDim.x; ++k) {
            double t, e;
            two_sum(S, ss[k], t, e);
            S = t;
            Cc += e + cc[k];
        }
        out[0] = S + Cc;
    }
}

// ---- gradients -------------------------------------------------------------------------
// One CTA (128 threads) per row atom i; G = zscale * Z = Q^{-1/2}.
// For ordered pairs (i, j):  g_c[i]    += 1/2 c_j g <G_ij, T>
//                            g_rbar[i] += 1/2 c_i c_j dg/dS <G_ij, T>
//                            gR[i]     -= 1/2 c_i c_j <G_ij, d(gT)/dr>,  r = R_j - R_i
// (both blocks (i,j) and (j,i) of the symmetric sum are folded into the factor 1/2).
// tq (optional): Tr (Q^{1/2})_ii per atom.  dE/d omega_bar_i = Tr (Z Q)_ii / (2 omega_bar_i) - 3/2
// exactly (diagonal and coupling terms of dQ/d omega_bar_i); two terms of ~1.5 cancel there, so
// a Z with a relative error e gives an absolute error ~e.  With tq (second order in the error
// of Z) the difference is taken from it instead.
__global__ void __launch_bounds__(128) k_mbd_grad(AtomBufs b, double beta, double a, const double *Z,
                                                  long long ld, double zscale, MbdGradOut o, const double *tq) {
    const int i = blockIdx.x;
    const double ci = b.ombar[i] * sqrt(b.abar0[i]);
    const double Ri[3] = {b.R[3 * i], b.R[3 * i + 1], b.R[3 * i + 2]};
    double acc[5] = {0, 0, 0, 0, 0};   // g_c, g_rbar, gR x3
    for (int j = threadIdx.x; j < b.N; j += 128) {
        if (j == i) continue;
        const double r[3] = {b.R[3 * j] - Ri[0], b.R[3 * j + 1] - Ri[1], b.R[3 * j + 2] - Ri[2]};
        const double rho2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], rho = sqrt(rho2);
        const double cj = b.ombar[j] * sqrt(b.abar0[j]);
        const Fermi g = fermi(rho, b.rbar[i] + b.rbar[j], beta, a);
        double G[9];
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) G[3 * x + y] = Z[(3LL * i + x) * ld + 3 * j + y];
        const double tr = G[0] + G[4] + G[8];
        double Gr[3], Gtr[3];
        for (int x = 0; x < 3; ++x) {
            Gr[x] = G[3 * x] * r[0] + G[3 * x + 1] * r[1] + G[3 * x + 2] * r[2];
            Gtr[x] = G[x] * r[0] + G[3 + x] * r[1] + G[6 + x] * r[2];
        }
        const double rGr = r[0] * Gr[0] + r[1] * Gr[1] + r[2] * Gr[2];
        const double ir = 1.0 / rho, ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
        const double P = ir3, W = -3.0 * ir5, dP = -3.0 * ir3 * ir, dW = 15.0 * ir5 * ir;
        const double GT = P * tr + W * rGr;
        acc[0] += 0.5 * zscale * cj * g.f * GT;
        acc[1] += 0.5 * zscale * ci * cj * g.df_dS * GT;
        const double pre = -0.5 * zscale * ci * cj;
        for (int c = 0; c < 3; ++c) {
            const double GdT = (dP * tr + dW * rGr) * r[c] * ir + W * (Gr[c] + Gtr[c]);
            acc[2 + c] += pre * (g.f * GdT + g.df_drho * r[c] * ir * GT);
        }
    }
    __shared__ double scratch[4 * 5];
    block_sum128<5>(acc, scratch);
    if (threadIdx.x == 0) {
        const double sa = sqrt(b.abar0[i]);
        const double trd = Z[(3LL * i) * ld + 3 * i] + Z[(3LL * i + 1) * ld + 3 * i + 1] +
                           Z[(3LL * i + 2) * ld + 3 * i + 2];
        const double g_om = tq ? tq[i] / (2.0 * b.ombar[i]) - 1.5
                               : 0.25 * zscale * trd * 2.0 * b.ombar[i] - 1.5 + acc[0] * sa;
        o.g_ombar[i] = g_om;
        o.g_abar0[i] = acc[0] * b.ombar[i] / (2.0 * sa);
        o.g_rbar[i] = acc[1];
        o.gR[3 * i] = acc[2];
        o.gR[3 * i + 1] = acc[3];
        o.gR[3 * i + 2] = acc[4];
    }
}

__global__ void k_chain(AtomBufs b, MbdGradOut o, double *h, double *g_a0, double *g_rv, double *H,
                        long long xstride) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    const double ab0 = b.abar0[i], x = ab0 / b.a0[i], x13 = cbrt(x), x23 = x13 * x13;
    const double g_om = o.g_ombar[i], g_rb = o.g_rbar[i];
    const double g_c6 = g_om * 4.0 / (3.0 * ab0 * ab0);
    const double g_ab0 = o.g_abar0[i] - g_om * 8.0 * b.c6bar[i] / (3.0 * ab0 * ab0 * ab0) +
                         g_rb * b.rv[i] / (3.0 * x23 * b.a0[i]);
    g_a0[i] = -g_rb * b.rv[i] / (3.0 * x23) * ab0 / (b.a0[i] * b.a0[i]);
    g_rv[i] = g_rb * x13;
    for (int k = 0; k < b.nf1; ++k) {
        const double hk = (k == 0) ? g_ab0 : g_c6 * 3.0 / kPi * b.wu[k] * 2.0 * b.abar[k * b.N + i];
        h[k * b.N + i] = hk;
        double *Hk = H + k * xstride + 9LL * i;
        for (int e = 0; e < 9; ++e) Hk[e] = (e % 4 == 0) ? hk : 0.0;
    }
}

// One CTA (128 threads) per row atom i; all frequencies per pair.
// With Ws = V_i X_j^T + X_i V_j^T (3x3, the blocks (i,j) and (j,i) of V X^T folded):
//   dE/d alpha_i(u) += -1/3 <Ws, dB/d alpha_i>,  dE/dR_vdW,i += -1/3 <Ws, dB/dS>,
//   dE/dR_i += +1/3 <Ws, dB/dr>  (r = R_j - R_i),  B = (1 - f) T^GG,
// plus the diagonal block: dE/d alpha_i(u) += -1/3 sum_x (V X^T)_{ix,ix} (-1/alpha_i^2).
// The per-pair arithmetic runs in T (double, or float in the reduced-precision modes);
// the per-thread and block sums are FP64.
// Dynamic shared memory: nf1 * 128 doubles of per-thread accumulators.
template <typename T> struct PairMath;
template <> struct PairMath<double> {
    static __device__ __forceinline__ Fermi fermi(double r, double S, double b, double a) { return pairs::fermi(r, S, b, a); }
    static __device__ __forceinline__ Radial radial(double r, double s) { return pairs::tgg_radial(r, s); }
};
template <> struct PairMath<float> {
    static __device__ __forceinline__ FermiF fermi(float r, float S, float b, float a) { return pairs::fermi_f(r, S, b, a); }
    static __device__ __forceinline__ RadialF radial(float r, float s) { return pairs::tgg_radial_f(r, s); }
};

// X, V ([nf1][xstride]), sig and al ([nf1][N], sigma_i(iu) and alpha_i(iu)) are read in T:
// the FP64 arrays, or FP32 copies of them in the reduced-precision modes.
template <typename T>
__global__ void __launch_bounds__(128) k_scs_grad(AtomBufs b, double beta, double a, const T *X, const T *V,
                                                  const T *sig, const T *al, long long xstride, double *g_a0,
                                                  double *g_om, double *g_rv, double *gR) {
    extern __shared__ double gal_s[];   // [nf1][128]
    const int i = blockIdx.x, t = threadIdx.x;
    for (int k = 0; k < b.nf1; ++k) gal_s[k * 128 + t] = 0.0;
    const double Ri[3] = {b.R[3 * i], b.R[3 * i + 1], b.R[3 * i + 2]};
    double acc[4] = {0, 0, 0, 0};   // g_rv, gR x3
    for (int j = t; j < b.N; j += 128) {
        if (j == i) continue;
        const T r[3] = {static_cast<T>(b.R[3 * j] - Ri[0]), static_cast<T>(b.R[3 * j + 1] - Ri[1]),
                        static_cast<T>(b.R[3 * j + 2] - Ri[2])};
        const T rho = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]), ir = T(1) / rho;
        const auto f = PairMath<T>::fermi(rho, static_cast<T>(b.rv[i] + b.rv[j]), static_cast<T>(beta), static_cast<T>(a));
        const T sr = T(1) - f.f;
        // Far pairs whose damping has rounded to f = 1 (1 - f = 0 and both derivatives 0)
        // contribute exact zeros at every frequency: beyond ~3.8 beta (R_i + R_j) in FP32,
        // ~7.1 in FP64.
        if (sr == T(0) && f.df_drho == T(0) && f.df_dS == T(0)) continue;
        T pacc[4] = {0, 0, 0, 0};
        for (int k = 0; k < b.nf1; ++k) {
            const T *Vk = V + k * xstride, *Xk = X + k * xstride;
            T Ws[9];
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) {
                    T w = 0;
                    for (int c = 0; c < 3; ++c)
                        w += Vk[9LL * i + 3 * x + c] * Xk[9LL * j + 3 * y + c] + Xk[9LL * i + 3 * x + c] * Vk[9LL * j + 3 * y + c];
                    Ws[3 * x + y] = w;
                }
            const T tr = Ws[0] + Ws[4] + Ws[8];
            T Wr[3], Wtr[3];
            for (int x = 0; x < 3; ++x) {
                Wr[x] = Ws[3 * x] * r[0] + Ws[3 * x + 1] * r[1] + Ws[3 * x + 2] * r[2];
                Wtr[x] = Ws[x] * r[0] + Ws[3 + x] * r[1] + Ws[6 + x] * r[2];
            }
            const T rWr = r[0] * Wr[0] + r[1] * Wr[1] + r[2] * Wr[2];
            const T si = sig[k * b.N + i], sj = sig[k * b.N + j];
            const T s = sqrt(si * si + sj * sj);
            const auto q = PairMath<T>::radial(rho, s);
            const T WT = q.P * tr + q.W * rWr;            // <Ws, T^GG>
            const T WTs = q.dPs * tr + q.dWs * rWr;       // <Ws, dT^GG/ds>
            // ds/d alpha_i = (sigma_i / s) * sigma_i / (3 alpha_i)
            const T dsda = si * si / (T(3) * s * al[k * b.N + i]);
            gal_s[k * 128 + t] += -1.0 / 3.0 * static_cast<double>(sr * WTs * dsda);
            pacc[0] += -f.df_dS * WT;
            for (int c = 0; c < 3; ++c) {
                const T WdT = (q.dP * tr + q.dW * rWr) * r[c] * ir + q.W * (Wr[c] + Wtr[c]);
                pacc[1 + c] += sr * WdT - f.df_drho * r[c] * ir * WT;
            }
        }
        acc[0] += -1.0 / 3.0 * static_cast<double>(pacc[0]);
        for (int c = 0; c < 3; ++c) acc[1 + c] += 1.0 / 3.0 * static_cast<double>(pacc[1 + c]);
    }
    __syncthreads();
    __shared__ double scratch[4 * 4];
    block_sum128<4>(acc, scratch);
    // reduce the per-frequency accumulators, add the diagonal block, chain to alpha0, omega
    if (t < b.nf1) {
        const int k = t;
        double sacc = 0.0;
        for (int e = 0; e < 128; ++e) sacc += gal_s[k * 128 + e];
        const T *Vk = V + k * xstride, *Xk = X + k * xstride;
        double wd = 0.0;
        for (int e = 0; e < 9; ++e) wd += static_cast<double>(Vk[9LL * i + e]) * static_cast<double>(Xk[9LL * i + e]);
        const double alk = b.al_u[k * b.N + i];
        sacc += -1.0 / 3.0 * wd * (-1.0 / (alk * alk));
        gal_s[k * 128] = sacc;
    }
    __syncthreads();
    if (t == 0) {
        double ga0 = 0.0, gom = 0.0;
        const double a0 = b.a0[i], om = b.om[i];
        for (int k = 0; k < b.nf1; ++k) {
            const double u = b.u[k], q = 1.0 + u * u / (om * om);
            const double gal = gal_s[k * 128];
            ga0 += gal / q;
            gom += gal * a0 * 2.0 * u * u / (om * om * om) / (q * q);
        }
        g_a0[i] += ga0;
        g_om[i] += gom;
        g_rv[i] += acc[0];
        gR[3 * i] += acc[1];
        gR[3 * i + 1] += acc[2];
        gR[3 * i + 2] += acc[3];
    }
}

// FP32 copies of X, V ([nf1][xstride] each) and of sigma(iu), alpha(iu) ([nf1][N] each),
// packed in that order into w.
__global__ void k_scs_grad_inputs_f32(const double *X, const double *V, const double *sig, const double *al,
                                      long long nx, long long na, float *w) {
    const long long total = 2 * nx + 2 * na;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        double v;
        if (e < nx) v = X[e];
        else if (e < 2 * nx) v = V[e - nx];
        else if (e < 2 * nx + na) v = sig[e - 2 * nx];
        else v = al[e - 2 * nx - na];
        w[e] = static_cast<float>(v);
    }
}

// TS pairwise dispersion (Secs. 2.6 and 2.7, Eq. pairwise with the TS oscillators of Eq. ts-scaling and
// the damping of Eq. fermi-damping, steepness 20): one CTA per atom i, threads over j.  For
// the pair (i, j) the energy is -C6_ij h(r), h = f/r^6, C6_ij = 3/2 a_i a_j w_i w_j / (w_i + w_j)
// (the two ordered terms of -1/2 sum_{i != j}).  Per atom: eatom[i] = -1/2 sum_j C6_ij h_ij;
// dE/dR_i = sum_j C6_ij h'(r) r_hat (r = R_j - R_i); dE/d a_i, dE/d w_i, dE/d R_vdW,i of the
// TS-scaled oscillators (b.a0, b.om, b.rv) into ga0, gom, grv.
__global__ void __launch_bounds__(128) k_ts_pairs(AtomBufs b, double s_r, double *eatom, double *gR, double *ga0,
                                                  double *gom, double *grv) {
    const int i = blockIdx.x;
    const double ai = b.a0[i], wi = b.om[i], rvi = b.rv[i];
    const double Ri[3] = {b.R[3 * i], b.R[3 * i + 1], b.R[3 * i + 2]};
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};   // e, gR x3, ga0, gom, grv
    for (int j = threadIdx.x; j < b.N; j += 128) {
        if (j == i) continue;
        const double r[3] = {b.R[3 * j] - Ri[0], b.R[3 * j + 1] - Ri[1], b.R[3 * j + 2] - Ri[2]};
        const double rho2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], rho = sqrt(rho2);
        const double aj = b.a0[j], wj = b.om[j];
        const double c6 = 1.5 * ai * aj * wi * wj / (wi + wj);
        const Fermi f = fermi(rho, rvi + b.rv[j], s_r, 20.0);
        const double ir6 = 1.0 / (rho2 * rho2 * rho2);
        const double h = f.f * ir6, dh = f.df_drho * ir6 - 6.0 * h / rho, dhS = f.df_dS * ir6;
        acc[0] += -0.5 * c6 * h;
        for (int c = 0; c < 3; ++c) acc[1 + c] += c6 * dh * r[c] / rho;
        acc[4] += -h * c6 / ai;
        acc[5] += -h * c6 * (1.0 / wi - 1.0 / (wi + wj));
        acc[6] += -c6 * dhS;
    }
    __shared__ double scratch[4 * 7];
    block_sum128<7>(acc, scratch);
    if (threadIdx.x == 0) {
        eatom[i] = acc[0];
        gR[3 * i] = acc[1];
        gR[3 * i + 1] = acc[2];
        gR[3 * i + 2] = acc[3];
        ga0[i] = acc[4];
        gom[i] = acc[5];
        grv[i] = acc[6];
    }
}

__global__ void k_ts_chain(AtomBufs b, const double *g_a0, const double *g_om, const double *g_rv,
                           const double *scale, double *gp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    const int N = b.N;
    const double w = scale ? scale[0] : 1.0;
    const double v = b.ratio[i], a0r = b.a0ref[i], v13 = cbrt(v);
    gp[i] = w * (g_a0[i] * v - g_om[i] * 8.0 * b.c6ref[i] / (3.0 * a0r * a0r * a0r));
    gp[N + i] = w * (g_om[i] * 4.0 / (3.0 * a0r * a0r));
    gp[2 * N + i] = w * (g_rv[i] * v13);
    gp[3 * N + i] = w * (g_a0[i] * a0r + g_rv[i] * b.rref[i] / (3.0 * v13 * v13));
}

__global__ void k_scale_copy(const double *x, int n, const double *scale, double *y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (scale ? scale[0] : 1.0) * x[i];
}

inline int cdiv(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

}  // namespace

void prepare_atoms(const AtomBufs &b, int *status, cudaStream_t s) {
    count_launches(1);
    k_prepare<<<cdiv(b.N, 128), 128, 0, s>>>(b, status);
}

void build_scs(const AtomBufs &b, double beta, double a, double *M, long long ld, long long mstride,
               int *status, cudaStream_t s) {
    dim3 grid(cdiv(b.N, 32), cdiv(b.N, 8));
    count_launches(1);
    k_build_scs<<<grid, dim3(32, 8), 0, s>>>(b, beta, a, M, ld, mstride, status);   // 18.6 KB static shared
    const int n = 3 * b.N;
    if (ld > n) {
        count_launches(1);
        k_pad_identity<<<dim3(cdiv((ld - n) * ld, 256), b.nf1), 256, 0, s>>>(M, ld, n, mstride);
    }
}

void pad_identity(double *M, long long ld, int n, int nf1, long long mstride, cudaStream_t s) {
    if (ld <= n) return;
    count_launches(1);
    k_pad_identity<<<dim3(cdiv((ld - n) * ld, 256), nf1), 256, 0, s>>>(M, ld, n, mstride);
}

void init_rhs_identity(double *X, long long ld, int n, int nf1, long long xstride, cudaStream_t s) {
    count_launches(1);
    k_rhs_identity<<<dim3(cdiv(ld, 256), nf1), 256, 0, s>>>(X, ld, n, xstride);
}

void contract_screen(const AtomBufs &b, const double *X, long long ld, long long xstride, int *status,
                     cudaStream_t s) {
    (void)ld;
    count_launches(1);
    k_contract_screen<<<cdiv(b.N, 128), 128, 0, s>>>(b, X, xstride, status);
}

void screened_params(const AtomBufs &b, int *status, cudaStream_t s) {
    count_launches(1);
    k_screened_params<<<cdiv(b.N, 128), 128, 0, s>>>(b, status);
}

void build_q(const AtomBufs &b, double beta, double a, double *Q, long long ld, int *status,
             cudaStream_t s) {
    dim3 grid(cdiv(b.N, 32), cdiv(b.N, 8));
    count_launches(1);
    k_build_q<<<grid, dim3(32, 8), 0, s>>>(b, beta, a, Q, ld, status);
    const int n = 3 * b.N;
    if (ld > n) {
        count_launches(1);
        k_pad_q<<<cdiv((ld - n) * ld, 256), 256, 0, s>>>(Q, ld, n, b.ombar);
    }
}

void energy_trace(const double *Y, long long ld, int n, const double *ombar, int N, double sqrt_s,
                  double *out, cudaStream_t s) {
    count_launches(1);
    k_energy<<<1, 256, 0, s>>>(Y, ld, n, ombar, N, sqrt_s, out);
}

void mbd_grad_pass(const AtomBufs &b, double beta, double a, const double *Z, long long ld,
                   double zscale, const MbdGradOut &o, cudaStream_t s, const double *tq) {
    count_launches(1);
    k_mbd_grad<<<b.N, 128, 0, s>>>(b, beta, a, Z, ld, zscale, o, tq);
}

void chain_screen(const AtomBufs &b, const MbdGradOut &o, double *h, double *g_a0, double *g_rv,
                  double *H, long long ld, long long xstride, cudaStream_t s) {
    // zero the padded rows of the adjoint right-hand sides, then fill the atom rows
    for (int k = 0; k < b.nf1; ++k)
        cudaMemsetAsync(H + k * xstride, 0, sizeof(double) * 3 * ld, s);
    count_launches(1);
    k_chain<<<cdiv(b.N, 128), 128, 0, s>>>(b, o, h, g_a0, g_rv, H, xstride);
}

void scs_grad_pass(const AtomBufs &b, double beta, double a, const double *X, const double *V,
                   long long xstride, double *g_a0, double *g_om, double *g_rv, double *gR, float *work32,
                   cudaStream_t s) {
    const size_t smem = sizeof(double) * b.nf1 * 128;
    if (work32) {
        const long long nx = xstride * b.nf1, na = static_cast<long long>(b.nf1) * b.N;
        float *X32 = work32, *V32 = work32 + nx, *sig32 = work32 + 2 * nx, *al32 = sig32 + na;
        count_launches(2);
        k_scs_grad_inputs_f32<<<cdiv(2 * nx + 2 * na, 256), 256, 0, s>>>(X, V, b.sig_u, b.al_u, nx, na, work32);
        k_scs_grad<float><<<b.N, 128, smem, s>>>(b, beta, a, X32, V32, sig32, al32, xstride, g_a0, g_om, g_rv, gR);
    } else {
        count_launches(1);
        k_scs_grad<double><<<b.N, 128, smem, s>>>(b, beta, a, X, V, b.sig_u, b.al_u, xstride, g_a0, g_om, g_rv,
                                                 gR);
    }
}

void nl_params(const AtomBufs &b, int *status, cudaStream_t s) {
    count_launches(1);
    k_nl_params<<<cdiv(b.N, 128), 128, 0, s>>>(b, status);
}

void nl_chain(const AtomBufs &b, const MbdGradOut &o, const double *scale, double *gp, cudaStream_t s) {
    count_launches(1);
    k_nl_chain<<<cdiv(b.N, 128), 128, 0, s>>>(b, o.g_abar0, o.g_ombar, o.g_rbar, scale, gp);
}

void ts_pairs(const AtomBufs &b, double s_r, double *eatom, double *gR, double *ga0, double *gom, double *grv,
              cudaStream_t s) {
    count_launches(1);
    k_ts_pairs<<<b.N, 128, 0, s>>>(b, s_r, eatom, gR, ga0, gom, grv);
}

void ts_chain(const AtomBufs &b, const double *g_a0, const double *g_om, const double *g_rv,
              const double *scale, double *gp, cudaStream_t s) {
    count_launches(1);
    k_ts_chain<<<cdiv(b.N, 128), 128, 0, s>>>(b, g_a0, g_om, g_rv, scale, gp);
}

void scale_copy(const double *x, int n, const double *scale, double *y, cudaStream_t s) {
    count_launches(1);
    k_scale_copy<<<cdiv(n, 256), 256, 0, s>>>(x, n, scale, y);
}

}  // namespace mbdgb
