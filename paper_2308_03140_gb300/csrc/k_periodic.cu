// Periodic MBD@rsSCS kernels for sm_103a (FP64): Sec. 2.2 (periodic boundary conditions)
// and the Ewald summation of the dipole tensor.
//
//  structure_factors   S[g][i] = e^{i G_g . R_i} for every reciprocal vector in use
//  build_scs_periodic  Gamma-point screening matrices: lattice sums of (1 - f) T^GG
//  build_q_periodic    Q(q) for every Bloch vector of the grid:
//                      T^lr(q)_ij = sum_n [T^erfc(r) - (1 - g(r)) T(r)] e^{-i q.r}
//                               + (4 pi/Omega) sum_G k^ k^T e^{-k^2/4 gamma^2} e^{i G.(R_j - R_i)}
//                               - delta_ij 4 gamma^3/(3 sqrt pi),   r = R_j + R_n - R_i, k = G + q
//  complex helpers     planar batched Newton-Schulz support (4M GEMMs on the FP64 kernel)
//  periodic_mbd_grad   dE = sum_q (1/nk) 1/4 Re Tr(Q(q)^{-1/2} dQ(q)) - 3/2 sum d omega_bar,
//                      for atoms, screened parameters and the lattice (Cartesian positions
//                      fixed; dk/dA_cd = -k_d A^{-1}_{.c}, dOmega/dA = Omega A^{-T})
//  scs_grad_periodic   the finite SCS adjoint pair pass summed over lattice images
//
// The reciprocal phase e^{+i G.(R_j - R_i)} with k = G + q follows from Poisson summation of
// sum_n T(r) e^{-i q.r}; the erfc numerator is the -grad grad of erfc(gamma r)/r; the
// damped-away part (1 - g) T is removed in real space because it decays exponentially.
#include "internal.h"
#include "pair_math.cuh"

namespace mbdgb {
namespace {

using namespace pairs;

constexpr int kQT = 16;   // atom tile edge of the pair-tile kernels (16 x 16 threads)
constexpr int kGC = 64;   // reciprocal vectors staged per chunk

__device__ __forceinline__ double frac_coord(const CellGeom &c, const double *v, int k) {
    return v[0] * c.Ainv[k] + v[1] * c.Ainv[3 + k] + v[2] * c.Ainv[6 + k];
}

// Lattice translations n with |x + n A| < rc: n_c in [-L_c - f_c(x), L_c - f_c(x)],
// L_c = rc |b_c| / (2 pi) (|f_c(r)| <= |r| |b_c| / 2 pi for any r).
__device__ __forceinline__ void image_box(const CellGeom &c, const double *x, int *lo, int *hi) {
    for (int k = 0; k < 3; ++k) {
        const double bn = sqrt(c.B[3 * k] * c.B[3 * k] + c.B[3 * k + 1] * c.B[3 * k + 1] + c.B[3 * k + 2] * c.B[3 * k + 2]);
        const double L = c.rc * bn / (2.0 * kPi) + 1e-9, f = frac_coord(c, x, k);
        lo[k] = static_cast<int>(ceil(-L - f));
        hi[k] = static_cast<int>(floor(L - f));
    }
}

// Symmetric 3x3 stored as xx, yy, zz, xy, xz, yz; contractions with P delta + W r r.
struct Sym6 { double v[6]; };
__device__ __forceinline__ double sym_tr(const double *w) { return w[0] + w[1] + w[2]; }
__device__ __forceinline__ void sym_mv(const double *w, const double *r, double *o) {
    o[0] = w[0] * r[0] + w[3] * r[1] + w[4] * r[2];
    o[1] = w[3] * r[0] + w[1] * r[1] + w[5] * r[2];
    o[2] = w[4] * r[0] + w[5] * r[1] + w[2] * r[2];
}

__global__ void k_structure_factors(const double *R, int N, const double *G, int nG, double2 *S) {
    const long long total = static_cast<long long>(nG) * N;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long g = e / N, i = e % N;
        const double ph = G[3 * g] * R[3 * i] + G[3 * g + 1] * R[3 * i + 1] + G[3 * g + 2] * R[3 * i + 2];
        double sn, cs;
        sincos(ph, &sn, &cs);
        S[e] = make_double2(cs, sn);
    }
}

// ---- Gamma-point screening matrices ------------------------------------------------
// Thread (i, j), j <= i, writes block (i, j) of every frequency's matrix and its mirror:
// delta_ij I / alpha_i + sum over images r = R_j - R_i + n A (0 < |r| < rc) of (1 - f) T^GG.
__global__ void k_build_scs_periodic(AtomBufs b, CellGeom c, double beta, double a, double *M, long long ld,
                                     long long mstride, int *status) {
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    if (i >= b.N || j > i) return;
    const double x[3] = {b.R[3 * j] - b.R[3 * i], b.R[3 * j + 1] - b.R[3 * i + 1], b.R[3 * j + 2] - b.R[3 * i + 2]};
    int lo[3], hi[3];
    image_box(c, x, lo, hi);
    const double S = b.rv[i] + b.rv[j];
    for (int k = 0; k < b.nf1; ++k) {
        const double si = b.sig_u[k * b.N + i], sj = b.sig_u[k * b.N + j], s = sqrt(si * si + sj * sj);
        double acc[6] = {0, 0, 0, 0, 0, 0};
        bool bad = false;
        for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
            for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
                for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
                    double r[3];
                    for (int e = 0; e < 3; ++e) r[e] = x[e] + n0 * c.A[e] + n1 * c.A[3 + e] + n2 * c.A[6 + e];
                    const double rho2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    if (rho2 >= c.rc * c.rc) continue;
                    if (rho2 < 1e-16) {
                        if (i != j || n0 || n1 || n2) bad = true;
                        continue;
                    }
                    const double rho = sqrt(rho2);
                    const Fermi f = fermi(rho, S, beta, a);
                    const Radial t = tgg_radial(rho, s);
                    const double sr = 1.0 - f.f;
                    acc[0] += sr * (t.P + t.W * r[0] * r[0]);
                    acc[1] += sr * (t.P + t.W * r[1] * r[1]);
                    acc[2] += sr * (t.P + t.W * r[2] * r[2]);
                    acc[3] += sr * t.W * r[0] * r[1];
                    acc[4] += sr * t.W * r[0] * r[2];
                    acc[5] += sr * t.W * r[1] * r[2];
                }
        if (bad) atomicOr(status, ST_INPUT);
        if (i == j) {
            const double d = 1.0 / b.al_u[k * b.N + i];
            acc[0] += d; acc[1] += d; acc[2] += d;
        }
        const double blk[9] = {acc[0], acc[3], acc[4], acc[3], acc[1], acc[5], acc[4], acc[5], acc[2]};
        double *Mk = M + k * mstride;
        for (int xx = 0; xx < 3; ++xx)
            for (int y = 0; y < 3; ++y) {
                Mk[(3LL * i + xx) * ld + 3 * j + y] = blk[3 * xx + y];
                Mk[(3LL * j + xx) * ld + 3 * i + y] = blk[3 * xx + y];
            }
    }
}

// ---- Q(q) for every Bloch vector ------------------------------------------------------
// grid (upper-triangle tile pairs, nk); thread (ty, tx) of tile (I, J) owns the atom pair
// (i, j) = (16 I + ty, 16 J + tx) when i <= j, and writes block (i, j) and its Hermitian
// mirror (j, i) = conj(block)^T (the 3x3 blocks are complex symmetric).
__device__ __forceinline__ void tile_pair(int t, int ntile, int &I, int &J) {
    I = 0;
    while (t >= ntile - I) { t -= ntile - I; ++I; }
    J = I + t;
}

// The reduced-precision staging of the gradient's reciprocal sum (F32: the mixed modes).
template <typename R> struct Vec2;
template <> struct Vec2<double> { using T = double2; };
template <> struct Vec2<float> { using T = float2; };
template <typename R>
__device__ __forceinline__ void stage_chunk_r(const PeriodicBufs &p, int N, const double *q, const int *gl, int g0,
                                              int m, int I, int J, R (*sk)[3], R *sc, R *sf, typename Vec2<R>::T (*sSi)[kQT],
                                              typename Vec2<R>::T (*sSj)[kQT], R *sG) {
    const double pre = 4.0 * kPi / p.cell.vol, i4g2 = 0.25 / (p.cell.gamma * p.cell.gamma);
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
        const int gi = gl[g0 + e];
        const double kx = p.G[3 * gi] + q[0], ky = p.G[3 * gi + 1] + q[1], kz = p.G[3 * gi + 2] + q[2];
        const double k2 = kx * kx + ky * ky + kz * kz;
        sk[e][0] = static_cast<R>(kx); sk[e][1] = static_cast<R>(ky); sk[e][2] = static_cast<R>(kz);
        sc[e] = static_cast<R>(pre * exp(-k2 * i4g2) / k2);
        sf[e] = static_cast<R>(2.0 / k2 + 2.0 * i4g2);
        sG[3 * e] = static_cast<R>(p.G[3 * gi]);
        sG[3 * e + 1] = static_cast<R>(p.G[3 * gi + 1]);
        sG[3 * e + 2] = static_cast<R>(p.G[3 * gi + 2]);
    }
    for (int e = threadIdx.x; e < m * 2 * kQT; e += blockDim.x) {
        const int gg = e / (2 * kQT), aa = e % (2 * kQT);
        const int atom = aa < kQT ? I * kQT + aa : J * kQT + aa - kQT;
        const double2 v = atom < N ? p.S[static_cast<long long>(gl[g0 + gg]) * N + atom] : make_double2(0.0, 0.0);
        typename Vec2<R>::T w;
        w.x = static_cast<R>(v.x);
        w.y = static_cast<R>(v.y);
        if (aa < kQT) sSi[gg][aa] = w; else sSj[gg][aa - kQT] = w;
    }
}

// Stage chunk [g0, g0 + m) of Bloch vector k's reciprocal list: k-vectors, the coefficient
// (4 pi/Omega) e^{-k^2/4 gamma^2}/k^2 and the structure factors of the tile's atoms.
__device__ __forceinline__ void stage_chunk(const PeriodicBufs &p, int N, const double *q, const int *gl, int g0,
                                            int m, int I, int J, double (*sk)[3], double *sc, double2 (*sSi)[kQT],
                                            double2 (*sSj)[kQT], double *sG) {
    const double pre = 4.0 * kPi / p.cell.vol, i4g2 = 0.25 / (p.cell.gamma * p.cell.gamma);
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
        const int gi = gl[g0 + e];
        const double kx = p.G[3 * gi] + q[0], ky = p.G[3 * gi + 1] + q[1], kz = p.G[3 * gi + 2] + q[2];
        const double k2 = kx * kx + ky * ky + kz * kz;
        sk[e][0] = kx; sk[e][1] = ky; sk[e][2] = kz;
        sc[e] = pre * exp(-k2 * i4g2) / k2;
        if (sG) { sG[3 * e] = p.G[3 * gi]; sG[3 * e + 1] = p.G[3 * gi + 1]; sG[3 * e + 2] = p.G[3 * gi + 2]; }
    }
    for (int e = threadIdx.x; e < m * 2 * kQT; e += blockDim.x) {
        const int gg = e / (2 * kQT), aa = e % (2 * kQT);
        const int atom = aa < kQT ? I * kQT + aa : J * kQT + aa - kQT;
        const double2 v = atom < N ? p.S[static_cast<long long>(gl[g0 + gg]) * N + atom] : make_double2(0.0, 0.0);
        if (aa < kQT) sSi[gg][aa] = v; else sSj[gg][aa - kQT] = v;
    }
}

__global__ void __launch_bounds__(256) k_build_q_periodic(AtomBufs b, PeriodicBufs p, double beta, double a,
                                                          double *Q, long long ld, int ntile, int *status) {
    const int kq = blockIdx.y;
    int I, J;
    tile_pair(blockIdx.x, ntile, I, J);
    const int ty = threadIdx.x / kQT, tx = threadIdx.x % kQT;
    const int i = I * kQT + ty, j = J * kQT + tx;
    const bool valid = i < b.N && j < b.N && (I < J || ty <= tx);
    const CellGeom &c = p.cell;
    const double q[3] = {p.kq[3 * kq], p.kq[3 * kq + 1], p.kq[3 * kq + 2]};
    double Tr[6] = {0, 0, 0, 0, 0, 0}, Ti[6] = {0, 0, 0, 0, 0, 0};
    if (valid) {   // real space
        const double x[3] = {b.R[3 * j] - b.R[3 * i], b.R[3 * j + 1] - b.R[3 * i + 1], b.R[3 * j + 2] - b.R[3 * i + 2]};
        const double S = b.rbar[i] + b.rbar[j];
        int lo[3], hi[3];
        image_box(c, x, lo, hi);
        bool bad = false;
        for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
            for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
                for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
                    double r[3];
                    for (int e = 0; e < 3; ++e) r[e] = x[e] + n0 * c.A[e] + n1 * c.A[3 + e] + n2 * c.A[6 + e];
                    const double rho2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    if (rho2 >= c.rc * c.rc) continue;
                    if (rho2 < 1e-16) {
                        if (i != j || n0 || n1 || n2) bad = true;
                        continue;
                    }
                    const double rho = sqrt(rho2);
                    const RadialT te = erfc_radial(rho, c.gamma), tb = bare_radial(rho);
                    const Fermi g = fermi(rho, S, beta, a);
                    const double P = te.P - (1.0 - g.f) * tb.P, W = te.W - (1.0 - g.f) * tb.W;
                    double sn, cs;
                    sincos(-(q[0] * r[0] + q[1] * r[1] + q[2] * r[2]), &sn, &cs);
                    const double F[6] = {P + W * r[0] * r[0], P + W * r[1] * r[1], P + W * r[2] * r[2],
                                         W * r[0] * r[1], W * r[0] * r[2], W * r[1] * r[2]};
#pragma unroll
                    for (int e = 0; e < 6; ++e) { Tr[e] += F[e] * cs; Ti[e] += F[e] * sn; }
                }
        if (bad) atomicOr(status, ST_INPUT);
    }
    // reciprocal space
    __shared__ double sk[kGC][3], sc[kGC];
    __shared__ double2 sSi[kGC][kQT], sSj[kGC][kQT];
    const int cnt = p.gcount[kq];
    const int *gl = p.glist + static_cast<long long>(kq) * p.maxG;
    for (int g0 = 0; g0 < cnt; g0 += kGC) {
        const int m = min(kGC, cnt - g0);
        __syncthreads();
        stage_chunk(p, b.N, q, gl, g0, m, I, J, sk, sc, sSi, sSj, nullptr);
        __syncthreads();
        if (valid)
            for (int gg = 0; gg < m; ++gg) {
                const double2 si = sSi[gg][ty], sj = sSj[gg][tx];
                const double cf = sc[gg];
                const double pr = cf * (si.x * sj.x + si.y * sj.y), pi = cf * (si.x * sj.y - si.y * sj.x);
                const double kx = sk[gg][0], ky = sk[gg][1], kz = sk[gg][2];
                const double kk[6] = {kx * kx, ky * ky, kz * kz, kx * ky, kx * kz, ky * kz};
#pragma unroll
                for (int e = 0; e < 6; ++e) { Tr[e] += pr * kk[e]; Ti[e] += pi * kk[e]; }
            }
    }
    if (!valid) return;
    if (i == j) {
        const double self = 4.0 * c.gamma * c.gamma * c.gamma / (3.0 * sqrt(kPi));
        Tr[0] -= self; Tr[1] -= self; Tr[2] -= self;
    }
    const double pre = b.ombar[i] * b.ombar[j] * sqrt(b.abar0[i] * b.abar0[j]);
    const int ix[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
    double *Qr = Q + static_cast<long long>(kq) * 2 * ld * ld, *Qi = Qr + ld * ld;
    const double w2 = b.ombar[i] * b.ombar[i];
    for (int xx = 0; xx < 3; ++xx)
        for (int y = 0; y < 3; ++y) {
            const double vr = pre * Tr[ix[3 * xx + y]] + (i == j && xx == y ? w2 : 0.0);
            const double vi = pre * Ti[ix[3 * xx + y]];
            Qr[(3LL * i + xx) * ld + 3 * j + y] = vr;
            Qi[(3LL * i + xx) * ld + 3 * j + y] = vi;
            if (i != j) {
                Qr[(3LL * j + y) * ld + 3 * i + xx] = vr;
                Qi[(3LL * j + y) * ld + 3 * i + xx] = -vi;
            }
        }
}

// Padding rows and columns n..ld-1 of every Q_k: omega_0^2 on the diagonal, zero couplings.
__global__ void k_pad_q_periodic(double *Q, long long ld, int n, const double *ombar) {
    const double d = ombar[0] * ombar[0];
    double *Qr = Q + static_cast<long long>(blockIdx.y) * 2 * ld * ld, *Qi = Qr + ld * ld;
    const long long rows = ld - n;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < rows * ld;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long r = n + e / ld, cidx = e % ld;
        Qr[r * ld + cidx] = (r == cidx) ? d : 0.0;
        Qr[cidx * ld + r] = (r == cidx) ? d : 0.0;
        Qi[r * ld + cidx] = 0.0;
        Qi[cidx * ld + r] = 0.0;
    }
}

// ---- batched complex helpers -------------------------------------------------------
__global__ void k_scale_all(double *Y, long long count, double scale) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < count;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        Y[e] *= scale;
}

__global__ void k_caxpby_identity(double *Z, const double *P, long long ld, long long total, double a, double b) {
    // total = nk * 2 ld^2; Z = a I + b P (P may be null for Z = a I)
    const long long m2 = ld * ld;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long w = e % (2 * m2);
        const bool re = w < m2;
        const long long rc = re ? w : w - m2;
        Z[e] = (re && rc / ld == rc % ld ? a : 0.0) + (P ? b * P[e] : 0.0);
    }
}

__device__ __forceinline__ double block_sum256(double v, double *sh) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;
}

// out[0] += sum_k sum_{p,q < n} |P_k - I|^2 (both planes)
__global__ void __launch_bounds__(256) k_cfrob_dev_identity(const double *P, long long ld, int n, int nk,
                                                            double *out) {
    __shared__ double sh[8];
    const long long per = static_cast<long long>(n) * n, total = per * nk;
    double acc = 0.0;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < total; e += static_cast<long long>(gridDim.x) * 256) {
        const long long k = e / per, w = e % per, r = w / n, cidx = w % n;
        const double *Pr = P + k * 2 * ld * ld;
        const double vr = Pr[r * ld + cidx] - (r == cidx ? 1.0 : 0.0), vi = Pr[ld * ld + r * ld + cidx];
        acc += vr * vr + vi * vi;
    }
    const double t = block_sum256(acc, sh);
    if (threadIdx.x == 0) atomicAdd(out, t);
}

// out[0] = max over k and rows of sum_q |Q_k[p][q]| (complex modulus), via the ordering
// of non-negative doubles as unsigned integers.
__global__ void k_cmax_abs_rowsum(const double *Q, long long ld, int nk, unsigned long long *out) {
    const long long row = blockIdx.x * static_cast<long long>(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= ld * nk) return;
    const long long k = row / ld, p = row % ld;
    const double *Qr = Q + k * 2 * ld * ld + p * ld, *Qi = Qr + ld * ld;
    double acc = 0.0;
    for (long long cidx = lane; cidx < ld; cidx += 32) acc += sqrt(Qr[cidx] * Qr[cidx] + Qi[cidx] * Qi[cidx]);
    acc = warp_sum(acc);
    if (lane == 0) atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(acc)));
}

// Lanczos on every Q_k: vectors planar [nk][2][ld].
__global__ void __launch_bounds__(1024) k_clanczos_init(double *v, double *vprev, long long ld) {
    __shared__ double sh[32];
    double *vk = v + blockIdx.x * 2 * ld, *pk = vprev + blockIdx.x * 2 * ld;
    double ss = 0.0;
    for (long long e = threadIdx.x; e < ld; e += 1024) {
        const double xv = sin(0.7548776662 * static_cast<double>(e) + 0.5698402910) + 0.25;
        vk[e] = xv;
        vk[ld + e] = 0.0;
        pk[e] = 0.0;
        pk[ld + e] = 0.0;
        ss += xv * xv;
    }
    double t = warp_sum(ss);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        t = warp_sum(sh[threadIdx.x]);
        if (threadIdx.x == 0) sh[0] = t;
    }
    __syncthreads();
    const double inv = 1.0 / sqrt(sh[0]);
    for (long long e = threadIdx.x; e < ld; e += 1024) vk[e] *= inv;
}

__global__ void k_cgemv(const double *Q, long long ld, const double *v, double *w) {
    const long long row = blockIdx.x * static_cast<long long>(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= ld) return;
    const long long k = blockIdx.y;
    const double *Qr = Q + k * 2 * ld * ld + row * ld, *Qi = Qr + ld * ld;
    const double *vr = v + k * 2 * ld, *vi = vr + ld;
    double ar = 0.0, ai = 0.0;
    for (long long cidx = lane; cidx < ld; cidx += 32) {
        ar += Qr[cidx] * vr[cidx] - Qi[cidx] * vi[cidx];
        ai += Qr[cidx] * vi[cidx] + Qi[cidx] * vr[cidx];
    }
    ar = warp_sum(ar);
    ai = warp_sum(ai);
    if (lane == 0) {
        w[k * 2 * ld + row] = ar;
        w[k * 2 * ld + ld + row] = ai;
    }
}

__device__ double block_sum1024c(double v, double *sh) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = (threadIdx.x < 32) ? sh[threadIdx.x] : 0.0;
    if (threadIdx.x < 32) t = warp_sum(t);
    __syncthreads();
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

// alpha = Re v^H w; w -= alpha v + beta_prev vprev; beta = |w|; vprev = v; v = w / beta.
__global__ void __launch_bounds__(1024) k_clanczos_update(double *w, double *v, double *vprev, long long ld,
                                                          double *coef, int steps, int j) {
    __shared__ double sh[32];
    const long long off = blockIdx.x * 2 * ld, m = 2 * ld;
    double *wk = w + off, *vk = v + off, *pk = vprev + off;
    double *ck = coef + static_cast<long long>(blockIdx.x) * 2 * steps;
    double d = 0.0;
    for (long long e = threadIdx.x; e < m; e += 1024) d += wk[e] * vk[e];
    const double alpha = block_sum1024c(d, sh);
    const double bprev = j > 0 ? ck[2 * j - 1] : 0.0;
    double ss = 0.0;
    for (long long e = threadIdx.x; e < m; e += 1024) {
        const double xv = wk[e] - alpha * vk[e] - bprev * pk[e];
        wk[e] = xv;
        ss += xv * xv;
    }
    const double beta = sqrt(block_sum1024c(ss, sh));
    const double inv = beta > 1e-300 ? 1.0 / beta : 0.0;
    for (long long e = threadIdx.x; e < m; e += 1024) {
        pk[e] = vk[e];
        vk[e] = wk[e] * inv;
    }
    if (threadIdx.x == 0) {
        ck[2 * j] = alpha;
        ck[2 * j + 1] = beta;
    }
}

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__global__ void k_energy_periodic(const double *Y, long long ld, int n, int nk, const double *ombar, int N,
                                  double scale, double *out) {
    double s = 0.0, cc = 0.0;
    const long long total = static_cast<long long>(n) * nk;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
        const long long k = e / n, pp = e % n;
        double t, er;
        two_sum(s, scale * Y[k * 2 * ld * ld + pp * ld + pp], t, er);
        s = t; cc += er;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double t, er;
        two_sum(s, -1.5 * ombar[i], t, er);
        s = t; cc += er;
    }
    __shared__ double ss[256], sc2[256];
    ss[threadIdx.x] = s;
    sc2[threadIdx.x] = cc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, C = 0.0;
        for (int k = 0; k < blockDim.x; ++k) {
            double t, er;
            two_sum(S, ss[k], t, er);
            S = t;
            C += er + sc2[k];
        }
        out[0] = S + C;
    }
}

// ---- MBD gradient of the periodic energy ---------------------------------------------
// Thread (i <= j) of tile (I, J) at Bloch vector k: with z = w_ij Z_k[i, j] (w_ij = zscale/(4 nk),
// doubled for i != j, which folds in block (j, i)), only the symmetric part zs of the
// block meets the (symmetric) tensors.  Accumulates
//   zT = Re <conj zs, T^lr> (the self term included for i = j), zS = Re <conj zs, dT^lr/dS>, zx = Re <conj zs, dT^lr/dx>,
//   zA = Re <conj zs, dT^lr/dA>,
// then g_c[i] += c_j zT, g_c[j] += c_i zT, g_rbar[i,j] += c_i c_j zS, gR[j] += c_i c_j zx,
// gR[i] -= c_i c_j zx, gA += c_i c_j zA (c_i = omega_bar_i sqrt(abar0_i)).
// Real-space sums in FP64; the reciprocal sum in R (double, or float for the mixed modes,
// whose Z carries errors far above FP32 rounding), each chunk of kGC vectors summed in R and
// added into FP64 totals.
template <typename R>
__global__ void __launch_bounds__(256) k_mbd_grad_periodic(AtomBufs b, PeriodicBufs p, double beta, double a,
                                                           const double *Z, long long ld, double zscale, int ntile,
                                                           double *g_c, double *g_rbar, double *gR, double *gA) {
    const int kq = blockIdx.y;
    int I, J;
    tile_pair(blockIdx.x, ntile, I, J);
    const int ty = threadIdx.x / kQT, tx = threadIdx.x % kQT;
    const int i = I * kQT + ty, j = J * kQT + tx;
    const bool valid = i < b.N && j < b.N && (I < J || ty <= tx);
    const CellGeom &c = p.cell;
    const double q[3] = {p.kq[3 * kq], p.kq[3 * kq + 1], p.kq[3 * kq + 2]};
    double zr[6] = {0, 0, 0, 0, 0, 0}, zi[6] = {0, 0, 0, 0, 0, 0}, x[3] = {0, 0, 0}, fx[3] = {0, 0, 0};
    double zT = 0.0, zS = 0.0, zx[3] = {0, 0, 0}, zA[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double su = 0.0, M1[3] = {0, 0, 0}, M2[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (valid) {
        const double w = 0.25 * zscale / p.nk * (i == j ? 1.0 : 2.0);
        const double *Zr = Z + static_cast<long long>(kq) * 2 * ld * ld, *Zi = Zr + ld * ld;
        const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
        for (int e = 0; e < 6; ++e) {
            const long long o1 = (3LL * i + ia[e]) * ld + 3 * j + ib[e], o2 = (3LL * i + ib[e]) * ld + 3 * j + ia[e];
            zr[e] = 0.5 * w * (Zr[o1] + Zr[o2]);
            zi[e] = 0.5 * w * (Zi[o1] + Zi[o2]);
        }
        for (int e = 0; e < 3; ++e) x[e] = b.R[3 * j + e] - b.R[3 * i + e];
        for (int k = 0; k < 3; ++k) fx[k] = frac_coord(c, x, k);
        // real space
        const double S = b.rbar[i] + b.rbar[j];
        int lo[3], hi[3];
        image_box(c, x, lo, hi);
        for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
            for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
                for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
                    const int nn[3] = {n0, n1, n2};
                    double r[3];
                    for (int e = 0; e < 3; ++e) r[e] = x[e] + n0 * c.A[e] + n1 * c.A[3 + e] + n2 * c.A[6 + e];
                    const double rho2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    if (rho2 >= c.rc * c.rc || rho2 < 1e-16) continue;
                    const double rho = sqrt(rho2), irho = 1.0 / rho;
                    const RadialT te = erfc_radial(rho, c.gamma), tb = bare_radial(rho);
                    const Fermi g = fermi(rho, S, beta, a);
                    const double sr = 1.0 - g.f;
                    const double P = te.P - sr * tb.P, W = te.W - sr * tb.W;
                    const double dP = te.dP - sr * tb.dP + g.df_drho * tb.P, dW = te.dW - sr * tb.dW + g.df_drho * tb.W;
                    double sn, cs;
                    sincos(-(q[0] * r[0] + q[1] * r[1] + q[2] * r[2]), &sn, &cs);
                    double wr[6], wi[6];
                    for (int e = 0; e < 6; ++e) {
                        wr[e] = zr[e] * cs + zi[e] * sn;
                        wi[e] = zr[e] * sn - zi[e] * cs;
                    }
                    double wrr[3], wir[3];
                    sym_mv(wr, r, wrr);
                    sym_mv(wi, r, wir);
                    const double trr = sym_tr(wr), tri = sym_tr(wi);
                    const double rwr = r[0] * wrr[0] + r[1] * wrr[1] + r[2] * wrr[2];
                    const double rwi = r[0] * wir[0] + r[1] * wir[1] + r[2] * wir[2];
                    const double Fwr = P * trr + W * rwr, Fwi = P * tri + W * rwi;
                    zT += Fwr;
                    zS += g.df_dS * (tb.P * trr + tb.W * rwr);
                    for (int d = 0; d < 3; ++d) {
                        const double dFw = (dP * trr + dW * rwr) * r[d] * irho + 2.0 * W * wrr[d];
                        zx[d] += dFw + q[d] * Fwi;
                        for (int k = 0; k < 3; ++k) zA[3 * k + d] += nn[k] * dFw - q[d] * fx[k] * Fwi;
                    }
                }
    }
    // reciprocal space
    using R2 = typename Vec2<R>::T;
    __shared__ R sk[kGC][3], sc[kGC], sf[kGC], sG[3 * kGC];
    __shared__ R2 sSi[kGC][kQT], sSj[kGC][kQT];
    const int cnt = p.gcount[kq];
    const int *gl = p.glist + static_cast<long long>(kq) * p.maxG;
    R zrr[6], zir[6];
    for (int e = 0; e < 6; ++e) {
        zrr[e] = static_cast<R>(zr[e]);
        zir[e] = static_cast<R>(zi[e]);
    }
    for (int g0 = 0; g0 < cnt; g0 += kGC) {
        const int m = min(kGC, cnt - g0);
        __syncthreads();
        stage_chunk_r<R>(p, b.N, q, gl, g0, m, I, J, sk, sc, sf, sSi, sSj, sG);
        __syncthreads();
        if (valid) {
            R su_c = 0, M1_c[3] = {0, 0, 0}, M2_c[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int gg = 0; gg < m; ++gg) {
                const R2 si = sSi[gg][ty], sj = sSj[gg][tx];
                const R er = si.x * sj.x + si.y * sj.y, ei = si.x * sj.y - si.y * sj.x;   // e^{i G.x}
                const R cf = sc[gg];
                const R kv[3] = {sk[gg][0], sk[gg][1], sk[gg][2]};
                R us[6], vs[6];
#pragma unroll
                for (int e = 0; e < 6; ++e) {
                    us[e] = zrr[e] * er + zir[e] * ei;
                    vs[e] = zrr[e] * ei - zir[e] * er;
                }
                const R uk[3] = {us[0] * kv[0] + us[3] * kv[1] + us[4] * kv[2], us[3] * kv[0] + us[1] * kv[1] + us[5] * kv[2],
                                 us[4] * kv[0] + us[5] * kv[1] + us[2] * kv[2]};
                const R vk[3] = {vs[0] * kv[0] + vs[3] * kv[1] + vs[4] * kv[2], vs[3] * kv[0] + vs[1] * kv[1] + vs[5] * kv[2],
                                 vs[4] * kv[0] + vs[5] * kv[1] + vs[2] * kv[2]};
                const R kuk = kv[0] * uk[0] + kv[1] * uk[1] + kv[2] * uk[2];
                const R kvk = kv[0] * vk[0] + kv[1] * vk[1] + kv[2] * vk[2];
                su_c += cf * kuk;
                const R cv = cf * kvk, f2 = kuk * sf[gg];   // sf = 2/k^2 + 1/(2 gamma^2)
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    M1_c[d] += sG[3 * gg + d] * cv;
                    const R De = cf * (R(2) * uk[d] - f2 * kv[d]);   // D_e at e = d
#pragma unroll
                    for (int dd = 0; dd < 3; ++dd) M2_c[3 * dd + d] += kv[dd] * De;   // M2[d'][e] = k_d' D_e
                }
            }
            su += static_cast<double>(su_c);
            for (int d = 0; d < 3; ++d) M1[d] += static_cast<double>(M1_c[d]);
            for (int e = 0; e < 9; ++e) M2[e] += static_cast<double>(M2_c[e]);
        }
    }
    if (!valid) return;
    zT += su;
    if (i == j) zT -= 4.0 * c.gamma * c.gamma * c.gamma / (3.0 * sqrt(kPi)) * (zr[0] + zr[1] + zr[2]);   // self term
    for (int d = 0; d < 3; ++d) zx[d] -= M1[d];
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) {
            double t = -c.Ainv[3 * d + k] * su + fx[k] * M1[d];
            for (int e = 0; e < 3; ++e) t -= M2[3 * d + e] * c.Ainv[3 * e + k];
            zA[3 * k + d] += t;
        }
    const double ci = b.ombar[i] * sqrt(b.abar0[i]), cj = b.ombar[j] * sqrt(b.abar0[j]), cij = ci * cj;
    if (i == j) {
        atomicAdd(&g_c[i], 2.0 * ci * zT);
        atomicAdd(&g_rbar[i], 2.0 * cij * zS);
    } else {
        atomicAdd(&g_c[i], cj * zT);
        atomicAdd(&g_c[j], ci * zT);
        atomicAdd(&g_rbar[i], cij * zS);
        atomicAdd(&g_rbar[j], cij * zS);
        for (int d = 0; d < 3; ++d) {
            atomicAdd(&gR[3 * j + d], cij * zx[d]);
            atomicAdd(&gR[3 * i + d], -cij * zx[d]);
        }
    }
    for (int e = 0; e < 9; ++e) atomicAdd(&gA[e], cij * zA[e]);
}

// g_ombar = zscale/(4 nk) sum_k Re Tr Z_k[i,i] 2 omega_bar_i - 3/2 + g_c sqrt(abar0), or, with tq_i
// = (1/nk) sum_k Re Tr (Q(q_k)^{1/2})_ii given, the same derivative as tq_i / (2 omega_bar_i) - 3/2
// (the diagonal and coupling terms of dQ/d omega_bar_i together, second order in the error of Z);
// g_abar0 = g_c omega_bar / (2 sqrt(abar0)).
__global__ void k_mbd_grad_periodic_finalize(AtomBufs b, const double *Z, long long ld, int nk, double zscale,
                                             const double *g_c, MbdGradOut o, const double *tq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    double d = 0.0;
    for (int k = 0; k < nk; ++k) {
        const double *Zr = Z + static_cast<long long>(k) * 2 * ld * ld;
        for (int xx = 0; xx < 3; ++xx) d += Zr[(3LL * i + xx) * ld + 3 * i + xx];
    }
    const double sa = sqrt(b.abar0[i]);
    o.g_ombar[i] = tq ? tq[i] / (2.0 * b.ombar[i]) - 1.5
                      : 0.25 * zscale / nk * d * 2.0 * b.ombar[i] - 1.5 + g_c[i] * sa;
    o.g_abar0[i] = g_c[i] * b.ombar[i] / (2.0 * sa);
}

// out[i] = (1/rows) sum_r x[r][i] (compensated).
__global__ void k_mean_rows(const double *x, int rows, int N, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0, c = 0.0;
    for (int r = 0; r < rows; ++r) {
        double t, e;
        two_sum(s, x[static_cast<long long>(r) * N + i], t, e);
        s = t;
        c += e;
    }
    out[i] = (s + c) / rows;
}

// ---- SCS adjoint over lattice images -------------------------------------------------
// One CTA (128 threads) per atom i; partners j = 0..N-1 including j = i (its images).
// With Ws = V_i X_j^T + X_i V_j^T per frequency (blocks (i,j) and (j,i) folded), every
// term of the finite pass is summed over the images r = R_j - R_i + n A, and
// dE/dA_cd += 1/2 (-1/3) n_c <Ws, dB/dr_d> (each unordered pair is visited from both ends).
__global__ void __launch_bounds__(128) k_scs_grad_periodic(AtomBufs b, CellGeom c, double beta, double a,
                                                           const double *X, const double *V, long long xstride,
                                                           double *g_a0, double *g_om, double *g_rv, double *gR,
                                                           double *gA_part) {
    extern __shared__ double gal_s[];   // [nf1][128]
    const int i = blockIdx.x, t = threadIdx.x;
    for (int k = 0; k < b.nf1; ++k) gal_s[k * 128 + t] = 0.0;
    double acc[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // g_rv, gR x3, gA x9
    for (int j = t; j < b.N; j += 128) {
        const double x[3] = {b.R[3 * j] - b.R[3 * i], b.R[3 * j + 1] - b.R[3 * i + 1], b.R[3 * j + 2] - b.R[3 * i + 2]};
        int lo[3], hi[3];
        image_box(c, x, lo, hi);
        const double S = b.rv[i] + b.rv[j];
        for (int k = 0; k < b.nf1; ++k) {
            const double *Vk = V + k * xstride, *Xk = X + k * xstride;
            double Ws[9];
            for (int xx = 0; xx < 3; ++xx)
                for (int y = 0; y < 3; ++y) {
                    double w = 0.0;
                    for (int cc = 0; cc < 3; ++cc)
                        w += Vk[9LL * i + 3 * xx + cc] * Xk[9LL * j + 3 * y + cc] +
                             Xk[9LL * i + 3 * xx + cc] * Vk[9LL * j + 3 * y + cc];
                    Ws[3 * xx + y] = w;
                }
            const double tr = Ws[0] + Ws[4] + Ws[8];
            const double si = b.sig_u[k * b.N + i], sj = b.sig_u[k * b.N + j], s = sqrt(si * si + sj * sj);
            const double dsda = si * si / (3.0 * s * b.al_u[k * b.N + i]);
            double gal = 0.0;
            for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
                for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
                    for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
                        const int nn[3] = {n0, n1, n2};
                        double r[3];
                        for (int e = 0; e < 3; ++e) r[e] = x[e] + n0 * c.A[e] + n1 * c.A[3 + e] + n2 * c.A[6 + e];
                        const double rho2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                        if (rho2 >= c.rc * c.rc || rho2 < 1e-16) continue;
                        const double rho = sqrt(rho2), ir = 1.0 / rho;
                        const Fermi f = fermi(rho, S, beta, a);
                        const double sr = 1.0 - f.f;
                        if (sr == 0.0 && f.df_drho == 0.0 && f.df_dS == 0.0) continue;   // exact zeros
                        double Wr[3], Wtr[3];
                        for (int xx = 0; xx < 3; ++xx) {
                            Wr[xx] = Ws[3 * xx] * r[0] + Ws[3 * xx + 1] * r[1] + Ws[3 * xx + 2] * r[2];
                            Wtr[xx] = Ws[xx] * r[0] + Ws[3 + xx] * r[1] + Ws[6 + xx] * r[2];
                        }
                        const double rWr = r[0] * Wr[0] + r[1] * Wr[1] + r[2] * Wr[2];
                        const Radial qd = tgg_radial(rho, s);
                        const double WT = qd.P * tr + qd.W * rWr;
                        const double WTs = qd.dPs * tr + qd.dWs * rWr;
                        gal += -1.0 / 3.0 * sr * WTs * dsda;
                        acc[0] += -1.0 / 3.0 * (-f.df_dS) * WT;
                        for (int cc = 0; cc < 3; ++cc) {
                            const double WdT = (qd.dP * tr + qd.dW * rWr) * r[cc] * ir + qd.W * (Wr[cc] + Wtr[cc]);
                            const double dB = sr * WdT - f.df_drho * r[cc] * ir * WT;   // <Ws, dB/dr_cc>
                            if (j != i) acc[1 + cc] += 1.0 / 3.0 * dB;
                            for (int kk = 0; kk < 3; ++kk) acc[4 + 3 * kk + cc] += -1.0 / 6.0 * nn[kk] * dB;
                        }
                    }
            gal_s[k * 128 + t] += gal;
        }
    }
    __syncthreads();
    __shared__ double scratch[4 * 13];
    block_sum128<13>(acc, scratch);
    if (t < b.nf1) {
        const int k = t;
        double sacc = 0.0;
        for (int e = 0; e < 128; ++e) sacc += gal_s[k * 128 + e];
        const double *Vk = V + k * xstride, *Xk = X + k * xstride;
        double wd = 0.0;
        for (int e = 0; e < 9; ++e) wd += Vk[9LL * i + e] * Xk[9LL * i + e];
        const double al = b.al_u[k * b.N + i];
        sacc += -1.0 / 3.0 * wd * (-1.0 / (al * al));
        gal_s[k * 128] = sacc;
    }
    __syncthreads();
    if (t == 0) {
        double ga0 = 0.0, gom = 0.0;
        const double a0 = b.a0[i], om = b.om[i];
        for (int k = 0; k < b.nf1; ++k) {
            const double u = b.u[k], qq = 1.0 + u * u / (om * om);
            const double gl = gal_s[k * 128];
            ga0 += gl / qq;
            gom += gl * a0 * 2.0 * u * u / (om * om * om) / (qq * qq);
        }
        g_a0[i] += ga0;
        g_om[i] += gom;
        g_rv[i] += acc[0];
        gR[3 * i] += acc[1];
        gR[3 * i + 1] += acc[2];
        gR[3 * i + 2] += acc[3];
        for (int e = 0; e < 9; ++e) gA_part[9LL * i + e] = acc[4 + e];
    }
}

// gA[e] += sum_i part[i][e] (fixed order).
__global__ void k_reduce_lattice(const double *part, int N, double *gA) {
    const int e = threadIdx.x;
    if (e >= 9) return;
    double s = 0.0;
    for (int i = 0; i < N; ++i) s += part[9LL * i + e];
    gA[e] += s;
}

inline int cdiv(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

}  // namespace

void structure_factors(const AtomBufs &b, const PeriodicBufs &p, cudaStream_t s) {
    count_launches(1);
    k_structure_factors<<<std::min(cdiv(static_cast<long long>(p.nG) * b.N, 256), 4096), 256, 0, s>>>(
        b.R, b.N, p.G, p.nG, p.S);
}

void build_scs_periodic(const AtomBufs &b, const CellGeom &c, double beta, double a, double *M, long long ld,
                        long long mstride, int *status, cudaStream_t s) {
    count_launches(1);
    k_build_scs_periodic<<<dim3(cdiv(b.N, 32), cdiv(b.N, 8)), dim3(32, 8), 0, s>>>(b, c, beta, a, M, ld, mstride,
                                                                                    status);
    pad_identity(M, ld, 3 * b.N, b.nf1, mstride, s);
}

void build_q_periodic(const AtomBufs &b, const PeriodicBufs &p, double beta, double a, double *Q, long long ld,
                      int n, int *status, cudaStream_t s) {
    const int ntile = cdiv(b.N, kQT);
    count_launches(1);
    k_build_q_periodic<<<dim3(ntile * (ntile + 1) / 2, p.nk), 256, 0, s>>>(b, p, beta, a, Q, ld, ntile, status);
    if (ld > n) {
        count_launches(1);
        k_pad_q_periodic<<<dim3(cdiv((ld - n) * ld, 256), p.nk), 256, 0, s>>>(Q, ld, n, b.ombar);
    }
}

namespace {
// Real symmetric embedding of the Hermitian Q(q_k) = A + iB (planar, slot k): M = [[A, -B],
// [B, A]] of order 2n in an lde x lde matrix, padded with the diagonal entry A_00 (inside the
// spectrum) and zero couplings.  Its eigenvalues are those of Q(q_k), each twice.
__global__ void k_embed_hermitian(const double *Q, long long ld, int n, int k, double *M, long long lde) {
    const double *Re = Q + static_cast<long long>(k) * 2 * ld * ld, *Im = Re + ld * ld;
    const long long total = lde * lde;
    const double pad = Re[0];
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long r = e / lde, c = e % lde;
        double v;
        if (r < 2LL * n && c < 2LL * n) {
            const long long rr = r < n ? r : r - n, cc = c < n ? c : c - n;
            const double a = Re[rr * ld + cc], b = Im[rr * ld + cc];
            v = (r < n) == (c < n) ? a : (r < n ? -b : b);
        } else {
            v = r == c ? pad : 0.0;
        }
        M[e] = v;
    }
}
// Planar slot k of Z (Re, Im) from the embedded matrix function Ze ~ M^{-1/2} =
// [[Re, -Im], [Im, Re]]: the first block column; zero outside the n x n block.
__global__ void k_extract_hermitian(const double *Ze, long long lde, int n, double *Z, long long ld, int k) {
    double *Re = Z + static_cast<long long>(k) * 2 * ld * ld, *Im = Re + ld * ld;
    const long long total = ld * ld;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long r = e / ld, c = e % ld;
        const bool in = r < n && c < n;
        Re[e] = in ? Ze[r * lde + c] : 0.0;
        Im[e] = in ? Ze[(r + n) * lde + c] : 0.0;
    }
}
// E = 1/(2 nk) sum_k e_k - 3/4 sum omega_bar, where e_k = 1/2 Tr M_k^{1/2} - 3/2 sum omega_bar is
// the mixed modes' corrected energy of the embedded matrix of Bloch vector k (Tr M_k^{1/2} =
// 2 Tr Q(q_k)^{1/2}); compensated sums.
__global__ void k_periodic_mixed_energy(const double *ek, int nk, const double *ombar, int N, double *out) {
    double s = 0.0, cc = 0.0;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        double t, er;
        two_sum(s, 0.5 * ek[k] / nk, t, er);
        s = t; cc += er;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double t, er;
        two_sum(s, -0.75 * ombar[i], t, er);
        s = t; cc += er;
    }
    __shared__ double ss[256], sc2[256];
    ss[threadIdx.x] = s;
    sc2[threadIdx.x] = cc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, C = 0.0;
        for (int q = 0; q < blockDim.x; ++q) {
            double t, er;
            two_sum(S, ss[q], t, er);
            S = t;
            C += er + sc2[q];
        }
        out[0] = S + C;
    }
}
}  // namespace

void embed_hermitian(const double *Q, long long ld, int n, int k, double *M, long long lde, cudaStream_t s) {
    count_launches(1);
    k_embed_hermitian<<<1216, 256, 0, s>>>(Q, ld, n, k, M, lde);
}

void extract_hermitian(const double *Ze, long long lde, int n, double *Z, long long ld, int k, cudaStream_t s) {
    count_launches(1);
    k_extract_hermitian<<<1216, 256, 0, s>>>(Ze, lde, n, Z, ld, k);
}

void periodic_mixed_energy(const double *ek, int nk, const double *ombar, int N, double *out, cudaStream_t s) {
    count_launches(1);
    k_periodic_mixed_energy<<<1, 256, 0, s>>>(ek, nk, ombar, N, out);
}

void cscale(double *Y, long long ld, int nk, double scale, cudaStream_t s) {
    count_launches(1);
    k_scale_all<<<1216, 256, 0, s>>>(Y, static_cast<long long>(nk) * 2 * ld * ld, scale);
}

void cset_identity(double *Z, long long ld, int nk, cudaStream_t s) {
    count_launches(1);
    k_caxpby_identity<<<1216, 256, 0, s>>>(Z, nullptr, ld, static_cast<long long>(nk) * 2 * ld * ld, 1.0, 0.0);
}

void caxpby_identity(double *Z, const double *P, long long ld, int nk, double a, double b, cudaStream_t s) {
    count_launches(1);
    k_caxpby_identity<<<1216, 256, 0, s>>>(Z, P, ld, static_cast<long long>(nk) * 2 * ld * ld, a, b);
}

void cfrob_dev_identity(const double *P, long long ld, int n, int nk, double *out, cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(double), s);
    count_launches(1);
    k_cfrob_dev_identity<<<1216, 256, 0, s>>>(P, ld, n, nk, out);
}

void cmax_abs_rowsum(const double *Q, long long ld, int nk, double *out, cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(double), s);
    count_launches(1);
    k_cmax_abs_rowsum<<<cdiv(ld * nk, 8), 256, 0, s>>>(Q, ld, nk, reinterpret_cast<unsigned long long *>(out));
}

void cgemm_f64(const double *A, const double *B, const double *D, double *C, long long ld, int nk, double alpha,
               double beta, bool herm, cudaStream_t s) {
    const long long m2 = ld * ld, st = 2 * m2;
    const int M = static_cast<int>(ld);
    const double *Ar = A, *Ai = A + m2, *Br = B, *Bi = B + m2;
    const double *Dr = D, *Di = D ? D + m2 : nullptr;
    double *Cr = C, *Ci = C + m2;
    // Re C = alpha (Ar Br - Ai Bi) + beta Re D;  Im C = alpha (Ar Bi + Ai Br) + beta Im D.
    // A Hermitian result has a symmetric real part and an antisymmetric imaginary part: each
    // of the two products that build a part then computes only the upper tiles of the partial
    // sum (the second reads the first's upper tiles through D = C) and mirrors them, with a
    // sign change for the imaginary part.
    const int mr = herm ? 2 : 0, mi = herm ? 3 : 0;
    gemm_f64(GemmArgs{Ar, Br, Dr, Cr, ld, ld, ld, ld, st, st, st, st, M, M, M, nk, alpha, beta, mr, 0}, s);
    gemm_f64(GemmArgs{Ai, Bi, Cr, Cr, ld, ld, ld, ld, st, st, st, st, M, M, M, nk, -alpha, 1.0, mr, 0}, s);
    gemm_f64(GemmArgs{Ar, Bi, Di, Ci, ld, ld, ld, ld, st, st, st, st, M, M, M, nk, alpha, beta, mi, 0}, s);
    gemm_f64(GemmArgs{Ai, Br, Ci, Ci, ld, ld, ld, ld, st, st, st, st, M, M, M, nk, alpha, 1.0, mi, 0}, s);
}

void clanczos_coefficients(const double *Q, long long ld, int nk, int steps, double *work, double *coef,
                           cudaStream_t s) {
    double *v = work, *vprev = work + nk * 2 * ld, *w = work + 2 * nk * 2 * ld;
    count_launches(1);
    k_clanczos_init<<<nk, 1024, 0, s>>>(v, vprev, ld);
    for (int j = 0; j < steps; ++j) {
        count_launches(2);
        k_cgemv<<<dim3(cdiv(ld, 8), nk), 256, 0, s>>>(Q, ld, v, w);
        k_clanczos_update<<<nk, 1024, 0, s>>>(w, v, vprev, ld, coef, steps, j);
    }
}

void energy_trace_periodic(const double *Y, long long ld, int n, int nk, const double *ombar, int N,
                           double sqrt_s, double *out, cudaStream_t s) {
    count_launches(1);
    k_energy_periodic<<<1, 256, 0, s>>>(Y, ld, n, nk, ombar, N, 0.5 * sqrt_s / nk, out);
}

void mean_rows(const double *x, int rows, int N, double *out, cudaStream_t s) {
    count_launches(1);
    k_mean_rows<<<cdiv(N, 128), 128, 0, s>>>(x, rows, N, out);
}

void periodic_mbd_grad(const AtomBufs &b, const PeriodicBufs &p, double beta, double a, const double *Z,
                       long long ld, double zscale, const MbdGradOut &o, double *work, double *gA, cudaStream_t s,
                       const double *tq, bool f32_recip) {
    double *g_c = work;
    cudaMemsetAsync(g_c, 0, sizeof(double) * b.N, s);
    cudaMemsetAsync(o.g_rbar, 0, sizeof(double) * b.N, s);
    cudaMemsetAsync(o.gR, 0, sizeof(double) * 3 * b.N, s);
    cudaMemsetAsync(gA, 0, sizeof(double) * 9, s);
    const int ntile = cdiv(b.N, kQT);
    count_launches(2);
    const dim3 grid(ntile * (ntile + 1) / 2, p.nk);
    if (f32_recip)
        k_mbd_grad_periodic<float><<<grid, 256, 0, s>>>(b, p, beta, a, Z, ld, zscale, ntile, g_c, o.g_rbar, o.gR, gA);
    else
        k_mbd_grad_periodic<double><<<grid, 256, 0, s>>>(b, p, beta, a, Z, ld, zscale, ntile, g_c, o.g_rbar, o.gR, gA);
    k_mbd_grad_periodic_finalize<<<cdiv(b.N, 128), 128, 0, s>>>(b, Z, ld, p.nk, zscale, g_c, o, tq);
}

void scs_grad_periodic(const AtomBufs &b, const CellGeom &c, double beta, double a, const double *X,
                       const double *V, long long xstride, double *g_a0, double *g_om, double *g_rv, double *gR,
                       double *gA_part, double *gA, cudaStream_t s) {
    count_launches(2);
    k_scs_grad_periodic<<<b.N, 128, sizeof(double) * b.nf1 * 128, s>>>(b, c, beta, a, X, V, xstride, g_a0, g_om,
                                                                       g_rv, gR, gA_part);
    k_reduce_lattice<<<1, 32, 0, s>>>(gA_part, b.N, gA);
}

}  // namespace mbdgb
