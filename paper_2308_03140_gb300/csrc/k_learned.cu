// Learned screening model (sm_103a): per-atom features, MLP inference and training.
//
// The paper has no learned part; the model stands in for the screening of Eqs. (scs) and
// (contraction) (Sec. 2.3):
//   features (122 per atom): for every other atom j of the same system at distance d < 24 bohr,
//     alpha0_j fc(d) exp(-(d - mu_m)^2 / (2 w^2)), m = 0..63, mu_m = (m + 1/2) w, w = 0.375
//     bohr (4 shells of 6 bohr x 16 Gaussians), fc(d) = (1 + cos(pi d / 24)) / 2; then the
//     atom's own TS-scaled alpha0, omega, R_vdW (Eq. ts-scaling) and volume ratio; then the
//     static screening moments: M_i = sum_j alpha0_j B_ij, B_ij = (1 - f_ij) T^GG_ij at u = 0
//     (Eqs. scs-sr-dipole, tgg, mayer, fermi-damping), m1 = Tr M_i / 3,
//     m2 = Tr(sum_j alpha0_j B_ij M_j) / 3, m3 = Tr(M_i M_i) / 3, and alpha0_i m1,
//     alpha0_i^2 m2, alpha0_i^2 m3; then (48 more) the terms of the Dyson series of Eq. scs at
//     the 16 grid points u_k (u_0 = 0 and the 15 Casimir-Polder nodes): with alpha_j(u) of
//     Eq. dyn-pol, B_ij(u) = (1 - f_ij) T^GG_ij at the widths of alpha(u), H^(0)_i = I and
//     H^(q)_i = sum_{j != i} alpha_j(u) B_ij(u) H^(q-1)_j, feature 74 + 3 k + q - 1 is
//     m_q,i(u_k) = Tr H^(q)_i / 3 (q = 1, 2, 3; all atoms of the system, no cutoff; FP32
//     pair arithmetic, FP64 warp sums);
//   MLP 122 -> 128 -> 128 -> 16 on standardised features, SiLU activations, FP16 weights and
//     biases, FP32 accumulation; output y_k = log(alpha_bar(u_k) / alpha(u_k)).
// Parameter layout of one ensemble member (FP16): W1 [122][128], b1 [128], W2 [128][128],
// b2 [128], W3 [128][16], b3 [16] (W[in][out], row-major), kParams halves in all.
#include <cuda_fp16.h>

#include "freq_grid.h"
#include "internal.h"
#include "pair_math.cuh"
#include "tc_ops.cuh"

namespace mbdgb {
namespace {

using namespace tcops;
using pairs::Fermi;
using pairs::Radial;

constexpr int kFS = 74, kNU = 16, kNQ = 3;   // static features; grid points and hops of the Dyson block
constexpr int kF = kFS + kNU * kNQ, kH = 128, kO = 16;
constexpr int oW1 = 0, ob1 = oW1 + kF * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH * kO, kParams = ob3 + kO;
constexpr int kTA = 32;          // atoms per CTA of the MLP kernels
constexpr double kPiL = 3.141592653589793238462643383279502884;
constexpr double kWidth = 0.375, kCut = 24.0;

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ int system_of(const int *offsets, int n_sys, int atom) {
    int lo = 0, hi = n_sys - 1;   // largest s with offsets[s] <= atom
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= atom) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// SCS coupling B = (1 - f) T^GG of the pair (i, j) at u = 0 (TS-scaled alpha0 and R_vdW,
// beta 0.83, a 6), as the 6 components xx, yy, zz, xy, xz, yz.
__device__ __forceinline__ void scs_coupling(const double *r, double rho, double a0i, double a0j, double rvi,
                                             double rvj, double *B) {
    const double cm = sqrt(2.0 / kPiL) / 3.0;
    const double si = cbrt(cm * a0i), sj = cbrt(cm * a0j);
    const Fermi f = pairs::fermi(rho, rvi + rvj, 0.83, 6.0);
    const Radial t = pairs::tgg_radial(rho, sqrt(si * si + sj * sj));
    const double sr = 1.0 - f.f;
    B[0] = sr * (t.P + t.W * r[0] * r[0]);
    B[1] = sr * (t.P + t.W * r[1] * r[1]);
    B[2] = sr * (t.P + t.W * r[2] * r[2]);
    B[3] = sr * t.W * r[0] * r[1];
    B[4] = sr * t.W * r[0] * r[2];
    B[5] = sr * t.W * r[1] * r[2];
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum128(double v, double *sh) {   // 128 threads, result in all
    v = warp_sum_d(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    return sh[0] + sh[1] + sh[2] + sh[3];
}

// One CTA of 128 threads per atom.  Thread t accumulates Gaussian t % 64 over the partners
// j = j0 + t / 64, + 2, ... (the Gaussian in FP32 from the FP64 distance offset d - mu, the sum in
// FP64); the threads also share the partners of the moment M_i (FP64, written to Mw [n][6]).
__global__ void __launch_bounds__(128) k_features(int n_atoms, int n_sys, const int *offsets, const double *R,
                                                  const double *a0ref, const double *c6ref, const double *rref,
                                                  const double *ratio, float *X, double *Mw) {
    __shared__ double part[2][64];
    __shared__ double red[4];
    const int atom = blockIdx.x, t = threadIdx.x;
    const int s = system_of(offsets, n_sys, atom);
    const int j0 = offsets[s], j1 = offsets[s + 1];
    const double xi = R[3 * atom], yi = R[3 * atom + 1], zi = R[3 * atom + 2];
    const int gidx = t & 63;
    const double mu = (gidx + 0.5) * kWidth;
    const float i2w2 = static_cast<float>(0.5 / (kWidth * kWidth));
    double acc = 0.0;
    for (int j = j0 + (t >> 6); j < j1; j += 2) {
        if (j == atom) continue;
        const double dx = R[3 * j] - xi, dy = R[3 * j + 1] - yi, dz = R[3 * j + 2] - zi;
        const double d = sqrt(dx * dx + dy * dy + dz * dz);
        if (d >= kCut) continue;
        const float w = static_cast<float>(a0ref[j] * ratio[j]) * 0.5f * (1.0f + cospif(static_cast<float>(d / kCut)));
        const float u = static_cast<float>(d - mu);
        acc += static_cast<double>(w * expf(-u * u * i2w2));
    }
    part[t >> 6][gidx] = acc;
    const double a0i = a0ref[atom] * ratio[atom], rvi = rref[atom] * cbrt(ratio[atom]);
    double M[6] = {0, 0, 0, 0, 0, 0};
    for (int j = j0 + t; j < j1; j += 128) {
        if (j == atom) continue;
        const double r[3] = {R[3 * j] - xi, R[3 * j + 1] - yi, R[3 * j + 2] - zi};
        const double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (d >= kCut) continue;
        const double a0j = a0ref[j] * ratio[j];
        double B[6];
        scs_coupling(r, d, a0i, a0j, rvi, rref[j] * cbrt(ratio[j]), B);
        for (int e = 0; e < 6; ++e) M[e] += a0j * B[e];
    }
    for (int e = 0; e < 6; ++e) M[e] = block_sum128(M[e], red);
    float *x = X + static_cast<long long>(atom) * kF;
    if (t < 64) x[t] = static_cast<float>(part[0][t] + part[1][t]);
    if (t == 0) {
        const double a0r = a0ref[atom], v = ratio[atom];
        x[64] = static_cast<float>(a0i);
        x[65] = static_cast<float>(4.0 * c6ref[atom] / (3.0 * a0r * a0r));
        x[66] = static_cast<float>(rvi);
        x[67] = static_cast<float>(v);
        for (int e = 0; e < 6; ++e) Mw[6LL * atom + e] = M[e];
    }
}

// Second pass: m1, m2 (two hops, needs every partner's M_j), m3 and their alpha0 multiples.
__global__ void k_feature_moments(int n_atoms, int n_sys, const int *offsets, const double *R, const double *a0ref,
                                  const double *rref, const double *ratio, const double *Mw, float *X) {
    const int atom = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (atom >= n_atoms) return;
    const int s = system_of(offsets, n_sys, atom);
    const int j0 = offsets[s], j1 = offsets[s + 1];
    const double xi = R[3 * atom], yi = R[3 * atom + 1], zi = R[3 * atom + 2];
    const double a0i = a0ref[atom] * ratio[atom], rvi = rref[atom] * cbrt(ratio[atom]);
    double t2 = 0.0;
    for (int j = j0 + lane; j < j1; j += 32) {
        if (j == atom) continue;
        const double r[3] = {R[3 * j] - xi, R[3 * j + 1] - yi, R[3 * j + 2] - zi};
        const double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (d >= kCut) continue;
        const double a0j = a0ref[j] * ratio[j];
        double B[6];
        scs_coupling(r, d, a0i, a0j, rvi, rref[j] * cbrt(ratio[j]), B);
        const double *Mj = Mw + 6LL * j;
        // Tr(B M_j) for symmetric B, M_j
        t2 += a0j * (B[0] * Mj[0] + B[1] * Mj[1] + B[2] * Mj[2] + 2.0 * (B[3] * Mj[3] + B[4] * Mj[4] + B[5] * Mj[5]));
    }
    t2 = warp_sum_d(t2);
    if (lane == 0) {
        const double *M = Mw + 6LL * atom;
        const double m1 = (M[0] + M[1] + M[2]) / 3.0, m2 = t2 / 3.0;
        const double m3 = (M[0] * M[0] + M[1] * M[1] + M[2] * M[2] +
                           2.0 * (M[3] * M[3] + M[4] * M[4] + M[5] * M[5])) / 3.0;
        float *x = X + static_cast<long long>(atom) * kF;
        x[68] = static_cast<float>(m1);
        x[69] = static_cast<float>(m2);
        x[70] = static_cast<float>(m3);
        x[71] = static_cast<float>(a0i * m1);
        x[72] = static_cast<float>(a0i * a0i * m2);
        x[73] = static_cast<float>(a0i * a0i * m3);
    }
}

// ---- Dyson block of the features (per grid point; FP32 pair arithmetic) -----------------
// Work of the forward pass (FP32, after the n x 6 FP64 static moments): P [n] (TS-scaled
// alpha0, omega, R_vdW), AS [16][n] (alpha(u_k), sigma(u_k)^2), H1 [16][n][6] (symmetric
// H^(1)), H2 [16][n][9] (H^(2), row-major).  The backward adds GQ [16][n] (dL/dm_q, q = 1..3),
// G2 [16][n][6] and G1 [16][n][9] (adjoints of H^(2), H^(1)) and FP [16][n][3] (FP64 partial
// forces per grid point).
struct GridU2 { float u2[kNU]; };
struct DysonFwd {
    float4 *P;
    float2 *AS;
    float *H1, *H2;
};
__host__ __device__ inline DysonFwd dyson_fwd(double *work, int n) {
    float *f = reinterpret_cast<float *>(work + 6LL * n);
    DysonFwd w;
    w.P = reinterpret_cast<float4 *>(f);
    w.AS = reinterpret_cast<float2 *>(f + 4LL * n);
    w.H1 = f + 36LL * n;
    w.H2 = f + 132LL * n;
    return w;
}
struct DysonAdj {
    float4 *GQ;
    float *G2, *G1;
    double *FP;
};
__host__ __device__ inline DysonAdj dyson_adj(double *adj, int n) {
    float *f = reinterpret_cast<float *>(adj + 6LL * n);
    DysonAdj w;
    w.GQ = reinterpret_cast<float4 *>(f);
    w.G2 = f + 64LL * n;
    w.G1 = f + 160LL * n;
    w.FP = adj + 6LL * n + 152LL * n;
    return w;
}
static_assert(6 + 276 / 2 == kLearnedWork, "forward work per atom");
static_assert(6 + 304 / 2 + 48 + 37 == kLearnedAdjointWork, "adjoint work per atom");

// 1 - f of the Fermi damping (beta 0.83, a 6) as e / (1 + e), e = exp(-a (d / (beta S) - 1)), and
// its derivative in d: the small values far beyond the damping radius keep their digits.
struct DampF { float sr, dsr; };
__device__ __forceinline__ DampF damp_f(float d, float S) {
    const float bS = 0.83f * S, e = expf(-6.0f * (d / bS - 1.0f));
    const float f = 1.0f / (1.0f + e), sr = e * f;
    return {sr, -6.0f * f * sr / bS};
}

// B = (1 - f) T^GG at separation r (|r| = d), width sqrt(sig2), as xx, yy, zz, xy, xz, yz.
__device__ __forceinline__ void dyson_coupling(const float *r, float d, float S, float sig2, float *B) {
    const DampF g = damp_f(d, S);
    const pairs::RadialF t = pairs::tgg_radial_f(d, sqrtf(sig2));
    const float P = g.sr * t.P, W = g.sr * t.W;
    B[0] = P + W * r[0] * r[0];
    B[1] = P + W * r[1] * r[1];
    B[2] = P + W * r[2] * r[2];
    B[3] = W * r[0] * r[1];
    B[4] = W * r[0] * r[2];
    B[5] = W * r[1] * r[2];
}

// sym 3x3 (6) times sym 3x3 (6) -> general row-major (9)
__device__ __forceinline__ void symsym(const float *A, const float *B, float *C) {
    const float a[9] = {A[0], A[3], A[4], A[3], A[1], A[5], A[4], A[5], A[2]};
    const float b[9] = {B[0], B[3], B[4], B[3], B[1], B[5], B[4], B[5], B[2]};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) C[3 * r + c] = a[3 * r] * b[c] + a[3 * r + 1] * b[3 + c] + a[3 * r + 2] * b[6 + c];
}

// The warp of grid point k and atom i: e = k n + i over the 16 n warps (consecutive warps take
// consecutive atoms of one grid point, so a CTA's warps read the same partner data).
struct WarpItem { int k, i, j0, j1; bool ok; };
__device__ __forceinline__ WarpItem warp_item(int n, int n_sys, const int *offsets) {
    const long long e = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    WarpItem w{0, 0, 0, 0, false};
    if (e >= static_cast<long long>(kNU) * n) return w;
    w.k = static_cast<int>(e / n);
    w.i = static_cast<int>(e % n);
    const int s = system_of(offsets, n_sys, w.i);
    w.j0 = offsets[s];
    w.j1 = offsets[s + 1];
    w.ok = true;
    return w;
}
__device__ __forceinline__ void sep(const double *R, int i, int j, float *r, float &d) {
    r[0] = static_cast<float>(R[3 * j] - R[3 * i]);
    r[1] = static_cast<float>(R[3 * j + 1] - R[3 * i + 1]);
    r[2] = static_cast<float>(R[3 * j + 2] - R[3 * i + 2]);
    d = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
}
template <int M>
__device__ __forceinline__ void warp_sum_store(const float *acc, float *out) {   // FP64 sums over the lanes
#pragma unroll
    for (int e = 0; e < M; ++e) {
        const double v = warp_sum_d(static_cast<double>(acc[e]));
        if ((threadIdx.x & 31) == 0) out[e] = static_cast<float>(v);
    }
}

// P and AS: thread per (k, i).
__global__ void k_dyson_prep(int n, const double *a0ref, const double *c6ref, const double *rref, const double *ratio,
                             GridU2 g, double *work) {
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (e >= static_cast<long long>(kNU) * n) return;
    const int k = static_cast<int>(e / n), i = static_cast<int>(e % n);
    const DysonFwd w = dyson_fwd(work, n);
    const double a0 = a0ref[i] * ratio[i], om = 4.0 * c6ref[i] / (3.0 * a0ref[i] * a0ref[i]);
    if (k == 0) w.P[i] = make_float4(static_cast<float>(a0), static_cast<float>(om),
                                     static_cast<float>(rref[i] * cbrt(ratio[i])), 0.0f);
    const double al = a0 / (1.0 + static_cast<double>(g.u2[k]) / (om * om));
    const double sg = cbrt(sqrt(2.0 / kPiL) / 3.0 * al);
    w.AS[e] = make_float2(static_cast<float>(al), static_cast<float>(sg * sg));
}

// Trace of B = (1 - f) T^GG at width sqrt(sig2): T^GG's trace is its Gaussian part alone,
// 2 z^2 th / d^3 (z = d / s, th = 2 z e^{-z^2} / sqrt(pi)), which the sum of its diagonal in FP32
// would leave to the cancellation of 3 P against W d^2.
__device__ __forceinline__ float dyson_trace(float d, float S, float sig2) {
    const float z = d * rsqrtf(sig2);
    if (z > pairs::kGaussFarF) return 0.0f;
    const float th = 1.1283791670955126f * z * expf(-z * z);
    return damp_f(d, S).sr * 2.0f * z * z * th / (d * d * d);
}

// HOP 1: H1_i = sum_j alpha_j B_ij (its trace from dyson_trace); HOP 2: H2_i = sum_j alpha_j
// B_ij H1_j; HOP 3: the trace of sum_j alpha_j B_ij H2_j.  X[i][74 + 3k + HOP - 1] = Tr / 3.
template <int HOP>
__global__ void k_dyson_hop(int n, int n_sys, const int *offsets, const double *R, double *work, float *X) {
    const WarpItem it = warp_item(n, n_sys, offsets);
    if (!it.ok) return;
    const int lane = threadIdx.x & 31, i = it.i, k = it.k;
    const DysonFwd w = dyson_fwd(work, n);
    const float rvi = w.P[i].z, sgi = w.AS[static_cast<long long>(k) * n + i].y;
    constexpr int M = HOP == 1 ? 7 : (HOP == 2 ? 9 : 1);   // HOP 1: H1 and its trace
    float acc[M];
#pragma unroll
    for (int e = 0; e < M; ++e) acc[e] = 0.0f;
    for (int j = it.j0 + lane; j < it.j1; j += 32) {
        if (j == i) continue;
        float r[3], d, B[6];
        sep(R, i, j, r, d);
        const float2 as = w.AS[static_cast<long long>(k) * n + j];
        dyson_coupling(r, d, rvi + w.P[j].z, sgi + as.y, B);
        if (HOP == 1) {
#pragma unroll
            for (int e = 0; e < 6; ++e) acc[e] += as.x * B[e];
            acc[6] += as.x * dyson_trace(d, rvi + w.P[j].z, sgi + as.y);
        } else if (HOP == 2) {
            const float *h = w.H1 + (static_cast<long long>(k) * n + j) * 6;
            const float hj[6] = {h[0], h[1], h[2], h[3], h[4], h[5]};
            float BH[9];
            symsym(B, hj, BH);
#pragma unroll
            for (int e = 0; e < 9; ++e) acc[e] += as.x * BH[e];
        } else {
            const float *h = w.H2 + (static_cast<long long>(k) * n + j) * 9;   // Tr(B H) = sum B o H (B symmetric)
            acc[0] += as.x * (B[0] * h[0] + B[1] * h[4] + B[2] * h[8] + B[3] * (h[1] + h[3]) + B[4] * (h[2] + h[6]) +
                              B[5] * (h[5] + h[7]));
        }
    }
    float out[M];
    warp_sum_store<M>(acc, out);
    if (lane == 0) {
        float tr;
        if (HOP == 1) {
            float *h = w.H1 + (static_cast<long long>(k) * n + i) * 6;
            for (int e = 0; e < 6; ++e) h[e] = out[e];
            tr = out[6];
        } else if (HOP == 2) {
            float *h = w.H2 + (static_cast<long long>(k) * n + i) * 9;
            for (int e = 0; e < 9; ++e) h[e] = out[e];
            tr = out[0] + out[4] + out[8];
        } else {
            tr = out[0];
        }
        X[static_cast<long long>(i) * kF + kFS + 3 * k + HOP - 1] = tr / 3.0f;
    }
}

// Backward of L = sum_{i,k,q} g_q,i(k) m_q,i(k), g = the members' summed feature gradient:
// GQ [k][i] = (g1, g2, g3).
__global__ void k_dyson_adj_prep(int n, int members, const float *dX, double *adj) {
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (e >= static_cast<long long>(kNU) * n) return;
    const int k = static_cast<int>(e / n), i = static_cast<int>(e % n);
    float g[3] = {0.0f, 0.0f, 0.0f};
    for (int m = 0; m < members; ++m)
        for (int q = 0; q < 3; ++q) g[q] += dX[(static_cast<long long>(m) * n + i) * kF + kFS + 3 * k + q];
    dyson_adj(adj, n).GQ[e] = make_float4(g[0], g[1], g[2], 0.0f);
}

// Adjoints of the hops (B_li = B_il): STEP 2: G2_i = g2_i I/3 + alpha_i sum_l B_il g3_l / 3
// (symmetric); STEP 1: G1_i = g1_i I/3 + alpha_i sum_l B_il G2_l.
template <int STEP>
__global__ void k_dyson_adj(int n, int n_sys, const int *offsets, const double *R, double *work, double *adj) {
    const WarpItem it = warp_item(n, n_sys, offsets);
    if (!it.ok) return;
    const int lane = threadIdx.x & 31, i = it.i, k = it.k;
    const DysonFwd w = dyson_fwd(work, n);
    const DysonAdj a = dyson_adj(adj, n);
    const float rvi = w.P[i].z;
    const float2 asi = w.AS[static_cast<long long>(k) * n + i];
    constexpr int M = STEP == 2 ? 6 : 9;
    float acc[M];
#pragma unroll
    for (int e = 0; e < M; ++e) acc[e] = 0.0f;
    for (int l = it.j0 + lane; l < it.j1; l += 32) {
        if (l == i) continue;
        float r[3], d, B[6];
        sep(R, i, l, r, d);
        dyson_coupling(r, d, rvi + w.P[l].z, asi.y + w.AS[static_cast<long long>(k) * n + l].y, B);
        if (STEP == 2) {
            const float g3 = a.GQ[static_cast<long long>(k) * n + l].z / 3.0f;
#pragma unroll
            for (int e = 0; e < 6; ++e) acc[e] += g3 * B[e];
        } else {
            const float *g = a.G2 + (static_cast<long long>(k) * n + l) * 6;
            const float gl[6] = {g[0], g[1], g[2], g[3], g[4], g[5]};
            float BG[9];
            symsym(B, gl, BG);
#pragma unroll
            for (int e = 0; e < 9; ++e) acc[e] += BG[e];
        }
    }
    float out[M];
    warp_sum_store<M>(acc, out);
    if (lane == 0) {
        const float4 gq = a.GQ[static_cast<long long>(k) * n + i];
        const float diag = (STEP == 2 ? gq.y : gq.x) / 3.0f;
        if (STEP == 2) {
            float *g = a.G2 + (static_cast<long long>(k) * n + i) * 6;
            for (int e = 0; e < 6; ++e) g[e] = asi.x * out[e] + (e < 3 ? diag : 0.0f);
        } else {
            float *g = a.G1 + (static_cast<long long>(k) * n + i) * 9;
            for (int e = 0; e < 9; ++e) g[e] = asi.x * out[e] + (e % 4 == 0 ? diag : 0.0f);
        }
    }
}

// Abar_ij = dL/dA_ij (A_ij = alpha_j B_ij) = G1_i + G2_i H1_j + (g3_i / 3) H2_j^T (row-major).
__device__ __forceinline__ void abar(const float *G1, const float *G2, float g3, const float *H1, const float *H2,
                                     float *out) {
    float GH[9];
    symsym(G2, H1, GH);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) out[3 * r + c] = G1[3 * r + c] + GH[3 * r + c] + g3 * H2[3 * c + r];
}

// FP[k][i] = dL/dR_i through grid point k: -sum_j <C_ij, dB/dr (r = R_j - R_i)> with C_ij the
// symmetric part of alpha_j Abar_ij + alpha_i Abar_ji.
__global__ void k_dyson_forces(int n, int n_sys, const int *offsets, const double *R, double *work, double *adj) {
    const WarpItem it = warp_item(n, n_sys, offsets);
    if (!it.ok) return;
    const int lane = threadIdx.x & 31, i = it.i, k = it.k;
    const DysonFwd w = dyson_fwd(work, n);
    const DysonAdj a = dyson_adj(adj, n);
    const long long ki = static_cast<long long>(k) * n + i;
    const float rvi = w.P[i].z;
    const float2 asi = w.AS[ki];
    float G1i[9], G2i[6], H1i[6], H2i[9];
    for (int e = 0; e < 9; ++e) G1i[e] = a.G1[ki * 9 + e], H2i[e] = w.H2[ki * 9 + e];
    for (int e = 0; e < 6; ++e) G2i[e] = a.G2[ki * 6 + e], H1i[e] = w.H1[ki * 6 + e];
    const float g3i = a.GQ[ki].z / 3.0f;
    float f[3] = {0.0f, 0.0f, 0.0f};
    for (int j = it.j0 + lane; j < it.j1; j += 32) {
        if (j == i) continue;
        const long long kj = static_cast<long long>(k) * n + j;
        float r[3], d;
        sep(R, i, j, r, d);
        const float2 asj = w.AS[kj];
        float Aij[9], Aji[9];
        abar(G1i, G2i, g3i, w.H1 + kj * 6, w.H2 + kj * 9, Aij);
        abar(a.G1 + kj * 9, a.G2 + kj * 6, a.GQ[kj].z / 3.0f, H1i, H2i, Aji);
        float M[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) M[e] = asj.x * Aij[e] + asi.x * Aji[e];
        const float C[6] = {M[0], M[4], M[8], 0.5f * (M[1] + M[3]), 0.5f * (M[2] + M[6]), 0.5f * (M[5] + M[7])};
        // <C, B> = sr (P tr C + W r.C.r); its gradient in r
        const DampF g = damp_f(d, rvi + w.P[j].z);
        const pairs::RadialF t = pairs::tgg_radial_f(d, sqrtf(asi.y + asj.y));
        const float Cr[3] = {C[0] * r[0] + C[3] * r[1] + C[4] * r[2], C[3] * r[0] + C[1] * r[1] + C[5] * r[2],
                             C[4] * r[0] + C[5] * r[1] + C[2] * r[2]};
        const float tr = C[0] + C[1] + C[2], rCr = r[0] * Cr[0] + r[1] * Cr[1] + r[2] * Cr[2];
        const float ir = 1.0f / d, CT = t.P * tr + t.W * rCr;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            f[c] -= g.dsr * r[c] * ir * CT + g.sr * ((t.dP * tr + t.dW * rCr) * r[c] * ir + 2.0f * t.W * Cr[c]);
    }
    for (int c = 0; c < 3; ++c) {
        const double v = warp_sum_d(static_cast<double>(f[c]));
        if (lane == 0) a.FP[ki * 3 + c] = v;
    }
}

// Shared layout of the MLP kernels: weights (FP16), standardised inputs, two hidden layers.
struct MlpSmem {
    __half *W;
    float *Xs, *h1, *h2;
};
__device__ __forceinline__ MlpSmem mlp_smem(char *base) {
    MlpSmem m;
    m.W = reinterpret_cast<__half *>(base);
    m.Xs = reinterpret_cast<float *>(base + ((kParams * 2 + 15) / 16) * 16);
    m.h1 = m.Xs + kTA * kF;
    m.h2 = m.h1 + kTA * kH;
    return m;
}
constexpr size_t kMlpSmem = ((kParams * 2 + 15) / 16) * 16 + sizeof(float) * (kTA * kF + 2 * kTA * kH);

__device__ __forceinline__ void load_params_and_inputs(const MlpSmem &m, const __half *P, const float *X,
                                                       const float *mean, const float *stdv, int a0, int B) {
    const int t = threadIdx.x;
    for (int e = t; e < kParams; e += blockDim.x) m.W[e] = P[e];
    for (int e = t; e < kTA * kF; e += blockDim.x) {
        const int a = e / kF, k = e % kF, atom = a0 + a;
        m.Xs[e] = atom < B ? (X[static_cast<long long>(atom) * kF + k] - mean[k]) / stdv[k] : 0.0f;
    }
    __syncthreads();
}

// ---- MLP forward on the tensor cores (tcgen05, kind::tf32) ---------------------------------
// One CTA of 128 threads per 128 atoms and ensemble member; thread t owns atom a0 + t, which is
// TMEM lane t of the accumulator.  Each layer Z = H W + b (M = 128 atoms, K = 128 inputs, the
// 122 features padded with zeros, N = 128 or 16) is one chain of tcgen05.mma: the FP32
// activations as TF32 hi + lo parts (hi = rna(h), lo = rna(h - hi)) against the weights,
// whose FP16 values are exact in TF32, H_hi W + H_lo W accumulated in TMEM.  The operands are
// written to shared memory by the threads in the K-major 128-byte-swizzled layout: element
// (row r, k) in slab k / 32 (r x 128 bytes each), 16-byte chunk ((k % 32) / 4) xor (r % 8).
constexpr int kMT = 128;                 // atoms per CTA
constexpr int kSlab = kMT * 128;         // bytes of one 32-element K slab of a 128-row operand
constexpr size_t kMlpTcSmem = 3 * 4 * static_cast<size_t>(kSlab) + 1024 + 64;
static_assert(kF <= 128 && kH == 128 && kO == 16, "layer shapes of the tensor-core MLP");
static_assert(6LL * kSlab == kLearnedPackedFloats, "packed weight images: six of 128 x 128 FP32");

__device__ __forceinline__ uint32_t swz(int r, int k) {
    const int kk = k & 31;
    return static_cast<uint32_t>((k >> 5) * kSlab + r * 128 + ((((kk >> 2) ^ (r & 7)) << 4) | ((kk & 3) << 2)));
}
__host__ __device__ constexpr uint32_t mlp_idesc(int n) {   // FP32 accumulator, TF32 A and B, K-major, M = 128
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(kMT >> 4) << 24);
}
__device__ __forceinline__ void mlp_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void put_split(uint8_t *hi, uint8_t *lo, int r, int k, float v) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(v));
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(l) : "f"(v - __uint_as_float(h)));
    *reinterpret_cast<uint32_t *>(hi + swz(r, k)) = h;
    *reinterpret_cast<uint32_t *>(lo + swz(r, k)) = l;
}
// B operand of a layer: row n = output unit, K = input (W is stored [in][out]); rows n < nout.
__device__ __forceinline__ void put_weights(uint8_t *Bs, const __half *W, int nin, int nout) {
    for (int e = threadIdx.x; e < nout * 128; e += blockDim.x) {
        const int k = e / nout, n = e % nout;   // consecutive threads: consecutive outputs of one input
        const float w = k < nin ? __half2float(W[k * nout + n]) : 0.0f;
        *reinterpret_cast<float *>(Bs + swz(n, k)) = w;
    }
}
// The six B operands of the tensor-core MLP of each member in their shared-memory layout
// (FP32, 64 KB each, zero where the layer has no row or input): 0-2 the forward's W1^T, W2^T,
// W3^T (rows = outputs), 3-5 the backward's W3, W2, W1 (rows = inputs).  Built once per model;
// the kernels then fetch each with one bulk copy.
constexpr int kImgFloats = 4 * kSlab / 4;
__global__ void k_mlp_pack(int members, const __half *params, float *packed) {
    const long long total = static_cast<long long>(members) * 6 * 128 * 128;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(e / (6 * 128 * 128)), img = static_cast<int>((e / (128 * 128)) % 6);
        const int n = static_cast<int>((e >> 7) & 127), k = static_cast<int>(e & 127);
        const __half *P = params + static_cast<long long>(m) * kParams;
        float w = 0.0f;
        switch (img) {
            case 0: w = k < kF ? __half2float(P[oW1 + k * kH + n]) : 0.0f; break;             // W1^T
            case 1: w = __half2float(P[oW2 + k * kH + n]); break;                             // W2^T
            case 2: w = n < kO ? __half2float(P[oW3 + k * kO + n]) : 0.0f; break;             // W3^T
            case 3: w = k < kO ? __half2float(P[oW3 + n * kO + k]) : 0.0f; break;             // W3
            case 4: w = __half2float(P[oW2 + n * kH + k]); break;                             // W2
            default: w = n < kF ? __half2float(P[oW1 + n * kH + k]) : 0.0f; break;            // W1
        }
        packed[(static_cast<long long>(m) * 6 + img) * kImgFloats + swz(n, k) / 4] = w;
    }
}

// Weights of the next product into Bs: one bulk copy of the packed image (thread 0 issues it,
// every thread waits for it before the MMA) or, without packed images, the threads' own
// converting writes.
struct WeightLoad {
    uint64_t *bar;
    uint32_t phase;
    bool pending;
};
__device__ __forceinline__ void weights_issue(uint8_t *Bs, const float *img, WeightLoad &wl) {
    if (threadIdx.x == 0) {
        mbar_expect_tx(wl.bar, 4 * kSlab);
        bulk_load(Bs, img, 4 * kSlab, wl.bar);
    }
    wl.pending = true;
}
__device__ __forceinline__ bool weights_wait(WeightLoad &wl, int *err) {
    const bool ok = mbar_wait(wl.bar, wl.phase, err);
    wl.phase ^= 1;
    wl.pending = false;
    return ok;
}
// Before the CTA exits: a copy still in flight (a wait that gave up earlier) must land first.
__device__ __forceinline__ void weights_drain(WeightLoad &wl, int *err) {
    if (wl.pending && threadIdx.x == 0) mbar_wait(wl.bar, wl.phase, err, kSpinCycles / 8);
}

// The layer's MMA chain (one thread) and its completion on bar; all threads wait (bounded).
__device__ __forceinline__ bool mlp_layer(uint32_t tmem, uint8_t *Ahi, uint8_t *Alo, uint8_t *Bs, int n,
                                          uint64_t *bar, uint32_t phase, int *err) {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0) {
        const uint32_t id = mlp_idesc(n);
        for (int sl = 0; sl < 4; ++sl)
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t b = sdesc(su32(Bs + sl * kSlab + kk * 32));   // rows n < N of each slab
                mlp_mma(tmem, sdesc(su32(Ahi + sl * kSlab + kk * 32)), b, id, (sl | kk) != 0 ? 1u : 0u);
                mlp_mma(tmem, sdesc(su32(Alo + sl * kSlab + kk * 32)), b, id, 1u);
            }
        mma_commit(bar);
    }
    const bool ok = mbar_wait(bar, phase, err);
    fence_after();
    return __syncthreads_and(ok) != 0;   // uniform over the CTA: every later barrier is reached by all
}

// grid (ceil(B / 128), members), 128 threads.  Y [member][B][16]; optional cache
// z [member][2][B][128] (pre-activations of both hidden layers).  A wait that times out raises
// ST_TC_TIMEOUT in *err and leaves NaN outputs.
__global__ void __launch_bounds__(128, 1) k_mlp_forward_tc(int B, const float *X, const float *mean,
                                                           const float *stdv, const __half *params, float *Y,
                                                           float *zcache, const float *packed, int *err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *Ahi = smem, *Alo = smem + 4 * kSlab, *Bs = smem + 8 * kSlab;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 12 * kSlab);
    WeightLoad wl{bar + 1, 0, false};
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 2);
    const int member = blockIdx.y, t = threadIdx.x, warp = t >> 5, a = blockIdx.x * kMT + t;
    const __half *P = params + static_cast<long long>(member) * kParams;
    const float *img = packed ? packed + static_cast<long long>(member) * 6 * kImgFloats : nullptr;
    if (t == 0) {
        mbar_init(bar, 1);
        mbar_init(wl.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (img) weights_issue(Bs, img, wl);   // W1^T under the writes of the features
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                     "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    // layer 1 operands: the standardised features of the CTA's atoms (read row by row, the
    // threads along the features), W1
    const int a0 = blockIdx.x * kMT;
    for (int e = t; e < kMT * 128; e += kMT) {
        const int row = e >> 7, k = e & 127, ar = a0 + row;
        const float x = (ar < B && k < kF) ? (X[static_cast<long long>(ar) * kF + k] - mean[k]) / stdv[k] : 0.0f;
        put_split(Ahi, Alo, row, k, x);
    }
    bool ok = true;
    if (img) ok = weights_wait(wl, err);
    else put_weights(Bs, P + oW1, kF, kH);
    fence_before();
    ok = __syncthreads_and(ok) != 0;
    fence_after();
    const uint32_t tmem = *tmem_slot + (static_cast<uint32_t>(warp * 32) << 16);
    float *z1 = zcache ? zcache + static_cast<long long>(member) * 2 * B * kH : nullptr;
    float *z2 = zcache ? z1 + static_cast<long long>(B) * kH : nullptr;
    uint32_t phase = 0;
    if (ok) ok = mlp_layer(*tmem_slot, Ahi, Alo, Bs, kH, bar, phase, err);
    if (ok && img) weights_issue(Bs, img + kImgFloats, wl);   // W2^T under the epilogue
    // hidden layers: z = acc + b -> cache; h = silu(z) -> the next layer's A operand
    for (int layer = 0; layer < 2 && ok; ++layer) {
        const __half *bias = P + (layer == 0 ? ob1 : ob2);
        float *zc = layer == 0 ? z1 : z2;
        for (int c0 = 0; c0 < kH; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + c0, r);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float z = __uint_as_float(r[j]) + __half2float(bias[c0 + j]);
                if (zc && a < B) zc[static_cast<long long>(a) * kH + c0 + j] = z;
                put_split(Ahi, Alo, t, c0 + j, a < B ? silu(z) : 0.0f);
            }
        }
        fence_before();
        __syncthreads();   // every thread's reads of TMEM and of the weights are done
        if (img) ok = weights_wait(wl, err);
        else if (layer == 0) put_weights(Bs, P + oW2, kH, kH);
        else put_weights(Bs, P + oW3, kH, kO);
        ok = __syncthreads_and(ok) != 0;
        phase ^= 1;
        if (ok) ok = mlp_layer(*tmem_slot, Ahi, Alo, Bs, layer == 0 ? kH : kO, bar, phase, err);
        if (ok && img && layer == 0) weights_issue(Bs, img + 2 * kImgFloats, wl);   // W3^T under the epilogue
    }
    // output layer: y = acc + b3 (16 columns).  The TMEM load is warp-collective: every lane
    // takes part (ok is uniform over the CTA), only the rows of real atoms are stored.
    uint32_t r[32];
    if (ok) tmem_ld32(tmem, r);   // columns 16..31 are not part of the product
    if (a < B) {
        float *y = Y + (static_cast<long long>(member) * B + a) * kO;
        for (int o = 0; o < kO; ++o) y[o] = ok ? __uint_as_float(r[o]) + __half2float(P[ob3 + o]) : __int_as_float(0x7fc00000);
    }
    if (!ok && t == 0) mbar_wait(bar, phase, err, kSpinCycles / 8);   // let a late chain finish before freeing TMEM
    weights_drain(wl, err);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(*tmem_slot), "r"(128));
    }
}

// B operand of a backward product: W used as stored ([in][out], row n = input unit), rows
// n < nin, K = the outputs k < nout (zero beyond).
__device__ __forceinline__ void put_weights_rows(uint8_t *Bs, const __half *W, int nin, int nout) {
    for (int e = threadIdx.x; e < 128 * 128; e += blockDim.x) {
        const int n = e >> 7, k = e & 127;   // consecutive threads: consecutive outputs of one row
        const float w = (n < nin && k < nout) ? __half2float(W[n * nout + k]) : 0.0f;
        *reinterpret_cast<float *>(Bs + swz(n, k)) = w;
    }
}

// Gradient of sum(dY * Y) with respect to the raw features on the tensor cores (the data
// path of the backward, without parameter gradients): dh2 = dY W3^T, dz2 = dh2 silu'(z2),
// dh1 = dz2 W2^T, dz1 = dh1 silu'(z1), dX = (dz1 W1^T) / std, each product as in the forward
// (TF32 hi/lo parts of the FP32 left factor against the exact weights, FP32 accumulation in
// TMEM).  grid (ceil(B / 128), members), 128 threads; zcache from the forward; a wait that
// times out raises ST_TC_TIMEOUT in *err and leaves NaN in dX.
__global__ void __launch_bounds__(128, 1) k_mlp_backward_dx_tc(int B, const float *stdv, const __half *params,
                                                               const float *zcache, const float *dY, float *dX,
                                                               const float *packed, int *err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *Ahi = smem, *Alo = smem + 4 * kSlab, *Bs = smem + 8 * kSlab;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 12 * kSlab);
    WeightLoad wl{bar + 1, 0, false};
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 2);
    const int member = blockIdx.y, t = threadIdx.x, warp = t >> 5, a0 = blockIdx.x * kMT, a = a0 + t;
    const __half *P = params + static_cast<long long>(member) * kParams;
    const float *img = packed ? packed + (static_cast<long long>(member) * 6 + 3) * kImgFloats : nullptr;
    const float *z1 = zcache + static_cast<long long>(member) * 2 * B * kH, *z2 = z1 + static_cast<long long>(B) * kH;
    if (t == 0) {
        mbar_init(bar, 1);
        mbar_init(wl.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (img) weights_issue(Bs, img, wl);   // W3 by rows under the writes of dY
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                     "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    // dY rows of the CTA's atoms (K = the 16 outputs), W3 by rows
    for (int e = t; e < kMT * 128; e += kMT) {
        const int row = e >> 7, k = e & 127, ar = a0 + row;
        const float v = (ar < B && k < kO) ? dY[(static_cast<long long>(member) * B + ar) * kO + k] : 0.0f;
        put_split(Ahi, Alo, row, k, v);
    }
    bool ok = true;
    if (img) ok = weights_wait(wl, err);
    else put_weights_rows(Bs, P + oW3, kH, kO);
    fence_before();
    ok = __syncthreads_and(ok) != 0;
    fence_after();
    const uint32_t tmem = *tmem_slot + (static_cast<uint32_t>(warp * 32) << 16);
    uint32_t phase = 0;
    if (ok) ok = mlp_layer(*tmem_slot, Ahi, Alo, Bs, kH, bar, phase, err);
    if (ok && img) weights_issue(Bs, img + kImgFloats, wl);   // W2 under the epilogue
    for (int layer = 0; layer < 2 && ok; ++layer) {   // dz2 from dh2, then dz1 from dh1
        const float *zc = layer == 0 ? z2 : z1;
        for (int c0 = 0; c0 < kH; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + c0, r);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float dz = a < B ? __uint_as_float(r[j]) * dsilu(zc[static_cast<long long>(a) * kH + c0 + j]) : 0.0f;
                put_split(Ahi, Alo, t, c0 + j, dz);
            }
        }
        fence_before();
        __syncthreads();   // every thread's reads of TMEM and of the weights are done
        if (img) ok = weights_wait(wl, err);
        else if (layer == 0) put_weights_rows(Bs, P + oW2, kH, kH);
        else put_weights_rows(Bs, P + oW1, kF, kH);
        ok = __syncthreads_and(ok) != 0;
        phase ^= 1;
        if (ok) ok = mlp_layer(*tmem_slot, Ahi, Alo, Bs, kH, bar, phase, err);
        if (ok && img && layer == 0) weights_issue(Bs, img + 2 * kImgFloats, wl);   // W1 under the epilogue
    }
    // dX = acc / std over the 122 features (TMEM loads on every lane, stores for real atoms)
    for (int c0 = 0; c0 < kH; c0 += 32) {
        uint32_t r[32];
        if (ok) tmem_ld32(tmem + c0, r);
        if (a < B)
            for (int j = 0; j < 32; ++j) {
                const int n = c0 + j;
                if (n < kF)
                    dX[(static_cast<long long>(member) * B + a) * kF + n] =
                        ok ? __uint_as_float(r[j]) / stdv[n] : __int_as_float(0x7fc00000);
            }
    }
    if (!ok && t == 0) mbar_wait(bar, phase, err, kSpinCycles / 8);   // let a late chain finish before freeing TMEM
    weights_drain(wl, err);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(*tmem_slot), "r"(128));
    }
}

// Backward of sum(dY * Y): grid (ceil(B / 32), members), 128 threads.  Needs the cache of the
// forward pass.  dX (optional) [member][B][74]: gradient with respect to the raw features.
// grad (optional) [member][kParams] FP32, accumulated (atomic adds of per-CTA sums).
__global__ void __launch_bounds__(128) k_mlp_backward(int B, const float *X, const float *mean, const float *stdv,
                                                      const __half *params, const float *zcache, const float *dY,
                                                      float *dX, float *grad) {
    extern __shared__ __align__(16) char smem[];
    const MlpSmem m = mlp_smem(smem);
    const int member = blockIdx.y, a0 = blockIdx.x * kTA, t = threadIdx.x;
    load_params_and_inputs(m, params + static_cast<long long>(member) * kParams, X, mean, stdv, a0, B);
    const float *z1 = zcache + static_cast<long long>(member) * 2 * B * kH, *z2 = z1 + static_cast<long long>(B) * kH;
    __shared__ float dy_s[kTA * kO];
    for (int e = t; e < kTA * kO; e += 128) {
        const int a = e / kO, o = e % kO;
        dy_s[e] = a0 + a < B ? dY[(static_cast<long long>(member) * B + a0 + a) * kO + o] : 0.0f;
    }
    // h1, h2 from the cached pre-activations (padding atoms: zero)
    for (int e = t; e < kTA * kH; e += 128) {
        const int a = e / kH, k = e % kH;
        const bool ok = a0 + a < B;
        m.h1[e] = ok ? silu(z1[static_cast<long long>(a0 + a) * kH + k]) : 0.0f;
        m.h2[e] = ok ? silu(z2[static_cast<long long>(a0 + a) * kH + k]) : 0.0f;
    }
    __syncthreads();
    float *g = grad ? grad + static_cast<long long>(member) * kParams : nullptr;
    if (g) {   // output layer: gW3[k][o] = sum_a h2[a][k] dy[a][o], gb3[o] = sum_a dy[a][o]
        for (int e = t; e < kH * kO; e += 128) {
            const int k = e / kO, o = e % kO;
            float s = 0.0f;
            for (int a = 0; a < kTA; ++a) s += m.h2[a * kH + k] * dy_s[a * kO + o];
            atomicAdd(&g[oW3 + e], s);
        }
        if (t < kO) {
            float s = 0.0f;
            for (int a = 0; a < kTA; ++a) s += dy_s[a * kO + t];
            atomicAdd(&g[ob3 + t], s);
        }
    }
    // dz2[a][t] = (sum_o dy[a][o] W3[t][o]) dsilu(z2[a][t]); kept in registers
    float dz[kTA];
    for (int a = 0; a < kTA; ++a) {
        float s = 0.0f;
#pragma unroll
        for (int o = 0; o < kO; ++o) s += dy_s[a * kO + o] * __half2float(m.W[oW3 + t * kO + o]);
        dz[a] = a0 + a < B ? s * dsilu(z2[static_cast<long long>(a0 + a) * kH + t]) : 0.0f;
    }
    if (g) {   // gW2[k][t] = sum_a h1[a][k] dz2[a][t]; gb2[t]
        float sb = 0.0f;
        for (int a = 0; a < kTA; ++a) sb += dz[a];
        atomicAdd(&g[ob2 + t], sb);
        for (int k = 0; k < kH; ++k) {
            float s = 0.0f;
#pragma unroll
            for (int a = 0; a < kTA; ++a) s += m.h1[a * kH + k] * dz[a];
            atomicAdd(&g[oW2 + k * kH + t], s);
        }
    }
    __syncthreads();   // h2 is no longer needed: reuse it for dz2
    for (int a = 0; a < kTA; ++a) m.h2[a * kH + t] = dz[a];
    __syncthreads();
    // dz1[a][t] = (sum_k dz2[a][k] W2[t][k]) dsilu(z1[a][t])
    for (int a = 0; a < kTA; ++a) {
        float s = 0.0f;
        for (int k = 0; k < kH; ++k) s += m.h2[a * kH + k] * __half2float(m.W[oW2 + t * kH + k]);
        dz[a] = a0 + a < B ? s * dsilu(z1[static_cast<long long>(a0 + a) * kH + t]) : 0.0f;
    }
    if (g) {   // gW1[k][t] = sum_a Xs[a][k] dz1[a][t]; gb1[t]
        float sb = 0.0f;
        for (int a = 0; a < kTA; ++a) sb += dz[a];
        atomicAdd(&g[ob1 + t], sb);
        for (int k = 0; k < kF; ++k) {
            float s = 0.0f;
#pragma unroll
            for (int a = 0; a < kTA; ++a) s += m.Xs[a * kF + k] * dz[a];
            atomicAdd(&g[oW1 + k * kH + t], s);
        }
    }
    if (dX) {
        __syncthreads();
        for (int a = 0; a < kTA; ++a) m.h1[a * kH + t] = dz[a];
        __syncthreads();
        for (int e = t; e < kTA * kF; e += 128) {
            const int a = e / kF, k = e % kF;
            if (a0 + a >= B) continue;
            float s = 0.0f;
            for (int j = 0; j < kH; ++j) s += m.h1[a * kH + j] * __half2float(m.W[oW1 + k * kH + j]);
            dX[(static_cast<long long>(member) * B + a0 + a) * kF + k] = s / stdv[k];
        }
    }
}

__global__ void k_mse_grad(long long n, const float *y, const float *t, float *dy, double *loss) {
    double acc = 0.0;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float d = y[e] - t[e];
        dy[e] = 2.0f * d / static_cast<float>(n);
        acc += static_cast<double>(d) * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, acc / static_cast<double>(n));
}

// Adam (Kingma and Ba): m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
// p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps); p16 = fp16(p) (round to nearest).
__global__ void k_adam(long long n, float *p, const float *g, float *mm, float *vv, float c1, float c2, float lr,
                       float b1, float b2, float eps, __half *p16) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float ge = g[e];
        const float me = b1 * mm[e] + (1.0f - b1) * ge, ve = b2 * vv[e] + (1.0f - b2) * ge * ge;
        mm[e] = me;
        vv[e] = ve;
        const float pe = p[e] - lr * (me / c1) / (sqrtf(ve / c2) + eps);
        p[e] = pe;
        if (p16) p16[e] = __float2half_rn(pe);
    }
}

// Y[i][k] = log(alpha_bar[k][i] / alpha_free[k][i]), the model's target (FP32).
__global__ void k_learned_targets(int n, const double *abar, const double *afree, float *Y) {
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (e >= static_cast<long long>(n) * kO) return;
    const int i = static_cast<int>(e / kO), k = static_cast<int>(e % kO);
    Y[e] = static_cast<float>(log(abar[static_cast<long long>(k) * n + i] / afree[static_cast<long long>(k) * n + i]));
}

__global__ void k_gather_rows(long long rows, int width, const int *idx, const float *src, float *dst) {
    const long long total = rows * width;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long r = e / width, c = e % width;
        dst[e] = src[static_cast<long long>(idx[r]) * width + c];
    }
}

__global__ void k_learned_alpha(int N, int members, int nf1, const double *al_u, const float *Y, double *abar,
                                double *spread) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * nf1) return;
    const int k = e / N, i = e % N;
    double ym = 0.0, s1 = 0.0, s2 = 0.0;
    const double al = al_u[k * N + i];
    for (int m = 0; m < members; ++m) {   // two passes: mean, then squared deviations
        const double y = Y[(static_cast<long long>(m) * N + i) * kO + k];
        ym += y;
        s1 += al * exp(y);
    }
    ym /= members;
    const double mean = s1 / members;
    for (int m = 0; m < members; ++m) {
        const double d = al * exp(static_cast<double>(Y[(static_cast<long long>(m) * N + i) * kO + k])) - mean;
        s2 += d * d;
    }
    abar[e] = al * exp(ym);
    spread[e] = sqrt(s2 / members);
}

// The energy-error estimate per atom: scale x the members' standard deviation of their
// first-order energies, D_m = sum_{k,i} h[k][i] alpha_i(u_k) (e^{y_m,i,k} - mean_m' e^{y_m',i,k}),
// over N.  One CTA of 1024 threads; the deviations are summed member by member (no cancellation
// against the mean energy).
__global__ void k_learned_estimate(int N, int nf1, int members, double scale, const double *h, const double *al_u,
                                   const float *Y, double *out) {
    __shared__ double sh[32];
    __shared__ double Dm[64];
    const int n = N * nf1;
    for (int m = 0; m < members; ++m) {
        double acc = 0.0;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int k = e / N, i = e % N;
            const float *y = Y + static_cast<long long>(i) * kO + k;
            float mean = 0.0f;
            for (int q = 0; q < members; ++q) mean += expf(y[static_cast<long long>(q) * N * kO]);
            mean /= static_cast<float>(members);
            acc += h[e] * al_u[e] * static_cast<double>(expf(y[static_cast<long long>(m) * N * kO]) - mean);
        }
        acc = warp_sum_d(acc);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (blockDim.x >> 5); ++w) t += sh[w];
            Dm[m] = t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int m = 0; m < members; ++m) v += Dm[m] * Dm[m];
        out[0] = scale * sqrt(v / members) / N;
    }
}


// ---- forces of the learned path --------------------------------------------------------
// dY[m][i][k] = h[k][i] alpha_bar[k][i] / M: the upstream gradient of each member's output
// (alpha_bar = alpha exp(mean_m y_m)).
__global__ void k_learned_dy(int N, int members, int nf1, const double *h, const double *abar, float *dY) {
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (e >= static_cast<long long>(members) * N * kO) return;
    const int k = static_cast<int>(e % kO), i = static_cast<int>((e / kO) % N);
    dY[e] = k < nf1 ? static_cast<float>(h[k * N + i] * abar[k * N + i] / members) : 0.0f;
}

// The members' summed gradient of the 74 static features: gs [N][74] (FP32).
__global__ void k_learned_gsum(int N, int members, const float *dX, float *gs) {
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (e >= static_cast<long long>(N) * kFS) return;
    const int i = static_cast<int>(e / kFS), k = static_cast<int>(e % kFS);
    float g = 0.0f;
    for (int m = 0; m < members; ++m) g += dX[(static_cast<long long>(m) * N + i) * kF + k];
    gs[e] = g;
}

// Upstream gradients of the static moments of atom i.
struct MomentGrad { double g1, g2, g3; };
__device__ __forceinline__ MomentGrad moment_grad(const float *gs, int i, double a0i) {
    const float *g = gs + static_cast<long long>(i) * kFS + 68;
    return {g[0] + a0i * g[3], g[1] + a0i * a0i * g[4], g[2] + a0i * a0i * g[5]};
}

// A_i = dE/dM_i = g1_i I/3 + 2 g3_i M_i/3 + (alpha0_i/3) sum_k g2_k B_ik (one CTA of 128
// threads per atom).
__global__ void __launch_bounds__(128) k_moment_adjoint(int N, const double *R, const double *a0ref,
                                                        const double *rref, const double *ratio, const double *Mw,
                                                        const float *gs, double *Aw) {
    __shared__ double red[4];
    const int i = blockIdx.x, t = threadIdx.x;
    const double a0i = a0ref[i] * ratio[i], rvi = rref[i] * cbrt(ratio[i]);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int k = t; k < N; k += 128) {
        if (k == i) continue;
        const double r[3] = {R[3 * k] - R[3 * i], R[3 * k + 1] - R[3 * i + 1], R[3 * k + 2] - R[3 * i + 2]};
        const double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (d >= kCut) continue;
        const double a0k = a0ref[k] * ratio[k];
        double B[6];
        scs_coupling(r, d, a0i, a0k, rvi, rref[k] * cbrt(ratio[k]), B);
        const double g2k = moment_grad(gs, k, a0k).g2;
        for (int e = 0; e < 6; ++e) acc[e] += g2k * B[e];
    }
    for (int e = 0; e < 6; ++e) acc[e] = block_sum128(acc[e], red);
    if (t == 0) {
        const MomentGrad gi = moment_grad(gs, i, a0i);
        const double *M = Mw + 6LL * i;
        for (int e = 0; e < 6; ++e)
            Aw[6LL * i + e] = (e < 3 ? gi.g1 / 3.0 : 0.0) + 2.0 * gi.g3 * M[e] / 3.0 + a0i / 3.0 * acc[e];
    }
}

// <C, dB/dr_c> for symmetric C (6 components) and B = (1 - f) T^GG at separation r.
__device__ __forceinline__ void coupling_grad(const double *r, double d, double a0i, double a0j, double rvi,
                                              double rvj, const double *C, double *out) {
    const double cm = sqrt(2.0 / kPiL) / 3.0;
    const double si = cbrt(cm * a0i), sj = cbrt(cm * a0j);
    const Fermi f = pairs::fermi(d, rvi + rvj, 0.83, 6.0);
    const Radial t = pairs::tgg_radial(d, sqrt(si * si + sj * sj));
    const double sr = 1.0 - f.f, ir = 1.0 / d;
    double Cr[3];
    Cr[0] = C[0] * r[0] + C[3] * r[1] + C[4] * r[2];
    Cr[1] = C[3] * r[0] + C[1] * r[1] + C[5] * r[2];
    Cr[2] = C[4] * r[0] + C[5] * r[1] + C[2] * r[2];
    const double tr = C[0] + C[1] + C[2], rCr = r[0] * Cr[0] + r[1] * Cr[1] + r[2] * Cr[2];
    const double CT = t.P * tr + t.W * rCr;
    for (int c = 0; c < 3; ++c)
        out[c] = -f.df_drho * r[c] * ir * CT + sr * ((t.dP * tr + t.dW * rCr) * r[c] * ir + 2.0 * t.W * Cr[c]);
}

// gR[i] += dE/dR_i through the features (one CTA of 128 threads per atom, fixed order):
//   radial:  -sum_j sum_k (gx_ik alpha0_j + gx_jk alpha0_i) phi_k'(d_ij) r^_ij (phi_k in FP32)
//   moments: -sum_j <C_ij + C_ji, dB/dr (r_ij)>,  C_ij = alpha0_j (A_i + g2_i M_j / 3)
//   Dyson block: the partial forces FP [16][N][3] of k_dyson_forces, in grid-point order.
__global__ void __launch_bounds__(128) k_learned_forces(int N, const double *R, const double *a0ref,
                                                        const double *rref, const double *ratio, const double *Mw,
                                                        const double *Aw, const float *gs, const double *FP,
                                                        double *gR) {
    __shared__ float gi_s[64];
    __shared__ double red[4];
    const int i = blockIdx.x, t = threadIdx.x;
    const double a0i = a0ref[i] * ratio[i], rvi = rref[i] * cbrt(ratio[i]);
    if (t < 64) gi_s[t] = gs[static_cast<long long>(i) * kFS + t];
    __syncthreads();
    const double g2i = moment_grad(gs, i, a0i).g2;
    const double *Mi = Mw + 6LL * i, *Ai = Aw + 6LL * i;
    const float i2w2 = static_cast<float>(0.5 / (kWidth * kWidth));
    double f[3] = {0, 0, 0};
    for (int j = t; j < N; j += 128) {
        if (j == i) continue;
        const double r[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
        const double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (d >= kCut) continue;
        const double a0j = a0ref[j] * ratio[j], rvj = rref[j] * cbrt(ratio[j]);
        // radial features
        const float df = static_cast<float>(d), x = df / static_cast<float>(kCut);
        const float fc = 0.5f * (1.0f + cospif(x)), dfc = -0.5f * static_cast<float>(kPiL / kCut) * sinpif(x);
        const float *gj = gs + static_cast<long long>(j) * kFS;
        const float a0jf = static_cast<float>(a0j), a0if = static_cast<float>(a0i);
        float sr = 0.0f;
        for (int k = 0; k < 64; ++k) {
            const float u = static_cast<float>(d - (k + 0.5) * kWidth), G = expf(-u * u * i2w2);
            sr += (gi_s[k] * a0jf + gj[k] * a0if) * G * (dfc - fc * u * 2.0f * i2w2);
        }
        for (int c = 0; c < 3; ++c) f[c] -= static_cast<double>(sr) * r[c] / d;
        // moments
        const double g2j = moment_grad(gs, j, a0j).g2;
        const double *Mj = Mw + 6LL * j, *Aj = Aw + 6LL * j;
        double C[6], dB[3];
        for (int e = 0; e < 6; ++e) C[e] = a0j * (Ai[e] + g2i * Mj[e] / 3.0) + a0i * (Aj[e] + g2j * Mi[e] / 3.0);
        coupling_grad(r, d, a0i, a0j, rvi, rvj, C, dB);
        for (int c = 0; c < 3; ++c) f[c] -= dB[c];
    }
    for (int c = 0; c < 3; ++c) f[c] = block_sum128(f[c], red);
    if (t == 0)
        for (int c = 0; c < 3; ++c) {
            double fd = 0.0;   // the Dyson block's grid points, in order
            for (int k = 0; k < kNU; ++k) fd += FP[(static_cast<long long>(k) * N + i) * 3 + c];
            gR[3 * i + c] += f[c] + fd;
        }
}

inline int cdiv(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

}  // namespace

int learned_param_count() { return kParams; }

void learned_dy(int N, int members, int nf1, const double *h, const double *abar, float *dY, cudaStream_t s) {
    count_launches(1);
    k_learned_dy<<<cdiv(static_cast<long long>(members) * N * kO, 256), 256, 0, s>>>(N, members, nf1, h, abar, dY);
}

void learned_forces(int N, const int *offsets, const double *R, const double *a0ref, const double *rref,
                    const double *ratio, double *work, const float *dX, int members, double *adjoint, double *gR,
                    cudaStream_t s) {
    const int wb = cdiv(static_cast<long long>(kNU) * N, 8), tb = cdiv(static_cast<long long>(kNU) * N, 256);
    float *gs = reinterpret_cast<float *>(adjoint + 206LL * N);   // [N][74] after the Dyson adjoints
    count_launches(7);
    k_dyson_adj_prep<<<tb, 256, 0, s>>>(N, members, dX, adjoint);
    k_learned_gsum<<<cdiv(static_cast<long long>(N) * kFS, 256), 256, 0, s>>>(N, members, dX, gs);
    k_dyson_adj<2><<<wb, 256, 0, s>>>(N, 1, offsets, R, work, adjoint);
    k_dyson_adj<1><<<wb, 256, 0, s>>>(N, 1, offsets, R, work, adjoint);
    k_dyson_forces<<<wb, 256, 0, s>>>(N, 1, offsets, R, work, adjoint);
    k_moment_adjoint<<<N, 128, 0, s>>>(N, R, a0ref, rref, ratio, work, gs, adjoint);
    k_learned_forces<<<N, 128, 0, s>>>(N, R, a0ref, rref, ratio, work, adjoint, gs, dyson_adj(adjoint, N).FP, gR);
}

void learned_alpha(int N, int members, int nf1, const double *al_u, const float *Y, double *abar, double *spread,
                   cudaStream_t s) {
    count_launches(1);
    k_learned_alpha<<<cdiv(static_cast<long long>(N) * nf1, 256), 256, 0, s>>>(N, members, nf1, al_u, Y, abar,
                                                                               spread);
}

void learned_estimate(int N, int nf1, int members, double scale, const double *h, const double *al_u,
                      const float *Y, double *out, cudaStream_t s) {
    count_launches(1);
    k_learned_estimate<<<1, 1024, 0, s>>>(N, nf1, members, scale, h, al_u, Y, out);
}

void scs_features(int n_atoms, int n_sys, const int *offsets, const double *R, const double *a0ref,
                  const double *c6ref, const double *rref, const double *ratio, float *X, double *work,
                  cudaStream_t s) {
    static GridU2 grid = [] {   // u_k^2 of the 16 points: 0 and the 15 Casimir-Polder nodes
        std::vector<double> u, wu;
        casimir_polder_grid(kNU - 1, u, wu);
        GridU2 g;
        for (int k = 0; k < kNU; ++k) g.u2[k] = static_cast<float>(u[k] * u[k]);
        return g;
    }();
    const int wb = cdiv(static_cast<long long>(kNU) * n_atoms, 8), tb = cdiv(static_cast<long long>(kNU) * n_atoms, 256);
    count_launches(6);
    k_features<<<n_atoms, 128, 0, s>>>(n_atoms, n_sys, offsets, R, a0ref, c6ref, rref, ratio, X, work);
    k_feature_moments<<<cdiv(n_atoms, 8), 256, 0, s>>>(n_atoms, n_sys, offsets, R, a0ref, rref, ratio, work, X);
    k_dyson_prep<<<tb, 256, 0, s>>>(n_atoms, a0ref, c6ref, rref, ratio, grid, work);
    k_dyson_hop<1><<<wb, 256, 0, s>>>(n_atoms, n_sys, offsets, R, work, X);
    k_dyson_hop<2><<<wb, 256, 0, s>>>(n_atoms, n_sys, offsets, R, work, X);
    k_dyson_hop<3><<<wb, 256, 0, s>>>(n_atoms, n_sys, offsets, R, work, X);
}

cudaError_t mlp_pack(int members, const void *params16, float *packed, cudaStream_t s) {
    count_launches(1);
    k_mlp_pack<<<std::min(cdiv(static_cast<long long>(members) * 6 * 128 * 128, 256), 2432), 256, 0, s>>>(
        members, static_cast<const __half *>(params16), packed);
    return cudaGetLastError();
}

cudaError_t mlp_forward(int B, int members, const float *X, const float *mean, const float *stdv,
                        const void *params16, float *Y, float *zcache, cudaStream_t s, int *err, const float *packed) {
    static int *own_err = nullptr;   // the timeout flag when the caller passes none
    if (!err) {
        if (!own_err) {
            cudaError_t e = cudaMalloc(&own_err, sizeof(int));
            if (e != cudaSuccess) return e;
            e = cudaMemset(own_err, 0, sizeof(int));
            if (e != cudaSuccess) return e;
        }
        err = own_err;
    }
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kMlpTcSmem));
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_mlp_forward_tc<<<dim3(cdiv(B, kMT), members), 128, kMlpTcSmem, s>>>(
        B, X, mean, stdv, static_cast<const __half *>(params16), Y, zcache, packed, err);
    return cudaGetLastError();
}

cudaError_t mlp_backward(int B, int members, const float *X, const float *mean, const float *stdv,
                         const void *params16, const float *zcache, const float *dY, float *dX, float *grad,
                         cudaStream_t s, const float *packed) {
    if (!grad) {   // the data path alone (the learned forces): on the tensor cores
        static int *own_err = nullptr;
        if (!own_err) {
            cudaError_t e = cudaMalloc(&own_err, sizeof(int));
            if (e != cudaSuccess) return e;
            e = cudaMemset(own_err, 0, sizeof(int));
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaFuncSetAttribute(k_mlp_backward_dx_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(kMlpTcSmem));
        if (e != cudaSuccess) return e;
        count_launches(1);
        k_mlp_backward_dx_tc<<<dim3(cdiv(B, kMT), members), 128, kMlpTcSmem, s>>>(
            B, stdv, static_cast<const __half *>(params16), zcache, dY, dX, packed, own_err);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kMlpSmem));
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_mlp_backward<<<dim3(cdiv(B, kTA), members), 128, kMlpSmem, s>>>(
        B, X, mean, stdv, static_cast<const __half *>(params16), zcache, dY, dX, grad);
    return cudaGetLastError();
}

void mse_grad(long long n, const float *y, const float *t, float *dy, double *loss, cudaStream_t s) {
    if (loss) cudaMemsetAsync(loss, 0, sizeof(double), s);
    count_launches(1);
    k_mse_grad<<<std::min(cdiv(n, 256), 1216), 256, 0, s>>>(n, y, t, dy, loss);
}

void adam_step(long long n, float *p, const float *g, float *m, float *v, int step, float lr, void *p16,
               cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, static_cast<float>(step)), c2 = 1.0f - powf(b2, static_cast<float>(step));
    count_launches(1);
    k_adam<<<std::min(cdiv(n, 256), 1216), 256, 0, s>>>(n, p, g, m, v, c1, c2, lr, b1, b2, 1e-8f,
                                                        static_cast<__half *>(p16));
}

void gather_rows(long long rows, int width, const int *idx, const float *src, float *dst, cudaStream_t s) {
    count_launches(1);
    k_gather_rows<<<std::min(cdiv(rows * width, 256), 4096), 256, 0, s>>>(rows, width, idx, src, dst);
}

}  // namespace mbdgb

// ---- C ABI (declared in include/mbd_gb300_kernels.h) ----------------------------------
#include "../../include/mbd_gb300.h"
#include "../../include/mbd_gb300_kernels.h"

extern "C" {

int mbdk_scs_features(void *stream, int n_atoms, int n_systems, const int *offsets, const double *coords,
                      const double *alpha0_ref, const double *c6_ref, const double *rvdw_ref,
                      const double *volume_ratio, float *X, double *work) {
    if (n_atoms < 1 || n_systems < 1 || !offsets || !coords || !alpha0_ref || !c6_ref || !rvdw_ref ||
        !volume_ratio || !X || !work)
        return MBD_ERR_INPUT;
    mbdgb::scs_features(n_atoms, n_systems, offsets, coords, alpha0_ref, c6_ref, rvdw_ref, volume_ratio, X, work,
                        static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

int mbdk_mlp_forward(void *stream, int n_atoms, int n_members, const float *X, const float *mean,
                     const float *std, const void *params_fp16, float *Y, float *zcache) {
    if (n_atoms < 1 || n_members < 1 || n_members > 65535 || !X || !mean || !std || !params_fp16 || !Y)
        return MBD_ERR_INPUT;
    return mbdgb::mlp_forward(n_atoms, n_members, X, mean, std, params_fp16, Y, zcache,
                              static_cast<cudaStream_t>(stream)) == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

int mbdk_mlp_backward(void *stream, int n_atoms, int n_members, const float *X, const float *mean,
                      const float *std, const void *params_fp16, const float *zcache, const float *dY,
                      float *dX, float *grad) {
    if (n_atoms < 1 || n_members < 1 || n_members > 65535 || !X || !mean || !std || !params_fp16 || !zcache ||
        !dY || (!dX && !grad))
        return MBD_ERR_INPUT;
    return mbdgb::mlp_backward(n_atoms, n_members, X, mean, std, params_fp16, zcache, dY, dX, grad,
                               static_cast<cudaStream_t>(stream)) == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

int mbdk_mse_grad(void *stream, long long n, const float *y, const float *t, float *dy, double *loss) {
    if (n < 1 || !y || !t || !dy) return MBD_ERR_INPUT;
    mbdgb::mse_grad(n, y, t, dy, loss, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

int mbdk_adam_step(void *stream, long long n, float *params, const float *grad, float *m, float *v, int step,
                   float lr, void *params_fp16) {
    if (n < 1 || step < 1 || !params || !grad || !m || !v || !(lr > 0.0f)) return MBD_ERR_INPUT;
    mbdgb::adam_step(n, params, grad, m, v, step, lr, params_fp16, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

int mbdk_learned_targets(void *stream, int n_atoms, const double *alpha_bar, const double *alpha_free, float *Y) {
    if (n_atoms < 1 || !alpha_bar || !alpha_free || !Y) return MBD_ERR_INPUT;
    mbdgb::count_launches(1);
    mbdgb::k_learned_targets<<<static_cast<int>((16LL * n_atoms + 255) / 256), 256, 0,
                               static_cast<cudaStream_t>(stream)>>>(n_atoms, alpha_bar, alpha_free, Y);
    return cudaGetLastError() == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

int mbdk_gather_rows(void *stream, long long rows, int width, const int *idx, const float *src, float *dst) {
    if (rows < 1 || width < 1 || !idx || !src || !dst) return MBD_ERR_INPUT;
    mbdgb::gather_rows(rows, width, idx, src, dst, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

}  // extern "C"
