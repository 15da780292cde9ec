// Learned screening model (sm_103a): per-atom features, MLP inference and training.
//
// The paper has no learned part; the model stands in for the screening of Eqs. (scs) and
// (contraction) (Sec. 2.3):
//   features (74 per atom): for every other atom j of the same system at distance d < 24 bohr,
//     alpha0_j fc(d) exp(-(d - mu_m)^2 / (2 w^2)), m = 0..63, mu_m = (m + 1/2) w, w = 0.375
//     bohr (4 shells of 6 bohr x 16 Gaussians), fc(d) = (1 + cos(pi d / 24)) / 2; then the
//     atom's own TS-scaled alpha0, omega, R_vdW (Eq. ts-scaling) and volume ratio; then the
//     static screening moments: M_i = sum_j alpha0_j B_ij, B_ij = (1 - f_ij) T^GG_ij at u = 0
//     (Eqs. scs-sr-dipole, tgg, mayer, fermi-damping), m1 = Tr M_i / 3,
//     m2 = Tr(sum_j alpha0_j B_ij M_j) / 3, m3 = Tr(M_i M_i) / 3, and alpha0_i m1,
//     alpha0_i^2 m2, alpha0_i^2 m3;
//   MLP 74 -> 128 -> 128 -> 16 on standardised features, SiLU activations, FP16 weights and
//     biases, FP32 accumulation; output y_k = log(alpha_bar(u_k) / alpha(u_k)).
// Parameter layout of one ensemble member (FP16): W1 [74][128], b1 [128], W2 [128][128],
// b2 [128], W3 [128][16], b3 [16] (W[in][out], row-major), kParams halves in all.
#include <cuda_fp16.h>

#include "internal.h"
#include "pair_math.cuh"

namespace mbdgb {
namespace {

using pairs::Fermi;
using pairs::Radial;

constexpr int kF = 74, kH = 128, kO = 16;
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

// One warp per atom; lane l accumulates Gaussians l and l + 32, and the lanes share the
// partner atoms for the moment M_i (written to Mw [n_atoms][6], FP64).
__global__ void k_features(int n_atoms, int n_sys, const int *offsets, const double *R, const double *a0ref,
                           const double *c6ref, const double *rref, const double *ratio, float *X, double *Mw) {
    const int atom = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (atom >= n_atoms) return;
    const int s = system_of(offsets, n_sys, atom);
    const int j0 = offsets[s], j1 = offsets[s + 1];
    const double xi = R[3 * atom], yi = R[3 * atom + 1], zi = R[3 * atom + 2];
    const double mu0 = (lane + 0.5) * kWidth, mu1 = (lane + 32.5) * kWidth, i2w2 = 0.5 / (kWidth * kWidth);
    double acc0 = 0.0, acc1 = 0.0;
    for (int j = j0; j < j1; ++j) {
        if (j == atom) continue;
        const double dx = R[3 * j] - xi, dy = R[3 * j + 1] - yi, dz = R[3 * j + 2] - zi;
        const double d = sqrt(dx * dx + dy * dy + dz * dz);
        if (d >= kCut) continue;
        const double w = a0ref[j] * ratio[j] * 0.5 * (1.0 + cos(kPiL * d / kCut));
        acc0 += w * exp(-(d - mu0) * (d - mu0) * i2w2);
        acc1 += w * exp(-(d - mu1) * (d - mu1) * i2w2);
    }
    float *x = X + static_cast<long long>(atom) * kF;
    x[lane] = static_cast<float>(acc0);
    x[lane + 32] = static_cast<float>(acc1);
    const double a0i = a0ref[atom] * ratio[atom], rvi = rref[atom] * cbrt(ratio[atom]);
    double M[6] = {0, 0, 0, 0, 0, 0};
    for (int j = j0 + lane; j < j1; j += 32) {
        if (j == atom) continue;
        const double r[3] = {R[3 * j] - xi, R[3 * j + 1] - yi, R[3 * j + 2] - zi};
        const double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (d >= kCut) continue;
        const double a0j = a0ref[j] * ratio[j];
        double B[6];
        scs_coupling(r, d, a0i, a0j, rvi, rref[j] * cbrt(ratio[j]), B);
        for (int e = 0; e < 6; ++e) M[e] += a0j * B[e];
    }
    for (int e = 0; e < 6; ++e) M[e] = warp_sum_d(M[e]);
    if (lane == 0) {
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

// z1, h1 and z2, h2 for the CTA's atoms (thread t owns hidden unit t).
__device__ __forceinline__ void hidden_layers(const MlpSmem &m, float *z1_out, float *z2_out, int a0, int B) {
    const int t = threadIdx.x;
    float acc[kTA];
    const float b1 = __half2float(m.W[ob1 + t]);
#pragma unroll
    for (int a = 0; a < kTA; ++a) acc[a] = b1;
    for (int k = 0; k < kF; ++k) {
        const float w = __half2float(m.W[oW1 + k * kH + t]);
#pragma unroll
        for (int a = 0; a < kTA; ++a) acc[a] += m.Xs[a * kF + k] * w;
    }
#pragma unroll
    for (int a = 0; a < kTA; ++a) {
        m.h1[a * kH + t] = silu(acc[a]);
        if (z1_out && a0 + a < B) z1_out[static_cast<long long>(a0 + a) * kH + t] = acc[a];
    }
    __syncthreads();
    const float b2 = __half2float(m.W[ob2 + t]);
#pragma unroll
    for (int a = 0; a < kTA; ++a) acc[a] = b2;
    for (int k = 0; k < kH; ++k) {
        const float w = __half2float(m.W[oW2 + k * kH + t]);
#pragma unroll
        for (int a = 0; a < kTA; ++a) acc[a] += m.h1[a * kH + k] * w;
    }
#pragma unroll
    for (int a = 0; a < kTA; ++a) {
        m.h2[a * kH + t] = silu(acc[a]);
        if (z2_out && a0 + a < B) z2_out[static_cast<long long>(a0 + a) * kH + t] = acc[a];
    }
    __syncthreads();
}

// grid (ceil(B / 32), members), 128 threads.  Y [member][B][16]; optional cache
// z [member][2][B][128] (pre-activations of both hidden layers).
__global__ void __launch_bounds__(128) k_mlp_forward(int B, const float *X, const float *mean, const float *stdv,
                                                     const __half *params, float *Y, float *zcache) {
    extern __shared__ __align__(16) char smem[];
    const MlpSmem m = mlp_smem(smem);
    const int member = blockIdx.y, a0 = blockIdx.x * kTA, t = threadIdx.x;
    load_params_and_inputs(m, params + static_cast<long long>(member) * kParams, X, mean, stdv, a0, B);
    float *z1 = zcache ? zcache + static_cast<long long>(member) * 2 * B * kH : nullptr;
    float *z2 = zcache ? z1 + static_cast<long long>(B) * kH : nullptr;
    hidden_layers(m, z1, z2, a0, B);
    // output layer: thread t computes (atom t / 16 + 8 q, output t % 16), q = 0..3
    const int o = t % kO;
    const float b3 = __half2float(m.W[ob3 + o]);
    for (int q = 0; q < kTA * kO / 128; ++q) {
        const int a = t / kO + 8 * q;
        float acc = b3;
        for (int k = 0; k < kH; ++k) acc += m.h2[a * kH + k] * __half2float(m.W[oW3 + k * kO + o]);
        if (a0 + a < B) Y[(static_cast<long long>(member) * B + a0 + a) * kO + o] = acc;
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

__global__ void k_learned_estimate(int n, int N, const double *h, const double *spread, double *out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int e = threadIdx.x; e < n; e += blockDim.x) acc += fabs(h[e] * spread[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (blockDim.x >> 5); ++w) t += sh[w];
        out[0] = t / N;
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

// Upstream gradients of the moments of atom i from the summed feature gradient gx.
struct MomentGrad { double g1, g2, g3; };
__device__ __forceinline__ MomentGrad moment_grad(const float *dX, int members, int N, int i, double a0i) {
    double g[6] = {0, 0, 0, 0, 0, 0};
    for (int m = 0; m < members; ++m)
        for (int e = 0; e < 6; ++e) g[e] += dX[(static_cast<long long>(m) * N + i) * kF + 68 + e];
    return {g[0] + a0i * g[3], g[1] + a0i * a0i * g[4], g[2] + a0i * a0i * g[5]};
}

// A_i = dE/dM_i = g1_i I/3 + 2 g3_i M_i/3 + (alpha0_i/3) sum_k g2_k B_ik (one warp per atom).
__global__ void k_moment_adjoint(int N, const double *R, const double *a0ref, const double *rref, const double *ratio,
                                 const double *Mw, const float *dX, int members, double *Aw) {
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const double a0i = a0ref[i] * ratio[i], rvi = rref[i] * cbrt(ratio[i]);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int k = lane; k < N; k += 32) {
        if (k == i) continue;
        const double r[3] = {R[3 * k] - R[3 * i], R[3 * k + 1] - R[3 * i + 1], R[3 * k + 2] - R[3 * i + 2]};
        const double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (d >= kCut) continue;
        const double a0k = a0ref[k] * ratio[k];
        double B[6];
        scs_coupling(r, d, a0i, a0k, rvi, rref[k] * cbrt(ratio[k]), B);
        const double g2k = moment_grad(dX, members, N, k, a0k).g2;
        for (int e = 0; e < 6; ++e) acc[e] += g2k * B[e];
    }
    for (int e = 0; e < 6; ++e) acc[e] = warp_sum_d(acc[e]);
    if (lane == 0) {
        const MomentGrad gi = moment_grad(dX, members, N, i, a0i);
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

// gR[i] += dE/dR_i through the features (one warp per atom, fixed order):
//   radial:  -sum_j sum_k (gx_ik alpha0_j + gx_jk alpha0_i) phi_k'(d_ij) r^_ij
//   moments: -sum_j <C_ij + C_ji, dB/dr (r_ij)>,  C_ij = alpha0_j (A_i + g2_i M_j / 3)
__global__ void k_learned_forces(int N, const double *R, const double *a0ref, const double *rref,
                                 const double *ratio, const double *Mw, const double *Aw, const float *dX,
                                 int members, double *gR) {
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const double a0i = a0ref[i] * ratio[i], rvi = rref[i] * cbrt(ratio[i]);
    const double g2i = moment_grad(dX, members, N, i, a0i).g2;
    const double *Mi = Mw + 6LL * i, *Ai = Aw + 6LL * i;
    const double i2w2 = 0.5 / (kWidth * kWidth);
    double f[3] = {0, 0, 0};
    for (int j = lane; j < N; j += 32) {
        if (j == i) continue;
        const double r[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
        const double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (d >= kCut) continue;
        const double a0j = a0ref[j] * ratio[j], rvj = rref[j] * cbrt(ratio[j]);
        // radial features
        const double fc = 0.5 * (1.0 + cos(kPiL * d / kCut)), dfc = -0.5 * kPiL / kCut * sin(kPiL * d / kCut);
        double s = 0.0;
        for (int k = 0; k < 64; ++k) {
            double gi = 0.0, gj = 0.0;
            for (int m = 0; m < members; ++m) {
                gi += dX[(static_cast<long long>(m) * N + i) * kF + k];
                gj += dX[(static_cast<long long>(m) * N + j) * kF + k];
            }
            const double mu = (k + 0.5) * kWidth, G = exp(-(d - mu) * (d - mu) * i2w2);
            s += (gi * a0j + gj * a0i) * (dfc * G + fc * G * (-(d - mu) * 2.0 * i2w2));
        }
        for (int c = 0; c < 3; ++c) f[c] -= s * r[c] / d;
        // moments
        const double g2j = moment_grad(dX, members, N, j, a0j).g2;
        const double *Mj = Mw + 6LL * j, *Aj = Aw + 6LL * j;
        double C[6], dB[3];
        for (int e = 0; e < 6; ++e) C[e] = a0j * (Ai[e] + g2i * Mj[e] / 3.0) + a0i * (Aj[e] + g2j * Mi[e] / 3.0);
        coupling_grad(r, d, a0i, a0j, rvi, rvj, C, dB);
        for (int c = 0; c < 3; ++c) f[c] -= dB[c];
    }
    for (int c = 0; c < 3; ++c) f[c] = warp_sum_d(f[c]);
    if (lane == 0)
        for (int c = 0; c < 3; ++c) gR[3 * i + c] += f[c];
}

inline int cdiv(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

}  // namespace

int learned_param_count() { return kParams; }

void learned_dy(int N, int members, int nf1, const double *h, const double *abar, float *dY, cudaStream_t s) {
    count_launches(1);
    k_learned_dy<<<cdiv(static_cast<long long>(members) * N * kO, 256), 256, 0, s>>>(N, members, nf1, h, abar, dY);
}

void learned_forces(int N, const double *R, const double *a0ref, const double *rref, const double *ratio,
                    const double *moments, const float *dX, int members, double *adjoint, double *gR, cudaStream_t s) {
    count_launches(2);
    k_moment_adjoint<<<cdiv(N, 8), 256, 0, s>>>(N, R, a0ref, rref, ratio, moments, dX, members, adjoint);
    k_learned_forces<<<cdiv(N, 8), 256, 0, s>>>(N, R, a0ref, rref, ratio, moments, adjoint, dX, members, gR);
}

void learned_alpha(int N, int members, int nf1, const double *al_u, const float *Y, double *abar, double *spread,
                   cudaStream_t s) {
    count_launches(1);
    k_learned_alpha<<<cdiv(static_cast<long long>(N) * nf1, 256), 256, 0, s>>>(N, members, nf1, al_u, Y, abar,
                                                                               spread);
}

void learned_estimate(int N, int nf1, const double *h, const double *spread, double *out, cudaStream_t s) {
    count_launches(1);
    k_learned_estimate<<<1, 1024, 0, s>>>(N * nf1, N, h, spread, out);
}

void scs_features(int n_atoms, int n_sys, const int *offsets, const double *R, const double *a0ref,
                  const double *c6ref, const double *rref, const double *ratio, float *X, double *work,
                  cudaStream_t s) {
    count_launches(2);
    k_features<<<cdiv(n_atoms, 8), 256, 0, s>>>(n_atoms, n_sys, offsets, R, a0ref, c6ref, rref, ratio, X, work);
    k_feature_moments<<<cdiv(n_atoms, 8), 256, 0, s>>>(n_atoms, n_sys, offsets, R, a0ref, rref, ratio, work, X);
}

cudaError_t mlp_forward(int B, int members, const float *X, const float *mean, const float *stdv,
                        const void *params16, float *Y, float *zcache, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kMlpSmem));
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_mlp_forward<<<dim3(cdiv(B, kTA), members), 128, kMlpSmem, s>>>(
        B, X, mean, stdv, static_cast<const __half *>(params16), Y, zcache);
    return cudaGetLastError();
}

cudaError_t mlp_backward(int B, int members, const float *X, const float *mean, const float *stdv,
                         const void *params16, const float *zcache, const float *dY, float *dX, float *grad,
                         cudaStream_t s) {
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

int mbdk_gather_rows(void *stream, long long rows, int width, const int *idx, const float *src, float *dst) {
    if (rows < 1 || width < 1 || !idx || !src || !dst) return MBD_ERR_INPUT;
    mbdgb::gather_rows(rows, width, idx, src, dst, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

}  // extern "C"
