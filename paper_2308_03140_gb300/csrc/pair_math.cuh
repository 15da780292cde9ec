// Helpers shared by the pair kernels (k_pairs.cu, k_periodic.cu): the Fermi damping
// function, the radial parts of the dipole tensors (host and device, so that the CPU tests
// can evaluate the kernels' own formulas) and warp/block sums (device).
// The dipole tensors are written T_ab = P delta_ab + W r_a r_b with radial P, W.
#pragma once
#include "internal.h"

namespace mbdgb {
namespace pairs {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTwoOverSqrtPi = 1.128379167095512573896158903121545172;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NV values per thread (blockDim.x == 128); result valid in thread 0.
template <int NV>
__device__ void block_sum128(double (&v)[NV], double *scratch /* [4][NV] */) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[w * NV + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = scratch[k] + scratch[NV + k] + scratch[2 * NV + k] + scratch[3 * NV + k];
    __syncthreads();
}

// Fermi function of Eq. (fermi-damping) and its derivatives with respect to the pair
// distance rho and the radius sum S.
struct Fermi { double f, df_drho, df_dS; };
__host__ __device__ __forceinline__ Fermi fermi(double rho, double S, double beta, double a) {
    const double x = rho / (beta * S);
    const double f = 1.0 / (1.0 + exp(-a * (x - 1.0)));
    const double dfx = a * f * (1.0 - f);
    return {f, dfx / (beta * S), -dfx * x / S};
}

// Radial parts of T^GG(r; s) (Eq. tgg): P = F1/r^3, W = (2 z^2 Th - 3 F1)/r^5 with
// z = r/s, Th = 2 z e^{-z^2}/sqrt(pi), F1 = erf z - Th; and d/dr, d/ds of both.
struct Radial { double P, W, dP, dW, dPs, dWs; };
// Beyond z = 8 the Gaussian parts vanish in FP64: erf z rounds to 1 and 2 z e^{-z^2}/sqrt(pi)
// < 1.5e-27, so P, W, dP, dW are those of the bare tensor to the last bit and s dP/ds,
// s dW/ds are below 1e-22 of dP, dW; the far branch skips erf and exp.
constexpr double kGaussFar = 8.0;
constexpr float kGaussFarF = 5.0f;   // FP32: erff(5) rounds to 1, 2 z e^{-z^2}/sqrt(pi) < 1e-10
__host__ __device__ __forceinline__ Radial tgg_radial(double rho, double s) {
    const double z = rho / s, z2 = z * z;
    if (z > kGaussFar) {
        const double ir = 1.0 / rho, ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
        Radial o;
        o.P = ir3;
        o.W = -3.0 * ir5;
        o.dP = -3.0 * ir3 * ir;
        o.dW = 15.0 * ir5 * ir;
        o.dPs = 0.0;
        o.dWs = 0.0;
        return o;
    }
    const double th = kTwoOverSqrtPi * z * exp(-z2);
    const double F1 = erf(z) - th;
    const double G = 2.0 * z2 * th - 3.0 * F1;
    const double ir = 1.0 / rho, ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
    Radial o;
    o.P = F1 * ir3;
    o.W = G * ir5;
    o.dP = 2.0 * z * th / s * ir3 - 3.0 * F1 * ir3 * ir;
    o.dW = -4.0 * z2 * z * th / s * ir5 - 5.0 * G * ir5 * ir;
    o.dPs = -2.0 * z2 * th / s * ir3;
    o.dWs = 4.0 * z2 * z2 * th / s * ir5;
    return o;
}

// Bare dipole tensor T = -grad grad 1/r, Eq. (dipole): P = 1/r^3, W = -3/r^5, and d/dr.
struct RadialT { double P, W, dP, dW; };
__host__ __device__ __forceinline__ RadialT bare_radial(double rho) {
    const double ir = 1.0 / rho, ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
    return {ir3, -3.0 * ir5, -3.0 * ir3 * ir, 15.0 * ir5 * ir};
}

// erfc-screened dipole tensor -grad grad erfc(gamma r)/r (Eq. terfc with the numerator
// -r_a r_b C + delta r^2 B): P = B/r^3, W = -C/r^5, x = gamma r, e = 2x e^{-x^2}/sqrt(pi),
// B = erfc x + e, C = 3 erfc x + e (3 + 2x^2); dB/dx = -2x e, dC/dx = -4x^3 e.
__host__ __device__ __forceinline__ RadialT erfc_radial(double rho, double gamma) {
    const double x = gamma * rho, ex = kTwoOverSqrtPi * x * exp(-x * x), ec = erfc(x);
    const double Bx = ec + ex, Cx = 3.0 * ec + ex * (3.0 + 2.0 * x * x);
    const double ir = 1.0 / rho, ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
    return {Bx * ir3, -Cx * ir5, -2.0 * gamma * x * ex * ir3 - 3.0 * Bx * ir3 * ir,
            4.0 * gamma * x * x * x * ex * ir5 + 5.0 * Cx * ir5 * ir};
}

// Single-precision versions of fermi and tgg_radial for the pair passes of the
// reduced-precision modes (same formulas).
struct FermiF { float f, df_drho, df_dS; };
__host__ __device__ __forceinline__ FermiF fermi_f(float rho, float S, float beta, float a) {
    const float x = rho / (beta * S);
    const float f = 1.0f / (1.0f + expf(-a * (x - 1.0f)));
    const float dfx = a * f * (1.0f - f);
    return {f, dfx / (beta * S), -dfx * x / S};
}
struct RadialF { float P, W, dP, dW, dPs, dWs; };
__host__ __device__ __forceinline__ RadialF tgg_radial_f(float rho, float s) {
    const float z = rho / s, z2 = z * z;
    if (z > kGaussFarF) {
        const float ir = 1.0f / rho, ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
        RadialF o;
        o.P = ir3;
        o.W = -3.0f * ir5;
        o.dP = -3.0f * ir3 * ir;
        o.dW = 15.0f * ir5 * ir;
        o.dPs = 0.0f;
        o.dWs = 0.0f;
        return o;
    }
    const float th = static_cast<float>(kTwoOverSqrtPi) * z * expf(-z2);
    const float F1 = erff(z) - th;
    const float G = 2.0f * z2 * th - 3.0f * F1;
    const float ir = 1.0f / rho, ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
    RadialF o;
    o.P = F1 * ir3;
    o.W = G * ir5;
    o.dP = 2.0f * z * th / s * ir3 - 3.0f * F1 * ir3 * ir;
    o.dW = -4.0f * z2 * z * th / s * ir5 - 5.0f * G * ir5 * ir;
    o.dPs = -2.0f * z2 * th / s * ir3;
    o.dWs = 4.0f * z2 * z2 * th / s * ir5;
    return o;
}

}  // namespace pairs
}  // namespace mbdgb
