// Error-free splitting of FP64 operands into tensor-core slices (FP64-accurate products on
// the TF32 tensor path; the paper has no counterpart, its FP64 products run on CPUs).
//
// A row r of A with max |A[r][:]| = m 2^e (1/2 <= m < 1) is scaled by 2^-e, so that every
// t = A[r][c] 2^-e has |t| < 1, and cut into kSlices slices of kSliceBits bits:
//     t = sum_p a_p 2^{-b (p+1)} + rem,   a_p integers, |a_p| < 2^b,   |rem| < 2^{-b kSlices},
// each a_p taken by truncation of the running remainder times 2^b (exact in FP64).  Slice p
// is stored as the FP32 value a_p 2^{e - b (p+1)}, exact in FP32 and in TF32 (b <= 11
// significant bits).  With both operands sliced this way (A by rows, op(B) by columns) every
// term of a slice product A_p op(B)_q for fixed (i, j) carries the same power of two
// 2^{e_i + f_j - b (p+q+2)} and an integer |a b| < 2^{2b}; over K' <= kSplitChunk terms the
// sum stays below 2^{2b} K' <= 2^22 times that unit, so the tensor core's FP32 accumulation
// is exact (with two bits to spare), as are the epilogue's FP32 chunk sums.  The products
// of weight p + q <= kSlices are kept (53): a dropped term is below 2^{2b - b (kSlices + 3)}
// = 2^-60 of 2^{e_i + f_j} per element of K, which keeps the result as accurate as an FP64
// GEMM's (the weight-9 products matter: without them the error reaches ~20 ulps of
// sum_k |A_ik| |B_kj| where an FP64 GEMM stays near 3).
#pragma once
#include "internal.h"

namespace mbdgb {
namespace split64 {

constexpr int kSliceBits = 6;
constexpr int kSlices = 9;          // 54 bits of each operand
constexpr int kSplitChunk = 1024;   // K per tensor-core product: 2^(2 kSliceBits) 1024 = 2^22

// Exponent e with |x| 2^-e < 1 for every |x| <= amax (0 for amax == 0), at least kMinExponent:
// the last slice's unit 2^{e - b kSlices} then stays an FP32 normal number (>= 2^-126), which
// the tensor cores do not flush.  A row whose largest element lies below 2^kMinExponent is
// sliced at that exponent: its slices are still exact, and it keeps an absolute accuracy of
// 2^-126 instead of a relative one.
constexpr int kMinExponent = -126 + kSliceBits * kSlices;   // -72
__host__ __device__ inline int scale_exponent(double amax) {
    if (!(amax > 0.0)) return 0;
    int e;
    frexp(amax, &e);
    return e < kMinExponent ? kMinExponent : e;
}

// The slices of x for the row exponent e: out[p] = a_p 2^{e - b (p+1)} (FP32, exact).
__host__ __device__ inline void slice(double x, int e, float *out) {
    double t = ldexp(x, -e);
    for (int p = 0; p < kSlices; ++p) {
        t *= static_cast<double>(1 << kSliceBits);
        const double a = trunc(t);
        t -= a;
        out[p] = static_cast<float>(ldexp(a, e - kSliceBits * (p + 1)));
    }
}

}  // namespace split64
}  // namespace mbdgb
