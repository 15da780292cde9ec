// Host run of the FP64 operand slicing of the CUDA library (split64::scale_exponent and
// split64::slice of csrc/split64.cuh, the functions k_row_exponents, k_row_slices and
// k_col_slices call), for the CPU tests.  Test infrastructure: built by
// tests/test_split64_host.py into tests/_build.
#include <cmath>

#include "split64.cuh"

using namespace mbdgb;

extern "C" int split64_slices_count() { return split64::kSlices; }
extern "C" int split64_slice_bits() { return split64::kSliceBits; }
extern "C" int split64_chunk() { return split64::kSplitChunk; }

// Row exponents and slices S [kSlices][rows][cols] of a row-major rows x cols matrix, as
// k_row_exponents and k_row_slices compute them.
extern "C" void split64_rows(const double *A, int rows, int cols, int *e, float *S) {
    const long long stride = static_cast<long long>(rows) * cols;
    for (int r = 0; r < rows; ++r) {
        double m = 0.0;
        for (int c = 0; c < cols; ++c) m = std::fmax(m, std::fabs(A[static_cast<long long>(r) * cols + c]));
        e[r] = split64::scale_exponent(m);
        for (int c = 0; c < cols; ++c) {
            float sl[split64::kSlices];
            split64::slice(A[static_cast<long long>(r) * cols + c], e[r], sl);
            for (int p = 0; p < split64::kSlices; ++p) S[p * stride + static_cast<long long>(r) * cols + c] = sl[p];
        }
    }
}
