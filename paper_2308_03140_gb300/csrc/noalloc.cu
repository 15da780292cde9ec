// Allocation-free factor-and-solve entry point (declared in include/mbd_gb300_kernels.h).
//
// Some callers cannot let a library allocate device memory: codes that hand all of
// the GPU's memory to their own pool up front (an electronic-structure or MD code
// with a fixed device-memory budget), and codes that must not pay the implicit
// device-wide synchronisation that cudaMalloc and cudaFree can cause in the middle
// of a time step.  For them this file keeps the scratch of factor-and-solve (the
// inverses of the 64x64 diagonal blocks of each Cholesky factor and the intermediate
// of the triangular solves) in a file-scope device array instead of caller- or
// library-allocated memory.
//
// The array is a fixed 16 MiB (2^21 doubles) that every GPU which loads the library
// holds until the process exits.  All calls on a device share it: two calls whose
// work overlaps on that GPU (different streams, or host threads) race on it and must
// be serialised by the caller.  Nothing in it needs to start at zero: the
// factorisation writes every scratch element before any kernel reads it.
#include <mutex>

#include "../../include/mbd_gb300.h"
#include "../../include/mbd_gb300_kernels.h"
#include "internal.h"

namespace {

constexpr long long kScratchDoubles = 1LL << 21;   // 16 MiB
__device__ __align__(256) double g_chol_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of g_chol_scratch on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device with
// that device current, and cached for the life of the process (a cudaDeviceReset of the
// device invalidates it; the header asks callers to reload the library after one).
int scratch_address(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MBD_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_chol_scratch) != cudaSuccess || !p) return MBD_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return MBD_OK;
}

}  // namespace

extern "C" int mbdk_cholesky_solve3_f64_noalloc(void *stream, double *A, long long ld, int batch,
                                                double *X, int *status) {
    if (ld <= 0 || ld % mbdgb::kTile || batch < 1 || !A || !X || !status) return MBD_ERR_INPUT;
    const long long dinv_n = static_cast<long long>(batch) * (ld / mbdgb::kTile) * 4096LL;
    const long long need = dinv_n + static_cast<long long>(batch) * 3 * ld;
    if (need > kScratchDoubles) return MBD_ERR_SCRATCH_LIMIT;
    double *scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    mbdgb::cholesky_f64(A, ld, ld * ld, batch, scratch, status, s);
    mbdgb::chol_solve3_f64(A, ld, ld * ld, batch, scratch, X, scratch + dinv_n, 3 * ld, s);
    return cudaGetLastError() == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}
