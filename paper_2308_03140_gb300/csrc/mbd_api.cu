// Host orchestration and C ABI of libmbdgb (declared in include/mbd_gb300.h).
//
// One evaluation is one stream-ordered pass over the device:
//   prepare_atoms -> build_scs (all frequencies) -> batched Cholesky -> X = A^{-1} E
//   -> contract_screen -> build_q -> Gershgorin scale -> coupled Newton-Schulz
//   -> energy; and for gradients: mbd_grad_pass -> chain_screen -> V = A^{-1} H
//   -> scs_grad_pass -> ts_chain.
// The host reads back one scalar per Newton-Schulz iteration (the convergence test)
// and the status word after the screening stage.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mbd_gb300.h"
#include "../../include/mbd_gb300_kernels.h"
#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "freq_grid.h"
#include "ns_schedule.h"

using namespace mbdgb;

namespace {
std::atomic<long long> g_launches{0};
// Refinement steps of the mixed screening solves: the FP32 factor's solution carries relative
// errors of a few 1e-7 in the screened polarizabilities, one step against the FP64 matrix
// brings them to about 1e-13 (screening matrices of kappa up to ~2e3).
constexpr int kRefineSteps = 1;
// Refinement steps of the mixed modes' adjoint solves V = A^{-1} H: the unrefined FP32 solve
// errs by at most kappa(A) eps32 ~ 1e-4 relative to the SCS part of the gradient; the TF32x3
// force error measured at 2000 atoms with it (3e-6 of the largest force) is well inside that.
constexpr int kAdjointRefineSteps = 0;
constexpr int kLanczosSteps = 48; // Lanczos steps of the spectrum estimate of Q
// ... and in the mixed modes for Q of order <= kLanczosSmallOrder: on the spectra of clusters of
// 70-500 atoms the mixed loop, which stops at its precision floor, takes the same number of
// steps (8-9) from a 24-step estimate as from a 48-step one (the lower estimate is then 3-10
// times higher, which only shortens the first steps), while the 24 steps save 48 of the
// evaluation's ~190 launches.  The FP64 loop, which converges further, can take one step
// more from it (11 against 10 on a 500-atom cluster) and keeps the 48.
constexpr int kLanczosStepsSmall = 24;
constexpr long long kLanczosSmallOrder = 2048;
// Precision floor of the TF32x3 Newton-Schulz iteration per unit of sqrt(n): |I - Z Y|_F
// settles at about 1.04e-7 sqrt(n) (8.1e-6 at n = 6000).  A step taken from a residual r whose
// exact successor bound 0.875 r^2 lies below this is the last useful one.  The coarser kinds
// (TF32, BF16x3) reach their floors above it and stop by the halving test alone.
constexpr double kMixedFloor = 1e-7;
// Periodic Newton-Schulz (FP64): Y' and Z' as Hermitian products (upper tiles only, real part
// mirrored, imaginary part mirrored with a sign change), a third fewer flops per step.
constexpr bool kHermitianNs = true;
constexpr int kLF = MBD_LEARNED_FEATURES;   // inputs of the learned screening model
// The FP64 path (screening, bounds, Newton-Schulz, gradients in FP64), with its Newton-Schulz
// products on the DMMA pipe (MBD_PREC_FP64) or FP64-accurate on the TF32 tensor cores.
inline bool fp64_path(int precision) { return precision == MBD_PREC_FP64 || precision == MBD_PREC_FP64_SPLIT; }
}  // namespace

void mbdgb::count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long mbdgb::launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

// Number of eigenvalues below x of the symmetric tridiagonal matrix (diag a, offdiag b)
// by the Sturm sequence of its LDL^T pivots.
int sturm_count(const std::vector<double> &a, const std::vector<double> &b, double x) {
    int cnt = 0;
    double d = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        const double off = i ? b[i - 1] * b[i - 1] : 0.0;
        d = a[i] - x - (i ? off / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// Smallest and largest eigenvalue of a symmetric tridiagonal matrix by bisection.
void tridiag_extremes(const std::vector<double> &a, const std::vector<double> &b, double &lo, double &hi) {
    double g0 = 1e300, g1 = -1e300;   // Gershgorin interval of the tridiagonal
    for (size_t i = 0; i < a.size(); ++i) {
        const double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < a.size() ? std::fabs(b[i]) : 0.0);
        g0 = std::min(g0, a[i] - r);
        g1 = std::max(g1, a[i] + r);
    }
    const int m = static_cast<int>(a.size());
    double l = g0, h = g1;
    for (int it = 0; it < 200; ++it) {   // smallest: count(x) >= 1
        const double mid = 0.5 * (l + h);
        if (sturm_count(a, b, mid) >= 1) h = mid; else l = mid;
    }
    lo = h;
    l = g0; h = g1;
    for (int it = 0; it < 200; ++it) {   // largest: count(x) >= m
        const double mid = 0.5 * (l + h);
        if (sturm_count(a, b, mid) >= m) h = mid; else l = mid;
    }
    hi = h;
}

}  // namespace

struct mbd_ctx {
    int device = 0;
    mbd_options opt{};
    cudaStream_t stream = nullptr;
    // problem
    int N = 0, n = 0, nf1 = 0, nb = 0;
    long long ld = 0;
    bool have_geom = false, have_params = false;
    std::vector<double> hR, ha0, hc6, hrr, hv;
    std::vector<double> hu, hwu;
    // device memory: one slab, carved
    void *slab = nullptr;
    size_t slab_bytes = 0;
    double *dR, *da0ref, *dc6ref, *drref, *dratio;
    double *da0, *dom, *drv, *dalu, *dsigu, *dabar, *dabar0, *dc6bar, *dombar, *drbar, *du, *dwu;
    double *dM, *ddinv, *dX, *dV, *dB;
    float *sM = nullptr, *sdinv = nullptr, *swork = nullptr;   // FP32 factors of the mixed modes
    uint32_t *spanel = nullptr;   // TF32x3 parts of the factor panels (tensor-core trailing updates)
    float *sgrad32 = nullptr;     // FP32 inputs of the reduced-precision SCS adjoint pair pass
    double *dlog = nullptr;       // per-frequency sums of the log-formula route: ln det, Tr A^2..4
    double *dtq = nullptr;        // Tr (Q^{1/2})_ii per atom from the mixed modes' FP64 correction
    bool tq_valid = false;
    double *dQ, *dZ, *dP, *dY2, *dZ2;
    // mixed-precision Newton-Schulz buffers (ld x ld each)
    float *fY = nullptr, *fZ = nullptr, *fY2 = nullptr, *fZ2 = nullptr, *fP = nullptr, *fPT = nullptr;
    void *hY[2] = {}, *hZ[2] = {}, *hY2[2] = {}, *hZ2[2] = {}, *hP[2] = {}, *hPT[2] = {};   // split operands
    double corr_resid = 0.0;   // |Zd Q Zd - I|_F of the mixed modes' correction
    // mixed modes on a cell: each Hermitian Q(q) as the real symmetric [[Re, -Im], [Im, Re]] of
    // order 2n (leading dimension lde), its FP64 workspaces
    long long lde = 0;
    double *eM = nullptr, *eV = nullptr, *eW = nullptr, *eVT = nullptr, *eZ = nullptr;
    double *dh, *dgomb, *dgab0, *dgrb, *dgR, *dga0, *dgom, *dgrv, *dgp;
    // periodic systems: cell, Bloch vectors and reciprocal lattice (host lists, device copies)
    bool periodic = false;
    int nk = 1, nG = 0, maxG = 0;
    CellGeom cell{};
    std::vector<double> hkq, hG;
    std::vector<int> hglist, hgcount;
    void *dsplit = nullptr;   // slices of the split FP64 GEMM (MBD_PREC_FP64_SPLIT)
    double *dkq = nullptr, *dG = nullptr, *dcoef = nullptr, *dlzw = nullptr, *dgA = nullptr, *dgAout = nullptr,
           *dgApart = nullptr, *dgc = nullptr, *dtsg = nullptr;
    int *dglist = nullptr, *dgcount = nullptr;
    double2 *dS = nullptr;
    bool have_lattice_grad = false;
    // learned screening model (host copy; device buffers in their own allocation)
    int members = 0;
    std::vector<uint16_t> hmodel;
    std::vector<float> hmean, hstd;
    bool model_dirty = false, force_plain = false;
    void *lslab = nullptr;
    size_t lbytes = 0;
    int lN = 0, lM = 0;
    void *dmodel = nullptr;
    float *dmeanstd = nullptr, *dfeat = nullptr, *dYl = nullptr;
    double *dspread = nullptr, *dmoments = nullptr, *dadj = nullptr;
    float *dzc = nullptr, *dXl = nullptr;   // MLP cache and feature gradient (learned forces)
    float *dpacked = nullptr;               // the members' weights in the MLP kernels' layout
    int *doffs = nullptr;
    double learned_est = 0.0;
    int learned_fallback = 0;
    bool last_learned = false;   // the last forward kept the learned model's screening
    double *dscal;   // [0] energy, [1] Gershgorin, [2] residual
    int *dstatus;
    // last results
    int ns_iter = 0;
    double ns_scale = 0.0, ns_resid = 0.0;
    bool have_result = false;
    bool have_screening = false;
    // state of the last forward evaluation, kept for mbd_backward_dev
    bool have_forward = false;
    long long eval_count = 0;  // successful evaluations of this context so far
    double *Zlast = nullptr;   // Newton-Schulz Z (Q^{-1/2} = zscale * Z)
    double zscale = 0.0;
    // exception
    int err_code = MBD_OK;
    std::string err_origin, err_msg;
    // profiling (CUDA events on the launch stream)
    bool profiling = false;
    std::vector<cudaEvent_t> events;
    int ev_used = 0;
    mbd_profile prof{};
};

namespace {

int fail(mbd_ctx *c, int code, const char *origin, const std::string &msg) {
    if (c) {
        c->err_code = code;
        c->err_origin = origin;
        c->err_msg = msg;
    }
    return code;
}

int cuda_fail(mbd_ctx *c, const char *origin, cudaError_t e) {
    return fail(c, MBD_ERR_CUDA, origin, std::string("CUDA error: ") + cudaGetErrorString(e));
}

#define MBD_CUDA(call, origin)                                  \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(ctx, origin, e_); \
    } while (0)

// Next free timing event of the context (created on first use, reused per evaluation).
cudaEvent_t next_event(mbd_ctx *ctx) {
    if (ctx->ev_used == static_cast<int>(ctx->events.size())) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->events.push_back(e);
    }
    return ctx->events[ctx->ev_used++];
}

struct Span { cudaEvent_t a = nullptr, b = nullptr; double flops = 0.0; };

// NVTX ranges of the evaluation stages on the host timeline (no-ops unless a profiler is
// attached); the range open at any return is closed by the destructor.
struct NvtxStages {
    bool open = false;
    void next(const char *name) {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    ~NvtxStages() {
        if (open) nvtxRangePop();
    }
};

void mark(mbd_ctx *ctx, cudaStream_t s, cudaEvent_t &e) {
    if (!ctx->profiling) return;
    e = next_event(ctx);
    if (e) cudaEventRecord(e, s);
}

double span_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (a && b && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) return ms;
    return 0.0;
}

void release(mbd_ctx *ctx) {
    if (ctx->slab) cudaFree(ctx->slab);
    ctx->slab = nullptr;
    ctx->slab_bytes = 0;
}

// Device buffers of the learned model for N atoms and M members (own allocation, resized on
// demand); uploads the model when it changed.
int ensure_learned(mbd_ctx *ctx) {
    const int N = ctx->N, M = ctx->members, nf1 = ctx->nf1;
    const size_t P = static_cast<size_t>(learned_param_count());
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    if (!ctx->lslab || ctx->lN != N || ctx->lM != M) {
        const size_t bytes = al(2 * P * M) + al(sizeof(float) * 2 * kLF) + al(sizeof(float) * kLF * N) +
                             al(sizeof(float) * M * N * 16) + al(sizeof(double) * nf1 * N) +
                             al(sizeof(double) * kLearnedWork * N) + al(sizeof(double) * kLearnedAdjointWork * N) +
                             al(sizeof(float) * M * 2 * N * 128) +
                             al(sizeof(float) * M * N * kLF) + al(sizeof(float) * M * kLearnedPackedFloats) +
                             al(sizeof(int) * 2);
        cudaError_t e = cudaSuccess;
        if (!ctx->lslab || ctx->lbytes < bytes) {   // re-carved in place when large enough
            if (ctx->lslab) cudaFree(ctx->lslab);
            ctx->lslab = nullptr;
            e = cudaMalloc(&ctx->lslab, bytes);
            if (e != cudaSuccess) return cuda_fail(ctx, "learned_screening", e);
            ctx->lbytes = bytes;
        }
        char *p = static_cast<char *>(ctx->lslab);
        ctx->dmodel = p; p += al(2 * P * M);
        ctx->dmeanstd = reinterpret_cast<float *>(p); p += al(sizeof(float) * 2 * kLF);
        ctx->dfeat = reinterpret_cast<float *>(p); p += al(sizeof(float) * kLF * N);
        ctx->dYl = reinterpret_cast<float *>(p); p += al(sizeof(float) * M * N * 16);
        ctx->dspread = reinterpret_cast<double *>(p); p += al(sizeof(double) * nf1 * N);
        ctx->dmoments = reinterpret_cast<double *>(p); p += al(sizeof(double) * kLearnedWork * N);
        ctx->dadj = reinterpret_cast<double *>(p); p += al(sizeof(double) * kLearnedAdjointWork * N);
        ctx->dzc = reinterpret_cast<float *>(p); p += al(sizeof(float) * M * 2 * N * 128);
        ctx->dXl = reinterpret_cast<float *>(p); p += al(sizeof(float) * M * N * kLF);
        ctx->dpacked = reinterpret_cast<float *>(p); p += al(sizeof(float) * M * kLearnedPackedFloats);
        ctx->doffs = reinterpret_cast<int *>(p);
        const int offs[2] = {0, N};
        e = cudaMemcpy(ctx->doffs, offs, sizeof(offs), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, "learned_screening", e);
        ctx->lN = N;
        ctx->lM = M;
        ctx->model_dirty = true;
    }
    if (ctx->model_dirty) {
        cudaError_t e = cudaMemcpy(ctx->dmodel, ctx->hmodel.data(), 2 * P * M, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(ctx->dmeanstd, ctx->hmean.data(), sizeof(float) * kLF, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(ctx->dmeanstd + kLF, ctx->hstd.data(), sizeof(float) * kLF, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = mlp_pack(M, ctx->dmodel, ctx->dpacked, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(ctx, "learned_screening", e);
        ctx->model_dirty = false;
    }
    return MBD_OK;
}

// Carves the workspace out of one allocation (256-byte aligned pieces).
int allocate(mbd_ctx *ctx) {
    const long long ld = ctx->ld, N = ctx->N, nf1 = ctx->nf1, nb = ctx->nb;
    const size_t mat = sizeof(double) * static_cast<size_t>(ld) * ld;
    std::vector<std::pair<double **, size_t>> plan = {
        {&ctx->dR, 3 * N}, {&ctx->da0ref, N}, {&ctx->dc6ref, N}, {&ctx->drref, N}, {&ctx->dratio, N},
        {&ctx->da0, N}, {&ctx->dom, N}, {&ctx->drv, N}, {&ctx->dalu, nf1 * N}, {&ctx->dsigu, nf1 * N},
        {&ctx->dabar, nf1 * N}, {&ctx->dabar0, N}, {&ctx->dc6bar, N}, {&ctx->dombar, N},
        {&ctx->drbar, N}, {&ctx->du, nf1}, {&ctx->dwu, nf1}, {&ctx->dlog, 4 * nf1}, {&ctx->dtq, N},
        {&ctx->ddinv, nf1 * nb * 4096}, {&ctx->dX, nf1 * ld * 3}, {&ctx->dV, nf1 * ld * 3},
        {&ctx->dB, nf1 * ld * 3},
        {&ctx->dh, nf1 * N}, {&ctx->dgomb, N}, {&ctx->dgab0, N}, {&ctx->dgrb, N}, {&ctx->dgR, 3 * N},
        {&ctx->dga0, N}, {&ctx->dgom, N}, {&ctx->dgrv, N}, {&ctx->dgp, 4 * N}, {&ctx->dscal, 8 + 2 * 64 + 1024},
    };
    const long long nk = ctx->nk;
    if (ctx->periodic) {
        plan.push_back({&ctx->dkq, 3 * nk});
        plan.push_back({&ctx->dG, 3LL * ctx->nG});
        plan.push_back({&ctx->dcoef, nk * 2 * kLanczosSteps});
        plan.push_back({&ctx->dlzw, 3 * nk * 2 * ld});
        plan.push_back({&ctx->dgA, 9});
        plan.push_back({&ctx->dgAout, 9});
        plan.push_back({&ctx->dgApart, 9 * N});
        plan.push_back({&ctx->dgc, N});
        plan.push_back({&ctx->dtsg, 2LL * ctx->nG});
        plan.push_back({reinterpret_cast<double **>(&ctx->dS), 2LL * ctx->nG * N});
        plan.push_back({reinterpret_cast<double **>(&ctx->dglist), (nk * ctx->maxG + 1) / 2});
        plan.push_back({reinterpret_cast<double **>(&ctx->dgcount), (nk + 1) / 2});
    }
    size_t bytes = 0;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    for (auto &p : plan) bytes += al(sizeof(double) * p.second);
    bytes += al(sizeof(int) * 4);
    const size_t small = bytes;
    bytes += nf1 * mat;          // screening matrices / factors
    // Q (= Y), Z, P, Y', Z': real, or nk planar complex matrices for a periodic system
    const size_t matq = ctx->periodic ? mat * 2 * static_cast<size_t>(nk) : mat;
    bytes += 5 * matq;
    const int prec = ctx->opt.precision;
    // the mixed modes' iteration buffers: the matrix order, or the order of a cell's embedded
    // Hermitian matrices
    const long long ldm = ctx->periodic ? ctx->lde : ld;
    const size_t mat32 = sizeof(float) * static_cast<size_t>(ldm) * ldm, mat16 = mat32 / 2;
    const size_t split_mat = prec == MBD_PREC_BF16X3 ? mat16 : (prec == MBD_PREC_TF32X3 ? mat32 : 0);
    if (!fp64_path(prec)) bytes += 6 * mat32;
    const size_t emat = sizeof(double) * static_cast<size_t>(ctx->lde) * ctx->lde;
    const bool embed = ctx->periodic && !fp64_path(prec);
    if (embed) bytes += 5 * emat;
    const size_t split_work = prec == MBD_PREC_FP64_SPLIT ? al(gemm_f64_split_work_bytes(static_cast<int>(ld),
                                                                                          static_cast<int>(ld),
                                                                                          static_cast<int>(ld)))
                                                          : 0;
    bytes += split_work;
    bytes += 12 * split_mat;
    // FP32 screening factors, their diagonal-block inverses and solve workspace
    const size_t panel_words = 2 * nf1 * static_cast<size_t>(ld) * kScsPanel;
    const size_t grad32 = 2 * nf1 * (3 * static_cast<size_t>(ld) + N);
    const size_t scs32 = !fp64_path(prec) && !ctx->periodic   // cells screen in FP64 (Gamma point)
                             ? nf1 * (mat / 2) + al(sizeof(float) * nf1 * nb * 4096) +
                                   al(sizeof(float) * 2 * nf1 * ld * 3) + al(sizeof(uint32_t) * panel_words) +
                                   al(sizeof(float) * grad32)
                             : 0;
    bytes += scs32;
    // A slab large enough for the new size is re-carved in place (systems of varying size in
    // a batch then reuse one allocation); otherwise it is replaced.
    cudaError_t e = cudaSuccess;
    if (!ctx->slab || ctx->slab_bytes < bytes) {
        release(ctx);
        e = cudaMalloc(&ctx->slab, bytes);
        if (e != cudaSuccess) return cuda_fail(ctx, "mbd_set_geometry", e);
        ctx->slab_bytes = bytes;
    }
    char *p = static_cast<char *>(ctx->slab);
    for (auto &q : plan) {
        *q.first = reinterpret_cast<double *>(p);
        p += al(sizeof(double) * q.second);
    }
    ctx->dstatus = reinterpret_cast<int *>(p);
    p = static_cast<char *>(ctx->slab) + small;
    ctx->dM = reinterpret_cast<double *>(p);
    p += nf1 * mat;
    double **mats[5] = {&ctx->dQ, &ctx->dZ, &ctx->dP, &ctx->dY2, &ctx->dZ2};
    for (auto m : mats) {
        *m = reinterpret_cast<double *>(p);
        p += matq;
    }
    if (split_work) {
        ctx->dsplit = p;
        p += split_work;
    }
    if (!fp64_path(prec)) {
        float **f32[6] = {&ctx->fY, &ctx->fZ, &ctx->fY2, &ctx->fZ2, &ctx->fP, &ctx->fPT};
        for (auto m : f32) {
            *m = reinterpret_cast<float *>(p);
            p += mat32;
        }
    }
    if (split_mat) {
        void **parts[6] = {ctx->hY, ctx->hZ, ctx->hY2, ctx->hZ2, ctx->hP, ctx->hPT};
        for (auto m : parts)
            for (int k = 0; k < 2; ++k) {
                m[k] = p;
                p += split_mat;
            }
    }
    if (embed) {
        double **em[5] = {&ctx->eM, &ctx->eV, &ctx->eW, &ctx->eVT, &ctx->eZ};
        for (auto m : em) {
            *m = reinterpret_cast<double *>(p);
            p += emat;
        }
    }
    if (scs32) {
        ctx->sM = reinterpret_cast<float *>(p);
        p += nf1 * (mat / 2);
        ctx->sdinv = reinterpret_cast<float *>(p);
        p += al(sizeof(float) * nf1 * nb * 4096);
        ctx->swork = reinterpret_cast<float *>(p);
        p += al(sizeof(float) * 2 * nf1 * ld * 3);
        ctx->spanel = reinterpret_cast<uint32_t *>(p);
        p += al(sizeof(uint32_t) * panel_words);
        ctx->sgrad32 = reinterpret_cast<float *>(p);
        p += al(sizeof(float) * grad32);
    }
    // Untouched parts of the factor buffers (strict upper triangles) are read by no
    // kernel; clearing them once keeps them finite.
    e = cudaMemset(ctx->slab, 0, bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, "mbd_set_geometry", e);
    e = cudaMemcpy(ctx->du, ctx->hu.data(), sizeof(double) * nf1, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->dwu, ctx->hwu.data(), sizeof(double) * nf1, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, "mbd_set_geometry", e);
    return MBD_OK;
}

// Uploads the Bloch vectors and reciprocal-vector lists of a periodic geometry.
int upload_periodic(mbd_ctx *ctx) {
    cudaError_t e = cudaMemcpy(ctx->dkq, ctx->hkq.data(), sizeof(double) * ctx->hkq.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->dG, ctx->hG.data(), sizeof(double) * ctx->hG.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->dglist, ctx->hglist.data(), sizeof(int) * ctx->hglist.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->dgcount, ctx->hgcount.data(), sizeof(int) * ctx->hgcount.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, "mbd_set_geometry", e);
    return MBD_OK;
}

PeriodicBufs periodic_bufs(mbd_ctx *ctx) {
    return PeriodicBufs{ctx->cell, ctx->nk, ctx->nG, ctx->maxG, ctx->dkq, ctx->dG, ctx->dglist, ctx->dgcount, ctx->dS};
}

// Host preparation of a periodic geometry: cell inverse and reciprocal vectors, Ewald
// parameters, Monkhorst-Pack Bloch vectors and the reciprocal vectors of each.
struct PeriodicSetup {
    CellGeom cell{};
    int nk = 0, nG = 0, maxG = 0;
    std::vector<double> kq, G;
    std::vector<int> glist, gcount;
    std::string msg;
};

int periodic_setup(const mbd_options &o, const double *A, const int *grid, PeriodicSetup &ps) {
    const double pi = 3.141592653589793238462643383279502884;
    for (int e = 0; e < 9; ++e)
        if (!std::isfinite(A[e])) { ps.msg = "non-finite lattice"; return MBD_ERR_INPUT; }
    for (int c = 0; c < 3; ++c)
        if (grid[c] < 1 || grid[c] > 64) { ps.msg = "k_grid entries must lie in 1..64"; return MBD_ERR_INPUT; }
    CellGeom &c = ps.cell;
    for (int e = 0; e < 9; ++e) c.A[e] = A[e];
    const double co[9] = {A[4] * A[8] - A[5] * A[7], -(A[3] * A[8] - A[5] * A[6]), A[3] * A[7] - A[4] * A[6],
                          -(A[1] * A[8] - A[2] * A[7]), A[0] * A[8] - A[2] * A[6], -(A[0] * A[7] - A[1] * A[6]),
                          A[1] * A[5] - A[2] * A[4], -(A[0] * A[5] - A[2] * A[3]), A[0] * A[4] - A[1] * A[3]};
    const double det = A[0] * co[0] + A[1] * co[1] + A[2] * co[2];
    if (!(std::fabs(det) > 1e-12)) { ps.msg = "singular lattice"; return MBD_ERR_INPUT; }
    for (int e = 0; e < 3; ++e)
        for (int k = 0; k < 3; ++k) c.Ainv[3 * e + k] = co[3 * k + e] / det;   // (A^{-1})_{ek}
    for (int k = 0; k < 3; ++k)
        for (int e = 0; e < 3; ++e) c.B[3 * k + e] = 2.0 * pi * c.Ainv[3 * e + k];
    c.vol = std::fabs(det);
    double g = o.ewald_gamma, rc = o.real_cutoff, kc = o.recip_cutoff;
    if (!(g > 0.0)) g = rc > 0.0 ? 6.0 / rc : 2.5 / std::cbrt(c.vol);
    if (!(rc > 0.0)) rc = 6.0 / g;
    if (!(kc > 0.0)) kc = 10.0 * g;
    c.gamma = g;
    c.rc = rc;
    c.kc = kc;
    auto norm = [](const double *v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); };
    // Monkhorst-Pack: kappa_c = (2m - n_c - 1)/(2 n_c), q = kappa B
    ps.nk = grid[0] * grid[1] * grid[2];
    double qmax = 0.0;
    for (int m0 = 1; m0 <= grid[0]; ++m0)
        for (int m1 = 1; m1 <= grid[1]; ++m1)
            for (int m2 = 1; m2 <= grid[2]; ++m2) {
                const double kap[3] = {(2.0 * m0 - grid[0] - 1) / (2.0 * grid[0]),
                                       (2.0 * m1 - grid[1] - 1) / (2.0 * grid[1]),
                                       (2.0 * m2 - grid[2] - 1) / (2.0 * grid[2])};
                double q[3];
                for (int e = 0; e < 3; ++e) q[e] = kap[0] * c.B[e] + kap[1] * c.B[3 + e] + kap[2] * c.B[6 + e];
                for (int e = 0; e < 3; ++e) ps.kq.push_back(q[e]);
                qmax = std::max(qmax, norm(q));
            }
    // every G = m B with |G + q| < kc for some q: |G| < kc + qmax, |m_c| <= (kc + qmax)|a_c|/(2 pi)
    const double gr = kc + qmax;
    int mm[3];
    for (int k = 0; k < 3; ++k) mm[k] = static_cast<int>(std::floor(gr * norm(c.A + 3 * k) / (2.0 * pi))) + 1;
    const long long box = (2LL * mm[0] + 1) * (2LL * mm[1] + 1) * (2LL * mm[2] + 1);
    if (box > 20000000LL) { ps.msg = "reciprocal cutoff too large for this cell"; return MBD_ERR_INPUT; }
    for (int m0 = -mm[0]; m0 <= mm[0]; ++m0)
        for (int m1 = -mm[1]; m1 <= mm[1]; ++m1)
            for (int m2 = -mm[2]; m2 <= mm[2]; ++m2) {
                double G[3];
                for (int e = 0; e < 3; ++e) G[e] = m0 * c.B[e] + m1 * c.B[3 + e] + m2 * c.B[6 + e];
                if (norm(G) < gr) for (int e = 0; e < 3; ++e) ps.G.push_back(G[e]);
            }
    ps.nG = static_cast<int>(ps.G.size() / 3);
    std::vector<std::vector<int>> lists(ps.nk);
    for (int k = 0; k < ps.nk; ++k)
        for (int gi = 0; gi < ps.nG; ++gi) {
            double kv[3];
            for (int e = 0; e < 3; ++e) kv[e] = ps.G[3 * gi + e] + ps.kq[3 * k + e];
            const double kk = norm(kv);
            if (kk < kc && kk > 1e-12) lists[k].push_back(gi);
        }
    ps.maxG = 1;
    for (auto &l : lists) ps.maxG = std::max(ps.maxG, static_cast<int>(l.size()));
    ps.glist.assign(static_cast<size_t>(ps.nk) * ps.maxG, 0);
    ps.gcount.assign(ps.nk, 0);
    for (int k = 0; k < ps.nk; ++k) {
        ps.gcount[k] = static_cast<int>(lists[k].size());
        for (size_t t = 0; t < lists[k].size(); ++t) ps.glist[static_cast<size_t>(k) * ps.maxG + t] = lists[k][t];
    }
    if (ps.nG == 0) ps.nG = 1, ps.G.assign(3, 0.0);   // keeps the device arrays non-empty
    return MBD_OK;
}

struct Inputs {
    const double *R, *a0ref, *c6ref, *rref, *ratio;
};
struct Outputs {
    double *energy, *grad_coords, *grad_params, *alpha_scs;   // device pointers or null
};

AtomBufs atom_bufs(mbd_ctx *ctx, const Inputs &in) {
    return AtomBufs{ctx->N, ctx->nf1, in.R, in.a0ref, in.c6ref, in.rref, in.ratio,
                    ctx->da0, ctx->dom, ctx->drv, ctx->dalu, ctx->dsigu, ctx->dabar,
                    ctx->dabar0, ctx->dc6bar, ctx->dombar, ctx->drbar, ctx->du, ctx->dwu};
}

// Gradient passes (Sec. 2.4) from the state of the last forward evaluation: the MBD
// pair pass on Q^{-1/2}, the chain through the screened parameters, the adjoint solves
// V = A^{-1} H with the kept factors, the SCS pair pass and the TS chain.  Outputs are
// scaled by *grad_energy (device scalar) when it is given.
void backward_passes(mbd_ctx *ctx, cudaStream_t s, const AtomBufs &b, const double *grad_energy,
                     double *grad_coords, double *grad_params) {
    const long long ld = ctx->ld, mat = ld * ld, xs = 3 * ld;
    const double beta = ctx->opt.beta, a = ctx->opt.a;
    MbdGradOut go{ctx->dgomb, ctx->dgab0, ctx->dgrb, ctx->dgR};
    mbd_grad_pass(b, beta, a, ctx->Zlast, ld, ctx->zscale, go, s, ctx->tq_valid ? ctx->dtq : nullptr);
    if (ctx->opt.scs_mode == MBD_SCS_NL) {   // MBD-NL: only the chain through Eqs. mbd-nl-*
        if (grad_params) nl_chain(b, go, grad_energy, grad_params, s);
        if (grad_coords) scale_copy(ctx->dgR, 3 * ctx->N, grad_energy, grad_coords, s);
        return;
    }
    const bool fp64 = fp64_path(ctx->opt.precision);
    chain_screen(b, go, ctx->dh, ctx->dga0, ctx->dgrv, fp64 ? ctx->dV : ctx->dB, ld, xs, s);
    cudaMemsetAsync(ctx->dgom, 0, sizeof(double) * ctx->N, s);
    if (fp64)
        chol_solve3_f64(ctx->dM, ld, mat, ctx->nf1, ctx->ddinv, ctx->dV, ctx->dB, xs, s);
    else
        refine_solve3(ctx->dM, ctx->sM, ctx->sdinv, ld, ctx->n, ctx->nf1, ctx->dB, ctx->dV, ctx->swork,
                      kAdjointRefineSteps, s);
    scs_grad_pass(b, beta, a, ctx->dX, ctx->dV, xs, ctx->dga0, ctx->dgom, ctx->dgrv, ctx->dgR,
                  fp64 ? nullptr : ctx->sgrad32, s);
    if (grad_params) ts_chain(b, ctx->dga0, ctx->dgom, ctx->dgrv, grad_energy, grad_params, s);
    if (grad_coords) scale_copy(ctx->dgR, 3 * ctx->N, grad_energy, grad_coords, s);
}

int read_status(mbd_ctx *ctx, cudaStream_t s, const char *origin) {
    int st = 0;
    MBD_CUDA(cudaMemcpyAsync(&st, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s), origin);
    MBD_CUDA(cudaStreamSynchronize(s), origin);
    MBD_CUDA(cudaGetLastError(), origin);
    if (st & ST_INPUT) return fail(ctx, MBD_ERR_INPUT, origin, "non-finite or non-positive input, or coincident atoms");
    if (st & ST_SCS_NOT_PD)
        return fail(ctx, MBD_ERR_SCS_NOT_PD, origin, "screening matrix alpha^-1 + T^scs is not positive definite");
    if (st & ST_NEG_ALPHA)
        return fail(ctx, MBD_ERR_SCS_NEG_ALPHA, origin, "screened static polarizability or C6 is not positive");
    return MBD_OK;
}


// Operand set of one matrix in the mixed modes: FP32 values and, for BF16x3, hi/lo.
struct MixMat {
    float *f;
    void *h, *l;
    const void *op0(bool split) const { return split ? static_cast<const void *>(h) : static_cast<const void *>(f); }
    const void *op1(bool split) const { return split ? static_cast<const void *>(l) : static_cast<const void *>(f); }
};

// The matrix of one mixed-precision matrix function and where its results go: Q (FP64,
// symmetric, ld x ld, valid n x n, decoupled padding), the FP64 workspaces V and W (ld^2
// doubles each) and VT (ld^2 doubles), the FP64 output Zd ~ Q^{-1/2}, and (if tq is not NULL)
// the traces of the first N diagonal 3x3 blocks of Q^{1/2}, second order in the error of Zd.
struct MixProblem {
    const double *Q;
    long long ld;
    int n;
    double *V, *W, *VT, *Zd;
    double *tq;
};

// Mixed-precision coupled Newton-Schulz (same scaled steps as the FP64 loop) on the
// tensor cores, stopped at the precision floor, then the FP64 correction:
// Zd = Z/sqrt(s) ~ Q^{-1/2}, V = Q Zd, W = Zd V, E = (3 Tr V - sum V o W)/4 - 3/2 sum w.
// The FP32 and split-part buffers of the context hold the iteration (ld^2 elements each).
int newton_schulz_mixed(mbd_ctx *ctx, cudaStream_t s, const MixProblem &pr, double sc, double lbound, double ubound,
                        double *energy_out, std::vector<Span> &spans, cudaEvent_t &e_corr) {
    const long long ld = pr.ld;
    const int n = pr.n, N = ctx->N, M = static_cast<int>(ld);
    const int kind = ctx->opt.precision == MBD_PREC_TF32 ? 0 : (ctx->opt.precision == MBD_PREC_BF16X3 ? 1 : 2);
    const bool split = kind != 0;
    const double nd = static_cast<double>(n);
    const double flops_full = 2.0 * nd * nd * nd, flops_sym = nd * nd * (nd + 1.0);
    MixMat Y{ctx->fY, ctx->hY[0], ctx->hY[1]}, Z{ctx->fZ, ctx->hZ[0], ctx->hZ[1]};
    MixMat Y2{ctx->fY2, ctx->hY2[0], ctx->hY2[1]}, Z2{ctx->fZ2, ctx->hZ2[0], ctx->hZ2[1]};
    MixMat P{ctx->fP, ctx->hP[0], ctx->hP[1]}, PT{ctx->fPT, ctx->hPT[0], ctx->hPT[1]};
    mixed_init(kind, pr.Q, ld, 1.0 / sc, Y.f, split ? Y.h : nullptr, Y.l, Z.f, Z.h, Z.l, s);
    // K stages per tensor-memory accumulation: the option, or the kind's default (BF16x3: 8,
    // i.e. 512 products per FP32 sum in tensor memory; TF32 and TF32x3: 2, i.e. 64 products)
    const int cstages = ctx->opt.tc_chunk_stages > 0 ? ctx->opt.tc_chunk_stages : (kind == 1 ? 8 : 2);
    // the correction's TF32x3 products keep short accumulations whatever the iteration's kind
    constexpr int kCorrectionChunk = 2;
    auto tc = [&](const TcOperands &op, TcArgs g, double flops) -> int {
        Span sp;
        sp.flops = flops;
        g.chunk_stages = cstages;
        mark(ctx, s, sp.a);
        const cudaError_t e = tc_gemm(kind, op, g, s);
        mark(ctx, s, sp.b);
        if (ctx->profiling) spans.push_back(sp);
        return e == cudaSuccess ? MBD_OK : cuda_fail(ctx, "newton_schulz_tc", e);
    };
    double *resid_dev = ctx->dscal + 2;
    double resid = 0.0, prev = 1e300;
    bool floor_reached = false;
    int it = 0;
    for (; it < ctx->opt.ns_max_iter; ++it) {
        MixMat Pk = Y, PTk = Y;   // P_0 = Y_0 (symmetric)
        if (it > 0) {
            MBD_CUDA(cudaMemsetAsync(resid_dev, 0, sizeof(double), s), "newton_schulz_tc");
            TcOperands op{Z.op0(split), Z.op1(split), Y.op0(split), Y.op1(split), ld, ld};
            TcArgs g{M, M, M, 1.f, 0.f, nullptr, ld, split ? nullptr : P.f, split ? P.h : nullptr,
                     split ? P.l : nullptr, split ? nullptr : PT.f, split ? PT.h : nullptr, split ? PT.l : nullptr,
                     resid_dev, n, 0, ctx->dstatus};
            int rc = tc(op, g, flops_full);   // P = Z Y (and its transpose), resid = |I - P|_F^2
            if (rc) return rc;
            Pk = P;
            PTk = PT;
            double r2 = 0.0;
            MBD_CUDA(cudaMemcpyAsync(&r2, resid_dev, sizeof(double), cudaMemcpyDeviceToHost, s), "newton_schulz_tc");
            MBD_CUDA(cudaStreamSynchronize(s), "newton_schulz_tc");
            resid = std::sqrt(r2);
            if (!std::isfinite(resid) || resid > 2.0 * std::sqrt(nd) + 1.0) {
                ctx->ns_iter = it;
                ctx->ns_resid = resid;
                return fail(ctx, MBD_ERR_NEG_EIGENVALUE, "newton_schulz_tc",
                            "Q has a non-positive eigenvalue (polarization catastrophe)");
            }
        }
        // The tensor-core phase ends at its precision floor (ns::mixed_last).
        const bool last = it > 0 && ns::mixed_last(resid, prev, ctx->opt.ns_tol, kMixedFloor * std::sqrt(nd));
        const ns::Coeffs cf = ns::step(lbound, ubound, last);
        const double c1 = cf.c1, c3 = cf.c3;
        {   // Y' = c1 Y + c3 Y P = NT(Y, P^T): symmetric
            TcOperands op{Y.op0(split), Y.op1(split), PTk.op0(split), PTk.op1(split), ld, ld};
            TcArgs g{M, M, M, static_cast<float>(c3), static_cast<float>(c1), Y.f, ld, Y2.f,
                     split ? Y2.h : nullptr, split ? Y2.l : nullptr, nullptr, nullptr, nullptr, nullptr, 0, 2,
                     ctx->dstatus};
            int rc = tc(op, g, flops_sym);
            if (rc) return rc;
        }
        if (it == 0) {
            mixed_axpby_identity(kind, Y.f, ld, static_cast<float>(c1), static_cast<float>(c3), Z2.f,
                                 split ? Z2.h : nullptr, Z2.l, s);
        } else {   // Z' = c1 Z + c3 P Z = NT(P, Z): symmetric
            TcOperands op{Pk.op0(split), Pk.op1(split), Z.op0(split), Z.op1(split), ld, ld};
            TcArgs g{M, M, M, static_cast<float>(c3), static_cast<float>(c1), Z.f, ld, Z2.f,
                     split ? Z2.h : nullptr, split ? Z2.l : nullptr, nullptr, nullptr, nullptr, nullptr, 0, 2,
                     ctx->dstatus};
            int rc = tc(op, g, flops_sym);
            if (rc) return rc;
        }
        std::swap(Y, Y2);
        std::swap(Z, Z2);
        if (it > 0) prev = resid;
        if (last) {
            floor_reached = true;
            ++it;
            break;
        }
    }
    ctx->ns_iter = it;
    ctx->ns_resid = resid;
    int st = 0;
    MBD_CUDA(cudaMemcpyAsync(&st, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s), "newton_schulz_tc");
    MBD_CUDA(cudaStreamSynchronize(s), "newton_schulz_tc");
    if (st & ST_TC_TIMEOUT) return fail(ctx, MBD_ERR_CUDA, "newton_schulz_tc", "tensor-core GEMM wait timed out");
    if (!floor_reached) return fail(ctx, MBD_ERR_NOT_CONVERGED, "newton_schulz_tc", "iteration cap reached");
    // ---- correction ----
    // With Zs ~ (Q/s)^{-1/2} (FP32 values of the iteration), Vs = (Q/s) Zs, Ws = Zs Vs:
    // Tr Q^{1/2} ~ sqrt(s) (3 Tr Vs - sum Vs o Ws)/2, second order in the error of Zs.
    // Tr Vs = sum (Q/s) o Zs is an exact FP64 dot.  Vs and Ws are FP64 sums of exact
    // diagonal scalings and TF32x3 tensor-core products of the off-diagonal parts (no
    // accumulator mixes a dominant term with many small ones; chunk sums in FP32 with
    // round-to-nearest), each product added once into its FP64 result.
    mark(ctx, s, e_corr);
    {
        // FP32 workspace: the iteration's matrices are free now.  Parts of offdiag(Q/s) and of
        // the full Zs feed the first product; offdiag(Zs) (reusing the Q parts) and Vs^T the
        // second.
        float *Qh = Y.f, *Ql = Y2.f, *Zs_h = P.f, *Zs_l = PT.f, *Zh = Qh, *Zl = Ql;
        float *VTh = reinterpret_cast<float *>(pr.VT), *VTl = VTh + ld * ld;
        double *V64 = pr.V, *W64 = pr.W;
        const float *Zs = Z.f;
        split_tf32_f64(pr.Q, ld, 1.0 / sc, 1, Qh, Ql, s);
        split_tf32_f32(Zs, ld, 0, Zs_h, Zs_l, s);
        diag_scale_rows_f64(pr.Q, Zs, ld, 1.0 / sc, V64, s);
        auto tc64 = [&](const TcOperands &op, const TcArgs &g) -> int {   // timed like the iteration's products
            Span sp;
            sp.flops = flops_full;
            mark(ctx, s, sp.a);
            const cudaError_t e = tc_gemm(2, op, g, s);
            mark(ctx, s, sp.b);
            if (ctx->profiling) spans.push_back(sp);
            return e == cudaSuccess ? MBD_OK : cuda_fail(ctx, "correction", e);
        };
        {   // Vs += offdiag(Q/s) Zs = NT(offdiag(Q/s), Zs) (Zs symmetric)
            TcOperands op{Qh, Ql, Zs_h, Zs_l, ld, ld};
            TcArgs g{M, M, M, 1.f, 0.f, nullptr, ld, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                     0, 0, ctx->dstatus, V64, kCorrectionChunk};
            if (int rc = tc64(op, g)) return rc;
        }
        split_tf32_f64_t(V64, ld, 1.0, VTh, VTl, s);
        split_tf32_f32(Zs, ld, 1, Zh, Zl, s);
        diag_scale_rows_f32(Zs, V64, ld, W64, s);
        {   // Ws += offdiag(Zs) Vs = NT(offdiag(Zs), Vs^T)
            TcOperands op{Zh, Zl, VTh, VTl, ld, ld};
            TcArgs g{M, M, M, 1.f, 0.f, nullptr, ld, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                     0, 0, ctx->dstatus, W64, kCorrectionChunk};
            if (int rc = tc64(op, g)) return rc;
        }
        energy_correction(pr.Q, 1.0 / sc, Zs, V64, W64, ld, n, std::sqrt(sc), ctx->dombar, N,
                          ctx->dscal + 8 + 2 * 64, energy_out, ctx->dscal + 3, s);
        if (pr.tq)   // diagonal blocks of Q^{1/2}, second order in the error of Zs, for dE/d omega_bar
            block_trace_sqrt(V64, W64, ld, N, std::sqrt(sc), pr.tq, s);
    }
    double *Zd = pr.Zd;
    to_f64(Z.f, ld, 1.0 / std::sqrt(sc), Zd, s);   // Q^{-1/2} for the gradient
    double c2 = 0.0;
    MBD_CUDA(cudaMemcpyAsync(&c2, ctx->dscal + 3, sizeof(double), cudaMemcpyDeviceToHost, s), "correction");
    MBD_CUDA(cudaStreamSynchronize(s), "correction");
    int st2 = 0;
    MBD_CUDA(cudaMemcpyAsync(&st2, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s), "correction");
    MBD_CUDA(cudaStreamSynchronize(s), "correction");
    if (st2 & ST_TC_TIMEOUT) return fail(ctx, MBD_ERR_CUDA, "correction", "tensor-core GEMM wait timed out");
    ctx->corr_resid = c2;
    // The corrected energy is second order in the error of Zs: with Zs = (Q/s)^{-1/2} (I + F),
    // Ws - I ~ 2F and the error of Tr Q^{1/2}/2 is about (3/4) Tr(Q^{1/2} F^2) <= (3/16) sqrt(s) r^2.
    // The split kinds claim the 1e-6 Ha/atom bar; a Z too poor for it is reported, not used.
    if (split && !(3.0 / 16.0 * std::sqrt(sc) * c2 * c2 / (n / 3) <= ctx->opt.mixed_max_error))
        return fail(ctx, MBD_ERR_NOT_CONVERGED, "correction",
                    "the tensor-core Q^{-1/2} is too inaccurate for the energy bar (mixed_max_error)");
    ctx->Zlast = Zd;
    ctx->zscale = 1.0;
    return MBD_OK;
}

// Gradient passes of a periodic system: the MBD pair pass over Bloch vectors (atoms,
// screened parameters, lattice), the chain through the screened parameters, the adjoint
// solves on the Gamma-point factors and the SCS pass over lattice images.
void backward_periodic(mbd_ctx *ctx, cudaStream_t s, const AtomBufs &b, const double *grad_energy,
                       double *grad_coords, double *grad_params) {
    const long long ld = ctx->ld, mat = ld * ld, xs = 3 * ld;
    const double beta = ctx->opt.beta, a = ctx->opt.a;
    const PeriodicBufs pb = periodic_bufs(ctx);
    MbdGradOut go{ctx->dgomb, ctx->dgab0, ctx->dgrb, ctx->dgR};
    const bool mixed = ctx->opt.precision != MBD_PREC_FP64 && ctx->opt.precision != MBD_PREC_FP64_SPLIT;
    periodic_mbd_grad(b, pb, beta, a, ctx->Zlast, ld, ctx->zscale, go, ctx->dgc, ctx->dgA, s,
                      ctx->tq_valid ? ctx->dtq : nullptr, mixed);
    if (ctx->opt.scs_mode == MBD_SCS_NL) {   // MBD-NL: no screening to differentiate
        if (grad_params) nl_chain(b, go, grad_energy, grad_params, s);
        if (grad_coords) scale_copy(ctx->dgR, 3 * ctx->N, grad_energy, grad_coords, s);
        scale_copy(ctx->dgA, 9, grad_energy, ctx->dgAout, s);
        ctx->have_lattice_grad = true;
        return;
    }
    chain_screen(b, go, ctx->dh, ctx->dga0, ctx->dgrv, ctx->dV, ld, xs, s);
    cudaMemsetAsync(ctx->dgom, 0, sizeof(double) * ctx->N, s);
    chol_solve3_f64(ctx->dM, ld, mat, ctx->nf1, ctx->ddinv, ctx->dV, ctx->dB, xs, s);
    scs_grad_periodic(b, ctx->cell, beta, a, ctx->dX, ctx->dV, xs, ctx->dga0, ctx->dgom, ctx->dgrv, ctx->dgR,
                      ctx->dgApart, ctx->dgA, s);
    if (grad_params) ts_chain(b, ctx->dga0, ctx->dgom, ctx->dgrv, grad_energy, grad_params, s);
    if (grad_coords) scale_copy(ctx->dgR, 3 * ctx->N, grad_energy, grad_coords, s);
    scale_copy(ctx->dgA, 9, grad_energy, ctx->dgAout, s);
    ctx->have_lattice_grad = true;
}

// Periodic evaluation (Secs. 2.2 and 2.3): Gamma-point screening, Q(q) for every Bloch vector of
// the grid, batched complex coupled Newton-Schulz (FP64, 4 real GEMMs per complex product;
// the tensor-core modes take each Q(q) as its real symmetric embedding through the finite
// matrix function), E = (1/nk) sum_q 1/2 Tr Q(q)^{1/2} - 3/2 sum omega_bar.
int run_periodic(mbd_ctx *ctx, cudaStream_t s, const Inputs &in, const Outputs &out, bool want_grad) {
    if (ctx->opt.scs_mode == MBD_SCS_LEARNED)
        return fail(ctx, MBD_ERR_UNSUPPORTED, "learned_screening", "learned screening is for finite systems");
    const int N = ctx->N, n = ctx->n, nf1 = ctx->nf1, nk = ctx->nk;
    const long long ld = ctx->ld, mat = ld * ld, xs = 3 * ld;
    const double beta = ctx->opt.beta, a = ctx->opt.a;
    ctx->have_result = false;
    ctx->have_screening = false;
    ctx->have_forward = false;
    ctx->have_lattice_grad = false;
    ctx->tq_valid = false;
    ctx->ev_used = 0;
    ctx->prof = mbd_profile{};
    const long long launches0 = launch_count();
    cudaEvent_t e_start = nullptr, e_scs = nullptr, e_ns = nullptr, e_grad = nullptr;
    std::vector<Span> gemms;
    const double nd = static_cast<double>(n);
    const double flops_cplx = 8.0 * nd * nd * nd * nk;   // one complex product per Bloch vector
    // herm: Hermitian result, upper tiles only (about half the work)
    auto timed_cgemm = [&](const double *A, const double *B, const double *D, double *C, double alpha, double bt,
                           bool herm) {
        Span sp;
        sp.flops = herm ? 4.0 * nd * nd * (nd + 1.0) * nk : flops_cplx;
        mark(ctx, s, sp.a);
        cgemm_f64(A, B, D, C, ld, nk, alpha, bt, herm, s);
        mark(ctx, s, sp.b);
        if (ctx->profiling) gemms.push_back(sp);
    };
    const AtomBufs b = atom_bufs(ctx, in);
    const PeriodicBufs pb = periodic_bufs(ctx);
    NvtxStages nv;
    nv.next("mbd screening (periodic)");
    mark(ctx, s, e_start);
    MBD_CUDA(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), s), "mbd_evaluate");
    // ---- Gamma-point screening (MBD-NL: the oscillators directly) ----
    if (ctx->opt.scs_mode == MBD_SCS_NL) {
        nl_params(b, ctx->dstatus, s);
        structure_factors(b, pb, s);
    } else {
        prepare_atoms(b, ctx->dstatus, s);
        structure_factors(b, pb, s);
        build_scs_periodic(b, ctx->cell, beta, a, ctx->dM, ld, mat, ctx->dstatus, s);
        cholesky_f64(ctx->dM, ld, mat, nf1, ctx->ddinv, ctx->dstatus, s);
        init_rhs_identity(ctx->dX, ld, n, nf1, xs, s);
        chol_solve3_f64(ctx->dM, ld, mat, nf1, ctx->ddinv, ctx->dX, ctx->dB, xs, s);
        contract_screen(b, ctx->dX, ld, xs, ctx->dstatus, s);
    }
    mark(ctx, s, e_scs);
    nv.next("mbd coupled oscillators and Newton-Schulz");
    int rc = read_status(ctx, s, "screening");
    if (rc) return rc;
    ctx->have_screening = true;
    // ---- Q(q) and the spectrum bounds ----
    build_q_periodic(b, pb, beta, a, ctx->dQ, ld, n, ctx->dstatus, s);
    cmax_abs_rowsum(ctx->dQ, ld, nk, ctx->dscal + 1, s);
    double sc = 0.0;
    MBD_CUDA(cudaMemcpyAsync(&sc, ctx->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, s), "newton_schulz");
    rc = read_status(ctx, s, "coupled_oscillator_matrix");
    if (rc) return rc;
    if (!(sc > 0.0) || !std::isfinite(sc)) return fail(ctx, MBD_ERR_INPUT, "newton_schulz", "invalid Q scale");
    double *energy_out = out.energy ? out.energy : ctx->dscal;
    std::vector<Span> tc_spans;
    if (!fp64_path(ctx->opt.precision)) {
        // ---- mixed modes: each Hermitian Q(q) as its real symmetric embedding [[Re, -Im],
        // [Im, Re]] (the same spectrum, twice) through the finite mixed-precision matrix function:
        // tensor-core iteration with its own scale and bounds, FP64 correction of the energy ----
        cudaEvent_t e_corr = nullptr;
        const long long lde = ctx->lde;
        const int ne = 2 * n, lzs = std::min(kLanczosSteps, static_cast<int>(lde));
        int it_max = 0;
        double res_max = 0.0, corr_max = 0.0, sc_max = 0.0;
        std::vector<double> lzk(2 * lzs);
        for (int k = 0; k < nk; ++k) {
            embed_hermitian(ctx->dQ, ld, n, k, ctx->eM, lde, s);
            max_abs_rowsum(ctx->eM, lde, static_cast<int>(lde), ctx->dscal + 1, s);
            double sk = 0.0;
            MBD_CUDA(cudaMemcpyAsync(&sk, ctx->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, s), "newton_schulz");
            lanczos_coefficients_f32(ctx->eM, ctx->fY, lde, lzs, ctx->eV, ctx->dscal + 8, s);
            MBD_CUDA(cudaMemcpyAsync(lzk.data(), ctx->dscal + 8, sizeof(double) * 2 * lzs, cudaMemcpyDeviceToHost, s),
                     "newton_schulz");
            MBD_CUDA(cudaStreamSynchronize(s), "newton_schulz");
            if (!(sk > 0.0) || !std::isfinite(sk)) return fail(ctx, MBD_ERR_INPUT, "newton_schulz", "invalid Q scale");
            double lo = 0.0, hi = sk;
            {
                std::vector<double> da, db;
                for (int j = 0; j < lzs; ++j) {
                    da.push_back(lzk[2 * j]);
                    if (j + 1 < lzs) db.push_back(lzk[2 * j + 1]);
                    if (!(lzk[2 * j + 1] > 1e-14 * sk)) break;
                }
                db.resize(da.empty() ? 0 : da.size() - 1);
                if (!da.empty()) tridiag_extremes(da, db, lo, hi);
            }
            double ub = 1.0;
            if (std::isfinite(hi) && hi > 0.0 && 1.05 * hi < sk) {
                sk = 1.05 * hi;
                ub = 1.05;
            }
            double lb = ns::lower_estimate(lo, sk);   // an estimate (ns_schedule.h)
            // Re Tr (Q(q_k)^{1/2})_ii: the first N diagonal blocks of M_k^{1/2}, into row k of dlzw
            const MixProblem pr{ctx->eM, lde, ne, ctx->eV, ctx->eW, ctx->eVT, ctx->eZ,
                                ctx->dlzw + static_cast<long long>(k) * N};
            const int rk = newton_schulz_mixed(ctx, s, pr, sk, lb, ub, ctx->dcoef + k, tc_spans, e_corr);
            if (rk) return rk;
            extract_hermitian(ctx->eZ, lde, n, ctx->dZ, ld, k, s);
            it_max = std::max(it_max, ctx->ns_iter);
            res_max = std::max(res_max, ctx->ns_resid);
            corr_max = std::max(corr_max, ctx->corr_resid);
            sc_max = std::max(sc_max, sk);
        }
        ctx->ns_iter = it_max;
        ctx->ns_resid = res_max;
        ctx->corr_resid = corr_max;
        ctx->ns_scale = sc_max;
        periodic_mixed_energy(ctx->dcoef, nk, ctx->dombar, N, energy_out, s);
        mean_rows(ctx->dlzw, nk, N, ctx->dtq, s);   // (1/nk) sum_q Re Tr (Q(q)^{1/2})_ii
        ctx->tq_valid = true;
        ctx->Zlast = ctx->dZ;
        ctx->zscale = 1.0;
    } else {
    const int lz_steps = std::min(kLanczosSteps, static_cast<int>(2 * ld));
    clanczos_coefficients(ctx->dQ, ld, nk, lz_steps, ctx->dlzw, ctx->dcoef, s);
    std::vector<double> lz(static_cast<size_t>(nk) * 2 * lz_steps);
    MBD_CUDA(cudaMemcpyAsync(lz.data(), ctx->dcoef, sizeof(double) * lz.size(), cudaMemcpyDeviceToHost, s),
             "newton_schulz");
    MBD_CUDA(cudaStreamSynchronize(s), "newton_schulz");
    double th_min = 1e300, th_max = 0.0;
    for (int k = 0; k < nk; ++k) {
        std::vector<double> da, db;
        const double *c = lz.data() + static_cast<size_t>(k) * 2 * lz_steps;
        for (int j = 0; j < lz_steps; ++j) {
            da.push_back(c[2 * j]);
            if (!(c[2 * j + 1] > 1e-14 * sc)) break;
            if (j + 1 < lz_steps) db.push_back(c[2 * j + 1]);
        }
        db.resize(da.empty() ? 0 : da.size() - 1);
        double lo = 0.0, hi = sc;
        if (!da.empty()) tridiag_extremes(da, db, lo, hi);
        th_min = std::min(th_min, lo);
        th_max = std::max(th_max, hi);
    }
    double ubound = 1.0;
    if (std::isfinite(th_max) && th_max > 0.0 && 1.05 * th_max < sc) {
        sc = 1.05 * th_max;
        ubound = 1.05;
    }
    ctx->ns_scale = sc;
    // the smallest over all Bloch vectors; an estimate, which may lie above the true bound
    // (that costs steps only, ns_schedule.h)
    double lbound = ns::lower_estimate(th_min, sc, 0.5);
    const double ss = std::sqrt(sc);
    // ---- batched complex coupled Newton-Schulz (same scaled steps as the finite path) ----
    double *Y = ctx->dQ, *Z = ctx->dZ, *P = ctx->dP, *Y2 = ctx->dY2, *Z2 = ctx->dZ2;
    cscale(Y, ld, nk, 1.0 / sc, s);
    cset_identity(Z, ld, nk, s);
    bool converged = false;
    double resid = 0.0;
    int it = 0;
    for (; it < ctx->opt.ns_max_iter; ++it) {
        const double *Pk = Y;
        if (it > 0) {
            timed_cgemm(Z, Y, nullptr, P, 1.0, 0.0, false);   // P = Z Y: not Hermitian in floating point
            Pk = P;
        }
        cfrob_dev_identity(Pk, ld, n, nk, ctx->dscal + 2, s);
        double r2 = 0.0;
        MBD_CUDA(cudaMemcpyAsync(&r2, ctx->dscal + 2, sizeof(double), cudaMemcpyDeviceToHost, s), "newton_schulz");
        MBD_CUDA(cudaStreamSynchronize(s), "newton_schulz");
        resid = std::sqrt(r2);
        if (!std::isfinite(resid) || resid > 2.0 * std::sqrt(nd * nk) + 1.0) {
            ctx->ns_iter = it;
            ctx->ns_resid = resid;
            return fail(ctx, MBD_ERR_NEG_EIGENVALUE, "newton_schulz",
                        "Q(q) has a non-positive eigenvalue (polarization catastrophe)");
        }
        const bool last = resid < ctx->opt.ns_tol;
        const ns::Coeffs cf = ns::step(lbound, ubound, last);
        const double c1 = cf.c1, c3 = cf.c3;
        timed_cgemm(Y, Pk, Y, Y2, c3, c1, kHermitianNs);   // Y' = c1 Y + c3 Y P (Hermitian: Y Z Y)
        if (it == 0) caxpby_identity(Z2, Pk, ld, nk, c1, c3, s);
        else timed_cgemm(Pk, Z, Z, Z2, c3, c1, kHermitianNs);   // Z' = c1 Z + c3 P Z (Hermitian: Z Y Z)
        std::swap(Y, Y2);
        std::swap(Z, Z2);
        if (last) {
            converged = true;
            ++it;
            break;
        }
    }
    ctx->ns_iter = it;
    ctx->ns_resid = resid;
    if (!converged) return fail(ctx, MBD_ERR_NOT_CONVERGED, "newton_schulz", "iteration cap reached");
    energy_trace_periodic(Y, ld, n, nk, ctx->dombar, N, ss, energy_out, s);
    ctx->Zlast = Z;
    ctx->zscale = 1.0 / ss;
    }
    mark(ctx, s, e_ns);
    nv.next("mbd gradient");
    if (want_grad) backward_periodic(ctx, s, b, nullptr, out.grad_coords, out.grad_params);
    if (out.alpha_scs)
        MBD_CUDA(cudaMemcpyAsync(out.alpha_scs, ctx->dabar0, sizeof(double) * N, cudaMemcpyDeviceToDevice, s),
                 "outputs");
    mark(ctx, s, e_grad);
    MBD_CUDA(cudaStreamSynchronize(s), "mbd_evaluate");
    MBD_CUDA(cudaGetLastError(), "mbd_evaluate");
    ctx->prof.launches = static_cast<int>(launch_count() - launches0);
    if (ctx->profiling) {
        mbd_profile &p = ctx->prof;
        p.gemm_launches = 4 * static_cast<int>(gemms.size());
        for (const Span &sp : gemms) {
            p.gemm_ms += span_ms(sp.a, sp.b);
            p.gemm_flops += sp.flops;
        }
        p.tc_launches = static_cast<int>(tc_spans.size());
        for (const Span &sp : tc_spans) {
            p.tc_ms += span_ms(sp.a, sp.b);
            p.tc_flops += sp.flops;
        }
        p.screening_ms = span_ms(e_start, e_scs);
        p.screening_flops = ctx->opt.scs_mode == MBD_SCS_NL ? 0.0 : nf1 * nd * nd * nd / 3.0;
        p.newton_schulz_ms = span_ms(e_scs, e_ns);
        p.gradient_ms = span_ms(e_ns, e_grad);
        p.total_ms = span_ms(e_start, e_grad);
    }
    ctx->have_result = true;
    ctx->have_forward = true;
    ++ctx->eval_count;
    return MBD_OK;
}

int run(mbd_ctx *ctx, cudaStream_t s, const Inputs &in, const Outputs &out, bool want_grad) {
    if (ctx->periodic) return run_periodic(ctx, s, in, out, want_grad);
    const int N = ctx->N, n = ctx->n, nf1 = ctx->nf1;
    const long long ld = ctx->ld, mat = ld * ld, xs = 3 * ld;
    const double beta = ctx->opt.beta, a = ctx->opt.a;
    ctx->have_result = false;
    ctx->have_screening = false;
    ctx->tq_valid = false;
    ctx->ev_used = 0;
    ctx->prof = mbd_profile{};
    const long long launches0 = launch_count();
    cudaEvent_t e_start = nullptr, e_scs = nullptr, e_ns = nullptr, e_grad = nullptr, e_corr = nullptr;
    std::vector<Span> gemms, tc_spans;
    cudaError_t split_err = cudaSuccess;   // first launch error of the split FP64 GEMM
    auto timed_gemm = [&](const GemmArgs &g, double flops) {
        Span sp;
        sp.flops = flops;
        mark(ctx, s, sp.a);
        if (ctx->opt.precision == MBD_PREC_FP64_SPLIT) {
            const cudaError_t e = gemm_f64_split(g.trans_b, g.mode, g.M, g.N, g.K, g.alpha, g.A, g.lda, g.B, g.ldb,
                                                 g.beta, g.D, g.ldd, g.C, g.ldc, ctx->dsplit, ctx->dstatus, s);
            if (e != cudaSuccess && split_err == cudaSuccess) split_err = e;
        } else {
            gemm_f64(g, s);
        }
        mark(ctx, s, sp.b);
        if (ctx->profiling) gemms.push_back(sp);
    };
    const double nd = static_cast<double>(ctx->n);
    const double flops_full = 2.0 * nd * nd * nd, flops_sym = nd * nd * (nd + 1.0);
    ctx->have_forward = false;
    const AtomBufs b = atom_bufs(ctx, in);
    NvtxStages nv;
    nv.next("mbd screening");
    mark(ctx, s, e_start);
    MBD_CUDA(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), s), "mbd_evaluate");
    // ---- screening (Sec. 2.3) ----
    const bool learned = ctx->opt.scs_mode == MBD_SCS_LEARNED && !ctx->force_plain;
    ctx->last_learned = false;
    if (learned) {   // model prediction of alpha_bar(iu) in place of the Dyson solves
        if (out.grad_params)
            return fail(ctx, MBD_ERR_UNSUPPORTED, "learned_screening",
                        "learned screening gives energies and coordinate gradients only");
        if (ctx->members < 1) return fail(ctx, MBD_ERR_STATE, "learned_screening", "no model set");
        int rc0 = ensure_learned(ctx);
        if (rc0) return rc0;
        prepare_atoms(b, ctx->dstatus, s);
        scs_features(N, 1, ctx->doffs, in.R, in.a0ref, in.c6ref, in.rref, in.ratio, ctx->dfeat, ctx->dmoments, s);
        const cudaError_t ef = mlp_forward(N, ctx->members, ctx->dfeat, ctx->dmeanstd, ctx->dmeanstd + kLF, ctx->dmodel,
                                           ctx->dYl, want_grad ? ctx->dzc : nullptr, s, nullptr, ctx->dpacked);
        if (ef != cudaSuccess) return cuda_fail(ctx, "learned_screening", ef);
        learned_alpha(N, ctx->members, nf1, ctx->dalu, ctx->dYl, ctx->dabar, ctx->dspread, s);
        screened_params(b, ctx->dstatus, s);
    } else if (ctx->opt.scs_mode == MBD_SCS_NL) {   // MBD-NL: oscillators set directly, no screening
        nl_params(b, ctx->dstatus, s);
    } else {
        prepare_atoms(b, ctx->dstatus, s);
        build_scs(b, beta, a, ctx->dM, ld, mat, ctx->dstatus, s);
        if (fp64_path(ctx->opt.precision)) {
            cholesky_f64(ctx->dM, ld, mat, nf1, ctx->ddinv, ctx->dstatus, s);
            init_rhs_identity(ctx->dX, ld, n, nf1, xs, s);
            chol_solve3_f64(ctx->dM, ld, mat, nf1, ctx->ddinv, ctx->dX, ctx->dB, xs, s);
        } else {   // FP32 factors, FP64-refined solutions
            MBD_CUDA(cholesky_f32_from_f64(ctx->dM, ctx->sM, ld, nf1, ctx->sdinv, ctx->spanel, ctx->dstatus, s),
                     "screening");
            init_rhs_identity(ctx->dB, ld, n, nf1, xs, s);
            refine_solve3(ctx->dM, ctx->sM, ctx->sdinv, ld, n, nf1, ctx->dB, ctx->dX, ctx->swork, kRefineSteps, s);
        }
        contract_screen(b, ctx->dX, ld, xs, ctx->dstatus, s);
    }
    mark(ctx, s, e_scs);
    nv.next("mbd coupled oscillators and Newton-Schulz");
    int rc = read_status(ctx, s, "screening");
    if (rc) return rc;
    ctx->have_screening = true;
    // ---- coupled-oscillator matrix and its square roots (Sec. 2.1) ----
    build_q(b, beta, a, ctx->dQ, ld, ctx->dstatus, s);
    max_abs_rowsum(ctx->dQ, ld, static_cast<int>(ld), ctx->dscal + 1, s);
    double sc = 0.0;
    MBD_CUDA(cudaMemcpyAsync(&sc, ctx->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, s), "newton_schulz");
    MBD_CUDA(cudaStreamSynchronize(s), "newton_schulz");
    rc = read_status(ctx, s, "coupled_oscillator_matrix");
    if (rc) return rc;
    if (!(sc > 0.0) || !std::isfinite(sc)) return fail(ctx, MBD_ERR_INPUT, "newton_schulz", "invalid Q scale");
    // Lanczos estimates of the extreme eigenvalues of Q (workspace: rows of P).  The
    // largest tightens the scale s of Y0 = Q/s (Lanczos converges fast at the top of the
    // spectrum; a 5 % margin keeps Y0's spectrum inside (0, 1]).  The smallest converges
    // slowly: after 48 steps its Ritz value is 3-6 times the smallest eigenvalue of Q
    // (500-2000 atom clusters), so a quarter of it is the lower bound of the scaled
    // iteration.  A bound on either side of the true one only costs steps (see below); on the
    // spectra of those clusters a quarter takes one step fewer than a half.
    const bool short_run = !fp64_path(ctx->opt.precision) && ld <= kLanczosSmallOrder;
    const int lz_steps = std::min(short_run ? kLanczosStepsSmall : kLanczosSteps, static_cast<int>(ld));
    if (fp64_path(ctx->opt.precision))
        lanczos_coefficients(ctx->dQ, ld, lz_steps, ctx->dP, ctx->dscal + 8, s);
    else   // the bounds need a few digits; the products read an FP32 copy of Q (in the FP32 Y buffer)
        lanczos_coefficients_f32(ctx->dQ, ctx->fY, ld, lz_steps, ctx->dP, ctx->dscal + 8, s);
    std::vector<double> lz(2 * lz_steps);
    MBD_CUDA(cudaMemcpyAsync(lz.data(), ctx->dscal + 8, sizeof(double) * 2 * lz_steps, cudaMemcpyDeviceToHost, s),
             "newton_schulz");
    MBD_CUDA(cudaStreamSynchronize(s), "newton_schulz");
    double th_min = 0.0, th_max = sc;
    {
        std::vector<double> da, db;
        for (int j = 0; j < lz_steps; ++j) {
            da.push_back(lz[2 * j]);
            if (j + 1 < lz_steps) db.push_back(lz[2 * j + 1]);
            if (!(lz[2 * j + 1] > 1e-14 * sc)) break;   // invariant subspace reached
        }
        db.resize(da.size() > 0 ? da.size() - 1 : 0);
        if (!da.empty()) tridiag_extremes(da, db, th_min, th_max);
    }
    // ubound: upper bound on sqrt(eig(Z Y)) for the first step: 1 under the Gershgorin
    // scale; 1.05 after tightening by the Lanczos estimate (tolerates an underestimate
    // of the largest eigenvalue by up to 16 %).
    double ubound = 1.0;
    if (std::isfinite(th_max) && th_max > 0.0 && 1.05 * th_max < sc) {
        sc = 1.05 * th_max;
        ubound = 1.05;
    }
    ctx->ns_scale = sc;
    double lbound = ns::lower_estimate(th_min, sc);   // estimated lower bound on sqrt(eig(Z Y))
    const double ss = std::sqrt(sc);
    double *energy_out = out.energy ? out.energy : ctx->dscal;
    if (fp64_path(ctx->opt.precision)) {
        double *Y = ctx->dQ, *Z = ctx->dZ, *P = ctx->dP, *Y2 = ctx->dY2, *Z2 = ctx->dZ2;
        scale_matrix(Y, ld, 1.0 / sc, s);
        set_identity(Z, ld, s);
        const int M = static_cast<int>(ld);
        bool converged = false;
        double resid = 0.0;
        int it = 0;
        for (; it < ctx->opt.ns_max_iter; ++it) {
            // P = Z Y (not symmetric once rounding separates Z and Y; computed in full)
            const double *Pk = Y;   // Z_0 = I: P_0 = Y_0
            if (it > 0) {
                GemmArgs g{Z, Y, nullptr, P, ld, ld, 0, ld, 0, 0, 0, 0, M, M, M, 1, 1.0, 0.0, 0, 0};
                timed_gemm(g, flops_full);
                Pk = P;
            }
            frob_dev_identity(Pk, ld, n, ctx->dscal + 2, s);
            double r2 = 0.0;
            MBD_CUDA(cudaMemcpyAsync(&r2, ctx->dscal + 2, sizeof(double), cudaMemcpyDeviceToHost, s), "newton_schulz");
            MBD_CUDA(cudaStreamSynchronize(s), "newton_schulz");
            resid = std::sqrt(r2);
            if (!std::isfinite(resid) || resid > 2.0 * std::sqrt(static_cast<double>(n)) + 1.0) {
                // For positive definite Q every eigenvalue of Z Y stays in (0, 1]; leaving that
                // range means an eigenvalue of Q is not positive.
                ctx->ns_iter = it;
                ctx->ns_resid = resid;
                return fail(ctx, MBD_ERR_NEG_EIGENVALUE, "newton_schulz",
                            "Q has a non-positive eigenvalue (polarization catastrophe)");
            }
            const bool last = resid < ctx->opt.ns_tol;
            const ns::Coeffs cf = ns::step(lbound, ubound, last);   // scaled step (ns_schedule.h)
            const double c1 = cf.c1, c3 = cf.c3;
            // Y' = Y T, Z' = T Z: Y' = c1 Y + c3 Y (Z Y) and Z' = c1 Z + c3 (Z Y) Z.  Y Z Y and
            // Z Y Z are symmetric for any symmetric Y, Z, so only their upper tiles are
            // computed.  (Using P^T in place of P, i.e. Y Y Z, breaks the coupling and makes
            // rounding errors grow by about sqrt(cond Q)/2 per step.)
            GemmArgs gy{Y, Pk, Y, Y2, ld, ld, ld, ld, 0, 0, 0, 0, M, M, M, 1, c3, c1, 2, 0};
            timed_gemm(gy, flops_sym);
            if (it == 0) {
                axpby_identity(Z2, Pk, ld, c1, c3, s);
            } else {
                GemmArgs gz{Pk, Z, Z, Z2, ld, ld, ld, ld, 0, 0, 0, 0, M, M, M, 1, c3, c1, 2, 0};
                timed_gemm(gz, flops_sym);
            }
            std::swap(Y, Y2);
            std::swap(Z, Z2);
            if (last) {
                converged = true;
                ++it;
                break;
            }
        }
        ctx->ns_iter = it;
        ctx->ns_resid = resid;
        if (split_err != cudaSuccess) return cuda_fail(ctx, "newton_schulz_split", split_err);
        if (ctx->opt.precision == MBD_PREC_FP64_SPLIT) {   // tensor-core waits are bounded: check them
            int st = 0;
            MBD_CUDA(cudaMemcpyAsync(&st, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s), "newton_schulz");
            MBD_CUDA(cudaStreamSynchronize(s), "newton_schulz");
            if (st & ST_TC_TIMEOUT) return fail(ctx, MBD_ERR_CUDA, "newton_schulz_split", "tensor-core GEMM wait timed out");
        }
        if (!converged)
            return fail(ctx, MBD_ERR_NOT_CONVERGED, "newton_schulz", "iteration cap reached");
        energy_trace(Y, ld, n, ctx->dombar, N, ss, energy_out, s);
        ctx->Zlast = Z;
        ctx->zscale = 1.0 / ss;
    } else {
        const MixProblem pr{ctx->dQ, ld, n, ctx->dP, ctx->dZ2, ctx->dY2, ctx->dZ, ctx->dtq};
        rc = newton_schulz_mixed(ctx, s, pr, sc, lbound, ubound, energy_out, tc_spans, e_corr);
        if (rc) return rc;
        ctx->tq_valid = true;
    }
    mark(ctx, s, e_ns);
    nv.next("mbd gradient");
    if (learned) {
        // energy-error estimate from the adjoints h = dE/d alpha_bar(u) and the members' spread;
        // above the threshold the evaluation is redone with plain screening
        MbdGradOut go{ctx->dgomb, ctx->dgab0, ctx->dgrb, ctx->dgR};
        mbd_grad_pass(b, beta, a, ctx->Zlast, ld, ctx->zscale, go, s, ctx->tq_valid ? ctx->dtq : nullptr);
        chain_screen(b, go, ctx->dh, ctx->dga0, ctx->dgrv, ctx->dV, ld, xs, s);
        learned_estimate(N, nf1, ctx->members, ctx->opt.learned_estimate_scale, ctx->dh, ctx->dalu, ctx->dYl,
                         ctx->dscal + 5, s);
        double est = 0.0;
        MBD_CUDA(cudaMemcpyAsync(&est, ctx->dscal + 5, sizeof(double), cudaMemcpyDeviceToHost, s), "learned_screening");
        MBD_CUDA(cudaStreamSynchronize(s), "learned_screening");
        ctx->learned_est = est;
        ctx->learned_fallback = 0;
        ctx->last_learned = est <= ctx->opt.learned_max_error;
        if (!(est <= ctx->opt.learned_max_error)) {
            // the profile of the plain re-run also counts the discarded learned attempt
            const int attempt_launches = static_cast<int>(launch_count() - launches0);
            double attempt_ms = 0.0;
            if (ctx->profiling && e_start && e_ns) {
                MBD_CUDA(cudaEventSynchronize(e_ns), "learned_screening");
                attempt_ms = span_ms(e_start, e_ns);
            }
            ctx->force_plain = true;
            const int rc2 = run(ctx, s, in, out, want_grad);
            ctx->force_plain = false;
            ctx->learned_est = est;
            ctx->learned_fallback = 1;
            ctx->prof.launches += attempt_launches;
            ctx->prof.total_ms += attempt_ms;
            return rc2;
        }
        if (want_grad) {
            // dE/dR = (MBD term at fixed screened parameters, in dgR) + sum h dalpha_bar/dR through
            // the members' outputs, the network and the features
            learned_dy(N, ctx->members, nf1, ctx->dh, ctx->dabar, ctx->dYl, s);
            const cudaError_t eb = mlp_backward(N, ctx->members, ctx->dfeat, ctx->dmeanstd, ctx->dmeanstd + kLF,
                                                ctx->dmodel, ctx->dzc, ctx->dYl, ctx->dXl, nullptr, s, ctx->dpacked);
            if (eb != cudaSuccess) return cuda_fail(ctx, "learned_screening", eb);
            learned_forces(N, ctx->doffs, in.R, in.a0ref, in.rref, in.ratio, ctx->dmoments, ctx->dXl, ctx->members,
                           ctx->dadj, ctx->dgR, s);
            if (out.grad_coords) scale_copy(ctx->dgR, 3 * N, nullptr, out.grad_coords, s);
        }
    }
    // ---- gradients (Sec. 2.4) ----
    if (want_grad && !learned) backward_passes(ctx, s, b, nullptr, out.grad_coords, out.grad_params);
    if (out.alpha_scs)
        MBD_CUDA(cudaMemcpyAsync(out.alpha_scs, ctx->dabar0, sizeof(double) * N, cudaMemcpyDeviceToDevice, s),
                 "outputs");
    mark(ctx, s, e_grad);
    MBD_CUDA(cudaStreamSynchronize(s), "mbd_evaluate");
    MBD_CUDA(cudaGetLastError(), "mbd_evaluate");
    ctx->prof.launches = static_cast<int>(launch_count() - launches0);
    if (ctx->profiling) {
        mbd_profile &p = ctx->prof;
        p.gemm_launches = static_cast<int>(gemms.size());
        for (const Span &sp : gemms) {
            p.gemm_ms += span_ms(sp.a, sp.b);
            p.gemm_flops += sp.flops;
        }
        p.tc_launches = static_cast<int>(tc_spans.size());
        for (const Span &sp : tc_spans) {
            p.tc_ms += span_ms(sp.a, sp.b);
            p.tc_flops += sp.flops;
        }
        if (e_corr) p.correction_ms = span_ms(e_corr, e_ns);
        p.screening_ms = span_ms(e_start, e_scs);
        p.screening_flops = ctx->opt.scs_mode == MBD_SCS_NL
                                ? 0.0
                                : nf1 * nd * nd * nd / 3.0;   // FP64, or FP32 in the mixed modes
        p.newton_schulz_ms = span_ms(e_scs, e_ns);
        p.gradient_ms = span_ms(e_ns, e_grad);
        p.total_ms = span_ms(e_start, e_grad);
    }
    ctx->have_result = true;
    ctx->have_forward = true;
    ++ctx->eval_count;
    return MBD_OK;
}

}  // namespace

extern "C" {

int mbd_default_options(mbd_options *opt) {
    if (!opt) return MBD_ERR_INPUT;
    opt->n_freq = 15;
    opt->beta = 0.83;
    opt->a = 6.0;
    opt->precision = MBD_PREC_FP64;
    opt->ns_tol = 1e-8;
    opt->ns_max_iter = 100;
    opt->tc_chunk_stages = 0;
    opt->ewald_gamma = 0.0;
    opt->real_cutoff = 0.0;
    opt->recip_cutoff = 0.0;
    opt->scs_mode = MBD_SCS_PLAIN;
    opt->learned_max_error = 1e-6;
    opt->mixed_max_error = 1e-7;
    opt->learned_estimate_scale = 1.0;
    return MBD_OK;
}

int mbd_create(mbd_ctx **out, int cuda_device, const mbd_options *opt) {
    if (!out) return MBD_ERR_INPUT;
    *out = nullptr;
    mbd_options o;
    if (opt) o = *opt; else mbd_default_options(&o);
    if (o.n_freq < 1 || o.n_freq + 1 > kMaxFreq || !(o.beta > 0) || !(o.a > 0) || o.ns_max_iter < 1 ||
        !(o.ns_tol > 0) || o.precision < MBD_PREC_FP64 || o.precision > MBD_PREC_FP64_SPLIT || o.tc_chunk_stages < 0 ||
        (o.scs_mode != MBD_SCS_PLAIN && o.scs_mode != MBD_SCS_LEARNED && o.scs_mode != MBD_SCS_NL) ||
        !(o.learned_max_error > 0) || !(o.mixed_max_error > 0) || !(o.learned_estimate_scale > 0) ||
        !std::isfinite(o.learned_estimate_scale) || (o.scs_mode == MBD_SCS_LEARNED && o.n_freq != 15))
        return MBD_ERR_INPUT;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cuda_device < 0 || cuda_device >= ndev)
        return MBD_ERR_CUDA;
    mbd_ctx *c = new mbd_ctx();
    c->device = cuda_device;
    c->opt = o;
    c->nf1 = o.n_freq + 1;
    casimir_polder_grid(o.n_freq, c->hu, c->hwu);
    if (cudaSetDevice(cuda_device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return MBD_ERR_CUDA;
    }
    *out = c;
    return MBD_OK;
}

int mbd_destroy(mbd_ctx *ctx) {
    if (!ctx) return MBD_OK;
    cudaSetDevice(ctx->device);
    release(ctx);
    if (ctx->lslab) cudaFree(ctx->lslab);
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return MBD_OK;
}

int mbd_set_geometry(mbd_ctx *ctx, int n_atoms, const double *coords, const double *lattice,
                     const int *k_grid) {
    if (!ctx) return MBD_ERR_INPUT;
    if ((lattice == nullptr) != (k_grid == nullptr))
        return fail(ctx, MBD_ERR_INPUT, "mbd_set_geometry", "lattice and k_grid are given together or not at all");
    if (n_atoms < 1 || !coords) return fail(ctx, MBD_ERR_INPUT, "mbd_set_geometry", "need n_atoms >= 1 and coords");
    for (int k = 0; k < 3 * n_atoms; ++k)
        if (!std::isfinite(coords[k])) return fail(ctx, MBD_ERR_INPUT, "mbd_set_geometry", "non-finite coordinate");
    const bool periodic = lattice != nullptr;
    PeriodicSetup ps;
    if (periodic) {
        if (ctx->opt.precision == MBD_PREC_FP64_SPLIT)
            return fail(ctx, MBD_ERR_UNSUPPORTED, "mbd_set_geometry",
                        "periodic systems run in FP64 or in the tensor-core modes, not with split FP64 products");
        const int rc = periodic_setup(ctx->opt, lattice, k_grid, ps);
        if (rc) return fail(ctx, rc, "mbd_set_geometry", ps.msg);
    }
    MBD_CUDA(cudaSetDevice(ctx->device), "mbd_set_geometry");
    const bool realloc = (n_atoms != ctx->N) || !ctx->slab || periodic != ctx->periodic ||
                         (periodic && (ps.nk != ctx->nk || ps.nG != ctx->nG || ps.maxG != ctx->maxG));
    ctx->N = n_atoms;
    ctx->n = 3 * n_atoms;
    ctx->ld = (ctx->n + 127) / 128 * 128;   // 128: the tensor-core tile (also a multiple of 64)
    ctx->lde = (2LL * ctx->n + 127) / 128 * 128;
    ctx->nb = static_cast<int>(ctx->ld / kTile);
    ctx->hR.assign(coords, coords + 3 * n_atoms);
    ctx->periodic = periodic;
    if (periodic) {
        ctx->cell = ps.cell;
        ctx->nk = ps.nk;
        ctx->nG = ps.nG;
        ctx->maxG = ps.maxG;
        ctx->hkq = ps.kq;
        ctx->hG = ps.G;
        ctx->hglist = ps.glist;
        ctx->hgcount = ps.gcount;
    } else {
        ctx->nk = 1;
        ctx->nG = ctx->maxG = 0;
    }
    ctx->have_lattice_grad = false;
    if (realloc) {
        ctx->have_params = false;
        ctx->have_forward = false;
        int rc = allocate(ctx);
        if (rc) { ctx->have_geom = false; return rc; }
    }
    if (periodic) {
        const int rc = upload_periodic(ctx);
        if (rc) { ctx->have_geom = false; return rc; }
    }
    ctx->have_geom = true;
    ctx->have_result = false;
    return MBD_OK;
}

int mbd_set_free_atom_params(mbd_ctx *ctx, const double *alpha0_ref, const double *c6_ref,
                             const double *rvdw_ref, const double *volume_ratio) {
    if (!ctx) return MBD_ERR_INPUT;
    if (!ctx->have_geom) return fail(ctx, MBD_ERR_STATE, "mbd_set_free_atom_params", "set the geometry first");
    if (!alpha0_ref || !c6_ref || !rvdw_ref || !volume_ratio)
        return fail(ctx, MBD_ERR_INPUT, "mbd_set_free_atom_params", "null parameter array");
    const int N = ctx->N;
    ctx->ha0.assign(alpha0_ref, alpha0_ref + N);
    ctx->hc6.assign(c6_ref, c6_ref + N);
    ctx->hrr.assign(rvdw_ref, rvdw_ref + N);
    ctx->hv.assign(volume_ratio, volume_ratio + N);
    ctx->have_params = true;
    ctx->have_result = false;
    return MBD_OK;
}

int mbd_evaluate(mbd_ctx *ctx, double *energy, double *grad_coords, double *grad_lattice,
                 double *grad_params, double *alpha_scs) {
    if (!ctx) return MBD_ERR_INPUT;
    if (!ctx->have_geom || !ctx->have_params)
        return fail(ctx, MBD_ERR_STATE, "mbd_evaluate", "set the geometry and the free-atom parameters first");
    if (grad_lattice && !ctx->periodic)
        return fail(ctx, MBD_ERR_UNSUPPORTED, "mbd_evaluate", "no lattice gradient for finite systems");
    if (!energy) return fail(ctx, MBD_ERR_INPUT, "mbd_evaluate", "energy pointer is required");
    MBD_CUDA(cudaSetDevice(ctx->device), "mbd_evaluate");
    const int N = ctx->N;
    cudaStream_t s = ctx->stream;
    MBD_CUDA(cudaMemcpyAsync(ctx->dR, ctx->hR.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s), "mbd_evaluate");
    MBD_CUDA(cudaMemcpyAsync(ctx->da0ref, ctx->ha0.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_evaluate");
    MBD_CUDA(cudaMemcpyAsync(ctx->dc6ref, ctx->hc6.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_evaluate");
    MBD_CUDA(cudaMemcpyAsync(ctx->drref, ctx->hrr.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_evaluate");
    MBD_CUDA(cudaMemcpyAsync(ctx->dratio, ctx->hv.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_evaluate");
    const bool want_grad = grad_coords || grad_params || grad_lattice;
    Inputs in{ctx->dR, ctx->da0ref, ctx->dc6ref, ctx->drref, ctx->dratio};
    Outputs o{ctx->dscal, nullptr, grad_params ? ctx->dgp : nullptr, nullptr};   // gradients stay in dgR
    int rc = run(ctx, s, in, o, want_grad);
    if (rc) return rc;
    double e = 0.0;
    MBD_CUDA(cudaMemcpyAsync(&e, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, s), "mbd_evaluate");
    if (grad_coords)
        MBD_CUDA(cudaMemcpyAsync(grad_coords, ctx->dgR, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s), "mbd_evaluate");
    if (grad_params)
        MBD_CUDA(cudaMemcpyAsync(grad_params, ctx->dgp, sizeof(double) * 4 * N, cudaMemcpyDeviceToHost, s), "mbd_evaluate");
    if (alpha_scs)
        MBD_CUDA(cudaMemcpyAsync(alpha_scs, ctx->dabar0, sizeof(double) * N, cudaMemcpyDeviceToHost, s), "mbd_evaluate");
    if (grad_lattice)
        MBD_CUDA(cudaMemcpyAsync(grad_lattice, ctx->dgAout, sizeof(double) * 9, cudaMemcpyDeviceToHost, s), "mbd_evaluate");
    MBD_CUDA(cudaStreamSynchronize(s), "mbd_evaluate");
    *energy = e;
    return MBD_OK;
}

int mbd_evaluate_dev(mbd_ctx *ctx, void *stream, int n_atoms, const double *coords, const double *alpha0_ref,
                     const double *c6_ref, const double *rvdw_ref, const double *volume_ratio, double *energy,
                     double *grad_coords, double *grad_params, double *alpha_scs) {
    if (!ctx) return MBD_ERR_INPUT;
    if (!ctx->have_geom) return fail(ctx, MBD_ERR_STATE, "mbd_evaluate_dev", "set the geometry first");
    if (n_atoms != ctx->N)
        return fail(ctx, MBD_ERR_INPUT, "mbd_evaluate_dev", "n_atoms differs from the geometry's size");
    if (!coords || !alpha0_ref || !c6_ref || !rvdw_ref || !volume_ratio || !energy)
        return fail(ctx, MBD_ERR_INPUT, "mbd_evaluate_dev", "null device pointer");
    MBD_CUDA(cudaSetDevice(ctx->device), "mbd_evaluate_dev");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool want_grad = grad_coords || grad_params;
    Inputs in{coords, alpha0_ref, c6_ref, rvdw_ref, volume_ratio};
    Outputs o{energy, grad_coords, grad_params, alpha_scs};
    return run(ctx, s, in, o, want_grad);
}

int mbd_get_evaluation_count(const mbd_ctx *ctx, long long *count) {
    if (!ctx || !count) return MBD_ERR_INPUT;
    *count = ctx->eval_count;
    return MBD_OK;
}

int mbd_backward_dev(mbd_ctx *ctx, void *stream, long long evaluation, int n_atoms, const double *coords,
                     const double *alpha0_ref, const double *c6_ref, const double *rvdw_ref,
                     const double *volume_ratio, const double *grad_energy, double *grad_coords,
                     double *grad_params) {
    if (!ctx) return MBD_ERR_INPUT;
    if (!ctx->have_forward)
        return fail(ctx, MBD_ERR_STATE, "mbd_backward_dev", "no forward evaluation to differentiate");
    if (evaluation != 0 && evaluation != ctx->eval_count)
        return fail(ctx, MBD_ERR_STATE, "mbd_backward_dev",
                    "the context's last evaluation is not the one to differentiate (evaluate it again first)");
    if (ctx->last_learned)
        return fail(ctx, MBD_ERR_UNSUPPORTED, "mbd_backward_dev",
                    "the last evaluation used learned screening; request its gradients from the evaluation");
    if (n_atoms != ctx->N || !coords || !alpha0_ref || !c6_ref || !rvdw_ref || !volume_ratio)
        return fail(ctx, MBD_ERR_INPUT, "mbd_backward_dev", "inputs must match the forward evaluation");
    MBD_CUDA(cudaSetDevice(ctx->device), "mbd_backward_dev");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Inputs in{coords, alpha0_ref, c6_ref, rvdw_ref, volume_ratio};
    if (ctx->periodic) backward_periodic(ctx, s, atom_bufs(ctx, in), grad_energy, grad_coords, grad_params);
    else backward_passes(ctx, s, atom_bufs(ctx, in), grad_energy, grad_coords, grad_params);
    MBD_CUDA(cudaStreamSynchronize(s), "mbd_backward_dev");
    MBD_CUDA(cudaGetLastError(), "mbd_backward_dev");
    return MBD_OK;
}

int mbd_set_scs_model(mbd_ctx *ctx, int n_members, const void *params_fp16, const float *mean, const float *std) {
    if (!ctx) return MBD_ERR_INPUT;
    if (n_members < 1 || n_members > 64 || !params_fp16 || !mean || !std)
        return fail(ctx, MBD_ERR_INPUT, "mbd_set_scs_model", "need 1..64 members, parameters, mean and std");
    for (int k = 0; k < kLF; ++k)
        if (!(std[k] > 0.0f) || !std::isfinite(mean[k]))
            return fail(ctx, MBD_ERR_INPUT, "mbd_set_scs_model", "feature std must be positive and mean finite");
    const size_t P = static_cast<size_t>(learned_param_count()) * n_members;
    const uint16_t *src = static_cast<const uint16_t *>(params_fp16);
    ctx->hmodel.assign(src, src + P);
    ctx->hmean.assign(mean, mean + kLF);
    ctx->hstd.assign(std, std + kLF);
    ctx->members = n_members;
    ctx->model_dirty = true;
    return MBD_OK;
}

int mbd_get_learned_stats(mbd_ctx *ctx, double *estimated_error, int *fell_back) {
    if (!ctx) return MBD_ERR_INPUT;
    if (estimated_error) *estimated_error = ctx->learned_est;
    if (fell_back) *fell_back = ctx->learned_fallback;
    return MBD_OK;
}

int mbd_screen(mbd_ctx *ctx, double *alpha_iu, double *alpha_free_iu, double *c6, double *omega, double *rvdw) {
    if (!ctx) return MBD_ERR_INPUT;
    if (!ctx->have_geom || !ctx->have_params)
        return fail(ctx, MBD_ERR_STATE, "mbd_screen", "set the geometry and the free-atom parameters first");
    if (ctx->opt.scs_mode == MBD_SCS_NL)
        return fail(ctx, MBD_ERR_UNSUPPORTED, "mbd_screen", "MBD-NL has no screening step");
    MBD_CUDA(cudaSetDevice(ctx->device), "mbd_screen");
    const int N = ctx->N, n = ctx->n, nf1 = ctx->nf1;
    const long long ld = ctx->ld, mat = ld * ld, xs = 3 * ld;
    cudaStream_t s = ctx->stream;
    MBD_CUDA(cudaMemcpyAsync(ctx->dR, ctx->hR.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s), "mbd_screen");
    MBD_CUDA(cudaMemcpyAsync(ctx->da0ref, ctx->ha0.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_screen");
    MBD_CUDA(cudaMemcpyAsync(ctx->dc6ref, ctx->hc6.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_screen");
    MBD_CUDA(cudaMemcpyAsync(ctx->drref, ctx->hrr.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_screen");
    MBD_CUDA(cudaMemcpyAsync(ctx->dratio, ctx->hv.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_screen");
    const AtomBufs b = atom_bufs(ctx, Inputs{ctx->dR, ctx->da0ref, ctx->dc6ref, ctx->drref, ctx->dratio});
    ctx->have_screening = false;
    MBD_CUDA(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), s), "mbd_screen");
    prepare_atoms(b, ctx->dstatus, s);
    if (ctx->periodic) build_scs_periodic(b, ctx->cell, ctx->opt.beta, ctx->opt.a, ctx->dM, ld, mat, ctx->dstatus, s);
    else build_scs(b, ctx->opt.beta, ctx->opt.a, ctx->dM, ld, mat, ctx->dstatus, s);
    if (fp64_path(ctx->opt.precision) || ctx->periodic) {
        cholesky_f64(ctx->dM, ld, mat, nf1, ctx->ddinv, ctx->dstatus, s);
        init_rhs_identity(ctx->dX, ld, n, nf1, xs, s);
        chol_solve3_f64(ctx->dM, ld, mat, nf1, ctx->ddinv, ctx->dX, ctx->dB, xs, s);
    } else {
        MBD_CUDA(cholesky_f32_from_f64(ctx->dM, ctx->sM, ld, nf1, ctx->sdinv, ctx->spanel, ctx->dstatus, s),
                 "mbd_screen");
        init_rhs_identity(ctx->dB, ld, n, nf1, xs, s);
        refine_solve3(ctx->dM, ctx->sM, ctx->sdinv, ld, n, nf1, ctx->dB, ctx->dX, ctx->swork, kRefineSteps, s);
    }
    contract_screen(b, ctx->dX, ld, xs, ctx->dstatus, s);
    int rc = read_status(ctx, s, "mbd_screen");
    if (rc) return rc;
    ctx->have_screening = true;
    if (alpha_free_iu)
        MBD_CUDA(cudaMemcpy(alpha_free_iu, ctx->dalu, sizeof(double) * N * nf1, cudaMemcpyDeviceToHost), "mbd_screen");
    return mbd_get_scs_detail(ctx, alpha_iu, c6, omega, rvdw);
}

int mbd_get_lattice_gradient(mbd_ctx *ctx, double *grad_lattice) {
    if (!ctx || !grad_lattice) return MBD_ERR_INPUT;
    if (!ctx->periodic || !ctx->have_lattice_grad)
        return fail(ctx, MBD_ERR_STATE, "mbd_get_lattice_gradient", "no lattice gradient has been computed");
    MBD_CUDA(cudaSetDevice(ctx->device), "mbd_get_lattice_gradient");
    MBD_CUDA(cudaMemcpy(grad_lattice, ctx->dgAout, sizeof(double) * 9, cudaMemcpyDeviceToHost), "mbd_get_lattice_gradient");
    return MBD_OK;
}

int mbd_get_scs_detail(mbd_ctx *ctx, double *alpha_iu, double *c6, double *omega, double *rvdw) {
    if (!ctx) return MBD_ERR_INPUT;
    if (!ctx->have_screening) return fail(ctx, MBD_ERR_STATE, "mbd_get_scs_detail", "no screening result");
    MBD_CUDA(cudaSetDevice(ctx->device), "mbd_get_scs_detail");
    const size_t N = ctx->N;
    if (alpha_iu) MBD_CUDA(cudaMemcpy(alpha_iu, ctx->dabar, sizeof(double) * N * ctx->nf1, cudaMemcpyDeviceToHost), "mbd_get_scs_detail");
    if (c6) MBD_CUDA(cudaMemcpy(c6, ctx->dc6bar, sizeof(double) * N, cudaMemcpyDeviceToHost), "mbd_get_scs_detail");
    if (omega) MBD_CUDA(cudaMemcpy(omega, ctx->dombar, sizeof(double) * N, cudaMemcpyDeviceToHost), "mbd_get_scs_detail");
    if (rvdw) MBD_CUDA(cudaMemcpy(rvdw, ctx->drbar, sizeof(double) * N, cudaMemcpyDeviceToHost), "mbd_get_scs_detail");
    return MBD_OK;
}

int mbd_ts_energy(mbd_ctx *ctx, double s_r, double *energy, double *grad_coords, double *grad_lattice,
                  double *grad_params) {
    if (!ctx) return MBD_ERR_INPUT;
    if (!energy || !(s_r > 0.0)) return fail(ctx, MBD_ERR_INPUT, "mbd_ts_energy", "energy is required; s_r > 0");
    if (!ctx->have_geom || !ctx->have_params)
        return fail(ctx, MBD_ERR_STATE, "mbd_ts_energy", "set the geometry and the free-atom parameters first");
    if (grad_lattice && !ctx->periodic)
        return fail(ctx, MBD_ERR_UNSUPPORTED, "mbd_ts_energy", "no lattice gradient for finite systems");
    if (ctx->opt.scs_mode == MBD_SCS_NL)
        return fail(ctx, MBD_ERR_UNSUPPORTED, "mbd_ts_energy", "TS takes the free-atom parameters of Eq. ts-scaling");
    MBD_CUDA(cudaSetDevice(ctx->device), "mbd_ts_energy");
    const int N = ctx->N;
    cudaStream_t s = ctx->stream;
    MBD_CUDA(cudaMemcpyAsync(ctx->dR, ctx->hR.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s), "mbd_ts_energy");
    MBD_CUDA(cudaMemcpyAsync(ctx->da0ref, ctx->ha0.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_ts_energy");
    MBD_CUDA(cudaMemcpyAsync(ctx->dc6ref, ctx->hc6.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_ts_energy");
    MBD_CUDA(cudaMemcpyAsync(ctx->drref, ctx->hrr.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_ts_energy");
    MBD_CUDA(cudaMemcpyAsync(ctx->dratio, ctx->hv.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "mbd_ts_energy");
    MBD_CUDA(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), s), "mbd_ts_energy");
    const AtomBufs b = atom_bufs(ctx, Inputs{ctx->dR, ctx->da0ref, ctx->dc6ref, ctx->drref, ctx->dratio});
    prepare_atoms(b, ctx->dstatus, s);   // TS-scaled oscillators (Eq. ts-scaling) and input checks
    // scratch: per-atom energies in dh, dE/d(a0, om, rv) in dga0, dgom, dgrv (and for a cell
    // the lattice parts in dgApart, their sum in dgA); the next evaluation rewrites all of
    // them before use
    if (ctx->periodic) {
        const PeriodicBufs pb = periodic_bufs(ctx);
        structure_factors(b, pb, s);   // e^{i G.R_i} of the current coordinates
        ts_periodic(b, pb, s_r, ctx->dtsg, ctx->dh, ctx->dgR, ctx->dga0, ctx->dgom, ctx->dgrv, ctx->dgApart,
                    ctx->dgA, ctx->dstatus, s);
    } else {
        ts_pairs(b, s_r, ctx->dh, ctx->dgR, ctx->dga0, ctx->dgom, ctx->dgrv, s);
    }
    if (grad_params) ts_chain(b, ctx->dga0, ctx->dgom, ctx->dgrv, nullptr, ctx->dgp, s);
    std::vector<double> ea(N);
    MBD_CUDA(cudaMemcpyAsync(ea.data(), ctx->dh, sizeof(double) * N, cudaMemcpyDeviceToHost, s), "mbd_ts_energy");
    if (grad_coords)
        MBD_CUDA(cudaMemcpyAsync(grad_coords, ctx->dgR, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s), "mbd_ts_energy");
    if (grad_lattice)
        MBD_CUDA(cudaMemcpyAsync(grad_lattice, ctx->dgA, sizeof(double) * 9, cudaMemcpyDeviceToHost, s), "mbd_ts_energy");
    if (grad_params)
        MBD_CUDA(cudaMemcpyAsync(grad_params, ctx->dgp, sizeof(double) * 4 * N, cudaMemcpyDeviceToHost, s), "mbd_ts_energy");
    ctx->have_forward = false;   // the gradient scratch of the last evaluation was reused
    int rc = read_status(ctx, s, "mbd_ts_energy");
    if (rc) return rc;
    double sum = 0.0, comp = 0.0;   // Neumaier sum of the per-atom energies
    for (double x : ea) {
        const double t = sum + x;
        comp += std::fabs(sum) >= std::fabs(x) ? (sum - t) + x : (x - t) + sum;
        sum = t;
    }
    *energy = sum + comp;
    return MBD_OK;
}

int mbd_log_energy(mbd_ctx *ctx, int max_order, double *energy, double *orders) {
    if (!ctx) return MBD_ERR_INPUT;
    if (!energy || max_order < 1 || max_order > 4 || (max_order > 1 && !orders))
        return fail(ctx, MBD_ERR_INPUT, "mbd_log_energy", "energy is required; max_order 1..4; orders for max_order > 1");
    if (ctx->periodic) return fail(ctx, MBD_ERR_UNSUPPORTED, "mbd_log_energy", "finite systems only");
    if (!ctx->have_screening)
        return fail(ctx, MBD_ERR_STATE, "mbd_log_energy", "no oscillators: evaluate the system first");
    MBD_CUDA(cudaSetDevice(ctx->device), "mbd_log_energy");
    cudaStream_t s = ctx->stream;
    const int N = ctx->N, nf = ctx->nf1 - 1;
    const long long ld = ctx->ld, mat = ld * ld;
    MBD_CUDA(cudaMemcpyAsync(ctx->dR, ctx->hR.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s),
             "mbd_log_energy");
    MBD_CUDA(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), s), "mbd_log_energy");
    const AtomBufs b = atom_bufs(ctx, Inputs{ctx->dR, ctx->da0ref, ctx->dc6ref, ctx->drref, ctx->dratio});
    double *A = ctx->dM + mat;   // the nodes u_1..u_nf in screening slots 1..nf
    double *sums = ctx->dlog;    // [4][nf]: sum ln L_pp, Tr A^2, Tr A^3, Tr A^4
    MBD_CUDA(build_lr_freq(b, ctx->opt.beta, ctx->opt.a, A, ld, mat, nf, ctx->dstatus, s), "mbd_log_energy");
    if (max_order >= 2) MBD_CUDA(batch_dot(A, A, mat, mat, nf, sums + nf, s), "mbd_log_energy");   // A symmetric
    if (max_order >= 3) {
        const int M = static_cast<int>(ld);
        for (int k = 0; k < nf; ++k) {   // P = A_k^2 (symmetric), then <P, A_k> and |P|^2
            GemmArgs g{A + k * mat, A + k * mat, nullptr, ctx->dP, ld, ld, 0, ld, 0, 0, 0, 0, M, M, M, 1, 1.0, 0.0, 2, 0};
            gemm_f64(g, s);
            MBD_CUDA(batch_dot(ctx->dP, A + k * mat, mat, 0, 1, sums + 2 * nf + k, s), "mbd_log_energy");
            if (max_order >= 4) MBD_CUDA(batch_dot(ctx->dP, ctx->dP, mat, 0, 1, sums + 3 * nf + k, s), "mbd_log_energy");
        }
    }
    add_identity_batch(A, ld, mat, nf, s);
    cholesky_f64(A, ld, mat, nf, ctx->ddinv, ctx->dstatus, s);
    logdiag_batch(A, ld, mat, nf, sums, ctx->dstatus, s);
    std::vector<double> h(4 * nf);
    MBD_CUDA(cudaMemcpyAsync(h.data(), sums, sizeof(double) * 4 * nf, cudaMemcpyDeviceToHost, s), "mbd_log_energy");
    ctx->have_forward = false;   // the screening buffers now hold these factors
    int rc = read_status(ctx, s, "mbd_log_energy");
    if (rc) return rc;
    const double inv2pi = 1.0 / (2.0 * 3.141592653589793238462643383279502884);
    double e = 0.0;
    for (int k = 0; k < nf; ++k) e += ctx->hwu[k + 1] * 2.0 * h[k];   // ln det = 2 sum ln L_pp
    *energy = e * inv2pi;
    for (int m = 2; m <= max_order; ++m) {
        double t = 0.0;
        for (int k = 0; k < nf; ++k) t += ctx->hwu[k + 1] * h[(m - 1) * nf + k];
        orders[m - 2] = -inv2pi * ((m % 2 == 0) ? 1.0 : -1.0) / m * t;   // -(-1)^m/m Tr A^m
    }
    return MBD_OK;
}

int mbd_get_stats(mbd_ctx *ctx, int *ns_iterations, double *ns_scale, double *ns_residual,
                  double *correction_residual) {
    if (!ctx) return MBD_ERR_INPUT;
    if (correction_residual) *correction_residual = fp64_path(ctx->opt.precision) ? 0.0 : ctx->corr_resid;
    if (ns_iterations) *ns_iterations = ctx->ns_iter;
    if (ns_scale) *ns_scale = ctx->ns_scale;
    if (ns_residual) *ns_residual = ctx->ns_resid;
    return MBD_OK;
}

int mbd_set_profiling(mbd_ctx *ctx, int enable) {
    if (!ctx) return MBD_ERR_INPUT;
    ctx->profiling = enable != 0;
    return MBD_OK;
}

int mbd_get_profile(mbd_ctx *ctx, mbd_profile *out) {
    if (!ctx || !out) return MBD_ERR_INPUT;
    *out = ctx->prof;
    return MBD_OK;
}

int mbd_get_exception(const mbd_ctx *ctx, int *code, char *origin, char *msg, size_t len) {
    if (!ctx) return MBD_ERR_INPUT;
    if (code) *code = ctx->err_code;
    if (origin && len) {
        std::strncpy(origin, ctx->err_origin.c_str(), len - 1);
        origin[len - 1] = '\0';
    }
    if (msg && len) {
        std::strncpy(msg, ctx->err_msg.c_str(), len - 1);
        msg[len - 1] = '\0';
    }
    return MBD_OK;
}

int mbdk_gemm_f64(void *stream, int trans_b, int mode, int M, int N, int K, double alpha,
                  const double *A, long long lda, const double *B, long long ldb, double beta,
                  const double *D, long long ldd, double *C, long long ldc) {
    if (M <= 0 || N <= 0 || K <= 0 || M % kTile || N % kTile || K % kTile || mode < 0 || mode > 3 ||
        (mode && M != N) || !A || !B || !C || (beta != 0.0 && !D) || (lda | ldb | ldc) & 1 ||
        (D && (ldd & 1)) || (trans_b != 0 && trans_b != 1))
        return MBD_ERR_INPUT;
    GemmArgs g{A, B, D, C, lda, ldb, ldd, ldc, 0, 0, 0, 0, M, N, K, 1, alpha, beta, mode, trans_b};
    gemm_f64(g, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

int mbdk_gemm_tc(void *stream, int kind, int mode, int M, int N, int K, float alpha, const void *A0,
                 const void *A1, long long lda, const void *B0, const void *B1, long long ldb, float beta,
                 const float *D, float *C, void *C_hi, void *C_lo, float *CT, long long ldc, int chunk_stages,
                 int *err) {
    if (!A0 || !B0 || (kind != 0 && (!A1 || !B1)) || ((C_hi != nullptr) != (C_lo != nullptr)) || chunk_stages < 0)
        return MBD_ERR_INPUT;
    TcOperands op{A0, kind != 0 ? A1 : A0, B0, kind != 0 ? B1 : B0, lda, ldb};
    TcArgs g{M, N, K, alpha, beta, D, ldc, C, C_hi, C_lo, CT, nullptr, nullptr, nullptr, 0, mode, err, nullptr,
             chunk_stages};
    const cudaError_t e = tc_gemm(kind, op, g, static_cast<cudaStream_t>(stream));
    if (e == cudaErrorInvalidValue) return MBD_ERR_INPUT;
    return e == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

int mbdk_tc_wait_check(void *stream, long long spin_cycles, int *err) {
    const cudaError_t e = tc_wait_probe(spin_cycles, err, static_cast<cudaStream_t>(stream));
    if (e == cudaErrorInvalidValue) return MBD_ERR_INPUT;
    return e == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

size_t mbdk_gemm_f64_split_work_bytes(int M, int N, int K) {
    if (M <= 0 || N <= 0 || K <= 0) return 0;
    return gemm_f64_split_work_bytes(M, N, K);
}

int mbdk_gemm_f64_split(void *stream, int trans_b, int M, int N, int K, double alpha, const double *A,
                        long long lda, const double *B, long long ldb, double beta, const double *D, long long ldd,
                        double *C, long long ldc, void *work, int *err) {
    if (M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 128 || K % 64 || !A || !B || !C || !work || !err ||
        (beta != 0.0 && !D) || ldc % 8 || lda < K || ldb < (trans_b ? K : N) || ldc < N ||
        (D && D != C && ldd < N) || (trans_b != 0 && trans_b != 1))
        return MBD_ERR_INPUT;
    const cudaError_t e = gemm_f64_split(trans_b, 0, M, N, K, alpha, A, lda, B, ldb, beta, D, ldd, C, ldc, work, err,
                                         static_cast<cudaStream_t>(stream));
    if (e == cudaErrorInvalidValue) return MBD_ERR_INPUT;
    return e == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

int mbdk_cholesky_f64(void *stream, double *A, long long ld, int batch, double *dinv, int *status) {
    if (ld <= 0 || ld % kTile || batch < 1 || !A || !dinv || !status) return MBD_ERR_INPUT;
    cholesky_f64(A, ld, ld * ld, batch, dinv, status, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

int mbdk_chol_solve3_f64(void *stream, const double *L, long long ld, int batch, const double *dinv,
                         double *X, double *work) {
    if (ld <= 0 || ld % kTile || batch < 1 || !L || !dinv || !X || !work || work == X) return MBD_ERR_INPUT;
    chol_solve3_f64(L, ld, ld * ld, batch, dinv, X, work, 3 * ld, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? MBD_OK : MBD_ERR_CUDA;
}

}  // extern "C"
