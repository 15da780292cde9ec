// Periodic TS pairwise dispersion for sm_103a (FP64): Secs. 2.6 and 2.7, the lattice sum of
// Eq. pairwise with the TS oscillators by the Ewald split of Eq. ts-ewald minus the
// real-space sum of the damped-away part.  The per-pair arithmetic is ts::pair_terms
// (ts_terms.cuh); here it is launched one CTA per atom.
//
//  ts_gtable        (t_G, rp_G) of every reciprocal vector in use (zero at |G| >= kc)
//  ts_periodic      per atom i: energy share, dE/d(alpha0, omega, R_vdW) of the TS-scaled
//                   oscillators, dE/dR_i and the lattice part of its ordered pairs
//  ts_lattice_sum   dE/dA = sum over atoms of the lattice parts (fixed order)
//
// Work per launch: N^2 pairs x (images within rc, ~60 flop each; nG reciprocal vectors,
// ~20 flop each from the structure factors).
#include "pair_math.cuh"
#include "ts_terms.cuh"

namespace mbdgb {
namespace {

using pairs::block_sum128;

__global__ void k_ts_gtable(const double *G, int nG, CellGeom c, double *tab) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nG) return;
    const double Gn = sqrt(G[3 * q] * G[3 * q] + G[3 * q + 1] * G[3 * q + 1] + G[3 * q + 2] * G[3 * q + 2]);
    const ts::Recip r = ts::recip_term(Gn, c.gamma, c.vol, c.kc);
    tab[2 * q] = r.t;
    tab[2 * q + 1] = r.rp;
}

// One CTA (128 threads) per atom i; partners j = 0..N-1, j = i standing for the images of i.
// acc: e, dE/da_i, dE/dw_i, dE/dR_vdW,i, dE/dR_i (3), lattice part (9).
__global__ void __launch_bounds__(128) k_ts_periodic(AtomBufs b, PeriodicBufs p, const double *tab, double s_r,
                                                     double *eatom, double *ga0, double *gom, double *grv,
                                                     double *gR, double *gA_part, int *status) {
    const int i = blockIdx.x;
    const double ai = b.a0[i], wi = b.om[i], rvi = b.rv[i];
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    bool bad = false;
    for (int j = threadIdx.x; j < b.N; j += 128) {
        const double x[3] = {b.R[3 * j] - b.R[3 * i], b.R[3 * j + 1] - b.R[3 * i + 1], b.R[3 * j + 2] - b.R[3 * i + 2]};
        const double aj = b.a0[j], wj = b.om[j];
        const double c6 = 1.5 * ai * aj * wi * wj / (wi + wj);
        ts::Pair o;
        ts::pair_terms(p.cell, x, j == i, c6, rvi + b.rv[j], s_r, p.nG, p.G, tab, p.S + i, p.S + j, b.N, o);
        acc[0] += o.e;
        acc[1] += -o.s * c6 / ai;
        acc[2] += -o.s * c6 * (1.0 / wi - 1.0 / (wi + wj));
        acc[3] += o.grv;
        for (int e = 0; e < 3; ++e) acc[4 + e] += o.gR[e];
        for (int e = 0; e < 9; ++e) acc[7 + e] += o.gA[e];
        bad = bad || o.bad;
    }
    if (bad) atomicOr(status, ST_INPUT);
    __shared__ double scratch[4 * 16];
    block_sum128<16>(acc, scratch);
    if (threadIdx.x == 0) {
        eatom[i] = acc[0];
        ga0[i] = acc[1];
        gom[i] = acc[2];
        grv[i] = acc[3];
        for (int e = 0; e < 3; ++e) gR[3 * i + e] = acc[4 + e];
        for (int e = 0; e < 9; ++e) gA_part[9LL * i + e] = acc[7 + e];
    }
}

__global__ void k_ts_lattice_sum(const double *part, int N, double *gA) {
    const int e = threadIdx.x;
    if (e >= 9) return;
    double s = 0.0;
    for (int i = 0; i < N; ++i) s += part[9LL * i + e];
    gA[e] = s;
}

inline int cdiv(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

}  // namespace

void ts_periodic(const AtomBufs &b, const PeriodicBufs &p, double s_r, double *tab, double *eatom, double *gR,
                 double *ga0, double *gom, double *grv, double *gA_part, double *gA, int *status, cudaStream_t s) {
    count_launches(3);
    k_ts_gtable<<<cdiv(p.nG, 128), 128, 0, s>>>(p.G, p.nG, p.cell, tab);
    k_ts_periodic<<<b.N, 128, 0, s>>>(b, p, tab, s_r, eatom, ga0, gom, grv, gR, gA_part, status);
    k_ts_lattice_sum<<<1, 32, 0, s>>>(gA_part, b.N, gA);
}

}  // namespace mbdgb
