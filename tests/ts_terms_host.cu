// Host run of the periodic TS pair arithmetic of the CUDA library (ts::pair_terms and
// ts::recip_term of csrc/ts_terms.cuh, the functions k_ts_gtable and k_ts_periodic call),
// accumulated per atom exactly as k_ts_periodic does but in plain loops, for the CPU tests.
// Test infrastructure: built by tests/test_ts_terms_host.py into tests/_build.
#include <cmath>
#include <vector>

#include "ts_terms.cuh"

using namespace mbdgb;

// Inputs: cell (A, A^-1, B = 2 pi A^-T row-major, volume), gamma, rc, kc; the TS-scaled
// oscillators a0, om, rv [N]; reciprocal vectors G [nG][3].  Outputs as the kernel's:
// eatom [N], ga0, gom, grv [N], gR [N][3], gA [9] (the per-atom lattice parts summed).
// Returns 1 if an image other than a self image lies at zero distance.
extern "C" int ts_host_periodic(int N, const double *R, const double *A, const double *Ainv, const double *B,
                                double vol, double gamma, double rc, double kc, const double *a0, const double *om,
                                const double *rv, double s_r, int nG, const double *G, double *eatom, double *ga0,
                                double *gom, double *grv, double *gR, double *gA) {
    CellGeom c{};
    for (int e = 0; e < 9; ++e) {
        c.A[e] = A[e];
        c.Ainv[e] = Ainv[e];
        c.B[e] = B[e];
    }
    c.vol = vol;
    c.gamma = gamma;
    c.rc = rc;
    c.kc = kc;
    std::vector<double> tab(2 * static_cast<size_t>(nG));
    for (int q = 0; q < nG; ++q) {
        const double Gn = std::sqrt(G[3 * q] * G[3 * q] + G[3 * q + 1] * G[3 * q + 1] + G[3 * q + 2] * G[3 * q + 2]);
        const ts::Recip r = ts::recip_term(Gn, gamma, vol, kc);
        tab[2 * q] = r.t;
        tab[2 * q + 1] = r.rp;
    }
    std::vector<double2> S(static_cast<size_t>(nG) * N);   // e^{i G.R_i}, [nG][N]
    for (int q = 0; q < nG; ++q)
        for (int i = 0; i < N; ++i) {
            const double ph = G[3 * q] * R[3 * i] + G[3 * q + 1] * R[3 * i + 1] + G[3 * q + 2] * R[3 * i + 2];
            S[static_cast<size_t>(q) * N + i] = make_double2(std::cos(ph), std::sin(ph));
        }
    int bad = 0;
    for (int e = 0; e < 9; ++e) gA[e] = 0.0;
    for (int i = 0; i < N; ++i) {
        double acc[16] = {};
        for (int j = 0; j < N; ++j) {
            const double x[3] = {R[3 * j] - R[3 * i], R[3 * j + 1] - R[3 * i + 1], R[3 * j + 2] - R[3 * i + 2]};
            const double c6 = 1.5 * a0[i] * a0[j] * om[i] * om[j] / (om[i] + om[j]);
            ts::Pair o;
            ts::pair_terms(c, x, j == i, c6, rv[i] + rv[j], s_r, nG, G, tab.data(), S.data() + i, S.data() + j, N, o);
            acc[0] += o.e;
            acc[1] += -o.s * c6 / a0[i];
            acc[2] += -o.s * c6 * (1.0 / om[i] - 1.0 / (om[i] + om[j]));
            acc[3] += o.grv;
            for (int e = 0; e < 3; ++e) acc[4 + e] += o.gR[e];
            for (int e = 0; e < 9; ++e) acc[7 + e] += o.gA[e];
            bad |= o.bad ? 1 : 0;
        }
        eatom[i] = acc[0];
        ga0[i] = acc[1];
        gom[i] = acc[2];
        grv[i] = acc[3];
        for (int e = 0; e < 3; ++e) gR[3 * i + e] = acc[4 + e];
        for (int e = 0; e < 9; ++e) gA[e] += acc[7 + e];
    }
    return bad;
}
