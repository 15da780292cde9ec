// Host build of the library's Casimir-Polder grid (csrc/freq_grid.h) for the CPU tests.
// Test infrastructure: built by tests/test_freq_grid_host.py into tests/_build.
#include <vector>

#include "freq_grid.h"

extern "C" void freq_grid_host(int n_freq, double *u, double *wu) {
    std::vector<double> uu, ww;
    mbdgb::casimir_polder_grid(n_freq, uu, ww);
    for (int k = 0; k <= n_freq; ++k) {
        u[k] = uu[k];
        wu[k] = ww[k];
    }
}
