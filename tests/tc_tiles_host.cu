// Host run of the tensor-core GEMM's work decomposition (csrc/tc_tiles.cuh) for the CPU tests.
// Test infrastructure: built by tests/test_tc_tiles_host.py into tests/_build.
#include "tc_tiles.cuh"

using namespace mbdgb::tctiles;

extern "C" int host_tile_count(int mode, int tm, int tn) { return tile_count(mode, tm, tn); }
extern "C" void host_grouped_tile(int bid, int mode, int tiles_m, int tiles_n, int *out) {
    grouped_tile(bid, mode, tiles_m, tiles_n, out[0], out[1]);
}
extern "C" int host_pair_tile_count(int mode, int tm, int tn) { return pair_tile_count(mode, tm, tn); }
extern "C" void host_pair_tile(int bid, int mode, int tiles_m, int tiles_n, int *out) {
    pair_tile(bid, mode, tiles_m, tiles_n, out[0], out[1]);
}
extern "C" int host_pair_tile_valid(int mode, int tiles_m, int TP, int tn, int rank) {
    return pair_tile_valid(mode, tiles_m, TP, tn, rank) ? 1 : 0;
}
extern "C" int host_wide_tile_count(int mode, int tm, int tn) { return wide_tile_count(mode, tm, tn); }
extern "C" void host_wide_tile(int bid, int mode, int tiles_m, int tiles_n, int *out) {
    wide_tile(bid, mode, tiles_m, tiles_n, out[0], out[1]);
}
extern "C" int host_wide_half_valid(int mode, int tiles_n, int tm, int TPn, int h) {
    return wide_half_valid(mode, tiles_n, tm, TPn, h) ? 1 : 0;
}
