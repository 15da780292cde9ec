// Work decomposition of the tensor-core GEMM (k_tc.cu) into output tiles of 128 x 128, shared
// by the device kernels and a host check (tests/tc_tiles_host.cu).
//
// Single-CTA form (k_tc_gemm): work item -> one 128 x 128 tile (tm, tn).
// CTA-pair form (k_tc_gemm2, tcgen05 cta_group::2): work item -> a pair tile of 256 x 128,
// tile rows 2 TP and 2 TP + 1 (one per CTA of the pair) of tile column tn.
// Wide form (k_tc_gemm_w): work item -> a wide tile of 128 x 256, tile row tm, tile columns
// 2 TPn and 2 TPn + 1 (one per half of the CTA's epilogue warps): the transposed pairs.
//
// Modes: 0 every tile; 1 the tiles on or below the diagonal (tm >= tn); 2 the tiles on or
// above it (tm <= tn).  Modes 1 and 2 are square (tiles_m == tiles_n).  A pair tile of mode 1
// or 2 that straddles the diagonal holds one tile outside the triangle, and the last pair row
// of an odd tile count one tile below the matrix: pair_tile_valid() tells the CTA whose tile it
// is to compute it without writing it.
//
// Tiles are taken in groups so that the CTAs resident at one time share operand panels in
// L2: mode 0 in groups of kTcGroup (pair) rows walked column by column; modes 1 and 2 in
// super-tiles of kTcGroup x kTcGroup tiles (kTcGroup/2 pair rows x kTcGroup columns in the
// pair form) of the triangle, column-major inside each.
#pragma once

namespace mbdgb {
namespace tctiles {

constexpr int kTcGroup = 8;

__host__ __device__ inline int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ inline int imax(int a, int b) { return a > b ? a : b; }

// ---- single-CTA tiles -------------------------------------------------------------------
__host__ __device__ inline int tile_count(int mode, int tiles_m, int tiles_n) {
    return mode == 0 ? tiles_m * tiles_n : tiles_n * (tiles_n + 1) / 2;
}

// Tile of work item `bid` (0 <= bid < tile_count).
__host__ __device__ inline void grouped_tile(int bid, int mode, int tiles_m, int tiles_n, int &tm, int &tn) {
    tm = tn = 0;
    if (mode == 0) {
        const int per_group = kTcGroup * tiles_n;
        const int g = bid / per_group, first = g * kTcGroup;
        const int rows = imin(kTcGroup, tiles_m - first), local = bid - g * per_group;
        tm = first + local % rows;
        tn = local / rows;
        return;
    }
    // upper triangle tm <= tn: kTcGroup x kTcGroup super-tiles in order, column-major inside
    // each; mode 1 takes the transposed tiles
    const int T = tiles_n, S = (T + kTcGroup - 1) / kTcGroup;
    int left = bid;
    bool found = false;
    for (int R = 0; R < S && !found; ++R) {        // super column of tn
        const int nr = imin(kTcGroup, T - R * kTcGroup);
        for (int C = 0; C <= R && !found; ++C) {   // super row of tm
            const int nc = imin(kTcGroup, T - C * kTcGroup);
            const int cnt = (C == R) ? nc * (nc + 1) / 2 : nc * nr;
            if (left < cnt) {
                if (C == R) {            // triangle of the diagonal super-tile: local c <= r
                    int r = 0;
                    while ((r + 1) * (r + 2) / 2 <= left) ++r;
                    tn = R * kTcGroup + r;
                    tm = C * kTcGroup + (left - r * (r + 1) / 2);
                } else {
                    tm = C * kTcGroup + left % nc;
                    tn = R * kTcGroup + left / nc;
                }
                found = true;
            } else {
                left -= cnt;
            }
        }
    }
    if (mode == 1) {
        const int t = tm;
        tm = tn;
        tn = t;
    }
}

// ---- CTA-pair tiles ---------------------------------------------------------------------
// Pair rows TP = 0 .. ceil(tiles_m / 2) - 1; in modes 1 and 2 a pair tile (TP, tn) is kept
// when either of its tiles lies in the triangle: mode 2 (upper) tn >= 2 TP, mode 1 (lower)
// tn <= 2 TP + 1.
__host__ __device__ inline int pair_rows(int tiles_m) { return (tiles_m + 1) / 2; }

// pair tiles of super-tile (C, R): pair rows [G2 C, G2 C + np), columns [G R, G R + nc)
__host__ __device__ inline int pair_super_count(int mode, int C, int R, int np, int nc) {
    if (mode == 2) {
        if (C < R) return np * nc;
        if (C > R) return 0;
        int cnt = 0;   // diagonal super-tile: local (p, c) kept when c >= 2 p
        for (int p = 0; p < np; ++p) cnt += imax(0, nc - 2 * p);
        return cnt;
    }
    // mode 1
    if (C > R) return np * nc;
    if (C < R) return 0;
    int cnt = 0;       // diagonal super-tile: local (p, c) kept when c <= 2 p + 1
    for (int p = 0; p < np; ++p) cnt += imin(nc, 2 * p + 2);
    return cnt;
}

__host__ __device__ inline int pair_tile_count(int mode, int tiles_m, int tiles_n) {
    const int P = pair_rows(tiles_m);
    if (mode == 0) return P * tiles_n;
    constexpr int G2 = kTcGroup / 2;
    const int T = tiles_n, S = (T + kTcGroup - 1) / kTcGroup;
    int total = 0;
    for (int C = 0; C < S; ++C)
        for (int R = 0; R < S; ++R) {
            const int np = imin(G2, P - C * G2), nc = imin(kTcGroup, T - R * kTcGroup);
            if (np > 0 && nc > 0) total += pair_super_count(mode, C, R, np, nc);
        }
    return total;
}

// Pair tile (TP, tn) of work item `bid` (0 <= bid < pair_tile_count).
__host__ __device__ inline void pair_tile(int bid, int mode, int tiles_m, int tiles_n, int &TP, int &tn) {
    const int P = pair_rows(tiles_m);
    TP = tn = 0;
    if (mode == 0) {
        const int per_group = kTcGroup * tiles_n;
        const int g = bid / per_group, first = g * kTcGroup;
        const int rows = imin(kTcGroup, P - first), local = bid - g * per_group;
        TP = first + local % rows;
        tn = local / rows;
        return;
    }
    constexpr int G2 = kTcGroup / 2;
    const int T = tiles_n, S = (T + kTcGroup - 1) / kTcGroup;
    int left = bid;
    // mode 2: super columns R outer, super rows C <= R inner; mode 1: super rows C outer,
    // super columns R <= C inner
    for (int a = 0; a < S; ++a)
        for (int b = 0; b <= a; ++b) {
            const int C = mode == 2 ? b : a, R = mode == 2 ? a : b;
            const int np = imin(G2, P - C * G2), nc = imin(kTcGroup, T - R * kTcGroup);
            if (np <= 0 || nc <= 0) continue;
            const int cnt = pair_super_count(mode, C, R, np, nc);
            if (left >= cnt) {
                left -= cnt;
                continue;
            }
            // column-major inside the super-tile, the kept pair rows of each column
            for (int c = 0; c < nc; ++c) {
                int p0 = 0, p1 = np;   // kept local pair rows [p0, p1) of local column c
                if (C == R) {
                    if (mode == 2) p1 = imin(np, c / 2 + 1);                 // 2 p <= c
                    else p0 = c / 2;                                        // 2 p + 1 >= c
                }
                const int k = imax(0, p1 - p0);
                if (left < k) {
                    TP = C * G2 + p0 + left;
                    tn = R * kTcGroup + c;
                    return;
                }
                left -= k;
            }
        }
}

// Whether the CTA of rank `rank` (0, 1) of pair tile (TP, tn) writes its tile (2 TP + rank, tn).
__host__ __device__ inline bool pair_tile_valid(int mode, int tiles_m, int TP, int tn, int rank) {
    const int tm = 2 * TP + rank;
    if (tm >= tiles_m) return false;
    if (mode == 1) return tm >= tn;
    if (mode == 2) return tm <= tn;
    return true;
}

// ---- wide tiles (128 x 256: tile row tm, tile columns 2 TPn and 2 TPn + 1) --------------
// The transpose of the CTA-pair decomposition: pairs of tile columns.  A wide tile of mode 2
// (upper) is kept when either half lies on or above the diagonal (2 TPn + 1 >= tm), of mode 1
// (lower) when either lies on or below it (2 TPn <= tm).
__host__ __device__ inline int transposed_mode(int mode) { return mode == 2 ? 1 : (mode == 1 ? 2 : 0); }

__host__ __device__ inline int wide_tile_count(int mode, int tiles_m, int tiles_n) {
    return pair_tile_count(transposed_mode(mode), tiles_n, tiles_m);
}

// Wide tile (tm, TPn) of work item `bid` (0 <= bid < wide_tile_count).
__host__ __device__ inline void wide_tile(int bid, int mode, int tiles_m, int tiles_n, int &tm, int &TPn) {
    pair_tile(bid, transposed_mode(mode), tiles_n, tiles_m, TPn, tm);
}

// Whether half h (0, 1) of wide tile (tm, TPn), the 128 x 128 tile (tm, 2 TPn + h), is written.
__host__ __device__ inline bool wide_half_valid(int mode, int tiles_n, int tm, int TPn, int h) {
    return pair_tile_valid(transposed_mode(mode), tiles_n, TPn, tm, h);
}

}  // namespace tctiles
}  // namespace mbdgb
