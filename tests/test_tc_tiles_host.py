"""The tensor-core GEMM's work decomposition (csrc/tc_tiles.cuh, run on the host through
tests/tc_tiles_host.cu): for every mode and a range of tile counts, the work items of the
single-CTA and the CTA-pair forms cover each tile the mode must write exactly once, and
nothing else is written.  CPU only."""
import ctypes as C
import os
import subprocess

import pytest

from paper_2308_03140_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2308_03140_gb300", "csrc")


@pytest.fixture(scope="module")
def host():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "tc_tiles_host.so")
    src = os.path.join(HERE, "tc_tiles_host.cu")
    deps = [src, os.path.join(CSRC, "tc_tiles.cuh")]
    if not os.path.exists(so) or any(os.path.getmtime(d) > os.path.getmtime(so) for d in deps):
        cmd = [build.nvcc(), *build.ARCH, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", f"-I{CSRC}", src,
               "-o", so]
        res = subprocess.run(cmd, capture_output=True, text=True)
        assert res.returncode == 0, res.stderr
    lib = C.CDLL(so)
    i = C.c_int
    lib.host_grouped_tile.argtypes = [i, i, i, i, C.c_void_p]
    lib.host_pair_tile.argtypes = [i, i, i, i, C.c_void_p]
    return lib


def required(mode, tm_n, tn_n):
    return {(a, b) for a in range(tm_n) for b in range(tn_n)
            if mode == 0 or (mode == 1 and a >= b) or (mode == 2 and a <= b)}


SIZES = [(1, 1), (2, 2), (3, 3), (7, 7), (8, 8), (9, 9), (16, 16), (17, 17), (47, 47), (48, 48), (188, 188),
         (3, 5), (10, 4), (47, 12)]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_single_cta_tiles_cover_the_mode_once(host, mode):
    out = (C.c_int * 2)()
    for tm_n, tn_n in SIZES:
        if mode and tm_n != tn_n:
            continue
        cnt = host.host_tile_count(mode, tm_n, tn_n)
        got = []
        for w in range(cnt):
            host.host_grouped_tile(w, mode, tm_n, tn_n, out)
            got.append((out[0], out[1]))
        assert len(set(got)) == len(got) == len(required(mode, tm_n, tn_n))
        assert set(got) == required(mode, tm_n, tn_n), (mode, tm_n)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_pair_tiles_cover_the_mode_once(host, mode):
    out = (C.c_int * 2)()
    for tm_n, tn_n in SIZES:
        if mode and tm_n != tn_n:
            continue
        cnt = host.host_pair_tile_count(mode, tm_n, tn_n)
        pairs, written = [], []
        for w in range(cnt):
            host.host_pair_tile(w, mode, tm_n, tn_n, out)
            TP, tn = out[0], out[1]
            assert 0 <= TP < (tm_n + 1) // 2 and 0 <= tn < tn_n, (mode, tm_n, w, TP, tn)
            pairs.append((TP, tn))
            for rank in (0, 1):
                if host.host_pair_tile_valid(mode, tm_n, TP, tn, rank):
                    written.append((2 * TP + rank, tn))
        assert len(set(pairs)) == len(pairs), (mode, tm_n)          # no pair tile twice
        assert len(set(written)) == len(written), (mode, tm_n)      # no tile written twice
        assert set(written) == required(mode, tm_n, tn_n), (mode, tm_n)
        # every pair tile writes at least one tile (no idle work items)
        assert all(host.host_pair_tile_valid(mode, tm_n, TP, tn, 0) or host.host_pair_tile_valid(mode, tm_n, TP, tn, 1)
                   for TP, tn in pairs)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_wide_tiles_cover_the_mode_once(host, mode):
    host.host_wide_tile.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]
    out = (C.c_int * 2)()
    for tm_n, tn_n in SIZES:
        if mode and tm_n != tn_n:
            continue
        cnt = host.host_wide_tile_count(mode, tm_n, tn_n)
        tiles, written = [], []
        for w in range(cnt):
            host.host_wide_tile(w, mode, tm_n, tn_n, out)
            tm, TPn = out[0], out[1]
            assert 0 <= tm < tm_n and 0 <= TPn < (tn_n + 1) // 2, (mode, tm_n, w, tm, TPn)
            tiles.append((tm, TPn))
            for h in (0, 1):
                if host.host_wide_half_valid(mode, tn_n, tm, TPn, h):
                    written.append((tm, 2 * TPn + h))
        assert len(set(tiles)) == len(tiles), (mode, tm_n)
        assert len(set(written)) == len(written), (mode, tm_n)
        assert set(written) == required(mode, tm_n, tn_n), (mode, tm_n, tn_n)
        assert all(host.host_wide_half_valid(mode, tn_n, tm, TPn, 0) or host.host_wide_half_valid(mode, tn_n, tm, TPn, 1)
                   for tm, TPn in tiles)
