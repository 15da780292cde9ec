"""The error-free operand splitting behind mbdk_gemm_f64_split (csrc/split64.cuh), compiled
for the host (tests/split64_host.cu), and an exact emulation of the split product on its
slices: the slices are exact FP32 (and TF32) values that add up to each entry within
2^-54 of its row's largest; every partial sum the tensor cores form over a K piece is an
integer multiple of its unit below 2^22, so FP32 holds it exactly; and the sum of the kept
slice products equals the FP64 product to FP64 accuracy.  CPU only; the device product is
checked in test_gpu_z_fp64_products.py."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from paper_2308_03140_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2308_03140_gb300", "csrc")


@pytest.fixture(scope="module")
def host():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "split64_host.so")
    src = os.path.join(HERE, "split64_host.cu")
    deps = [src, os.path.join(CSRC, "split64.cuh"), os.path.join(CSRC, "internal.h")]
    if not os.path.exists(so) or any(os.path.getmtime(d) > os.path.getmtime(so) for d in deps):
        cmd = [build.nvcc(), *build.ARCH, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", f"-I{CSRC}", src,
               "-o", so]
        res = subprocess.run(cmd, capture_output=True, text=True)
        assert res.returncode == 0, res.stderr
    return C.CDLL(so)


def slices(lib, A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    rows, cols = A.shape
    S_n = lib.split64_slices_count()
    e = np.zeros(rows, dtype=np.int32)
    S = np.zeros((S_n, rows, cols), dtype=np.float32)
    lib.split64_rows(A.ctypes.data_as(C.c_void_p), rows, cols, e.ctypes.data_as(C.c_void_p),
                     S.ctypes.data_as(C.c_void_p))
    return e, S


def tf32_exact(x):
    # a TF32 operand keeps the top 19 bits of the FP32 word: exact iff the low 13 are zero
    return np.all((x.view(np.uint32) & np.uint32(0x1FFF)) == 0)


def test_slices_are_exact_and_reconstruct(host):
    rng = np.random.default_rng(1)
    A = rng.normal(size=(40, 70)) * np.exp(rng.uniform(-8, 8, size=(40, 1)))   # rows of very different size
    A[3] = 0.0
    A[5, :10] = 1e-300                                                          # tiny entries in a normal row
    e, S = slices(host, A)
    b, n = host.split64_slice_bits(), host.split64_slices_count()
    assert b * n >= 53
    assert tf32_exact(S)
    for p in range(n):   # slice p is an integer of at most b bits times 2^(e - b (p + 1))
        a = np.ldexp(S[p].astype(np.float64), (-(e - b * (p + 1)))[:, None])
        assert np.all(a == np.round(a)) and np.abs(a).max() < 2 ** b
    recon = S.astype(np.float64).sum(0)
    rowmax = np.abs(A).max(1, keepdims=True)
    assert np.all(np.abs(recon - A) <= 2.0 ** (-b * n) * np.ldexp(1.0, e)[:, None])
    assert np.all(np.abs(recon - A) <= 2.0 ** -53 * rowmax)
    assert np.all(S[:, 3] == 0)


def test_emulated_split_product_is_fp64_accurate(host):
    # the product as the device forms it: slice products of weight p + q <= n over K pieces of
    # at most the chunk, each piece's sums in units of 2^(e_i + f_j - b (p + q + 2))
    rng = np.random.default_rng(2)
    M, N, K = 48, 40, 2300
    A = rng.normal(size=(M, K)) * np.exp(rng.uniform(-3, 3, size=(M, 1)))
    B = rng.normal(size=(K, N)) * np.exp(rng.uniform(-3, 3, size=(1, N)))
    eA, SA = slices(host, A)
    eB, SB = slices(host, np.ascontiguousarray(B.T))   # op(B) by columns = rows of B^T
    b, n, chunk = host.split64_slice_bits(), host.split64_slices_count(), host.split64_chunk()
    Cacc = np.zeros((M, N))
    worst = 0.0
    for p in range(n):
        for q in range(min(n, n + 1 - p)):
            ia = np.ldexp(SA[p].astype(np.float64), (-(eA - b * (p + 1)))[:, None])   # integers
            ib = np.ldexp(SB[q].astype(np.float64), (-(eB - b * (q + 1)))[:, None])
            for k0 in range(0, K, chunk):
                part = ia[:, k0:k0 + chunk] @ ib[:, k0:k0 + chunk].T               # exact: < 2^53
                worst = max(worst, np.abs(part).max(),
                            np.abs(np.cumsum(ia[:, k0:k0 + chunk, None] * ib.T[None, k0:k0 + chunk], 1)).max())
                unit = np.ldexp(1.0, (eA[:, None] + eB[None, :] - b * (p + q + 2)))
                Cacc += part * unit                                                  # FP64 additions
    assert worst < 2 ** 22          # every partial sum exact in FP32, two bits to spare
    exact = (np.array(A, dtype=np.longdouble) @ np.array(B, dtype=np.longdouble)).astype(np.float64)
    scale = np.abs(A) @ np.abs(B)
    fp64 = np.abs(A @ B - exact) / scale                  # an FP64 GEMM's own error, in units of |A||B|
    err = np.abs(Cacc - exact) / scale
    assert err.max() <= 2 * fp64.max() + 2.0 ** -52 and err.max() <= 8 * 2.0 ** -53


def test_tiny_rows_keep_normal_slices(host):
    # a row whose largest element lies below 2^-72 is sliced at exponent -72, so that the last
    # slice's unit 2^-126 is still an FP32 normal (the tensor cores flush subnormals): every
    # non-zero slice value is normal, the slices are exact, and the row is rebuilt to 2^-126
    rng = np.random.default_rng(3)
    A = rng.normal(size=(4, 50))
    A[1] *= 1e-25
    A[2] *= 1e-35
    e, S = slices(host, A)
    assert e[1] == -72 and e[2] == -72
    nz = S[S != 0].astype(np.float64)
    assert np.all(np.abs(nz) >= 2.0 ** -126)
    recon = S.astype(np.float64).sum(0)
    assert np.all(np.abs(recon[1:3] - A[1:3]) <= 2.0 ** -126)
    assert np.all(np.abs(recon[[0, 3]] - A[[0, 3]]) <= 2.0 ** -53 * np.abs(A[[0, 3]]).max(1, keepdims=True))
