"""The radial formulas of the pair kernels (csrc/pair_math.cuh, evaluated on the host through
tests/pair_math_host.cu) against the oracle's dipole tensors and damping function (Eqs.
dipole, tgg, terfc, fermi-damping): T = P I + W r r^T equals the oracle's T, T^GG and T^erfc,
the radial derivatives equal central differences of the oracle's tensors, and the FP32
versions of the reduced-precision modes agree with the FP64 ones to FP32 accuracy.  CPU only."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as o
from paper_2308_03140_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2308_03140_gb300", "csrc")


@pytest.fixture(scope="module")
def host():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "pair_math_host.so")
    src = os.path.join(HERE, "pair_math_host.cu")
    deps = [src, os.path.join(CSRC, "pair_math.cuh"), os.path.join(CSRC, "internal.h")]
    if not os.path.exists(so) or any(os.path.getmtime(d) > os.path.getmtime(so) for d in deps):
        cmd = [build.nvcc(), *build.ARCH, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", f"-I{CSRC}", src,
               "-o", so]
        res = subprocess.run(cmd, capture_output=True, text=True)
        assert res.returncode == 0, res.stderr
    lib = C.CDLL(so)
    d, f = C.c_double, C.c_float
    lib.host_fermi.argtypes = [d, d, d, d, C.c_void_p]
    lib.host_fermi_f.argtypes = [f, f, f, f, C.c_void_p]
    lib.host_tgg.argtypes = [d, d, C.c_void_p]
    lib.host_tgg_f.argtypes = [f, f, C.c_void_p]
    lib.host_bare.argtypes = [d, C.c_void_p]
    lib.host_erfc.argtypes = [d, d, C.c_void_p]
    return lib


def call(fn, *args, n, dtype=np.float64):
    out = np.zeros(n, dtype=dtype)
    fn(*args, out.ctypes.data_as(C.c_void_p))
    return out


def tensor(P, W, r):
    return P * np.eye(3) + W * np.outer(r, r)


def rvecs():
    rng = np.random.default_rng(4)
    for rho in (0.9, 2.3, 4.0, 7.5, 15.0):
        v = rng.normal(size=3)
        yield rho * v / np.linalg.norm(v)


def fd_tensor(fn, r, h=1e-6):
    return np.array([(fn(r + h * e) - fn(r - h * e)) / (2 * h) for e in np.eye(3)])   # [c][a][b]


def radial_deriv_tensor(P, W, dP, dW, r):
    rho = np.linalg.norm(r)
    out = []
    for c in range(3):
        e = np.eye(3)[c]
        out.append(dP * r[c] / rho * np.eye(3) + dW * r[c] / rho * np.outer(r, r) + W * (np.outer(e, r) + np.outer(r, e)))
    return np.array(out)


def test_bare_and_gaussian_dipole_tensors(host):
    for r in rvecs():
        rho = np.linalg.norm(r)
        P, W, dP, dW = call(host.host_bare, rho, n=4)
        assert np.allclose(tensor(P, W, r), o.T_bare(r), rtol=1e-14, atol=0)
        ref = fd_tensor(o.T_bare, r)
        assert np.allclose(radial_deriv_tensor(P, W, dP, dW, r), ref, atol=1e-7 * np.abs(ref).max())
        for s in (0.6, 1.5, 3.0):
            P, W, dP, dW, dPs, dWs = call(host.host_tgg, rho, s, n=6)
            T = o.T_gg(r, s)
            assert np.allclose(tensor(P, W, r), T, rtol=1e-13, atol=1e-15 * np.abs(T).max())
            ref = fd_tensor(lambda x: o.T_gg(x, s), r)
            assert np.allclose(radial_deriv_tensor(P, W, dP, dW, r), ref, atol=1e-7 * np.abs(ref).max())
            h = 1e-6 * s
            refs = (o.T_gg(r, s + h) - o.T_gg(r, s - h)) / (2 * h)
            # far beyond the width the s-derivative is ~e^{-z^2}: compare on the tensor's scale
            assert np.allclose(tensor(dPs, dWs, r), refs, atol=1e-7 * np.abs(refs).max() + 1e-9 * np.abs(T).max() / s)
            # FP32: W = (2 z^2 Th - 3 F1)/r^5 cancels at short range, costing a few digits
            Pf = call(host.host_tgg_f, np.float32(rho), np.float32(s), n=6, dtype=np.float32)
            assert np.allclose(Pf[:2], [P, W], rtol=2e-4, atol=2e-6 * max(abs(P), abs(W)))


def test_erfc_screened_tensor(host):
    for r in rvecs():
        rho = np.linalg.norm(r)
        for g in (0.15, 0.3, 0.6):
            P, W, dP, dW = call(host.host_erfc, rho, g, n=4)
            T = o.T_erfc(r, g)
            assert np.allclose(tensor(P, W, r), T, rtol=1e-12, atol=1e-14 * np.abs(T).max() + 1e-300)
            ref = fd_tensor(lambda x: o.T_erfc(x, g), r)
            assert np.allclose(radial_deriv_tensor(P, W, dP, dW, r), ref, atol=1e-7 * np.abs(ref).max() + 1e-300)


def test_fermi_damping(host):
    for rho, S, beta, a in ((3.0, 7.0, 0.83, 6.0), (6.5, 7.0, 0.83, 6.0), (12.0, 6.2, 0.94, 20.0), (5.5, 6.2, 0.94, 20.0)):
        f, dfr, dfs = call(host.host_fermi, rho, S, beta, a, n=3)
        assert f == pytest.approx(o.fermi(rho, S, beta, a), rel=1e-14, abs=1e-300)
        h = 1e-6
        assert dfr == pytest.approx((o.fermi(rho + h, S, beta, a) - o.fermi(rho - h, S, beta, a)) / (2 * h), rel=1e-7,
                                    abs=1e-8)
        assert dfs == pytest.approx((o.fermi(rho, S + h, beta, a) - o.fermi(rho, S - h, beta, a)) / (2 * h), rel=1e-7,
                                    abs=1e-8)
        ff = call(host.host_fermi_f, np.float32(rho), np.float32(S), np.float32(beta), np.float32(a), n=3,
                  dtype=np.float32)
        assert np.allclose(ff, [f, dfr, dfs], rtol=1e-5, atol=1e-6)


def test_gaussian_tensor_far_branch_is_exact(host):
    # beyond z = r/s = 8 the Gaussian parts round away in FP64: the far branch returns the bare
    # tensor's radial parts, which the full formula reproduces to the last bit (host libm), and
    # it joins the full formula continuously at the boundary
    for s in (0.7, 1.3, 2.1):
        for z in (8.0000001, 9.0, 13.0, 40.0):
            rho = z * s
            far = call(host.host_tgg, rho, s, n=6)
            bare = call(host.host_bare, rho, n=4)
            assert np.array_equal(far[:4], bare) and far[4] == 0.0 and far[5] == 0.0
            x = np.array([rho, 0.0, 0.0])
            T = o.T_gg(x, s)
            assert np.allclose(tensor(far[0], far[1], x), T, rtol=2e-15, atol=0)
        inside = call(host.host_tgg, 7.9999999 * s, s, n=6)   # the full formula just inside
        assert np.allclose(inside[:4], call(host.host_bare, 7.9999999 * s, n=4), rtol=1e-15, atol=0)
        assert abs(inside[4]) < 1e-22 * abs(inside[2]) * s and abs(inside[5]) < 1e-22 * abs(inside[3]) * s
        for z in (5.0001, 6.0, 11.0):   # FP32 branch beyond z = 5
            rf = call(host.host_tgg_f, np.float32(z * s), np.float32(s), n=6, dtype=np.float32)
            assert rf[4] == 0.0 and rf[5] == 0.0
            assert np.allclose(rf[:4], call(host.host_bare, float(np.float32(z * s)), n=4), rtol=1e-6, atol=0)


def test_far_damping_rounds_to_one_with_zero_derivatives(host):
    # the SCS adjoint pair passes skip pairs whose damping has rounded to f = 1: then 1 - f
    # and both derivatives are exactly zero, so every term of the pair is an exact zero
    beta, a, S = 0.83, 6.0, 7.0
    for eta in (7.2, 9.0, 20.0):            # FP64: e^{-6 (eta - 1)} below half an ulp of 1
        f, dfr, dfs = call(host.host_fermi, eta * beta * S, S, beta, a, n=3)
        assert f == 1.0 and dfr == 0.0 and dfs == 0.0
    for eta in (3.8, 5.0, 9.0):             # FP32: below 2^-24 from eta ~ 3.77
        ff = call(host.host_fermi_f, np.float32(eta * beta * S), np.float32(S), np.float32(beta), np.float32(a), n=3,
                  dtype=np.float32)
        assert ff[0] == 1.0 and ff[1] == 0.0 and ff[2] == 0.0
    f, dfr, dfs = call(host.host_fermi, 6.0 * beta * S, S, beta, a, n=3)   # nearer: small but nonzero
    assert f < 1.0 and dfr > 0.0 and dfs < 0.0


def test_screening_matrix_with_the_far_branch_matches_the_oracle(host):
    # the screening matrices of a 300-atom cluster at all 16 grid points, formed with the
    # kernel's formulas (far branch of T^GG included), against the oracle's builder
    from paper_2308_03140_gb300 import synthetic as syn
    s = syn.sphere_cluster(300, seed=1300)
    a0, om, rv = s.alpha0_ref * s.ratio, 4 * s.c6_ref / (3 * s.alpha0_ref ** 2), s.rvdw_ref * np.cbrt(s.ratio)
    u, _ = o.freq_grid(15)
    R = np.ascontiguousarray(s.coords)
    host.host_scs_matrix.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                     C.c_double, C.c_void_p]
    n = 3 * len(R)
    far = 0
    for k in range(16):
        al = np.ascontiguousarray(a0 / (1 + u[k] ** 2 / om ** 2))
        sig = np.ascontiguousarray(np.cbrt(np.sqrt(2 / np.pi) * al / 3))
        M = np.zeros((n, n))
        host.host_scs_matrix(len(R), R.ctypes.data_as(C.c_void_p), al.ctypes.data_as(C.c_void_p),
                             sig.ctypes.data_as(C.c_void_p), np.ascontiguousarray(rv).ctypes.data_as(C.c_void_p),
                             0.83, 6.0, M.ctypes.data_as(C.c_void_p))
        ref = o.scs_matrix(R, al, rv)
        assert np.abs(M - ref).max() <= 1e-14 * np.abs(ref).max(), k
        d = np.linalg.norm(R[:, None] - R[None], axis=-1)
        far += np.sum(d / np.sqrt(sig[:, None] ** 2 + sig[None] ** 2) > 8)
    assert far > 0.5 * 16 * len(R) ** 2     # most pair-frequency evaluations took the far branch
