"""The Newton-Schulz schedule of the library (csrc/ns_schedule.h: step coefficients, the lower
bound from the Lanczos minimum, the mixed loop's stopping test), run on the host on the exact
spectrum of Q for a 500-atom cluster of the bench recipe (Q from the oracle's builders, the
screening by LAPACK, the 48-step Lanczos Ritz value from the library's start vector).  In
exact arithmetic the coupled iteration acts on each eigenvalue alone, so the step counts and
the final residuals follow from the spectrum.  Also checks the facts the schedule rests on:
the exact bound of a plain step and the behaviour of a scaled step below its lower bound.
CPU only."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest
import scipy.linalg as sl

import oracle as o
from oracle import oracle as oc
from paper_2308_03140_gb300 import synthetic as syn

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2308_03140_gb300", "csrc")


@pytest.fixture(scope="module")
def host():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "ns_schedule_host.so")
    src = os.path.join(HERE, "ns_schedule_host.cpp")
    deps = [src, os.path.join(CSRC, "ns_schedule.h")]
    if not os.path.exists(so) or any(os.path.getmtime(d) > os.path.getmtime(so) for d in deps):
        res = subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", f"-I{CSRC}", src, "-o", so],
                             capture_output=True, text=True)
        assert res.returncode == 0, res.stderr
    lib = C.CDLL(so)
    d = C.c_double
    lib.ns_scalar_run.argtypes = [C.c_void_p, C.c_int, d, d, C.c_int, d, d, d, C.POINTER(d)]
    lib.ns_scalar_run.restype = C.c_int
    return lib


@pytest.fixture(scope="module")
def spectrum():
    s = syn.sphere_cluster(500, seed=1500)
    N = s.n_atoms
    a0, om, rv = s.alpha0_ref * s.ratio, 4 * s.c6_ref / (3 * s.alpha0_ref ** 2), s.rvdw_ref * np.cbrt(s.ratio)
    u, _ = o.freq_grid(15)
    ab = np.zeros((16, N))
    for k in range(16):
        al = a0 / (1 + u[k] ** 2 / om ** 2)
        M = oc.scs_matrix(s.coords, al, rv)
        cf = sl.cho_factor(M, lower=True, check_finite=False)
        ab[k] = sl.cho_solve(cf, np.tile(np.eye(3), (N, 1)), check_finite=False).reshape(N, 3, 3).trace(
            axis1=1, axis2=2) / 3
    _, (abar0, _, ombar, rbar) = oc.screened_params(ab, a0, rv)
    Q = oc.mbd_q(s.coords, abar0, ombar, rbar)
    lam = sl.eigvalsh(Q, check_finite=False)
    # 48-step Lanczos from the library's start vector (rows padded to a multiple of 128 with
    # the decoupled diagonal omega_bar_0^2)
    n = Q.shape[0]
    ld = (n + 127) // 128 * 128
    Qp = np.zeros((ld, ld))
    Qp[:n, :n] = Q
    Qp[np.arange(n, ld), np.arange(n, ld)] = ombar[0] ** 2
    p = np.arange(ld)
    v = np.sin(0.7548776662 * p + 0.5698402910) + 0.25
    v /= np.linalg.norm(v)
    vp, beta, al, be = np.zeros(ld), 0.0, [], []
    for _ in range(48):
        w = Qp @ v - beta * vp
        alpha = v @ w
        w -= alpha * v
        beta = np.linalg.norm(w)
        al.append(alpha)
        be.append(beta)
        vp, v = v, w / beta
    ritz = np.linalg.eigvalsh(np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1))
    k = 24   # the library's shorter run for matrices of order <= 2048 (this one: 1500)
    ritz24 = np.linalg.eigvalsh(np.diag(al[:k]) + np.diag(be[:k - 1], 1) + np.diag(be[:k - 1], -1))
    return lam, ritz.min(), ritz24.min()


def run(lib, lam, ritz, fraction, mixed, tol, floor_el):
    r = C.c_double()
    lam = np.ascontiguousarray(lam)
    it = lib.ns_scalar_run(lam.ctypes.data_as(C.c_void_p), len(lam), ritz, fraction, mixed, tol, 1e-7, floor_el,
                           C.byref(r))
    return it, r.value


def test_plain_step_bound_and_scaled_step_below_its_bound():
    e = np.linspace(-0.5, 0.5, 2001)
    x = 1 - e
    assert np.all(np.abs(1 - x * (1.5 - 0.5 * x) ** 2) <= 0.875 * e ** 2 + 1e-15)
    for l, u in ((1e-3, 1.05), (0.02, 1.0), (0.3, 1.0)):
        al = np.sqrt(3 / (u * u + u * l + l * l))
        z = np.linspace(1e-6, l, 500)
        f = 0.5 * al * z * (3 - al * al * z * z)
        assert np.all(np.diff(f) > 0) and np.all(f / z >= al - 1e-12) and al >= 1 - 1e-12


def test_schedule_on_the_spectrum(host, spectrum):
    lam, ritz, ritz24 = spectrum
    assert 2.5 < ritz / lam.min() < 4          # the Lanczos minimum lags the spectrum's bottom
    # mixed loop with the TF32x3 precision floor: the floor test stops it at 9 steps, one
    # step below the old half-minimum bound, with the exact residual below the floor
    it, r = run(host, lam, ritz, 0.25, 1, 1e-8, 1.04e-7)
    it_half, _ = run(host, lam, ritz, 0.5, 1, 1e-8, 1.04e-7)
    assert it == 9 and it <= it_half and r < 1.04e-7 * np.sqrt(len(lam))
    # FP64 loop: one step after |I - P| < 1e-8, converged to the last bits
    it64, r64 = run(host, lam, ritz, 0.25, 0, 1e-8, 0.0)
    assert it64 <= 12 and r64 < 1e-13
    # the bound on either side of the true one only costs steps: far above and far below
    for frac in (4.0, 1e-3):
        it_x, r_x = run(host, lam, ritz, frac, 0, 1e-8, 0.0)
        assert r_x < 1e-13 and it_x <= it64 + 6
    # the 24-step estimate that the mixed modes use for matrices of order <= 2048: a higher Ritz
    # minimum and no more steps of the mixed loop (the FP64 loop, which keeps 48, would take one more)
    assert ritz24 > ritz
    it24, r24 = run(host, lam, ritz24, 0.25, 1, 1e-8, 1.04e-7)
    assert it24 <= it and r24 < 1.04e-7 * np.sqrt(len(lam))
    it24_64, r24_64 = run(host, lam, ritz24, 0.25, 0, 1e-8, 0.0)
    assert it24_64 <= it64 + 1 and r24_64 < 1e-13
