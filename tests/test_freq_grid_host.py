"""The library's imaginary-frequency grid (csrc/freq_grid.h, Sec. 3.3: Gauss-Legendre nodes
mapped by u = 0.6 (1 + x) / (1 - x)), built on the host: nodes and weights against numpy's
Gauss-Legendre rule under the same map, u_0 = 0 with weight 0, and the integral of a Lorentzian
(the Casimir-Polder form) against its closed form.  CPU only."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2308_03140_gb300", "csrc")


@pytest.fixture(scope="module")
def grid():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "freq_grid_host.so")
    src = os.path.join(HERE, "freq_grid_host.cpp")
    deps = [src, os.path.join(CSRC, "freq_grid.h")]
    if not os.path.exists(so) or any(os.path.getmtime(d) > os.path.getmtime(so) for d in deps):
        res = subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", f"-I{CSRC}", src, "-o", so],
                             capture_output=True, text=True)
        assert res.returncode == 0, res.stderr
    lib = C.CDLL(so)
    lib.freq_grid_host.argtypes = [C.c_int, C.c_void_p, C.c_void_p]

    def run(n):
        u, w = np.zeros(n + 1), np.zeros(n + 1)
        lib.freq_grid_host(n, u.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p))
        return u, w
    return run


@pytest.mark.parametrize("n", [1, 4, 15, 40])
def test_grid_is_the_mapped_gauss_legendre_rule(grid, n):
    u, w = grid(n)
    x, wx = np.polynomial.legendre.leggauss(n)
    assert u[0] == 0.0 and w[0] == 0.0
    assert np.allclose(u[1:], 0.6 * (1 + x) / (1 - x), rtol=1e-13, atol=0)
    assert np.allclose(w[1:], wx * 1.2 / (1 - x) ** 2, rtol=1e-12, atol=0)
    assert np.all(np.diff(u[1:]) > 0)


def test_grid_integrates_the_casimir_polder_form(grid):
    # integral_0^inf du / (1 + u^2/w^2)^2 = pi w / 4: the shape of alpha(iu)^2 for one
    # oscillator, which the 15-point rule integrates to the accuracy Sec. 3.3 states
    u, wu = grid(15)
    for om in (0.3, 0.7, 1.5):
        val = np.sum(wu / (1 + u ** 2 / om ** 2) ** 2)
        assert val == pytest.approx(np.pi * om / 4, rel=2e-7)
