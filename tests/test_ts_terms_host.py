"""The periodic TS pair arithmetic of the CUDA library (csrc/ts_terms.cuh: the functions the
kernels k_ts_gtable and k_ts_periodic call) compiled for the host and summed over all ordered
pairs (tests/ts_terms_host.cu), against the oracle (oracle/ts_pairwise.py, itself pinned in
test_oracle_ts_pins.py): energy, coordinate and lattice gradients and the gradients with
respect to the TS-scaled oscillators.  This checks the kernel's per-pair terms, signs and
factors without a GPU; the launch itself is checked against the oracle in test_gpu_ts.py.
CPU only."""
import ctypes as C
import math
import os
import subprocess

import numpy as np
import pytest

from oracle import ts_pairwise as T
from paper_2308_03140_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2308_03140_gb300", "csrc")
S_R = 0.94


@pytest.fixture(scope="module")
def host():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "ts_terms_host.so")
    src = os.path.join(HERE, "ts_terms_host.cu")
    deps = [src] + [os.path.join(CSRC, f) for f in ("ts_terms.cuh", "internal.h")]
    if not os.path.exists(so) or any(os.path.getmtime(d) > os.path.getmtime(so) for d in deps):
        cmd = [build.nvcc(), *build.ARCH, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
               f"-I{CSRC}", src, "-o", so]
        res = subprocess.run(cmd, capture_output=True, text=True)
        assert res.returncode == 0, res.stderr
    lib = C.CDLL(so)
    lib.ts_host_periodic.restype = C.c_int
    return lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def run_host(lib, R, A, a0, om, rv, gamma, rc, kc, Gmax):
    R = np.ascontiguousarray(R, float)
    A = np.ascontiguousarray(A, float)
    Ainv = np.ascontiguousarray(np.linalg.inv(A))
    B = np.ascontiguousarray(2 * math.pi * Ainv.T)
    N = len(R)
    # every G = m B with |G| < Gmax; those with |G| >= kc carry zero weight, as in the
    # library's list (which serves all Bloch vectors of a k-grid)
    mm = [int(math.ceil(Gmax * np.linalg.norm(A[c]) / (2 * math.pi))) + 1 for c in range(3)]
    ms = np.array(np.meshgrid(*[np.arange(-m, m + 1) for m in mm], indexing="ij")).reshape(3, -1).T
    G = ms @ B
    G = np.ascontiguousarray(G[np.linalg.norm(G, axis=1) < Gmax])
    out = [np.zeros(N) for _ in range(4)] + [np.zeros((N, 3)), np.zeros(9)]
    bad = lib.ts_host_periodic(N, _p(R), _p(A), _p(Ainv), _p(B), C.c_double(abs(np.linalg.det(A))),
                               C.c_double(gamma), C.c_double(rc), C.c_double(kc), _p(a0), _p(om), _p(rv),
                               C.c_double(S_R), len(G), _p(G), *[_p(x) for x in out])
    eatom, ga0, gom, grv, gR, gA = out
    return bad, eatom.sum(), ga0, gom, grv, gR, gA.reshape(3, 3)


def oracle_parts(R, A, p, gamma, rc, kc):
    a0, om, rv = T.ts_params(*p)
    C6 = T.c6_matrix(a0, om)
    s = T.ewald_inverse_r6(R, A, gamma, rc, kc) - T.damped_away_sum(R, A, rv, S_R, rc)
    gR, gA, grv = T._periodic_geometry_grad(R, A, C6, rv, gamma, rc, kc, S_R, T.D_TS)
    ga0, gom = T._c6_chain(a0, om, -0.5 * s)
    return -0.5 * float(np.sum(C6 * s)), ga0, gom, grv, gR, gA


def scaled(p):
    # the TS scaling written out here (Eq. ts-scaling), so that neither side feeds the other
    a0ref, c6ref, rref, v = p
    return a0ref * v, 4 * c6ref / (3 * a0ref ** 2), rref * np.cbrt(v)


@pytest.mark.parametrize("case", ["small_cell", "dilute_cell"])
def test_host_pair_terms_match_the_oracle(host, case):
    if case == "small_cell":
        rng = np.random.default_rng(3)
        A = np.array([[9.0, 0, 0], [1.0, 8.5, 0], [-0.6, 0.8, 9.5]])
        N, gamma = 4, 0.3
    else:
        rng = np.random.default_rng(21)
        A = np.array([[14.0, 0, 0], [-1.2, 13.1, 0], [0.9, 1.4, 15.2]])
        N, gamma = 9, 0.22
    R = rng.uniform(0, 1, (N, 3)) @ A
    p = [rng.uniform(4, 12, N), rng.uniform(5, 50, N), rng.uniform(3, 4, N), rng.uniform(0.7, 1.0, N)]
    rc, kc = 6.5 / gamma, 10.5 * gamma
    bad, E, ga0, gom, grv, gR, gA = run_host(host, R, A, *scaled(p), gamma, rc, kc, 1.2 * kc)
    E_o, ga0_o, gom_o, grv_o, gR_o, gA_o = oracle_parts(R, A, p, gamma, rc, kc)
    assert bad == 0
    assert E == pytest.approx(E_o, rel=1e-12, abs=0)
    for got, ref in ((ga0, ga0_o), (gom, gom_o), (grv, grv_o), (gR, gR_o), (gA, gA_o)):
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_host_flags_coincident_atoms(host):
    A = np.eye(3) * 9.0
    R = np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 10.0]])     # the second atom is an image of the first
    ones = np.ones(2)
    bad, *_ = run_host(host, R, A, 8 * ones, 0.4 * ones, 3.5 * ones, 0.3, 20.0, 3.0, 3.0)
    assert bad == 1


def test_host_pair_terms_full_cell_properties(host):
    # the 256-atom triclinic cell at the two Ewald splits of the GPU property test: the
    # kernel's arithmetic gives the same energy and gradients (7e-14 and 2e-12 here), forces
    # that sum to zero and a symmetric strain derivative
    from paper_2308_03140_gb300 import synthetic as syn
    c = syn.workload("cell256")
    p = (c.alpha0_ref, c.c6_ref, c.rvdw_ref, c.ratio)
    res = [run_host(host, c.coords, c.lattice, *scaled(p), g, 6.5 / g, 10.5 * g, 10.5 * g) for g in (0.2, 0.26)]
    (b1, E1, *g1), (b2, E2, *g2) = res
    assert b1 == 0 and b2 == 0
    assert E2 == pytest.approx(E1, rel=1e-12, abs=0)
    for x, y in zip(g1, g2):
        assert np.abs(x - y).max() <= 1e-10 * np.abs(x).max()
    gR, gA = g1[3], g1[4]
    assert np.abs(gR.sum(0)).max() <= 1e-13 * np.abs(gR).max()
    strain = c.coords.T @ gR + c.lattice.T @ gA
    assert np.abs(strain - strain.T).max() <= 1e-12 * np.abs(strain).max()
