"""Pins of the TS pairwise oracle (oracle/ts_pairwise.py; Secs. 2.6 and 2.7, Eqs. pairwise,
ts-scaling, fermi-damping, ts-ewald): closed forms, the Casimir-Polder quadrature of the combination
rule, central differences, the kernels of the Ewald split by numerical integration, gamma
invariance and the plain lattice sum.  CPU only."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import gammainc

import oracle as o
from oracle import ts_pairwise as T

S_R = 0.94


def test_two_atoms_closed_form():
    a0ref, c6ref, rref, v = np.array([9.0, 6.0]), np.array([40.0, 12.0]), np.array([3.6, 3.2]), np.array([0.8, 0.9])
    d = 7.3
    R = np.array([[0.0, 0.0, 0.0], [0.0, d, 0.0]])
    a = a0ref * v
    w = 4 * c6ref / (3 * a0ref ** 2)
    rv = rref * np.cbrt(v)
    c6 = 1.5 * a[0] * a[1] / (1 / w[0] + 1 / w[1])
    f = 1 / (1 + math.exp(-20 * (d / (S_R * (rv[0] + rv[1])) - 1)))
    assert T.ts_energy(R, a0ref, c6ref, rref, v, S_R) == pytest.approx(-c6 * f / d ** 6, rel=1e-14, abs=0)
    # homonuclear C6 scales as v^2 (Eq. ts-scaling)
    C6 = T.c6_matrix(*T.ts_params(a0ref, c6ref, rref, v)[:2])
    assert np.allclose(np.diag(C6), c6ref * v ** 2, rtol=1e-14)


def test_combination_rule_is_casimir_polder():
    # C6_ij = 3/pi int_0^inf alpha_i(iu) alpha_j(iu) du for single oscillators, on a fine grid
    a, w = np.array([9.0, 5.5]), np.array([0.45, 0.8])
    u, wu = o.freq_grid(60)
    al = a[:, None] / (1 + u[None, :] ** 2 / w[:, None] ** 2)
    cp = 3 / math.pi * np.sum(wu * al[0] * al[1])
    assert T.c6_matrix(a, w)[0, 1] == pytest.approx(cp, rel=1e-12, abs=0)


def test_finite_gradients_central_differences():
    rng = np.random.default_rng(7)
    N = 5
    R = rng.uniform(0, 9, (N, 3))
    p = [rng.uniform(4, 12, N), rng.uniform(5, 50, N), rng.uniform(3, 4, N), rng.uniform(0.7, 1.0, N)]
    E, gR, gp = T.ts_energy(R, *p, S_R, grad=True)
    h = 1e-6
    for k in range(N):
        for c in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[k, c] += h
            Rm[k, c] -= h
            fd = (T.ts_energy(Rp, *p, S_R) - T.ts_energy(Rm, *p, S_R)) / (2 * h)
            assert fd == pytest.approx(gR[k, c], rel=1e-6, abs=1e-13)
    for q in range(4):
        for k in range(N):
            hh = 1e-6 * p[q][k]
            up = [x.copy() for x in p]
            dn = [x.copy() for x in p]
            up[q][k] += hh
            dn[q][k] -= hh
            fd = (T.ts_energy(R, *up, S_R) - T.ts_energy(R, *dn, S_R)) / (2 * hh)
            assert fd == pytest.approx(gp[q, k], rel=1e-6, abs=1e-13), (q, k)
    assert np.abs(gR.sum(0)).max() < 1e-15


def test_ewald_split_kernels():
    g = 0.3
    # long-range part of the split: LR(r) = 1/2 int_0^{g^2} t^2 e^{-r^2 t} dt = P(3, g^2 r^2) / r^6
    # (regularized lower incomplete gamma); real-space kernel + LR = 1/r^6
    def lr(r):
        return gammainc(3, g * g * r * r) / r ** 6 if r > 0 else g ** 6 / 6
    for r in (0.7, 2.0, 5.5, 11.0):
        direct = 0.5 * quad(lambda t: t * t * math.exp(-r * r * t), 0, g * g, epsabs=0, epsrel=1e-13)[0]
        assert lr(r) == pytest.approx(direct, rel=1e-12)
        assert g ** 6 * T.phi_r(g * r) + lr(r) == pytest.approx(1 / r ** 6, rel=1e-11)
    # reciprocal kernel = 3D Fourier transform of LR: 4 pi / G int_0^inf LR(r) r sin(G r) dr
    for G in (0.2, 0.6, 1.4):
        # infinite-range sine quadrature uses the absolute tolerance only; the integral is ~1e-4
        ft = 4 * math.pi / G * quad(lambda r: lr(r) * r, 0, np.inf, weight="sin", wvar=G, epsabs=1e-16,
                                    limlst=200)[0]
        assert g ** 3 * T.phi_k(G / g) == pytest.approx(ft, rel=1e-8)
    ft0 = 4 * math.pi * quad(lambda r: lr(r) * r * r, 0, np.inf, epsabs=0, epsrel=1e-12)[0]
    assert g ** 3 * T.phi_k(0.0) == pytest.approx(ft0, rel=1e-9)
    assert T.phi_k(0.0) == pytest.approx(math.pi ** 1.5 / 3, rel=1e-15)
    # the self correction is the long-range part at r = 0
    assert lr(1e-6) == pytest.approx(g ** 6 / 6, rel=1e-9)


@pytest.fixture(scope="module")
def cell():
    rng = np.random.default_rng(3)
    A = np.array([[9.0, 0, 0], [1.0, 8.5, 0], [-0.6, 0.8, 9.5]])
    N = 4
    R = rng.uniform(0, 1, (N, 3)) @ A
    p = [rng.uniform(4, 12, N), rng.uniform(5, 50, N), rng.uniform(3, 4, N), rng.uniform(0.7, 1, N)]
    return R, A, p


def test_periodic_ewald_gamma_invariance_and_direct_sum(cell):
    R, A, p = cell
    E1 = T.ts_energy_periodic(R, A, *p, gamma=0.25, rc=6.5 / 0.25, kc=10 * 0.25, s_r=S_R)
    E2 = T.ts_energy_periodic(R, A, *p, gamma=0.35, rc=6.5 / 0.35, kc=10 * 0.35, s_r=S_R)
    assert E2 == pytest.approx(E1, rel=1e-9, abs=0)
    Ed = T.ts_energy_periodic_direct(R, A, *p, r_big=300.0, s_r=S_R)   # absolutely convergent sum
    assert Ed == pytest.approx(E1, rel=1e-8, abs=0)


def test_periodic_large_box_limit():
    # a 3-atom molecule in a cubic box of edge L: E_box - E_finite is the image energy
    # -1/2 sum_ij C6_ij sum_{n != 0} f/|R_ij + n L|^6, here summed over |n L| < 8 L plus the
    # continuum tail 4 pi / (3 L^3 (8 L)^3); it falls off about as L^-6
    R = np.array([[0.0, 0.0, 0.0], [7.0, 0.0, 0.0], [0.0, 7.5, 1.0]])
    p = [np.array([9.0, 6.0, 11.0]), np.array([40.0, 12.0, 30.0]), np.array([3.6, 3.2, 3.9]), np.array([0.8, 0.9, 0.85])]
    a0, om, rv = T.ts_params(*p)
    C6 = T.c6_matrix(a0, om)
    E_fin = T.ts_energy(R, *p, S_R)
    ns = np.array(np.meshgrid(*[np.arange(-8, 9)] * 3, indexing="ij")).reshape(3, -1).T
    ns = ns[(np.linalg.norm(ns, axis=1) > 0) & (np.linalg.norm(ns, axis=1) < 8)]
    diffs = []
    for L in (40.0, 80.0):
        E_box = T.ts_energy_periodic(R, np.eye(3) * L, *p, gamma=6.5 / 30, rc=30.0, kc=10 * 6.5 / 30, s_r=S_R)
        img = 0.0
        for i in range(3):
            for j in range(3):
                d = np.linalg.norm(R[j] - R[i] + ns * L, axis=1)
                f = 1 / (1 + np.exp(-20 * (d / (S_R * (rv[i] + rv[j])) - 1)))
                img += -0.5 * C6[i, j] * (np.sum(f / d ** 6) + 4 * math.pi / (3 * L ** 3 * (8 * L) ** 3))
        assert E_box - E_fin == pytest.approx(img, rel=1e-4)
        diffs.append(E_box - E_fin)
    assert diffs[0] < 0 and abs(diffs[0]) < 1e-3 * abs(E_fin)
    assert 50 < diffs[0] / diffs[1] < 80


def test_periodic_gradients_central_differences(cell):
    # tight cutoffs so that no image or G vector crosses them within the difference step
    R, A, p = cell
    g, rc, kc = 0.3, 7 / 0.3, 12 * 0.3
    E, gR, gA, gp = T.ts_energy_periodic(R, A, *p, g, rc, kc, s_r=S_R, grad=True)
    assert E == pytest.approx(T.ts_energy_periodic(R, A, *p, g, rc, kc, s_r=S_R), rel=1e-15, abs=0)

    def en(R_=R, A_=A, p_=p):
        return T.ts_energy_periodic(R_, A_, *p_, g, rc, kc, s_r=S_R)
    h = 1e-5
    for i in range(len(R)):
        for c in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, c] += h
            Rm[i, c] -= h
            assert (en(R_=Rp) - en(R_=Rm)) / (2 * h) == pytest.approx(gR[i, c], abs=1e-8 * np.abs(gR).max())
    for f in range(3):
        for c in range(3):
            Ap, Am = A.copy(), A.copy()
            Ap[f, c] += h
            Am[f, c] -= h
            assert (en(A_=Ap) - en(A_=Am)) / (2 * h) == pytest.approx(gA[f, c], abs=1e-8 * np.abs(gA).max())
    for q in range(4):
        for k in range(len(R)):
            hh = 1e-6 * p[q][k]
            up = [x.copy() for x in p]
            dn = [x.copy() for x in p]
            up[q][k] += hh
            dn[q][k] -= hh
            assert (en(p_=up) - en(p_=dn)) / (2 * hh) == pytest.approx(gp[q, k], abs=1e-7 * np.abs(gp[q]).max())
    assert np.abs(gR.sum(0)).max() < 1e-15


def test_periodic_lattice_gradient_is_the_direct_sum_virial(cell):
    # homogeneous strain R -> R (I + e), A -> A (I + e): dE/de = R^T gR + A^T gA, and for the
    # plain lattice sum of -1/2 C6 f/r^6 the same derivative is the virial
    # -1/2 sum C6 F'(r) r r^T / r (F = f/r^6) to r_big plus its continuum tail
    # -1/2 C6 (-8 pi / (3 Omega r_big^3)) I; this route has no Ewald split at all
    R, A, p = cell
    _, gR, gA, _ = T.ts_energy_periodic(R, A, *p, 0.3, 7 / 0.3, 12 * 0.3, s_r=S_R, grad=True)
    strain = R.T @ gR + A.T @ gA
    a0, om, rv = T.ts_params(*p)
    C6 = T.c6_matrix(a0, om)
    Om = abs(np.linalg.det(A))
    rb = 150.0
    shifts = T._images(A, rb)
    vir = np.zeros((3, 3))
    for i in range(len(R)):
        for j in range(len(R)):
            v = R[j] + shifts - R[i]
            r = np.linalg.norm(v, axis=1)
            s = (r > 1e-12) & (r < rb)
            v, r = v[s], r[s]
            f, dfr, _ = T.fermi(r, rv[i] + rv[j], S_R)
            vir += -0.5 * C6[i, j] * (((dfr / r ** 6 - 6 * f / r ** 7) / r)[:, None] * v).T @ v
            vir += -0.5 * C6[i, j] * (-8 * math.pi / (3 * Om * rb ** 3)) * np.eye(3)
    assert np.abs(strain - vir).max() < 1e-6 * np.abs(vir).max()
    assert np.allclose(strain, strain.T, atol=1e-12 * np.abs(strain).max())
