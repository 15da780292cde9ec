"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(closed forms, limits, library routines, finite differences), independent of the
oracle's own formulas.  CPU only."""
import math

import numpy as np
import pytest

import oracle as o
from paper_2308_03140_gb300 import synthetic as syn

BETA, A_DAMP = 0.83, 6.0


def rand_r(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v) * rng.uniform(1.5, 6.0)


def hessian_fd(phi, r, h=1e-4):
    """Central-difference Hessian of a scalar function of a 3-vector."""
    H = np.zeros((3, 3))
    E = np.eye(3) * h
    for a in range(3):
        for b in range(3):
            H[a, b] = (phi(r + E[a] + E[b]) - phi(r + E[a] - E[b])
                       - phi(r - E[a] + E[b]) + phi(r - E[a] - E[b])) / (4 * h * h)
    return H


# ---- frequency grid (Sec. 3.3) -------------------------------------------------------
def test_gauss_legendre_matches_numpy():
    for n in (1, 2, 5, 15, 24):
        x, w = o.gauss_legendre(n)
        xn, wn = np.polynomial.legendre.leggauss(n)
        assert np.max(np.abs(x - xn)) < 1e-14
        assert np.max(np.abs(w - wn)) < 1e-14


def test_casimir_polder_quadrature_single_oscillator():
    # (3/pi) int_0^inf alpha0^2/(1+u^2/w^2)^2 du = 3/4 w alpha0^2 exactly (Eq. osc-param).
    u, wu = o.freq_grid(15)
    assert u[0] == 0.0 and wu[0] == 0.0
    for om in (0.3, 0.6, 1.0, 2.0):
        a0 = 7.0
        quad = 3 / math.pi * np.sum(wu[1:] * (a0 / (1 + u[1:] ** 2 / om ** 2)) ** 2)
        assert abs(quad / (0.75 * om * a0 ** 2) - 1) < 2e-6
    # near the grid's own scale the rule is far better (exponential convergence, Sec. 3.3)
    om = 0.6
    quad = 3 / math.pi * np.sum(wu[1:] * (1 / (1 + u[1:] ** 2 / om ** 2)) ** 2)
    assert abs(quad / (0.75 * om) - 1) < 1e-9


# ---- dipole tensors (Eqs. dipole, tgg, terfc) ----------------------------------------
def test_T_bare_is_minus_hessian_of_coulomb():
    rng = np.random.default_rng(1)
    for _ in range(5):
        r = rand_r(rng)
        H = hessian_fd(lambda x: 1 / np.linalg.norm(x), r)
        assert np.allclose(o.T_bare(r), -H, rtol=0, atol=2e-7 * np.abs(H).max() + 1e-9)


def test_T_gg_is_minus_hessian_of_gaussian_potential():
    rng = np.random.default_rng(2)
    for _ in range(5):
        r, s = rand_r(rng), rng.uniform(0.8, 3.0)
        H = hessian_fd(lambda x: math.erf(np.linalg.norm(x) / s) / np.linalg.norm(x), r)
        assert np.allclose(o.T_gg(r, s), -H, rtol=0, atol=2e-7 * np.abs(H).max() + 1e-9)


def test_T_erfc_is_minus_hessian_of_screened_potential():
    rng = np.random.default_rng(3)
    for _ in range(5):
        r, g = rand_r(rng), rng.uniform(0.1, 0.8)
        H = hessian_fd(lambda x: math.erfc(g * np.linalg.norm(x)) / np.linalg.norm(x), r)
        assert np.allclose(o.T_erfc(r, g), -H, rtol=0, atol=2e-7 * np.abs(H).max() + 1e-9)


def test_tensor_limits_and_split():
    rng = np.random.default_rng(4)
    for _ in range(5):
        r = rand_r(rng)
        T = o.T_bare(r)
        assert np.allclose(o.T_gg(r, 1e-3), T, rtol=1e-13, atol=1e-15)       # sigma -> 0
        assert np.allclose(o.T_erfc(r, 1e-7), T, rtol=1e-10, atol=1e-15)      # gamma -> 0
        s = rng.uniform(0.8, 3.0)
        # erf(r/s)/r = 1/r - erfc(r/s)/r
        assert np.allclose(o.T_gg(r, s), T - o.T_erfc(r, 1 / s), rtol=1e-12, atol=1e-15)
        assert abs(np.trace(T)) < 1e-14 * np.abs(T).max()     # bare T is traceless
        assert np.allclose(o.T_gg(r, s), o.T_gg(r, s).T)
    # bare tensor along z: diag(1, 1, -2)/R^3
    R = 3.7
    assert np.allclose(o.T_bare([0, 0, R]), np.diag([1, 1, -2]) / R ** 3, atol=1e-16)


def test_tensor_derivatives_fd():
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(4):
        r, s = rand_r(rng), rng.uniform(0.8, 3.0)
        d_bare = o.T_bare_deriv(r)
        d_gg, d_s = o.T_gg_deriv(r, s)
        for c in range(3):
            e = np.zeros(3); e[c] = h
            fd = (o.T_bare(r + e) - o.T_bare(r - e)) / (2 * h)
            assert np.allclose(d_bare[c], fd, atol=1e-8 * np.abs(fd).max() + 1e-12)
            fd = (o.T_gg(r + e, s) - o.T_gg(r - e, s)) / (2 * h)
            assert np.allclose(d_gg[c], fd, atol=1e-8 * np.abs(fd).max() + 1e-12)
        fd = (o.T_gg(r, s + h) - o.T_gg(r, s - h)) / (2 * h)
        scale = max(np.abs(fd).max(), np.abs(o.T_gg(r, s)).max())   # FD roundoff ~ eps |T| / h
        assert np.allclose(d_s, fd, atol=1e-8 * scale)


def test_fermi_damping_limits():
    assert o.fermi(0.83 * 7.0, 7.0, 0.83, 6.0) == pytest.approx(0.5, abs=1e-15)   # eta = 1
    assert o.fermi(1e3, 7.0, 0.83, 6.0) == pytest.approx(1.0, abs=1e-15)
    assert o.fermi(1e-3, 7.0, 0.83, 20.0) < 1e-8


# ---- dense linear algebra --------------------------------------------------------------
def test_gauss_jordan_and_jacobi_vs_numpy():
    rng = np.random.default_rng(6)
    for n in (1, 3, 17, 48):
        A = rng.normal(size=(n, n)); A = A + A.T + 2 * n * np.eye(n)
        Ai = o.inverse(A)
        assert np.allclose(Ai, np.linalg.inv(A), rtol=1e-12, atol=1e-14)
        assert np.allclose(A @ Ai, np.eye(n), atol=1e-12)
        lam, V = o.eigh(A)
        assert np.allclose(np.sort(lam), np.linalg.eigvalsh(A), rtol=1e-13, atol=1e-12)
        assert np.allclose(A @ V, V * lam, atol=1e-10)
        assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)


# ---- screening (Eqs. scs, contraction) -----------------------------------------------
def test_two_atom_scs_closed_form():
    # per axis the 6x6 system splits into 2x2 blocks [[1/a1, t],[t, 1/a2]]; the row sum of
    # the inverse of the first row is (1/a2 - t)/(1/(a1 a2) - t^2).
    R = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 4.2]])
    a0, om, rv = np.array([6.0, 9.0]), np.array([0.5, 0.8]), np.array([3.2, 3.6])
    u, _ = o.freq_grid(15)
    ab = o.scs(R, a0, om, rv, BETA, A_DAMP, 15)
    for k in (0, 3, 9, 15):
        al = a0 / (1 + u[k] ** 2 / om ** 2)
        s = math.hypot(*[(math.sqrt(2 / math.pi) * x / 3) ** (1 / 3) for x in al])
        f = o.fermi(4.2, rv.sum(), BETA, A_DAMP)
        t = np.diag((1 - f) * o.T_gg([0, 0, 4.2], s))
        det = 1 / (al[0] * al[1]) - t ** 2
        ref1 = np.mean((1 / al[1] - t) / det)
        ref2 = np.mean((1 / al[0] - t) / det)
        assert ab[k, 0] == pytest.approx(ref1, rel=1e-13)
        assert ab[k, 1] == pytest.approx(ref2, rel=1e-13)


def test_isolated_atoms_are_unscreened():
    # atoms 1e3 bohr apart: alpha_bar = alpha, C6bar = 3/4 w a0^2 up to quadrature error.
    R = np.array([[0.0, 0, 0], [1e3, 0, 0], [0, 1e3, 0]])
    a0, om, rv = np.array([5.0, 8.0, 11.0]), np.array([0.45, 0.6, 0.9]), np.array([3.1, 3.5, 3.9])
    ab = o.scs(R, a0, om, rv)
    u, _ = o.freq_grid(15)
    al = a0[None, :] / (1 + u[:, None] ** 2 / om[None, :] ** 2)
    assert np.allclose(ab, al, rtol=1e-8)
    rc, (abar0, c6, ombar, rbar) = o.screened_params(ab, a0, rv)
    assert rc == o.OK
    assert np.allclose(c6, 0.75 * om * a0 ** 2, rtol=2e-6)
    assert np.allclose(rbar, rv, rtol=1e-8)


# ---- MBD energy (Eqs. q-matrix, mbd-energy, pairwise) -------------------------------
def two_osc_energy(a, w, R, g):
    """Exact energy of two coupled isotropic oscillators along z (per-axis 2x2 modes)."""
    E = 0.0
    for t in (g / R ** 3, g / R ** 3, -2 * g / R ** 3):
        m = 0.5 * (w[0] ** 2 + w[1] ** 2)
        d = math.sqrt((0.5 * (w[0] ** 2 - w[1] ** 2)) ** 2 + w[0] ** 2 * w[1] ** 2 * a[0] * a[1] * t * t)
        E += 0.5 * (math.sqrt(m + d) + math.sqrt(m - d))
    return E - 1.5 * (w[0] + w[1])


def test_two_oscillator_closed_form():
    for R, a, w, rd in [(5.0, (8.0, 5.0), (0.5, 0.9), (3.0, 3.4)),
                        (7.5, (11.0, 11.0), (0.7, 0.7), (3.7, 3.7)),
                        (4.0, (4.0, 12.0), (2.0, 0.1), (1.0, 1.0))]:
        pos = np.array([[0, 0, 0], [0, 0, R]], float)
        g = o.fermi(R, sum(rd), BETA, A_DAMP)
        E = o.mbd_energy(pos, np.array(a), np.array(w), np.array(rd), BETA, A_DAMP)
        # E is a difference of terms of size 3/2 sum(w): roundoff is relative to those
        assert abs(E - two_osc_energy(a, w, R, g)) < 50 * 2.2e-16 * 1.5 * sum(w)
    # identical atoms: (w/2) sum_a (sqrt(1 + a t_a) + sqrt(1 - a t_a) - 2)
    R, a, w = 6.0, 9.0, 0.6
    pos = np.array([[0, 0, 0], [0, 0, R]], float)
    E = o.mbd_energy(pos, np.array([a, a]), np.array([w, w]), np.array([1e-3, 1e-3]), BETA, A_DAMP)
    ref = sum(w / 2 * (math.sqrt(1 + a * t) + math.sqrt(1 - a * t) - 2)
              for t in (1 / R ** 3, 1 / R ** 3, -2 / R ** 3))
    assert abs(E - ref) < 50 * 2.2e-16 * 3 * w


def test_second_order_limit_is_pairwise():
    # E(lambda alpha)/lambda^2 -> -sum_{i<j} C6ij f / R^6, f = R^6/6 Tr(T_lr^2) = g^2 (Eq. pairwise)
    sy = syn.cube_cluster(6, 12.0, 3.0, seed=11)
    R, a0, om, rd = sy.coords, sy.alpha0_ref, 4 * sy.c6_ref / (3 * sy.alpha0_ref ** 2), sy.rvdw_ref
    E2 = 0.0
    for i in range(6):
        for j in range(i + 1, 6):
            d = np.linalg.norm(R[j] - R[i])
            c6 = 1.5 * a0[i] * a0[j] / (1 / om[i] + 1 / om[j])
            g = o.fermi(d, rd[i] + rd[j], BETA, A_DAMP)
            E2 -= c6 * g * g / d ** 6
    ests = []
    for lam in (1e-2, 5e-3):   # smaller lambda drowns E in the roundoff of 3/2 sum(w)
        ests.append(o.mbd_energy(R, lam * a0, om, rd, BETA, A_DAMP) / lam ** 2)
    # the third-order term is O(lambda); Richardson removes it
    rich = 2 * ests[1] - ests[0]
    assert rich == pytest.approx(E2, rel=2e-6)
    assert ests[0] == pytest.approx(E2, rel=2e-4)
    assert not ests[0] == pytest.approx(E2, rel=1e-6)   # the many-body correction is visible


def test_catastrophe_detected():
    # alpha t_z = -2 alpha/R^3 < -1 with no damping: Q has a negative eigenvalue (Sec. 2.1)
    pos = np.array([[0, 0, 0], [0, 0, 2.5]], float)
    with pytest.raises(o.OracleError) as e:
        o.mbd_energy(pos, np.array([50.0, 50.0]), np.array([0.5, 0.5]), np.array([0.05, 0.05]))
    assert e.value.code == o.ERR_NEG_EIGENVALUE


def test_dense_literal_cluster_gives_negative_screened_alpha():
    sy = syn.fcc_jitter_cluster(60, density=0.08, seed=1099)
    with pytest.raises(o.OracleError) as e:
        o.mbd_rsscs_energy(*o.system_args(sy))
    assert e.value.code == o.ERR_SCS_NEG_ALPHA


def test_energy_invariances():
    sy = syn.cube_cluster(7, 9.0, 2.5, seed=12)
    args = list(o.system_args(sy))
    E = o.mbd_rsscs_energy(*args)
    th = 0.7
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(1.1), -math.sin(1.1)], [0, math.sin(1.1), math.cos(1.1)]])
    moved = sy.coords @ (Rz @ Rx).T + np.array([3.0, -2.0, 11.0])
    assert o.mbd_rsscs_energy(moved, *args[1:]) == pytest.approx(E, rel=1e-12)
    perm = np.random.default_rng(0).permutation(7)
    assert o.mbd_rsscs_energy(*[x[perm] for x in args]) == pytest.approx(E, rel=1e-12)


# ---- gradients (Eqs. mbd-gradient, scs-gradient) -------------------------------------
@pytest.fixture(scope="module")
def small_grad():
    sy = syn.cube_cluster(5, 7.0, 2.5, seed=7)
    args = list(o.system_args(sy))
    fwd = o.mbd_rsscs_gradient(*args, mode="forward")
    adj = o.mbd_rsscs_gradient(*args, mode="adjoint")
    return args, fwd, adj


def test_gradient_forward_equals_adjoint(small_grad):
    _, (E1, gR1, gp1), (E2, gR2, gp2) = small_grad
    assert E1 == E2
    assert np.allclose(gR1, gR2, rtol=1e-10, atol=1e-15)
    assert np.allclose(gp1, gp2, rtol=1e-10, atol=1e-15)


def test_gradient_central_differences(small_grad):
    args, _, (E, gR, gp) = small_grad
    h = 1e-4
    for i in range(len(args[0])):
        for c in range(3):
            Rp, Rm = args[0].copy(), args[0].copy()
            Rp[i, c] += h; Rm[i, c] -= h
            fd = (o.mbd_rsscs_energy(Rp, *args[1:]) - o.mbd_rsscs_energy(Rm, *args[1:])) / (2 * h)
            assert abs(fd - gR[i, c]) < 1e-9
    for k in range(4):
        for i in range(len(args[0])):
            a = [x.copy() for x in args]
            hh = 1e-5 * a[k + 1][i]
            a[k + 1][i] += hh; Ep = o.mbd_rsscs_energy(*a)
            a[k + 1][i] -= 2 * hh; Em = o.mbd_rsscs_energy(*a)
            assert abs((Ep - Em) / (2 * hh) - gp[k, i]) < 1e-8 * max(1.0, abs(gp[k, i]))


def test_gradient_invariances(small_grad):
    args, _, (E, gR, gp) = small_grad
    assert np.abs(gR.sum(0)).max() < 1e-15          # translation
    torque = np.cross(args[0], gR).sum(0)
    assert np.abs(torque).max() < 1e-14             # rotation


def test_gradient_from_dense_steps_equals_the_adjoint_gradient():
    # the 2000-atom reference gradient takes the oracle's adjoint pieces with LAPACK dense steps;
    # on a small cluster it must equal the oracle's own gradient (Gauss-Jordan, Jacobi)
    sy = syn.cube_cluster(10, 11.0, 2.5, seed=77)
    args = o.system_args(sy)
    E_ref, gR_ref, gp_ref = o.mbd_rsscs_gradient(*args, mode="adjoint")
    R, a0r, c6r, rr, v = args
    a0, om, rv = o.ts_scaling(a0r, c6r, rr, v)
    u, _ = o.freq_grid(15)
    n = 3 * sy.n_atoms
    E3 = np.zeros((n, 3))
    for c in range(3):
        E3[c::3, c] = 1.0
    Ms = [o.scs_matrix(R, o.dyn_alpha(a0, om, u[k]), rv) for k in range(16)]
    X = np.array([np.linalg.solve(M, E3) for M in Ms])
    ab = (X[:, 0::3, 0] + X[:, 1::3, 1] + X[:, 2::3, 2]) / 3.0
    rc, (abar0, c6bar, ombar, rbar) = o.screened_params(ab, a0, rv)
    lam, C = np.linalg.eigh(o.mbd_q(R, abar0, ombar, rbar))
    Z = (C / np.sqrt(lam)) @ C.T
    gR, gp = o.gradient_from_dense_steps(R, a0r, c6r, rr, v, ab, X, Z, lambda k, H: np.linalg.solve(Ms[k], H))
    # LAPACK against Jacobi / Gauss-Jordan: ~1e-11 of the largest component (rounding of Z and
    # of the solves, through the cancellations of the force sums)
    assert np.allclose(gR, gR_ref, rtol=0, atol=1e-9 * np.abs(gR_ref).max())
    for k in range(4):
        assert np.allclose(gp[k], gp_ref[k], rtol=0, atol=1e-9 * np.abs(gp_ref[k]).max())
