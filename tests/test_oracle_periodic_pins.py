"""Pins of the periodic oracle (oracle/mbd_periodic.c) against what the mathematics fixes.

Sec. 2.2 (periodic boundary conditions) and the Ewald summation of the dipole tensor.
Each pin is chosen so that a plausible slip (a wrong phase sign, a missing self term, a wrong reciprocal
prefactor, a dropped image, a wrong lattice chain rule) fails it:
- gamma-invariance of the Ewald sum (phase, prefactor, self term, erfc numerator);
- Hermiticity and T(-q) = conj T(q);
- central differences of every analytic derivative;
- Brillouin-zone folding of a supercell, invariance under lattice translations;
- the large-cell limit of the periodic energy equals the finite oracle's energy, which is
  itself pinned by closed forms (test_oracle_pins.py).
All CPU; each test runs in about a second.
"""
import numpy as np
import pytest

from oracle import oracle as o

CELL = np.array([[8.0, 0.0, 0.0], [0.9, 7.6, 0.0], [-0.6, 0.7, 8.4]])
FRAC = np.array([[0.1, 0.2, 0.15], [0.55, 0.45, 0.6], [0.3, 0.8, 0.75]])


def params(N, seed=7):
    rng = np.random.default_rng(seed)
    return (rng.uniform(4, 12, N), rng.uniform(5, 50, N), rng.uniform(3, 4, N), rng.uniform(0.7, 1.0, N))


def ewald_set(gamma, rc=None):
    return gamma, (6.5 / gamma if rc is None else rc), 11.0 * gamma


def test_reciprocal_cell():
    B, vol = o.cell_reciprocal(CELL)
    assert np.allclose(CELL @ B.T, 2 * np.pi * np.eye(3), atol=1e-13)
    assert vol == pytest.approx(abs(np.linalg.det(CELL)), rel=1e-14)


def test_monkhorst_pack():
    k = o.monkhorst_pack([4, 4, 4])
    assert k.shape == (64, 3)
    assert set(np.round(k[:, 0], 12)) == {-0.375, -0.125, 0.125, 0.375}
    assert np.allclose(k.sum(0), 0.0)
    assert not np.any(np.all(np.abs(k) < 1e-12, axis=1))          # even grid: no Gamma point
    assert np.any(np.all(np.abs(o.monkhorst_pack([3, 3, 3])) < 1e-12, axis=1))


def test_T_erfc_derivative_vs_fd():
    r, g, h = np.array([1.3, -2.2, 0.7]), 0.4, 1e-6
    dT = o.T_erfc_deriv(r, g)
    for c in range(3):
        e = np.zeros(3); e[c] = h
        fd = (o.T_erfc(r + e, g) - o.T_erfc(r - e, g)) / (2 * h)
        assert np.abs(fd - dT[c]).max() < 1e-8 * np.abs(dT).max()


def test_ewald_gamma_invariance():
    """Eq. (ewald): the split parameter only moves terms between the two sums."""
    R = FRAC @ CELL
    kap = np.array([0.25, -0.125, 0.375])
    T1 = o.ewald_T(R, CELL, kap, *ewald_set(0.30))
    T2 = o.ewald_T(R, CELL, kap, *ewald_set(0.45))
    assert np.abs(T1 - T2).max() < 1e-10 * np.abs(T1).max()


def test_ewald_cutoff_convergence():
    R = FRAC @ CELL
    kap = np.array([0.125, 0.375, -0.375])
    T1 = o.ewald_T(R, CELL, kap, 0.35, 6.5 / 0.35, 11 * 0.35)
    T2 = o.ewald_T(R, CELL, kap, 0.35, 8.0 / 0.35, 14 * 0.35)
    assert np.abs(T1 - T2).max() < 1e-12 * np.abs(T1).max()


def test_ewald_hermitian_and_time_reversal():
    R = FRAC @ CELL
    kap = np.array([0.25, -0.125, 0.375])
    T = o.ewald_T(R, CELL, kap, *ewald_set(0.35))
    assert np.abs(T - T.conj().T).max() < 1e-15
    Tm = o.ewald_T(R, CELL, -kap, *ewald_set(0.35))
    assert np.abs(Tm - T.conj()).max() < 1e-15


def test_ewald_lattice_translation():
    """With the phase on the full separation R_nij (reading of the reciprocal phase), moving an
    atom by a lattice vector only relabels the images: T(q) is unchanged, while a
    non-lattice shift of one atom does change it."""
    R = FRAC @ CELL
    kap = np.array([0.25, -0.125, 0.375])
    T = o.ewald_T(R, CELL, kap, *ewald_set(0.35))
    R2 = R.copy(); R2[2] += CELL[1] - 2 * CELL[0]
    assert np.abs(o.ewald_T(R2, CELL, kap, *ewald_set(0.35)) - T).max() < 1e-13 * np.abs(T).max()
    R3 = R.copy(); R3[2] += 0.5 * CELL[1]
    assert np.abs(o.ewald_T(R3, CELL, kap, *ewald_set(0.35)) - T).max() > 1e-3 * np.abs(T).max()


@pytest.mark.parametrize("same", [0, 1])
def test_tlr_block_derivatives_vs_fd(same):
    kap, g, rc, kc, S, h = np.array([0.25, -0.125, 0.375]), 0.3, 20.0, 3.0, 5.5, 1e-5
    x = np.zeros(3) if same else (FRAC[1] - FRAC[0]) @ CELL
    T, dx, dS, dA = o.tlr_block(CELL, x, same, kap, g, rc, kc, rsum=S, derivs=True)
    blk = lambda A=CELL, x=x, S=S: o.tlr_block(A, x, same, kap, g, rc, kc, rsum=S)
    scale = np.abs(T).max()
    if not same:
        for d in range(3):
            e = np.zeros(3); e[d] = h
            assert np.abs((blk(x=x + e) - blk(x=x - e)) / (2 * h) - dx[d]).max() < 1e-8 * scale
    assert np.abs((blk(S=S + h) - blk(S=S - h)) / (2 * h) - dS).max() < 1e-8 * scale
    for c in range(3):
        for d in range(3):
            Ap, Am = CELL.copy(), CELL.copy()
            Ap[c, d] += h; Am[c, d] -= h
            assert np.abs((blk(A=Ap) - blk(A=Am)) / (2 * h) - dA[c, d]).max() < 1e-8 * scale


def test_hermitian_sqrt_vs_numpy():
    R = FRAC @ CELL
    Q = o.periodic_q(R, CELL, np.array([0.25, 0.25, -0.25]), np.array([5.0, 7.0, 9.0]),
                     np.array([0.6, 0.5, 0.7]), np.array([3.5, 3.3, 3.7]), *ewald_set(0.35))
    assert np.abs(Q - Q.conj().T).max() < 1e-15
    h, lam, Z = o.hermitian_sqrt(Q, want_z=True)
    w, U = np.linalg.eigh(Q)
    assert np.abs(lam - w).max() < 1e-13
    assert h == pytest.approx(0.5 * np.sqrt(w).sum(), rel=1e-14)
    assert np.abs(Z - (U * w ** -0.5) @ U.conj().T).max() < 1e-13


def test_periodic_scs_matrix_reduces_to_finite():
    """No image inside the cutoff: the Gamma-point SCS matrix is the finite one."""
    R = np.array([[0.0, 0.0, 0.0], [3.1, 0.4, -0.5], [0.9, 3.3, 1.2]]) + 5.0
    al, rv = np.array([6.0, 8.0, 5.0]), np.array([3.4, 3.6, 3.2])
    M = o.periodic_scs_matrix(R, np.eye(3) * 60.0, al, rv, rc=40.0)
    assert np.abs(M - o.scs_matrix(R, al, rv)).max() < 1e-15


def test_periodic_scs_matrix_images():
    """Self images: block (i,i) holds sum_{n != 0} (1 - f) T^GG(n A); the matrix is symmetric."""
    R = FRAC @ CELL
    al, rv = np.array([6.0, 8.0, 5.0]), np.array([3.4, 3.6, 3.2])
    M = o.periodic_scs_matrix(R, CELL, al, rv, rc=25.0)
    assert np.abs(M - M.T).max() < 1e-15
    s = np.sqrt(2) * (np.sqrt(2 / np.pi) * al[0] / 3) ** (1 / 3)
    blk = np.diag([1 / al[0]] * 3)
    for n in np.ndindex(9, 9, 9):
        r = (np.array(n) - 4) @ CELL
        d = np.linalg.norm(r)
        if 0 < d < 25.0:
            blk = blk + (1 - o.fermi(d, 2 * rv[0], 0.83, 6.0)) * o.T_gg(r, s)
    assert np.abs(M[:3, :3] - blk).max() < 1e-14


def test_energy_brillouin_zone_folding():
    """A 1x1x2 supercell on a 2x2x2 grid samples the same Bloch vectors as the cell on 2x2x4."""
    R = FRAC @ CELL
    p = params(3)
    set_ = ewald_set(0.35)
    E = o.periodic_rsscs_energy(R, CELL, o.monkhorst_pack([2, 2, 4]), *p, *set_)
    A2 = CELL.copy(); A2[2] *= 2
    R2 = np.vstack([R, R + CELL[2]])
    E2 = o.periodic_rsscs_energy(R2, A2, o.monkhorst_pack([2, 2, 2]), *[np.tile(x, 2) for x in p], *set_)
    assert E2 == pytest.approx(2 * E, rel=1e-10)


def test_energy_invariances():
    R = FRAC @ CELL
    p = params(3)
    kap = o.monkhorst_pack([2, 2, 2])
    E = o.periodic_rsscs_energy(R, CELL, kap, *p, *ewald_set(0.35, rc=20.0))
    R2 = R.copy(); R2[1] += CELL[0] - CELL[2]
    assert o.periodic_rsscs_energy(R2, CELL, kap, *p, *ewald_set(0.35, rc=20.0)) == pytest.approx(E, rel=1e-12)
    assert o.periodic_rsscs_energy(R + [0.3, -1.1, 0.7], CELL, kap, *p, *ewald_set(0.35, rc=20.0)) == \
        pytest.approx(E, rel=1e-12)
    # gamma only moves terms between the Ewald sums (cutoff of the damped sums held at 20 bohr)
    assert o.periodic_rsscs_energy(R, CELL, kap, *p, *ewald_set(0.5, rc=20.0)) == pytest.approx(E, rel=1e-10)


def test_energy_large_cell_limit_is_finite_energy():
    """A molecule in a cubic cell of edge L: E(L) = E_finite + c/L^3 + O(L^-6) (the dipolar
    image field); the extrapolation to L -> infinity recovers the finite oracle's energy."""
    R = np.array([[0.0, 0.0, 0.0], [3.1, 0.4, -0.5], [0.9, 3.3, 1.2]]) + 5.0
    p = params(3)
    Ef = o.mbd_rsscs_energy(R, *p)
    kap = np.array([[0.25, 0.25, 0.25]])
    Ls = np.array([40.0, 60.0, 80.0])
    Es = []
    for L in Ls:
        g = 4.5 / L
        Es.append(o.periodic_rsscs_energy(R, np.eye(3) * L, kap, *p, g, 6.5 / g, 10 * g))
    M = np.stack([np.ones(3), Ls ** -3, Ls ** -6], 1)
    E_inf = np.linalg.solve(M, np.array(Es))[0]
    assert abs(Es[0] - Ef) > 1e-7                       # the images do matter at L = 40
    assert abs(E_inf - Ef) < 5e-3 * abs(Es[0] - Ef)


def test_gradients_vs_central_differences():
    R = FRAC @ CELL
    p = params(3)
    kap = o.monkhorst_pack([2, 2, 2])
    set_ = ewald_set(0.35)
    E, gR, gA, gp = o.periodic_rsscs_gradient(R, CELL, kap, *p, *set_)
    en = lambda R_=R, A_=CELL, p_=p: o.periodic_rsscs_energy(R_, A_, kap, *p_, *set_)
    assert E == pytest.approx(en(), rel=1e-14)
    h = 1e-4
    for i in range(3):
        for d in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, d] += h; Rm[i, d] -= h
            assert (en(R_=Rp) - en(R_=Rm)) / (2 * h) == pytest.approx(gR[i, d], abs=1e-10)
    for c in range(3):
        for d in range(3):
            Ap, Am = CELL.copy(), CELL.copy()
            Ap[c, d] += h; Am[c, d] -= h
            assert (en(A_=Ap) - en(A_=Am)) / (2 * h) == pytest.approx(gA[c, d], abs=1e-10)
    for k in range(4):
        for i in range(3):
            pp = [x.copy() for x in p]
            hh = 1e-5 * pp[k][i]
            pp[k][i] += hh; Ep = en(p_=pp)
            pp[k][i] -= 2 * hh; Em = en(p_=pp)
            assert (Ep - Em) / (2 * hh) == pytest.approx(gp[k, i], abs=1e-9)
    assert np.abs(gR.sum(0)).max() < 1e-15                # translation invariance


def test_lattice_gradient_strain_identity():
    """With Cartesian positions fixed, a uniform scaling of everything (cell and atoms) by
    (1 + e) changes E at first order by e (sum_cd A_cd dE/dA_cd + sum_i R_i . dE/dR_i)."""
    R = FRAC @ CELL
    p = params(3)
    kap = o.monkhorst_pack([2, 2, 2])
    set_ = ewald_set(0.35)
    _, gR, gA, _ = o.periodic_rsscs_gradient(R, CELL, kap, *p, *set_)
    e = 1e-5
    Ep = o.periodic_rsscs_energy(R * (1 + e), CELL * (1 + e), kap, *p, *set_)
    Em = o.periodic_rsscs_energy(R * (1 - e), CELL * (1 - e), kap, *p, *set_)
    assert (Ep - Em) / (2 * e) == pytest.approx((CELL * gA).sum() + (R * gR).sum(), rel=1e-6)
