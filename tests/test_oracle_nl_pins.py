"""Pins of the MBD-NL oracle (oracle/mbd_oracle.c: orc_mbd_nl; Sec. 2.7, paragraph MBD-NL,
Eqs. mbd-nl-scaling, mbd-nl-rvdw) against hand-computed parameters, the closed form of two
coupled oscillators, central differences and invariances.  CPU only."""
import math

import numpy as np
import pytest

import oracle as o

BETA, A_DAMP = 0.83, 6.0

# alpha0_ref = 2^7 and 3^7 make alpha0_ref^(1/7) exact; ra = 0.9^3, 0.7^3 make ra^(1/3) exact
A0REF = np.array([128.0, 2187.0])
C6REF = np.array([30.0, 60.0])
RA = np.array([0.729, 0.343])
RW = np.array([1.25, 0.8])
ALPHA0 = np.array([128.0 * 0.729, 2187.0 * 0.343])
OMEGA = np.array([4 * 30.0 / (3 * 128.0 ** 2) * 1.25, 4 * 60.0 / (3 * 2187.0 ** 2) * 0.8])
RDAMP = np.array([2.5 * 2 * 0.9, 2.5 * 3 * 0.7])


def two_osc_energy(a, w, R, g):
    """Exact energy of two coupled isotropic oscillators along z (per-axis 2x2 modes of the
    coupled-oscillator matrix with coupling w_i w_j sqrt(a_i a_j) g T, T = diag(1, 1, -2)/R^3)."""
    E = 0.0
    for t in (g / R ** 3, g / R ** 3, -2 * g / R ** 3):
        m = 0.5 * (w[0] ** 2 + w[1] ** 2)
        d = math.sqrt((0.5 * (w[0] ** 2 - w[1] ** 2)) ** 2 + w[0] ** 2 * w[1] ** 2 * a[0] * a[1] * t * t)
        E += 0.5 * (math.sqrt(m + d) + math.sqrt(m - d))
    return E - 1.5 * (w[0] + w[1])


def test_nl_parametrization_closed_form():
    R = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 9.0]])
    _, par = o.mbd_nl(R, A0REF, C6REF, RA, RW, BETA, A_DAMP, detail=True)
    assert np.allclose(par[0], ALPHA0, rtol=1e-15, atol=0)
    assert np.allclose(par[1], OMEGA, rtol=1e-15, atol=0)
    assert np.allclose(par[2], [4.5, 5.25], rtol=1e-14, atol=0)


@pytest.mark.parametrize("d", [5.0, 7.5, 12.0])
def test_nl_two_atom_closed_form(d):
    R = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, d]])
    E = o.mbd_nl(R, A0REF, C6REF, RA, RW, BETA, A_DAMP)
    g = 1.0 / (1.0 + math.exp(-A_DAMP * (d / (BETA * (4.5 + 5.25)) - 1.0)))   # Fermi damping
    ref = two_osc_energy(ALPHA0, OMEGA, d, g)
    assert abs(E - ref) < 50 * 2.2e-16 * 1.5 * OMEGA.sum()
    assert E < 0


def _system(seed, N=5):
    rng = np.random.default_rng(seed)
    R = rng.uniform(0, 9, (N, 3))
    while min(np.linalg.norm(R[i] - R[j]) for i in range(N) for j in range(i)) < 2.5:
        R = rng.uniform(0, 9, (N, 3))
    return (R, rng.uniform(4, 12, N), rng.uniform(5, 50, N), rng.uniform(0.7, 1.0, N),
            rng.uniform(0.85, 1.2, N))


def test_nl_gradients_central_differences():
    R, a0, c6, ra, rw = _system(1)
    E, gR, gp = o.mbd_nl(R, a0, c6, ra, rw, BETA, A_DAMP, grad=True)
    # E (~1e-3 Ha) is a difference of terms of ~4 Ha taken through the Jacobi eigensolver, so
    # its roundoff (~1e-13) bounds the differences absolutely, as in the rsSCS pins
    h = 1e-4
    for k in range(R.shape[0]):
        for c in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[k, c] += h
            Rm[k, c] -= h
            fd = (o.mbd_nl(Rp, a0, c6, ra, rw, BETA, A_DAMP) - o.mbd_nl(Rm, a0, c6, ra, rw, BETA, A_DAMP)) / (2 * h)
            assert abs(fd - gR[k, c]) < 1e-9, (k, c)
    args = [a0, c6, ra, rw]
    for p in range(4):
        for k in range(R.shape[0]):
            hp = 1e-5 * args[p][k]
            up = [x.copy() for x in args]
            dn = [x.copy() for x in args]
            up[p][k] += hp
            dn[p][k] -= hp
            fd = (o.mbd_nl(R, *up, BETA, A_DAMP) - o.mbd_nl(R, *dn, BETA, A_DAMP)) / (2 * hp)
            assert abs(fd - gp[p, k]) < 1e-8 * max(1.0, abs(gp[p, k])), (p, k)


def test_nl_invariances():
    R, a0, c6, ra, rw = _system(2, N=6)
    E, gR, _ = o.mbd_nl(R, a0, c6, ra, rw, BETA, A_DAMP, grad=True)
    Qm, _ = np.linalg.qr(np.random.default_rng(3).normal(size=(3, 3)))
    E2, gR2, _ = o.mbd_nl(R @ Qm.T + [1.0, -2.0, 0.5], a0, c6, ra, rw, BETA, A_DAMP, grad=True)
    assert E2 == pytest.approx(E, rel=1e-12)
    assert np.allclose(gR2, gR @ Qm.T, atol=1e-14)
    assert np.abs(gR.sum(0)).max() < 1e-15            # no net force
    assert np.abs(np.cross(R, gR).sum(0)).max() < 1e-14   # no net torque
    p = np.random.default_rng(4).permutation(6)
    assert o.mbd_nl(R[p], a0[p], c6[p], ra[p], rw[p], BETA, A_DAMP) == pytest.approx(E, rel=1e-13)


def test_nl_rejects_nonpositive_ratios():
    R, a0, c6, ra, rw = _system(5, N=3)
    ra[1] = 0.0
    with pytest.raises(Exception):
        o.mbd_nl(R, a0, c6, ra, rw, BETA, A_DAMP)
