"""Pins of the log-formula energy route of the oracle (oracle/mbd_oracle.c:
orc_mbd_log_energy; Sec. 2.5, Eqs. log-formula and rpa) against the diagonalization route,
the closed-form pairwise (second-order) energy and the two-oscillator closed form.  CPU only."""
import math

import numpy as np
import pytest

import oracle as o
from paper_2308_03140_gb300 import synthetic as syn

BETA, A_DAMP = 0.83, 6.0


def cluster(n=6, seed=11):
    sy = syn.cube_cluster(n, 12.0, 3.0, seed=seed)
    a0 = sy.alpha0_ref
    return sy.coords, a0, 4 * sy.c6_ref / (3 * a0 ** 2), sy.rvdw_ref


def test_log_route_equals_diagonalization_route():
    R, a0, om, rd = cluster()
    E_eig = o.mbd_energy(R, a0, om, rd, BETA, A_DAMP)
    E_log, _ = o.mbd_log_energy(R, a0, om, rd, BETA, A_DAMP, n_freq=40)
    # both are ~1e-3 Ha: the diagonalization route is a difference of terms ~3/2 sum(omega)
    assert abs(E_log - E_eig) < 50 * 2.2e-16 * 1.5 * om.sum()
    E15, _ = o.mbd_log_energy(R, a0, om, rd, BETA, A_DAMP, n_freq=15)
    assert E15 == pytest.approx(E_eig, rel=1e-8, abs=0)      # the default grid's quadrature error
    assert not E15 == pytest.approx(E_eig, rel=1e-12, abs=0)


def test_second_order_is_the_pairwise_energy():
    # E^(2) = -sum_{i<j} C6_ij g_ij^2 / R_ij^6, C6_ij = 3/pi int alpha_i alpha_j du
    #       = 3/2 alpha0_i alpha0_j omega_i omega_j / (omega_i + omega_j)
    R, a0, om, rd = cluster()
    _, orders = o.mbd_log_energy(R, a0, om, rd, BETA, A_DAMP, n_freq=40, max_order=2)
    E2 = 0.0
    for i in range(len(a0)):
        for j in range(i + 1, len(a0)):
            d = np.linalg.norm(R[j] - R[i])
            c6 = 1.5 * a0[i] * a0[j] * om[i] * om[j] / (om[i] + om[j])
            g = 1.0 / (1.0 + math.exp(-A_DAMP * (d / (BETA * (rd[i] + rd[j])) - 1.0)))
            E2 -= c6 * g * g / d ** 6
    assert orders[0] == pytest.approx(E2, rel=1e-12, abs=0)


def test_orders_sum_to_the_log_energy():
    R, a0, om, rd = cluster()
    E_log, orders = o.mbd_log_energy(R, a0, om, rd, BETA, A_DAMP, n_freq=15, max_order=14)
    assert orders.sum() == pytest.approx(E_log, rel=1e-10, abs=0)
    assert orders[0] < 0 and abs(orders[1]) < abs(orders[0])   # pairwise term dominates


def test_two_atoms_closed_form():
    d, a, w, rd = 5.0, (8.0, 5.0), (0.5, 0.9), (3.0, 3.4)
    R = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, d]])
    E, _ = o.mbd_log_energy(R, np.array(a), np.array(w), np.array(rd), BETA, A_DAMP, n_freq=60)
    g = 1.0 / (1.0 + math.exp(-A_DAMP * (d / (BETA * sum(rd)) - 1.0)))
    ref = 0.0
    for t in (g / d ** 3, g / d ** 3, -2 * g / d ** 3):   # per axis: 2x2 modes
        m = 0.5 * (w[0] ** 2 + w[1] ** 2)
        q = math.sqrt((0.5 * (w[0] ** 2 - w[1] ** 2)) ** 2 + w[0] ** 2 * w[1] ** 2 * a[0] * a[1] * t * t)
        ref += 0.5 * (math.sqrt(m + q) + math.sqrt(m - q))
    ref -= 1.5 * (w[0] + w[1])
    assert abs(E - ref) < 1e-13


def test_order_signs_and_quadrature():
    # one 2x2 block: A = [[0, c], [c, 0]] has eigenvalues +-c; Tr A^m = 2 c^m (m even), 0 (odd)
    d, a, w, rd = 6.0, (8.0, 8.0), (0.6, 0.6), (1e-3, 1e-3)   # g = 1: no damping
    R = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, d]])
    E, orders = o.mbd_log_energy(R, np.array(a), np.array(w), np.array(rd), BETA, A_DAMP, n_freq=60,
                                 max_order=4)
    assert abs(orders[1]) < 1e-16                                  # Tr A^3 = 0 for two atoms
    # E^(4) = -1/(2 pi) int du 1/4 Tr A^4 with Tr A^4 = 2 alpha(u)^4 (1 + 1 + 16)/d^12
    u, wu = o.freq_grid(60)
    al = a[0] / (1 + u[1:] ** 2 / w[0] ** 2)
    ref4 = -1 / (2 * math.pi) * np.sum(wu[1:] * 0.25 * 2 * al ** 4 * 18 / d ** 12)
    assert orders[2] == pytest.approx(ref4, rel=1e-12, abs=0)
