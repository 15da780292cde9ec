"""GPU parity of MBD-NL (Sec. 2.7, paragraph MBD-NL: no screening, oscillators from
Eqs. mbd-nl-scaling and mbd-nl-rvdw) through the C ABI against the CPU oracle
(oracle/mbd_oracle.c: orc_mbd_nl).

Tolerances as for MBD@rsSCS: energy 1e-10 relative, coordinate gradients 1e-8 Ha/bohr,
parameter gradients 1e-8 relative to the largest of their kind (FP64 path); the TF32x3
arm within the method's 1e-6 Ha/atom of the FP64 path, forces within 0.1 of the largest.
Periodic systems: the oracle's Q(q) (oracle/mbd_periodic.c) with LAPACK eigenvalues as the
dense step; gradients against central differences of that energy."""
import math

import numpy as np
import pytest

import oracle as o
from paper_2308_03140_gb300 import binding, build
from paper_2308_03140_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

BETA, A_DAMP = 0.83, 6.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def nl_inputs(sysm, seed):
    ra, rw = syn.nl_ratios(sysm.n_atoms, seed)
    return sysm.coords, sysm.alpha0_ref, sysm.c6_ref, ra, rw


def gpu_nl(R, a0, c6, ra, rw, precision=binding.MBD_PREC_FP64, lattice=None, k_grid=None, **opt):
    m = binding.MBD(0, precision=precision, scs_mode=binding.MBD_SCS_NL, **opt)
    m.set_geometry(R, lattice, k_grid)
    m.set_nl_params(a0, c6, ra, rw)
    return m


@pytest.mark.parametrize("which", ["three", "finite32", "n90"])
def test_nl_parity_fp64(which):
    if which == "three":
        sysm = syn.cube_cluster(3, 7.0, 2.5, seed=31)
    elif which == "finite32":
        sysm = syn.workload("finite32")
    else:
        sysm = syn.sphere_cluster(90, seed=1090)   # 3N = 270: several tiles and a ragged tail
    R, a0, c6, ra, rw = nl_inputs(sysm, seed=77)
    E_ref, gR_ref, gp_ref, par = o.mbd_nl(R, a0, c6, ra, rw, BETA, A_DAMP, grad=True, detail=True)
    with gpu_nl(R, a0, c6, ra, rw) as m:
        E, gR, gp, al = m.evaluate(True)
        det = m.scs_detail()
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref), (E, E_ref)
    assert np.max(np.abs(gR - gR_ref)) <= 1e-8
    for k in range(4):
        assert np.max(np.abs(gp[k] - gp_ref[k])) <= 1e-8 * max(np.max(np.abs(gp_ref[k])), 1e-3), k
    assert np.allclose(al, par[0], rtol=1e-14, atol=0)
    assert np.allclose(det["omega"], par[1], rtol=1e-14, atol=0)
    assert np.allclose(det["rvdw"], par[2], rtol=1e-14, atol=0)
    assert np.allclose(det["c6"], 0.75 * par[0] ** 2 * par[1], rtol=1e-14)


def test_nl_tf32x3_matches_fp64_at_500_atoms():
    sysm = syn.sphere_cluster(500, seed=1500)
    R, a0, c6, ra, rw = nl_inputs(sysm, seed=78)
    out = {}
    for p in (binding.MBD_PREC_FP64, binding.MBD_PREC_TF32X3):
        with gpu_nl(R, a0, c6, ra, rw, precision=p) as m:
            out[p] = m.evaluate(True)
    E64, gR64 = out[binding.MBD_PREC_FP64][:2]
    E, gR = out[binding.MBD_PREC_TF32X3][:2]
    assert abs(E - E64) / 500 <= 1e-6, (E, E64)
    assert np.max(np.abs(gR - gR64)) <= 0.1 * np.max(np.abs(gR64))


def periodic_nl_energy(R, A, grid, a0, c6, ra, rw, gamma, rc, kc):
    """Oracle Q(q) of the MBD-NL oscillators for every Bloch vector of the grid, LAPACK
    eigenvalues: E = (1/n_k) sum_q 1/2 Tr Q(q)^(1/2) - 3/2 sum omega."""
    _, par = o.mbd_nl(R, a0, c6, ra, rw, BETA, A_DAMP, detail=True)   # the oscillators (alpha0, omega, R_damp)
    kap = o.monkhorst_pack(grid)
    terms = []
    for k in kap:
        lam = np.linalg.eigvalsh(o.periodic_q(R, A, k, par[0], par[1], par[2], gamma, rc, kc, BETA, A_DAMP))
        assert lam[0] > 0
        terms += list(0.5 * np.sqrt(lam) / len(kap))
    return math.fsum(terms + list(-1.5 * par[1]))


def test_nl_periodic_parity():
    from test_gpu_periodic import small_cell
    R, A, p = small_cell(8, 10.0, seed=12)
    a0, c6 = p[0], p[1]
    ra, rw = syn.nl_ratios(8, seed=79)
    grid, g, rc, kc = (2, 2, 2), 0.3, 6.5 / 0.3, 11 * 0.3
    E_ref = periodic_nl_energy(R, A, grid, a0, c6, ra, rw, g, rc, kc)
    with gpu_nl(R, a0, c6, ra, rw, lattice=A, k_grid=grid, ewald_gamma=g, real_cutoff=rc, recip_cutoff=kc) as m:
        E, gR, gp, _ = m.evaluate(True)
        gA = m.lattice_gradient()
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref), (E, E_ref)
    h = 1e-4
    for (i, c) in [(0, 0), (3, 2), (7, 1)]:
        Rp, Rm = R.copy(), R.copy()
        Rp[i, c] += h
        Rm[i, c] -= h
        fd = (periodic_nl_energy(Rp, A, grid, a0, c6, ra, rw, g, rc, kc) -
              periodic_nl_energy(Rm, A, grid, a0, c6, ra, rw, g, rc, kc)) / (2 * h)
        assert abs(fd - gR[i, c]) < 1e-9, (i, c, fd, gR[i, c])
    dA = np.random.default_rng(5).normal(size=(3, 3))
    dA /= np.linalg.norm(dA)
    fd = (periodic_nl_energy(R, A + h * dA, grid, a0, c6, ra, rw, g, rc, kc) -
          periodic_nl_energy(R, A - h * dA, grid, a0, c6, ra, rw, g, rc, kc)) / (2 * h)
    assert abs(fd - float((gA * dA).sum())) < 1e-8
    hh = 1e-5 * rw[2]
    up, dn = rw.copy(), rw.copy()
    up[2] += hh
    dn[2] -= hh
    fd = (periodic_nl_energy(R, A, grid, a0, c6, ra, up, g, rc, kc) -
          periodic_nl_energy(R, A, grid, a0, c6, ra, dn, g, rc, kc)) / (2 * hh)
    assert abs(fd - gp[3, 2]) < 1e-8 * max(1.0, abs(gp[3, 2]))


def test_nl_input_errors_and_no_screening():
    sysm = syn.cube_cluster(3, 7.0, 2.5, seed=31)
    R, a0, c6, ra, rw = nl_inputs(sysm, seed=77)
    with gpu_nl(R, a0, c6, ra, rw) as m:
        with pytest.raises(binding.MBDError) as e:
            m.screen()
        assert e.value.code == 8
        bad = rw.copy()
        bad[1] = -1.0
        m.set_nl_params(a0, c6, ra, bad)
        with pytest.raises(binding.MBDError) as e:
            m.evaluate(False)
        assert e.value.code == 1
