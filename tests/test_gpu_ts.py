"""GPU parity of the TS pairwise energy and gradients (Secs. 2.6 and 2.7: Eqs. pairwise,
ts-scaling, fermi-damping, ts-ewald; mbd_ts_energy) against the CPU oracle
(oracle/ts_pairwise.py), for clusters and for cells.  FP64 on both sides: energy 1e-12
relative, coordinate and lattice gradients 1e-10 relative to the largest, parameter
gradients 1e-10 relative to the largest of their kind."""
import numpy as np
import pytest

from oracle import ts_pairwise as T
from paper_2308_03140_gb300 import binding, build
from paper_2308_03140_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

S_R = 0.94


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


@pytest.mark.parametrize("which", ["three", "finite32", "n90"])
def test_ts_parity(which):
    sysm = {"three": lambda: syn.cube_cluster(3, 7.0, 2.5, seed=31), "finite32": lambda: syn.workload("finite32"),
            "n90": lambda: syn.sphere_cluster(90, seed=1090)}[which]()
    args = (sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)
    E_ref, gR_ref, gp_ref = T.ts_energy(sysm.coords, *args, S_R, grad=True)
    with binding.MBD(0) as m:
        m.set_geometry(sysm.coords)
        m.set_free_atom_params(*args)
        E, gR, gp = m.ts_energy(S_R)
        E0, _, _ = m.ts_energy(S_R, gradients=False)
    assert E == pytest.approx(E_ref, rel=1e-12, abs=0) and E0 == E
    assert np.abs(gR - gR_ref).max() <= 1e-10 * np.abs(gR_ref).max()
    for k in range(4):
        assert np.abs(gp[k] - gp_ref[k]).max() <= 1e-10 * np.abs(gp_ref[k]).max(), k
    assert np.abs(gR.sum(0)).max() <= 1e-14


def test_ts_errors():
    sysm = syn.workload("finite32")
    args = (sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)
    with binding.MBD(0) as m:
        m.set_geometry(sysm.coords)
        m.set_free_atom_params(*args)
        with pytest.raises(binding.MBDError) as e:
            m.ts_energy(0.0)
        assert e.value.code == 1
    with binding.MBD(0, scs_mode=binding.MBD_SCS_NL) as m:
        m.set_geometry(sysm.coords)
        m.set_free_atom_params(*args)
        with pytest.raises(binding.MBDError) as e:
            m.ts_energy(S_R)
        assert e.value.code == 8
    with binding.MBD(0) as m:                 # no lattice gradient for a finite system
        m.set_geometry(sysm.coords)
        m.set_free_atom_params(*args)
        with pytest.raises(binding.MBDError) as e:
            m.ts_energy(S_R, lattice=True)
        assert e.value.code == 8


def periodic_case(which):
    if which == "cell4":
        rng = np.random.default_rng(3)
        A = np.array([[9.0, 0, 0], [1.0, 8.5, 0], [-0.6, 0.8, 9.5]])
        R = rng.uniform(0, 1, (4, 3)) @ A
        args = (rng.uniform(4, 12, 4), rng.uniform(5, 50, 4), rng.uniform(3, 4, 4), rng.uniform(0.7, 1, 4))
        return R, A, args, 0.3
    c = syn.triclinic_cell(24, edge=(13.0, 15.0), seed=2024)
    return c.coords, c.lattice, (c.alpha0_ref, c.c6_ref, c.rvdw_ref, c.ratio), 0.22


@pytest.mark.parametrize("which", ["cell4", "cell24"])
def test_ts_periodic_parity(which):
    # Eq. ts-ewald minus the damped-away part, per cell, with coordinate, lattice and
    # parameter gradients; the k-grid plays no part
    R, A, args, gamma = periodic_case(which)
    rc, kc = 6.5 / gamma, 10.5 * gamma
    E_ref, gR_ref, gA_ref, gp_ref = T.ts_energy_periodic(R, A, *args, gamma, rc, kc, s_r=S_R, grad=True)
    with binding.MBD(0, ewald_gamma=gamma, real_cutoff=rc, recip_cutoff=kc) as m:
        m.set_geometry(R, A, (2, 2, 2))
        m.set_free_atom_params(*args)
        E, gR, gp, gA = m.ts_energy(S_R, lattice=True)
        E0, _, _ = m.ts_energy(S_R, gradients=False)
    assert E == pytest.approx(E_ref, rel=1e-12, abs=0) and E0 == E
    assert np.abs(gR - gR_ref).max() <= 1e-10 * np.abs(gR_ref).max()
    assert np.abs(gA - gA_ref).max() <= 1e-10 * np.abs(gA_ref).max()
    for k in range(4):
        assert np.abs(gp[k] - gp_ref[k]).max() <= 1e-10 * np.abs(gp_ref[k]).max(), k


def test_ts_periodic_full_cell_properties():
    # the 256-atom triclinic cell (edges 20-26 bohr): the oracle is too slow here, so the
    # checks are properties that hold at any size: the Ewald split gamma does not change the
    # energy or its gradients, the forces sum to zero, and the strain derivative
    # R^T dE/dR + A^T dE/dA is symmetric (rotational invariance)
    c = syn.workload("cell256")
    args = (c.alpha0_ref, c.c6_ref, c.rvdw_ref, c.ratio)
    out = []
    for gamma in (0.2, 0.26):
        with binding.MBD(0, ewald_gamma=gamma, real_cutoff=6.5 / gamma, recip_cutoff=10.5 * gamma) as m:
            m.set_geometry(c.coords, c.lattice, (1, 1, 1))
            m.set_free_atom_params(*args)
            out.append(m.ts_energy(S_R, lattice=True))
    (E1, gR1, gp1, gA1), (E2, gR2, gp2, gA2) = out
    assert E2 == pytest.approx(E1, rel=1e-10, abs=0)
    assert np.abs(gR2 - gR1).max() <= 1e-8 * np.abs(gR1).max()
    assert np.abs(gA2 - gA1).max() <= 1e-8 * np.abs(gA1).max()
    assert np.abs(gp2 - gp1).max() <= 1e-8 * np.abs(gp1).max()
    assert np.abs(gR1.sum(0)).max() <= 1e-12 * np.abs(gR1).max()
    strain = c.coords.T @ gR1 + c.lattice.T @ gA1
    assert np.abs(strain - strain.T).max() <= 1e-9 * np.abs(strain).max()
