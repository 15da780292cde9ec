"""GPU parity of the TS pairwise energy and gradients (Secs. 2.6 and 2.7: Eqs. pairwise, ts-scaling,
fermi-damping; mbd_ts_energy) against the CPU oracle (oracle/ts_pairwise.py).  FP64 on both
sides: energy 1e-12 relative, coordinate gradients 1e-10 relative to the largest, parameter
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
    with binding.MBD(0) as m:
        m.set_geometry(sysm.coords[:4], np.eye(3) * 20.0, (1, 1, 1))
        m.set_free_atom_params(*[a[:4] for a in args])
        with pytest.raises(binding.MBDError) as e:
            m.ts_energy(S_R)
        assert e.value.code == 8
