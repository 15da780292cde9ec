"""Failure paths of the library on the GPU, made on the host (no device fault): the
Newton-Schulz iteration cap and the polarization catastrophe (Q not positive definite,
Sec. 2.1), each returned as its status code."""
import numpy as np
import pytest

import oracle as o
from paper_2308_03140_gb300 import binding, build
from paper_2308_03140_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


@pytest.mark.parametrize("precision", [binding.MBD_PREC_FP64, binding.MBD_PREC_TF32X3])
def test_iteration_cap_is_reported(precision):
    sysm = syn.workload("finite32")
    with binding.MBD(0, precision=precision, ns_max_iter=1) as m:
        m.set_geometry(sysm.coords)
        m.set_free_atom_params(sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)
        with pytest.raises(binding.MBDError) as e:
            m.evaluate(False)
        assert e.value.code == 5          # MBD_ERR_NOT_CONVERGED
        assert m.stats()["ns_iterations"] == 1


def test_polarization_catastrophe_is_reported():
    # two MBD-NL oscillators with alpha0 = 2500 at 12 bohr: alpha0 2 g / R^3 = 1.78 > 1, so the
    # axial mode of Q has a negative eigenvalue (the oracle agrees)
    R = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 12.0]])
    a0ref, c6ref, ra, rw = np.full(2, 5000.0), np.full(2, 300.0), np.full(2, 0.5), np.ones(2)
    with pytest.raises(o.OracleError) as e:
        o.mbd_nl(R, a0ref, c6ref, ra, rw)
    assert e.value.code == o.ERR_NEG_EIGENVALUE
    with binding.MBD(0, scs_mode=binding.MBD_SCS_NL) as m:
        m.set_geometry(R)
        m.set_nl_params(a0ref, c6ref, ra, rw)
        with pytest.raises(binding.MBDError) as e:
            m.evaluate(False)
        assert e.value.code == 2          # MBD_ERR_NEG_EIGENVALUE
