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


def test_tensor_core_wait_times_out_with_status():
    # the GEMM's bounded wait on a barrier that nothing arrives at (no copy or MMA in flight):
    # it gives up after its budget and raises the timeout bit; the context stays usable
    import torch
    dev = torch.device("cuda:0")
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    assert binding.mbdk_tc_wait_check(err, 2_000_000) == 0
    torch.cuda.synchronize()
    assert err.item() == 8               # ST_TC_TIMEOUT
    assert binding.mbdk_tc_wait_check(err, 0) == 1   # MBD_ERR_INPUT: budget out of range
    # a GEMM on the same context still runs and is correct
    A = torch.randn(128, 64, dtype=torch.float32, device=dev)
    C = torch.zeros(128, 128, dtype=torch.float32, device=dev)
    err.zero_()
    assert binding.mbdk_gemm_tc(0, A, A, C, err=err) == 0
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = A.double() @ A.double().T
    assert (C.double() - ref).abs().max().item() <= 2e-3 * (A.double().abs() @ A.double().abs().T).max().item()


@pytest.mark.parametrize("precision", [binding.MBD_PREC_BF16X3, binding.MBD_PREC_TF32X3])
def test_mixed_correction_check_reports_a_poor_inverse_root(precision):
    # the split kinds estimate the energy error their Q^{-1/2} leaves after the FP64 correction;
    # with the bar set below what any reduced-precision iteration reaches, the evaluation fails
    # with MBD_ERR_NOT_CONVERGED instead of returning an energy outside it
    sysm = syn.workload("finite32")
    with binding.MBD(0, precision=precision, mixed_max_error=1e-30) as m:
        m.set_geometry(sysm.coords)
        m.set_free_atom_params(sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)
        with pytest.raises(binding.MBDError) as e:
            m.evaluate(False)
        assert e.value.code == 5          # MBD_ERR_NOT_CONVERGED
    with binding.MBD(0, precision=precision) as m:   # the default bar passes
        m.set_geometry(sysm.coords)
        m.set_free_atom_params(sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)
        m.evaluate(False)
