"""The torch.autograd.Function wrapper: backward = the library's hand-written reverse
pass, checked against the CPU oracle's gradient, central differences of the GPU energy,
and torch.autograd.gradcheck."""
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


def _tensors(sysm, requires_grad=True):
    import torch
    dev = torch.device("cuda:0")
    return [torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev,
                         requires_grad=requires_grad)
            for x in (sysm.coords, sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)]


def test_autograd_backward_matches_oracle_gradient():
    import torch
    from paper_2308_03140_gb300.autograd import MBDEnergy
    sysm = syn.workload("finite32")
    E_ref, gR_ref, gp_ref = o.mbd_rsscs_gradient(*o.system_args(sysm), mode="adjoint")
    mod = MBDEnergy(sysm.n_atoms)
    ins = _tensors(sysm)
    E = mod(*ins)
    (3.0 * E).backward()                     # the incoming gradient scales the result
    assert abs(E.item() - E_ref) <= 1e-10 * abs(E_ref)
    assert np.max(np.abs(ins[0].grad.cpu().numpy() - 3.0 * gR_ref)) <= 3e-8
    for k in range(4):
        g = ins[k + 1].grad.cpu().numpy()
        assert np.max(np.abs(g - 3.0 * gp_ref[k])) <= 3e-8 * max(1.0, np.max(np.abs(gp_ref[k])))


def test_autograd_gradcheck_small_system():
    import torch
    from paper_2308_03140_gb300.autograd import MBDEnergy
    sysm = syn.cube_cluster(4, 6.5, 2.5, seed=21)
    mod = MBDEnergy(sysm.n_atoms)
    ins = _tensors(sysm)
    assert torch.autograd.gradcheck(lambda *x: mod(*x), tuple(ins), eps=1e-6, atol=1e-8, rtol=1e-5)


def test_backward_without_forward_is_an_error():
    import torch
    sysm = syn.cube_cluster(3, 6.0, 2.5, seed=5)
    ins = _tensors(sysm, requires_grad=False)
    with binding.MBD(0) as m:
        m.set_geometry(sysm.coords)
        gR = torch.empty(3, 3, dtype=torch.float64, device=ins[0].device)
        with pytest.raises(binding.MBDError) as e:
            m.backward_dev(*ins, grad_coords=gR)
        assert e.value.code == 7


def test_two_forwards_on_one_context_before_backward():
    # E = f(x1) + f(x2) on one module: the second forward replaces the device state of the
    # first, so the first's backward must evaluate again, not differentiate the second state
    import torch
    from paper_2308_03140_gb300.autograd import MBDEnergy
    s1 = syn.cube_cluster(6, 8.0, 2.5, seed=31)
    s2 = syn.cube_cluster(6, 8.0, 2.5, seed=32)
    mod = MBDEnergy(6)
    x1, x2 = _tensors(s1), _tensors(s2)
    E = mod(*x1) + 2.0 * mod(*x2)
    E.backward()
    for sysm, x, w in ((s1, x1, 1.0), (s2, x2, 2.0)):
        _, gR_ref, gp_ref = o.mbd_rsscs_gradient(*o.system_args(sysm), mode="adjoint")
        assert np.max(np.abs(x[0].grad.cpu().numpy() - w * gR_ref)) <= 3e-8
        for k in range(4):
            assert np.max(np.abs(x[k + 1].grad.cpu().numpy() - w * gp_ref[k])) <= 3e-8 * max(1.0, np.abs(gp_ref[k]).max())


def test_backward_of_a_replaced_evaluation_is_an_error():
    import torch
    s1 = syn.cube_cluster(4, 7.0, 2.5, seed=41)
    s2 = syn.cube_cluster(4, 7.0, 2.5, seed=42)
    x1, x2 = _tensors(s1, requires_grad=False), _tensors(s2, requires_grad=False)
    dev = x1[0].device
    with binding.MBD(0) as m:
        m.set_geometry(s1.coords)
        e = torch.empty(1, dtype=torch.float64, device=dev)
        m.evaluate_dev(*x1, e)
        first = m.evaluation_count()
        m.evaluate_dev(*x2, e)
        assert m.evaluation_count() == first + 1
        gR = torch.empty(4, 3, dtype=torch.float64, device=dev)
        with pytest.raises(binding.MBDError) as err:
            m.backward_dev(*x1, grad_coords=gR, evaluation=first)
        assert err.value.code == 7   # MBD_ERR_STATE
        m.backward_dev(*x2, grad_coords=gR, evaluation=first + 1)
        _, gR_ref, _ = o.mbd_rsscs_gradient(*o.system_args(s2), mode="adjoint")
        assert np.max(np.abs(gR.cpu().numpy() - gR_ref)) <= 3e-8
