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
