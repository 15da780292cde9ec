"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: energy 1e-10 relative, gradients 1e-8 Ha/bohr (coordinates) and
1e-8 relative-to-max for parameter gradients, screened polarizabilities 1e-11
relative."""
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


def gpu_eval(sys, gradients=True):
    with binding.MBD(0) as m:
        m.set_geometry(sys.coords)
        m.set_free_atom_params(sys.alpha0_ref, sys.c6_ref, sys.rvdw_ref, sys.ratio)
        E, gR, gp, al = m.evaluate(gradients)
        return E, gR, gp, al, m.scs_detail(), m.stats()


def check_against_oracle(sys, grad=True):
    args = o.system_args(sys)
    E_ref, det = o.mbd_rsscs_energy(*args, detail=True)
    E, gR, gp, al, det_g, st = gpu_eval(sys, grad)
    N = sys.n_atoms
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref) + 1e-15, (E, E_ref, st)
    assert np.allclose(det_g["alpha_bar"], det["alpha_bar"], rtol=1e-11, atol=0)
    assert np.allclose(det_g["c6"], det["c6"], rtol=1e-11)
    assert np.allclose(det_g["omega"], det["omega"], rtol=1e-11)
    assert np.allclose(det_g["rvdw"], det["rvdw"], rtol=1e-11)
    assert np.allclose(al, det["alpha_bar"][0], rtol=1e-11)
    if grad:
        _, gR_ref, gp_ref = o.mbd_rsscs_gradient(*args, mode="adjoint")
        assert np.max(np.abs(gR - gR_ref)) <= 1e-8, np.max(np.abs(gR - gR_ref))
        for k in range(4):
            scale = np.max(np.abs(gp_ref[k]))
            assert np.max(np.abs(gp[k] - gp_ref[k])) <= 1e-8 * max(scale, 1e-3), k
    return E, st


def test_parity_finite32():
    E, st = check_against_oracle(syn.workload("finite32"))
    assert 5 <= st["ns_iterations"] <= 40


@pytest.mark.parametrize("n_atoms,seed", [(1, 1), (2, 2), (5, 3), (21, 4), (22, 5), (45, 6)])
def test_parity_sizes_and_ragged_tiles(n_atoms, seed):
    # n = 3N: 3, 6, 15 (one ragged tile), 63, 66 (tile + ragged tail), 135 (three tiles)
    edge = max(4.0, (n_atoms / 0.0117) ** (1 / 3))
    sys = syn.cube_cluster(n_atoms, edge, 2.5, seed=seed)
    check_against_oracle(sys)


def test_single_atom_has_zero_energy_and_unscreened_alpha():
    sys = syn.cube_cluster(1, 5.0, 2.5, seed=9)
    E, gR, gp, al, det, _ = gpu_eval(sys)
    assert abs(E) < 1e-14
    assert np.allclose(al, sys.alpha0_ref * sys.ratio, rtol=1e-13)
    assert np.all(gR == 0.0)


def test_dense_literal_cluster_reports_negative_alpha():
    sys = syn.fcc_jitter_cluster(60, density=0.08, seed=1099)
    with pytest.raises(binding.MBDError) as e:
        gpu_eval(sys)
    assert e.value.code == 3


def test_invalid_inputs_reported():
    sys = syn.cube_cluster(4, 6.0, 2.5, seed=4)
    bad = syn.System(sys.coords.copy(), sys.alpha0_ref.copy(), sys.c6_ref, sys.rvdw_ref, sys.ratio)
    bad.coords[1] = bad.coords[0]
    with pytest.raises(binding.MBDError) as e:
        gpu_eval(bad)
    assert e.value.code == 1
    bad = syn.System(sys.coords, sys.alpha0_ref.copy(), sys.c6_ref, sys.rvdw_ref, sys.ratio)
    bad.alpha0_ref[2] = np.nan
    with pytest.raises(binding.MBDError) as e:
        gpu_eval(bad)
    assert e.value.code == 1


def test_device_variant_matches_host_variant():
    import torch
    sys = syn.workload("finite32")
    E, gR, gp, al, _, _ = gpu_eval(sys)
    dev = torch.device("cuda:0")
    t = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev)
    N = sys.n_atoms
    e_t = torch.zeros(1, dtype=torch.float64, device=dev)
    gR_t = torch.zeros(N, 3, dtype=torch.float64, device=dev)
    gp_t = torch.zeros(4, N, dtype=torch.float64, device=dev)
    al_t = torch.zeros(N, dtype=torch.float64, device=dev)
    with binding.MBD(0) as m:
        m.set_geometry(sys.coords)
        m.evaluate_dev(t(sys.coords), t(sys.alpha0_ref), t(sys.c6_ref), t(sys.rvdw_ref), t(sys.ratio),
                       e_t, gR_t, gp_t, al_t)
    assert e_t.item() == E
    assert np.array_equal(gR_t.cpu().numpy(), gR)
    assert np.array_equal(gp_t.cpu().numpy(), gp)
    assert np.array_equal(al_t.cpu().numpy(), al)


def test_repeated_calls_are_deterministic():
    sys = syn.workload("finite32")
    with binding.MBD(0) as m:
        m.set_geometry(sys.coords)
        m.set_free_atom_params(sys.alpha0_ref, sys.c6_ref, sys.rvdw_ref, sys.ratio)
        r1 = m.evaluate(True)
        r2 = m.evaluate(True)
    assert r1[0] == r2[0]
    assert np.array_equal(r1[1], r2[1]) and np.array_equal(r1[2], r2[2])
