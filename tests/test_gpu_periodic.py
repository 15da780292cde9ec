"""GPU parity of the periodic path (Sec. 2.2, Ewald summation) through the C ABI against the
CPU oracle (oracle/mbd_periodic.c).

Tolerances: energy 1e-10 relative; coordinate and lattice gradients 1e-8 Ha/bohr; parameter
gradients 1e-8 relative to the largest of their kind; screened polarizabilities 1e-11
relative.  Both sides use the same Ewald split, cutoffs and Monkhorst-Pack grid."""
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


def small_cell(N, edge, seed, dmin=2.4):
    """N atoms in a skewed cell of about `edge` bohr, minimum-image separation dmin."""
    rng = np.random.default_rng(seed)
    A = np.array([[edge, 0.0, 0.0], [0.11 * edge, 0.95 * edge, 0.0], [-0.07 * edge, 0.09 * edge, 1.05 * edge]])
    frac = []
    shifts = np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij")).reshape(3, -1).T @ A
    while len(frac) < N:
        f = rng.uniform(0, 1, 3)
        ok = True
        for g in frac:
            d = (g - f) - np.round(g - f)
            if np.min(np.linalg.norm(d @ A + shifts, axis=1)) < dmin:
                ok = False
                break
        if ok:
            frac.append(f)
    R = np.array(frac) @ A
    p = syn.draw_params(rng, N)
    return R, A, p


def run_both(R, A, p, grid, gamma, rc, kc, grad=True):
    kap = o.monkhorst_pack(grid)
    E_ref, det = o.periodic_rsscs_energy(R, A, kap, *p, gamma, rc, kc, detail=True)
    with binding.MBD(0, ewald_gamma=gamma, real_cutoff=rc, recip_cutoff=kc) as m:
        m.set_geometry(R, A, grid)
        m.set_free_atom_params(*p)
        E, gR, gp, al = m.evaluate(grad)
        gA = m.lattice_gradient() if grad else None
        det_g, st = m.scs_detail(), m.stats()
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref), (E, E_ref, st)
    assert np.allclose(det_g["alpha_bar"], det["alpha_bar"], rtol=1e-11, atol=0)
    assert np.allclose(det_g["omega"], det["omega"], rtol=1e-11)
    assert np.allclose(al, det["alpha_bar"][0], rtol=1e-11)
    if grad:
        _, gR_ref, gA_ref, gp_ref = o.periodic_rsscs_gradient(R, A, kap, *p, gamma, rc, kc)
        assert np.max(np.abs(gR - gR_ref)) <= 1e-8, np.max(np.abs(gR - gR_ref))
        assert np.max(np.abs(gA - gA_ref)) <= 1e-8, (gA, gA_ref)
        for k in range(4):
            scale = np.max(np.abs(gp_ref[k]))
            assert np.max(np.abs(gp[k] - gp_ref[k])) <= 1e-8 * max(scale, 1e-3), k
    return E, st


def test_periodic_parity_small_cell():
    R, A, p = small_cell(3, 8.0, seed=11)
    run_both(R, A, p, (2, 2, 2), 0.35, 6.5 / 0.35, 11 * 0.35)


@pytest.mark.parametrize("N,edge,grid,seed", [(8, 10.0, (2, 2, 2), 12), (24, 12.5, (1, 2, 3), 13),
                                              (45, 15.0, (2, 1, 2), 14)])
def test_periodic_parity_tiles_and_grids(N, edge, grid, seed):
    # n = 24, 72 (one ragged 128 tile, padded), 135 (two tiles, ragged); odd grids contain Gamma
    R, A, p = small_cell(N, edge, seed)
    run_both(R, A, p, grid, 0.3, 6.5 / 0.3, 11 * 0.3)


def test_periodic_automatic_ewald_parameters_match_gamma_invariance():
    """Automatic Ewald parameters (gamma = 6/rc from the cutoff, kc = 10 gamma) against the
    oracle at another split: the energy does not depend on gamma.  The automatic reciprocal
    cutoff truncates the sum at exp(-25) of its leading term, a few 1e-9 of the energy."""
    R, A, p = small_cell(8, 10.0, seed=15)
    with binding.MBD(0, real_cutoff=26.0) as m:   # gamma = 6/26 from the cutoff
        m.set_geometry(R, A, (2, 2, 2))
        m.set_free_atom_params(*p)
        E, *_ = m.evaluate(False)
    E_ref = o.periodic_rsscs_energy(R, A, o.monkhorst_pack((2, 2, 2)), *p, 0.4, 26.0, 4.6)
    assert E == pytest.approx(E_ref, rel=1e-8)


def test_periodic_input_errors():
    R, A, p = small_cell(3, 8.0, seed=11)
    with binding.MBD(0) as m:
        with pytest.raises(binding.MBDError) as e:
            m.set_geometry(R, A, None)
        assert e.value.code == 1
        with pytest.raises(binding.MBDError) as e:
            m.set_geometry(R, np.zeros((3, 3)), (2, 2, 2))
        assert e.value.code == 1
        with pytest.raises(binding.MBDError) as e:
            m.set_geometry(R, A, (0, 2, 2))
        assert e.value.code == 1
    with binding.MBD(0, precision=binding.MBD_PREC_FP64_SPLIT) as m:
        with pytest.raises(binding.MBDError) as e:
            m.set_geometry(R, A, (2, 2, 2))
        assert e.value.code == 8


def test_periodic_lattice_gradient_state():
    R, A, p = small_cell(3, 8.0, seed=11)
    with binding.MBD(0, ewald_gamma=0.35) as m:
        m.set_geometry(R, A, (2, 2, 2))
        m.set_free_atom_params(*p)
        with pytest.raises(binding.MBDError):
            m.lattice_gradient()
        m.evaluate(False)
        with pytest.raises(binding.MBDError):
            m.lattice_gradient()
        m.evaluate(True)
        assert np.all(np.isfinite(m.lattice_gradient()))


# Mixed modes on a cell: each Hermitian Q(q) as its real symmetric embedding through the finite
# tensor-core matrix function with the FP64 correction.  Bounds a few times the largest errors
# measured on these cells (printed by the test): energy per atom (TF32x3 1.5e-8, BF16x3
# 1.7e-8), and the coordinate, lattice and parameter gradients relative to their largest
# components (TF32x3 2.6e-5, BF16x3 1.8e-4; the gradients take the tensor-core Q(q)^{-1/2}
# at first order).
MIXED_CELL = {binding.MBD_PREC_TF32X3: (5e-8, 2e-4), binding.MBD_PREC_BF16X3: (1e-7, 1e-3)}


def _mixed_vs(R, A, p, grid, gamma, rc, kc, precision, E_ref, gR_ref, gA_ref, gp_ref):
    with binding.MBD(0, precision=precision, ewald_gamma=gamma, real_cutoff=rc, recip_cutoff=kc) as m:
        m.set_geometry(R, A, grid)
        m.set_free_atom_params(*p)
        E, gR, gp, al = m.evaluate(True)
        gA = m.lattice_gradient()
        st = m.stats()
    N = R.shape[0]
    de = abs(E - E_ref) / N
    fr = np.abs(gR - gR_ref).max() / np.abs(gR_ref).max()
    lr = np.abs(gA - gA_ref).max() / np.abs(gA_ref).max()
    pr = max(np.abs(gp[k] - gp_ref[k]).max() / np.abs(gp_ref[k]).max() for k in range(4))
    print(f"cell N {N} precision {precision}: |dE|/N {de:.3e}, force {fr:.3e}, lattice {lr:.3e}, params {pr:.3e}, "
          f"iterations {st['ns_iterations']}")
    e_b, g_b = MIXED_CELL[precision]
    assert de <= e_b, (E, E_ref, st)
    assert fr <= g_b and lr <= g_b and pr <= g_b, (fr, lr, pr)
    return st


@pytest.mark.parametrize("precision", [binding.MBD_PREC_TF32X3, binding.MBD_PREC_BF16X3])
@pytest.mark.parametrize("N,edge,grid,seed", [(8, 10.0, (2, 2, 2), 12), (45, 15.0, (2, 1, 2), 14)])
def test_periodic_mixed_modes_against_the_oracle(N, edge, grid, seed, precision):
    R, A, p = small_cell(N, edge, seed)
    gamma, rc, kc = 0.3, 6.5 / 0.3, 11 * 0.3
    kap = o.monkhorst_pack(grid)
    E_ref = o.periodic_rsscs_energy(R, A, kap, *p, gamma, rc, kc)
    _, gR_ref, gA_ref, gp_ref = o.periodic_rsscs_gradient(R, A, kap, *p, gamma, rc, kc)
    _mixed_vs(R, A, p, grid, gamma, rc, kc, precision, E_ref, gR_ref, gA_ref, gp_ref)


@pytest.mark.parametrize("precision", [binding.MBD_PREC_TF32X3, binding.MBD_PREC_BF16X3])
def test_periodic_mixed_modes_at_the_256_atom_cell(precision):
    # against the oracle-checked FP64 path on the same cell (64 Bloch vectors)
    s = syn.workload("cell256")
    g, rc, kc = 0.2, 30.0, 2.0
    with binding.MBD(0, ewald_gamma=g, real_cutoff=rc, recip_cutoff=kc) as m:
        m.set_geometry(s.coords, s.lattice, s.k_grid)
        m.set_free_atom_params(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
        E64, gR64, gp64, _ = m.evaluate(True)
        gA64 = m.lattice_gradient()
    _mixed_vs(s.coords, s.lattice, (s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio), s.k_grid, g, rc, kc, precision,
              E64, gR64, gA64, gp64)
