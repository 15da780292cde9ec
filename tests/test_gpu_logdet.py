"""GPU parity of the log-formula energy route (Eq. log-formula) and its many-body orders
(Eq. rpa) through the C ABI (mbd_log_energy) against the CPU oracle (orc_mbd_log_energy),
with the oscillators the oracle's own screening gives (orc_mbd_rsscs_energy detail).

Tolerances: energy and orders 1e-10 relative (FP64 on both sides, the same 15-point grid).
Cross-route: the log energy on the 15-point grid against the Newton-Schulz energy of the
same evaluation within 1e-8 relative up to 90 atoms and 5e-8 at 500 (the grid's quadrature
error: ~1e-9 at 32 atoms, 1.7e-8 at 500)."""
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


def system(which):
    return syn.workload("finite32") if which == "finite32" else syn.sphere_cluster(90, seed=1090)


@pytest.mark.parametrize("which", ["finite32", "n90"])
def test_log_energy_parity_and_cross_route(which):
    sysm = system(which)
    args = o.system_args(sysm)
    _, det = o.mbd_rsscs_energy(*args, detail=True)
    E_ref, ord_ref = o.mbd_log_energy(sysm.coords, det["alpha_bar"][0], det["omega"], det["rvdw"], BETA, A_DAMP,
                                      n_freq=15, max_order=4)
    with binding.MBD(0) as m:
        m.set_geometry(sysm.coords)
        m.set_free_atom_params(sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)
        E_ns = m.evaluate(False)[0]
        E_log, orders = m.log_energy(4)
        E_log2, orders2 = m.log_energy(2)            # orders 3 and 4 skipped: same energy
    assert abs(E_log - E_ref) <= 1e-10 * abs(E_ref), (E_log, E_ref)
    assert np.allclose(orders, ord_ref, rtol=1e-10, atol=0), (orders, ord_ref)
    assert E_log2 == E_log                                  # same factors, fixed-order sums
    assert orders2[0] == pytest.approx(orders[0], rel=1e-13, abs=0)   # block sums combined by atomics
    assert abs(E_log - E_ns) <= 1e-8 * abs(E_ns), (E_log, E_ns)
    assert orders[0] < 0 < orders[1]   # attractive pairwise term, repulsive three-body term


def test_log_energy_after_mixed_and_nl_evaluations():
    sysm = syn.sphere_cluster(500, seed=1500)
    E = {}
    for p in (binding.MBD_PREC_FP64, binding.MBD_PREC_TF32X3):
        with binding.MBD(0, precision=p) as m:
            m.set_geometry(sysm.coords)
            m.set_free_atom_params(sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)
            E[p] = (m.evaluate(False)[0],) + m.log_energy(2)
    # the mixed screening's oscillators agree with FP64 to ~1e-13, so the log energies agree
    assert E[binding.MBD_PREC_TF32X3][1] == pytest.approx(E[binding.MBD_PREC_FP64][1], rel=1e-10, abs=0)
    # the 15-point grid's quadrature error grows with the system: 1.7e-8 relative at 500 atoms
    # (the oracle's log route on a finer grid closes it), ~1e-9 at 32
    assert abs(E[binding.MBD_PREC_FP64][1] - E[binding.MBD_PREC_FP64][0]) <= 5e-8 * abs(E[binding.MBD_PREC_FP64][0])
    # MBD-NL: the log route of its oscillators against the oracle's diagonalization
    ra, rw = syn.nl_ratios(32, seed=80)
    s32 = syn.workload("finite32")
    E_nl, _, _, par = o.mbd_nl(s32.coords, s32.alpha0_ref, s32.c6_ref, ra, rw, BETA, A_DAMP, grad=True, detail=True)
    E_ref, _ = o.mbd_log_energy(s32.coords, par[0], par[1], par[2], BETA, A_DAMP, n_freq=15, max_order=2)
    with binding.MBD(0, scs_mode=binding.MBD_SCS_NL) as m:
        m.set_geometry(s32.coords)
        m.set_nl_params(s32.alpha0_ref, s32.c6_ref, ra, rw)
        m.evaluate(False)
        E_log, _ = m.log_energy(2)
    assert abs(E_log - E_ref) <= 1e-10 * abs(E_ref)
    assert abs(E_log - E_nl) <= 1e-8 * abs(E_nl)


def test_log_energy_errors():
    sysm = syn.workload("finite32")
    with binding.MBD(0) as m:
        m.set_geometry(sysm.coords)
        m.set_free_atom_params(sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)
        with pytest.raises(binding.MBDError) as e:
            m.log_energy(2)                  # no evaluation yet
        assert e.value.code == 7
        m.evaluate(False)
        with pytest.raises(binding.MBDError) as e:
            m.log_energy(5)
        assert e.value.code == 1
        # the call reuses the screening buffers: a new evaluation restores the state
        E1 = m.evaluate(True)[0]
        m.log_energy(3)
        E2, gR, _, _ = m.evaluate(True)
        assert E2 == pytest.approx(E1, rel=1e-12, abs=0) and np.all(np.isfinite(gR))
