"""GPU checks at the full benchmark sizes, in the launch configuration bench.py times.

The plain CPU oracle is too slow for a 6000 x 6000 problem (Gauss-Jordan, Jacobi), so here
the reference is assembled from the oracle's own matrix builders (oracle/mbd_oracle.c,
oracle/mbd_periodic.c) with LAPACK (numpy.linalg.solve / eigvalsh) as the dense step:
- screening: M(u) from the oracle, X = M^{-1} 1 by LU, alpha_bar by Eq. (contraction);
- screened parameters by the oracle (Eqs. casimir-polder, scale-rvdw-scs);
- Q (finite) or Q(q) (periodic, every Bloch vector of the grid up to time reversal,
  Q(-q) = conj Q(q) has the same spectrum) from the oracle, E from its eigenvalues.
Tolerances as for the small cases: energy 1e-10 relative (FP64 path), screened
polarizabilities 1e-11 relative; the TF32x3 and BF16x3 arms within 1e-7 Ha/atom of the
reference (the method's bar is 1e-6).  Gradients of the finite cluster are compared element by
element with the oracle's adjoint gradient (its MBD and SCS pair passes and chains, in C) on
the same LAPACK dense steps: Z = Q^{-1/2} from the eigenvectors of Q and the adjoint solves
with the Cholesky factors of M(u); FP64 to 1e-8 Ha/bohr.  Both systems are also checked
through properties that hold at any size: zero net force (translations), zero net torque
(rotations, finite system), and central differences of the GPU energy along a random
direction.
"""
import math

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


def reference_screening(scs_matrix_of_alpha, a0, om, rv, N):
    u, _ = o.freq_grid(15)
    n = 3 * N
    E3 = np.zeros((n, 3))
    for c in range(3):
        E3[c::3, c] = 1.0
    ab = np.zeros((16, N))
    for k in range(16):
        X = np.linalg.solve(scs_matrix_of_alpha(o.dyn_alpha(a0, om, u[k])), E3)
        ab[k] = (X[0::3, 0] + X[1::3, 1] + X[2::3, 2]) / 3.0
    rc, (abar0, c6bar, ombar, rbar) = o.screened_params(ab, a0, rv)
    assert rc == 0
    return ab, abar0, ombar, rbar


@pytest.fixture(scope="module")
def finite_dense():
    """The 2000-atom cluster's reference with LAPACK dense steps: Cholesky factors of the 16
    screening matrices (kept for the adjoint solves), X = M^{-1} E, alpha_bar, the energy
    from the eigenvalues of Q and Z = Q^{-1/2} from its eigenvectors."""
    import scipy.linalg as sl
    s = syn.workload("finite2000")
    R, a0r, c6r, rr, v = o.system_args(s)
    a0, om, rv = o.ts_scaling(a0r, c6r, rr, v)
    u, _ = o.freq_grid(15)
    n = 3 * s.n_atoms
    E3 = np.zeros((n, 3))
    for c in range(3):
        E3[c::3, c] = 1.0
    factors, X = [], np.zeros((16, n, 3))
    for k in range(16):
        f = sl.cho_factor(o.scs_matrix(R, o.dyn_alpha(a0, om, u[k]), rv), lower=True, check_finite=False)
        factors.append(f)
        X[k] = sl.cho_solve(f, E3, check_finite=False)
    ab = (X[:, 0::3, 0] + X[:, 1::3, 1] + X[:, 2::3, 2]) / 3.0
    rc, (abar0, c6bar, ombar, rbar) = o.screened_params(ab, a0, rv)
    assert rc == 0
    lam, C = np.linalg.eigh(o.mbd_q(R, abar0, ombar, rbar))
    assert lam[0] > 0
    E = math.fsum(list(0.5 * np.sqrt(lam)) + list(-1.5 * ombar))
    Z = (C / np.sqrt(lam)) @ C.T
    return dict(s=s, E=E, ab=ab, X=X, Z=Z, factors=factors)


@pytest.fixture(scope="module")
def finite_ref(finite_dense):
    d = finite_dense
    return d["s"], d["E"], d["ab"]


@pytest.fixture(scope="module")
def finite_grad_ref(finite_dense):
    """The oracle's adjoint gradient of the 2000-atom cluster (its pair passes and chains) on
    the LAPACK dense steps of finite_dense."""
    import scipy.linalg as sl
    d = finite_dense
    s = d["s"]
    gR, gp = o.gradient_from_dense_steps(*o.system_args(s), d["ab"], d["X"], d["Z"],
                                         lambda k, H: sl.cho_solve(d["factors"][k], H, check_finite=False))
    return gR, gp


@pytest.fixture(scope="module")
def periodic_ref():
    s = syn.workload("cell256")
    R, a0r, c6r, rr, v = o.system_args(s)
    a0, om, rv = o.ts_scaling(a0r, c6r, rr, v)
    g, rc, kc = 0.2, 30.0, 2.0
    ab, abar0, ombar, rbar = reference_screening(lambda al: o.periodic_scs_matrix(R, s.lattice, al, rv, rc),
                                                 a0, om, rv, s.n_atoms)
    kap = o.monkhorst_pack(s.k_grid)
    half = kap[kap[:, 0] > 0]          # the other half is -kappa: same spectrum
    assert 2 * len(half) == len(kap)
    terms = []
    for k in half:
        lam = np.linalg.eigvalsh(o.periodic_q(R, s.lattice, k, abar0, ombar, rbar, g, rc, kc))
        assert lam[0] > 0
        terms += list(0.5 * np.sqrt(lam) * 2.0 / len(kap))
    E = math.fsum(terms + list(-1.5 * ombar))
    return s, E, ab


def gpu(s, precision=binding.MBD_PREC_FP64, gradients=True, **opt):
    m = binding.MBD(0, precision=precision, **opt)
    m.set_geometry(s.coords, s.lattice, s.k_grid)
    m.set_free_atom_params(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
    E, gR, gp, al = m.evaluate(gradients)
    return m, E, gR, gp


def directional_check(m, s, E0, gR, h=1e-3, seed=0):
    d = np.random.default_rng(seed).normal(size=s.coords.shape)
    d /= np.linalg.norm(d)
    es = []
    for sg in (1, -1):
        m.set_geometry(s.coords + sg * h * d, s.lattice, s.k_grid)
        m.set_free_atom_params(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
        es.append(m.evaluate(False)[0])
    fd = (es[0] - es[1]) / (2 * h)
    assert fd == pytest.approx(float((gR * d).sum()), rel=1e-5, abs=1e-10)


def test_finite2000_fp64_energy_and_screening(finite_ref):
    s, E_ref, ab = finite_ref
    m, E, gR, gp = gpu(s)
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref), (E, E_ref)
    assert np.allclose(m.scs_detail()["alpha_bar"], ab, rtol=1e-11, atol=0)
    assert np.abs(gR.sum(0)).max() < 1e-12
    assert np.abs(np.cross(s.coords, gR).sum(0)).max() < 1e-10
    directional_check(m, s, E, gR)
    m.close()


def test_finite2000_fp64_gradients_elementwise(finite_ref, finite_grad_ref):
    # every force and parameter-gradient component against the oracle's adjoint gradient
    s, _, _ = finite_ref
    gR_ref, gp_ref = finite_grad_ref
    m, E, gR, gp = gpu(s)
    m.close()
    assert np.abs(gR - gR_ref).max() <= 1e-8, np.abs(gR - gR_ref).max()
    for k in range(4):
        assert np.abs(gp[k] - gp_ref[k]).max() <= 1e-8 * max(1.0, np.abs(gp_ref[k]).max()), k


@pytest.mark.parametrize("precision,f_bound,p_bound", [(binding.MBD_PREC_TF32X3, 5e-5, 5e-5),
                                                       (binding.MBD_PREC_BF16X3, 5e-4, 5e-4)])
def test_finite2000_mixed_energy_and_forces(finite_ref, finite_grad_ref, precision, f_bound, p_bound):
    s, E_ref, ab = finite_ref
    m, E, gR, gp = gpu(s, precision)
    ab_tc = m.scs_detail()["alpha_bar"]
    m.close()
    assert abs(E - E_ref) / s.n_atoms <= 1e-7, (E, E_ref)
    # FP32 factorization, the solve refined once against the FP64 screening matrices
    assert np.allclose(ab_tc, ab, rtol=1e-10, atol=0)
    m64, E64, gR64, gp64 = gpu(s)
    m64.close()
    gR_ref, gp_ref = finite_grad_ref
    fo = np.abs(gR - gR_ref).max() / np.abs(gR_ref).max()
    assert fo <= f_bound, fo   # element by element against the oracle's gradient as well
    # forces of the mixed mode come from the Newton-Schulz Z of the tensor-core iteration;
    # bounds a few times the errors measured at this size (4.9e-6 TF32x3, 7.9e-5 BF16x3)
    fr = np.abs(gR - gR64).max() / np.abs(gR64).max()
    pr = max(np.abs(gp[k] - gp64[k]).max() / np.abs(gp64[k]).max() for k in range(4))
    print(f"precision {precision} N 2000: force err {fr:.3e}, param err {pr:.3e} of max")
    assert fr <= f_bound
    assert pr <= p_bound


def test_cell256_fp64_energy_screening_and_gradients(periodic_ref):
    s, E_ref, ab = periodic_ref
    m, E, gR, gp = gpu(s, real_cutoff=30.0)
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref), (E, E_ref)
    assert np.allclose(m.scs_detail()["alpha_bar"], ab, rtol=1e-11, atol=0)
    gA = m.lattice_gradient()
    assert np.abs(gR.sum(0)).max() < 1e-12
    directional_check(m, s, E, gR)
    # lattice: a random strain direction of A at fixed Cartesian positions
    dA = np.random.default_rng(1).normal(size=(3, 3))
    dA /= np.linalg.norm(dA)
    es = []
    for sg in (1, -1):
        m.set_geometry(s.coords, s.lattice + sg * 1e-3 * dA, s.k_grid)
        m.set_free_atom_params(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
        es.append(m.evaluate(False)[0])
    assert (es[0] - es[1]) / 2e-3 == pytest.approx(float((gA * dA).sum()), rel=1e-5, abs=1e-10)
    m.close()
