"""GPU tests of FP64 products: the antisymmetric mirror mode of the FP64 GEMM (mode 3, for the
imaginary parts of Hermitian products), and the FP64-accurate split GEMM (mbdk_gemm_f64_split: operands cut into exact
TF32 slices, slice products on the tcgen05 tensor cores, exact FP32 partial sums added in
FP64) against the host's FP64 product, and the FP64
path with its Newton-Schulz products on it (MBD_PREC_FP64_SPLIT) against the oracle and the
plain FP64 path.  Its slicing and an exact emulation of the product are checked on the CPU in
test_split64_host.py, which also fixes the tolerances used here."""
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


def _dev():
    import torch
    return torch.device("cuda:0")


@pytest.mark.parametrize("trans_b", [True, False])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 1152), (384, 128, 2112)])
def test_gemm_f64_split_is_fp64_accurate(M, N, K, trans_b):
    # FP64-accurate products on the TF32 tensor cores by error-free slicing: against the
    # exact product (long double on the host) within a few FP64 roundings of |A||B|, for
    # rows and columns of very different size, K over one and several 1024 pieces
    import torch
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(M, K)) * np.exp(rng.uniform(-6, 6, size=(M, 1)))
    B = rng.normal(size=(N, K)) * np.exp(rng.uniform(-6, 6, size=(N, 1)))
    # reference: the host's FP64 product (within a few ulps of |A||B| of the exact one; an
    # extended-precision product would be software-emulated on some hosts)
    exact = A @ B.T
    scale = np.abs(A) @ np.abs(B).T
    Bop = B if trans_b else np.ascontiguousarray(B.T)
    dA, dB = torch.tensor(A, device=_dev()), torch.tensor(Bop, device=_dev())
    C = torch.full((M, N), 7.0, dtype=torch.float64, device=_dev())
    err = binding.mbdk_gemm_f64_split(dA, dB, C, trans_b=trans_b)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = C.cpu().numpy()
    # an FP64 GEMM of these operands errs by up to ~3.5 ulps of |A||B|; the exact emulation of
    # this algorithm on the host gives 4.1 (K = 64) and 1.7 (K = 1152); a lost slice or a
    # rounded partial sum would show as ~2^-22
    assert np.all(np.abs(got - exact) <= 12 * 2.0 ** -53 * scale), np.abs((got - exact) / scale).max()
    # alpha, beta, and D aliasing C: C = -0.5 A B^T + 1.5 C
    D = rng.normal(size=(M, N))
    C2 = torch.tensor(D, device=_dev())
    binding.mbdk_gemm_f64_split(dA, dB, C2, alpha=-0.5, beta=1.5, D=C2, trans_b=trans_b)
    C3 = torch.zeros(M, N, dtype=torch.float64, device=_dev())
    binding.mbdk_gemm_f64_split(dA, dB, C3, alpha=-0.5, beta=1.5, D=torch.tensor(D, device=_dev()), trans_b=trans_b)
    torch.cuda.synchronize()
    ref = -0.5 * exact + 1.5 * D
    tol = 16 * 2.0 ** -53 * (0.5 * scale + 1.5 * np.abs(D))
    assert np.all(np.abs(C2.cpu().numpy() - ref) <= tol) and np.all(np.abs(C3.cpu().numpy() - ref) <= tol)


def test_gemm_f64_split_rejects_bad_shapes():
    import torch
    A = torch.zeros(128, 64, dtype=torch.float64, device=_dev())
    B = torch.zeros(96, 64, dtype=torch.float64, device=_dev())     # N not a multiple of 128
    C = torch.zeros(128, 96, dtype=torch.float64, device=_dev())
    with pytest.raises(binding.MBDError) as e:
        binding.mbdk_gemm_f64_split(A, B, C)
    assert e.value.code == 1


@pytest.mark.parametrize("workload", ["finite32", "n90"])
def test_fp64_split_path_matches_oracle_and_fp64_path(workload):
    sysm = syn.workload("finite32") if workload == "finite32" else syn.sphere_cluster(90, seed=1090)
    E_ref, gR_ref, gp_ref = o.mbd_rsscs_gradient(*o.system_args(sysm), mode="adjoint")
    out = {}
    for prec in (binding.MBD_PREC_FP64, binding.MBD_PREC_FP64_SPLIT):
        with binding.MBD(0, precision=prec) as m:
            m.set_geometry(sysm.coords)
            m.set_free_atom_params(sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)
            out[prec] = m.evaluate(True)[:3] + (m.stats(),)
    E, gR, gp, st = out[binding.MBD_PREC_FP64_SPLIT]
    E64, gR64, gp64, st64 = out[binding.MBD_PREC_FP64]
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref), (E, E_ref)
    assert np.abs(gR - gR_ref).max() <= 1e-8 * np.abs(gR_ref).max()
    # both paths are FP64-accurate; E is a small difference of terms of order sum(omega)
    assert abs(E - E64) <= 1e-11 * abs(E64) and np.abs(gR - gR64).max() <= 1e-9 * np.abs(gR64).max()
    assert abs(st["ns_iterations"] - st64["ns_iterations"]) <= 1


def test_gemm_f64_antisymmetric_mirror_mode():
    # S K S with S symmetric and K antisymmetric is antisymmetric: mode 3 computes the upper
    # tiles and writes their negatives below; P = K S first (mode 0, non-transposed path)
    import torch
    n = 192
    g = torch.Generator(device="cpu").manual_seed(3)
    X = torch.randn(n, n, generator=g, dtype=torch.float64)
    S, K = (X + X.T).to(_dev()), (X - X.T).to(_dev())
    P = torch.empty(n, n, dtype=torch.float64, device=_dev())
    binding.mbdk_gemm_f64(K, S, P, mode=0, trans_b=False)
    C = torch.full((n, n), float("nan"), dtype=torch.float64, device=_dev())
    D = torch.randn(n, n, generator=g, dtype=torch.float64)
    D = (D - D.T).to(_dev())
    binding.mbdk_gemm_f64(S, P, C, alpha=0.5, beta=2.0, D=D, mode=3, trans_b=False)
    torch.cuda.synchronize()
    ref = 0.5 * (S @ K @ S) + 2.0 * D
    assert torch.allclose(C, ref, rtol=1e-12, atol=1e-10)
    tiles = torch.arange(n, device=_dev()) // 64
    lower = tiles[:, None] > tiles[None, :]
    assert torch.equal(C[lower], -C.T[lower])          # mirrored entries are exact negatives
