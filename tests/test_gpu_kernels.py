"""Kernel-level GPU tests of the dense FP64 building blocks against plain torch
float64 references (matmul, Cholesky, triangular solves)."""
import numpy as np
import pytest

from paper_2308_03140_gb300 import binding, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def _dev():
    import torch
    return torch.device("cuda:0")


@pytest.mark.parametrize("trans_b", [True, False])
@pytest.mark.parametrize("M,N,K", [(64, 64, 64), (192, 128, 320), (256, 64, 64), (384, 384, 192)])
def test_gemm_full(M, N, K, trans_b):
    import torch
    g = torch.Generator(device="cpu").manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g, dtype=torch.float64)
    B = torch.randn(N, K, generator=g, dtype=torch.float64)
    D = torch.randn(M, N, generator=g, dtype=torch.float64)
    C = torch.zeros(M, N, dtype=torch.float64, device=_dev())
    Bop = B if trans_b else B.T.contiguous()
    binding.mbdk_gemm_f64(A.to(_dev()), Bop.to(_dev()), C, alpha=-0.5, beta=1.5, D=D.to(_dev()), mode=0,
                          trans_b=trans_b)
    ref = -0.5 * A @ B.T + 1.5 * D          # CPU float64 reference
    torch.cuda.synchronize()
    # FP64 products of N(0,1) data: error bound ~ K eps |A||B|
    assert torch.allclose(C.cpu(), ref, rtol=0, atol=4 * K * 2.3e-16 * 4)


@pytest.mark.parametrize("trans_b", [True, False])
def test_gemm_is_exact_on_integer_data(trans_b):
    # integers below 2^20 with K = 256: every product and partial sum is exact in FP64,
    # so a full-precision FP64 tensor path must reproduce the integer result bit for bit.
    import torch
    g = torch.Generator(device="cpu").manual_seed(5)
    M = N = 128; K = 256
    Ai = torch.randint(-(2 ** 20), 2 ** 20, (M, K), generator=g, dtype=torch.int64)
    Bi = torch.randint(-(2 ** 20), 2 ** 20, (N, K), generator=g, dtype=torch.int64)
    ref = Ai @ Bi.T
    Bop = Bi if trans_b else Bi.T.contiguous()
    C = torch.zeros(M, N, dtype=torch.float64, device=_dev())
    binding.mbdk_gemm_f64(Ai.double().to(_dev()), Bop.double().to(_dev()), C, mode=0, trans_b=trans_b)
    torch.cuda.synchronize()
    assert torch.equal(C.cpu().to(torch.int64), ref)


@pytest.mark.parametrize("n", [64, 128, 192, 320])
def test_gemm_nt_symmetric_modes(n):
    import torch
    g = torch.Generator(device="cpu").manual_seed(n)
    X = torch.randn(n, n, generator=g, dtype=torch.float64)
    S = (X + X.T).to(_dev())
    T = torch.linalg.matrix_exp(0.01 * (X + X.T)).to(_dev())   # commutes with nothing in general
    C = torch.full((n, n), float("nan"), dtype=torch.float64, device=_dev())
    binding.mbdk_gemm_f64(S, S, C, mode=2)                      # S S^T is symmetric
    ref = S @ S.T
    torch.cuda.synchronize()
    assert torch.allclose(C, ref, rtol=1e-13, atol=1e-11)
    # Y Z Y with symmetric Y, Z, through the non-transposed path: P = Z Y, then Y P
    P = torch.empty(n, n, dtype=torch.float64, device=_dev())
    binding.mbdk_gemm_f64(T, S, P, mode=0, trans_b=False)
    C3 = torch.full((n, n), float("nan"), dtype=torch.float64, device=_dev())
    binding.mbdk_gemm_f64(S, P, C3, mode=2, trans_b=False)
    torch.cuda.synchronize()
    ref3 = S @ T @ S
    assert torch.allclose(C3, ref3, rtol=1e-12, atol=1e-10)
    C2 = torch.zeros(n, n, dtype=torch.float64, device=_dev())
    binding.mbdk_gemm_f64(S, T, C2, mode=1)
    ref2 = S @ T.T
    tri = torch.ones(n // 64, n // 64).tril().repeat_interleave(64, 0).repeat_interleave(64, 1).bool().to(_dev())
    assert torch.allclose(C2[tri], ref2[tri], rtol=1e-13, atol=1e-11)
    assert torch.all(C2[~tri] == 0)


@pytest.mark.parametrize("ld,batch", [(64, 1), (128, 3), (192, 2), (448, 16)])
def test_cholesky_and_solves(ld, batch):
    import torch
    g = torch.Generator(device="cpu").manual_seed(ld * 7 + batch)
    X = torch.randn(batch, ld, ld, generator=g, dtype=torch.float64)
    A = X @ X.transpose(1, 2) / ld + torch.eye(ld, dtype=torch.float64)
    Ad = A.to(_dev()).contiguous()
    # poison the upper triangle: the factorisation must read the lower triangle only
    upper = torch.ones(ld, ld, dtype=torch.bool).triu(1).to(_dev())
    Ad[:, upper] = float("nan")
    dinv = torch.zeros(batch * (ld // 64) * 4096, dtype=torch.float64, device=_dev())
    status = torch.zeros(1, dtype=torch.int32, device=_dev())
    binding.mbdk_cholesky_f64(Ad, dinv, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    Lref = torch.linalg.cholesky(A)
    low = ~upper.cpu()
    assert torch.allclose(Ad.cpu()[:, low], Lref[:, low], rtol=1e-12, atol=1e-12)
    Bm = torch.randn(batch, ld, 3, generator=g, dtype=torch.float64)
    Xd = Bm.to(_dev()).contiguous()
    binding.mbdk_chol_solve3_f64(Ad, dinv, Xd)
    torch.cuda.synchronize()
    ref = torch.linalg.solve(A, Bm)
    assert torch.allclose(Xd.cpu(), ref, rtol=1e-10, atol=1e-11)


def test_cholesky_flags_indefinite():
    import torch
    ld = 128
    A = torch.eye(ld, dtype=torch.float64)
    A[70, 70] = -1.0
    Ad = A.unsqueeze(0).to(_dev()).contiguous()
    dinv = torch.zeros(2 * 4096, dtype=torch.float64, device=_dev())
    status = torch.zeros(1, dtype=torch.int32, device=_dev())
    binding.mbdk_cholesky_f64(Ad, dinv, status)
    torch.cuda.synchronize()
    assert status.item() & 2
