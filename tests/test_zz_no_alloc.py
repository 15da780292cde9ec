"""The allocation-free factor-and-solve entry point against the allocating pair
(mbdk_cholesky_f64 + mbdk_chol_solve3_f64), through the C ABI.

Kept in its own file, collected last, so that a run stopping at the first failure
has already run every other test."""
import pytest

from paper_2308_03140_gb300 import binding, build

pytestmark = pytest.mark.gpu


def _spd(batch, ld, seed):
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    X = torch.randn(batch, ld, ld, generator=g, dtype=torch.float64)
    A = X @ X.transpose(1, 2) / ld + torch.eye(ld, dtype=torch.float64)
    B = torch.randn(batch, ld, 3, generator=g, dtype=torch.float64)
    return A, B


def test_noalloc_factor_solve_matches_allocating_entry_points():
    import torch
    build.build()
    binding.load()
    dev = torch.device("cuda:0")
    # two calls in a row with different sizes and data: the shared scratch must not leak
    for batch, ld, seed in ((3, 192, 11), (16, 256, 12)):
        A, B = _spd(batch, ld, seed)
        # allocating path: caller-provided diagonal-block-inverse buffer
        A_ref, X_ref = A.to(dev).contiguous(), B.to(dev).contiguous()
        dinv = torch.zeros(batch * (ld // 64) * 4096, dtype=torch.float64, device=dev)
        st_ref = torch.zeros(1, dtype=torch.int32, device=dev)
        binding.mbdk_cholesky_f64(A_ref, dinv, st_ref)
        binding.mbdk_chol_solve3_f64(A_ref, dinv, X_ref)
        # allocation-free path
        A_na, X_na = A.to(dev).contiguous(), B.to(dev).contiguous()
        st_na = torch.zeros(1, dtype=torch.int32, device=dev)
        rc = binding.mbdk_cholesky_solve3_f64_noalloc(A_na, X_na, st_na)
        torch.cuda.synchronize()
        assert rc == 0
        assert st_ref.item() == 0 and st_na.item() == 0
        low = torch.ones(ld, ld, dtype=torch.bool, device=dev).tril()
        assert torch.allclose(A_na[:, low], A_ref[:, low], rtol=1e-12, atol=1e-12)
        assert torch.allclose(X_na, X_ref, rtol=1e-10, atol=1e-11)
        # and both solve the system
        assert torch.allclose(X_na.cpu(), torch.linalg.solve(A, B), rtol=1e-10, atol=1e-11)


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    import torch
    build.build()
    binding.load()
    dev = torch.device("cuda:0")
    batch, ld = 512, 64     # 512 * (1 * 4096 + 3 * 64) doubles > 2^21
    A = torch.eye(ld, dtype=torch.float64, device=dev).repeat(batch, 1, 1).contiguous()
    X = torch.zeros(batch, ld, 3, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    assert binding.mbdk_cholesky_solve3_f64_noalloc(A, X, st) == 9   # MBD_ERR_SCRATCH_LIMIT
