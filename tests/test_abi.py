"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/mbd_gb300.h declares (no GPU needed: no compute call is made)."""
import ctypes as C
import os
import re

import pytest

from paper_2308_03140_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|size_t)\s+(mbdk?_\w+)\s*\(", txt, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    decl = declared_symbols()
    assert decl, "no declarations found"
    assert decl == set(binding.EXPORTS)
    for name in decl:
        assert hasattr(lib, name), name


def test_default_options(lib):
    opt = binding.mbd_options()
    assert lib.mbd_default_options(C.byref(opt)) == 0
    assert opt.n_freq == 15 and opt.beta == 0.83 and opt.a == 6.0
    assert lib.mbd_default_options(None) == 1   # MBD_ERR_INPUT


def test_library_is_sm103a_only():
    # the build passes exactly one -gencode, for sm_103a
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _create(lib, **fields):
    opt = binding.mbd_options()
    lib.mbd_default_options(C.byref(opt))
    for k, v in fields.items():
        setattr(opt, k, v)
    h = C.c_void_p()
    return lib.mbd_create(C.byref(h), 0, C.byref(opt)), h


@pytest.mark.parametrize("field,value", [("n_freq", 0), ("n_freq", 10 ** 6), ("beta", 0.0), ("a", -1.0),
                                         ("ns_max_iter", 0), ("ns_tol", 0.0), ("precision", 9),
                                         ("tc_chunk_stages", -1), ("scs_mode", 3), ("learned_max_error", 0.0),
                                         ("mixed_max_error", 0.0), ("learned_estimate_scale", 0.0),
                                         ("learned_estimate_scale", float("inf"))])
def test_create_rejects_invalid_options_before_touching_the_device(lib, field, value):
    rc, h = _create(lib, **{field: value})
    assert rc == 1 and not h.value   # MBD_ERR_INPUT, no context


def test_learned_mode_needs_the_models_frequency_grid(lib):
    rc, h = _create(lib, scs_mode=binding.MBD_SCS_LEARNED, n_freq=10)
    assert rc == 1 and not h.value


def test_create_accepts_every_method_and_precision(lib):
    # valid options pass validation; without a GPU the device query then fails (MBD_ERR_CUDA)
    import torch
    for mode in (binding.MBD_SCS_PLAIN, binding.MBD_SCS_LEARNED, binding.MBD_SCS_NL):
        for prec in (binding.MBD_PREC_FP64, binding.MBD_PREC_TF32, binding.MBD_PREC_BF16X3, binding.MBD_PREC_TF32X3,
                     binding.MBD_PREC_FP64_SPLIT):
            rc, h = _create(lib, scs_mode=mode, precision=prec)
            if torch.cuda.is_available():
                assert rc == 0
                lib.mbd_destroy(h)
            else:
                assert rc == 6 and not h.value   # MBD_ERR_CUDA
    assert lib.mbd_destroy(None) == 0


def test_binding_marshalling():
    import numpy as np
    import torch
    a = binding._f64([[1, 2, 3], [4, 5, 6]], (-1, 3))
    assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == (2, 3)
    b = binding._f64(np.arange(12.0).reshape(3, 4)[:, ::2])   # strided input is copied densely
    assert b.flags.c_contiguous and b.tolist() == [[0.0, 2.0], [4.0, 6.0], [8.0, 10.0]]
    with pytest.raises(ValueError):
        binding._f64([1.0, 2.0], (-1, 3))
    t = torch.zeros(4, 6, dtype=torch.float64)
    assert binding._tptr(t).value == t.data_ptr() and binding._tptr(None) is None
    with pytest.raises(ValueError):
        binding._tptr(t.t())                                  # a transposed view is refused


def test_null_context_calls_return_input_error(lib):
    # every context call checks its handle before any device work; this also exercises the
    # argument marshalling of each signature (ctypes raises on a count mismatch)
    E = C.c_double()
    assert lib.mbd_ts_energy(None, 0.94, C.byref(E), None, None, None) == 1
    assert lib.mbd_log_energy(None, 2, C.byref(E), None) == 1
    assert lib.mbd_evaluate(None, C.byref(E), None, None, None, None) == 1
    with pytest.raises(TypeError):
        lib.mbd_ts_energy(None, 0.94, C.byref(E), None, None)      # the old five-argument form


def test_split_gemm_entry_checks_arguments_before_any_device_work(lib):
    # sizes are validated first (no device call); the workspace size is plain arithmetic
    assert lib.mbdk_gemm_f64_split_work_bytes(128, 256, 64) == 9 * (128 + 256) * 64 * 4 + (128 + 256) * 4
    assert lib.mbdk_gemm_f64_split_work_bytes(0, 256, 64) == 0
    args = dict(trans_b=1, M=128, N=96, K=64)   # N not a multiple of 128
    rc = lib.mbdk_gemm_f64_split(None, args["trans_b"], args["M"], args["N"], args["K"], 1.0, None, 64, None, 64,
                                 0.0, None, 0, None, 96, None, None)
    assert rc == 1
