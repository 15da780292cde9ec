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
            names |= set(re.findall(r"^\s*int\s+(mbdk?_\w+)\s*\(", txt, flags=re.M))
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
