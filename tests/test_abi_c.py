"""The C ABI as a C program sees it (no GPU needed): tests/abi_c_check.c includes both public
headers under -std=c99 -pedantic -Wall -Wextra -Werror, links against libmbdgb.so and runs.
The struct layouts it prints must equal the ctypes structs of the binding (the two clients
of one ABI), the defaults must be the documented ones, and the calls that must fail before
any device work return their documented codes."""
import os
import shutil
import subprocess

import pytest

from paper_2308_03140_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "_build")


@pytest.fixture(scope="module")
def report():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    os.makedirs(OUT, exist_ok=True)
    exe = os.path.join(OUT, "abi_c_check")
    libdir = os.path.dirname(lib)
    cmd = [cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-O1",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_c_check.c"),
           "-L", libdir, "-lmbdgb", f"-Wl,-rpath,{libdir}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.splitlines()
    sizes = {l.split()[1]: int(l.split()[2]) for l in lines if l.startswith("sizeof ")}
    offsets = {(l.split()[1], l.split()[2]): int(l.split()[3]) for l in lines if l.startswith("offset ")}
    rcs = {l.split()[1]: int(l.split()[2]) for l in lines if l.startswith("rc ")}
    defaults = next(l for l in lines if l.startswith("default ")).split()[1:]
    defaults = dict(zip(defaults[0::2], defaults[1::2]))
    misc = {l.split()[0]: l.split()[1] for l in lines if l.startswith(("ctx_after", "split_work"))}
    return sizes, offsets, rcs, defaults, misc


@pytest.mark.parametrize("name,struct", [("mbd_options", binding.mbd_options), ("mbd_profile", binding.mbd_profile)])
def test_struct_layouts_match_the_binding(report, name, struct):
    sizes, offsets, _, _, _ = report
    import ctypes as C
    assert sizes[name] == C.sizeof(struct)
    fields = [f for f, _ in struct._fields_]
    assert {f for (s, f) in offsets if s == name} == set(fields)
    for f in fields:
        assert offsets[(name, f)] == getattr(struct, f).offset, f


def test_defaults_seen_from_c(report):
    _, _, rcs, d, _ = report
    assert rcs["default_options"] == 0 and rcs["default_options_null"] == 1
    assert int(d["n_freq"]) == 15 and float(d["beta"]) == 0.83 and float(d["a"]) == 6.0
    assert int(d["precision"]) == binding.MBD_PREC_FP64 and float(d["ns_tol"]) == 1e-8
    assert int(d["ns_max_iter"]) == 100 and int(d["tc_chunk_stages"]) == 0
    assert int(d["scs_mode"]) == binding.MBD_SCS_PLAIN
    assert float(d["learned_max_error"]) == 1e-6 and float(d["mixed_max_error"]) == 1e-7
    assert float(d["learned_estimate_scale"]) == 1.0


def test_calls_that_fail_before_device_work(report):
    _, _, rcs, _, misc = report
    assert rcs["create_bad_n_freq"] == 1 and misc["ctx_after_failed_create"] == "null"   # MBD_ERR_INPUT
    assert rcs["create_null_out"] == 1
    assert rcs["destroy_null"] == 0
    assert rcs["evaluate_null"] == 1 and rcs["evaluation_count_null"] == 1 and rcs["exception_null"] == 1
    assert int(misc["split_work_bytes"]) == 9 * (128 + 256) * 64 * 4 + (128 + 256) * 4
