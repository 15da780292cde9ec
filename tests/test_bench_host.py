"""Host arithmetic of bench.py's JSON line (no GPU): the roofline object of the dominant kernel
from per-step profiles, the peaks it divides by, the DRAM traffic it quotes only for the
captured source, and the per-result errors of an arm against the FP64 path."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2308_03140_gb300 import binding  # noqa: E402  (constants only; the library is not loaded)


def _profs(steps, tc_ms, tc_flops, tc_launches, gemm_ms=0.0, gemm_flops=0.0, gemm_launches=0):
    return [dict(tc_ms=tc_ms, tc_flops=tc_flops, tc_launches=tc_launches, gemm_ms=gemm_ms,
                 gemm_flops=gemm_flops, gemm_launches=gemm_launches) for _ in range(steps)]


@pytest.fixture
def peaks(monkeypatch):
    p = {"bf16_tflops_sustained": 1500.0, "hbm_gbs": 7000.0}
    monkeypatch.setattr(bench, "measured_peaks", lambda: p)
    return p


def test_tensor_core_roofline_per_kind(peaks):
    # 4 steps, each 30 launches of 1e15 algorithmic flop in 2000 ms of kernel time
    profs = _profs(4, 2000.0, 30e15, 30)
    for prec, name, ratio, products in ((binding.MBD_PREC_BF16X3, "bf16x3", 1.0, 3),
                                        (binding.MBD_PREC_TF32X3, "tf32x3", 0.5, 3),
                                        (binding.MBD_PREC_TF32, "tf32", 0.5, 1)):
        r = bench.roofline_of(binding, name, prec, profs, 10000.0, 4, "finite2000")
        assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
        assert r["achieved"] == pytest.approx(4 * 30e15 / 8.0 / 1e12)    # flop / s over all launches
        assert r["peak"] == pytest.approx(1500.0 * ratio / products)
        assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
        assert r["launches_per_step"] == 30 and r["avg_launch_ms"] == pytest.approx(8000.0 / 120)
        assert r["flops_per_launch"] == pytest.approx(1e15)
        assert r["share_of_step"] == pytest.approx(0.8)
        assert r["peak_source"].startswith("of measured")
        assert r["traffic"] is None   # no capture for this workload


def test_fp64_roofline_and_fallback_peak(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: None)
    profs = _profs(2, 0.0, 0.0, 0, gemm_ms=500.0, gemm_flops=4e14, gemm_launches=20)
    r = bench.roofline_of(binding, "fp64", binding.MBD_PREC_FP64, profs, 1000.0, 2, "finite8000")
    assert r["peak"] == pytest.approx(1700.0 * 1.25 / 2250.0)
    assert r["peak_source"].startswith("of fallback")
    assert r["achieved"] == pytest.approx(8e14 / 1.0 / 1e12)
    assert r["traffic"] is None


def test_traffic_only_for_the_captured_source(peaks, monkeypatch):
    rec = bench.TC_GEMM_TRAFFIC[("bf16x3", "finite8000")]
    profs = _profs(1, 100.0, 1e15, 30)
    monkeypatch.setattr(bench, "tc_region_sha16", lambda path: rec["k_tc_region_sha16"])
    r = bench.roofline_of(binding, "bf16x3", binding.MBD_PREC_BF16X3, profs, 200.0, 1, "finite8000")
    assert r["traffic"] == rec["bytes"] and r["traffic_launch"] == rec["source"]
    assert os.path.exists(os.path.join(ROOT, rec["source"]))
    monkeypatch.setattr(bench, "tc_region_sha16", lambda path: "0" * 16)
    r = bench.roofline_of(binding, "bf16x3", binding.MBD_PREC_BF16X3, profs, 200.0, 1, "finite8000")
    assert r["traffic"] is None and r["traffic_launch"] is None


def test_region_hashes_read_the_sources():
    # the hash functions find their regions in the present sources (a renamed marker line
    # would make them raise, and the bench would then fail instead of quoting stale traffic)
    csrc = os.path.join(ROOT, "paper_2308_03140_gb300", "csrc")
    for f, path in ((bench.tc_region_sha16, "k_tc.cu"), (bench.gemm_region_sha16, "k_dense.cu")):
        h = f(os.path.join(csrc, path))
        assert len(h) == 16 and int(h, 16) >= 0


def test_errors_against_the_fp64_path():
    rng = np.random.default_rng(3)
    N = 5
    ref = {"energy": -1.0, "gR": rng.normal(size=(N, 3)), "gp": rng.normal(size=(4, N)), "gA": None}
    arm = {"energy": -1.0 + 5e-8, "gR": ref["gR"].copy(), "gp": ref["gp"].copy(), "gA": None}
    arm["gR"][2, 1] += 1e-6
    arm["gp"][3, 4] -= 2e-6
    e = bench.errors_vs(arm, ref, N)
    assert e["delta_e_per_atom_ha"] == pytest.approx(1e-8)
    assert e["max_force_err_ha_bohr"] == pytest.approx(1e-6)
    assert e["max_force_err_rel"] == pytest.approx(1e-6 / np.abs(ref["gR"]).max())
    assert e["max_param_grad_err"] == pytest.approx(2e-6)
    rel = e["max_param_grad_err_rel"]
    assert rel[:3] == [0.0, 0.0, 0.0] and rel[3] == pytest.approx(2e-6 / np.abs(ref["gp"][3]).max())
    assert "max_lattice_grad_err_rel" not in e
    # learned arms have no parameter gradients; cells add the lattice gradient
    arm2 = dict(arm, gp=None, gA=np.eye(3) * 1.001)
    e2 = bench.errors_vs(arm2, dict(ref, gA=np.eye(3)), N)
    assert "max_param_grad_err" not in e2
    assert e2["max_lattice_grad_err_rel"] == pytest.approx(1e-3)


def test_cpu_baseline_object():
    # the GPU arm's cpu_baseline on a tiny sample: the contract's keys, the extrapolation labelled
    cb = bench.cpu_baseline("finite8000", 12, 8000)
    assert cb["kind"] == "oracle" and cb["unit"] == "solves/s" and cb["cores"] >= 1
    assert cb["extrapolated"] is True and "12-atom cluster" in cb["sample"] and "upper bound" in cb["sample"]
    assert cb["value"] == pytest.approx(1.0 / (cb["sample_seconds"] * (8000 / 12) ** 3))


def test_clock_sampler_parses_the_nvidia_smi_rows(tmp_path):
    # rows as `nvidia-smi --format=csv,noheader,nounits` prints them for the sampler's fields
    rows = ["0, 2055, 2070, 1100.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2040, 2070, 1380.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = bench.ClockSampler(0)
    cs.proc, cs.path = _Proc(), str(p)
    c = cs.stop()
    assert c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"] and c["power_w_max"] == pytest.approx(1380.2)
    assert not os.path.exists(p)
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_reference_arm_prints_on_rank_zero_only():
    import subprocess
    base = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
            "--gpus", "2"]
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run(base, capture_output=True, text=True, cwd=ROOT, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
