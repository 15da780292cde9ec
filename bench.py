#!/usr/bin/env python3
"""Benchmark: MBD@rsSCS energy + analytic gradient solves per second on GB300.

One step = one full evaluation (TS scaling, screening at 16 frequency points, Q, coupled
Newton-Schulz Q^{+-1/2}, energy, and all gradients) of the 8000-atom finite cluster
(0.08 atoms/A^3, minimum separation 2.2 bohr; Q is 24000 x 24000) in BF16x3 arithmetic,
inputs resident in HBM.  `e2e` repeats the measurement through the C ABI with host buffers
(host-to-device copies of the inputs and device-to-host copies of energy, gradients and
screened polarizabilities inside the timed region).  Beside it, on the same inputs: the
TF32x3 arm, the FP64 path (one evaluation) against which each arm's energy, force and
parameter-gradient errors are stated; then further workloads, each with its own FP64 arm:
the 2000-atom cluster (Q 6000 x 6000: BF16x3, TF32x3 and the learned screening), the
256-atom cell with 64 Bloch vectors, and a batch of clusters of 50-500 atoms with plain and
learned screening (with and without its fallback).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per GPU, launched by torch.distributed.run);
a single finite Q does not shard.  `--impl reference` times the CPU oracle (the
plain FP64 reference implementation) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MBD energy+gradient solves/s & TFLOP/s vs FP64 GPU path at |ΔE|≤1e-6 Ha/atom"
UNIT = "solves/s"
WORKLOAD = "finite8000"
# Ewald split, real-space and reciprocal cutoffs of the periodic workload (real-space cutoff
# 30 bohr; gamma = 6/30, k_c = 10 gamma)
PERIODIC_EWALD = (0.2, 30.0, 2.0)
N_TARGET = {"finite2000": 2000, "cell256": 256, "finite8000": 8000, "batch4096": 275}
# nominal FP64 : dense BF16 tensor rate of the part (1.25 TFLOP/s : 2250 TFLOP/s)
FP64_OVER_BF16 = 1.25 / 2250.0
# DRAM bytes (read + write) per k_gemm_nn launch from the committed ncu capture
# (profiles/k_gemm_nn_finite2000.md), valid while the GEMM's own source (its tile code,
# kernels and launcher in k_dense.cu) keeps the captured hash.
GEMM_NN_TRAFFIC = {"bytes": 6.309694e9 + 0.289604352e9, "k_gemm_region_sha16": "3aeb35fc6cf2af16",
                   "source": "profiles/k_gemm_nn_finite2000.md"}


def gemm_region_sha16(path):
    """sha256 (first 16 hex) of the FP64 GEMM's source in k_dense.cu: from its tile
    constants to the k_gemm_nn kernel, plus the gemm_f64 launcher."""
    import hashlib
    lines = open(path).read().splitlines()
    i = next(k for k, l in enumerate(lines) if l.startswith("constexpr int BM = "))
    j = next(k for k, l in enumerate(lines) if "k_gemm_nn(GemmArgs g" in l)
    a = next(k for k, l in enumerate(lines) if l.startswith("void gemm_f64("))
    b = next(k for k in range(a, len(lines)) if lines[k] == "}")
    return hashlib.sha256("\n".join(lines[i:j + 1] + lines[a:b + 1]).encode()).hexdigest()[:16]
# DRAM bytes per tensor-core GEMM launch from committed captures, keyed by (precision,
# workload): the mean over the 28 Newton-Schulz and 2 correction products of one BF16x3 step
# of the 8000-atom cluster (1-pass dram__bytes capture of the full-size step;
# profiles/launches_finite8000_bf16x3.md), valid while the GEMM's own source in k_tc.cu (tile
# constants through the tc_gemm dispatcher) keeps the captured hash.
TC_GEMM_TRAFFIC = {("bf16x3", "finite8000"): {"bytes": 52.238774485e9,
                                               "k_tc_region_sha16": "eb40cbc36ad4f016",
                                               "launch": "mean of the 30 Newton-Schulz and correction products "
                                                         "of one step, order 24064",
                                               "source": "profiles/launches_finite8000_bf16x3.md"}}


def tc_region_sha16(path):
    """sha256 (first 16 hex) of the tensor-core GEMM's source in k_tc.cu: from its tile
    constants through the tc_gemm dispatcher (device helpers, kernel, tensor maps, launch)."""
    import hashlib
    lines = open(path).read().splitlines()
    i = next(k for k, l in enumerate(lines) if l.startswith("constexpr int TM = 128"))
    a = next(k for k, l in enumerate(lines) if l.startswith("cudaError_t tc_gemm("))
    b = next(k for k in range(a, len(lines)) if lines[k] == "}")
    return hashlib.sha256("\n".join(lines[i:b + 1]).encode()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("finite2000", "cell256", "finite8000", "batch4096"), default=WORKLOAD,
                    help="finite2000: the 2000-atom cluster; cell256: the periodic cell (64 Bloch vectors); "
                         "finite8000: the large cluster; batch4096: the varlen cluster batch with the learned "
                         "screening model beside plain screening")
    ap.add_argument("--order", type=int, default=6016, help="--kernel tc_gemm_sym: matrix order (multiple of 128)")
    ap.add_argument("--batch-clusters", type=int, default=64,
                    help="batch4096: clusters of the batch evaluated per step (the first ones of the recipe)")
    ap.add_argument("--precision", choices=("bf16x3", "tf32x3", "tf32", "fp64", "fp64split"), default="bf16x3",
                    help="matrix-function arithmetic of the timed arm (the FP64 path is measured beside it)")
    ap.add_argument("--also", default="tf32x3",
                    help="comma-separated further arithmetic arms timed on the same workload ('' for none)")
    ap.add_argument("--other-steps", type=int, default=3, help="timed steps of each further arm (1 warm-up)")
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed steps of the FP64 comparison arm (0: skip; no warm-up at 4000 atoms or more)")
    ap.add_argument("--e2e-steps", type=int, default=5, help="steps of the end-to-end measurement (at most --steps)")
    ap.add_argument("--learned-arm", type=int, default=1,
                    help="1: the finite extra workloads also time the learned screening (no fallback) beside plain")
    ap.add_argument("--extra-workload", default="finite2000,cell256,batch4096",
                    help="comma-separated further workloads measured after the first ('' for none): finite2000 "
                         "and cell256 in the timed arm's and --also arithmetic with their own FP64 arm; batch4096 "
                         "= --batch-clusters clusters of the varlen batch, plain against learned screening")
    ap.add_argument("--extra-steps", type=int, default=5, help="timed steps of each further workload (1 warm-up)")
    ap.add_argument("--extra-fp64-steps", type=int, default=1, help="timed FP64 steps of each further workload")
    ap.add_argument("--cpu-sample-atoms", type=int, default=320,
                    help="atoms of the bounded oracle sample (same recipe, extrapolated by n^3)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--method", choices=("rsscs", "nl"), default="rsscs",
                    help="rsscs: MBD@rsSCS (the headline); nl: MBD-NL (Sec. 2.7: no screening, oscillators "
                         "from the free-atom reference and density-functional ratios drawn by "
                         "synthetic.nl_ratios(N, seed=7000))")
    ap.add_argument("--kernel", choices=("tc_gemm_sym", "tc_gemm_sym6016", "tc_gemm_update", "log_energy_finite2000",
                                         "ts_finite2000", "ts_cell256", "gemm_f64_split6016"),
                    default=None,
                    help="time one kernel or route alone instead of the workload: tc_gemm_sym = the "
                         "symmetric Newton-Schulz product in the --precision split kind (bf16x3 or tf32x3) at order "
                         "--order (k_tc_gemm mode 2, the library chunk lengths; at 6016 a small case for profilers, about "
                         "0.9 GB on the device; tc_gemm_sym6016 is the same at 6016); tc_gemm_update = the "
                         "trailing update of the screening's FP32 Cholesky, C = D - L21 L21^T on the lower tiles of "
                         "order --order with a 512-column panel (k_tc_gemm mode 1, one matrix); "
                         "log_energy_finite2000 = the log-formula energy route (mbd_log_energy, orders 2) of the "
                         "2000-atom cluster after a TF32x3 evaluation; ts_finite2000 = the TS pairwise energy "
                         "and gradients (mbd_ts_energy) of the 2000-atom cluster; ts_cell256 = the same per cell of "
                         "the 256-atom triclinic cell with the lattice gradient (Eq. ts-ewald); "
                         "gemm_f64_split6016 = the FP64-accurate split GEMM against the FP64 GEMM at order 6016")
    args = ap.parse_args()
    args.also = [x for x in args.also.split(",") if x]
    args.extra_workload = [x for x in args.extra_workload.split(",") if x]
    for x in args.extra_workload:
        if x not in ("finite2000", "cell256", "finite8000", "batch4096"):
            ap.error(f"--extra-workload: unknown workload {x}")
    for x in args.also:
        if x not in ("bf16x3", "tf32x3", "tf32", "fp64split"):
            ap.error(f"--also: unknown arithmetic {x}")
    return args


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = max((num(r[2]) for r in rows if num(r[2]) is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def sample_system(workload: str, n_sample: int):
    """Bounded same-recipe sample of a workload for the CPU oracle: a cluster of n_sample
    atoms (finite), or a cell of n_sample atoms with edges scaled to keep the density and the
    same k-grid and cutoffs (periodic)."""
    from paper_2308_03140_gb300 import synthetic as syn
    if workload == "cell256":
        f = (n_sample / 256.0) ** (1.0 / 3.0)
        return syn.triclinic_cell(n_sample, edge=(20.0 * f, 26.0 * f), seed=2000)
    return syn.sphere_cluster(n_sample, seed=1000)


NL_SEED = 7000   # stream of the MBD-NL density-functional ratios of a workload


def oracle_solve(sysm, method="rsscs"):
    """One energy+gradient by the CPU oracle (as it stands)."""
    import oracle as o
    if method == "nl":
        from paper_2308_03140_gb300 import synthetic as syn
        ra, rw = syn.nl_ratios(sysm.n_atoms, NL_SEED)
        if sysm.lattice is not None:
            raise ValueError("the oracle's MBD-NL arm covers finite systems")
        return o.mbd_nl(sysm.coords, sysm.alpha0_ref, sysm.c6_ref, ra, rw, grad=True)
    if sysm.lattice is not None:
        g, rc, kc = PERIODIC_EWALD
        return o.periodic_rsscs_gradient(sysm.coords, sysm.lattice, o.monkhorst_pack(sysm.k_grid),
                                         sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio, g, rc, kc)
    return o.mbd_rsscs_gradient(*o.system_args(sysm), mode="adjoint")


def cpu_baseline(workload: str, n_sample: int, n_target: int, method: str = "rsscs"):
    """Times the CPU oracle (as it stands) on a same-recipe sample of n_sample atoms and
    extrapolates to n_target atoms by the cubic cost of its dense stages."""
    sysm = sample_system(workload, n_sample)
    t0 = time.perf_counter()
    oracle_solve(sysm, method)
    dt = time.perf_counter() - t0
    scale = (n_target / n_sample) ** 3
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    kind = "cell" if sysm.lattice is not None else "cluster"
    return {"value": 1.0 / (dt * scale), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"energy+gradient of a {n_sample}-atom {kind} of the same recipe in "
                      f"{dt:.2f} s, extrapolated by (n/{n_sample})^3 to {n_target} atoms (the oracle's cost "
                      f"grows faster than n^3 at these sizes, so the extrapolated rate is an upper bound)",
            "sample_seconds": dt, "extrapolated": True}


def reduce_max(x: float, world: int, device) -> float:
    """The largest x over the ranks of the process group (x itself when world == 1): the
    timed region of a multi-rank run ends when its slowest rank does."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds_max


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    n_target = N_TARGET[args.workload]
    n_s = min(args.cpu_sample_atoms, 200) if args.workload != "cell256" else 32
    sysm = sample_system(args.workload, n_s)
    for _ in range(args.warmup):
        oracle_solve(sysm, args.method)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_solve(sysm, args.method)
        times.append(time.perf_counter() - t0)
    dt = sum(times)
    scale = (n_target / n_s) ** 3
    value = args.steps / (dt * scale)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    kind = "cell" if sysm.lattice is not None else "cluster"
    from paper_2308_03140_gb300 import synthetic as syn
    full = syn.workload(args.workload)
    sample = (f"each step one energy+gradient of a {n_s}-atom {kind} of the same recipe (measured: "
              f"{1e3 * dt / args.steps:.0f} ms per step), extrapolated by ({n_target}/{n_s})^3 to the workload "
              f"(the oracle's cost grows faster than n^3 at these sizes, so the extrapolated rate is an upper bound)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "ms_per_step_extrapolated": 1e3 * dt * scale / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "precision": "fp64", "data": "synthetic",
            "config": workload_config(args.workload, args.method, n_target, world, full.lattice is not None, full),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "sample_atoms": n_s, "extrapolated": True},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(workload, method, n_atoms, world, periodic=False, sysm=None):
    """The workload's description, shared by both arms of the bench (so their configs match)."""
    import numpy as np
    n = 3 * n_atoms
    cfg = {"workload": workload, "method": "MBD-NL" if method == "nl" else "MBD@rsSCS", "n_atoms": n_atoms,
           "matrix_order": n, "n_freq": 15,
           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}
    if periodic:
        nk = int(np.prod(sysm.k_grid))
        cfg["l2"] = (f"inputs larger than L2: 5 Newton-Schulz sets of {nk} complex {n}x{n} matrices "
                     f"({16 * n * n * nk / 1e6:.0f} MB each set)")
        cfg.update({"lattice_bohr": np.asarray(sysm.lattice).round(4).tolist(), "k_grid": list(sysm.k_grid),
                    "ewald_gamma": PERIODIC_EWALD[0], "real_cutoff_bohr": PERIODIC_EWALD[1],
                    "recip_cutoff_per_bohr": PERIODIC_EWALD[2]})
    else:
        cfg["l2"] = (f"inputs larger than L2: 16 screening matrices + 5 Newton-Schulz matrices of "
                     f"{8 * n * n / 1e6:.0f} MB each per step")
    return cfg


PRECISIONS = ("fp64", "tf32", "bf16x3", "tf32x3", "fp64split")


def precision_code(binding, name):
    return {"fp64": binding.MBD_PREC_FP64, "tf32": binding.MBD_PREC_TF32, "bf16x3": binding.MBD_PREC_BF16X3,
            "tf32x3": binding.MBD_PREC_TF32X3, "fp64split": binding.MBD_PREC_FP64_SPLIT}[name]


def time_arm(binding, dev, stream, sysm, p3, p4, precision, scs_mode, steps, warmup, barrier=None,
             max_over_ranks=None, clocks=None, learned=None):
    """One context, `warmup` untimed and `steps` timed device evaluations (energy and all
    gradients, inputs resident in HBM) bracketed by CUDA events on the launch stream.  With
    `learned` (the model file's arrays) the screening is the learned model's, without its
    fallback, and the gradients are the coordinate ones (learned mode has no parameter
    gradients).  Returns the timing, the last results (host copies) and the per-step profiles."""
    import numpy as np
    import torch
    N = sysm.n_atoms
    periodic = sysm.lattice is not None
    T = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev)
    inp = [T(sysm.coords), T(sysm.alpha0_ref), T(sysm.c6_ref), T(p3), T(p4)]
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    gR = torch.zeros(N, 3, dtype=torch.float64, device=dev)
    gp = torch.zeros(4, N, dtype=torch.float64, device=dev)
    al = torch.zeros(N, dtype=torch.float64, device=dev)
    ewald = dict(ewald_gamma=PERIODIC_EWALD[0], real_cutoff=PERIODIC_EWALD[1],
                 recip_cutoff=PERIODIC_EWALD[2]) if periodic else {}
    lopt = dict(scs_mode=binding.MBD_SCS_LEARNED, learned_max_error=1e300) if learned is not None else \
        dict(scs_mode=scs_mode)
    m = binding.MBD(dev.index or 0, precision=precision, **lopt, **ewald)
    if learned is not None:
        m.set_scs_model(learned["params16"], learned["mean"], learned["std"])
        gp = None
    m.set_geometry(sysm.coords, sysm.lattice, sysm.k_grid)
    m.set_free_atom_params(sysm.alpha0_ref, sysm.c6_ref, p3, p4)

    def step():
        m.evaluate_dev(*inp, energy, gR, gp, al, stream=stream)

    for _ in range(warmup):
        step()
    m.set_profiling(True)
    if barrier:
        barrier()
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    profs = []
    for _ in range(steps):
        step()
        profs.append(m.profile())
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop() if clocks else None
    if barrier:
        barrier()
    ms = ev0.elapsed_time(ev1)
    if max_over_ranks:
        ms = max_over_ranks(ms)
    m.set_profiling(False)
    out = {"ms": ms, "steps": steps, "warmup": warmup, "energy": energy.item(), "gR": gR.cpu().numpy().copy(),
           "gp": gp.cpu().numpy().copy() if gp is not None else None, "profs": profs, "stats": m.stats(),
           "clocks": clk, "ctx": m,
           "gA": m.lattice_gradient() if periodic else None}
    return out


def errors_vs(arm, ref, N):
    """Per-result error of an arm against the FP64 path on the same inputs."""
    import numpy as np
    gpr = np.abs(ref["gp"]).max(axis=1)
    params = {} if arm["gp"] is None else {
        "max_param_grad_err": float(np.abs(arm["gp"] - ref["gp"]).max()),
        "max_param_grad_err_rel": [float(np.abs(arm["gp"][k] - ref["gp"][k]).max() / gpr[k]) for k in range(4)]}
    return {"delta_e_per_atom_ha": (arm["energy"] - ref["energy"]) / N,
            "max_force_err_ha_bohr": float(np.abs(arm["gR"] - ref["gR"]).max()),
            "max_force_ha_bohr": float(np.abs(ref["gR"]).max()),
            "max_force_err_rel": float(np.abs(arm["gR"] - ref["gR"]).max() / np.abs(ref["gR"]).max()),
            **params,
            **({"max_lattice_grad_err_rel": float(np.abs(arm["gA"] - ref["gA"]).max() / np.abs(ref["gA"]).max())}
               if arm.get("gA") is not None and ref.get("gA") is not None else {})}


def roofline_of(binding, args_precision, precision, profs, ms, steps, workload):
    """Roofline of the dominant kernel of an arm from the library's CUDA-event profile."""
    gemm_ms = sum(p["gemm_ms"] for p in profs)
    gemm_flops = sum(p["gemm_flops"] for p in profs)
    gemm_launches = sum(p["gemm_launches"] for p in profs)
    peaks = measured_peaks()
    bf16_sus = peaks.get("bf16_tflops_sustained") if peaks else None
    src = "of measured" if bf16_sus else "of fallback"
    bf16_sus = bf16_sus or 1700.0
    if precision == binding.MBD_PREC_FP64_SPLIT:
        kernel = "k_tc_gemm<TF32> slice products of the split FP64 GEMM (Newton-Schulz products)"
        k_ms, k_flops, k_launches = gemm_ms, gemm_flops, gemm_launches
        peak = bf16_sus * 0.5 / 53
        peak_src = (f"{src}: bf16_tflops_sustained x nominal TF32/BF16 rate (0.5) / 53 slice products per "
                    "algorithmic product")
        traffic, tsrc = None, None
    elif precision == binding.MBD_PREC_FP64:
        kernel = "k_gemm_nn (FP64 mma.sync m8n8k4, Newton-Schulz products)"
        k_ms, k_flops, k_launches = gemm_ms, gemm_flops, gemm_launches
        peak = bf16_sus * FP64_OVER_BF16
        peak_src = f"{src}: bf16_tflops_sustained x nominal FP64/BF16 ratio (1.25/2250)"
        cur = gemm_region_sha16(os.path.join(ROOT, "paper_2308_03140_gb300", "csrc", "k_dense.cu"))
        ok = workload == "finite2000" and cur == GEMM_NN_TRAFFIC["k_gemm_region_sha16"]
        traffic, tsrc = (GEMM_NN_TRAFFIC["bytes"], GEMM_NN_TRAFFIC["source"]) if ok else (None, None)
    else:
        kernel = "k_tc_gemm (tcgen05 + TMA + TMEM; Newton-Schulz and correction products)"
        k_ms = sum(p["tc_ms"] for p in profs)
        k_flops = sum(p["tc_flops"] for p in profs)
        k_launches = sum(p["tc_launches"] for p in profs)
        per_kind = {binding.MBD_PREC_TF32: (0.5, 1, "TF32"), binding.MBD_PREC_BF16X3: (1.0, 3, "BF16x3"),
                    binding.MBD_PREC_TF32X3: (0.5, 3, "TF32x3")}[precision]
        peak = bf16_sus * per_kind[0] / per_kind[1]
        peak_src = (f"{src}: bf16_tflops_sustained x nominal {per_kind[2][:4]}/BF16 rate ({per_kind[0]}) / "
                    f"{per_kind[1]} tensor products per algorithmic product")
        cur = tc_region_sha16(os.path.join(ROOT, "paper_2308_03140_gb300", "csrc", "k_tc.cu"))
        rec = TC_GEMM_TRAFFIC.get((args_precision, workload))
        traffic, tsrc = ((rec["bytes"], rec["source"]) if rec and cur == rec["k_tc_region_sha16"] else (None, None))
    achieved = k_flops / (k_ms / 1e3) / 1e12 if k_ms > 0 else None
    return {"kernel": kernel, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "traffic_unit": "bytes per launch (ncu capture)", "traffic_launch": tsrc, "peak_source": peak_src,
            "launches_per_step": k_launches / steps, "avg_launch_ms": k_ms / max(k_launches, 1),
            "flops_per_launch": k_flops / max(k_launches, 1), "share_of_step": k_ms / ms if ms > 0 else None}


def stage_means(profs):
    return {k: statistics.mean(p[k] for p in profs) for k in
            ("screening_ms", "newton_schulz_ms", "correction_ms", "gradient_ms", "total_ms")}


def run_ours(args):
    import numpy as np
    import torch
    from paper_2308_03140_gb300 import binding, build
    from paper_2308_03140_gb300 import synthetic as syn
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    build.build()
    binding.load()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, world, dev)

    sysm = syn.workload(args.workload)
    periodic = sysm.lattice is not None
    if periodic and args.precision == "fp64split":
        args.precision = "fp64"   # cells have no split-FP64 path
    N = sysm.n_atoms
    nl = args.method == "nl"
    # per-atom parameter slots 3 and 4: R_vdW,ref and the volume ratio, or the MBD-NL ratios
    p3, p4 = syn.nl_ratios(N, NL_SEED) if nl else (sysm.rvdw_ref, sysm.ratio)
    scs_mode = binding.MBD_SCS_NL if nl else binding.MBD_SCS_PLAIN
    stream = torch.cuda.Stream(device=dev)
    precision = precision_code(binding, args.precision)
    main = time_arm(binding, dev, stream, sysm, p3, p4, precision, scs_mode, args.steps, args.warmup, barrier,
                    max_over_ranks, ClockSampler(local))
    m = main["ctx"]
    ms = main["ms"]
    value = whole_job_rate(args.steps, world, ms / 1e3)

    # end to end through the C ABI with host buffers: inputs uploaded, energy and gradients
    # read back inside the timed region, every step
    e2e_steps = min(args.steps, args.e2e_steps)
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        m.set_geometry(sysm.coords, sysm.lattice, sysm.k_grid)
        m.set_free_atom_params(sysm.alpha0_ref, sysm.c6_ref, p3, p4)
        E_h, gR_h, gp_h, al_h = m.evaluate(True)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * e2e_steps / e2e_s, "unit": UNIT, "steps": e2e_steps,
           "h2d_bytes_per_step": 8 * (3 * N + 4 * N),
           "d2h_bytes_per_step": 8 * (1 + 3 * N + 4 * N + N + (9 if periodic else 0))}
    if periodic:
        e2e["h2d_bytes_per_step"] += 8 * 9 + 4 * 3   # lattice and k-grid
    st = main["stats"]
    profs = main["profs"]
    m.close()
    main["ctx"] = None
    torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if precision == binding.MBD_PREC_FP64 else f"{args.precision}+f32+f64",
        "precision": args.precision, "data": "synthetic",
        "config": workload_config(args.workload, args.method, N, world, periodic, sysm),
    }
    exec_flops = sum(p["gemm_flops"] + p["tc_flops"] + p["screening_flops"] for p in profs) / args.steps
    n = 3 * N
    line["tflops"] = exec_flops / (ms / args.steps / 1e3) / 1e12
    # the work the method needs at least (finite systems): 16 Cholesky factorisations with
    # their 3-RHS solves (none for MBD-NL) and ~9 n^3 for an eigendecomposition of Q
    line["tflops_algorithmic_min"] = (None if periodic else
                                      ((0.0 if nl else 16.0 * (n ** 3 / 3.0 + 12.0 * n ** 2)) + 9.0 * n ** 3)
                                      / (ms / args.steps / 1e3) / 1e12)
    line["roofline"] = roofline_of(binding, args.precision, precision, profs, ms, args.steps, args.workload)
    line["e2e"] = e2e
    line["clocks"] = main["clocks"]
    line["gpu_launches"] = sum(p["launches"] for p in profs)
    line["energy_ha"] = main["energy"]
    line["energy_per_atom_ha"] = main["energy"] / N
    line["ns_iterations"] = st["ns_iterations"]
    line["stage_ms"] = stage_means(profs)
    line["ns_residual"] = st["ns_residual"]
    line["correction_residual"] = st["correction_residual"]

    # other arithmetic on the same workload (same API, fewer steps), then the FP64 path, against
    # which every arm's error is stated
    arms = {}
    for other in args.also:
        if other == args.precision or (periodic and other == "fp64split"):
            continue
        a = time_arm(binding, dev, stream, sysm, p3, p4, precision_code(binding, other), scs_mode,
                     max(1, args.other_steps), 1, barrier, max_over_ranks)
        a["ctx"].close()
        arms[other] = a
        torch.cuda.empty_cache()
    fp64 = None
    if precision != binding.MBD_PREC_FP64 and args.fp64_steps > 0:
        fw = 0 if N >= 4000 else 1   # the large cluster's FP64 evaluation takes minutes: no warm-up
        f = time_arm(binding, dev, stream, sysm, p3, p4, binding.MBD_PREC_FP64, scs_mode, args.fp64_steps, fw,
                     barrier, max_over_ranks)
        f["ctx"].close()
        torch.cuda.empty_cache()
        fp64 = {"value": world * args.fp64_steps / (f["ms"] / 1e3), "unit": UNIT,
                "ms_per_step": f["ms"] / args.fp64_steps, "steps": args.fp64_steps, "warmup": fw,
                "energy_ha": f["energy"], "ns_iterations": f["stats"]["ns_iterations"],
                "stage_ms": stage_means(f["profs"]),
                "roofline": roofline_of(binding, "fp64", binding.MBD_PREC_FP64, f["profs"], f["ms"],
                                        args.fp64_steps, args.workload),
                "errors_of": {args.precision: errors_vs(main, f, N),
                              **{k: errors_vs(a, f, N) for k, a in arms.items()}}}
    line["fp64_path"] = fp64
    line["other_precisions"] = {k: {"value": world * a["steps"] / (a["ms"] / 1e3), "unit": UNIT,
                                    "ms_per_step": a["ms"] / a["steps"], "steps": a["steps"], "warmup": 1,
                                    "energy_ha": a["energy"], "ns_iterations": a["stats"]["ns_iterations"],
                                    "stage_ms": stage_means(a["profs"]),
                                    "roofline": roofline_of(binding, k, precision_code(binding, k), a["profs"],
                                                            a["ms"], a["steps"], args.workload)}
                                for k, a in arms.items()}
    # further workloads (the 2000-atom cluster, the 256-atom cell), each measured the same way
    # with fewer steps, and the varlen cluster batch with the learned screening beside plain
    for xw in args.extra_workload:
        if xw == args.workload:
            continue
        if xw == "batch4096":
            if not nl:
                line[xw] = batch_section(binding, local, args, args.precision)
            continue
        xs = syn.workload(xw)
        xper = xs.lattice is not None
        xp3, xp4 = syn.nl_ratios(xs.n_atoms, NL_SEED) if nl else (xs.rvdw_ref, xs.ratio)
        sec = {"config": workload_config(xw, args.method, xs.n_atoms, world, xper, xs)}
        xarms = {}
        xk = max(1, min(args.steps, args.extra_steps))
        for name in [args.precision] + [a for a in args.also if a != args.precision]:
            if xper and name == "fp64split":
                continue
            a = time_arm(binding, dev, stream, xs, xp3, xp4, precision_code(binding, name), scs_mode, xk, 1,
                         barrier, max_over_ranks)
            a["ctx"].close()
            xarms[name] = a
            sec[name] = {"value": world * xk / (a["ms"] / 1e3), "unit": UNIT,
                         "ms_per_step": a["ms"] / xk, "steps": xk, "warmup": 1,
                         "energy_ha": a["energy"], "ns_iterations": a["stats"]["ns_iterations"],
                         "stage_ms": stage_means(a["profs"]),
                         "roofline": roofline_of(binding, name, precision_code(binding, name), a["profs"], a["ms"],
                                                 xk, xw)}
        if not xper and not nl and args.learned_arm:   # the learned screening (no fallback) with the same matrix function
            model = np.load(os.path.join(ROOT, "paper_2308_03140_gb300", "learned_scs_model.npz"))
            a = time_arm(binding, dev, stream, xs, xp3, xp4, precision_code(binding, args.precision), scs_mode, xk, 1,
                         barrier, max_over_ranks, learned=model)
            a["ctx"].close()
            name = f"learned_{args.precision}"
            xarms[name] = a
            sec[name] = {"value": world * xk / (a["ms"] / 1e3), "unit": UNIT, "ms_per_step": a["ms"] / xk,
                         "steps": xk, "warmup": 1, "energy_ha": a["energy"], "gradients": "energy and coordinates",
                         "stage_ms": stage_means(a["profs"])}
        if args.extra_fp64_steps > 0:
            f = time_arm(binding, dev, stream, xs, xp3, xp4, binding.MBD_PREC_FP64, scs_mode, args.extra_fp64_steps,
                         1, barrier, max_over_ranks)
            f["ctx"].close()
            sec["fp64_path"] = {"value": world * args.extra_fp64_steps / (f["ms"] / 1e3), "unit": UNIT,
                                "ms_per_step": f["ms"] / args.extra_fp64_steps, "steps": args.extra_fp64_steps,
                                "warmup": 1, "energy_ha": f["energy"], "ns_iterations": f["stats"]["ns_iterations"],
                                "stage_ms": stage_means(f["profs"]),
                                "roofline": roofline_of(binding, "fp64", binding.MBD_PREC_FP64, f["profs"], f["ms"],
                                                        args.extra_fp64_steps, xw),
                                "errors_of": {k: errors_vs(a, f, xs.n_atoms) for k, a in xarms.items()}}
        torch.cuda.empty_cache()
        line[xw] = sec
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if not (nl and periodic):
            line["cpu_baseline"] = cpu_baseline(args.workload, 32 if periodic else args.cpu_sample_atoms, N,
                                                args.method)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batch_section(binding, local, args, precision_name):
    """The first --batch-clusters clusters of the varlen batch (sizes U{50..500}): energy +
    coordinate gradients per cluster through the library API, plain screening against the learned
    model with its fallback at 1e-6 Ha/atom and without fallback, on the same clusters; one pass
    per arm after one warm-up pass.  Device time from the library's profile, host time around
    each pass (inputs uploaded and outputs read back for every cluster)."""
    import numpy as np
    import torch
    from paper_2308_03140_gb300 import synthetic as syn
    K = args.batch_clusters
    systems = syn.cluster_batch(K)
    model = np.load(os.path.join(ROOT, "paper_2308_03140_gb300", "learned_scs_model.npz"))
    precision = precision_code(binding, precision_name)
    scale = float(model["estimate_scale"]) if "estimate_scale" in model.files else 1.0
    arms = {"plain": dict(), "learned": dict(scs_mode=binding.MBD_SCS_LEARNED, learned_max_error=1e-6,
                                             learned_estimate_scale=scale),
            "learned_no_fallback": dict(scs_mode=binding.MBD_SCS_LEARNED, learned_max_error=1e300),
            "plain_fp64": dict(precision=binding.MBD_PREC_FP64)}
    ctxs = {}
    for name, opt in arms.items():
        m = binding.MBD(local, **{"precision": precision, **opt})
        if opt.get("scs_mode") == binding.MBD_SCS_LEARNED:
            m.set_scs_model(model["params16"], model["mean"], model["std"])
        m.set_profiling(True)
        ctxs[name] = m
    launches = {}

    def one_pass(name, record=None):
        m = ctxs[name]
        dev_ms, fb = 0.0, 0
        for s in systems:
            m.set_geometry(s.coords)
            m.set_free_atom_params(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
            E, gR, _, _ = m.evaluate(True, param_gradients=name.startswith("plain"))
            prof = m.profile()
            dev_ms += prof["total_ms"]
            launches[name] = launches.get(name, 0) + prof["launches"]
            if name.startswith("learned"):
                fb += int(m.learned_stats()["fell_back"])
            if record is not None:
                record.append((E, gR))
        return dev_ms, fb

    results, ref, records = {}, [], {}
    one_pass("plain", ref)   # reference energies and forces (also the plain arm's warm-up)
    for name in arms:
        if name != "plain":
            one_pass(name)   # warm-up
        torch.cuda.synchronize()
        launches[name] = 0
        rec = []
        t0 = time.perf_counter()
        dev_ms, fb = one_pass(name, rec)
        wall = time.perf_counter() - t0
        results[name] = {"solves_per_s_device": K / (dev_ms / 1e3), "solves_per_s_e2e": K / wall,
                         "fallback_fraction": fb / K if name.startswith("learned") else None,
                         "gpu_launches": launches[name]}
        records[name] = rec

    def errors(rec, against):
        dE = [abs(e - er) / s.n_atoms for (e, _), (er, _), s in zip(rec, against, systems)]
        dF = [float(np.abs(g - gr).max()) for (_, g), (_, gr) in zip(rec, against)]
        return {"mean_abs_de_per_atom_ha": float(np.mean(dE)), "max_abs_de_per_atom_ha": float(np.max(dE)),
                "fraction_within_1e-6": float(np.mean(np.array(dE) <= 1e-6)), "max_force_err_ha_bohr": float(np.max(dF))}

    for name in arms:   # against plain screening with the same matrix function, and against the FP64 path
        if name != "plain":
            results[name].update(errors(records[name], ref))
        if name != "plain_fp64":
            results[name]["vs_fp64_path"] = errors(records[name], records["plain_fp64"])
    for m in ctxs.values():
        m.close()
    return {"config": {"workload": "batch4096", "clusters": K, "mean_atoms": float(np.mean([s.n_atoms for s in systems])),
                       "sizes": "U{50..500}, the first clusters of the 4096-cluster recipe", "precision": precision_name,
                       "learned_model": "paper_2308_03140_gb300/learned_scs_model.npz (4 members, trained on 20000 "
                                        "perturbed plain-screening solves)", "estimate_scale": scale},
            "arms": results}


def run_batch(args):
    """The varlen cluster batch alone (see batch_section), as one JSON line whose value is the
    learned arm's device solves/s."""
    import numpy as np
    import torch
    from paper_2308_03140_gb300 import binding, build
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    build.build()
    binding.load()
    clocks = ClockSampler(local)
    clocks.start()
    sec = batch_section(binding, local, args, args.precision)
    clk = clocks.stop()
    res = sec["arms"]
    K = args.batch_clusters
    line = {
        "metric": METRIC, "value": res["learned"]["solves_per_s_device"], "unit": UNIT, "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": 1e3 * K / res["learned"]["solves_per_s_device"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": f"{args.precision}+f32+f16",
        "data": "synthetic", "config": sec["config"], "arms": res,
        "e2e": {"value": res["learned"]["solves_per_s_e2e"], "unit": UNIT},
        "clocks": clk, "gpu_launches": res["learned"]["gpu_launches"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_kernel(args):
    """One kernel alone, --warmup + --steps launches, CUDA-event time per launch: the
    symmetric split product Z' = c3 P Z + c1 Z of the Newton-Schulz iteration (k_tc_gemm mode
    2, the library's accumulation lengths: 8 stages for bf16x3, 2 for tf32x3) at order --order
    (default 6016, the 2000-atom cluster's), operands
    as hi/lo parts of the --precision kind (bf16x3 or tf32x3), FP32 output and its parts; or
    (--kernel tc_gemm_update) the screening's trailing update C -= L21 L21^T of a 512-column
    panel on the lower tiles (mode 1, 8-stage accumulation as in the factorisation, in place)."""
    import torch
    from paper_2308_03140_gb300 import binding
    binding.load()
    dev = torch.device("cuda:0")
    n = args.order
    kind = 1 if args.precision == "bf16x3" else 2
    update = args.kernel == "tc_gemm_update"
    K = 512 if update else n
    g = torch.Generator(device="cpu").manual_seed(7)
    S = torch.randn(n, K, generator=g, dtype=torch.float32) / K ** 0.5
    if not update:
        S = (S + S.T)
    S = S.to(dev)
    if kind == 2:
        hi = ((S.view(torch.int32) + 0x1000) & ~0x1FFF).view(torch.float32)
        lo = (S - hi).contiguous()
        pdt = torch.float32
    else:
        hi = S.to(torch.bfloat16)
        lo = (S - hi.float()).to(torch.bfloat16)
        pdt = torch.bfloat16
    C = torch.empty(n, n, dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    chunk = 8 if kind == 1 else 2   # the library's accumulation lengths for the kind
    if update:
        chunk = 8   # the screening's accumulation length
        C.copy_(torch.randn(n, n, generator=g, dtype=torch.float32).to(dev))

        def launch():   # C = C - S S^T on the lower tiles (in place, as the factorisation does)
            rc = binding.mbdk_gemm_tc(kind, hi, hi, C, A1=lo, B1=lo, alpha=-1.0, beta=1.0, D=C, mode=1, err=err,
                                      chunk_stages=chunk)
            if rc:
                raise RuntimeError(f"mbdk_gemm_tc returned {rc}")
    else:
        Ch, Cl = torch.empty(n, n, dtype=pdt, device=dev), torch.empty(n, n, dtype=pdt, device=dev)

        def launch():
            rc = binding.mbdk_gemm_tc(kind, hi, hi, C, A1=lo, B1=lo, alpha=-0.5, beta=1.5, D=S, C_hi=Ch, C_lo=Cl,
                                      mode=2, err=err, chunk_stages=chunk)
            if rc:
                raise RuntimeError(f"mbdk_gemm_tc returned {rc}")

    for _ in range(args.warmup):
        launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        launch()
    e1.record()
    torch.cuda.synchronize()
    if err.item():
        raise RuntimeError("tensor-core wait timed out")
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    if update:   # algorithmic: the lower tiles (tm >= tn) of the n x n x 512 product
        t = n // 128
        flops = 2.0 * 128 * 128 * K * t * (t + 1) / 2
    else:        # algorithmic: upper triangle of a symmetric n x n x n product
        flops = float(n) * n * (n + 1)
    form = os.environ.get("MBDGB_TC_FORM", "wide")
    print(json.dumps({"kernel": f"k_tc_gemm ({form} form) <{args.precision}> mode {1 if update else 2}", "order": n,
                      "K": K, "chunk_stages": chunk, "launches": args.steps, "ms_per_launch": ms,
                      "tflops_algorithmic": flops / (ms / 1e3) / 1e12}))
    return 0


def run_split_gemm(args):
    """The FP64-accurate split GEMM (mbdk_gemm_f64_split) at order 6016 against the FP64
    tensor-pipe GEMM (mbdk_gemm_f64) on the same operands (a symmetric matrix of the scale of
    the Newton-Schulz iterates, times itself): CUDA-event time per call of each, algorithmic
    TFLOP/s (2 n^3), and the largest difference between the two results in units of
    sum_k |A_ik| |B_kj| (both are FP64-accurate, so a few 2^-53)."""
    import torch
    from paper_2308_03140_gb300 import binding
    binding.load()
    dev = torch.device("cuda:0")
    n = 6016
    g = torch.Generator(device="cpu").manual_seed(11)
    S = torch.randn(n, n, generator=g, dtype=torch.float64) / n ** 0.5
    S = (S + S.T).to(dev)
    C1 = torch.empty(n, n, dtype=torch.float64, device=dev)
    C2 = torch.empty_like(C1)
    work = torch.empty(int(binding.load().mbdk_gemm_f64_split_work_bytes(n, n, n)), dtype=torch.uint8, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / max(args.steps, 1)

    ms_split = timed(lambda: binding.mbdk_gemm_f64_split(S, S, C1, trans_b=True, work=work, err=err))
    ms_f64 = timed(lambda: binding.mbdk_gemm_f64(S, S, C2, trans_b=True))
    if err.item():
        raise RuntimeError("tensor-core wait timed out")
    absS = S.abs()
    scale = absS @ absS.T
    diff = float(((C1 - C2).abs() / scale).max()) / 2.0 ** -53
    flops = 2.0 * n ** 3
    print(json.dumps({"kernel": "mbdk_gemm_f64_split (k_row_exponents, k_row_slices, 318 x k_tc_gemm<TF32>)",
                      "order": n, "calls": args.steps, "ms_per_call": ms_split,
                      "tflops_algorithmic": flops / (ms_split / 1e3) / 1e12, "fp64_gemm_ms_per_call": ms_f64,
                      "fp64_gemm_tflops": flops / (ms_f64 / 1e3) / 1e12, "speedup_vs_fp64_gemm": ms_f64 / ms_split,
                      "max_diff_ulps_of_abs_product": diff}))
    return 0


def run_log_energy(args):
    """The log-formula route (Eq. log-formula, FP64 Cholesky factors of I + A_k at the 15
    nodes) of the 2000-atom cluster: --warmup + --steps calls after one TF32x3 evaluation,
    host-clock time per call (the call synchronises), its Cholesky rate against the FP64
    peak, the energy against the Newton-Schulz route, and the oracle's log route timed on a
    100-atom sample of the same recipe (extrapolated by n^3)."""
    from paper_2308_03140_gb300 import binding, build
    from paper_2308_03140_gb300 import synthetic as syn
    build.build()
    binding.load()
    sysm = syn.workload("finite2000")
    m = binding.MBD(0, precision=binding.MBD_PREC_TF32X3)
    m.set_geometry(sysm.coords)
    m.set_free_atom_params(sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)
    E_ns = m.evaluate(False)[0]
    for _ in range(args.warmup):
        m.log_energy(2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        E_log, orders = m.log_energy(2)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    m.close()
    ld = 6016
    chol_flops = 15 * ld ** 3 / 3.0
    peaks = measured_peaks()
    bf16 = (peaks or {}).get("bf16_tflops_sustained") or 1700.0
    fp64_peak = bf16 * FP64_OVER_BF16
    line = {"kernel": "mbd_log_energy (k_build_lr_freq, batched FP64 Cholesky, k_logdiag_batch)",
            "workload": "finite2000", "n_freq": 15, "calls": args.steps, "ms_per_call": 1e3 * dt,
            "cholesky_tflops": chol_flops / dt / 1e12, "fp64_peak_tflops": fp64_peak,
            "frac_of_fp64_peak": chol_flops / dt / 1e12 / fp64_peak,
            "peak_source": ("of measured" if peaks else "of fallback") + ": bf16_tflops_sustained x nominal FP64/BF16 "
                           "(1.25/2250)",
            "energy_log_ha": E_log, "energy_ns_ha": E_ns, "delta_per_atom_ha": (E_log - E_ns) / sysm.n_atoms,
            "pairwise_order_ha": float(orders[0])}
    if not args.no_cpu_baseline:
        import oracle as o
        s100 = sample_system("finite2000", 100)
        _, det = o.mbd_rsscs_energy(*o.system_args(s100), detail=True)
        t1 = time.perf_counter()
        o.mbd_log_energy(s100.coords, det["alpha_bar"][0], det["omega"], det["rvdw"], n_freq=15, max_order=2)
        ts = time.perf_counter() - t1
        line["cpu_baseline"] = {"value": 1.0 / (ts * (2000 / 100) ** 3), "unit": "calls/s",
                                "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
                                "kind": "oracle", "sample": f"log route of a 100-atom cluster in {ts:.2f} s, "
                                                            "extrapolated by (n/100)^3 to 2000 atoms"}
    print(json.dumps(line), flush=True)
    return 0


def run_ts(args):
    """The TS pairwise energy and gradients (mbd_ts_energy, s_R = 0.94): host-clock time per
    call, inputs uploaded and gradients read back each call, and the pair pass's rate against
    the FP64 rate.  ts_finite2000: the 2000-atom cluster (about 60 flop per ordered pair); the
    oracle's TS on an 800-atom sample of the same recipe, extrapolated by n^2.  ts_cell256:
    the 256-atom triclinic cell per cell, with the lattice gradient, by Eq. ts-ewald (gamma
    0.2/bohr, real-space cutoff 30 bohr, reciprocal cutoff 2.0/bohr; about 60 flop per pair
    image and 20 per pair and reciprocal vector); the oracle on the cell's first 32 atoms in
    the same lattice, extrapolated by n^2."""
    import numpy as np

    from paper_2308_03140_gb300 import binding, build
    from paper_2308_03140_gb300 import synthetic as syn
    build.build()
    binding.load()
    cell = args.kernel == "ts_cell256"
    sysm = syn.workload("cell256" if cell else "finite2000")
    N = sysm.n_atoms
    args_p = (sysm.alpha0_ref, sysm.c6_ref, sysm.rvdw_ref, sysm.ratio)
    gamma, rc, kc = 0.2, 30.0, 2.0
    if cell:
        m = binding.MBD(0, ewald_gamma=gamma, real_cutoff=rc, recip_cutoff=kc)
        m.set_geometry(sysm.coords, sysm.lattice, (1, 1, 1))   # the k-grid plays no part in TS
    else:
        m = binding.MBD(0)
        m.set_geometry(sysm.coords)
    m.set_free_atom_params(*args_p)
    for _ in range(args.warmup):
        m.ts_energy(0.94, lattice=cell)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        E = m.ts_energy(0.94, lattice=cell)[0]
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    m.close()
    peaks = measured_peaks()
    bf16 = (peaks or {}).get("bf16_tflops_sustained") or 1700.0
    fp64_peak = bf16 * FP64_OVER_BF16
    if cell:
        A = np.asarray(sysm.lattice)
        vol = abs(np.linalg.det(A))
        B = 2 * np.pi * np.linalg.inv(A).T
        mm = [int(np.ceil(kc * np.linalg.norm(A[c]) / (2 * np.pi))) + 1 for c in range(3)]
        ms = np.array(np.meshgrid(*[np.arange(-q, q + 1) for q in mm], indexing="ij")).reshape(3, -1).T
        n_g = int(np.sum(np.linalg.norm(ms @ B, axis=1) < kc))
        images = 4.0 / 3.0 * np.pi * rc ** 3 / vol
        flops = float(N * N) * (60.0 * images + 20.0 * n_g)
        kernel = "mbd_ts_energy (k_prepare, k_structure_factors, k_ts_gtable, k_ts_periodic, k_ts_chain)"
    else:
        flops = 60.0 * N * (N - 1)
        kernel = "mbd_ts_energy (k_prepare, k_ts_pairs, k_ts_chain)"
    line = {"kernel": kernel, "workload": "cell256" if cell else "finite2000",
            "calls": args.steps, "ms_per_call": 1e3 * dt, "solves_per_s": 1.0 / dt, "energy_ha": E,
            "alu_tflops_per_call": flops / dt / 1e12, "fp64_peak_tflops": fp64_peak,
            "frac_of_fp64_peak": flops / dt / 1e12 / fp64_peak,
            "note": "host-clock time per call including the uploads and the gradient read-back"}
    if cell:
        line["note"] += f"; {n_g} reciprocal vectors and ~{images:.1f} images per pair"
    if not args.no_cpu_baseline:
        from oracle import ts_pairwise as T
        if cell:
            ns = 32
            sub = [a[:ns] for a in (sysm.coords,) + args_p]
            t1 = time.perf_counter()
            T.ts_energy_periodic(sub[0], sysm.lattice, *sub[1:], gamma, rc, kc, s_r=0.94, grad=True)
            what = f"periodic TS of the cell's first {ns} atoms (same lattice)"
        else:
            ns = 800
            smp = sample_system("finite2000", ns)
            t1 = time.perf_counter()
            T.ts_energy(smp.coords, smp.alpha0_ref, smp.c6_ref, smp.rvdw_ref, smp.ratio, 0.94, grad=True)
            what = f"TS of an {ns}-atom cluster"
        ts = time.perf_counter() - t1
        line["cpu_baseline"] = {"value": 1.0 / (ts * (N / ns) ** 2), "unit": "solves/s", "cores": 1,
                                "kind": "oracle", "sample": f"{what} in {ts:.2f} s (numpy), "
                                                            f"extrapolated by (n/{ns})^2 to {N} atoms"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.kernel == "log_energy_finite2000":
        return run_log_energy(args)
    if args.kernel in ("ts_finite2000", "ts_cell256"):
        return run_ts(args)
    if args.kernel == "gemm_f64_split6016":
        return run_split_gemm(args)
    if args.kernel:
        return run_kernel(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch4096":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
