"""Learned screening model: training data from plain screening, training on the GPU with the
library's own kernels, and packing for mbd_set_scs_model.

The paper has no learned part.  The model (features, network, output encoding) is described
in include/mbd_gb300_kernels.h: per-atom features of the local geometry and of the first
terms of the Dyson series at every grid point, an MLP 122 -> 128 -> 128 -> 16 with FP16
weights and FP32 accumulation, output y = log(alpha_bar(iu) / alpha(iu)) on the 16 grid
points, an ensemble whose spread drives the fallback to plain screening.  Training minimises
the mean squared error of y against the plain-screening targets with Adam; every forward,
backward, loss and update step and the targets run in the library's kernels
(mbdk_scs_features, mbdk_learned_targets, mbdk_mlp_forward/backward, mbdk_mse_grad,
mbdk_adam_step, mbdk_gather_rows); PyTorch provides device memory, and the feature
standardisation statistics are computed once on the host.  The error estimate's scale is
fitted on held-out clusters after training (calibrate).
"""
from __future__ import annotations

import numpy as np

from . import binding
from . import synthetic as syn

P = binding.LEARNED_PARAMS
F = binding.LEARNED_FEATURES
LAYERS = ((F, 128), (128, 128), (128, 16))


def init_params(members: int, seed: int) -> np.ndarray:
    """FP32 parameters [members, P]: weights N(0, 1/fan_in) (the last layer scaled by 0.1, so
    an untrained member predicts y close to 0, i.e. no screening), zero biases."""
    rng = np.random.default_rng(seed)
    out = np.zeros((members, P), dtype=np.float32)
    for m in range(members):
        parts = []
        for li, (fi, fo) in enumerate(LAYERS):
            W = rng.normal(0.0, 1.0 / np.sqrt(fi), (fi, fo)) * (0.1 if li == 2 else 1.0)
            parts += [W.ravel(), np.zeros(fo)]
        out[m] = np.concatenate(parts)
    return out


def perturbed_cluster(index: int, seed0: int = 100_000, n_range=(50, 500)):
    """Training cluster `index`: a sphere cluster of the batch recipe (size U{50..500}, seed
    seed0 + index, disjoint from the evaluation batch's seeds 4000 + i) with positions moved by
    N(0, 0.1 bohr) and parameters scaled by U[0.95, 1.05]."""
    rng = np.random.default_rng(10_000_000 + seed0 + index)
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    s = syn.sphere_cluster(n, seed=seed0 + index, name=f"cluster{index}")
    s.coords = s.coords + rng.normal(0.0, 0.1, s.coords.shape)
    for f in ("alpha0_ref", "c6_ref", "rvdw_ref", "ratio"):
        setattr(s, f, getattr(s, f) * rng.uniform(0.95, 1.05, s.n_atoms))
    return s


def training_data(systems, device: int = 0):
    """Features X [n_atoms, F] (torch float32, CUDA) and targets y [n_atoms, 16] of the
    systems, with plain screening (mixed-precision factorisation with FP64 refinement) as the
    teacher."""
    import torch
    dev = torch.device(f"cuda:{device}")
    feats, targets = [], []
    m = binding.MBD(device, precision=binding.MBD_PREC_TF32X3)
    for s in systems:
        m.set_geometry(s.coords)
        m.set_free_atom_params(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
        d = m.screen()
        ab = torch.tensor(d["alpha_bar"], dtype=torch.float64, device=dev).contiguous()
        af = torch.tensor(d["alpha_free"], dtype=torch.float64, device=dev).contiguous()
        Yk = torch.empty(s.n_atoms, 16, dtype=torch.float32, device=dev)
        binding.mbdk_learned_targets(ab, af, Yk)
        targets.append(Yk)
        feats.append(features([s], dev))
    m.close()
    return torch.cat(feats).contiguous(), torch.cat(targets).contiguous()


def features(systems, dev):
    import torch
    offsets = np.concatenate([[0], np.cumsum([s.n_atoms for s in systems])]).astype(np.int32)
    cat = lambda f: torch.tensor(np.concatenate([np.ravel(getattr(s, f)) for s in systems]), dtype=torch.float64,
                                 device=dev)
    X = torch.zeros(int(offsets[-1]), F, dtype=torch.float32, device=dev)
    binding.mbdk_scs_features(torch.tensor(offsets, device=dev), cat("coords"), cat("alpha0_ref"), cat("c6_ref"),
                              cat("rvdw_ref"), cat("ratio"), X)
    return X


class Ensemble:
    """Ensemble of members trained on the same data from different initial weights and batch
    orders; FP32 master parameters with FP16 copies on the GPU."""

    def __init__(self, members: int = 4, seed: int = 0, device: int = 0):
        import torch
        self.dev = torch.device(f"cuda:{device}")
        self.members = members
        self.p32 = torch.tensor(init_params(members, seed), device=self.dev)
        self.p16 = self.p32.to(torch.float16)
        self.mean = torch.zeros(F, dtype=torch.float32, device=self.dev)
        self.std = torch.ones(F, dtype=torch.float32, device=self.dev)
        self.seed = seed
        self.estimate_scale = 1.0

    def set_standardisation(self, X):
        """Feature mean and standard deviation over the training set; the floor 1e-5 |mean| +
        1e-12 keeps constant features finite without flattening the small Dyson terms of the
        high frequencies (down to ~1e-9), while values below 1e-12 (the Gaussian tail of the
        first-order term for far pairs) stay near zero after standardisation."""
        import torch
        Xh = X.cpu().numpy().astype(np.float64)
        mu = Xh.mean(0)
        self.mean = torch.tensor(mu, dtype=torch.float32, device=self.dev)
        self.std = torch.tensor(np.maximum(Xh.std(0), 1e-5 * np.abs(mu) + 1e-12), dtype=torch.float32, device=self.dev)
        self.estimate_scale = 1.0

    def fit(self, X, Y, steps: int = 2000, batch: int = 4096, lr: float = 2e-3, log_every: int = 0):
        """Adam on the mean squared error of y; every member draws its own batches.
        Returns the loss history (one value per step, mean over members)."""
        import torch
        M, B = self.members, min(batch, X.shape[0])
        m = torch.zeros_like(self.p32)
        v = torch.zeros_like(self.p32)
        grad = torch.zeros_like(self.p32)
        Xb = torch.zeros(B, F, dtype=torch.float32, device=self.dev)
        Yb = torch.zeros(B, 16, dtype=torch.float32, device=self.dev)
        Yp = torch.zeros(M, B, 16, dtype=torch.float32, device=self.dev)
        dY = torch.zeros(M, B, 16, dtype=torch.float32, device=self.dev)
        z = torch.zeros(M, 2, B, 128, dtype=torch.float32, device=self.dev)
        loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        rng = np.random.default_rng(self.seed + 17)
        hist = []
        for step in range(1, steps + 1):
            grad.zero_()
            total = 0.0
            for k in range(M):   # each member: its own batch, forward with cache, backward
                idx = torch.tensor(rng.integers(0, X.shape[0], B).astype(np.int32), device=self.dev)
                binding.mbdk_gather_rows(idx, X, Xb)
                binding.mbdk_gather_rows(idx, Y, Yb)
                pk = self.p16[k:k + 1]
                binding.mbdk_mlp_forward(Xb, self.mean, self.std, pk, Yp[k:k + 1], z[k:k + 1])
                binding.mbdk_mse_grad(Yp[k], Yb, dY[k], loss)
                binding.mbdk_mlp_backward(Xb, self.mean, self.std, pk, z[k:k + 1], dY[k:k + 1], None,
                                          grad[k:k + 1])
                total += loss.item() if (log_every or step == steps) else 0.0
            binding.mbdk_adam_step(self.p32, grad, m, v, step, lr, self.p16)
            hist.append(total / M)
            if log_every and step % log_every == 0:
                print(f"step {step} loss {total / M:.3e}", flush=True)
        return hist

    def predict(self, X):
        import torch
        Y = torch.zeros(self.members, X.shape[0], 16, dtype=torch.float32, device=self.dev)
        binding.mbdk_mlp_forward(X, self.mean, self.std, self.p16, Y)
        return Y

    def model(self):
        """(params16 [members, P] float16, mean [F], std [F]) for MBD.set_scs_model."""
        return self.p16.cpu().numpy(), self.mean.cpu().numpy(), self.std.cpu().numpy()

    def save(self, path: str):
        p16, mean, std = self.model()
        np.savez(path, params16=p16, mean=mean, std=std, estimate_scale=np.float64(self.estimate_scale))


def evaluate_accuracy(ens, systems, device: int = 0, threshold: float = 1e-6, scale: float | None = None,
                      precision: int = binding.MBD_PREC_TF32X3):
    """Learned against plain screening (the same matrix function, `precision`) on the systems:
    per system |dE|/N, the estimate per atom at the estimate scale (the ensemble's when None)
    and whether the learned evaluation would fall back at `threshold`."""
    p16, mean, std = ens.model()
    scale = ens.estimate_scale if scale is None else scale
    rows = []
    with binding.MBD(device, precision=precision) as plain, \
            binding.MBD(device, precision=precision, scs_mode=binding.MBD_SCS_LEARNED, learned_max_error=1e300,
                        learned_estimate_scale=scale) as lm:
        lm.set_scs_model(p16, mean, std)
        for s in systems:
            for m in (plain, lm):
                m.set_geometry(s.coords)
                m.set_free_atom_params(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
            E0 = plain.evaluate(False)[0]
            E1 = lm.evaluate(False)[0]
            est = lm.learned_stats()["estimated_error_per_atom"]
            rows.append((s.n_atoms, abs(E1 - E0) / s.n_atoms, est, est > threshold))
    return rows


def calibrate(ens, systems, quantile: float = 0.95, device: int = 0):
    """Scale of the error estimate: the `quantile` of |dE|/N over the unscaled estimate on
    held-out systems, so that the scaled estimate bounds the true error on that fraction of
    them.  Sets ens.estimate_scale and returns it."""
    rows = evaluate_accuracy(ens, systems, device=device, scale=1.0)
    ratio = np.array([r[1] / r[2] for r in rows if r[2] > 0])
    ens.estimate_scale = float(np.quantile(ratio, quantile)) if ratio.size else 1.0
    return ens.estimate_scale


def main(argv=None):
    """Train the learned screening model on the GPU and save it:
    python -m paper_2308_03140_gb300.learned --solves 20000 --out model.npz"""
    import argparse
    import time
    import torch
    from . import build
    ap = argparse.ArgumentParser()
    ap.add_argument("--solves", type=int, default=20000)
    ap.add_argument("--members", type=int, default=4)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--eval", type=int, default=64, help="held-out clusters of the batch recipe")
    ap.add_argument("--calib", type=int, default=256,
                    help="held-out perturbed clusters (seeds after the training set's) that fit the estimate scale")
    ap.add_argument("--quantile", type=float, default=0.95)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    build.build()
    binding.load()
    t0 = time.time()
    Xs, Ys = [], []
    for c0 in range(0, a.solves, 500):
        X, Y = training_data([perturbed_cluster(i) for i in range(c0, min(a.solves, c0 + 500))])
        Xs.append(X)
        Ys.append(Y)
    X, Y = torch.cat(Xs).contiguous(), torch.cat(Ys).contiguous()
    t1 = time.time()
    ens = Ensemble(members=a.members, seed=0)
    ens.set_standardisation(X)
    hist = ens.fit(X, Y, steps=a.steps, batch=a.batch, lr=a.lr, log_every=500)
    t2 = time.time()
    if a.calib:
        scale = calibrate(ens, [perturbed_cluster(a.solves + 50_000 + i) for i in range(a.calib)], a.quantile)
        print(f"estimate scale {scale:.3f} ({a.quantile:.2f} quantile of |dE| / estimate over {a.calib} clusters, "
              f"{time.time() - t2:.1f} s)", flush=True)
    ens.save(a.out)
    var = float(((Y - Y.mean(0)) ** 2).mean())
    print(f"training set: {a.solves} solves, {X.shape[0]} atoms, {t1 - t0:.1f} s; training {t2 - t1:.1f} s; "
          f"final loss {hist[-1]:.3e} (target variance {var:.3e})", flush=True)
    rows = evaluate_accuracy(ens, syn.cluster_batch(a.eval) if a.eval else [])
    if rows:
        err = np.array([r[1] for r in rows])
        est = np.array([r[2] for r in rows])
        fb = np.mean([r[3] for r in rows])
        ok = np.mean([(r[1] <= 1e-6) for r in rows if not r[3]]) if not all(r[3] for r in rows) else float("nan")
        print(f"held-out {len(rows)} clusters: |dE|/atom mean {err.mean():.3e} max {err.max():.3e}; "
              f"within 1e-6: {np.mean(err <= 1e-6):.2f}; estimate mean {est.mean():.3e}; fallback fraction at "
              f"1e-6: {fb:.2f}; accepted clusters within 1e-6: {ok:.2f}", flush=True)


if __name__ == "__main__":
    main()
