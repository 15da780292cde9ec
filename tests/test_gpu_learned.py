"""GPU parity of the learned-screening kernels (csrc/k_learned.cu, through the C ABI) against
the FP64 oracle (oracle/learned_scs.py).

Tolerances follow the arithmetic: the static features are computed in FP64 and stored in
FP32 (relative 1e-6); the Dyson block (features 74..121) takes its pair terms in FP32 with FP64
sums over the partners (3e-5 of each column's largest magnitude); the MLP forward runs on the
tensor cores (TF32 hi/lo parts of the activations against the FP16 weights, which are exact in
TF32, FP32 accumulation) and the backward in FP32 SIMT, both against weights that the oracle
uses exactly (relative 2e-5 against the largest magnitude of each output); Adam in FP32
(1e-6)."""
import numpy as np
import pytest

from oracle import learned_scs as LS
import oracle as o
from paper_2308_03140_gb300 import binding, build
from paper_2308_03140_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def T(x, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dt, device=DEV)


def batch_of_systems(sizes=(7, 30, 1, 55), seed=0):
    systems = [syn.sphere_cluster(n, seed=seed + k) for k, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum([s.n_atoms for s in systems])]).astype(np.int32)
    cat = lambda f: np.concatenate([getattr(s, f) for s in systems])
    return systems, offsets, cat("coords").reshape(-1, 3), cat("alpha0_ref"), cat("c6_ref"), cat("rvdw_ref"), cat("ratio")


def random_params(members, seed=1):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(members):
        out.append([(rng.normal(0, 1 / np.sqrt(i), (i, n)), rng.normal(0, 0.2, n)) for i, n in LS.LAYERS])
    return out


def pack16(member_params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in member_params]).astype(np.float16)


def test_features_match_oracle_varlen_batch():
    systems, offsets, R, a0r, c6r, rr, v = batch_of_systems()
    X = torch.zeros(R.shape[0], binding.LEARNED_FEATURES, dtype=torch.float32, device=DEV)
    binding.mbdk_scs_features(T(offsets, torch.int32), T(R), T(a0r), T(c6r), T(rr), T(v), X)
    Xg = X.cpu().numpy()
    Xo = []
    for s in systems:
        a0, om, rv = o.ts_scaling(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
        Xo.append(LS.features(s.coords, a0, om, rv, s.ratio))
    Xo = np.concatenate(Xo)
    st = LS.N_FEAT_STATIC
    assert np.allclose(Xg[:, :st], Xo[:, :st], rtol=1e-6, atol=1e-6 * max(1.0, np.abs(Xo[:, :st]).max()))
    # the Dyson block against the scale of each feature over the batch, with an absolute floor of
    # 1e-12 (the standardisation's floor on the std): at the highest frequencies the first-order
    # term of far pairs is the Gaussian tail of T^GG's trace, which the oracle's FP64 trace of the
    # full tensor leaves at its cancellation level (~1e-20) and the kernel takes as 0
    col = np.abs(Xo[:, st:]).max(0)
    bad = np.abs(Xg[:, st:] - Xo[:, st:]) - (3e-5 * col + 1e-12)
    assert np.all(bad <= 0), (np.argmax(bad.max(0)), bad.max())


@pytest.mark.parametrize("B", [1, 31, 32, 77, 128, 300])
def test_mlp_forward_backward_match_oracle(B):
    rng = np.random.default_rng(B)
    F = binding.LEARNED_FEATURES
    X = rng.normal(2.0, 3.0, (B, F))
    mean, std = rng.normal(2.0, 0.1, F), rng.uniform(2.0, 4.0, F)
    members = random_params(2, seed=B)
    p16 = np.stack([pack16(m) for m in members])
    P = [LS.round_fp16(m) for m in members]
    Xs = (X.astype(np.float32).astype(np.float64) - mean.astype(np.float32)) / std.astype(np.float32)
    Xg, mg, sg = T(X, torch.float32), T(mean, torch.float32), T(std, torch.float32)
    pg = torch.tensor(p16.view(np.int16), device=DEV).view(torch.float16)
    Y = torch.zeros(2, B, 16, dtype=torch.float32, device=DEV)
    z = torch.zeros(2, 2, B, 128, dtype=torch.float32, device=DEV)
    binding.mbdk_mlp_forward(Xg, mg, sg, pg, Y, z)
    dY = rng.normal(size=(2, B, 16))
    dX = torch.zeros(2, B, F, dtype=torch.float32, device=DEV)
    grad = torch.zeros(2, binding.LEARNED_PARAMS, dtype=torch.float32, device=DEV)
    binding.mbdk_mlp_backward(Xg, mg, sg, pg, z, T(dY, torch.float32), dX, grad)
    dX_tc = torch.zeros(2, B, F, dtype=torch.float32, device=DEV)   # the data path alone: tensor cores
    binding.mbdk_mlp_backward(Xg, mg, sg, pg, z, T(dY, torch.float32), dX_tc, None)
    for mi in range(2):
        y, cache = LS.forward(Xs, P[mi])
        Yg = Y[mi].cpu().numpy()
        assert np.abs(Yg - y).max() <= 2e-5 * max(1.0, np.abs(y).max())
        grads, dXs = LS.backward(dY[mi].astype(np.float32).astype(np.float64), P[mi], cache)
        g_ref = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
        gg = grad[mi].cpu().numpy()
        assert np.abs(gg - g_ref).max() <= 2e-5 * max(1.0, np.abs(g_ref).max())
        dX_ref = dXs / std.astype(np.float32)
        assert np.abs(dX[mi].cpu().numpy() - dX_ref).max() <= 2e-5 * max(1.0, np.abs(dX_ref).max())
        assert np.abs(dX_tc[mi].cpu().numpy() - dX_ref).max() <= 2e-5 * max(1.0, np.abs(dX_ref).max())


def test_mse_adam_and_gather_match_oracle():
    rng = np.random.default_rng(7)
    y, t = rng.normal(size=(50, 16)), rng.normal(size=(50, 16))
    dy = torch.zeros(50, 16, dtype=torch.float32, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    binding.mbdk_mse_grad(T(y, torch.float32), T(t, torch.float32), dy, loss)
    l_ref, g_ref = LS.mse_loss_grad(y.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64))
    assert loss.item() == pytest.approx(l_ref, rel=1e-6)
    assert np.allclose(dy.cpu().numpy(), g_ref, rtol=1e-5, atol=1e-9)
    n = 1000
    p, g = rng.normal(size=n), rng.normal(size=n)
    m, v = rng.normal(0, 0.1, n), rng.uniform(0, 0.1, n)
    pg, mg, vg = T(p, torch.float32), T(m, torch.float32), T(v, torch.float32)
    p16 = torch.zeros(n, dtype=torch.float16, device=DEV)
    binding.mbdk_adam_step(pg, T(g, torch.float32), mg, vg, 3, 1e-2, p16)
    f = lambda a: a.astype(np.float32).astype(np.float64)
    pr, mr, vr = f(p), f(m), f(v)
    LS.adam_step(pr, f(g), mr, vr, 3, 1e-2)
    assert np.allclose(pg.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
    assert np.allclose(mg.cpu().numpy(), mr, rtol=1e-5, atol=1e-7)
    assert np.array_equal(p16.cpu().numpy(), pg.cpu().numpy().astype(np.float16))
    src = T(rng.normal(size=(40, 5)), torch.float32)
    idx = T(rng.integers(0, 40, 17), torch.int32)
    dst = torch.zeros(17, 5, dtype=torch.float32, device=DEV)
    binding.mbdk_gather_rows(idx, src, dst)
    assert torch.equal(dst, src[idx.long()])


# ---- learned mode of the MBD evaluation ------------------------------------------------
def oracle_energy_from_alpha_bar(s, ab):
    """Oracle MBD energy from given screened alpha_bar(u) rows (Eqs. casimir-polder,
    scale-rvdw-scs, q-matrix, mbd-energy)."""
    a0, om, rv = o.ts_scaling(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
    rc, (abar0, c6, ombar, rbar) = o.screened_params(ab, a0, rv)
    return o.mbd_energy(s.coords, abar0, ombar, rbar)


def learned_eval(s, params16, mean, std, **opt):
    with binding.MBD(0, scs_mode=binding.MBD_SCS_LEARNED, **opt) as m:
        m.set_geometry(s.coords)
        m.set_free_atom_params(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
        m.set_scs_model(params16, mean, std)
        E = m.evaluate(False)[0]
        return E, m.scs_detail(), m.learned_stats()


def test_zero_model_gives_the_unscreened_energy():
    s = syn.sphere_cluster(40, seed=3)
    p16 = np.zeros((2, binding.LEARNED_PARAMS), np.float16)
    F = binding.LEARNED_FEATURES
    E, det, st = learned_eval(s, p16, np.zeros(F), np.ones(F), learned_max_error=1.0)
    a0, om, rv = o.ts_scaling(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
    u, _ = o.freq_grid(15)
    ab = np.stack([o.dyn_alpha(a0, om, uk) for uk in u])
    assert np.allclose(det["alpha_bar"], ab, rtol=1e-14)
    assert E == pytest.approx(oracle_energy_from_alpha_bar(s, ab), rel=1e-10)
    assert st["estimated_error_per_atom"] == 0.0 and not st["fell_back"]


def test_random_model_matches_oracle_prediction():
    s = syn.sphere_cluster(60, seed=4)
    members = random_params(3, seed=9)
    members = [[(W * 0.05, b * 0.05) for W, b in mp] for mp in members]
    p16 = np.stack([pack16(mp) for mp in members])
    a0, om, rv = o.ts_scaling(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
    X = LS.features(s.coords, a0, om, rv, s.ratio)
    mean, std = X.mean(0), np.maximum(X.std(0), 1e-3)
    Xs = (X - mean) / std
    u, _ = o.freq_grid(15)
    alpha_u = np.stack([o.dyn_alpha(a0, om, uk) for uk in u])
    ab_ref, spread = LS.predict_alpha_bar(Xs, [LS.round_fp16(mp) for mp in members], alpha_u)
    E, det, st = learned_eval(s, p16, mean, std, learned_max_error=1.0)
    assert np.allclose(det["alpha_bar"], ab_ref, rtol=2e-5)
    assert E == pytest.approx(oracle_energy_from_alpha_bar(s, ab_ref), rel=1e-4)
    assert st["estimated_error_per_atom"] > 0.0 and not st["fell_back"]
    _, _, st2 = learned_eval(s, p16, mean, std, learned_max_error=1.0, learned_estimate_scale=0.25)
    assert st2["estimated_error_per_atom"] == pytest.approx(0.25 * st["estimated_error_per_atom"], rel=1e-12)


def test_fallback_reproduces_plain_screening():
    s = syn.sphere_cluster(50, seed=5)
    members = [[(W * 0.05, b * 0.05) for W, b in mp] for mp in random_params(2, seed=11)]
    p16 = np.stack([pack16(mp) for mp in members])
    F = binding.LEARNED_FEATURES
    E, det, st = learned_eval(s, p16, np.zeros(F), np.ones(F) * 10.0, learned_max_error=1e-14)
    assert st["fell_back"]
    E_ref = o.mbd_rsscs_energy(*o.system_args(s))
    assert E == pytest.approx(E_ref, rel=1e-10)


def test_learned_mode_rejects_gradients_and_periodic_systems():
    s = syn.sphere_cluster(20, seed=6)
    with binding.MBD(0, scs_mode=binding.MBD_SCS_LEARNED) as m:
        m.set_geometry(s.coords)
        m.set_free_atom_params(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
        with pytest.raises(binding.MBDError) as e:
            m.evaluate(False)
        assert e.value.code == 7                      # no model set
        F = binding.LEARNED_FEATURES
        m.set_scs_model(np.zeros((1, binding.LEARNED_PARAMS), np.float16), np.zeros(F), np.ones(F))
        with pytest.raises(binding.MBDError) as e:
            m.evaluate(True)                          # parameter gradients: not in learned mode
        assert e.value.code == 8


def oracle_learned_energy(R, s, members, mean, std):
    """FP64 oracle of the learned path: features -> members (FP16 weights) -> alpha_bar -> MBD."""
    a0, om, rv = o.ts_scaling(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
    X = LS.features(R, a0, om, rv, s.ratio)
    Xs = (X - mean.astype(np.float32).astype(np.float64)) / std.astype(np.float32).astype(np.float64)
    u, _ = o.freq_grid(15)
    alpha_u = np.stack([o.dyn_alpha(a0, om, uk) for uk in u])
    ab, _ = LS.predict_alpha_bar(Xs, [LS.round_fp16(mp) for mp in members], alpha_u)
    rc, (abar0, c6, ombar, rbar) = o.screened_params(ab, a0, rv)
    return o.mbd_energy(R, abar0, ombar, rbar)


def test_learned_forces_match_oracle_finite_differences():
    s = syn.sphere_cluster(14, seed=8)
    members = [[(W * 0.05, b * 0.05) for W, b in mp] for mp in random_params(2, seed=21)]
    p16 = np.stack([pack16(mp) for mp in members])
    a0, om, rv = o.ts_scaling(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
    X = LS.features(s.coords, a0, om, rv, s.ratio)
    mean, std = X.mean(0), np.maximum(X.std(0), 1e-3)
    with binding.MBD(0, scs_mode=binding.MBD_SCS_LEARNED, learned_max_error=1.0) as m:
        m.set_geometry(s.coords)
        m.set_free_atom_params(s.alpha0_ref, s.c6_ref, s.rvdw_ref, s.ratio)
        m.set_scs_model(p16, mean, std)
        E, gR, gp, _ = m.evaluate(True, param_gradients=False)
        assert gp is None and not m.learned_stats()["fell_back"]
    assert E == pytest.approx(oracle_learned_energy(s.coords, s, members, mean, std), rel=1e-5)
    h = 1e-4
    fd = np.zeros_like(gR)
    for i in range(s.n_atoms):
        for c in range(3):
            Rp, Rm = s.coords.copy(), s.coords.copy()
            Rp[i, c] += h; Rm[i, c] -= h
            fd[i, c] = (oracle_learned_energy(Rp, s, members, mean, std) -
                        oracle_learned_energy(Rm, s, members, mean, std)) / (2 * h)
    assert np.abs(gR - fd).max() <= 1e-4 * np.abs(fd).max() + 1e-9, (np.abs(gR - fd).max(), np.abs(fd).max())
    assert np.abs(gR.sum(0)).max() < 1e-6 * np.abs(gR).max()


def test_training_on_the_gpu_gains_over_the_unscreened_model():
    """A short training run (our kernels end to end) recovers most of the screening
    correction on held-out clusters: |E_learned - E_rsSCS| is a small fraction of
    |E_unscreened - E_rsSCS|, and the learned screening stage is faster than the Dyson solves."""
    from paper_2308_03140_gb300 import learned
    train = [learned.perturbed_cluster(i, n_range=(50, 160)) for i in range(120)]
    test = [learned.perturbed_cluster(10_000 + i, n_range=(50, 160)) for i in range(6)]
    X, Y = learned.training_data(train)
    ens = learned.Ensemble(members=4, seed=0)
    ens.set_standardisation(X)
    hist = ens.fit(X, Y, steps=1500, batch=2048, lr=2e-3)
    assert hist[-1] < 0.5 * float(((Y - Y.mean(0)) ** 2).mean())   # well over half the variance explained
    p16, mean, std = ens.model()
    zero = np.zeros_like(p16[:1])
    errs_l, errs_0 = [], []
    for s in test:
        E_ref = binding.evaluate_system(s, gradients=False)[0]
        E_l, _, st = learned_eval(s, p16, mean, std, learned_max_error=1.0)
        E_0, _, _ = learned_eval(s, zero, mean, std, learned_max_error=1.0)
        errs_l.append(abs(E_l - E_ref) / s.n_atoms)
        errs_0.append(abs(E_0 - E_ref) / s.n_atoms)
    assert np.mean(errs_l) < 0.2 * np.mean(errs_0), (errs_l, errs_0)
