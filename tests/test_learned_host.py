"""Host parts of the learned-screening trainer (no GPU): the initial parameters' layout (the
order mbd_set_scs_model reads: W1, b1, W2, b2, W3, b3 per member), and the training clusters'
recipe (sizes, the base cluster of seed 100000 + i, the stated perturbations)."""
import numpy as np

from paper_2308_03140_gb300 import binding, learned
from paper_2308_03140_gb300 import synthetic as syn


def test_initial_parameters_layout():
    p = learned.init_params(3, seed=5)
    assert p.shape == (3, binding.LEARNED_PARAMS) and p.dtype == np.float32
    F, H, O = binding.LEARNED_FEATURES, 128, binding.LEARNED_OUTPUTS
    sizes = [F * H, H, H * H, H, H * O, O]
    assert sum(sizes) == binding.LEARNED_PARAMS
    parts = np.split(p[0], np.cumsum(sizes)[:-1])
    W1, b1, W2, b2, W3, b3 = parts
    assert not b1.any() and not b2.any() and not b3.any()
    # N(0, 1/fan_in) weights, the last layer scaled by 0.1
    assert abs(W1.std() * np.sqrt(F) - 1) < 0.05 and abs(W2.std() * np.sqrt(H) - 1) < 0.05
    assert abs(W3.std() * np.sqrt(H) / 0.1 - 1) < 0.1
    assert not np.array_equal(p[0], p[1])                      # members start apart
    assert np.array_equal(p, learned.init_params(3, seed=5))  # reproducible


def test_training_clusters_recipe():
    for i in (0, 7, 123):
        s = learned.perturbed_cluster(i)
        assert 50 <= s.n_atoms <= 500
        base = syn.sphere_cluster(s.n_atoms, seed=100_000 + i)
        d = s.coords - base.coords
        assert abs(d.std() - 0.1) < 0.02 and abs(d.mean()) < 0.02      # positions + N(0, 0.1 bohr)
        for f in ("alpha0_ref", "c6_ref", "rvdw_ref", "ratio"):
            r = getattr(s, f) / getattr(base, f)
            assert r.min() >= 0.95 and r.max() <= 1.05            # parameters x U[0.95, 1.05]
        t = learned.perturbed_cluster(i)
        assert np.array_equal(s.coords, t.coords)
