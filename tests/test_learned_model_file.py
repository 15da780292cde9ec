"""The committed learned-screening model (paper_2308_03140_gb300/learned_scs_model.npz, the
file bench.py's learned arms load) has the layout mbd_set_scs_model takes: FP16 parameters
of whole ensemble members, feature statistics of the model's feature count with a positive
spread, and a positive, finite estimate scale."""
import os

import numpy as np

from paper_2308_03140_gb300 import binding

PATH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2308_03140_gb300",
                    "learned_scs_model.npz")


def test_model_file_layout():
    d = np.load(PATH)
    assert set(d.files) == {"params16", "mean", "std", "estimate_scale"}
    p = d["params16"]
    assert p.dtype == np.float16 and p.ndim == 2 and p.shape[1] == binding.LEARNED_PARAMS and p.shape[0] >= 2
    assert np.all(np.isfinite(p.astype(np.float64)))
    for k in ("mean", "std"):
        assert d[k].dtype == np.float32 and d[k].shape == (binding.LEARNED_FEATURES,)
        assert np.all(np.isfinite(d[k]))
    assert np.all(d["std"] > 0)
    sc = float(d["estimate_scale"])
    assert np.isfinite(sc) and 0 < sc < 100
    # the members differ (an ensemble of one repeated member has no spread to estimate from)
    assert all(np.any(p[0] != p[m]) for m in range(1, p.shape[0]))
