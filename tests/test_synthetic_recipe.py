"""The seeded synthetic inputs follow their stated recipe (host, no GPU): atom counts, the
sphere radius of the cluster density 0.08 atoms/A^3, minimum separations (minimum image for
the cell), cell edges and angles, parameter ranges, the varlen batch's size range, and
reproducibility from the seed."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_2308_03140_gb300 import synthetic as syn

RHO = 0.08 * 0.529177210903 ** 3   # atoms per bohr^3


def _min_distance(R):
    d, _ = cKDTree(R).query(R, k=2)
    return d[:, 1].min()


def _params_in_range(s):
    assert np.all((s.alpha0_ref >= 4) & (s.alpha0_ref <= 12))
    assert np.all((s.c6_ref >= 5) & (s.c6_ref <= 50))
    assert np.all((s.rvdw_ref >= 3) & (s.rvdw_ref <= 4))
    assert np.all((s.ratio >= 0.7) & (s.ratio <= 1.0))


@pytest.mark.parametrize("name,n", [("finite2000", 2000), ("finite8000", 8000)])
def test_sphere_clusters(name, n):
    s = syn.workload(name)
    assert s.n_atoms == n and s.lattice is None and s.k_grid is None
    radius = (3 * n / (4 * math.pi * RHO)) ** (1 / 3)
    assert np.linalg.norm(s.coords, axis=1).max() <= radius + 1e-9
    assert _min_distance(s.coords) >= 2.2 - 1e-12
    _params_in_range(s)
    t = syn.workload(name)
    assert np.array_equal(s.coords, t.coords) and np.array_equal(s.ratio, t.ratio)


def test_radius_of_the_large_cluster():
    # 8000 atoms at 0.01186 atoms/bohr^3: a sphere of 54.4 bohr
    assert (3 * 8000 / (4 * math.pi * RHO)) ** (1 / 3) == pytest.approx(54.4, abs=0.05)


def test_small_cube_cluster():
    s = syn.workload("finite32")
    assert s.n_atoms == 32
    assert s.coords.min() >= 0 and s.coords.max() <= 14.0
    assert _min_distance(s.coords) >= 2.5 - 1e-12
    _params_in_range(s)


def test_triclinic_cell():
    s = syn.workload("cell256")
    A = np.asarray(s.lattice)
    assert s.n_atoms == 256 and tuple(s.k_grid) == (4, 4, 4)
    edges = np.linalg.norm(A, axis=1)
    assert np.all((edges >= 20) & (edges <= 26))
    ang = [math.degrees(math.acos(A[i] @ A[j] / (edges[i] * edges[j]))) for i, j in ((1, 2), (0, 2), (0, 1))]
    assert all(80 <= x <= 100 for x in ang)
    assert A[0, 1] == 0 and A[0, 2] == 0 and A[1, 2] == 0       # a along x, b in the xy plane
    # minimum-image separation >= 2.5 bohr: fractional differences wrapped to [-1/2, 1/2)
    f = s.coords @ np.linalg.inv(A)
    df = f[:, None, :] - f[None, :, :]
    df -= np.round(df)
    d = np.linalg.norm(df @ A, axis=-1)
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 2.5 - 1e-9
    _params_in_range(s)


def test_cluster_batch_sizes_and_seeds():
    b = syn.cluster_batch(64)
    sizes = np.array([c.n_atoms for c in b])
    assert sizes.min() >= 50 and sizes.max() <= 500 and len(b) == 64
    c5 = syn.sphere_cluster(int(sizes[5]), seed=4005)
    assert np.array_equal(b[5].coords, c5.coords)
    assert _min_distance(b[5].coords) >= 2.2 - 1e-12
