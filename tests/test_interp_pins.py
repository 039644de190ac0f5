"""Pins of the source-interpolation oracle (nearest DOF, Sec. 2.5 and the
nearest-point decomposition of Sec. 3.2) against a library k-d tree, the
tie rule, and a brute-force Voronoi check."""
import numpy as np
from scipy.spatial import cKDTree

from oracle import interp as I


def test_nearest_source_matches_a_kd_tree():
    rng = np.random.default_rng(4)
    S = rng.uniform(-1, 1, (500, 3))
    X = rng.uniform(-1.2, 1.2, (3000, 3))
    idx = I.nearest_source(X, S)
    d, j = cKDTree(S).query(X)
    assert np.allclose(np.linalg.norm(X - S[idx], axis=1), d, rtol=0, atol=1e-15)
    assert np.array_equal(idx, j)        # random points: no ties


def test_ties_go_to_the_lowest_index_and_cells_are_voronoi():
    S = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 0, 0], [0.5, 0, 0]])
    X = np.array([[0.25, 0, 0], [0.75, 0, 0], [-1, 0, 0], [0.1, 0.3, 0]])
    # (0.25, 0, 0): sources 0, 2 and 3 are 0.25 away -> 0; (0.75, 0, 0): 1 and 3 -> 1
    assert list(I.nearest_source(X, S)) == [0, 1, 0, 0]
    rng = np.random.default_rng(7)
    S = rng.uniform(-1, 1, (40, 3))
    X = rng.uniform(-1, 1, (200, 3))
    idx = I.nearest_source(X, S)
    for x, k in zip(X, idx):
        assert np.all(np.linalg.norm(S - x, axis=1) >= np.linalg.norm(S[k] - x) - 1e-15)
