"""Plain FP64 CPU oracle of point location on a tetrahedral mesh (Sec. 2.5:
source positions are placed in the mesh elements that hold them).

TEST INFRASTRUCTURE ONLY: a definition for the GPU locator to be checked
against.  Only the test suite imports it; it shares no code with the CUDA
library.

The element holding a point x is the one whose smallest barycentric
coordinate at x is largest, ties to the lowest element index; x lies in the
mesh when that coordinate is >= -1e-10.  The barycentric coordinates of x in
element e are the solution l of the 4 x 4 system [1 1 1 1; x0 x1 x2 x3] l =
[1; x] (one column per vertex), solved here by LU for every element (brute
force, small meshes only).
"""
from __future__ import annotations

import numpy as np

TOL = 1e-10


def barycentric(nodes, tets, x):
    """(m, 4) barycentric coordinates of point x in every element."""
    V = np.asarray(nodes, dtype=np.float64)[np.asarray(tets)]          # (m, 4, 3)
    M = np.ones((V.shape[0], 4, 4))
    M[:, 1:, :] = np.transpose(V, (0, 2, 1))
    rhs = np.broadcast_to(np.concatenate([[1.0], np.asarray(x, dtype=np.float64)]), (V.shape[0], 4))
    return np.linalg.solve(M, rhs[..., None])[..., 0]


def locate_points(nodes, tets, pos):
    """Element index holding each point (-1 outside the mesh)."""
    out = np.empty(len(pos), dtype=np.int64)
    for p, x in enumerate(np.atleast_2d(pos)):
        score = barycentric(nodes, tets, x).min(axis=1)
        e = int(np.argmax(score))                      # first maximum: the lowest index on ties
        out[p] = e if score[e] >= -TOL else -1
    return out
