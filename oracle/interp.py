"""Plain FP64 CPU oracle of the source interpolation (Sec. 2.5 keeps an index
array that links mesh nodes to DOFs; Sec. 3.2 groups DOFs around random
centres by distance).

TEST INFRASTRUCTURE ONLY: the definition the CUDA path of zi_nearest_source
is checked against.  Only the test suite imports it; it shares no code with
the CUDA library.

Reading: the interpolation index of a point (a mesh node, or a centre of a
decomposition) is the nearest DOF position by Euclidean distance, ties to
the lowest DOF index; distances are compared as FP64 squared distances
(dx*dx + dy*dy) + dz*dz, each operation rounded once.
"""
from __future__ import annotations

import numpy as np


def nearest_source(points, sources, chunk: int = 2048):
    """Index of the nearest source for every point (brute force)."""
    X = np.atleast_2d(np.asarray(points, dtype=np.float64))
    S = np.atleast_2d(np.asarray(sources, dtype=np.float64))
    out = np.empty(X.shape[0], dtype=np.int64)
    for s in range(0, X.shape[0], chunk):
        d = X[s:s + chunk, None, :] - S[None, :, :]
        d2 = (d[:, :, 0] * d[:, :, 0] + d[:, :, 1] * d[:, :, 1]) + d[:, :, 2] * d[:, :, 2]
        out[s:s + chunk] = np.argmin(d2, axis=1)  # first minimum: the lowest index on ties
    return out
