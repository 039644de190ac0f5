"""Plain FP64 CPU oracle of the segmentation mesher (Sec. 2.5, "mesh tool").

TEST INFRASTRUCTURE ONLY: a definition for a GPU mesher to be checked
against.  Only the test suite imports it; it shares no code with the CUDA
library.

Sec. 2.5 builds a uniform tetrahedral mesh out of a surface segmentation: one
closed triangle surface per compartment, worked through from the inside out;
surfaces are allowed to cross; when a tetrahedron touches several
compartments, a number given to each compartment settles which one it joins
(smaller numbers win).  The reading taken here:

* grid and tets: the Kuhn grid of the sphere mesher (zi_oracle.mesh_from_grid)
  over the cube [-N h, N h]^3, N = ceil(max |coordinate of the outermost
  surface| / h) + 1, six tets per cube in PERMS order, orientation fixed by
  swapping the last two vertices;
* node label: the first compartment (innermost first) whose surface has
  winding number >= 1/2 at the node, or "outside";
* tet label: among its four node labels, the compartment of the highest
  priority (lowest value; ties to the inner compartment), "outside" ranking
  below every compartment; tets labelled "outside" (all four nodes outside)
  are dropped;
* kept nodes: the vertices of kept tets, numbered by ascending grid index;
  kept tets in (cube, permutation) order; boundary faces as in mesh_from_grid.

The winding number of a closed, outward-oriented surface at a point is the
sum of the signed solid angles of its triangles over 4 pi (1 inside, 0
outside); the solid angle of a triangle uses the formula of Van Oosterom and
Strackee, tan(Omega/2) = A.(B x C) / (|A||B||C| + (A.B)|C| + (B.C)|A| + (C.A)|B|)
with A, B, C the vertices relative to the point.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import zi_oracle as O

OUTSIDE = -1


def winding_number(points, verts, tris, chunk: int = 4096):
    """Winding number at points (k,3) of the closed surface (verts, tris)."""
    points = np.atleast_2d(np.asarray(points, dtype=np.float64))
    T = np.asarray(verts, dtype=np.float64)[np.asarray(tris)]          # (t, 3, 3)
    out = np.empty(points.shape[0])
    for s in range(0, points.shape[0], chunk):
        P = points[s:s + chunk]
        A = T[None, :, 0, :] - P[:, None, :]
        B = T[None, :, 1, :] - P[:, None, :]
        C = T[None, :, 2, :] - P[:, None, :]
        a, b, c = (np.linalg.norm(X, axis=2) for X in (A, B, C))
        num = np.einsum("ktd,ktd->kt", A, np.cross(B, C))
        den = (a * b * c + np.einsum("ktd,ktd->kt", A, B) * c + np.einsum("ktd,ktd->kt", B, C) * a
               + np.einsum("ktd,ktd->kt", C, A) * b)
        out[s:s + chunk] = np.sum(2.0 * np.arctan2(num, den), axis=1) / (4.0 * math.pi)
    return out


def node_labels(points, surfaces):
    """First compartment (innermost first) containing each point, or OUTSIDE."""
    lab = np.full(np.atleast_2d(points).shape[0], OUTSIDE, dtype=np.int64)
    for c, (verts, tris) in enumerate(surfaces):
        inside = (winding_number(points, verts, tris) >= 0.5) & (lab == OUTSIDE)
        lab[inside] = c
    return lab


def tet_label(node_lab, priority):
    """Label of a tet from its four node labels (rule in the module header)."""
    best, best_key = OUTSIDE, (math.inf, math.inf)
    for c in node_lab:
        if c == OUTSIDE:
            continue
        key = (priority[c], c)
        if key < best_key:
            best, best_key = int(c), key
    return best


def mesh_from_surfaces(h: float, surfaces, priority):
    """Kuhn-grid mesh of a surface segmentation: dict(nodes, tets, labels,
    bfaces, N, h, node_label (grid), grid_index (kept nodes))."""
    h = float(h)
    R = max(float(np.max(np.abs(v))) for v, _ in surfaces)
    N = int(math.ceil(R / h)) + 1
    G, Gc = 2 * N + 1, 2 * N
    gI, gJ, gK = np.meshgrid(np.arange(G), np.arange(G), np.arange(G), indexing="ij")
    grid_pts = np.stack([(gI.ravel() - N) * h, (gJ.ravel() - N) * h, (gK.ravel() - N) * h], axis=1)
    glab = node_labels(grid_pts, surfaces)

    cubes = np.arange(Gc ** 3)
    cI, cJ, cK = np.unravel_index(cubes, (Gc, Gc, Gc))
    base = np.stack([cI, cJ, cK], axis=1)
    gt = np.empty((cubes.size, 6, 4), dtype=np.int64)       # grid indices of the tet vertices
    for k, (a, b, c) in enumerate(O.PERMS):
        v0 = base.copy()
        v1 = v0.copy(); v1[:, a] += 1
        v2 = v1.copy(); v2[:, b] += 1
        v3 = v0 + 1
        for slot, v in enumerate((v0, v1, v2, v3)):
            gt[:, k, slot] = (v[:, 0] * G + v[:, 1]) * G + v[:, 2]
    gt = gt.reshape(-1, 4)
    # tet_label for every tet at once: rank the compartments by (priority, index), take the best rank
    C = len(surfaces)
    order = sorted(range(C), key=lambda c: (priority[c], c))
    rank = np.empty(C + 1, dtype=np.int64)
    rank[np.array(order)] = np.arange(C)
    rank[C] = C                                                 # OUTSIDE ranks last
    best = np.min(rank[np.where(glab[gt] == OUTSIDE, C, glab[gt])], axis=1)
    labels = np.where(best == C, OUTSIDE, np.append(np.array(order), OUTSIDE)[best])
    keep = labels != OUTSIDE
    gt, labels = gt[keep], labels[keep]

    used = np.unique(gt)
    node_id = np.full(G ** 3, -1, dtype=np.int64)
    node_id[used] = np.arange(used.size)
    nodes = grid_pts[used]
    tets = node_id[gt]
    e1 = nodes[tets[:, 1]] - nodes[tets[:, 0]]
    e2 = nodes[tets[:, 2]] - nodes[tets[:, 0]]
    e3 = nodes[tets[:, 3]] - nodes[tets[:, 0]]
    neg = np.einsum("mi,mi->m", e1, np.cross(e2, e3)) < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    tets = tets.astype(np.int32)
    return dict(nodes=nodes, tets=tets, labels=labels.astype(np.int32), bfaces=O.boundary_faces(tets), N=N, h=h,
                node_label=glab, grid_index=used)
