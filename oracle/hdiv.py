"""Plain FP64 CPU oracle of the H(div) source model (Sec. 2.1, "Primary
current model").

TEST INFRASTRUCTURE ONLY: the definition the CUDA path of zi_source_stencil
is checked against.  Only the test suite and the benchmark's CPU leg import
it; it shares no code with the CUDA library.

The paper's primary current is a combination of divergence-conforming basis
functions: the face functions of the tetrahedron that holds a source (the
4-source Whitney stencil) and, in the 10-source stencil, its six edge
functions as well.  A Cartesian source (three orientations per position) is
interpolated from the stencil by position-based optimisation (PBO).  The
paper names these but does not write them out; what follows is the reading
this project takes.

Stencil sources of tet T = (v_0, v_1, v_2, v_3):

* face source k (k = 0..3): the lowest-order Raviart-Thomas function of the
  face opposite v_k, with unit flux from T into the neighbour N_k across that
  face.  Its divergence is -1/|T| on T and +1/|N_k| on N_k and its normal
  component is continuous, so its load f_i = int J . grad psi_i
  (the right-hand side of the weak form, App. A.1) is 1/4 at the vertex o_k
  of N_k opposite the face and -1/4 at v_k.  Its dipole moment int J is
  c(N_k) - c(T) = (x(o_k) - x(v_k)) / 4, placed at the face centroid.
  A face on the mesh boundary has no neighbour and no face source.
* edge source (a, b) (a < b, the six vertex pairs of T): a pair of opposite
  unit monopoles at the edge's end nodes, load e_{v_b} - e_{v_a}, moment
  x(v_b) - x(v_a), placed at the edge midpoint.

Every stencil source's load satisfies f . psi = d . grad psi for every linear
psi: it is a discrete dipole of moment d.

PBO coefficients of a source at x0 with moment q: w minimises

    J(w) = || sum_k w_k d_k (c_k - x0)^T / s ||_F^2
           + lam * sum_k (1 + |c_k - x0|^2 / s^2) |d_k|^2 w_k^2

subject to sum_k w_k d_k = q, with s the mean edge length of T.  The
constraint reproduces the dipole moment exactly (so every linear potential
sees exactly the point dipole); the first term is the source's first
(quadrupole-order) moment about x0; the second prefers small coefficients on
far sources.  The Cartesian source of orientation e_d has load column
F[:, 3p + d] = sum_k w_k^(d) f_k.  A library dense solve of the KKT system
serves as the step.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

WHITNEY4 = 0
PBO10 = 1
EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def face_neighbours(tets: np.ndarray, which: np.ndarray):
    """For tets `which` and each local face k (opposite vertex k): the tet on
    the other side of that face and its vertex not on the face, or (-1, -1)
    on the mesh boundary.  Plain definition: the other tet holding all three
    face nodes, found through the node-to-tet incidence."""
    m = tets.shape[0]
    n = int(tets.max()) + 1
    inc = sp.csr_matrix((np.ones(4 * m), (tets.ravel(), np.repeat(np.arange(m), 4))), shape=(n, m))
    nbr = np.full((which.size, 4), -1, dtype=np.int64)
    opp = np.full((which.size, 4), -1, dtype=np.int64)
    for r, t in enumerate(which):
        v = tets[t]
        for k in range(4):
            face = [int(v[j]) for j in range(4) if j != k]
            common = set(inc[face[0]].indices)
            for a in face[1:]:
                common &= set(inc[a].indices)
            common.discard(int(t))
            if len(common) > 1:
                raise ValueError("face shared by more than two tets")
            if common:
                u = common.pop()
                nbr[r, k] = u
                (o,) = [int(x) for x in tets[u] if x not in face]
                opp[r, k] = o
    return nbr, opp


def stencil(nodes, tet, opp, model):
    """Sources of one tet: (loads, moments d (K,3), positions c (K,3)), with
    loads a list of ((node, weight), (node, weight)) pairs."""
    X = nodes[tet]
    loads, d, c = [], [], []
    for k in range(4):
        if opp[k] < 0:
            continue
        face = [j for j in range(4) if j != k]
        xo = nodes[opp[k]]
        loads.append(((int(opp[k]), 0.25), (int(tet[k]), -0.25)))
        d.append((xo - X[k]) / 4.0)
        c.append(X[face].mean(axis=0))
    if model == PBO10:
        for a, b in EDGES:
            loads.append(((int(tet[b]), 1.0), (int(tet[a]), -1.0)))
            d.append(X[b] - X[a])
            c.append(0.5 * (X[a] + X[b]))
    elif model != WHITNEY4:
        raise ValueError("model must be WHITNEY4 or PBO10")
    return loads, np.array(d), np.array(c)


def mean_edge(X):
    return np.mean([np.linalg.norm(X[b] - X[a]) for a, b in EDGES])


def pbo_coefficients(x0, d, c, s, lam):
    """w (K x 3): the minimiser of J subject to D w = e_j, one column per
    Cartesian orientation j, from the KKT system
        [2H  D^T] [w ]   [0  ]
        [D   0  ] [mu] = [e_j],   H = M^T M + lam diag((1 + rho_k^2) |d_k|^2),
    M the 9 x K matrix whose column k is vec(d_k (c_k - x0)^T / s)."""
    K = d.shape[0]
    r = (c - x0) / s
    M = np.stack([np.outer(d[k], r[k]).ravel() for k in range(K)], axis=1)
    H = M.T @ M + lam * np.diag((1.0 + np.sum(r * r, axis=1)) * np.sum(d * d, axis=1))
    KKT = np.zeros((K + 3, K + 3))
    KKT[:K, :K] = 2.0 * H
    KKT[:K, K:] = d
    KKT[K:, :K] = d.T
    rhs = np.zeros((K + 3, 3))
    rhs[K:, :] = np.eye(3)
    return np.linalg.solve(KKT, rhs)[:K]


def objective(w, x0, d, c, s, lam):
    """J(w) of one orientation (for checks)."""
    r = (c - x0) / s
    first = sum(w[k] * np.outer(d[k], r[k]) for k in range(d.shape[0]))
    reg = lam * np.sum((1.0 + np.sum(r * r, axis=1)) * np.sum(d * d, axis=1) * w * w)
    return float(np.sum(first * first) + reg)


def source_matrix_hdiv(nodes, tets, dip_tet, pos, model=PBO10, lam=1e-2):
    """F (n x 3P, sparse) of the Cartesian H(div) sources at positions pos in
    tets dip_tet: column 3p + d is sum_k w_k^(d) f_k over tet dip_tet[p]'s
    stencil."""
    n = nodes.shape[0]
    dip_tet = np.asarray(dip_tet, dtype=np.int64)
    _, opp = face_neighbours(tets, dip_tet)
    rows, cols, vals = [], [], []
    for p, t in enumerate(dip_tet):
        loads, d, c = stencil(nodes, tets[t], opp[p], model)
        w = pbo_coefficients(pos[p], d, c, mean_edge(nodes[tets[t]]), lam)
        for k, pair in enumerate(loads):
            for node, a in pair:
                for j in range(3):
                    rows.append(node)
                    cols.append(3 * p + j)
                    vals.append(a * w[k, j])
    return sp.coo_matrix((vals, (rows, cols)), shape=(n, 3 * dip_tet.size)).tocsc()
