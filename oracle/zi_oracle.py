"""Plain FP64 CPU oracle for the FEM lead-field build (App. A of the paper).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously correct
definition that the CUDA path is checked against.  Only the test suite, the
package smoke check and the CPU-baseline leg of the benchmark may import it;
the product path never does, and it shares no code with the CUDA library
(the only common module is the seeded input generator, which holds none of the
method's arithmetic).

What it computes, step by step, in the paper's notation:

* a0  mesh: regular grid of step h, cubes kept when their centre lies inside
      the outer sphere, six Kuhn tetrahedra per cube, shell labels by the
      centre radius.  The paper's own mesher (Sec. 2.5 "Mesh tool") is
      replaced by this stand-in; the conventions below are the reading used.
* a1  element geometry: grad(lambda_a) = rows 2..4 of inv([1 x_a]),
      vol = |det| / 6, K_e = vol * grad^T Sigma_e grad (App. A.1, a_ij).
* a2  assembly of A on the mesh-graph pattern (explicit zeros kept).
* a3  complete electrode model terms, App. A.1: A += 1/z_l int psi_i psi_j,
      b_il = 1/z_l int psi_i, c_ll = |e_l| / z_l, with z_l = Z_l * area_l
      (the reading that keeps the constant null space of the block system);
      grounding row/column i' (App. A.1).
* a5  transfer matrix T = A^-1 B (App. A.4), here by a sparse direct solve:
      the exact result that PCG approaches.
* a7  source matrix F, F_{i,3p+d} = d psi_i / d x_d at the dipole position
      (partial integration; the paper's G equals -F), columns ordered
      position p, then x, y, z (Sec. 2.5).
* a8  L = R (C - B^T T)^-1 T^T F (App. A.2, Eq. aku rearranged), or for point
      electrodes with electrode 1 as reference, L = T^T F.
* a9  linearised EIT (App. A.3): y = R M^-1 I with M = C - B^T A^-1 B and
      dy_{p,k}/d log s_m = -u_p^T K_m w_k, u_p = T M^-1 I_p, w_k = T M^-1 R e_k.

A library sparse direct solver (SuperLU through scipy) and library COO->CSR
summation serve as steps; nothing here is blocked, fused or reordered beyond
what those definitions state.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# Permutations of the axes (x, y, z) in lexicographic order; tet k of a cube
# follows the path v0 -> v0+e_a -> v0+e_a+e_b -> v0+(1,1,1) for PERMS[k].
PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
# Outward-oriented faces of a positively oriented tet, face f opposite vertex f.
FACES = ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1))


class OracleError(ValueError):
    pass


# ---------------------------------------------------------------------------
# a0: grid mesh (stand-in for the paper's uniform tetrahedral mesher)
# ---------------------------------------------------------------------------

def grid_half_width(h: float, r_out: float) -> int:
    """N: grid indices run over [-N, N] on each axis, N = ceil(R/h) + 1."""
    return int(math.ceil(r_out / h)) + 1


def shell_thresholds(h: float, radii) -> list:
    """Centre test |c| < R  <=>  (2i+1)^2 + (2j+1)^2 + (2k+1)^2 < (2R/h)^2,
    with (2R/h) and its square formed in FP64 in exactly this order."""
    out = []
    for R in radii:
        t = 2.0 * float(R) / float(h)
        out.append(t * t)
    return out


def mesh_from_grid(h: float, radii):
    """Regular-grid Kuhn mesh of the ball r < radii[-1] with shell labels.

    Returns dict(nodes (n,3) f64, tets (m,4) i32, labels (m,) i32,
    bfaces (nb,3) i32, N, cube_of_tet (m,) grid cube linear index).

    Conventions (the paper is silent on all of them):
      - node (I,J,K), I = i+N in [0, 2N], at ((I-N)h, (J-N)h, (K-N)h);
        kept iff it is a corner of a kept cube; numbered by ascending
        (I*G + J)*G + K, G = 2N+1.
      - cube (I,J,K), I in [0, 2N), kept iff its centre is inside radii[-1];
        label = index of the first shell whose radius exceeds the centre radius.
      - kept cubes in ascending (I*2N + J)*2N + K order, six tets each in
        PERMS order; a tet with negative signed volume has its last two
        vertices swapped.
      - boundary faces: faces belonging to exactly one tet, ordered by
        (tet, local face), vertex triples from FACES (outward).
    """
    radii = [float(r) for r in radii]
    N = grid_half_width(h, radii[-1])
    G = 2 * N + 1
    Gc = 2 * N
    odd = 2 * (np.arange(Gc, dtype=np.int64) - N) + 1
    sq = (odd[:, None, None] ** 2 + odd[None, :, None] ** 2 + odd[None, None, :] ** 2)
    thr = shell_thresholds(h, radii)
    keep = sq.astype(np.float64) < thr[-1]
    label_grid = np.zeros(sq.shape, dtype=np.int32)
    for t in thr[:-1]:
        label_grid += (sq.astype(np.float64) >= t).astype(np.int32)

    # nodes: corner of any kept cube
    kn = np.zeros((G, G, G), dtype=bool)
    for dI in (0, 1):
        for dJ in (0, 1):
            for dK in (0, 1):
                kn[dI:dI + Gc, dJ:dJ + Gc, dK:dK + Gc] |= keep
    node_flat = kn.ravel()
    node_id = np.full(G ** 3, -1, dtype=np.int64)
    node_id[node_flat] = np.arange(int(node_flat.sum()))
    gi = np.nonzero(node_flat)[0]
    I, J, K = np.unravel_index(gi, (G, G, G))
    nodes = np.stack([(I - N).astype(np.float64) * h,
                      (J - N).astype(np.float64) * h,
                      (K - N).astype(np.float64) * h], axis=1)

    cubes = np.nonzero(keep.ravel())[0]
    cI, cJ, cK = np.unravel_index(cubes, (Gc, Gc, Gc))
    base = np.stack([cI, cJ, cK], axis=1)
    tets = np.empty((cubes.size, 6, 4), dtype=np.int64)
    for k, (a, b, c) in enumerate(PERMS):
        v0 = base.copy()
        v1 = v0.copy(); v1[:, a] += 1
        v2 = v1.copy(); v2[:, b] += 1
        v3 = v0 + 1
        for slot, v in enumerate((v0, v1, v2, v3)):
            tets[:, k, slot] = node_id[(v[:, 0] * G + v[:, 1]) * G + v[:, 2]]
    tets = tets.reshape(-1, 4)
    labels = np.repeat(label_grid.ravel()[cubes], 6).astype(np.int32)
    cube_of_tet = np.repeat(cubes, 6)

    # orientation: swap the last two vertices where the signed volume is < 0
    e1 = nodes[tets[:, 1]] - nodes[tets[:, 0]]
    e2 = nodes[tets[:, 2]] - nodes[tets[:, 0]]
    e3 = nodes[tets[:, 3]] - nodes[tets[:, 0]]
    det = np.einsum("mi,mi->m", e1, np.cross(e2, e3))
    neg = det < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    tets = tets.astype(np.int32)
    bfaces = boundary_faces(tets)
    return dict(nodes=nodes, tets=tets, labels=labels, bfaces=bfaces, N=N,
                cube_of_tet=cube_of_tet, h=float(h), radii=tuple(radii))


def boundary_faces(tets: np.ndarray) -> np.ndarray:
    """Faces used by exactly one tet, found by sorting all 4m vertex triples;
    returned in (tet, local face) order with FACES' outward vertex order."""
    m = tets.shape[0]
    faces = np.stack([tets[:, list(f)] for f in FACES], axis=1).reshape(-1, 3)
    key = np.sort(faces, axis=1).astype(np.int64)
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    ks = key[order]
    same_next = np.all(ks[1:] == ks[:-1], axis=1)
    dup = np.zeros(4 * m, dtype=bool)
    dup[:-1] |= same_next
    dup[1:] |= same_next
    single = np.zeros(4 * m, dtype=bool)
    single[order] = ~dup
    return faces[single].astype(np.int32)


# ---------------------------------------------------------------------------
# a1: element geometry and stiffness (App. A.1 a_ij, Sec. 2.1.2 tensor rows)
# ---------------------------------------------------------------------------

def element_geometry(nodes: np.ndarray, tets: np.ndarray):
    """grad(lambda) (m,4,3) and volume (m,): lambda_a(x) = ([1 x] inv(M))_a
    with M the 4x4 matrix whose row a is [1, x_a]."""
    m = tets.shape[0]
    M = np.ones((m, 4, 4), dtype=np.float64)
    M[:, :, 1:] = nodes[tets]
    det = np.linalg.det(M)
    if np.any(~(det > 0)):
        raise OracleError("non-positive element volume")
    inv = np.linalg.inv(M)
    grads = np.transpose(inv[:, 1:, :], (0, 2, 1))  # (m, a, d) = inv[d+1, a]
    return grads, det / 6.0


def sigma_tensor(sigma6: np.ndarray) -> np.ndarray:
    """6-tuples (s11, s22, s33, s12, s13, s23) -> symmetric 3x3 tensors."""
    s = np.asarray(sigma6, dtype=np.float64)
    S = np.empty((s.shape[0], 3, 3))
    S[:, 0, 0] = s[:, 0]; S[:, 1, 1] = s[:, 1]; S[:, 2, 2] = s[:, 2]
    S[:, 0, 1] = S[:, 1, 0] = s[:, 3]
    S[:, 0, 2] = S[:, 2, 0] = s[:, 4]
    S[:, 1, 2] = S[:, 2, 1] = s[:, 5]
    return S


def element_stiffness(grads: np.ndarray, vol: np.ndarray, sigma6: np.ndarray) -> np.ndarray:
    """K_e[a,b] = vol * grad(lambda_a)^T Sigma_e grad(lambda_b)."""
    S = sigma_tensor(sigma6)
    if not np.all(np.isfinite(S)):
        raise OracleError("non-finite conductivity")
    return vol[:, None, None] * np.einsum("mai,mij,mbj->mab", grads, S, grads)


def stiffness_triplets(tets: np.ndarray, Ke: np.ndarray):
    """(rows, cols, values) of every element contribution K_e[a, b]."""
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    return rows, cols, Ke.reshape(-1)


def csr_from_triplets(n: int, rows, cols, vals) -> sp.csr_matrix:
    """Sum of the triplets on their union pattern.  COO -> CSR conversion sums
    duplicates and keeps explicit zeros, so the pattern is the mesh graph
    whatever the values (sparse matrix *addition* would drop exact zeros)."""
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def assemble_stiffness(n: int, tets: np.ndarray, Ke: np.ndarray) -> sp.csr_matrix:
    """A_vol = sum_e K_e scattered on the mesh-graph pattern (explicit zeros
    are kept so the pattern does not depend on sigma)."""
    return csr_from_triplets(n, *stiffness_triplets(tets, Ke))


# ---------------------------------------------------------------------------
# electrodes and the complete electrode model (App. A.1)
# ---------------------------------------------------------------------------

def triangle_areas(nodes: np.ndarray, tri: np.ndarray) -> np.ndarray:
    p0, p1, p2 = nodes[tri[:, 0]], nodes[tri[:, 1]], nodes[tri[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=1)


def electrode_patches(nodes, bfaces, centres, radius):
    """Boundary triangles of electrode l: centroid (p0+p1+p2)/3 within
    Euclidean distance `radius` of centre l (d^2 < radius^2, FP64, summed in
    x, y, z order).  Returns (tri index array, electrode of each) in
    electrode-major, triangle-ascending order."""
    p0, p1, p2 = nodes[bfaces[:, 0]], nodes[bfaces[:, 1]], nodes[bfaces[:, 2]]
    cen = (p0 + p1 + p2) / 3.0
    r2 = radius * radius
    tri_l, el_l = [], []
    owner = np.full(bfaces.shape[0], -1, dtype=np.int64)
    for l in range(centres.shape[0]):
        d = cen - centres[l]
        d2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
        sel = np.nonzero(d2 < r2)[0]
        if sel.size == 0:
            raise OracleError("electrode %d covers no boundary triangle" % l)
        if np.any(owner[sel] >= 0):
            raise OracleError("electrode patches overlap")
        owner[sel] = l
        tri_l.append(sel)
        el_l.append(np.full(sel.size, l))
    return np.concatenate(tri_l), np.concatenate(el_l)


def point_electrode_nodes(nodes, bfaces, centres):
    """Nearest boundary node to each centre (squared distance in FP64, summed
    in x, y, z order; ties go to the lowest node index)."""
    bn = np.unique(bfaces)
    out = np.empty(centres.shape[0], dtype=np.int64)
    for l in range(centres.shape[0]):
        d = nodes[bn] - centres[l]
        d2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
        out[l] = bn[int(np.argmin(d2))]
    if np.unique(out).size != out.size:
        raise OracleError("two electrodes on the same node")
    return out


def cem_terms(n, nodes, bfaces, tri, el, z, n_el):
    """A_cem (triplets rows, cols, values), B (n x L dense), C (L,) for the
    complete electrode model with z_l = Z_l * |e_l|:
        A_cem[i,j] = sum_l 1/z_l int_{e_l} psi_i psi_j   (P1 surface mass,
                     area/12 * (2 on the diagonal, 1 off it))
        B[i,l]     = 1/z_l int_{e_l} psi_i              (area/3 per vertex)
        C[l]       = |e_l| / z_l."""
    t = bfaces[tri]
    area = triangle_areas(nodes, t)
    w = 1.0 / z[el]
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            rows.append(t[:, a]); cols.append(t[:, b])
            vals.append(w * area / 12.0 * (2.0 if a == b else 1.0))
    A_cem = (np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    B = np.zeros((n, n_el))
    for a in range(3):
        np.add.at(B, (t[:, a], el), w * area / 3.0)
    C = np.zeros(n_el)
    np.add.at(C, el, area)
    C = C / z
    return A_cem, B, C


def ground_node_cem(bfaces, tri):
    """i': the lowest-index boundary node that no electrode patch touches."""
    bn = np.unique(bfaces)
    covered = np.unique(bfaces[tri])
    free = np.setdiff1d(bn, covered)
    if free.size == 0:
        raise OracleError("no boundary node outside the electrodes")
    return int(free[0])


def pin(A: sp.csr_matrix, ip: int) -> sp.csr_matrix:
    """Grounding (App. A.1): a_{i'i'} = 1 and a_{i'j} = 0; the column is zeroed
    too so A stays symmetric (the solution has t_{i'} = 0 either way)."""
    A = A.tocsr(copy=True)
    r = A.indptr
    rows = np.repeat(np.arange(A.shape[0]), np.diff(r))
    A.data[(rows == ip) | (A.indices == ip)] = 0.0
    A.data[(rows == ip) & (A.indices == ip)] = 1.0
    return A


# ---------------------------------------------------------------------------
# sources: partial-integration dipoles (Sec. 2.1.1 classical model)
# ---------------------------------------------------------------------------

def locate_dipoles(mesh, pos):
    """Tet containing each dipole: cube = floor(x/h) per axis; inside the cube,
    the Kuhn tet PERMS[k] whose axis order sorts the fractional coordinates in
    descending order (first such k on ties).  Raises if the cube is not kept."""
    h, N = mesh["h"], mesh["N"]
    Gc = 2 * N
    s = pos / h
    cell = np.floor(s)
    f = s - cell
    ci = cell.astype(np.int64) + N
    if np.any(ci < 0) or np.any(ci >= Gc):
        raise OracleError("dipole outside the grid")
    lin = (ci[:, 0] * Gc + ci[:, 1]) * Gc + ci[:, 2]
    cube_rank = np.full(Gc ** 3, -1, dtype=np.int64)
    kept = mesh["cube_of_tet"][::6]
    cube_rank[kept] = np.arange(kept.size)
    rank = cube_rank[lin]
    if np.any(rank < 0):
        raise OracleError("dipole outside the mesh")
    perm = np.full(pos.shape[0], -1, dtype=np.int64)
    for k in range(5, -1, -1):
        a, b, c = PERMS[k]
        ok = (f[:, a] >= f[:, b]) & (f[:, b] >= f[:, c])
        perm[ok] = k
    return rank * 6 + perm


def source_matrix(n, nodes, tets, dip_tet):
    """F (n x 3P, sparse): F[i, 3p+d] = d lambda_i / d x_d on the tet holding
    dipole p, for its four vertices i."""
    grads, _ = element_geometry(nodes, tets[dip_tet])
    P = dip_tet.size
    rows = np.repeat(tets[dip_tet], 3, axis=0)          # (3P, 4): rows of column 3p+d
    cols = np.repeat(np.arange(3 * P), 4).reshape(3 * P, 4)
    vals = np.transpose(grads, (0, 2, 1)).reshape(3 * P, 4)  # [p, d, a]
    return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(n, 3 * P)).tocsc()


# ---------------------------------------------------------------------------
# system, transfer matrix, lead field
# ---------------------------------------------------------------------------

class System:
    """Assembled and grounded FEM system of one head.

    Attributes: n, A (pinned CSR), A_unpinned, B (n x Lc dense RHS), C (L,)
    or None, ip, mode ("cem" / "point"), el_nodes (point mode), tri/el (cem),
    Ke (m,4,4), grads, vol."""

    def __init__(self, mesh, sigma6, centres, model, radius=0.0, z=None):
        nodes, tets, bfaces = mesh["nodes"], mesh["tets"], mesh["bfaces"]
        n = nodes.shape[0]
        self.mesh, self.n, self.mode = mesh, n, model
        self.grads, self.vol = element_geometry(nodes, tets)
        self.Ke = element_stiffness(self.grads, self.vol, sigma6)
        r, c, v = stiffness_triplets(tets, self.Ke)
        A = csr_from_triplets(n, r, c, v)
        self.n_el = centres.shape[0]
        if model == "cem":
            z = np.asarray(z, dtype=np.float64)
            self.tri, self.el = electrode_patches(nodes, bfaces, centres, radius)
            (rc, cc, vc), B, C = cem_terms(n, nodes, bfaces, self.tri, self.el, z, self.n_el)
            A = csr_from_triplets(n, np.concatenate([r, rc]), np.concatenate([c, cc]),
                                  np.concatenate([v, vc]))
            self.ip = ground_node_cem(bfaces, self.tri)
            self.B_unpinned = B.copy()
            B[self.ip, :] = 0.0
            self.B, self.C, self.z = B, C, z
        elif model == "point":
            self.el_nodes = point_electrode_nodes(nodes, bfaces, centres)
            self.ip = int(self.el_nodes[0])
            B = np.zeros((n, self.n_el - 1))
            B[self.el_nodes[1:], np.arange(self.n_el - 1)] = 1.0
            self.B, self.C = B, None
        else:
            raise OracleError("unknown electrode model %r" % model)
        self.A_unpinned = A
        self.A = pin(A, self.ip)
        self._lu = None

    def factor(self):
        """Sparse direct factorisation of the grounded A (SuperLU, no
        pivoting: A is SPD), on A permuted by geometric nested dissection."""
        if self._lu is None:
            self._perm = nested_dissection(self.mesh["nodes"])
            p = self._perm
            Ap = self.A[p][:, p].tocsc()
            self._lu = spla.splu(Ap, permc_spec="NATURAL", diag_pivot_thresh=0.0,
                                 options=dict(SymmetricMode=True))
        return self._lu

    def solve(self, rhs):
        rhs = np.asarray(rhs, dtype=np.float64)
        lu = self.factor()
        p = self._perm
        x = np.empty_like(rhs)
        x[p] = lu.solve(np.ascontiguousarray(rhs[p]))
        return x

    def transfer(self):
        """T = A^-1 B, one column per electrode (App. A.4)."""
        return self.solve(self.B)


def nested_dissection(nodes: np.ndarray, leaf: int = 64) -> np.ndarray:
    """Fill-reducing ordering for grid meshes: split along the longest axis at
    the grid plane nearest the median; the plane's nodes separate the halves
    because Kuhn-tet edges span at most one grid step per axis.  Separators
    are numbered after both halves."""
    out = []

    def rec(idx):
        if idx.size <= leaf:
            out.append(idx)
            return
        X = nodes[idx]
        ax = int(np.argmax(X.max(0) - X.min(0)))
        v = X[:, ax]
        planes = np.unique(v)
        p = planes[np.argmin(np.abs(planes - np.median(v)))]
        left, right, sep = idx[v < p], idx[v > p], idx[v == p]
        if left.size == 0 or right.size == 0:
            out.append(idx)
            return
        rec(left)
        rec(right)
        out.append(sep)

    rec(np.arange(nodes.shape[0]))
    return np.concatenate(out)


def average_reference(L: int) -> np.ndarray:
    """R with r_jj = 1 - 1/L and r_ij = -1/L (App. A.1)."""
    return np.eye(L) - np.full((L, L), 1.0 / L)


def leadfield(system: System, F, T=None):
    """EEG lead field (App. A.2): L = R (C - B^T T)^-1 T^T F for the complete
    electrode model; L = T^T F for point electrodes referenced to electrode 1."""
    if T is None:
        T = system.transfer()
    TtF = np.asarray((F.T @ T).T)
    if system.mode == "point":
        return TtF
    S = np.diag(system.C) - system.B.T @ T
    return average_reference(system.n_el) @ np.linalg.solve(S, TtF)


def block_system_solution(system: System, rhs_u, I=None):
    """Solve the full CEM block system [[A, -B], [-B^T, C]] [z; v] = [rhs_u; I]
    directly (grounded by the i' row), returning (z, v).  Cross-check of the
    Schur-complement route."""
    n, Le = system.n, system.n_el
    A = system.A
    Bm = sp.csr_matrix(system.B)
    K = sp.bmat([[A, -Bm], [-Bm.T, sp.diags(system.C)]], format="csc")
    b = np.zeros(n + Le)
    b[:n] = rhs_u
    b[system.ip] = 0.0
    if I is not None:
        b[n:] = I
    x = spla.spsolve(K, b)
    return x[:n], x[n:]


# ---------------------------------------------------------------------------
# linearised EIT (App. A.3)
# ---------------------------------------------------------------------------

def eit_forward(system: System, I_pat, T=None):
    """Voltages y_p = R M^-1 I_p, M = C - B^T T; returns (y (np x L), M, T)."""
    if T is None:
        T = system.transfer()
    M = np.diag(system.C) - system.B.T @ T
    R = average_reference(system.n_el)
    y = (R @ np.linalg.solve(M, np.asarray(I_pat).T)).T
    return y, M, T


def eit_jacobian(system: System, I_pat, T=None):
    """J[p, k, m] = d y_{p,k} / d log s_m = -u_p^T K_m w_k with
    u_p = T M^-1 I_p and w_k = T M^-1 R e_k (App. A.3); K_m is element m's
    stiffness at the current conductivity (dA / d log s_m = K_m)."""
    y, M, T = eit_forward(system, I_pat, T)
    Minv = np.linalg.inv(M)
    R = average_reference(system.n_el)
    U = T @ (Minv @ np.asarray(I_pat).T)       # n x np
    W = T @ (Minv @ R)                          # n x L
    tets = system.mesh["tets"]
    Um = U[tets]                                # m x 4 x np
    Wm = W[tets]                                # m x 4 x L
    J = -np.einsum("map,mab,mbk->pkm", Um, system.Ke, Wm)
    return J, y


def eit_vjp(system: System, I_pat, grad_y, T=None):
    """sum_{p,k} grad_y[p,k] J[p,k,m] for every element m."""
    J, y = eit_jacobian(system, I_pat, T)
    return np.einsum("pk,pkm->m", grad_y, J)


# ---------------------------------------------------------------------------
# one-call helpers
# ---------------------------------------------------------------------------

def build_head(spec, workloads):
    """Mesh, conductivity, electrodes and dipoles of a HeadSpec; returns
    (mesh, sigma6, centres, z, pos, q)."""
    mesh = mesh_from_grid(spec.h, spec.radii)
    s6 = workloads.conductivity(spec, mesh["nodes"], mesh["tets"], mesh["labels"])
    centres, z = workloads.electrode_inputs(spec)
    pos, q = workloads.dipole_inputs(spec)
    return mesh, s6, centres, z, pos, q


def leadfield_from_spec(spec, workloads):
    """The whole LF build for a HeadSpec: returns (L, system, mesh, F, T)."""
    mesh, s6, centres, z, pos, q = build_head(spec, workloads)
    system = System(mesh, s6, centres, spec.electrode_model,
                    radius=spec.electrode_radius, z=z)
    dip_tet = locate_dipoles(mesh, pos)
    F = source_matrix(system.n, mesh["nodes"], mesh["tets"], dip_tet)
    T = system.transfer()
    L = leadfield(system, F, T)
    return L, system, mesh, F, T
