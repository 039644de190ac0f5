"""Pins for the CPU oracle: each check comes from the paper's definitions or
from mathematics the oracle does not itself use (closed forms, invariants,
brute force, an analytic solution), so that a dropped term, a wrong sign or a
transposed operand in the oracle fails one of them."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import analytic, zi_oracle as O
from paper_1811_07717_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# element stiffness (App. A.1, a_ij = int sigma grad psi_i . grad psi_j)
# --------------------------------------------------------------------------

def test_reference_tet_stiffness_closed_form():
    nodes = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    g, vol = O.element_geometry(nodes, tets)
    K = O.element_stiffness(g, vol, np.array([[1.0, 1.0, 1.0, 0, 0, 0]]))[0]
    expect = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    assert abs(vol[0] - 1.0 / 6.0) < 1e-16
    assert np.max(np.abs(K - expect)) < 1e-15


def test_anisotropic_tet_stiffness_closed_form():
    # scaled reference tet, diagonal tensor: K = vol * diag-weighted gradient products
    s = 0.5
    nodes = np.array([[0, 0, 0], [s, 0, 0], [0, s, 0], [0, 0, s]], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    g, vol = O.element_geometry(nodes, tets)
    sig = np.array([[2.0, 3.0, 5.0, 0.0, 0.0, 0.0]])
    K = O.element_stiffness(g, vol, sig)[0]
    # grads: lambda_1 = x/s, lambda_2 = y/s, lambda_3 = z/s, lambda_0 = 1 - sum
    d = np.array([2.0, 3.0, 5.0])
    v = s ** 3 / 6.0
    expect = np.zeros((4, 4))
    for a in range(3):
        expect[a + 1, a + 1] = v * d[a] / s ** 2
        expect[0, a + 1] = expect[a + 1, 0] = -v * d[a] / s ** 2
    expect[0, 0] = v * d.sum() / s ** 2
    assert np.max(np.abs(K - expect)) < 1e-14 * np.max(np.abs(expect))
    # an off-diagonal tensor entry couples x and y gradients: K[1,2] = vol*s12/s^2
    sig2 = np.array([[2.0, 3.0, 5.0, 0.7, 0.0, 0.0]])
    K2 = O.element_stiffness(g, vol, sig2)[0]
    assert abs(K2[1, 2] - v * 0.7 / s ** 2) < 1e-15


def test_kuhn_interior_row_is_seven_point_stencil():
    h, sig = 0.2, 0.33
    mesh = O.mesh_from_grid(h, [1.0])
    g, vol = O.element_geometry(mesh["nodes"], mesh["tets"])
    m = mesh["tets"].shape[0]
    Ke = O.element_stiffness(g, vol, np.tile([sig, sig, sig, 0, 0, 0], (m, 1)))
    A = O.assemble_stiffness(mesh["nodes"].shape[0], mesh["tets"], Ke)
    # the centre node (0,0,0) is interior
    i = int(np.nonzero(np.all(mesh["nodes"] == 0.0, axis=1))[0][0])
    cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
    vals = A.data[A.indptr[i]:A.indptr[i + 1]]
    assert cols.size == 15  # self + 6 axis + 8 diagonal-edge neighbours
    for c, v in zip(cols, vals):
        d = (mesh["nodes"][c] - mesh["nodes"][i]) / h
        k = int(round(np.abs(d).sum()))
        if k == 0:
            assert abs(v - 6 * h * sig) < 1e-15
        elif k == 1:
            assert abs(v + h * sig) < 1e-15
        else:
            assert abs(v) < 1e-16


# --------------------------------------------------------------------------
# mesh (stand-in for the paper's mesher)
# --------------------------------------------------------------------------

def _brute_force_mesh(h, R):
    """Straight loops over the grid: kept cubes, node numbering, tets."""
    N = int(math.ceil(R / h)) + 1
    G, Gc = 2 * N + 1, 2 * N
    keep = {}
    for I in range(Gc):
        for J in range(Gc):
            for K in range(Gc):
                c = [((I - N) + 0.5) * h, ((J - N) + 0.5) * h, ((K - N) + 0.5) * h]
                keep[(I, J, K)] = (c[0] ** 2 + c[1] ** 2 + c[2] ** 2) < R * R
    used = set()
    for (I, J, K), k in keep.items():
        if k:
            for d in [(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1)]:
                used.add((I + d[0], J + d[1], K + d[2]))
    order = sorted(used, key=lambda t: (t[0] * G + t[1]) * G + t[2])
    nid = {t: i for i, t in enumerate(order)}
    nodes = [((t[0] - N) * h, (t[1] - N) * h, (t[2] - N) * h) for t in order]
    tets = []
    for I in range(Gc):
        for J in range(Gc):
            for K in range(Gc):
                if not keep[(I, J, K)]:
                    continue
                for (a, b, c) in O.PERMS:
                    v = [I, J, K]
                    path = [tuple(v)]
                    v[a] += 1; path.append(tuple(v))
                    v[b] += 1; path.append(tuple(v))
                    path.append((I + 1, J + 1, K + 1))
                    ids = [nid[p] for p in path]
                    # odd permutations give a negatively oriented tet
                    odd = (a, b, c) in ((0, 2, 1), (1, 0, 2), (2, 1, 0))
                    if odd:
                        ids[2], ids[3] = ids[3], ids[2]
                    tets.append(ids)
    return np.array(nodes), np.array(tets)


@pytest.mark.parametrize("h,R", [(0.45, 1.0), (0.3, 1.0), (0.21, 0.7)])
def test_mesh_matches_brute_force(h, R):
    mesh = O.mesh_from_grid(h, [R])
    nodes, tets = _brute_force_mesh(h, R)
    assert np.array_equal(mesh["nodes"], nodes)
    assert np.array_equal(mesh["tets"], tets)


def test_mesh_counts_golden():
    """Node/tet/boundary-face counts of the grid meshes, written by
    tests/golden/make_golden.py from a brute-force count."""
    with open(os.path.join(GOLDEN, "mesh_counts.json")) as f:
        gold = json.load(f)
    for row in gold["rows"]:
        mesh = O.mesh_from_grid(row["h"], row["radii"])
        assert mesh["nodes"].shape[0] == row["n"]
        assert mesh["tets"].shape[0] == row["m"]
        assert mesh["bfaces"].shape[0] == row["nb"]
        assert list(np.bincount(mesh["labels"], minlength=len(row["radii"]))) == row["labels"]


@pytest.mark.parametrize("h", [0.25, 0.1])
def test_mesh_is_a_closed_conforming_positive_mesh(h):
    mesh = O.mesh_from_grid(h, [0.5, 0.8, 1.0])
    nodes, tets, bf = mesh["nodes"], mesh["tets"], mesh["bfaces"]
    g, vol = O.element_geometry(nodes, tets)
    assert np.all(vol > 0)
    assert abs(vol.sum() - (tets.shape[0] // 6) * h ** 3) < 1e-12 * vol.sum()
    # every face is in one or two tets
    faces = np.sort(np.stack([tets[:, list(f)] for f in O.FACES], 1).reshape(-1, 3), 1)
    _, cnt = np.unique(faces, axis=0, return_counts=True)
    assert set(np.unique(cnt)) <= {1, 2}
    assert np.sum(cnt == 1) == bf.shape[0]
    # the boundary is a closed 2-manifold with Euler characteristic 2
    edges = np.sort(np.concatenate([bf[:, [0, 1]], bf[:, [1, 2]], bf[:, [2, 0]]]), 1)
    ue, ecnt = np.unique(edges, axis=0, return_counts=True)
    assert np.all(ecnt == 2)
    V = np.unique(bf).size
    assert V - ue.shape[0] + bf.shape[0] == 2
    # outward orientation: divergence theorem int x.n dS = 3 |Omega|
    p0, p1, p2 = nodes[bf[:, 0]], nodes[bf[:, 1]], nodes[bf[:, 2]]
    nA = 0.5 * np.cross(p1 - p0, p2 - p0)
    flux = np.sum(np.einsum("fi,fi->f", (p0 + p1 + p2) / 3.0, nA))
    assert abs(flux - 3 * vol.sum()) < 1e-10 * vol.sum()


def test_shell_labels_follow_centre_radius():
    h, radii = 0.1, [0.5, 0.8, 1.0]
    mesh = O.mesh_from_grid(h, radii)
    c = mesh["nodes"][mesh["tets"]].mean(axis=1)
    # centroid of a Kuhn tet is not the cube centre; use the cube's min corner + h/2
    corner = mesh["nodes"][mesh["tets"]].min(axis=1)
    cc = np.linalg.norm(corner + h / 2, axis=1)
    expect = np.searchsorted(np.array(radii), cc, side="right")
    assert np.array_equal(mesh["labels"], expect)
    assert np.all(np.linalg.norm(c, axis=1) < 1.0 + h)


# --------------------------------------------------------------------------
# assembled matrix
# --------------------------------------------------------------------------

def _small_system(h=0.25, aniso=True, model="cem", radii=(0.5, 0.7, 1.0), ne=8):
    spec = W.HeadSpec("t", tuple(radii), (0.33, 0.02, 0.33), h, ne, model, 10, 0.4,
                      electrode_radius=0.3, contact_impedance=0.05,
                      skull_aniso=(0.002, 0.02) if aniso else None, seed=7)
    mesh, s6, centres, z, pos, q = O.build_head(spec, W)
    system = O.System(mesh, s6, centres, model, radius=spec.electrode_radius, z=z)
    return spec, mesh, s6, system, pos, q


def test_stiffness_symmetric_zero_rowsum_psd_with_constant_nullspace():
    spec, mesh, s6, sysm, _, _ = _small_system(h=0.3)
    n = sysm.n
    Av = O.assemble_stiffness(n, mesh["tets"], sysm.Ke)
    D = Av.toarray()
    assert np.max(np.abs(D - D.T)) < 1e-15 * np.max(np.abs(D))
    assert np.max(np.abs(D.sum(1))) < 1e-14 * np.max(np.abs(D))
    ev = np.linalg.eigvalsh(D)
    assert abs(ev[0]) < 1e-12 * ev[-1]
    assert ev[1] > 1e-8 * ev[-1]
    # after CEM terms and grounding: SPD
    Ap = sysm.A.toarray()
    assert np.max(np.abs(Ap - Ap.T)) < 1e-15 * np.max(np.abs(Ap))
    assert np.linalg.eigvalsh(Ap)[0] > 0


def test_patch_test_linear_potential_reproduced():
    """Constant anisotropic sigma, u = a.x + c: interior rows of A u vanish, and
    the Neumann problem with the exact boundary flux reproduces u."""
    mesh = O.mesh_from_grid(0.2, [1.0])
    nodes, tets, bf = mesh["nodes"], mesh["tets"], mesh["bfaces"]
    m, n = tets.shape[0], nodes.shape[0]
    s6 = np.tile([0.7, 0.4, 0.9, 0.1, -0.2, 0.05], (m, 1))
    g, vol = O.element_geometry(nodes, tets)
    A = O.assemble_stiffness(n, tets, O.element_stiffness(g, vol, s6))
    a = np.array([0.3, -1.1, 0.8])
    u = nodes @ a + 0.25
    r = A @ u
    interior = np.setdiff1d(np.arange(n), np.unique(bf))
    assert np.max(np.abs(r[interior])) < 1e-13
    # consistent Neumann load f_i = sum_faces (S a . n) area / 3
    S = O.sigma_tensor(s6[:1])[0]
    p0, p1, p2 = nodes[bf[:, 0]], nodes[bf[:, 1]], nodes[bf[:, 2]]
    nA = 0.5 * np.cross(p1 - p0, p2 - p0)
    flux = nA @ (S @ a)
    f = np.zeros(n)
    for k in range(3):
        np.add.at(f, bf[:, k], flux / 3.0)
    ip = int(np.unique(bf)[0])
    Ap = O.pin(A, ip)
    f[ip] = 0.0
    import scipy.sparse.linalg as spla
    x = spla.spsolve(Ap.tocsc(), f)
    assert np.max(np.abs(x - (u - u[ip]))) < 1e-12


def test_pin_zeroes_row_and_column():
    spec, mesh, s6, sysm, _, _ = _small_system(h=0.3)
    A = sysm.A.toarray()
    ip = sysm.ip
    e = np.zeros(sysm.n); e[ip] = 1.0
    assert np.array_equal(A[ip], e) and np.array_equal(A[:, ip], e)
    assert np.all(sysm.B[ip] == 0)


# --------------------------------------------------------------------------
# complete electrode model (App. A.1)
# --------------------------------------------------------------------------

def test_cem_constant_nullspace_identities():
    """[A -B; -B^T C] [1; 1] = 0 before grounding: A 1 = B 1 and B^T 1 = C."""
    spec, mesh, s6, sysm, _, _ = _small_system(h=0.2)
    A = sysm.A_unpinned
    B = sysm.B_unpinned
    one = np.ones(sysm.n)
    lhs = A @ one
    scale = np.max(np.abs(A.data))
    assert np.max(np.abs(lhs - B.sum(1))) < 1e-13 * scale
    assert np.max(np.abs(B.sum(0) - sysm.C)) < 1e-13 * np.max(sysm.C)
    # C l * z l is the patch area
    areas = np.bincount(sysm.el, O.triangle_areas(mesh["nodes"], mesh["bfaces"][sysm.tri]),
                        minlength=sysm.n_el)
    assert np.allclose(sysm.C * sysm.z, areas, rtol=1e-14, atol=0)


def test_cem_patches_are_disjoint_and_near_centres():
    spec, mesh, s6, sysm, _, _ = _small_system(h=0.2)
    assert np.unique(sysm.tri).size == sysm.tri.size
    centres, _ = W.electrode_inputs(spec)
    cen = mesh["nodes"][mesh["bfaces"][sysm.tri]].mean(axis=1)
    d = np.linalg.norm(cen - centres[sysm.el], axis=1)
    assert np.all(d < spec.electrode_radius)


def test_lead_field_equals_block_system_solution():
    """L x via the transfer matrix equals R v from a direct solve of the full
    block system [[A, -B], [-B^T, C]] [z; v] = [-G x; 0] (Eq. u_system)."""
    spec, mesh, s6, sysm, pos, q = _small_system(h=0.2)
    dip = O.locate_dipoles(mesh, pos)
    F = O.source_matrix(sysm.n, mesh["nodes"], mesh["tets"], dip)
    L = O.leadfield(sysm, F)
    rng = np.random.default_rng(0)
    R = O.average_reference(sysm.n_el)
    for _ in range(5):
        x = rng.standard_normal(F.shape[1])
        _, v = O.block_system_solution(sysm, F @ x)
        y = R @ v
        assert np.linalg.norm(L @ x - y) <= 1e-10 * np.linalg.norm(y)


def test_lead_field_invariant_to_ground_node():
    spec, mesh, s6, sysm, pos, q = _small_system(h=0.2)
    dip = O.locate_dipoles(mesh, pos)
    F = O.source_matrix(sysm.n, mesh["nodes"], mesh["tets"], dip)
    L1 = O.leadfield(sysm, F)
    bn = np.unique(mesh["bfaces"])
    covered = np.unique(mesh["bfaces"][sysm.tri])
    free = np.setdiff1d(bn, covered)
    ip2 = int(free[len(free) // 2])
    sysm.ip = ip2
    sysm.A = O.pin(sysm.A_unpinned, ip2)
    sysm.B = sysm.B_unpinned.copy(); sysm.B[ip2] = 0
    sysm._lu = None
    L2 = O.leadfield(sysm, F)
    assert np.linalg.norm(L1 - L2) <= 1e-10 * np.linalg.norm(L1)


def test_point_electrode_lead_field_by_reciprocity():
    """T route (one solve per electrode) equals direct forward solves A u = F q
    per dipole, read at the electrode nodes."""
    spec = W.unit_sphere_point(h=0.2, n_electrodes=12, n_dipoles=10)
    L, sysm, mesh, F, T = O.leadfield_from_spec(spec, W)
    U = sysm.solve(F.toarray())
    Ld = U[sysm.el_nodes[1:], :] - U[sysm.el_nodes[0], :]
    assert np.linalg.norm(L - Ld) <= 1e-11 * np.linalg.norm(L)


def test_transfer_solve_residual_and_dense_solve():
    spec, mesh, s6, sysm, _, _ = _small_system(h=0.3)
    T = sysm.transfer()
    Td = np.linalg.solve(sysm.A.toarray(), sysm.B)
    assert np.max(np.abs(T - Td)) <= 1e-12 * np.max(np.abs(Td))
    res = np.linalg.norm(sysm.A @ T - sysm.B) / np.linalg.norm(sysm.B)
    assert res < 1e-13


# --------------------------------------------------------------------------
# sources
# --------------------------------------------------------------------------

def test_dipoles_located_inside_their_tets_and_gradients_sum_to_zero():
    spec = W.three_shell(0.006, 16, 500, seed=11)
    mesh = O.mesh_from_grid(spec.h, spec.radii)
    pos, q = W.dipole_inputs(spec)
    dip = O.locate_dipoles(mesh, pos)
    X = mesh["nodes"][mesh["tets"][dip]]          # P x 4 x 3
    M = np.ones((dip.size, 4, 4)); M[:, :, 1:] = X
    rhs = np.concatenate([np.ones((dip.size, 1)), pos], 1)[:, :, None]
    lam = np.linalg.solve(np.transpose(M, (0, 2, 1)), rhs)[:, :, 0]
    assert np.all(lam > -1e-12) and np.allclose(lam.sum(1), 1.0)
    F = O.source_matrix(mesh["nodes"].shape[0], mesh["nodes"], mesh["tets"], dip)
    assert np.max(np.abs(np.asarray(F.sum(0)))) < 1e-9 * np.max(np.abs(F.data))
    # grad lambda applied to the edge vectors gives the identity
    g, _ = O.element_geometry(mesh["nodes"], mesh["tets"][dip[:5]])
    for p in range(5):
        for a in range(4):
            for b in range(4):
                val = g[p, a] @ (X[p, b] - X[p, 0])
                assert abs(val - (float(a == b) - float(a == 0))) < 1e-12


def test_dipole_tie_goes_to_first_permutation():
    mesh = O.mesh_from_grid(0.25, [1.0])
    # point on the main diagonal of a cube: all fractional parts equal
    pos = np.array([[0.1, 0.1, 0.1], [0.05, 0.2, 0.2]])
    dip = O.locate_dipoles(mesh, pos)
    assert dip[0] % 6 == 0
    # f = (0.2, 0.8, 0.8): descending orders (1,2,0) and (2,1,0); first is index 3
    assert dip[1] % 6 == 3


# --------------------------------------------------------------------------
# analytic homogeneous sphere
# --------------------------------------------------------------------------

def test_analytic_sphere_potential_satisfies_neumann_and_laplace():
    rng = np.random.default_rng(3)
    R, sig = 1.0, 0.33
    for _ in range(3):
        r0 = rng.standard_normal(3); r0 *= 0.7 * rng.random() / np.linalg.norm(r0)
        q = rng.standard_normal(3)
        pts = rng.standard_normal((20, 3)); pts /= np.linalg.norm(pts, axis=1, keepdims=True)
        eps = 1e-6
        du = (analytic.sphere_dipole_potential(pts * (R + eps), r0, q, sig, R)
              - analytic.sphere_dipole_potential(pts * (R - eps), r0, q, sig, R)) / (2 * eps)
        u = analytic.sphere_dipole_potential(pts * R, r0, q, sig, R)
        assert np.max(np.abs(du)) < 1e-6 * np.max(np.abs(u))
        # the image part u - u_inf is harmonic: 7-point finite-difference Laplacian
        def u_img(x):
            d = x - r0
            uinf = (d @ q) / (4 * math.pi * sig * np.linalg.norm(d, axis=1) ** 3)
            return analytic.sphere_dipole_potential(x, r0, q, sig, R) - uinf
        x = rng.standard_normal((6, 3)) * 0.3
        hh = 1e-3
        lap = -6 * u_img(x)
        for d in range(3):
            e = np.zeros(3); e[d] = hh
            lap += u_img(x + e) + u_img(x - e)
        lap /= hh * hh
        # second differences of u_img along one axis, for scale
        e = np.array([hh, 0, 0])
        d2 = np.abs(u_img(x + e) + u_img(x - e) - 2 * u_img(x)) / hh ** 2
        assert np.max(np.abs(lap)) < 1e-5 * max(np.max(d2), np.max(np.abs(u_img(x))))


def test_analytic_sphere_reduces_to_infinite_medium_for_large_radius():
    r0 = np.array([0.1, -0.2, 0.3]); q = np.array([0.3, 0.5, -0.2])
    pts = np.array([[0.5, 0.5, 0.0], [-0.4, 0.1, 0.2]])
    u = analytic.sphere_dipole_potential(pts, r0, q, 1.0, 1e4)
    d = pts - r0
    uinf = (d @ q) / (4 * math.pi * np.linalg.norm(d, axis=1) ** 3)
    assert np.allclose(u, uinf, rtol=1e-9)


def _analytic_error(h):
    spec = W.unit_sphere_point(h=h, n_electrodes=16, n_dipoles=40)
    L, sysm, mesh, F, T = O.leadfield_from_spec(spec, W)
    pos, q = W.dipole_inputs(spec)
    en = sysm.el_nodes
    sel = np.nonzero(np.linalg.norm(pos, axis=1) < 0.6)[0]
    Lq = np.stack([L[:, 3 * p:3 * p + 3] @ q[p] for p in sel], 1)
    ua = np.stack([analytic.sphere_dipole_potential(mesh["nodes"][en], pos[p], q[p], 0.33, 1.0)
                   for p in sel], 1)
    ua = ua[1:] - ua[0]
    return np.linalg.norm(Lq - ua) / np.linalg.norm(ua)


def test_fem_lead_field_converges_to_analytic_sphere():
    """Sign and scale of L (G = -F, Eq. u_system) against the analytic ball;
    the staircase boundary gives O(h) error, so the pin is a monotone decrease
    with observed order near one."""
    e = [_analytic_error(h) for h in (0.2, 0.1, 0.05)]
    assert e[0] > e[1] > e[2]
    assert e[1] < 0.2 and e[2] < 0.1
    assert math.log(e[0] / e[2]) / math.log(4.0) > 0.6


# --------------------------------------------------------------------------
# linearised EIT (App. A.3)
# --------------------------------------------------------------------------

def _eit_system(h=0.2, ne=16):
    spec = W.unit_sphere_cem(h=h, n_electrodes=ne)
    mesh, s6, centres, z, pos, q = O.build_head(spec, W)
    return spec, mesh, s6, centres, z


def _eit_y(mesh, s6, centres, z, spec, I):
    sysm = O.System(mesh, s6, centres, "cem", radius=spec.electrode_radius, z=z)
    y, _, _ = O.eit_forward(sysm, I)
    return y


def test_eit_jacobian_matches_central_differences():
    spec, mesh, s6, centres, z = _eit_system(h=0.2, ne=16)
    I = W.injection_patterns(spec.n_electrodes)
    sysm = O.System(mesh, s6, centres, "cem", radius=spec.electrode_radius, z=z)
    J, y = O.eit_jacobian(sysm, I)
    rng = np.random.default_rng(5)
    els = rng.choice(mesh["tets"].shape[0], 12, replace=False)
    eps = 1e-6
    for m in els:
        sp_ = s6.copy(); sp_[m] *= math.exp(eps)
        sm_ = s6.copy(); sm_[m] *= math.exp(-eps)
        fd = (_eit_y(mesh, sp_, centres, z, spec, I) - _eit_y(mesh, sm_, centres, z, spec, I)) / (2 * eps)
        # FD noise: solve rounding (~1e-15 |y|) over the 2e-6 step
        assert np.linalg.norm(fd - J[:, :, m]) <= 1e-6 * np.linalg.norm(J[:, :, m]) + 1e-9 * np.linalg.norm(y)


def test_eit_homogeneity_sum_rule():
    """y is homogeneous of degree -1 in (sigma, 1/z): sum_m J_m plus the
    derivative in a common log-scale of 1/z equals -y."""
    spec, mesh, s6, centres, z = _eit_system(h=0.2, ne=16)
    I = W.injection_patterns(spec.n_electrodes)
    sysm = O.System(mesh, s6, centres, "cem", radius=spec.electrode_radius, z=z)
    J, y = O.eit_jacobian(sysm, I)
    eps = 1e-5
    dz = (_eit_y(mesh, s6, centres, z * math.exp(-eps), spec, I)
          - _eit_y(mesh, s6, centres, z * math.exp(eps), spec, I)) / (2 * eps)
    lhs = J.sum(axis=2) + dz
    assert np.linalg.norm(lhs + y) <= 1e-7 * np.linalg.norm(y)


def test_eit_transfer_impedance_reciprocity():
    """Voltage across pair b from a current at pair a equals the voltage across
    a from the same current at b (M is symmetric)."""
    spec, mesh, s6, centres, z = _eit_system(h=0.2, ne=16)
    sysm = O.System(mesh, s6, centres, "cem", radius=spec.electrode_radius, z=z)
    I = W.injection_patterns(spec.n_electrodes)
    y, M, T = O.eit_forward(sysm, I)
    Vab = I @ y.T  # [b, a] = I_b . y_a  (R drops out since sum I_b = 0)
    assert np.max(np.abs(Vab - Vab.T)) <= 1e-10 * np.max(np.abs(Vab))


def test_average_reference_matrix():
    """R (App. A.1): r_jj = 1 - 1/L, r_ij = -1/L; R 1 = 0, R^2 = R, and R v is v
    minus its mean."""
    L = 7
    R = O.average_reference(L)
    assert np.allclose(np.diag(R), 1 - 1 / L) and abs(R[0, 1] + 1 / L) < 1e-16
    assert np.max(np.abs(R @ np.ones(L))) < 1e-15
    v = np.arange(L, dtype=float) ** 2
    assert np.allclose(R @ v, v - v.mean())


def test_pattern_is_the_mesh_graph_whatever_the_values():
    """The CSR pattern of A (with CEM terms) is {(i, j): i, j share a tet},
    independent of sigma: an isotropic sigma (exactly-zero couplings on the
    Kuhn diagonals of exact coordinates) gives the same pattern."""
    spec, mesh, s6, sysm, _, _ = _small_system(h=0.25, aniso=False)
    tets = mesh["tets"]
    pairs = set()
    for t in tets:
        for a in t:
            for b in t:
                pairs.add((int(a), int(b)))
    A = sysm.A_unpinned
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    got = set(zip(rows.tolist(), A.indices.tolist()))
    assert got == pairs


# --------------------------------------------------------------------------
# CPU block PCG baseline (Sec. 2.3.1 iteration) against the direct solve
# --------------------------------------------------------------------------

def test_cpu_block_pcg_matches_direct_solve():
    from oracle import cpu_pcg
    spec = W.three_shell(0.006, 16, 10, seed=21, electrode_radius=0.009)
    mesh = O.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"], mesh["tets"], mesh["labels"])
    centres, z = W.electrode_inputs(spec)
    system = O.System(mesh, s6, centres, spec.electrode_model, radius=spec.electrode_radius, z=z)
    T_direct = system.transfer()
    counts = set()
    for precond in (0, 1):
        for threads in (1, 3):
            T, iters, k = cpu_pcg.block_pcg(system.A, system.B, tol=1e-12, precond=precond, threads=threads)
            # |T - T*| <= kappa-scaled residual; the residual itself is at the stop test
            assert np.linalg.norm(T - T_direct) <= 1e-9 * np.linalg.norm(T_direct)
            res = np.linalg.norm(system.A @ T - system.B, axis=0) / np.linalg.norm(system.B, axis=0)
            assert np.all(res <= 1e-12 * (1 + 1e-6))
            assert k == iters.max() and k > 10
            counts.add((precond, k))
    # the thread split changes only the summation order of the dots
    assert len({k for _, k in counts}) <= 2


def test_assembled_couplings_are_noise_or_genuine():
    """The solver copies drop couplings below 2^-40 sqrt(a_ii a_jj) as assembly
    noise (FP64) and below 2^-24 (FP32).  That is safe because the assembled
    off-diagonal entries fall into two separated groups: the exact zeros of the
    Kuhn diagonal edges (isotropic elements), which come out at rounding level,
    and genuine couplings far above both cuts -- isotropic and anisotropic
    heads alike."""
    for aniso in (None, (0.00132, 0.0132)):
        spec = W.three_shell(0.006, 16, 10, seed=2, skull_aniso=aniso)
        mesh = O.mesh_from_grid(spec.h, spec.radii)
        s6 = W.conductivity(spec, mesh["nodes"], mesh["tets"], mesh["labels"])
        centres, z = W.electrode_inputs(spec)
        system = O.System(mesh, s6, centres, spec.electrode_model, radius=spec.electrode_radius, z=z)
        A = system.A.tocoo()
        d = np.abs(system.A.diagonal())
        off = A.row != A.col
        rel = np.abs(A.data[off]) / np.sqrt(d[A.row[off]] * d[A.col[off]])
        noise = rel <= 2.0 ** -40
        assert noise.sum() > 0.3 * off.sum()            # the diagonal edges are there
        assert np.all(rel[noise] < 1e-14)               # and at rounding level
        assert np.all(rel[~noise] > 2.0 ** -24)         # everything else survives both cuts


def test_difference_form_operator_is_the_matrix():
    """Reading P20: the inner FP32 solve applies A as c_i p_i + sum_{j != i}
    a_ij (p_j - p_i) with c_i the row sum.  In exact arithmetic that is A p
    (checked here in FP64 on the oracle's assembled CEM matrix), and in FP32
    it is far closer to A p than the plain form on a smooth vector."""
    spec = W.three_shell(0.006, 16, 10, seed=2, skull_aniso=(0.00132, 0.0132))
    mesh = O.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"], mesh["tets"], mesh["labels"])
    centres, z = W.electrode_inputs(spec)
    system = O.System(mesh, s6, centres, spec.electrode_model, radius=spec.electrode_radius, z=z)
    A = system.A.tocoo()
    c = np.asarray(system.A.sum(axis=1)).ravel()
    off = A.row != A.col

    def diff_form(p, dtype):
        a = A.data[off].astype(dtype)
        t = a * (p[A.col[off]].astype(dtype) - p[A.row[off]].astype(dtype))
        q = np.zeros(A.shape[0], dtype=dtype)
        np.add.at(q, A.row[off], t)
        return q + c.astype(dtype) * p.astype(dtype)

    rng = np.random.default_rng(0)
    p = rng.standard_normal(A.shape[0])
    exact = system.A @ p
    assert np.linalg.norm(diff_form(p, np.float64) - exact) <= 1e-12 * np.linalg.norm(exact)
    # a smooth vector (a linear function plus a constant), stored in FP32 as the inner solve stores its
    # direction; the exact product is A applied to that stored vector.  On the stiffness rows a linear
    # function lies in the kernel of A, so A p cancels in the plain form but not in the difference form.
    x = mesh["nodes"]
    ps = (1.0 + 0.3 * x[:, 0] / 0.092 + 0.2 * x[:, 2] / 0.092).astype(np.float32).astype(np.float64)
    ex = system.A @ ps
    plain = (system.A.astype(np.float32) @ ps.astype(np.float32)).astype(np.float64)
    diff = diff_form(ps, np.float32).astype(np.float64)
    scale = abs(system.A) @ np.abs(ps)
    interior = np.abs(ex) < 1e-6 * scale
    assert interior.sum() > A.shape[0] // 4
    err_plain = np.abs(plain - ex)
    err_diff = np.abs(diff - ex)
    assert np.linalg.norm(err_diff) < 0.2 * np.linalg.norm(err_plain)
    assert np.linalg.norm(err_diff[interior]) < 0.02 * np.linalg.norm(err_plain[interior])


def test_point_electrodes_are_the_nearest_boundary_nodes():
    """Electrode placement (reading P6 / step 2): against a k-d tree over the
    boundary nodes, the lowest index on an exact tie, and a duplicate raises."""
    from scipy.spatial import cKDTree
    mesh = O.mesh_from_grid(0.1, (1.0,))
    nodes, bf = mesh["nodes"], mesh["bfaces"]
    bn = np.unique(bf)
    centres = W.fibonacci_points(40, 1.0)
    got = O.point_electrode_nodes(nodes, bf, centres)
    d, j = cKDTree(nodes[bn]).query(centres)
    assert np.allclose(np.linalg.norm(nodes[got] - centres, axis=1), d, atol=1e-15)
    # a centre exactly halfway between two boundary nodes (h = 1/8: exact coordinates) takes the lower index
    m8 = O.mesh_from_grid(0.125, (1.0,))
    n8, b8 = m8["nodes"], m8["bfaces"]
    bn8 = np.unique(b8)
    a = bn8[0]
    b = next(c for c in bn8[1:] if np.sum(n8[c] != n8[a]) == 1 and np.abs(n8[c] - n8[a]).max() == 0.125)
    mid = 0.5 * (n8[a] + n8[b])
    dd = np.sum((n8[bn8] - mid) ** 2, axis=1)
    assert np.sum(dd == dd.min()) >= 2
    assert O.point_electrode_nodes(n8, b8, mid[None, :])[0] == min(a, b)
    with pytest.raises(O.OracleError):
        O.point_electrode_nodes(nodes, bf, np.vstack([centres[:1], centres[:1]]))
