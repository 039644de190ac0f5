"""Pins of the segmentation-mesher oracle (Sec. 2.5, "mesh tool") against
mathematics it does not use itself: the winding number against half-space
tests on convex polyhedra and against ray-crossing parity on a non-convex
surface, node labels of nested spheres against their radii, the priority
rule recounted by brute force (and its monotonicity), a conforming mesh with
a closed boundary, and compartment volumes converging with h."""
import math

import numpy as np

from oracle import segmesh as S, zi_oracle as O
from paper_1811_07717_gb300 import workloads as W


def test_winding_number_of_a_convex_polyhedron_is_the_half_space_test():
    V, T = W.icosphere(2, 1.0)
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    off = np.einsum("ij,ij->i", n, V[T[:, 0]])
    rng = np.random.default_rng(1)
    P = rng.uniform(-1.3, 1.3, (2000, 3))
    side = P @ n.T - off[None, :]                # < 0 on the inner side of every face
    inside = np.all(side < 0, axis=1)
    clear = np.min(np.abs(side) / np.linalg.norm(n, axis=1)[None, :], axis=1) > 1e-6
    wn = S.winding_number(P[clear], V, T)
    assert np.allclose(wn, inside[clear].astype(float), atol=1e-9)
    assert 200 < inside.sum() < 1800


def _notched_box():
    """A closed non-convex surface: the unit cube with a square notch cut into
    its top face (an L-shaped prism extruded along y), outward triangles."""
    # profile in the x-z plane (counterclockwise): an L shape
    prof = np.array([[0, 0], [1, 0], [1, 1], [0.6, 1], [0.6, 0.5], [0, 0.5]], dtype=float)
    k = prof.shape[0]
    V = np.array([[x, 0.0, z] for x, z in prof] + [[x, 1.0, z] for x, z in prof])
    tris = []
    for i in range(k):
        j = (i + 1) % k
        tris += [(i, k + j, j), (i, k + i, k + j)]
    # caps: fan triangulation of the L (convex pieces: [0,1,2,3,4] and [0,4,5])
    for a, b, c in [(0, 1, 4), (1, 2, 3), (1, 3, 4), (0, 4, 5)]:
        tris += [(a, b, c), (k + a, k + c, k + b)]
    V = V - 0.5
    T = np.array(tris)
    # closed and consistently oriented: every directed edge has its reverse
    directed = {(a, b) for t in T for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
    assert all((b, a) in directed for a, b in directed) and len(directed) == 3 * T.shape[0]
    # outward: positive enclosed volume (0.5 * 1 + 0.4 * 0.5 of the unit cube)
    vol = np.einsum("ij,ij->i", V[T[:, 0]], np.cross(V[T[:, 1]], V[T[:, 2]])).sum() / 6
    assert abs(vol - 0.7) < 1e-12
    return V, T


def _ray_parity(P, V, T, d):
    """Crossings of the ray P + t d (t > 0) with the triangles (Moller-Trumbore), mod 2."""
    out = np.zeros(P.shape[0], dtype=int)
    for a, b, c in V[T]:
        e1, e2 = b - a, c - a
        pv = np.cross(d, e2)
        det = e1 @ pv
        if abs(det) < 1e-14:
            continue
        tv = P - a
        u = tv @ pv / det
        qv = np.cross(tv, e1)
        v = qv @ d / det
        t = qv @ e2 / det
        out += ((u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)).astype(int)
    return out % 2


def test_winding_number_of_a_non_convex_surface_is_the_ray_parity():
    V, T = _notched_box()
    rng = np.random.default_rng(2)
    P = rng.uniform(-0.7, 0.7, (1500, 3))
    d = np.array([0.3127, 0.1789, 0.9325])
    d /= np.linalg.norm(d)
    par = _ray_parity(P, V, T, d)
    wn = S.winding_number(P, V, T)
    assert np.all(np.minimum(np.abs(wn), np.abs(wn - 1)) < 1e-9)
    assert np.array_equal(np.rint(wn).astype(int), par)
    # the notch is outside, the box's lower half inside
    assert S.winding_number(np.array([[-0.2, 0.0, 0.25]]), V, T)[0] < 0.5
    assert S.winding_number(np.array([[0.0, 0.0, -0.3]]), V, T)[0] > 0.5


def _shells(level=3, radii=(0.8, 0.86, 1.0)):
    return [W.icosphere(level, r) for r in radii]


def test_node_labels_of_nested_spheres_follow_the_radii():
    radii = (0.8, 0.86, 1.0)
    surf = _shells(3, radii)
    rng = np.random.default_rng(3)
    P = rng.uniform(-1.1, 1.1, (3000, 3))
    r = np.linalg.norm(P, axis=1)
    # facets of an icosphere lie within radius * (1 - cos(max edge angle)) of the sphere
    V, T = W.icosphere(3, 1.0)
    edge = np.max(np.linalg.norm(V[T[:, 0]] - V[T[:, 1]], axis=1))
    sag = edge * edge / 2
    clear = np.all(np.abs(r[:, None] - np.array(radii)[None, :]) > sag * 1.1, axis=1)
    lab = S.node_labels(P[clear], surf)
    exact = np.searchsorted(np.array(radii), r[clear], side="right")
    exact[exact == len(radii)] = S.OUTSIDE
    assert np.array_equal(lab, exact)


def test_mesh_is_conforming_and_labelled_by_priority():
    surf = _shells(2)
    prio = (3, 1, 2)       # skull (compartment 1) first, as for a thin layer
    mesh = S.mesh_from_surfaces(0.2, surf, prio)
    nodes, tets = mesh["nodes"], mesh["tets"]
    # positive volumes
    e1 = nodes[tets[:, 1]] - nodes[tets[:, 0]]
    det = np.einsum("mi,mi->m", e1, np.cross(nodes[tets[:, 2]] - nodes[tets[:, 0]], nodes[tets[:, 3]] - nodes[tets[:, 0]]))
    assert np.all(det > 0)
    # every face in one or two tets; the boundary surface is a closed 2-manifold with Euler characteristic 2
    faces = np.sort(np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]]), axis=1)
    _, cnt = np.unique(faces, axis=0, return_counts=True)
    assert cnt.max() == 2
    bf = mesh["bfaces"]
    edges = np.unique(np.sort(np.concatenate([bf[:, [0, 1]], bf[:, [1, 2]], bf[:, [0, 2]]]), axis=1), axis=0)
    assert np.unique(bf).size - edges.shape[0] + bf.shape[0] == 2
    # labels: the best-priority node label, recounted from the grid labels
    glab = mesh["node_label"]
    gidx = mesh["grid_index"][tets]
    for t in range(0, tets.shape[0], 7):
        cands = [c for c in glab[gidx[t]] if c != S.OUTSIDE]
        assert cands
        assert mesh["labels"][t] == min(cands, key=lambda c: (prio[c], c))
    # raising the skull's priority never shrinks it; lowering it never grows it
    low = S.mesh_from_surfaces(0.2, surf, (1, 3, 2))
    assert np.sum(mesh["labels"] == 1) >= np.sum(low["labels"] == 1)
    assert tets.shape[0] == low["tets"].shape[0]        # the kept set does not depend on priorities


def test_compartment_volumes_converge():
    """The labelled volumes approach the spheres' with h (the any-node rule
    and the priorities bias them outward by at most a cell layer)."""
    radii = (0.8, 0.86, 1.0)
    surf = _shells(3, radii)
    exact = np.array([4 / 3 * math.pi * radii[0] ** 3] + [4 / 3 * math.pi * (radii[c] ** 3 - radii[c - 1] ** 3)
                                                         for c in (1, 2)])
    err = []
    for h in (0.2, 0.1):
        mesh = S.mesh_from_surfaces(h, surf, (1, 2, 3))
        _, vol = O.element_geometry(mesh["nodes"], mesh["tets"])
        got = np.array([vol[mesh["labels"] == c].sum() for c in range(3)])
        err.append(np.abs(got / exact - 1))
        # every label is the rule's: recount with the scalar definition
        glab, gidx = mesh["node_label"], mesh["grid_index"][mesh["tets"]]
        for t in range(0, mesh["tets"].shape[0], 11):
            assert mesh["labels"][t] == S.tet_label(glab[gidx[t]], (1, 2, 3))
    assert np.all(err[1] < 0.25)
    assert err[1][0] < 0.7 * err[0][0] and np.abs(err[1]).sum() < np.abs(err[0]).sum()


def _locate_brute_force(nodes, tets, pos):
    """The tet whose smallest barycentric coordinate at the point is largest."""
    M = np.ones((tets.shape[0], 4, 4))
    M[:, :, 1:] = nodes[tets]
    inv = np.linalg.inv(M)
    out = np.empty(pos.shape[0], dtype=np.int64)
    for p, x in enumerate(pos):
        lam = np.einsum("mji,j->mi", inv, np.concatenate([[1.0], x]))
        out[p] = np.argmax(lam.min(axis=1))
    return out


def test_lead_field_on_a_segmentation_mesh_converges_to_the_analytic_ball():
    """End to end: the mesh of one icosphere surface feeds the EEG build, and
    its lead field approaches the homogeneous-ball potential as h falls."""
    from oracle import analytic
    errs = []
    for h in (0.2, 0.1):
        spec = W.unit_sphere_point(h=h, n_electrodes=16, n_dipoles=40)
        mesh = S.mesh_from_surfaces(h, [W.icosphere(3, 1.0)], (1,))
        s6 = W.conductivity(spec, mesh["nodes"], mesh["tets"], mesh["labels"])
        centres, _ = W.electrode_inputs(spec)
        pos, q = W.dipole_inputs(spec)
        sysm = O.System(mesh, s6, centres, "point")
        dip = _locate_brute_force(mesh["nodes"], mesh["tets"], pos)
        L = O.leadfield(sysm, O.source_matrix(sysm.n, mesh["nodes"], mesh["tets"], dip))
        sel = np.nonzero(np.linalg.norm(pos, axis=1) < 0.6)[0]
        Lq = np.stack([L[:, 3 * p:3 * p + 3] @ q[p] for p in sel], 1)
        ua = np.stack([analytic.sphere_dipole_potential(mesh["nodes"][sysm.el_nodes], pos[p], q[p], 0.33, 1.0)
                       for p in sel], 1)
        ua = ua[1:] - ua[0]
        errs.append(np.linalg.norm(Lq - ua) / np.linalg.norm(ua))
    assert errs[1] < 0.6 * errs[0] and errs[1] < 0.2
