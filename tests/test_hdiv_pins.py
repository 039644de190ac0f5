"""Pins of the H(div) source oracle (Sec. 2.1, "Primary current model")
against mathematics it does not use itself: the face source's load and moment
are integrals of the lowest-order Raviart-Thomas function, every stencil
source is a discrete dipole for linear potentials, the PBO coefficients are
the constrained minimiser found by an independent optimiser, the neighbour
table agrees with a brute-force search, and the lead field of the Cartesian
H(div) sources converges to the analytic ball faster than partial
integration (the paper's accuracy claim for this model)."""
import math

import numpy as np
import pytest
from scipy.linalg import null_space
from scipy.optimize import minimize

from oracle import analytic, hdiv as HD, zi_oracle as O
from paper_1811_07717_gb300 import workloads as W


def tet_grads(X):
    """Gradients of the barycentric coordinates of tet X (4 x 3), from the
    inverse of [1 x]."""
    M = np.hstack([np.ones((4, 1)), X])
    return np.linalg.inv(M)[1:].T          # row a = grad lambda_a


def test_face_source_load_and_moment_are_raviart_thomas_integrals():
    """Two random tets sharing a face; the RT0 function with unit flux from T
    into N is (x - x_v)/(3|T|) on T and -(x - x_o)/(3|N|) on N.  Its loads
    int w . grad psi_i and its moment int w (exact by the centroid rule, w
    being linear) are what the stencil uses: +-1/4 at o and v, (x_o - x_v)/4."""
    rng = np.random.default_rng(11)
    for _ in range(5):
        face = rng.standard_normal((3, 3))
        nrm = np.cross(face[1] - face[0], face[2] - face[0])
        xv = face.mean(0) + nrm * rng.uniform(0.3, 1.0) + 0.3 * rng.standard_normal(3)
        xo = face.mean(0) - nrm * rng.uniform(0.3, 1.0) + 0.3 * rng.standard_normal(3)
        XT = np.vstack([face, xv])        # T = (f0, f1, f2, v); the face is opposite local vertex 3
        XN = np.vstack([face, xo])
        vT = abs(np.linalg.det(XT[:3] - XT[3])) / 6
        vN = abs(np.linalg.det(XN[:3] - XN[3])) / 6
        # unit flux through the face: normal component times area
        area = 0.5 * np.linalg.norm(nrm)
        n_out = nrm / np.linalg.norm(nrm) * np.sign(nrm @ (face.mean(0) - xv))
        assert abs((face.mean(0) - xv) @ n_out / (3 * vT) * area - 1.0) < 1e-12
        wT = lambda x: (x - xv) / (3 * vT)
        wN = lambda x: -(x - xo) / (3 * vN)
        cT, cN = XT.mean(0), XN.mean(0)
        gT, gN = tet_grads(XT), tet_grads(XN)
        load = {}
        for a in range(4):
            load[("T", a)] = vT * wT(cT) @ gT[a]
            load[("N", a)] = vN * wN(cN) @ gN[a]
        # face nodes: contributions from both sides cancel
        for a in range(3):
            assert abs(load[("T", a)] + load[("N", a)]) < 1e-12
        assert abs(load[("T", 3)] - (-0.25)) < 1e-12
        assert abs(load[("N", 3)] - 0.25) < 1e-12
        moment = vT * wT(cT) + vN * wN(cN)
        assert np.allclose(moment, (xo - xv) / 4, atol=1e-12)
        # the oracle's stencil for T (face 3 has neighbour vertex "o")
        nodes = np.vstack([XT, xo])
        loads, d, c = HD.stencil(nodes, np.array([0, 1, 2, 3]), np.array([-1, -1, -1, 4]), HD.WHITNEY4)
        assert loads == [((4, 0.25), (3, -0.25))]
        assert np.allclose(d[0], moment, atol=1e-12)
        assert np.allclose(c[0], face.mean(0))


def _small_mesh(h=0.25):
    return O.mesh_from_grid(h, (1.0,))


def test_stencil_sources_are_discrete_dipoles_for_linear_potentials():
    mesh = _small_mesh()
    nodes, tets = mesh["nodes"], mesh["tets"]
    rng = np.random.default_rng(4)
    which = rng.choice(tets.shape[0], 20, replace=False)
    _, opp = HD.face_neighbours(tets, which)
    for r, t in enumerate(which):
        loads, d, c = HD.stencil(nodes, tets[t], opp[r], HD.PBO10)
        assert len(loads) == 6 + int(np.sum(opp[r] >= 0))
        for _ in range(3):
            g, c0 = rng.standard_normal(3), rng.standard_normal()
            psi = nodes @ g + c0
            for k, pair in enumerate(loads):
                assert abs(sum(a * psi[i] for i, a in pair) - d[k] @ g) < 1e-12


def test_face_neighbours_match_brute_force():
    mesh = _small_mesh(0.3)
    tets = mesh["tets"]
    which = np.arange(0, tets.shape[0], 7)
    nbr, opp = HD.face_neighbours(tets, which)
    sets = [frozenset(int(x) for x in t) for t in tets]
    n_boundary = 0
    for r, t in enumerate(which):
        for k in range(4):
            face = sets[t] - {int(tets[t][k])}
            hits = [u for u in range(tets.shape[0]) if u != t and face <= sets[u]]
            assert len(hits) <= 1
            if hits:
                assert nbr[r, k] == hits[0]
                assert opp[r, k] == next(iter(sets[hits[0]] - face))
                # the neighbour's opposite vertex lies across the face plane from v_k
                X = mesh["nodes"]
                f = sorted(face)
                nrm = np.cross(X[f[1]] - X[f[0]], X[f[2]] - X[f[0]])
                assert (np.dot(X[tets[t][k]] - X[f[0]], nrm) * np.dot(X[opp[r, k]] - X[f[0]], nrm)) < 0
            else:
                n_boundary += 1
                assert nbr[r, k] == -1 and opp[r, k] == -1
    assert n_boundary > 0


@pytest.mark.parametrize("model", [HD.WHITNEY4, HD.PBO10])
def test_pbo_coefficients_are_the_constrained_minimiser(model):
    """D w = e_j exactly, and an independent optimiser (SLSQP with the
    equality constraint, and the null-space parametrisation of the
    constraint) finds the same minimiser."""
    mesh = _small_mesh()
    nodes, tets = mesh["nodes"], mesh["tets"]
    rng = np.random.default_rng(8)
    pos = rng.standard_normal((4, 3)) * 0.3
    dip = O.locate_dipoles(mesh, pos)
    _, opp = HD.face_neighbours(tets, dip)
    lam = 1e-2
    for p in range(4):
        loads, d, c = HD.stencil(nodes, tets[dip[p]], opp[p], model)
        s = HD.mean_edge(nodes[tets[dip[p]]])
        w = HD.pbo_coefficients(pos[p], d, c, s, lam)
        assert np.allclose(d.T @ w, np.eye(3), atol=1e-11)
        N = null_space(d.T)
        for j in range(3):
            wp = np.linalg.lstsq(d.T, np.eye(3)[:, j], rcond=None)[0]
            f = lambda z: HD.objective(wp + N @ z, pos[p], d, c, s, lam)
            z = minimize(f, np.zeros(N.shape[1]), method="BFGS", options=dict(gtol=1e-12)).x
            w_ns = wp + N @ z
            cons = {"type": "eq", "fun": lambda v: d.T @ v - np.eye(3)[:, j]}
            w_sq = minimize(lambda v: HD.objective(v, pos[p], d, c, s, lam), wp, method="SLSQP",
                            constraints=[cons], options=dict(ftol=1e-15, maxiter=500)).x
            scale = np.max(np.abs(w[:, j]))
            assert np.max(np.abs(w_ns - w[:, j])) < 1e-5 * scale
            assert np.max(np.abs(w_sq - w[:, j])) < 1e-4 * scale
            jw = HD.objective(w[:, j], pos[p], d, c, s, lam)
            for _ in range(5):
                assert HD.objective(w[:, j] + N @ (1e-3 * rng.standard_normal(N.shape[1])),
                                    pos[p], d, c, s, lam) >= jw


def test_pbo_scales_inversely_with_the_mesh():
    """Scaling the mesh and the dipole position by a scales every coefficient
    (and so the load of a unit moment) by 1/a."""
    mesh = _small_mesh()
    nodes, tets = mesh["nodes"], mesh["tets"]
    pos = np.array([[0.11, -0.07, 0.23]])
    dip = O.locate_dipoles(mesh, pos)
    F1 = HD.source_matrix_hdiv(nodes, tets, dip, pos).toarray()
    F2 = HD.source_matrix_hdiv(3.0 * nodes, tets, dip, 3.0 * pos).toarray()
    assert np.allclose(F2 * 3.0, F1, rtol=1e-10, atol=1e-12 * np.abs(F1).max())


def test_whitney_on_a_boundary_tet_still_reproduces_the_moment():
    """A tet with a face on the mesh boundary has three face sources; they
    still span the three orientations."""
    mesh = _small_mesh()
    tets, nodes = mesh["tets"], mesh["nodes"]
    _, opp = HD.face_neighbours(tets, np.arange(0, tets.shape[0], 3))
    rows = np.nonzero(np.sum(opp < 0, axis=1) == 1)[0][:6]
    assert rows.size == 6
    for r in rows:
        t = 3 * r
        loads, d, c = HD.stencil(nodes, tets[t], opp[r], HD.WHITNEY4)
        assert len(loads) == 3
        w = HD.pbo_coefficients(nodes[tets[t]].mean(0), d, c, HD.mean_edge(nodes[tets[t]]), 1e-2)
        assert np.allclose(d.T @ w, np.eye(3), atol=1e-11)


def test_hdiv_lead_field_converges_to_the_analytic_ball_faster_than_partial_integration():
    """Sec. 2.1: the H(div) model is more accurate than partial integration.
    On the homogeneous unit ball both the Whitney and the PBO 10-source
    Cartesian sources beat partial integration at every h, and the PBO error
    falls with order near one."""
    errs = {}
    for h in (0.2, 0.1, 0.05):
        spec = W.unit_sphere_point(h=h, n_electrodes=16, n_dipoles=40)
        mesh, s6, centres, z, pos, q = O.build_head(spec, W)
        sysm = O.System(mesh, s6, centres, "point")
        T = sysm.transfer()
        dip = O.locate_dipoles(mesh, pos)
        sel = np.nonzero(np.linalg.norm(pos, axis=1) < 0.6)[0]
        ua = np.stack([analytic.sphere_dipole_potential(mesh["nodes"][sysm.el_nodes], pos[p], q[p], 0.33, 1.0)
                       for p in sel], 1)
        ua = ua[1:] - ua[0]
        Fs = {"pi": O.source_matrix(sysm.n, mesh["nodes"], mesh["tets"], dip),
              "w4": HD.source_matrix_hdiv(mesh["nodes"], mesh["tets"], dip, pos, HD.WHITNEY4),
              "pbo10": HD.source_matrix_hdiv(mesh["nodes"], mesh["tets"], dip, pos, HD.PBO10)}
        for name, F in Fs.items():
            L = O.leadfield(sysm, F, T)
            Lq = np.stack([L[:, 3 * p:3 * p + 3] @ q[p] for p in sel], 1)
            errs[(name, h)] = np.linalg.norm(Lq - ua) / np.linalg.norm(ua)
    for h in (0.2, 0.1, 0.05):
        assert errs[("pbo10", h)] < errs[("w4", h)] < errs[("pi", h)]
    e = [errs[("pbo10", h)] for h in (0.2, 0.1, 0.05)]
    assert e[0] > e[1] > e[2] and e[2] < 0.05
    assert math.log(e[0] / e[2]) / math.log(4.0) > 0.8
