"""Pins of the MEG oracle (App. A.2 by way of the Biot-Savart formula) against
mathematics it does not use itself: Sarvas' closed form for a spherically
symmetric conductor (self-checked: curl- and divergence-free outside, radial
component of the primary current alone, no field from radial or central
dipoles), the quadrature rule against adaptive cubature, the transfer route
against direct forward solves, invariance to the grounding node, and the
FEM lead field converging to the closed form, with the volume-current part
vanishing for radial sensors as the mesh is refined."""
import math

import numpy as np
import pytest
from scipy.integrate import tplquad

from oracle import analytic, meg as M, zi_oracle as O
from paper_1811_07717_gb300 import workloads as W


def test_sarvas_closed_form_checks():
    rng = np.random.default_rng(2)
    for _ in range(4):
        r0 = rng.standard_normal(3)
        r0 *= 0.7 * rng.random() / np.linalg.norm(r0)
        q = rng.standard_normal(3)
        pts = rng.standard_normal((10, 3))
        pts *= (1.1 + rng.random((10, 1))) / np.linalg.norm(pts, axis=1, keepdims=True)
        B = analytic.sarvas_field(pts, r0, q)
        # the radial component is that of the primary current alone
        rhat = pts / np.linalg.norm(pts, axis=1, keepdims=True)
        Bp = analytic.primary_field(pts, r0, q)
        assert np.allclose(np.sum(B * rhat, 1), np.sum(Bp * rhat, 1), rtol=1e-10, atol=1e-14 * np.abs(B).max())
        # curl- and divergence-free outside the conductor (central differences)
        e = 1e-5
        J = np.zeros((pts.shape[0], 3, 3))  # J[:, i, j] = dB_i / dx_j
        for j in range(3):
            dx = np.zeros(3)
            dx[j] = e
            J[:, :, j] = (analytic.sarvas_field(pts + dx, r0, q) - analytic.sarvas_field(pts - dx, r0, q)) / (2 * e)
        scale = np.abs(J).max()
        curl = np.stack([J[:, 2, 1] - J[:, 1, 2], J[:, 0, 2] - J[:, 2, 0], J[:, 1, 0] - J[:, 0, 1]], 1)
        assert np.abs(curl).max() < 1e-7 * scale
        assert np.abs(np.trace(J, axis1=1, axis2=2)).max() < 1e-7 * scale
    # radial dipoles and dipoles at the centre have no external field
    pts = np.array([[0.0, 0.0, 1.5], [1.2, 0.3, -0.4]])
    r0 = np.array([0.1, -0.2, 0.3])
    assert np.abs(analytic.sarvas_field(pts, r0, 2.0 * r0)).max() < 1e-22
    assert np.abs(analytic.sarvas_field(pts, np.zeros(3) + 1e-300, np.array([0.3, 0.1, 0.2]))).max() < 1e-20


def test_quadrature_rule_is_degree_two_and_converges_with_distance():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((4, 3))
    vol = abs(np.linalg.det(X[1:] - X[0])) / 6
    pts = M.quadrature_points(X)
    # barycentric coordinates of the points; int lambda_a lambda_b = vol (1 + delta_ab) / 20
    lam = np.linalg.solve(np.hstack([np.ones((4, 1)), X]).T, np.hstack([np.ones((4, 1)), pts]).T).T
    for a in range(4):
        for b in range(4):
            assert abs(vol / 4 * np.sum(lam[:, a] * lam[:, b]) - vol * (1 + (a == b)) / 20) < 1e-14
    # against adaptive cubature on the reference tet: error falls like (size / distance)^3
    Xr = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    errs = []
    for dist in (2.0, 4.0):
        r = np.array([dist, 0.3 * dist, 0.2 * dist])
        ref = np.array([tplquad(lambda z, y, x, c=c: (r[c] - (x, y, z)[c]) / np.linalg.norm(r - np.array([x, y, z])) ** 3,
                                0, 1, lambda x: 0, lambda x: 1 - x, lambda x, y: 0, lambda x, y: 1 - x - y,
                                epsabs=1e-13, epsrel=1e-11)[0] for c in range(3)])
        errs.append(np.linalg.norm(M.kernel_integral(Xr, 1 / 6, r) - ref) / np.linalg.norm(ref))
    assert errs[0] < 5e-3 and errs[1] < errs[0] / 8


def _sphere(h, Ns=24, tilt=0.6, n_dipoles=40, roll=0):
    spec = W.unit_sphere_point(h=h, n_electrodes=16, n_dipoles=n_dipoles)
    mesh, s6, centres, z, pos, q = O.build_head(spec, W)
    sysm = O.System(mesh, s6, np.roll(centres, roll, axis=0), "point")
    sp_, sd = W.meg_sensors(Ns, 1.2, tilt=tilt)
    dip = O.locate_dipoles(mesh, pos)
    F = O.source_matrix(sysm.n, mesh["nodes"], mesh["tets"], dip)
    return mesh, s6, sysm, sp_, sd, pos, q, F


def test_transfer_route_equals_forward_solves_and_is_blind_to_grounding():
    mesh, s6, sysm, sp_, sd, pos, q, F = _sphere(0.2)
    L = M.meg_leadfield(sysm, s6, sp_, sd, pos, F)
    # forward route: u = A^-1 F (grounded), then Bm^T u
    Bm = M.meg_rhs(sysm, s6, sp_, sd)
    Fd = F.toarray()
    Fd[sysm.ip, :] = 0.0
    u = sysm.solve(Fd)
    L_fwd = M.primary(sp_, sd, pos) + Bm.T @ u
    assert np.linalg.norm(L - L_fwd) <= 1e-11 * np.linalg.norm(L)
    # another grounding node gives the same lead field
    _, _, sys2, _, _, _, _, _ = _sphere(0.2, roll=5)
    assert sys2.ip != sysm.ip
    L2 = M.meg_leadfield(sys2, s6, sp_, sd, pos, F)
    assert np.linalg.norm(L2 - L) <= 1e-11 * np.linalg.norm(L)


def test_meg_lead_field_converges_to_sarvas():
    errs, prim = [], []
    for h in (0.2, 0.1, 0.05):
        mesh, s6, sysm, sp_, sd, pos, q, F = _sphere(h)
        L = M.meg_leadfield(sysm, s6, sp_, sd, pos, F)
        sel = np.nonzero(np.linalg.norm(pos, axis=1) < 0.6)[0]
        Lq = np.stack([L[:, 3 * p:3 * p + 3] @ q[p] for p in sel], 1)
        Ba = np.stack([np.sum(analytic.sarvas_field(sp_, pos[p], q[p]) * sd, 1) for p in sel], 1)
        Bp = np.stack([np.sum(analytic.primary_field(sp_, pos[p], q[p]) * sd, 1) for p in sel], 1)
        errs.append(np.linalg.norm(Lq - Ba) / np.linalg.norm(Ba))
        prim.append(np.linalg.norm(Bp - Ba) / np.linalg.norm(Ba))
    assert min(prim) > 1.0              # the volume currents matter for tilted sensors
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.1
    assert math.log(errs[0] / errs[2]) / math.log(4.0) > 0.8


def test_radial_sensors_see_no_volume_current_in_the_limit():
    """For a spherically symmetric conductor the radial field is the primary
    one; the FEM volume part for radial sensors falls with h."""
    rel = []
    for h in (0.2, 0.1, 0.05):
        mesh, s6, sysm, sp_, sd, pos, q, F = _sphere(h, tilt=0.0)
        Tm = M.meg_transfer(sysm, s6, sp_, sd)
        rel.append(np.linalg.norm(np.asarray((F.T @ Tm).T)) / np.linalg.norm(M.primary(sp_, sd, pos)))
    assert rel[0] > rel[1] > rel[2] and rel[2] < 0.02


def test_hdiv_sources_beat_partial_integration_for_meg_too():
    """The H(div) sources' accuracy (Sec. 2.1) carries over to the magnetic
    lead field: against Sarvas, PBO10 < Whitney < partial integration."""
    from oracle import hdiv as HD
    for h in (0.2, 0.1):
        mesh, s6, sysm, sp_, sd, pos, q, F = _sphere(h)
        Tm = M.meg_transfer(sysm, s6, sp_, sd)
        dip = O.locate_dipoles(mesh, pos)
        sel = np.nonzero(np.linalg.norm(pos, axis=1) < 0.6)[0]
        Ba = np.stack([np.sum(analytic.sarvas_field(sp_, pos[p], q[p]) * sd, 1) for p in sel], 1)
        errs = []
        for Fm in (F, HD.source_matrix_hdiv(mesh["nodes"], mesh["tets"], dip, pos, HD.WHITNEY4),
                   HD.source_matrix_hdiv(mesh["nodes"], mesh["tets"], dip, pos, HD.PBO10)):
            L = M.meg_leadfield(sysm, s6, sp_, sd, pos, Fm, Tm=Tm)
            Lq = np.stack([L[:, 3 * p:3 * p + 3] @ q[p] for p in sel], 1)
            errs.append(np.linalg.norm(Lq - Ba) / np.linalg.norm(Ba))
        assert errs[2] < errs[1] < errs[0]


def test_meg_lead_field_is_blind_to_a_global_conductivity_scale():
    """Scaling every conductivity by a scales A and Bm alike, so T_meg and the
    MEG lead field do not change (the EEG lead field scales by 1/a)."""
    mesh, s6, sysm, sp_, sd, pos, q, F = _sphere(0.2)
    L1 = M.meg_leadfield(sysm, s6, sp_, sd, pos, F)
    centres = W.electrode_inputs(W.unit_sphere_point(h=0.2, n_electrodes=16, n_dipoles=40))[0]
    sys3 = O.System(mesh, 3.0 * s6, centres, "point")
    L3 = M.meg_leadfield(sys3, 3.0 * s6, sp_, sd, pos, F)
    assert np.linalg.norm(L3 - L1) <= 1e-11 * np.linalg.norm(L1)
    assert np.linalg.norm(O.leadfield(sys3, F) * 3.0 - O.leadfield(sysm, F)) <= 1e-11 * np.linalg.norm(O.leadfield(sysm, F))
