"""Plain FP64 CPU oracle of the MEG lead field (App. A.2 points to the
Biot-Savart law for the magnetic counterpart of the EEG lead field).

TEST INFRASTRUCTURE ONLY: the definition the CUDA path of zi_meg_rhs /
zi_meg_transfer / zi_meg_leadfield is checked against.  Only the test suite
and the benchmark's CPU leg import it; it shares no code with the CUDA
library.

The field of the total current J^p - sigma grad u (Sec. 2.1) at a sensor r_s
outside the head, read along the sensor's unit orientation n_s, is by
Biot-Savart

    b_s = mu0/(4 pi) [ q . ((r_s - x0) x n_s) / |r_s - x0|^3           (primary dipole q at x0)
                       - sum_e (sigma_e grad u_e) . (G_e(r_s) x n_s) ],  (volume current)
    G_e(r) = int_e (r - r') / |r - r'|^3 dV'.

With u = sum_i u_i psi_i (P1), the volume part is Bm^T u, where

    Bm[i, s] = -mu0/(4 pi) sum_{e containing i} grad psi_i|_e . sigma_e (G_e(r_s) x n_s).

The potential of the Cartesian source columns solves A u = F (the EEG
system, Eq. u_system), so the volume part of the lead field is
(A^-1 Bm)^T F = T_meg^T F: one solve per sensor, the same transfer-matrix
route as the EEG lead field.  Row i' of Bm is zeroed with the grounding (the
volume part is blind to a constant in u, since the gradients of a tet's four
basis functions sum to zero).

G_e is integrated by the 4-point degree-2 rule for tetrahedra (barycentric
points (a, b, b, b) and permutations, a = (5 + 3 sqrt 5)/20,
b = (5 - sqrt 5)/20, weights |e|/4).  mu0/(4 pi) = 1e-7 T m/A.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import zi_oracle as O

MU0_OVER_4PI = 1e-7
QA = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
QB = (5.0 - math.sqrt(5.0)) / 20.0


def quadrature_points(X):
    """The rule's four points of tet X (4 x 3): point k has weight a on vertex k."""
    W = np.full((4, 4), QB)
    np.fill_diagonal(W, QA)
    return W @ X


def kernel_integral(X, vol, r):
    """G_e(r) for tet X of volume vol by the 4-point rule."""
    pts = quadrature_points(X)
    d = r[None, :] - pts
    return vol / 4.0 * np.sum(d / np.linalg.norm(d, axis=1)[:, None] ** 3, axis=0)


def meg_rhs(system, sigma6, sens_pos, sens_dir):
    """Bm (n x Ns), row i' zeroed; one sensor at a time over all tets."""
    mesh = system.mesh
    nodes, tets = mesh["nodes"], mesh["tets"]
    grads, vol = system.grads, system.vol                 # grads[e, a] = grad psi_{tets[e,a]} on e
    Sig = O.sigma_tensor(sigma6)
    W = np.full((4, 4), QB)
    np.fill_diagonal(W, QA)
    pts = np.einsum("kj,ejd->ekd", W, nodes[tets])       # (m, 4 points, 3)
    Ns = sens_pos.shape[0]
    Bm = np.zeros((nodes.shape[0], Ns))
    for s in range(Ns):
        d = sens_pos[s][None, None, :] - pts
        G = vol[:, None] / 4.0 * np.sum(d / np.linalg.norm(d, axis=2)[:, :, None] ** 3, axis=1)
        V = np.einsum("eij,ej->ei", Sig, np.cross(G, sens_dir[s][None, :]))
        contrib = -MU0_OVER_4PI * np.einsum("ead,ed->ea", grads, V)
        np.add.at(Bm[:, s], tets, contrib)
    Bm[system.ip, :] = 0.0
    return Bm


def primary(sens_pos, sens_dir, pos):
    """Ns x 3P: the primary-current field of unit Cartesian dipoles, column 3p + d."""
    Ns, P = sens_pos.shape[0], pos.shape[0]
    out = np.zeros((Ns, 3 * P))
    for p in range(P):
        a = sens_pos - pos[p]
        c = np.cross(a, sens_dir) / np.linalg.norm(a, axis=1)[:, None] ** 3
        out[:, 3 * p:3 * p + 3] = MU0_OVER_4PI * c
    return out


def meg_transfer(system, sigma6, sens_pos, sens_dir):
    return system.solve(meg_rhs(system, sigma6, sens_pos, sens_dir))


def meg_leadfield(system, sigma6, sens_pos, sens_dir, pos, F, Tm=None):
    """L_meg (Ns x 3P) = primary + T_meg^T F."""
    if Tm is None:
        Tm = meg_transfer(system, sigma6, sens_pos, sens_dir)
    return primary(sens_pos, sens_dir, pos) + np.asarray((F.T @ Tm).T)
