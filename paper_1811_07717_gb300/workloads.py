"""Seeded synthetic inputs for the FEM lead-field build.

This module only draws and lays out inputs: head geometry parameters, the
conductivity field per element, electrode centres and dipoles.  It holds none
of the method's arithmetic (no geometry of elements, no assembly, no solves),
so that the CUDA path and the CPU oracle can both read the same inputs without
sharing any code of the method itself.

Units are SI throughout: metres, S/m, Ohm*m^2 (contact impedance z = Z*area).

The workloads stand in for the paper's head models (Sec. 2.7): spheres meshed
as regular grids split into Kuhn tetrahedra, with one to three shells
(brain / skull / scalp), the electrode counts and source counts of the paper's
experiments (Sec. 2.7, Sec. 2.1 "Hardware requirements" for the 1 mm scale).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class HeadSpec:
    """One seeded head model.

    radii:       ascending shell radii (m); the last one is the outer surface.
    sigma:       isotropic conductivity per shell (S/m), same length as radii.
    h:           grid step (m).
    n_electrodes, electrode_model: "point" (nearest surface node, electrode 1
                 is the reference) or "cem" (complete electrode model).
    electrode_radius (m), contact_impedance z (Ohm*m^2) for "cem".
    n_dipoles:   source positions, three Cartesian orientations each.
    dipole_rmax: dipoles are uniform in the ball r < dipole_rmax.
    skull_aniso: None, or (sigma_radial, sigma_tangential) for shell 1.
    """

    name: str
    radii: tuple
    sigma: tuple
    h: float
    n_electrodes: int
    electrode_model: str
    n_dipoles: int
    dipole_rmax: float
    electrode_radius: float = 0.0
    contact_impedance: float = 0.0
    skull_aniso: tuple | None = None
    seed: int = 0
    extra: dict = field(default_factory=dict)


def unit_sphere_point(h: float = 0.1, n_electrodes: int = 16, n_dipoles: int = 300,
                      seed: int = 1) -> HeadSpec:
    """Homogeneous unit ball, sigma = 0.33 S/m, point electrodes."""
    return HeadSpec("unit_sphere_point_h%g" % h, (1.0,), (0.33,), h, n_electrodes,
                    "point", n_dipoles, 0.8, seed=seed)


def unit_sphere_cem(h: float = 0.1, n_electrodes: int = 32, n_dipoles: int = 50,
                    seed: int = 5) -> HeadSpec:
    """Homogeneous unit ball with complete-model electrodes of radius 0.15 and
    contact impedance 0.1 (unit-sphere units); used for finite-difference
    checks of the linearised EIT Jacobian."""
    return HeadSpec("unit_sphere_cem_h%g" % h, (1.0,), (0.33,), h, n_electrodes, "cem",
                    n_dipoles, 0.8, electrode_radius=0.15, contact_impedance=0.1, seed=seed)


def three_shell(h: float = 0.002, n_electrodes: int = 128, n_dipoles: int = 20000,
                seed: int = 2, r_out: float = 0.092, skull_aniso=None,
                electrode_radius: float = 0.005) -> HeadSpec:
    """Three-shell head: brain / skull / scalp with radii scaled from
    80 / 86 / 92 mm, sigma 0.33 / 0.0132 / 0.33 S/m, 5 mm electrodes with
    2 kOhm*mm^2 contact impedance, dipoles uniform in r < 78/92 * r_out."""
    s = r_out / 0.092
    radii = (0.080 * s, 0.086 * s, r_out)
    return HeadSpec("three_shell_h%gmm_L%d" % (h * 1e3, n_electrodes), radii,
                    (0.33, 0.0132, 0.33), h, n_electrodes, "cem", n_dipoles, 0.078 * s,
                    electrode_radius=electrode_radius, contact_impedance=2e-3,
                    skull_aniso=skull_aniso, seed=seed)


def config_unit_sphere() -> HeadSpec:
    """Plain method, FP64: unit sphere, h = 0.1, 16 point electrodes, 300 dipoles."""
    return unit_sphere_point(0.1, 16, 300, seed=1)


def config_three_shell_2mm() -> HeadSpec:
    """Three-shell sphere, h = 2 mm, 128 CEM electrodes, 20k dipoles."""
    return three_shell(0.002, 128, 20000, seed=2)


def config_three_shell_1mm_aniso() -> HeadSpec:
    """h = 1 mm, transversely anisotropic skull (radial 0.00132, tangential
    0.0132 S/m), 256 electrodes, 100k dipoles."""
    return three_shell(0.001, 256, 100000, seed=3, skull_aniso=(0.00132, 0.0132))


def config_eit_2mm() -> HeadSpec:
    """Linearised EIT: h = 2 mm three-shell mesh with 32 scalp electrodes."""
    return three_shell(0.002, 32, 0, seed=5)


def config_batch(n_heads: int = 24, seed: int = 4, h_choices=(0.0015, 0.002, 0.003),
                 le_choices=(32, 64, 128, 256), dip_range=(5000, 30000),
                 r_range=(0.080, 0.100)) -> list:
    """Batch of seeded three-shell heads of uneven size: outer radius uniform in
    80-100 mm, h from {1.5, 2, 3} mm, electrode count from {32, 64, 128, 256},
    5k-30k dipoles, dipoles in r < 0.848 * r_out."""
    rng = np.random.default_rng(seed)
    heads = []
    for b in range(n_heads):
        r_out = float(rng.uniform(*r_range))
        h = float(h_choices[int(rng.integers(len(h_choices)))])
        le = int(le_choices[int(rng.integers(len(le_choices)))])
        nd = int(rng.integers(dip_range[0], dip_range[1] + 1))
        spec = three_shell(h, le, nd, seed=1000 + b, r_out=r_out)
        spec.dipole_rmax = 0.848 * r_out
        spec.name = "batch%02d_h%gmm_R%.1fmm_L%d" % (b, h * 1e3, r_out * 1e3, le)
        heads.append(spec)
    return heads


# ---------------------------------------------------------------------------
# drawn inputs
# ---------------------------------------------------------------------------

def fibonacci_points(n: int, radius: float) -> np.ndarray:
    """n near-uniform points on the sphere of the given radius (golden-angle
    spiral): z_i = 1 - (2i+1)/n, phi_i = i*pi*(3 - sqrt(5))."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    return radius * np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def random_dipoles(n: int, rmax: float, seed: int):
    """Positions uniform in the ball r < rmax (r = rmax*u^(1/3), isotropic
    direction) and unit moments with isotropic direction."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rmax * rng.random(n) ** (1.0 / 3.0)
    pos = d * r[:, None]
    q = rng.standard_normal((n, 3))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return np.ascontiguousarray(pos), np.ascontiguousarray(q)


def conductivity(spec: HeadSpec, nodes: np.ndarray, tets: np.ndarray,
                 labels: np.ndarray) -> np.ndarray:
    """Per-element conductivity 6-tuples (s11, s22, s33, s12, s13, s23), the
    row layout of Sec. 2.1.2.  Isotropic per shell; with skull_aniso the skull
    tensor is s_t*I + (s_r - s_t) rr^T, r the unit vector to the element
    centroid."""
    m = tets.shape[0]
    sig = np.asarray(spec.sigma, dtype=np.float64)[labels]
    s6 = np.zeros((m, 6), dtype=np.float64)
    s6[:, 0] = sig
    s6[:, 1] = sig
    s6[:, 2] = sig
    if spec.skull_aniso is not None:
        sr, st = spec.skull_aniso
        sk = np.nonzero(labels == 1)[0]
        c = nodes[tets[sk]].mean(axis=1)
        r = c / np.linalg.norm(c, axis=1, keepdims=True)
        s6[sk, 0] = st + (sr - st) * r[:, 0] * r[:, 0]
        s6[sk, 1] = st + (sr - st) * r[:, 1] * r[:, 1]
        s6[sk, 2] = st + (sr - st) * r[:, 2] * r[:, 2]
        s6[sk, 3] = (sr - st) * r[:, 0] * r[:, 1]
        s6[sk, 4] = (sr - st) * r[:, 0] * r[:, 2]
        s6[sk, 5] = (sr - st) * r[:, 1] * r[:, 2]
    return s6


def electrode_inputs(spec: HeadSpec):
    """Electrode centres on the outer sphere, and per-electrode contact
    impedance (CEM) as arrays."""
    centres = fibonacci_points(spec.n_electrodes, spec.radii[-1])
    z = np.full(spec.n_electrodes, spec.contact_impedance, dtype=np.float64)
    return centres, z


def dipole_inputs(spec: HeadSpec):
    return random_dipoles(spec.n_dipoles, spec.dipole_rmax, spec.seed)


def injection_patterns(n_electrodes: int, amplitude: float = 1e-3) -> np.ndarray:
    """Adjacent-pair current patterns I_p = a*(e_p - e_{p+1}), p = 1..L-1,
    as a (L-1) x L array."""
    n = n_electrodes
    I = np.zeros((n - 1, n), dtype=np.float64)
    for p in range(n - 1):
        I[p, p] = amplitude
        I[p, p + 1] = -amplitude
    return I


def meg_sensors(n: int, radius: float, tilt: float = 0.6):
    """n magnetometers on the golden-angle spiral at the given radius, unit
    orientation radial + tilt * (a tangential direction), normalised.  The
    tilt gives every sensor a tangential component, which the volume
    currents of a spherical head do reach."""
    pos = fibonacci_points(n, radius)
    rhat = pos / np.linalg.norm(pos, axis=1, keepdims=True)
    ref = np.where(np.abs(rhat[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    t = np.cross(ref, rhat)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    d = rhat + tilt * t
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.ascontiguousarray(pos), np.ascontiguousarray(d)


def icosphere(level: int, radius: float = 1.0, centre=(0.0, 0.0, 0.0)):
    """Closed triangle surface of a sphere: the icosahedron with every
    triangle split into four `level` times, vertices projected to the sphere;
    triangles oriented outward.  Returns (verts (v,3), tris (t,3) int32)."""
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0), (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
         (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                mid[key] = len(verts) - 1
            return mid[key]
        nf = []
        for a, b, c in f:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    V = np.array(verts) * radius + np.asarray(centre, dtype=np.float64)
    T = np.array(f, dtype=np.int32)
    # outward orientation: the normal points away from the centre
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    flip = np.einsum("ij,ij->i", n, V[T].mean(axis=1) - np.asarray(centre)) < 0
    T[flip, 1], T[flip, 2] = T[flip, 2].copy(), T[flip, 1].copy()
    return V, T
