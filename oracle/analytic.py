"""Analytic potential of a current dipole in a homogeneous insulated ball.

TEST INFRASTRUCTURE ONLY (part of the oracle; see zi_oracle.py's header).

Derived from the governing equation div(sigma grad u) = div J^p of Sec. 2
with J^p = q delta(r - r0) and the no-flux condition of the complete electrode
model's first boundary condition (App. A.1, (I)) on the whole sphere:

  u = u_inf + u_c,
  u_inf(r) = q.(r - r0) / (4 pi sigma |r - r0|^3),
  u_c(r)   = 1/(4 pi sigma) q . grad_{r0} sum_{n>=1} (n+1)/n * |r0|^n |r|^n / R^(2n+1)
                                                 * P_n(rhat . r0hat),

the image term chosen mode by mode so that du/dr = 0 at |r| = R (expand
1/|r - r0| in Legendre polynomials; each exterior mode |r0|^n/|r|^(n+1) gets
the interior partner with matching radial derivative).  Valid for
|r| < R^2/|r0|.  grad_{r0}[rho^n P_n(c)] = n rho^(n-1) P_n(c) r0hat
+ rho^(n-1) P_n'(c) (rhat - c r0hat), with Bonnet's recurrence for P_n and
P'_{n+1} = P'_{n-1} + (2n+1) P_n for the derivatives.
"""
from __future__ import annotations

import math

import numpy as np


def sphere_dipole_potential(r, r0, q, sigma: float, R: float, nterms: int = 400) -> np.ndarray:
    """Potential at points r (k,3) of a dipole q (3,) at r0 (3,) in a ball of
    radius R and conductivity sigma with an insulating surface."""
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    r0 = np.asarray(r0, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    d = r - r0
    dn = np.linalg.norm(d, axis=1)
    u_inf = (d @ q) / (4.0 * math.pi * sigma * dn ** 3)

    rn = np.linalg.norm(r, axis=1)
    rho0 = float(np.linalg.norm(r0))
    rhat = r / np.where(rn > 0, rn, 1.0)[:, None]
    if rho0 < 1e-300:
        # only the n = 1 mode survives: 2 |r| (q.rhat) / R^3
        u_c = 2.0 * rn * (rhat @ q) / R ** 3
        return u_inf + u_c / (4.0 * math.pi * sigma)
    r0hat = r0 / rho0
    c = np.clip(rhat @ r0hat, -1.0, 1.0)
    q_r0 = float(q @ r0hat)
    q_r = rhat @ q
    # Legendre recurrences
    P_prev = np.ones_like(c)      # P_0
    P_cur = c.copy()              # P_1
    dP_prev = np.zeros_like(c)    # P_0'
    dP_cur = np.ones_like(c)      # P_1'
    u_c = np.zeros_like(c)
    x = rn * rho0 / (R * R)       # geometric ratio of the series
    scale = np.ones_like(c)       # (|r| rho0 / R^2)^(n-1)
    for n in range(1, nterms + 1):
        # term: (n+1)/n * |r|^n / R^(2n+1) * rho0^(n-1) * [n P_n q.r0hat + P_n' (q.rhat - c q.r0hat)]
        coef = (n + 1.0) / n * (rn / (R ** 3)) * scale
        u_c += coef * (n * P_cur * q_r0 + dP_cur * (q_r - c * q_r0))
        # advance to n+1
        P_next = ((2 * n + 1) * c * P_cur - n * P_prev) / (n + 1)
        dP_next = dP_prev + (2 * n + 1) * P_cur
        P_prev, P_cur = P_cur, P_next
        dP_prev, dP_cur = dP_cur, dP_next
        scale = scale * x
    return u_inf + u_c / (4.0 * math.pi * sigma)


MU0_OVER_4PI = 1e-7  # T m / A


def sarvas_field(r, r0, q) -> np.ndarray:
    """Magnetic field outside a spherically symmetric conductor centred at the
    origin, at points r (k,3), of a current dipole q (3,) at r0 (3,) inside it
    (Sarvas' closed form, which follows from B = -mu0 grad U outside the
    conductor and the radial component being that of the primary current
    alone):
        a = r - r0,  F = |a| (|r||a| + |r|^2 - r0.r),
        grad F = (|a|^2/|r| + a.r/|a| + 2|a| + 2|r|) r - (|a| + 2|r| + a.r/|a|) r0,
        B = mu0/(4 pi F^2) (F q x r0 - ((q x r0).r) grad F).
    Independent of the radial conductivity profile."""
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    r0 = np.asarray(r0, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    a = r - r0
    an = np.linalg.norm(a, axis=1)
    rn = np.linalg.norm(r, axis=1)
    ar = np.sum(a * r, axis=1)
    F = an * (rn * an + rn * rn - r @ r0)
    gF = ((an * an / rn + ar / an + 2.0 * an + 2.0 * rn)[:, None] * r
          - (an + 2.0 * rn + ar / an)[:, None] * r0[None, :])
    qx = np.cross(q, r0)
    return MU0_OVER_4PI / (F * F)[:, None] * (F[:, None] * qx[None, :] - (r @ qx)[:, None] * gF)


def primary_field(r, r0, q) -> np.ndarray:
    """Biot-Savart field of the primary current alone, mu0/(4 pi) q x (r - r0)/|r - r0|^3."""
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    a = r - np.asarray(r0, dtype=np.float64)
    return MU0_OVER_4PI * np.cross(np.asarray(q, dtype=np.float64), a) / np.linalg.norm(a, axis=1)[:, None] ** 3
