"""Plain FP64 CPU oracle of the IAS MAP inversion (App. B of the paper).

TEST INFRASTRUCTURE ONLY: the definition the CUDA path of zi_ias_map is
checked against.  Only the test suite and the benchmark's CPU leg import it;
it shares no code with the CUDA library.

The iterative alternating sequential (IAS) scheme alternates between the two
conditional maximisers of the posterior:

  x-step  x = D_theta L^T (L D_theta L^T + nu^2 I)^-1 y,   D_theta = diag(theta)
          (the paper writes L_k = L D^{1/2} and x = D^{1/2} L_k^T (L_k L_k^T +
          nu^2 I)^-1 y; theta > 0 in both hypermodels, so D^{1/2} D^{1/2} = D);
  theta-step, per source i:
          gamma hypermodel (G):          theta_i = theta0/2 (eta + sqrt(eta^2 + 2 x_i^2 / theta0)),
                                         eta = beta - 3/2;
          inverse-gamma hypermodel (IG): theta_i = (theta0 + x_i^2 / 2) / kappa, kappa = beta + 3/2;

starting from theta = (theta0, ..., theta0), for a fixed number of rounds.
Each data column y (a time sample) is inverted independently with its own
theta.  A library dense solve serves as the step (L D L^T + nu^2 I)^-1 y.
"""
from __future__ import annotations

import numpy as np

HYPER_G = 0
HYPER_IG = 1


def theta_update(x, theta0, beta, hyper):
    """The theta-step of App. B, elementwise."""
    x2 = np.asarray(x, dtype=np.float64) ** 2
    if hyper == HYPER_G:
        eta = beta - 1.5
        return 0.5 * theta0 * (eta + np.sqrt(eta * eta + 2.0 * x2 / theta0))
    if hyper == HYPER_IG:
        kappa = beta + 1.5
        return (theta0 + 0.5 * x2) / kappa
    raise ValueError("hypermodel must be HYPER_G or HYPER_IG")


def x_step(L, y, theta, nu):
    """x = D L^T (L D L^T + nu^2 I)^-1 y for one data column."""
    M = (L * theta[None, :]) @ L.T + nu * nu * np.eye(L.shape[0])
    z = np.linalg.solve(M, y)
    return theta * (L.T @ z)


def ias_map(L, Y, nu, theta0, beta, hyper, iters):
    """IAS MAP estimates for every column of Y (Le x T): returns x (n x T)
    and theta (n x T) after `iters` rounds (each round an x-step from the
    current theta, then a theta-step from that x)."""
    L = np.asarray(L, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    n = L.shape[1]
    X = np.zeros((n, Y.shape[1]))
    TH = np.full((n, Y.shape[1]), float(theta0))
    for t in range(Y.shape[1]):
        theta = TH[:, t].copy()
        x = np.zeros(n)
        for _ in range(iters):
            x = x_step(L, Y[:, t], theta, nu)
            theta = theta_update(x, theta0, beta, hyper)
        X[:, t] = x
        TH[:, t] = theta
    return X, TH


def neg_log_posterior(L, y, x, theta, nu, theta0, beta, hyper):
    """The function IAS minimises alternately (up to constants): the Gaussian
    likelihood, the conditionally Gaussian prior x_i ~ N(0, theta_i) and the
    hyperprior of theta_i, G (a gamma density) or IG (an inverse-gamma one)."""
    r = y - L @ x
    f = 0.5 * (r @ r) / (nu * nu) + np.sum(0.5 * x * x / theta + 0.5 * np.log(theta))
    if hyper == HYPER_G:
        f += np.sum(theta / theta0 - (beta - 1.0) * np.log(theta))
    else:
        f += np.sum(theta0 / theta + (beta + 1.0) * np.log(theta))
    return float(f)
