"""Pins of the IAS oracle (App. B) against mathematics it does not use itself:
the x-step equals the minimiser of the penalised least-squares problem (solved
in the source space), the theta-step is a stationary point of the hyperprior
objective, and the alternation never increases the objective."""
import numpy as np
import pytest

from oracle import ias as I


def problem(seed=0, Le=12, n=40, T=3):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((Le, n))
    x_true = np.zeros((n, T))
    x_true[rng.choice(n, 3, replace=False), :] = rng.standard_normal((3, T)) * 2.0
    Y = L @ x_true + 0.05 * rng.standard_normal((Le, T))
    return L, Y


def test_x_step_minimises_the_penalised_least_squares():
    L, Y = problem()
    rng = np.random.default_rng(3)
    theta = rng.uniform(0.1, 2.0, L.shape[1])
    nu = 0.3
    x = I.x_step(L, Y[:, 0], theta, nu)
    # normal equations in the source space: (L^T L / nu^2 + D^-1) x = L^T y / nu^2
    H = L.T @ L / nu ** 2 + np.diag(1.0 / theta)
    x_ref = np.linalg.solve(H, L.T @ Y[:, 0] / nu ** 2)
    assert np.allclose(x, x_ref, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("hyper", [I.HYPER_G, I.HYPER_IG])
def test_theta_step_is_stationary(hyper):
    rng = np.random.default_rng(5)
    x = rng.standard_normal(50) * 3.0
    theta0, beta = 0.7, 2.3
    th = I.theta_update(x, theta0, beta, hyper)
    assert np.all(th > 0)
    # d/dtheta of x^2/(2 theta) + log(theta)/2 + hyperprior term, by central differences
    def f(t):
        base = 0.5 * x * x / t + 0.5 * np.log(t)
        if hyper == I.HYPER_G:
            return base + t / theta0 - (beta - 1.0) * np.log(t)
        return base + theta0 / t + (beta + 1.0) * np.log(t)
    eps = 1e-6 * th
    grad = (f(th + eps) - f(th - eps)) / (2 * eps)
    scale = 0.5 * x * x / th ** 2 + 1.0 / th
    assert np.all(np.abs(grad) <= 1e-6 * scale)
    # and it is the minimum along theta
    assert np.all(f(th) <= f(th * 1.01)) and np.all(f(th) <= f(th * 0.99))


@pytest.mark.parametrize("hyper", [I.HYPER_G, I.HYPER_IG])
def test_alternation_never_increases_the_objective(hyper):
    L, Y = problem(seed=1)
    nu, theta0, beta = 0.05, 0.1, 1.8
    y = Y[:, 0]
    theta = np.full(L.shape[1], theta0)
    x = np.zeros(L.shape[1])
    f_prev = np.inf
    for _ in range(15):
        x = I.x_step(L, y, theta, nu)
        f_x = I.neg_log_posterior(L, y, x, theta, nu, theta0, beta, hyper)
        assert f_x <= f_prev * (1 + 1e-12) + 1e-12
        theta = I.theta_update(x, theta0, beta, hyper)
        f_t = I.neg_log_posterior(L, y, x, theta, nu, theta0, beta, hyper)
        assert f_t <= f_x * (1 + 1e-12) + 1e-12
        f_prev = f_t


def test_columns_are_independent_and_the_g_model_sparsifies():
    L, Y = problem(seed=2)
    X, TH = I.ias_map(L, Y, 0.05, 0.05, 1.6, I.HYPER_G, 25)
    for t in range(Y.shape[1]):
        x1, _ = I.ias_map(L, Y[:, t], 0.05, 0.05, 1.6, I.HYPER_G, 25)
        assert np.allclose(X[:, t], x1[:, 0], rtol=0, atol=0)
    # a gamma hypermodel with small eta concentrates the estimate on few sources
    share = np.sort(np.abs(X[:, 0]))[::-1]
    assert share[:6].sum() > 0.8 * share.sum()
