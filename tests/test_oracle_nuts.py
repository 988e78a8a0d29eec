"""Pins of the oracle's multinomial NUTS and its leapfrog integrator.

* Leapfrog on a Gaussian target is a linear map with a closed form (the
  discretised harmonic oscillator); compared to 1e-13.
* Leapfrog is reversible: L steps, flip p, L steps returns to the start.
* Exact-start stationarity on N(mu, diag sigma^2): moments at steps 1 and 10,
  and a million-draw 1-D check of the variance and fourth moment.
* Logistic-regression density and gradient special values; the NUTS posterior
  itself on logistic regression has no closed form (parity unpinned there).
"""
import numpy as np

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W


def _leapfrog_matrix(eps, omega2):
    a = eps * eps * omega2
    return np.array([[1 - a / 2, eps], [-eps * omega2 * (1 - a / 4), 1 - a / 2]])


def test_leapfrog_matches_harmonic_oscillator_closed_form():
    w = W.gauss_diag(d=6)
    rng = np.random.default_rng(0)
    x0 = rng.standard_normal(6)
    p0 = rng.standard_normal(6)
    for eps, n in [(0.1, 1), (0.05, 37), (0.3, 200)]:
        x, p = O.leapfrog("gauss_diag", w["params"], x0, p0, eps, n)
        for k in range(6):
            M = np.linalg.matrix_power(_leapfrog_matrix(eps, 1 / w["sd"][k] ** 2), n)
            ex = M @ np.array([x0[k] - w["mu"][k], p0[k]])
            assert abs(x[k] - w["mu"][k] - ex[0]) < 1e-13 * max(1, n / 10)
            assert abs(p[k] - ex[1]) < 1e-13 * max(1, n / 10)


def test_leapfrog_reversibility_logreg():
    w = W.logreg(n=200, d=5)
    rng = np.random.default_rng(1)
    x0 = w["beta_true"] + 0.1 * rng.standard_normal(5)
    p0 = rng.standard_normal(5)
    L = 64
    x, p = O.leapfrog("logreg", w["params"], x0, p0, 0.01, L, n_data=200)
    xb, pb = O.leapfrog("logreg", w["params"], x, -p, 0.01, L, n_data=200)
    assert np.max(np.abs(xb - x0)) < 1e-12 * L
    assert np.max(np.abs(-pb - p0)) < 1e-12 * L * 100


def test_logreg_density_special_values():
    w = W.logreg(n=300, d=7)
    v, g = O.logp("logreg", w["params"], np.zeros(7), n_data=300, grad=True)
    assert abs(v + 300 * np.log(2)) < 1e-9
    assert np.allclose(g, w["X"].T @ (w["y"] - 0.5), atol=1e-10)
    rng = np.random.default_rng(2)
    b = rng.standard_normal(7)
    v, g = O.logp("logreg", w["params"], b, n_data=300, grad=True)
    h = 1e-6
    num = np.array([(O.logp("logreg", w["params"], b + h * e, n_data=300)
                     - O.logp("logreg", w["params"], b - h * e, n_data=300)) / (2 * h)
                    for e in np.eye(7)])
    assert np.allclose(num, g, rtol=1e-6, atol=1e-5)


def test_gauss_diag_exact_start_moments():
    w = W.gauss_diag(d=8)
    m = 3000
    x0 = W.x0_gauss_diag_exact(w, m)
    r = O.run("nuts", "gauss_diag", w["params"], x0, 10, seed=2, algo_params=[0.2, 10, 1000.0])
    for i in (0, 9):
        x = r["samples"][:, i, :]
        z = (x - w["mu"]) / w["sd"]
        assert np.all(np.abs(z.mean(0)) < 4 / np.sqrt(m))
        assert np.all(np.abs(z.var(0) - 1) < 4 * np.sqrt(2 / m))
        q = (z ** 2).sum(1)
        assert abs(q.mean() - 8) < 4 * np.sqrt(16 / m)
    c, depth = r["counts"], r["aux"]
    assert c.min() >= 1 and c.max() <= 1023
    assert np.all(c <= 2 ** depth - 1)
    assert depth.max() <= 10 and depth.min() >= 1


def test_one_dimensional_invariance_million_draws():
    # a coarse step (eps = 0.9) makes the multinomial / progressive choices matter
    params = np.array([0.0, 1.0])
    m = 400_000
    x0 = np.random.default_rng(3).standard_normal((m, 1))
    r = O.run("nuts", "gauss_diag", params, x0, 1, seed=5, algo_params=[0.9, 10, 1000.0])
    x = r["samples"][:, 0, 0]
    assert abs(x.mean()) < 4 / np.sqrt(m)
    assert abs(x.var() - 1) < 4 * np.sqrt(2 / m)
    assert abs((x ** 4).mean() - 3) < 4 * np.sqrt(96 / m)
    assert (x != x0[:, 0]).mean() > 0.9


def test_divergence_ends_the_transition():
    # a huge step on a stiff Gaussian diverges immediately: the first subtree is
    # discarded and the chain stays put after one leapfrog
    params = np.array([0.0, 0.01])
    x0 = np.zeros((4, 1))
    r = O.run("nuts", "gauss_diag", params, x0, 3, seed=1, algo_params=[50.0, 10, 1000.0])
    assert np.all(r["samples"] == 0.0)
    assert np.all(r["counts"] == 1) and np.all(r["aux"] == 1)


def test_logreg_short_run_deterministic():
    w = W.logreg(n=1000, d=25)
    x0 = W.x0_logreg(w, 4)
    a = O.run("nuts", "logreg", w["params"], x0, 5, seed=1, n_data=1000,
              algo_params=[0.05, 10, 1000.0], n_threads=1)
    b = O.run("nuts", "logreg", w["params"], x0, 5, seed=1, n_data=1000,
              algo_params=[0.05, 10, 1000.0], n_threads=2)
    assert np.array_equal(a["samples"], b["samples"])
    assert a["counts"].min() >= 1


def test_nuts_logreg_posterior_matches_importance_sampling():
    # Logistic regression has no closed-form posterior, so the oracle's NUTS (the configuration's
    # eps = 0.05, depth <= 10) is checked against a different estimator of the same posterior
    # expectations: self-normalised importance sampling from a multivariate t (10 degrees of
    # freedom) centred at the posterior mode with the Laplace covariance H^-1 widened by 1.2^2,
    # H = X^T W X + I, W = diag(s (1 - s)), s = sigmoid(X beta_MAP).  The mode comes from Newton's
    # method on the oracle's log density and gradient; the importance weights use the log
    # posterior written with numpy.  NUTS chain means and second moments must agree with the
    # importance-sampling estimates within 4 combined Monte Carlo standard errors (the posterior
    # is visibly skewed here, its mean up to ~0.5 sd from the mode, so the mode itself is no pin).
    w = W.logreg(1000, 25)
    X, y = w["X"], w["y"]
    b = np.zeros(25)
    for _ in range(30):
        _, g = O.logp("logreg", w["params"], b, n_data=1000, grad=True)
        s = 1.0 / (1.0 + np.exp(-(X @ b)))
        H = X.T @ (X * (s * (1 - s))[:, None]) + np.eye(25)
        b = b + np.linalg.solve(H, g)
    _, g = O.logp("logreg", w["params"], b, n_data=1000, grad=True)
    assert np.abs(g).max() < 1e-9
    s = 1.0 / (1.0 + np.exp(-(X @ b)))
    H = X.T @ (X * (s * (1 - s))[:, None]) + np.eye(25)
    C = np.linalg.cholesky(np.linalg.inv(H) * 1.2 ** 2)
    rng = np.random.default_rng(17)
    N, nu = 200_000, 10.0
    zt = rng.standard_normal((N, 25)) / np.sqrt(rng.chisquare(nu, (N, 1)) / nu)
    beta = b + zt @ C.T
    eta = beta @ X.T
    logpost = eta @ y - np.logaddexp(0.0, eta).sum(1) - 0.5 * (beta ** 2).sum(1)
    logq = -0.5 * (nu + 25) * np.log1p((zt ** 2).sum(1) / nu)
    lw = logpost - logq
    wt = np.exp(lw - lw.max())
    wt /= wt.sum()
    assert 1.0 / (wt ** 2).sum() > 0.1 * N          # the proposal covers the posterior
    f = np.concatenate([beta, beta ** 2], axis=1)
    is_mean = wt @ f
    is_se = np.sqrt((wt[:, None] ** 2 * (f - is_mean) ** 2).sum(0))
    m, n, burn = 48, 250, 50
    r = O.run("nuts", "logreg", w["params"], W.x0_logreg(w, m), n, seed=3, n_data=1000,
              algo_params=[0.05, 10, 1000.0])
    xs = r["samples"][:, burn:, :]
    cm = np.concatenate([xs.mean(1), (xs ** 2).mean(1)], axis=1)
    mean, mcse = cm.mean(0), cm.std(0, ddof=1) / np.sqrt(m)
    z = np.abs(mean - is_mean) / np.sqrt(mcse ** 2 + is_se ** 2)
    assert z.max() <= 4.0, z
