"""Pins of the oracle's mixture-of-Gaussians target (Sec. 7.3's NUTS workload: equicorrelated
unit-variance components, modes on the principal direction) and of NUTS on it.

* The log-density equals the mixture written with scipy's multivariate normal (explicit
  covariance matrix, its own factorisation), up to the common Gaussian normaliser the target
  drops; several correlations, including a negative one.
* The gradient equals central finite differences of the log-density.
* One component with rho = 0 is the standard normal around its mean.
* NUTS started from exact draws of the paper's 100-d target keeps the mode occupancies and the
  within-mode moments (exact-start stationarity), and its trajectory lengths show the paper's
  heavy tail at the chosen step size.
"""
import math

import numpy as np
import pytest
from scipy.special import logsumexp
from scipy.stats import multivariate_normal

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W


def _mixture(d, K, rho, seed):
    r = np.random.default_rng(seed)
    w = r.uniform(0.2, 2.0, K)
    mu = r.normal(0.0, 2.0, (K, d))
    return np.concatenate([[rho], w, mu.ravel()]), w, mu


@pytest.mark.parametrize("rho", [0.0, 0.6, -0.2, 0.95])
def test_logp_matches_scipy_mixture(rho):
    d, K = 5, 3
    params, w, mu = _mixture(d, K, rho, 3)
    S = (1 - rho) * np.eye(d) + rho * np.ones((d, d))
    norm = -0.5 * d * math.log(2 * math.pi) - 0.5 * np.linalg.slogdet(S)[1]
    r = np.random.default_rng(4)
    for _ in range(20):
        x = r.normal(0.0, 3.0, d)
        ref = logsumexp([math.log(w[k]) + multivariate_normal(mu[k], S).logpdf(x) for k in range(K)]) - norm
        got = O.logp("mog", params, x, n_data=K)
        assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref))


@pytest.mark.parametrize("rho", [0.3, 0.99])
def test_gradient_matches_finite_differences(rho):
    d, K = 7, 3
    params, _, _ = _mixture(d, K, rho, 5)
    r = np.random.default_rng(6)
    for _ in range(5):
        x = r.normal(0.0, 2.0, d)
        _, g = O.logp("mog", params, x, n_data=K, grad=True)
        h = 1e-6
        fd = np.array([(O.logp("mog", params, x + h * e, n_data=K) - O.logp("mog", params, x - h * e, n_data=K))
                       / (2 * h) for e in np.eye(d)])
        assert np.max(np.abs(g - fd)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_one_uncorrelated_component_is_the_standard_normal():
    d = 9
    mu = np.arange(d, dtype=np.float64) * 0.3
    params = np.concatenate([[0.0], [2.5], mu])
    x = np.random.default_rng(7).normal(size=d)
    v, g = O.logp("mog", params, x, n_data=1, grad=True)
    assert abs(v - (math.log(2.5) - 0.5 * np.sum((x - mu) ** 2))) < 1e-13
    assert np.max(np.abs(g + (x - mu))) < 1e-14


def test_nuts_keeps_the_papers_mixture_stationary():
    # d = 100, rho = 0.99, modes at -10 * 1, 0, 10 * 1 (equal weights), eps = 0.044, depth <= 10
    w = W.mog(100)
    m = 3000
    x0 = W.x0_mog_exact(w, m)
    r = O.run("nuts", "mog", w["params"], x0, 3, seed=2, n_data=3, algo_params=[0.044, 10, 1000.0],
              store=False)
    x = r["x_final"]
    xbar = x.mean(1)
    mode = np.argmin(np.abs(xbar[:, None] - np.array([-10.0, 0.0, 10.0])[None, :]), axis=1)
    frac = np.bincount(mode, minlength=3) / m
    assert np.all(np.abs(frac - 1 / 3) < 4 * math.sqrt((1 / 3) * (2 / 3) / m))
    # within a mode: the coordinate mean has variance rho + (1 - rho) / d, the residuals about
    # it have mean square (1 - rho) (d - 1) / d per coordinate
    off = xbar - np.array([-10.0, 0.0, 10.0])[mode]
    v_par = 0.99 + 0.01 / 100
    assert abs(off.var() - v_par) < 4 * v_par * math.sqrt(2.0 / m)
    res = ((x - xbar[:, None]) ** 2).sum(1) / 99      # (1 - rho) chi2_99 / 99 per chain
    assert abs(res.mean() - 0.01) < 4 * 0.01 * math.sqrt(2.0 / 99 / m)
    # trajectory lengths: mostly short, a tail reaching the depth cap
    c = r["counts"].ravel()
    assert np.mean(c < 20) > 0.8 and c.max() >= 1000
