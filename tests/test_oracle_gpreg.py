"""Pins of the oracle's GP-regression hyperparameter likelihood (Sec. 7.2: ESS over (sigma, tau,
lambda) with N(0, I) priors): the marginal likelihood equals scipy's multivariate normal density
with the explicit covariance; lambda = 0 has a closed form (Sherman-Morrison / matrix
determinant lemma); signs of the hyperparameters do not matter; a singular covariance gives
-inf; and ESS on it moves the chains while keeping the likelihood finite."""
import math

import numpy as np
import pytest
from scipy.stats import multivariate_normal

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W


@pytest.mark.parametrize("n", [25, 100])
def test_likelihood_matches_scipy(n):
    w = W.gp_reg(n)
    r = np.random.default_rng(5)
    for _ in range(12):
        th = r.normal(0.0, 1.0, 3)
        C = th[1] ** 2 * np.exp(-th[2] ** 2 * w["D"]) + th[0] ** 2 * np.eye(n)
        ref = multivariate_normal(np.zeros(n), C, allow_singular=False).logpdf(w["y"])
        got = O.logp("gp_reg", w["params"], th, n_data=n)
        assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref))


def test_lambda_zero_closed_form():
    # C = tau^2 1 1^T + sigma^2 I: det = sigma^(2(n-1)) (sigma^2 + n tau^2),
    # y^T C^-1 y = (|y|^2 - tau^2 (1^T y)^2 / (sigma^2 + n tau^2)) / sigma^2
    n = 40
    w = W.gp_reg(n)
    y = w["y"]
    for s, t in [(0.5, 1.2), (1.5, 0.3)]:
        s2, t2 = s * s, t * t
        logdet = (n - 1) * math.log(s2) + math.log(s2 + n * t2)
        quad = (y @ y - t2 * y.sum() ** 2 / (s2 + n * t2)) / s2
        ref = -0.5 * quad - 0.5 * logdet - 0.5 * n * math.log(2 * math.pi)
        got = O.logp("gp_reg", w["params"], np.array([s, t, 0.0]), n_data=n)
        assert abs(got - ref) < 1e-10 * abs(ref)


def test_signs_do_not_matter_and_singular_covariance_is_minus_infinity():
    n = 25
    w = W.gp_reg(n)
    th = np.array([0.3, 0.8, 0.6])
    v = O.logp("gp_reg", w["params"], th, n_data=n)
    for sg in ([-1, 1, 1], [1, -1, 1], [1, 1, -1], [-1, -1, -1]):
        assert O.logp("gp_reg", w["params"], th * np.array(sg), n_data=n) == v
    assert O.logp("gp_reg", w["params"], np.array([0.0, 1.0, 0.0]), n_data=n) == -math.inf


def test_ess_moves_the_hyperparameters():
    w = W.gp_reg(25)
    x0 = W.x0_gp_reg(w, 16)
    r = O.run("ess", "gp_reg", w["params"], x0, 30, seed=2, n_data=25)
    assert np.all(np.isfinite(r["samples"]))
    assert np.mean(np.abs(np.diff(r["samples"], axis=1)) > 0) > 0.9
    assert r["counts"].max() > 3 * max(1.0, np.median(r["counts"]))
