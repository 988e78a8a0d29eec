"""Pins of the oracle's elliptical slice sampler (appendix Alg. 8).

Conjugate-Gaussian closed form, the flat-likelihood special case, and the
bracket invariant.  Chains start from exact posterior draws, so the samples at
every step are i.i.d. across chains and the Monte Carlo standard error is plain
sd/sqrt(m).
"""
import numpy as np
from scipy import stats

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W


def _chi2_check(x, mean, cov, label):
    # (x - mu)^T C^-1 (x - mu) ~ chi^2_d; its mean over m i.i.d. rows is d +- sqrt(2d/m)
    d = mean.size
    Ci = np.linalg.inv(cov)
    r = x - mean
    q = np.einsum("ij,jk,ik->i", r, Ci, r)
    m = x.shape[0]
    assert abs(q.mean() - d) < 4 * np.sqrt(2 * d / m), (label, q.mean())
    return q


def test_conjugate_gaussian_exact_start_moments():
    w = W.gauss_conj(d=16)
    m, n = 2048, 40
    x0 = W.x0_gauss_posterior(w, m)
    r = O.run("ess", "gauss_conj", w["params"], x0, n, seed=1)
    sd = np.sqrt(np.diag(w["post_cov"]))
    for i in (0, 9, 39):
        xi = r["samples"][:, i, :]
        # per-dimension mean within 4 standard errors
        assert np.all(np.abs(xi.mean(0) - w["post_mean"]) < 4 * sd / np.sqrt(m)), i
        _chi2_check(xi, w["post_mean"], w["post_cov"], i)
    # the chains move: a sample differs from its predecessor
    assert np.mean(np.all(r["samples"][:, 1:] == r["samples"][:, :-1], axis=2)) < 1e-3
    assert r["counts"].min() >= 0


def test_conjugate_gaussian_long_run_moments():
    # 128 chains x 1000 samples from x0 = 0, first 10 % discarded; batch-means MCSE
    w = W.gauss_conj(d=16)
    m, n = 128, 1000
    r = O.run("ess", "gauss_conj", w["params"], W.x0_zeros(m, 16), n, seed=1)
    kept = r["samples"][:, n // 10:, :]
    chain_means = kept.mean(1)                       # (m, d): one batch per chain
    mcse = chain_means.std(0, ddof=1) / np.sqrt(m)
    assert np.all(np.abs(chain_means.mean(0) - w["post_mean"]) < 4 * mcse)
    var = kept.reshape(-1, 16).var(0)
    assert np.all(np.abs(var / np.diag(w["post_cov"]) - 1) < 0.1)


def test_flat_likelihood_never_shrinks_and_keeps_prior():
    # f == 1: the first proposal is always accepted (N = 0) and the chain is the
    # prior-preserving rotation x cos(theta) + nu sin(theta): exact N(0, Sigma) draws
    w = W.flat(d=8)
    Sigma = w["L"] @ w["L"].T
    m = 4000
    x0 = W.x0_normal(m, 8) @ w["L"].T
    r = O.run("ess", "flat", w["params"], x0, 5, seed=3)
    assert np.all(r["counts"] == 0)
    for i in range(5):
        _chi2_check(r["samples"][:, i], np.zeros(8), Sigma, i)
    # x' is a rotation in the (x, nu) plane: with nu from an independent draw the
    # sample is not equal to x, and successive samples are correlated like
    # cos(theta) with theta ~ U(0, 2 pi): E[x' x^T] = E[cos theta] Sigma = 0
    c = (r["samples"][:, 1] * r["samples"][:, 0]).sum(0) / m
    assert np.all(np.abs(c) < 6 * np.diag(Sigma) / np.sqrt(m))


def test_bracket_invariant_and_shrinking():
    # after every shrink: theta_min <= 0 <= theta_max, theta in the bracket, and the
    # bracket strictly narrows (Alg. 8 shrink step)
    w = W.gp_logit(d=32)
    x = np.zeros(32)
    lp = O.logp("gp_logit", w["params"], x)
    total = 0
    for i in range(300):
        x_new, n, tr = O.ess_trace("gp_logit", w["params"], x, seed=4, chain=0, sample=i)
        total += n
        widths = tr[:, 2] - tr[:, 1]
        assert np.all(tr[:, 1] <= 0) and np.all(tr[:, 2] >= 0)
        assert np.all(tr[:, 1] <= tr[:, 0]) and np.all(tr[:, 0] <= tr[:, 2])
        assert np.all(np.diff(widths) < 0)
        assert np.all(widths <= 2 * np.pi)
        lp_new = O.logp("gp_logit", w["params"], x_new)
        x = x_new
        lp = lp_new
    assert total > 100  # the invariant was exercised


def test_likelihood_special_values():
    # log f at the data: Gaussian likelihood is 0 at x = y; the logistic
    # likelihood at x = 0 is -d log 2
    w = W.gauss_conj(d=16)
    assert O.logp("gauss_conj", w["params"], w["y"]) == 0.0
    g = W.gp_logit(d=64)
    assert abs(O.logp("gp_logit", g["params"], np.zeros(64)) + 64 * np.log(2)) < 1e-12
    # large |x| does not overflow the softplus
    v = O.logp("gp_logit", g["params"], 800 * g["s"])
    assert np.isfinite(v) and v <= 0 and abs(v) < 1e-300
    v = O.logp("gp_logit", g["params"], -800 * g["s"])
    assert abs(v + 800 * 64) < 1e-9


def test_runs_are_deterministic_and_chain_keyed():
    w = W.gauss_conj(d=16)
    x0 = W.x0_zeros(6, 16)
    a = O.run("ess", "gauss_conj", w["params"], x0, 20, seed=1, n_threads=1)
    b = O.run("ess", "gauss_conj", w["params"], x0, 20, seed=1, n_threads=3)
    assert np.array_equal(a["samples"], b["samples"])
    # chain j of a run started at chain0 = 2 equals chain 2 + j of the full run
    c = O.run("ess", "gauss_conj", w["params"], x0[2:], 20, seed=1, chain0=2)
    assert np.array_equal(c["samples"], a["samples"][2:])
