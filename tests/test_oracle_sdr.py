"""Pins of the oracle's symmetric delayed rejection (re-centred tries, Mira 2001; the sampler of
Sec. 7.1's toy experiment): exact detailed balance of the enumerated M-try transition on a
discrete ring, stationarity of N(0, 1) and of a diagonal Gaussian from exact starts with the
paper's settings (M = 100 tries, proposal sd 0.1), and the one-try case reducing to the
random-walk Metropolis step of the 3-stage sampler."""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W


def _ring_transition(logpi, M):
    """Transition matrix of symmetric DR on a ring: every try moves the last rejected point
    (initially x) by +-1 with probability 1/2 each; try k is accepted with the oracle's
    alpha_k(x, pi*, y_k); after M rejections the chain stays."""
    R = len(logpi)
    P = np.zeros((R, R))
    for x in range(R):
        for steps in itertools.product((-1, 1), repeat=M):
            w = 0.5 ** M           # probability of this proposal sequence
            centre, lp_star, stay = x, -math.inf, 1.0
            for k, st in enumerate(steps):
                y = (centre + st) % R
                a = math.exp(O.sdr_log_alpha(logpi[x], lp_star, logpi[y]))
                P[x, y] += w * stay * a
                stay *= 1.0 - a
                lp_star = max(lp_star, logpi[y])
                centre = y
            P[x, x] += w * stay
    return P


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_symmetric_dr_detailed_balance_on_ring(M):
    rng = np.random.default_rng(7)
    pi = rng.uniform(0.05, 1.0, size=7)
    pi /= pi.sum()
    logpi = np.log(pi)
    P = _ring_transition(logpi, M)
    assert np.allclose(P.sum(1), 1.0, atol=1e-13)
    flux = pi[:, None] * P
    assert np.max(np.abs(flux - flux.T)) < 1e-13
    assert np.allclose(pi @ P, pi, atol=1e-13)
    if M >= 2:  # later tries add moves: more probability leaves each state than with one try
        assert np.all(np.diag(P) < np.diag(_ring_transition(logpi, 1)) + 1e-15)


def test_a_wrong_acceptance_breaks_the_ring_balance():
    # the same enumeration with the un-telescoped ratio pi(y) / pi(x) at every try (a plausible
    # mistake) is not reversible: the pin above detects the formula, not just any DR
    rng = np.random.default_rng(7)
    pi = rng.uniform(0.05, 1.0, size=7)
    pi /= pi.sum()
    logpi = np.log(pi)
    R, M = 7, 3
    P = np.zeros((R, R))
    for x in range(R):
        for steps in itertools.product((-1, 1), repeat=M):
            w, centre, stay = 0.5 ** M, x, 1.0
            for st in steps:
                y = (centre + st) % R
                a = min(1.0, math.exp(logpi[y] - logpi[x]))
                P[x, y] += w * stay * a
                stay *= 1.0 - a
                centre = y
            P[x, x] += w * stay
    flux = pi[:, None] * P
    assert np.max(np.abs(flux - flux.T)) > 1e-4


def test_one_try_is_the_random_walk_metropolis_step_of_the_staged_sampler():
    # symmetric DR with M = 1 and the 3-stage sampler with one stage both make one x-centred
    # Gaussian proposal from the same draws and accept with min(1, pi(y)/pi(x))
    w = W.gauss_diag(4)
    x0 = W.x0_gauss_diag_exact(w, 64)
    a = O.run("sdr", "gauss_diag", w["params"], x0, 50, seed=3, algo_params=[1, 0.7])
    b = O.run("dr", "gauss_diag", w["params"], x0, 50, seed=3, algo_params=[1, 0.7, 1.0])
    assert np.array_equal(a["samples"], b["samples"])
    assert np.array_equal(a["counts"], b["counts"])


def test_paper_setting_keeps_standard_normal_stationary():
    # N(0, 1), M = 100 tries of sd 0.1 (Sec. 7.1), 200k chains from exact draws, 3 transitions:
    # the cross-chain moments stay those of N(0, 1) (i.i.d. over chains: MCSE = sd / sqrt(m))
    m = 200_000
    w = {"params": np.array([0.0, 1.0])}
    x0 = np.random.default_rng(11).standard_normal((m, 1))
    r = O.run("sdr", "gauss_diag", w["params"], x0, 3, seed=9, algo_params=[100, 0.1], store=False)
    x = r["x_final"][:, 0]
    assert abs(x.mean()) < 4 / math.sqrt(m)
    assert abs(x.var() - 1.0) < 4 * math.sqrt(2.0 / m)
    assert abs(np.mean(x ** 4) - 3.0) < 4 * math.sqrt(96.0 / m)
    # tries are used: the proposal is small, so most samples accept early but some need many
    assert r["counts"].max() > 5 and r["counts"].min() >= 1


def test_diagonal_gaussian_stationary_with_many_tries():
    w = W.gauss_diag(3)
    m = 100_000
    x0 = W.x0_gauss_diag_exact(w, m)
    r = O.run("sdr", "gauss_diag", w["params"], x0, 2, seed=4, algo_params=[20, 0.5], store=False)
    mu, sd = w["params"][:3], w["params"][3:]
    z = (r["x_final"] - mu) / sd
    assert np.all(np.abs(z.mean(0)) < 4 / math.sqrt(m))
    assert np.all(np.abs(z.var(0) - 1.0) < 4 * math.sqrt(2.0 / m))
