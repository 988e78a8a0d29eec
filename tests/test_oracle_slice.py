"""Pins of the oracle's slice sampler (Neal 2003 stepping-out and shrinkage on a random line;
Fig. 2's two-loop FSM): exact loop counts on a flat target, the triangular step law of the
no-expansion case, and exact-start stationarity on a diagonal Gaussian, the funnel and a
two-mode mixture."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W

FLAT = np.array([0.0, 1e9])   # N(0, 1e18) in one dimension: log pi is constant to ~1e-16


def test_flat_target_uses_every_expansion_step_and_accepts_the_first_proposal():
    # every end is inside the slice, so the left and right loops take all m - 1 steps
    # between them and the first proposal is accepted: N = m evaluations, one proposal
    x0 = np.zeros((500, 1))
    for m in (1, 2, 7, 50):
        r = O.run("slice", "gauss_diag", FLAT, x0, 4, seed=2, algo_params=[1.5, m])
        assert np.all(r["counts"] == m)
        assert np.all(r["aux"] == 1)


def test_without_expansion_the_step_is_triangular():
    # m = 1: the interval is [-w V, w - w V] around x, the proposal theta = w (U - V): the
    # difference of two uniforms, triangular on [-w, w]
    # (along the line's direction u = sign(z_0), so that a lopsided interval is not hidden by the
    # direction's random sign)
    w = 2.0
    m = 200_000
    x0 = np.zeros((m, 1))
    r = O.run("slice", "gauss_diag", FLAT, x0, 1, seed=7, algo_params=[w, 1], store=False)
    u = np.sign([O.normals(7, c, 0, 0, 0, 1)[0] for c in range(m)])
    step = r["x_final"][:, 0] * u
    tri = stats.triang(c=0.5, loc=-w, scale=2 * w)
    assert stats.kstest(step, tri.cdf).pvalue > 1e-3
    assert np.all(np.abs(step) < w)


def test_standard_normal_and_diagonal_gaussian_stay_stationary():
    w = W.gauss_diag(3)
    m = 100_000
    x0 = W.x0_gauss_diag_exact(w, m)
    r = O.run("slice", "gauss_diag", w["params"], x0, 3, seed=4, algo_params=[1.0, 50], store=False)
    z = (r["x_final"] - w["mu"]) / w["sd"]
    assert np.all(np.abs(z.mean(0)) < 4 / math.sqrt(m))
    assert np.all(np.abs(z.var(0) - 1.0) < 4 * math.sqrt(2.0 / m))
    assert np.all(np.abs((z ** 4).mean(0) - 3.0) < 4 * math.sqrt(96.0 / m))
    # the random line through x changes direction each sample: samples move
    assert np.mean(np.abs(r["x_final"] - x0) > 0) > 0.99


@pytest.mark.parametrize("w,m_exp", [(4.0, 1), (0.5, 100)])
def test_standard_normal_moments_after_ten_transitions(w, m_exp):
    # 400k one-dimensional chains, ten transitions: a shrink rule that keeps too much of the
    # interval, or an interval not placed uniformly around x, moves the variance by >> 4 sigma
    m = 400_000
    x0 = np.random.default_rng(3).standard_normal((m, 1))
    r = O.run("slice", "gauss_diag", np.array([0.0, 1.0]), x0, 10, seed=7, algo_params=[w, m_exp], store=False)
    x = r["x_final"][:, 0]
    assert abs(x.mean()) < 4 / math.sqrt(m)
    assert abs(x.var() - 1.0) < 4 * math.sqrt(2.0 / m)
    assert abs(np.mean(x ** 4) - 3.0) < 4 * math.sqrt(96.0 / m)


def test_funnel_neck_stays_stationary():
    # v ~ N(0, 9): the interval widths needed range over orders of magnitude (many expansion
    # steps in the mouth, many shrinks in the neck)
    m = 100_000
    x0 = W.x0_funnel_exact(m)
    r = O.run("slice", "funnel", np.zeros(1), x0, 3, seed=5, algo_params=[1.0, 100], store=False)
    v = r["x_final"][:, 0] / 3.0
    assert abs(v.mean()) < 4 / math.sqrt(m)
    assert abs(v.var() - 1.0) < 4 * math.sqrt(2.0 / m)
    c = r["counts"]
    assert c.max() > 3 * np.median(c)


def test_two_mode_mixture_keeps_its_weights():
    w = W.mog(2, rho=0.5, offsets=(-1.5, 1.5), weights=(1.0, 3.0))
    m = 100_000
    x0 = W.x0_mog_exact(w, m)
    r = O.run("slice", "mog", w["params"], x0, 4, seed=6, n_data=2, algo_params=[2.0, 20], store=False)
    # P(mean coordinate > 0) under the mixture: 1/4 P(N(-1.5, 0.75) > 0) + 3/4 P(N(1.5, 0.75) > 0)
    s = math.sqrt(0.5 + 0.5 / 2)
    p = 0.25 * stats.norm.sf(1.5 / s) + 0.75 * stats.norm.sf(-1.5 / s)
    frac = np.mean(r["x_final"].mean(1) > 0)
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / m)


@pytest.mark.parametrize("bad", [[0.0, 10], [-1.0, 10], [1.0, 0]])
def test_bad_parameters_are_rejected(bad):
    with pytest.raises(ValueError):
        O.run("slice", "gauss_diag", FLAT, np.zeros((2, 1)), 1, seed=1, algo_params=bad)
