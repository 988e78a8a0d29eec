"""The oracle's single-transition entry point reproduces its runs: started from the state a run
was in before sample t, with sample index t, it moves to the run's sample t with the same loop
count (the per-transition parity tests of single precision rely on this)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W


def _cases():
    g = W.gauss_conj(6)
    f = W.funnel(10)
    mg = W.mog(12, rho=0.9, offsets=(-2.0, 2.0))
    return [
        ("ess", "gauss_conj", g["params"], 0, None, W.x0_normal(6, 6, scale=0.5)),
        ("dr", "funnel", f["params"], 0, [3, 1.0, 0.5], W.x0_funnel_exact(6)),
        ("sdr", "mog", mg["params"], 2, [30, 0.3], W.x0_mog_exact(mg, 6)),
        ("nuts", "mog", mg["params"], 2, [0.1, 8, 1000.0], W.x0_mog_exact(mg, 6)),
    ]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_single_transitions_reproduce_a_run(case):
    algo, kind, params, n_data, ap, x0 = case
    m, n = x0.shape[0], 7
    run = O.run(algo, kind, params, x0, n, seed=5, chain0=3, n_data=n_data, algo_params=ap)
    starts = np.concatenate([x0[:, None, :], run["samples"][:, :-1, :]], axis=1).reshape(m * n, -1)
    chains = np.repeat(np.arange(3, 3 + m), n)
    samples = np.tile(np.arange(n), m)
    t = O.transitions(algo, kind, params, starts, chains, samples, seed=5, n_data=n_data, algo_params=ap)
    assert np.array_equal(t["x"], run["samples"].reshape(m * n, -1))
    assert np.array_equal(t["counts"], run["counts"].ravel())
    assert np.array_equal(t["aux"], run["aux"].ravel())


def test_decision_margin_of_a_one_stage_dr_transition():
    # One delayed-rejection stage makes exactly one decision, log u < log alpha_1 with
    # alpha_1 = min(1, pi(y) / pi(x)); the recorded margin is |log u - log alpha_1| /
    # max(1, |log alpha_1|), rebuilt here from the oracle's own random numbers and log density.
    w = W.gauss_diag(3)
    x = W.x0_gauss_diag_exact(w, 5)
    chains, samples = np.arange(5), np.array([0, 4, 9, 2, 7])
    t = O.transitions("dr", "gauss_diag", w["params"], x, chains, samples, seed=8, algo_params=[1, 0.7, 1.0])
    D = 1  # ceil(3 / 4) normal blocks
    for i in range(5):
        z = O.normals(8, int(chains[i]), int(samples[i]), 0, 0, 3)
        y = x[i] + 0.7 * z
        la = min(0.0, O.logp("gauss_diag", w["params"], y) - O.logp("gauss_diag", w["params"], x[i]))
        b = O.philox4x32_10([D, int(samples[i]), 0, 0], [int(chains[i]), 8])
        lu = np.log(O.uniform(b[0], b[1]))
        assert t["margin"][i] == pytest.approx(abs(lu - la) / max(1.0, abs(la)), rel=1e-12)
        assert t["counts"][i] == 1


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_margins_are_recorded_and_do_not_change_the_transition(case):
    # the transitions above reproduce runs bit for bit with the margin bookkeeping on; every
    # transition makes at least one decision, so every margin is finite and non-negative
    algo, kind, params, n_data, ap, x0 = case
    m = x0.shape[0]
    t = O.transitions(algo, kind, params, x0, np.arange(m), np.zeros(m, dtype=int), seed=5,
                      n_data=n_data, algo_params=ap)
    assert np.all(np.isfinite(t["margin"])) and np.all(t["margin"] >= 0)
