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
