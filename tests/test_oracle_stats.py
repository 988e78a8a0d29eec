"""Pins of the R(m) estimator (Sec. 4.2, "Scale of potential speed-ups").

R(m) = E max_j N_j / E N_1.  For N/B ~ Bernoulli(p) the paper gives
R(m) = (1 - (1-p)^m) / p; for any law on the integers E max over m i.i.d.
draws = sum_{k>=0} (1 - F(k)^m).
"""
import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("m,p", [(1, 0.3), (8, 0.1), (64, 0.02)])
def test_bernoulli_closed_form(m, p):
    rng = np.random.default_rng(m)
    n = 200_000
    B = 10
    counts = (B * (rng.uniform(size=(m, n)) < p)).astype(np.int32)
    R = O.R_hat(counts)
    exact = (1 - (1 - p) ** m) / p
    assert abs(R / exact - 1) < 0.03


def test_geometric_expected_max_formula():
    rng = np.random.default_rng(7)
    m, n, q = 32, 50_000, 0.3
    counts = rng.geometric(q, size=(m, n)).astype(np.int32) - 1   # support 0, 1, 2, ...
    k = np.arange(0, 400)
    F = 1 - (1 - q) ** (k + 1)
    e_max = np.sum(1 - F ** m)
    e_n = (1 - q) / q
    assert abs(O.R_hat(counts) / (e_max / e_n) - 1) < 0.02


def test_single_chain_and_constant_counts():
    assert O.R_hat(np.full((1, 100), 5, np.int32)) == 1.0
    assert O.R_hat(np.full((16, 100), 3, np.int32)) == 1.0
    assert O.R_hat(np.zeros((4, 10), np.int32)) == 1.0
