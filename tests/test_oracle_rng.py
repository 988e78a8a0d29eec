"""Pins of the oracle's counter-based RNG (Philox4x32-10) and its conversions."""
import numpy as np
import pytest
from scipy import stats

from conftest import load_kat
from oracle import oracle as O


@pytest.mark.parametrize("ctr,key,out", load_kat())
def test_philox_known_answers(ctr, key, out):
    # published known-answer vectors of Philox4x32-10 (Salmon et al., SC'11)
    assert O.philox4x32_10(ctr, key) == out


def test_uniform_endpoints_are_open():
    # u = ((hi:lo >> 12) + 1/2) 2^-52: smallest 2^-53, largest 1 - 2^-53, never 0 or 1
    assert O.uniform(0, 0) == 2.0 ** -53
    assert O.uniform(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert O.uniform(0x80000000, 0) == 0.5 + 2.0 ** -53


def test_uniform_is_uniform():
    ws = [O.philox4x32_10([i, 7, 3, 0], [11, 13]) for i in range(20000)]
    u = np.array([O.uniform(w[0], w[1]) for w in ws])
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_box_muller_normals():
    # 40000 normals: mean 0, variance 1, normal CDF (Kolmogorov-Smirnov), and the
    # two members of a Box-Muller pair are uncorrelated
    z = np.concatenate([O.normals(5, c, 3, 0, 0, 40) for c in range(1000)])
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 4 * np.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    pairs = z.reshape(-1, 2)
    assert abs(np.corrcoef(pairs.T)[0, 1]) < 4 / np.sqrt(len(pairs))


def test_streams_are_keyed_by_chain_sample_tag_draw():
    base = O.normals(9, 1, 2, 0, 0, 8)
    assert np.array_equal(base, O.normals(9, 1, 2, 0, 0, 8))
    for args in [(9, 2, 2, 0, 0), (9, 1, 3, 0, 0), (9, 1, 2, 1, 0), (9, 1, 2, 0, 4), (10, 1, 2, 0, 0)]:
        assert not np.allclose(base, O.normals(*args, 8))
    # normals 4q .. 4q+3 come from draw q: starting at draw 1 shifts by one block
    assert np.array_equal(base[4:], O.normals(9, 1, 2, 0, 1, 4))


def test_uniform32_endpoints():
    assert O.uniform32(0) == 2.0 ** -33
    assert O.uniform32(0xFFFFFFFF) == 1.0 - 2.0 ** -33
