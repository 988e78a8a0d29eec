"""The engine hands the device blocks of closed jobs to later jobs: a job in a reused block
gives exactly the samples of a job in a fresh one, and the moments read back into caller arrays
equal the sums over its samples."""
import numpy as np
import pytest

from paper_2503_17405_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_reused_blocks_and_moments():
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    w = W.gauss_conj(16)
    x0 = W.x0_normal(256, 16, scale=0.5)
    fresh = fsmc.Engine(0)
    tg = fresh.target("gauss_conj", 16, w["params"])
    j = fresh.job(tg, "ess", 256, 50, x0=x0, seed=3, prec="fp32")
    j.run()
    ref = j.samples()
    j.close()
    fresh.close()

    eng = fsmc.Engine(0)
    tg = eng.target("gauss_conj", 16, w["params"])
    for m, n, store in ((300, 60, True), (256, 50, False), (256, 40, True)):  # leave blocks behind
        k = eng.job(tg, "ess", m, n, x0=W.x0_normal(m, 16), seed=9, prec="fp32", store=store)
        k.run()
        k.close()
    assert eng.bytes_in_use() < 1 << 20  # only the target's copies are accounted for
    j = eng.job(tg, "ess", 256, 50, x0=x0, seed=3, prec="fp32")
    j.run()
    assert np.array_equal(j.samples(), ref)
    sx, sx2, nk = np.zeros((256, 16)), np.zeros((256, 16)), np.zeros(256, dtype=np.int64)
    j.moments(sx, sx2, nk)
    xs = ref.astype(np.float64)
    assert np.all(nk == 50)
    assert np.allclose(sx, xs.sum(1), rtol=1e-5, atol=1e-4)
    assert np.allclose(sx2, (xs ** 2).sum(1), rtol=1e-5, atol=1e-4)
    with pytest.raises(ValueError):
        j.moments(np.zeros((256, 15)), sx2, nk)
    j.close()
    eng.close()
