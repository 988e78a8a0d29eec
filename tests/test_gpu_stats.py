"""Run statistics (Sec. 4.1-4.2) read through fsmc_read_stats, which reduces the [m][n] loop
counts on the device: R(m) = mean_i max_j N_ij / mean_ij N_ij must equal the oracle's R_hat on
the same counts, and mean N, mean max N, the sample and state totals must equal direct sums."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    e = fsmc.Engine(0)
    yield e
    e.close()


def _check(job, counts, steps, tmin):
    st = job.stats()
    c = counts[:, :tmin]
    assert st["R_hat"] == pytest.approx(O.R_hat(np.ascontiguousarray(c)), rel=1e-13)
    assert st["mean_N"] == pytest.approx(c.mean(dtype=np.float64), rel=1e-13)
    assert st["mean_max_N"] == pytest.approx(c.max(axis=0).mean(dtype=np.float64), rel=1e-13)
    assert st["fsm_steps"] == int(steps.sum())
    return st


def _read_stats_ms(job, reps=7):
    job.stats()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        job.stats()
        ts.append((time.perf_counter() - t0) * 1e3)
    return float(np.median(ts))


def test_ess_gp_logit_full_size_stats_match_oracle(eng):
    # the headline configuration: 16384 chains x 2000 samples, FP32 (131 MB of loop counts)
    w = W.gp_logit(256)
    m, n = 16384, 2000
    tg = eng.target("gp_logit", 256, w["params"])
    job = eng.job(tg, "ess", m, n, x0=W.x0_zeros(m, 256), seed=1, prec="fp32")
    job.run("fsm")
    counts, _, steps = job.loop_counts()
    st = _check(job, counts, steps, n)
    assert st["samples_done"] == m * n
    assert 3.5 < st["R_hat"] < 5.5
    ms = _read_stats_ms(job)
    print("read_stats at 16384 x 2000:", ms, "ms; R_hat", st["R_hat"])
    assert ms < 1.0
    job.close()


def test_dr_funnel_full_size_stats_match_oracle(eng):
    # the delayed-rejection configuration: 65536 chains x 5000 samples, FP32 (1.3 GB of counts)
    m, n = 65536, 5000
    tg = eng.target("funnel", 10)
    job = eng.job(tg, "dr", m, n, x0=W.x0_funnel_exact(m), seed=1, prec="fp32",
                  dr={"n_stages": 3, "scale0": 1.0, "factor": 0.5})
    job.run("fsm")
    counts, _, steps = job.loop_counts()
    st = _check(job, counts, steps, n)
    assert st["samples_done"] == m * n
    job.close()


def test_partial_run_stats_cover_completed_samples_only(eng):
    # after a partial run chains stand at different sample counts: the statistics use the samples
    # i < min_j t_j that every chain has, and samples_done counts every emitted sample
    w = W.gauss_conj(16)
    m, n = 1000, 400
    tg = eng.target("gauss_conj", 16, w["params"])
    job = eng.job(tg, "ess", m, n, x0=W.x0_normal(m, 16), seed=3, prec="fp32",
                  tuning={"lanes_per_chain": 1, "steps_per_launch": 16})
    job.run("fsm", max_fsm_steps=300)
    counts, _, steps = job.loop_counts()
    t = (counts >= 0).sum(axis=1)
    tmin = int(t.min())
    assert 0 < tmin < n and t.max() > tmin
    st = _check(job, counts, steps, tmin)
    assert st["samples_done"] == int(t.sum())
    job.close()


def test_sync_iterations_and_error_word_in_the_record(eng):
    m, n = 4096, 200
    tg = eng.target("funnel", 10)
    job = eng.job(tg, "dr", m, n, x0=W.x0_funnel_exact(m), seed=2, prec="fp32",
                  dr={"n_stages": 3, "scale0": 1.0, "factor": 0.5})
    job.run("sync")
    counts, _, steps = job.loop_counts()
    st = _check(job, counts, steps, n)
    assert st["sync_iterations"] == int(counts.max(axis=0).sum())
    assert st["error_word"] == 0
    job.close()
