"""Failure detection without a GPU fault: every failure here is made on the host or by a bounded
device wait that is told to expect an arrival that never comes.  Nothing traps, faults or hangs;
after each failure the device is shown to still answer by a run that succeeds.

  * a grid-barrier wait of the synchronised kernel runs out -> FSMC_ETIMEOUT, error bit 2;
  * a log density that is NaN everywhere (a NaN label in the logistic-regression data) is
    treated as -inf: every proposal is rejected and error bit 4 is set;
  * ESS on the GP-logit target from a state with a NaN coordinate: no proposal clears the
    threshold, every sample ends at the shrink cap (bits 1 and 4) with the state unchanged;
  * a running submitted job is cancelled -> FSMC_ECANCELED, while a job beside it finishes with
    the samples it has when run alone;
  * a job larger than the device's memory, under a budget that admits it -> FSMC_ENOMEM.
"""
import time

import numpy as np
import pytest

from paper_2503_17405_b300 import fsmc, workloads as W

pytestmark = pytest.mark.gpu

DR = {"n_stages": 3, "scale0": 1.0, "factor": 0.5}


@pytest.fixture(scope="module")
def eng():
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    e = fsmc.Engine(0)
    yield e
    e.close()


@pytest.mark.parametrize("algo", ["dr", "ess"])
def test_sync_barrier_wait_runs_out_and_reports_timeout(eng, algo):
    from paper_2503_17405_b300 import fsmc
    m, n = 4096, 50
    if algo == "dr":
        tg = eng.target("funnel", 10)
        kw, x0 = {"dr": DR}, W.x0_funnel_exact(m)
    else:
        w = W.gp_logit(64)
        tg = eng.target("gp_logit", 64, w["params"])
        kw, x0 = {}, W.x0_zeros(m, 64)
    bad = eng.job(tg, algo, m, n, x0=x0, seed=1, prec="fp32",
                  tuning={"barrier_spin_limit": 1 << 14, "barrier_test_missing": 1}, **kw)
    t0 = time.perf_counter()
    with pytest.raises(fsmc.FsmcError) as ei:
        bad.run("sync")
    elapsed = time.perf_counter() - t0
    assert ei.value.status == fsmc.ETIMEOUT
    assert bad.stats()["error_word"] & 2
    assert elapsed < 30.0
    bad.close()
    # the device still answers: the same job without the hook runs, and matches the FSM run
    good = eng.job(tg, algo, m, n, x0=x0, seed=1, prec="fp32", **kw)
    good.run("sync")
    ref = eng.job(tg, algo, m, n, x0=x0, seed=1, prec="fp32", **kw)
    ref.run("fsm")
    assert good.stats()["error_word"] == 0
    assert np.array_equal(good.samples(), ref.samples())
    good.close()
    ref.close()


def test_barrier_hook_is_checked(eng):
    from paper_2503_17405_b300 import fsmc
    tg = eng.target("funnel", 10)
    for bad in ({"barrier_test_missing": 2}, {"barrier_spin_limit": -1}):
        with pytest.raises(fsmc.FsmcError) as ei:
            eng.job(tg, "dr", 64, 4, dr=DR, tuning=bad)
        assert ei.value.status == fsmc.EINVAL


@pytest.mark.parametrize("algo", ["dr", "nuts"])
def test_nan_log_density_rejects_every_proposal_and_sets_the_error_bit(eng, algo):
    w = W.logreg(50, 5)
    params = np.array(w["params"], dtype=np.float64)
    params[50 * 5 + 7] = np.nan          # label 7
    tg = eng.target("logreg", 5, params, n_data=50)
    m, n = 256, 20
    x0 = W.x0_logreg(w, m)
    kw = {"dr": DR} if algo == "dr" else {"nuts": {"eps": 0.05, "max_depth": 6, "max_dH": 1000.0}}
    for mode in ("fsm", "sync"):
        job = eng.job(tg, algo, m, n, x0=x0, seed=1, prec="fp32", **kw)
        job.run(mode)
        st = job.stats()
        assert st["error_word"] & 4, st["error_word"]
        xs = job.samples()
        assert np.array_equal(xs, np.broadcast_to(x0.astype(np.float32)[:, None, :], xs.shape))
        counts, depth, _ = job.loop_counts()
        if algo == "dr":
            assert np.all(counts == 3)       # every stage tried and rejected
        else:
            assert np.all(counts == 1) and np.all(depth == 1)  # the first leaf diverges
        job.close()


@pytest.mark.parametrize("lanes", [32, 1])
def test_ess_gp_logit_from_a_nan_state_ends_every_sample_at_the_shrink_cap(eng, lanes):
    d = 256 if lanes == 32 else 16
    w = W.gp_logit(d)
    tg = eng.target("gp_logit", d, w["params"])
    m, n = 64, 2
    x0 = W.x0_zeros(m, d)
    x0[5, 3] = np.nan
    for mode in ("fsm", "sync"):
        job = eng.job(tg, "ess", m, n, x0=x0, seed=1, prec="fp32", tuning={"lanes_per_chain": lanes})
        with pytest.raises(fsmc.FsmcError, match="shrink cap"):   # the run completes, then reports
            job.run(mode)
        st = job.stats()
        assert st["error_word"] & 5 == 5, st["error_word"]
        assert st["samples_done"] == m * n
        counts, _, _ = job.loop_counts()
        assert np.all(counts[5] == 10000)   # the shrink cap
        assert np.all(np.isnan(job.samples(5, 1)[0, :, 3]))
        assert np.all(counts[np.arange(m) != 5] < 10000)
        job.close()


def test_cancel_a_running_submitted_job(eng):
    from paper_2503_17405_b300 import fsmc
    w = W.logreg(1000, 25)
    tg = eng.target("logreg", 25, w["params"], n_data=1000)
    nuts = {"eps": 0.05, "max_depth": 10, "max_dH": 1000.0}
    long_job = eng.job(tg, "nuts", 4096, 20000, x0=W.x0_logreg(w, 4096), seed=1, prec="fp32", store=False,
                       nuts=nuts)
    g = W.gauss_conj(16)
    tg2 = eng.target("gauss_conj", 16, g["params"])
    x2 = W.x0_normal(256, 16)
    side = eng.job(tg2, "ess", 256, 300, x0=x2, seed=4, prec="fp32")
    long_job.submit("fsm")
    side.submit("fsm")
    deadline = time.time() + 60
    while long_job.progress()[0] == 0 and time.time() < deadline:
        time.sleep(0.01)
    assert long_job.progress()[0] > 0, "the long job never started"
    long_job.cancel()
    eng.wait_all(120.0)
    with pytest.raises(fsmc.FsmcError) as ei:
        long_job.poll()
    assert ei.value.status == fsmc.ECANCELED
    mn, done = long_job.progress()
    assert not done and mn < 20000
    assert side.poll()[0]
    alone = eng.job(tg2, "ess", 256, 300, x0=x2, seed=4, prec="fp32")
    alone.run("fsm")
    assert np.array_equal(side.loop_counts()[0], alone.loop_counts()[0])
    assert np.array_equal(side.samples(), alone.samples())
    for j in (long_job, side, alone):
        j.close()


def test_allocation_larger_than_the_device_reports_enomem(eng):
    from paper_2503_17405_b300 import fsmc
    big = fsmc.Engine(0, hbm_budget_bytes=1 << 50)     # a budget beyond the device's memory
    try:
        w = W.gp_logit(256)
        tg = big.target("gp_logit", 256, w["params"])
        job = big.job(tg, "ess", 16384, 20000, prec="fp32")   # 335 GB of stored samples
        with pytest.raises(fsmc.FsmcError) as ei:
            job.run("fsm")
        assert ei.value.status == fsmc.ENOMEM
        job.close()
        ok = big.job(tg, "ess", 64, 20, prec="fp32")
        ok.run("fsm")
        assert ok.progress() == (20, True)
        ok.close()
    finally:
        big.close()
