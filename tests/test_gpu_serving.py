"""Continuous batching: jobs submitted while others run are admitted as memory frees up,
their work shares fused launches, and every result equals the same job run alone."""
import time

import numpy as np
import pytest

from paper_2503_17405_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _specs():
    g64, g200 = W.gp_logit(64), W.gp_logit(200)
    lr10, lr40 = W.logreg(500, 10), W.logreg(300, 40)
    return [
        dict(kind="gp_logit", w=g64, algo="ess", m=256, n=120, x0=W.x0_zeros(256, 64)),
        dict(kind="logreg", w=lr10, algo="nuts", m=64, n=40, x0=W.x0_logreg(lr10, 64)),
        dict(kind="gp_logit", w=g200, algo="ess", m=128, n=90, x0=W.x0_zeros(128, 200)),
        dict(kind="logreg", w=lr40, algo="nuts", m=32, n=30, x0=W.x0_logreg(lr40, 32)),
        dict(kind="gp_logit", w=g64, algo="ess", m=100, n=60, x0=W.x0_normal(100, 64, scale=0.1)),
    ]


def _make(eng, s, seed):
    w = s["w"]
    tg = eng.target(s["kind"], w["d"], w["params"], n_data=w["n_data"])
    return eng.job(tg, s["algo"], s["m"], s["n"], x0=s["x0"], seed=seed, prec="fp32",
                   nuts={"eps": 0.05, "max_depth": 10, "max_dH": 1000.0})


@pytest.fixture(scope="module")
def alone():
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    eng = fsmc.Engine(0)
    out = []
    for k, s in enumerate(_specs()):
        job = _make(eng, s, 10 + k)
        job.run("fsm")
        out.append((job.samples(), job.loop_counts()[0], job.bytes()))
    eng.close()
    return out


def _serve(alone, budget_jobs, mode):
    from paper_2503_17405_b300 import fsmc
    specs = _specs()
    budget = 0
    if budget_jobs:
        # room for the two largest jobs at once (plus the targets): forces queueing
        sizes = sorted(b for _, _, b in alone)
        budget = sum(sizes[-budget_jobs:]) + (64 << 20)
    eng = fsmc.Engine(0, hbm_budget_bytes=budget)
    jobs = []
    for k, s in enumerate(specs):
        job = _make(eng, s, 10 + k)
        job.submit(mode)
        jobs.append(job)
        time.sleep(0.01)  # arrivals while earlier jobs are on the GPU
    results = [None] * len(jobs)
    lat = [None] * len(jobs)
    t_end = time.time() + 300
    while any(r is None for r in results):
        assert time.time() < t_end, "serving did not finish"
        for k, job in enumerate(jobs):
            if results[k] is None:
                done, latency = job.poll()
                if done:
                    results[k] = (job.samples(), job.loop_counts()[0])
                    lat[k] = latency
                    job.close()   # frees its memory for queued jobs
        time.sleep(0.002)
    eng.wait_all(10.0)
    eng.close()
    return results, lat


@pytest.mark.parametrize("budget_jobs", [0, 2])
def test_results_in_the_mix_equal_results_alone(alone, budget_jobs):
    results, lat = _serve(alone, budget_jobs, "fsm")
    for k, ((xs, cs), (xa, ca, _)) in enumerate(zip(results, alone)):
        assert np.array_equal(cs, ca), k
        assert np.array_equal(xs, xa), k
    assert all(l > 0 for l in lat)


def test_synchronised_one_at_a_time_baseline(alone):
    # the synchronised kernels evaluate the logistic gradient per warp (the FSM kernel batches
    # it over a block), so compare at the FP32 parity tolerance
    from parity import compare
    results, lat = _serve(alone, 0, "sync")
    for k, ((xs, cs), (xa, ca, _)) in enumerate(zip(results, alone)):
        r = compare(xs, cs, xa, ca, "fp32")
        assert r["flipped"] <= max(1, cs.shape[0] // 8), k


def test_oversized_job_is_refused_not_hung(alone):
    from paper_2503_17405_b300 import fsmc
    eng = fsmc.Engine(0, hbm_budget_bytes=8 << 20)
    s = _specs()[0]
    job = _make(eng, s, 10)
    job.submit("fsm")
    t_end = time.time() + 30
    while True:
        try:
            done, _ = job.poll()
        except fsmc.FsmcError as e:
            assert e.status == fsmc.EADMIT
            break
        assert time.time() < t_end
        time.sleep(0.01)
    eng.close()
