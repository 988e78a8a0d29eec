"""The autotuner: it returns a valid launch shape, caches it, and jobs run with it."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W
from parity import compare

pytestmark = pytest.mark.gpu


def test_autotune_ess_dr_nuts_and_cache(tmp_path):
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    eng = fsmc.Engine(0)
    cache = str(tmp_path / "tune.txt")
    w = W.gp_logit(64)
    tg = eng.target("gp_logit", 64, w["params"])
    t1 = eng.autotune(tg, "ess", 2048, cache_path=cache)
    assert t1["lanes_per_chain"] in (1, 8, 16, 32) and t1["steps_per_launch"] > 0
    assert t1["generator"] in (1, 2) and t1["ring_slots"] > 0
    assert os.path.exists(cache)
    assert eng.autotune(tg, "ess", 2048, cache_path=cache) == t1   # served from the cache
    job = eng.job(tg, "ess", 64, 80, x0=W.x0_zeros(64, 64), seed=1, prec="fp32", tuning=t1)
    job.run()
    ref = O.run("ess", "gp_logit", w["params"], W.x0_zeros(64, 64), 80, seed=1)
    c, _, _ = job.loop_counts()
    compare(job.samples(), c, ref["samples"], ref["counts"], "fp32")
    fun = eng.target("funnel", 10)
    td = eng.autotune(fun, "dr", 8192, cache_path=cache)
    assert td["lanes_per_chain"] == 1 and td["threads_per_block"] in (64, 128, 256)
    lr = W.logreg(500, 10)
    tl = eng.target("logreg", 10, lr["params"], n_data=500)
    tn = eng.autotune(tl, "nuts", 512, cache_path=cache)
    assert tn["steps_per_launch"] in (32, 128, 256)
    assert len(open(cache).read().strip().splitlines()) == 3
    eng.close()
