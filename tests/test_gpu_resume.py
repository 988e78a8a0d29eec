"""Checkpoint / resume (fsmc_job_snapshot, fsmc_job_restore) for every sampler: a run stopped part
way, snapshotted, restored into a fresh job and finished gives the samples and loop counts of an
uninterrupted run bit for bit (the chains' states, FSM state ids, per-state variables, sample
counters and the keyed random numbers are all in the snapshot or derived from it)."""
import numpy as np
import pytest

from paper_2503_17405_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    e = fsmc.Engine(0)
    yield e
    e.close()


def _cases():
    lr = W.logreg(200, 6)
    mg = W.mog(12, rho=0.9, offsets=(-2.0, 2.0))
    return {
        "dr_funnel": ("dr", "funnel", 10, None, 0, W.x0_funnel_exact(384), {"dr": {"n_stages": 3, "scale0": 1.0, "factor": 0.5}}),
        "sdr_funnel": ("dr", "funnel", 10, None, 0, W.x0_funnel_exact(256),
                       {"dr": {"n_stages": 30, "scale0": 0.3, "factor": 1.0, "symmetric": 1}}),
        "slice_funnel": ("slice", "funnel", 10, None, 0, W.x0_funnel_exact(384), {"slice": {"w": 1.0, "m": 50}}),
        "nuts_logreg": ("nuts", "logreg", 6, lr["params"], 200, W.x0_logreg(lr, 96),
                        {"nuts": {"eps": 0.05, "max_depth": 8, "max_dH": 1000.0}}),
        "nuts_mog": ("nuts", "mog", 12, mg["params"], 2, W.x0_mog_exact(mg, 64),
                     {"nuts": {"eps": 0.1, "max_depth": 8, "max_dH": 1000.0}}),
    }


@pytest.mark.parametrize("name", list(_cases()))
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_resume_from_snapshot_is_bit_exact(eng, name, prec):
    algo, kind, d, params, n_data, x0, kw = _cases()[name]
    m, n = x0.shape[0], 120
    tg = eng.target(kind, d, params, n_data=n_data)
    tu = {"steps_per_launch": 16}
    whole = eng.job(tg, algo, m, n, x0=x0, seed=3, prec=prec, tuning=tu, **kw)
    whole.run("fsm")
    part = eng.job(tg, algo, m, n, x0=x0, seed=3, prec=prec, tuning=tu, **kw)
    part.run("fsm", max_fsm_steps=40)
    mn, done = part.progress()
    assert not done
    blob = part.snapshot()
    part.close()
    fresh = eng.job(tg, algo, m, n, x0=x0, seed=3, prec=prec, tuning=tu, **kw)
    fresh.restore(blob)
    assert fresh.progress()[0] == mn
    fresh.run("fsm")
    cw, aw, _ = whole.loop_counts()
    cf, af, _ = fresh.loop_counts()
    assert np.array_equal(cf, cw) and np.array_equal(af, aw)
    assert np.array_equal(fresh.samples(), whole.samples())
    whole.close()
    fresh.close()


def test_restore_rejects_a_snapshot_of_another_shape(eng):
    from paper_2503_17405_b300 import fsmc
    tg = eng.target("funnel", 10)
    a = eng.job(tg, "dr", 64, 20, x0=W.x0_funnel_exact(64), dr={"n_stages": 3, "scale0": 1.0, "factor": 0.5})
    a.run("fsm", max_fsm_steps=8)
    blob = a.snapshot()
    b = eng.job(tg, "dr", 32, 20, x0=W.x0_funnel_exact(32), dr={"n_stages": 3, "scale0": 1.0, "factor": 0.5})
    with pytest.raises(fsmc.FsmcError):
        b.restore(blob)
    with pytest.raises(fsmc.FsmcError):
        a.restore(blob[:-8])
    a.close()
    b.close()
