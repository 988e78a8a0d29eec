"""The paper's step-form ablations (tuning.step_form = 2) on the CUDA kernels: the ESS bundled
step without amortisation (both states' log-density calls every step, one masked; Sec. 3.3 /
App. B) and DR with its PROPOSE body unrolled into four states run one per step (not condensed,
Sec. 7.1) compute exactly the samples and loop counts of the default forms; only the work per
sample differs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W
from parity import compare

pytestmark = pytest.mark.gpu

DR = {"n_stages": 3, "scale0": 1.0, "factor": 0.5}


@pytest.fixture(scope="module")
def eng():
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    e = fsmc.Engine(0)
    yield e
    e.close()


@pytest.mark.parametrize("lanes", [1, 32])
def test_ess_not_amortised_gives_identical_samples(eng, lanes):
    w = W.gauss_conj(16)
    m, n = 300, 200
    x0 = W.x0_normal(m, 16, scale=0.5)
    tg = eng.target("gauss_conj", 16, w["params"])
    out = []
    for form in (1, 2):
        job = eng.job(tg, "ess", m, n, x0=x0, seed=3, prec="fp32",
                      tuning={"lanes_per_chain": lanes, "steps_per_launch": 24, "step_form": form})
        assert job.tuning()["step_form"] == form
        job.run("fsm")
        c, _, steps = job.loop_counts()
        out.append((job.samples(), c, steps))
        job.close()
    (xa, ca, sa), (xb, cb, sb) = out
    assert np.array_equal(ca, cb)
    assert np.array_equal(xa, xb)
    # one state per log-density evaluation in both forms: N + 1 per sample
    assert np.array_equal(sa, (ca + 1).sum(1)) and np.array_equal(sb, sa)


def test_dr_not_condensed_gives_identical_samples_in_four_states_per_stage(eng):
    m, n = 400, 300
    x0 = W.x0_funnel_exact(m)
    w = W.funnel(10)
    tg = eng.target("funnel", 10, w["params"])
    out = []
    for form in (1, 2):
        job = eng.job(tg, "dr", m, n, x0=x0, seed=5, prec="fp64", dr=DR,
                      tuning={"steps_per_launch": 37, "step_form": form})
        job.run("fsm")
        c, _, steps = job.loop_counts()
        out.append((job.samples(), c, steps))
        job.close()
    (xa, ca, sa), (xb, cb, sb) = out
    assert np.array_equal(ca, cb)
    assert np.array_equal(xa, xb)
    assert np.array_equal(sa, ca.sum(1))             # condensed: one state per stage tried
    assert np.array_equal(sb, 4 * ca.sum(1))         # draw, evaluate, ratio, decide per stage
    # and both follow the oracle (FP64: 1e-10, identical stage counts)
    ref = O.run("dr", "funnel", np.zeros(1), x0, n, seed=5, algo_params=[3, 1.0, 0.5])
    r = compare(xb, cb, ref["samples"], ref["counts"], "fp64")
    assert r["max_err"] <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_symmetric_dr_four_states_per_try_on_the_papers_toy(eng, prec):
    # Sec. 7.1's toy: N(0, 1), re-centred tries of sd 0.1, at most M = 100 tries; a launch budget
    # that splits samples and tries across launches
    m, n = 512, 200
    x0 = np.random.default_rng(5).standard_normal((m, 1))
    tg = eng.target("gauss_diag", 1, np.array([0.0, 1.0]))
    sdr = {"n_stages": 100, "scale0": 0.1, "factor": 1.0, "symmetric": 1}
    out = []
    for form in (1, 2):
        job = eng.job(tg, "dr", m, n, x0=x0, seed=8, prec=prec, dr=sdr,
                      tuning={"steps_per_launch": 41, "step_form": form})
        job.run("fsm")
        c, _, steps = job.loop_counts()
        out.append((job.samples(), c, steps))
        job.close()
    (xa, ca, sa), (xb, cb, sb) = out
    assert np.array_equal(ca, cb)
    assert np.array_equal(xa, xb)
    assert np.array_equal(sa, ca.sum(1)) and np.array_equal(sb, 4 * ca.sum(1))
    assert ca.max() > 5  # some samples need many tries
    if prec == "fp64":
        ref = O.run("sdr", "gauss_diag", np.array([0.0, 1.0]), x0, n, seed=8, algo_params=[100, 0.1])
        r = compare(xb, cb, ref["samples"], ref["counts"], "fp64")
        assert r["max_err"] <= 1e-10


def test_step_form_limits(eng):
    from paper_2503_17405_b300 import fsmc
    lr = W.logreg(200, 5)
    tl = eng.target("logreg", 5, lr["params"], n_data=200)
    with pytest.raises(fsmc.FsmcError):
        eng.job(tl, "nuts", 64, 10, prec="fp32", nuts={"eps": 0.05, "max_depth": 6, "max_dH": 1000.0},
                tuning={"step_form": 2})
    w = W.gauss_conj(16)
    tg = eng.target("gauss_conj", 16, w["params"])
    job = eng.job(tg, "ess", 32, 10, prec="fp32", tuning={"step_form": 2})
    with pytest.raises(fsmc.FsmcError):
        job.submit("fsm")  # serving runs the default step forms only
    job.close()
