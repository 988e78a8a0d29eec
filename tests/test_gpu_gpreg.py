"""ESS on Sec. 7.2's GP-regression hyperparameters with the likelihood evaluated warp-wide (a
chain per warp, the n x n covariance factorised in shared memory) against the FP64 oracle,
through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W
from parity import compare, transitions_agree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    e = fsmc.Engine(0)
    yield e
    e.close()


def _job(eng, w, x0, n, prec, mode, tuning=None, seed=2):
    tg = eng.target("gp_reg", 3, w["params"], n_data=w["n_data"])
    job = eng.job(tg, "ess", x0.shape[0], n, x0=x0, seed=seed, prec=prec, tuning=tuning)
    job.run(mode)
    return job


@pytest.mark.parametrize("n_data", [25, 100, 219])
@pytest.mark.parametrize("mode", ["fsm", "sync"])
def test_fp64_matches_oracle(eng, n_data, mode):
    w = W.gp_reg(n_data)
    x0 = W.x0_gp_reg(w, 20)
    n = 25
    job = _job(eng, w, x0, n, "fp64", mode)
    ref = O.run("ess", "gp_reg", w["params"], x0, n, seed=2, n_data=n_data)
    counts, _, steps = job.loop_counts()
    compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    if mode == "fsm":
        assert np.array_equal(steps, (counts + 1).sum(1))   # one likelihood per FSM step
    else:
        assert job.stats()["sync_iterations"] >= int((counts.max(0) + 1).sum())
    job.close()


def test_fp32_fsm_equals_sync_and_partial_runs(eng):
    w = W.gp_reg(100)
    x0 = W.x0_gp_reg(w, 40)
    n = 40
    a = _job(eng, w, x0, n, "fp32", "fsm")
    b = _job(eng, w, x0, n, "fp32", "sync")
    c = _job(eng, w, x0, n, "fp32", "fsm", tuning={"steps_per_launch": 3})
    (ca, _, _), (cb, _, _), (cc, _, _) = a.loop_counts(), b.loop_counts(), c.loop_counts()
    assert np.array_equal(ca, cb) and np.array_equal(a.samples(), b.samples())
    assert np.array_equal(ca, cc) and np.array_equal(a.samples(), c.samples())
    for j in (a, b, c):
        j.close()


@pytest.mark.parametrize("n_data", [25, 100, 319])
def test_fp32_transition_by_transition_against_the_oracle(eng, n_data):
    w = W.gp_reg(n_data)
    x0 = W.x0_gp_reg(w, 32).astype(np.float32).astype(np.float64)
    m, n = x0.shape[0], 40
    job = _job(eng, w, x0, n, "fp32", "fsm")
    xs = job.samples().astype(np.float64)
    counts, _, _ = job.loop_counts()
    job.close()
    starts = np.concatenate([x0[:, None, :], xs[:, :-1, :]], axis=1).reshape(m * n, -1)
    ref = O.transitions("ess", "gp_reg", w["params"], starts, np.repeat(np.arange(m), n), np.tile(np.arange(n), m),
                        seed=2, n_data=n_data)
    transitions_agree(xs.reshape(m * n, -1), counts.ravel(), ref, "fp32 gp_reg n=%d" % n_data)


@pytest.mark.parametrize("mode", ["fsm", "sync"])
def test_fp64_papers_largest_size_matches_oracle(eng, mode):
    # n = 400 (Sec. 7.2's largest): the rows beyond shared memory live in the CTA's scratch block
    w = W.gp_reg(400)
    x0 = W.x0_gp_reg(w, 6)
    n = 6
    job = _job(eng, w, x0, n, "fp64", mode)
    ref = O.run("ess", "gp_reg", w["params"], x0, n, seed=2, n_data=400)
    counts, _, _ = job.loop_counts()
    compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    job.close()


def test_fp32_papers_largest_size_transitions(eng):
    w = W.gp_reg(400)
    x0 = W.x0_gp_reg(w, 8).astype(np.float32).astype(np.float64)
    m, n = x0.shape[0], 8
    job = _job(eng, w, x0, n, "fp32", "fsm")
    xs = job.samples().astype(np.float64)
    counts, _, _ = job.loop_counts()
    job.close()
    starts = np.concatenate([x0[:, None, :], xs[:, :-1, :]], axis=1).reshape(m * n, -1)
    ref = O.transitions("ess", "gp_reg", w["params"], starts, np.repeat(np.arange(m), n), np.tile(np.arange(n), m),
                        seed=2, n_data=400)
    transitions_agree(xs.reshape(m * n, -1), counts.ravel(), ref, "fp32 gp_reg n=400")


def test_limits_and_argument_checks(eng):
    from paper_2503_17405_b300 import fsmc
    big = W.gp_reg(513)
    with pytest.raises(fsmc.FsmcError):
        eng.target("gp_reg", 3, big["params"], n_data=513)        # over the size limit
    w = W.gp_reg(25)
    with pytest.raises(fsmc.FsmcError):
        eng.target("gp_reg", 2, w["params"][1:], n_data=25)      # d must be 3
    tg = eng.target("gp_reg", 3, w["params"], n_data=25)
    with pytest.raises(fsmc.FsmcError):
        eng.job(tg, "ess", 4, 4, tuning={"lanes_per_chain": 16})
    with pytest.raises(fsmc.FsmcError):
        eng.job(tg, "nuts", 4, 4)
    job = eng.job(tg, "ess", 4, 4)
    with pytest.raises(fsmc.FsmcError):
        job.submit("fsm")
    job.close()
