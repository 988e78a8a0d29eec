"""The slice sampler (Fig. 2's two-loop FSM: stepping out, then shrinkage) on the CUDA kernels
against the FP64 oracle, through the C ABI: FSM and synchronised kernels, loop counts, partial
runs, the synchronised loop structure, and argument checks."""
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


def _cases():
    g = W.gauss_diag(3)
    mg = W.mog(5, rho=0.6, offsets=(-2.0, 2.0), weights=(1.0, 2.0))
    return {
        "gauss_diag": (g, W.x0_gauss_diag_exact(g, 96), {"w": 1.0, "m": 20}),
        "funnel": (dict(kind="funnel", d=10, n_data=0, params=np.zeros(0)), W.x0_funnel_exact(96),
                   {"w": 1.0, "m": 100}),
        "mog": (mg, W.x0_mog_exact(mg, 96), {"w": 2.0, "m": 8}),
    }


def _job(eng, w, x0, sl, n, prec, mode, tuning=None, seed=3):
    tg = eng.target(w["kind"], w["d"], w["params"] if w["params"].size else None, n_data=w["n_data"])
    job = eng.job(tg, "slice", x0.shape[0], n, x0=x0, seed=seed, prec=prec, slice=sl, tuning=tuning)
    job.run(mode)
    return job


@pytest.mark.parametrize("mode", ["fsm", "sync"])
@pytest.mark.parametrize("name", ["gauss_diag", "funnel", "mog"])
def test_fp64_matches_oracle(eng, name, mode):
    w, x0, sl = _cases()[name]
    n = 120
    job = _job(eng, w, x0, sl, n, "fp64", mode)
    ref = O.run("slice", w["kind"], w["params"], x0, n, seed=3, n_data=w["n_data"], algo_params=[sl["w"], sl["m"]])
    counts, props, steps = job.loop_counts()
    compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert np.array_equal(props, ref["aux"])
    if mode == "fsm":
        assert np.array_equal(steps, counts.sum(1))   # one log-density evaluation per FSM step
    else:
        # three loops in sequence per sample, each run until its slowest chain leaves it
        assert job.stats()["sync_iterations"] >= int(counts.max(0).sum())
    job.close()


def test_fp32_fsm_equals_sync_and_partial_runs(eng):
    w, x0, sl = _cases()["funnel"]
    n = 200
    a = _job(eng, w, x0, sl, n, "fp32", "fsm")
    b = _job(eng, w, x0, sl, n, "fp32", "sync")
    c = _job(eng, w, x0, sl, n, "fp32", "fsm", tuning={"steps_per_launch": 3})
    xa, xb, xc = a.samples(), b.samples(), c.samples()
    (ca, pa, _), (cb, pb, _), (cc, pc, _) = a.loop_counts(), b.loop_counts(), c.loop_counts()
    assert np.array_equal(ca, cb) and np.array_equal(pa, pb) and np.array_equal(xa, xb)
    assert np.array_equal(ca, cc) and np.array_equal(xa, xc)
    for j in (a, b, c):
        j.close()


def test_fp32_transition_by_transition_against_the_oracle(eng):
    w, x0, sl = _cases()["funnel"]
    x0 = x0.astype(np.float32).astype(np.float64)
    m, n = x0.shape[0], 150
    job = _job(eng, w, x0, sl, n, "fp32", "fsm")
    xs = job.samples().astype(np.float64)
    counts, _, _ = job.loop_counts()
    job.close()
    starts = np.concatenate([x0[:, None, :], xs[:, :-1, :]], axis=1).reshape(m * n, -1)
    ref = O.transitions("slice", "funnel", w["params"], starts, np.repeat(np.arange(m), n), np.tile(np.arange(n), m),
                        seed=3, algo_params=[sl["w"], sl["m"]])
    transitions_agree(xs.reshape(m * n, -1), counts.ravel(), ref, "fp32 slice")


def test_flat_target_takes_every_expansion_step(eng):
    flat = dict(kind="gauss_diag", d=2, n_data=0, params=np.array([0.0, 0.0, 1e9, 1e9]))
    x0 = np.zeros((64, 2))
    for m_lim in (1, 5, 40):
        job = _job(eng, flat, x0, {"w": 1.0, "m": m_lim}, 6, "fp64", "fsm")
        counts, props, _ = job.loop_counts()
        assert np.all(counts == m_lim) and np.all(props == 1)
        job.close()


def test_argument_checks(eng):
    from paper_2503_17405_b300 import fsmc
    g = W.gauss_diag(3)
    tg = eng.target("gauss_diag", 3, g["params"])
    for bad in ({"w": 0.0, "m": 10}, {"w": -1.0, "m": 10}, {"w": 1.0, "m": 0}):
        with pytest.raises(fsmc.FsmcError):
            eng.job(tg, "slice", 8, 4, slice=bad)
    with pytest.raises(fsmc.FsmcError):
        eng.job(tg, "slice", 8, 4, tuning={"step_form": 2})
    job = eng.job(tg, "slice", 8, 4)
    with pytest.raises(fsmc.FsmcError):
        job.submit("fsm")
    job.close()
    wide = W.gauss_diag(40)
    tw = eng.target("gauss_diag", 40, wide["params"])
    with pytest.raises(fsmc.FsmcError):
        eng.job(tw, "slice", 8, 4, tuning={"lanes_per_chain": 1})   # a chain per thread: d <= 32
    assert eng.job(tw, "slice", 8, 4).tuning()["lanes_per_chain"] == 32


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_moments_only_mode_matches_stored_samples(eng, prec, rtol):
    # moments-only slice jobs keep each chain's compensated sums in shared memory during a launch
    w, x0, sl = _cases()["funnel"]
    n = 300
    tg = eng.target(w["kind"], w["d"], None)
    jobs = []
    for store in (True, False):
        j = eng.job(tg, "slice", x0.shape[0], n, x0=x0, seed=3, prec=prec, store=store, slice=sl,
                    tuning={"steps_per_launch": 64})
        j.run("fsm")
        jobs.append(j)
    xs = jobs[0].samples()
    sx, sx2, nk = jobs[1].moments()
    assert np.all(nk == n)
    assert np.allclose(sx, xs.sum(1), rtol=rtol, atol=rtol * n)
    assert np.allclose(sx2, (xs ** 2).sum(1), rtol=rtol, atol=rtol * n)
    for j in jobs:
        j.close()


# ---- a chain per warp (d > 32) ------------------------------------------------------------------
def _wide_cases():
    g = W.gauss_diag(100)
    f = W.funnel(50)
    mg = W.mog(64, rho=0.5, offsets=(-3.0, 3.0))
    return {
        "gauss_diag_d100": (g, 0, W.x0_gauss_diag_exact(g, 96)),
        "funnel_d50": (f, 0, W.x0_funnel_exact(96, d=50)),
        "mog_d64": (mg, 2, W.x0_mog_exact(mg, 96)),
    }


@pytest.mark.parametrize("mode", ["fsm", "sync"])
@pytest.mark.parametrize("name", ["gauss_diag_d100", "funnel_d50", "mog_d64"])
def test_fp64_chain_per_warp_matches_oracle(eng, name, mode):
    w, n_data, x0 = _wide_cases()[name]
    m, n = x0.shape[0], 60
    sl = {"w": 1.0, "m": 30}
    tg = eng.target(w["kind"], w["d"], w["params"] if w["params"].size else None, n_data=n_data)
    job = eng.job(tg, "slice", m, n, x0=x0, seed=4, prec="fp64", slice=sl, tuning={"steps_per_launch": 25})
    assert job.tuning()["lanes_per_chain"] == 32
    job.run(mode)
    ref = O.run("slice", w["kind"], w["params"], x0, n, seed=4, n_data=n_data, algo_params=[1.0, 30])
    counts, props, _ = job.loop_counts()
    r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert r["max_err"] <= 1e-10
    assert np.array_equal(props, ref["aux"])
    job.close()


def test_fp32_chain_per_warp_fsm_equals_sync(eng):
    w, n_data, x0 = _wide_cases()["gauss_diag_d100"]
    m, n = x0.shape[0], 80
    tg = eng.target(w["kind"], w["d"], w["params"])
    a = eng.job(tg, "slice", m, n, x0=x0, seed=2, prec="fp32")
    b = eng.job(tg, "slice", m, n, x0=x0, seed=2, prec="fp32")
    a.run("fsm")
    b.run("sync")
    (ca, pa, _), (cb, pb, _) = a.loop_counts(), b.loop_counts()
    assert np.array_equal(ca, cb) and np.array_equal(pa, pb) and np.array_equal(a.samples(), b.samples())
    ref = O.transitions("slice", w["kind"], w["params"],
                        np.concatenate([x0.astype(np.float32).astype(np.float64)[:, None, :],
                                        a.samples()[:, :-1, :]], axis=1).reshape(m * n, -1),
                        np.repeat(np.arange(m), n), np.tile(np.arange(n), m), seed=2, algo_params=[1.0, 100])
    transitions_agree(a.samples().reshape(m * n, -1), ca.ravel(), ref, "fp32 slice chain per warp d=100")
    a.close()
    b.close()
