"""Sec. 7.3's NUTS target on the CUDA kernels: the 100-d equicorrelated mixture of Gaussians
(rho = 0.99, modes at -10 * 1, 0, 10 * 1), NUTS in the FSM and synchronised kernels against the
FP64 oracle, a general mixture (unequal weights, negative correlation, ragged lanes), DR on a
mixture, and the target's argument checks."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W
from parity import compare, sample_errors, transitions_agree

pytestmark = pytest.mark.gpu

NUTS = {"eps": 0.044, "max_depth": 10, "max_dH": 1000.0}


@pytest.fixture(scope="module")
def eng():
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    e = fsmc.Engine(0)
    yield e
    e.close()


def _nuts(eng, w, m, n, x0, prec, mode, nuts=NUTS, seed=1):
    tg = eng.target("mog", w["d"], w["params"], n_data=w["n_data"])
    job = eng.job(tg, "nuts", m, n, x0=x0, seed=seed, prec=prec, nuts=nuts)
    job.run(mode)
    return job


def _oracle_nuts(w, x0, n, nuts=NUTS, seed=1):
    return O.run("nuts", "mog", w["params"], x0, n, seed=seed, n_data=w["n_data"],
                 algo_params=[nuts["eps"], nuts["max_depth"], nuts["max_dH"]])


@pytest.mark.parametrize("mode", ["fsm", "sync"])
def test_fp64_papers_mixture_matches_oracle(eng, mode):
    w = W.mog(100)
    m, n = 48, 40
    x0 = W.x0_mog_exact(w, m)
    job = _nuts(eng, w, m, n, x0, "fp64", mode)
    ref = _oracle_nuts(w, x0, n)
    counts, depth, steps = job.loop_counts()
    compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert np.array_equal(depth, ref["aux"])
    assert counts.max() >= 500          # the heavy tail of trajectory lengths is exercised
    if mode == "fsm":
        assert np.array_equal(steps, counts.sum(1))
    job.close()


def test_fp64_general_mixture_matches_oracle(eng):
    # d = 37 (two registers per lane, ragged), K = 4, unequal weights, negative correlation
    d, K = 37, 4
    r = np.random.default_rng(21)
    mu = r.normal(0.0, 1.5, (K, d))
    wts = r.uniform(0.3, 2.0, K)
    rho = -0.02
    w = dict(kind="mog", d=d, n_data=K, params=np.concatenate([[rho], wts, mu.ravel()]))
    m, n = 40, 60
    x0 = mu[r.integers(0, K, m)] + 0.5 * r.standard_normal((m, d))
    nuts = {"eps": 0.15, "max_depth": 8, "max_dH": 1000.0}
    for mode in ("fsm", "sync"):
        job = _nuts(eng, w, m, n, x0, "fp64", mode, nuts=nuts, seed=3)
        ref = _oracle_nuts(w, x0, n, nuts=nuts, seed=3)
        counts, _, _ = job.loop_counts()
        compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
        job.close()


def test_fp32_papers_mixture_transition_by_transition(eng):
    # Every FP32 transition against the FP64 oracle's transition from the same (FP32) state with
    # the same random numbers.  Trajectories of up to 1023 leapfrog steps on this ill-conditioned
    # target (condition number (1 + 99 rho) / (1 - rho) ~ 1e4) make whole-chain comparison end at
    # the first near-tie of a multinomial or U-turn decision, and such a flip can move the sample
    # by less than the usual flip threshold (to another leaf of the same trajectory); one
    # transition at a time, rounding error and flipped decisions separate cleanly.
    w = W.mog(100)
    m, n = 64, 60
    x0 = W.x0_mog_exact(w, m).astype(np.float32).astype(np.float64)
    job = _nuts(eng, w, m, n, x0, "fp32", "fsm")
    xs = job.samples().astype(np.float64)
    counts, _, _ = job.loop_counts()
    job.close()
    starts = np.concatenate([x0[:, None, :], xs[:, :-1, :]], axis=1).reshape(m * n, -1)
    ref = O.transitions("nuts", "mog", w["params"], starts, np.repeat(np.arange(m), n), np.tile(np.arange(n), m),
                        seed=1, n_data=3, algo_params=[NUTS["eps"], NUTS["max_depth"], NUTS["max_dH"]])
    ok = transitions_agree(xs.reshape(m * n, -1), counts.ravel(), ref, "fp32 mog")
    assert sample_errors(xs.reshape(m * n, -1), ref["x"])[ok].max() <= 2e-5


def test_fp32_fsm_and_sync_agree(eng):
    w = W.mog(100)
    m, n = 256, 30
    x0 = W.x0_mog_exact(w, m)
    a = _nuts(eng, w, m, n, x0, "fp32", "fsm")
    b = _nuts(eng, w, m, n, x0, "fp32", "sync")
    ca, _, _ = a.loop_counts()
    cb, _, _ = b.loop_counts()
    r = compare(a.samples(), ca, b.samples(), cb, "fp32")
    print("fp32 mog FSM vs sync:", r["flipped"], "flipped of", m)
    assert r["flipped"] <= m // 8
    st = b.stats()
    assert st["sync_iterations"] >= int(cb.max(0).sum())
    a.close()
    b.close()


@pytest.mark.parametrize("symmetric", [0, 1])
def test_fp64_dr_on_a_mixture_matches_oracle(eng, symmetric):
    w = W.mog(10, rho=0.5, offsets=(-3.0, 0.0, 3.0), weights=(1.0, 2.0, 1.0))
    m, n = 128, 150
    x0 = W.x0_mog_exact(w, m)
    tg = eng.target("mog", 10, w["params"], n_data=3)
    if symmetric:
        dr, algo, ap = {"n_stages": 20, "scale0": 0.4, "factor": 1.0, "symmetric": 1}, "sdr", [20, 0.4]
    else:
        dr, algo, ap = {"n_stages": 3, "scale0": 1.0, "factor": 0.5}, "dr", [3, 1.0, 0.5]
    for mode in ("fsm", "sync"):
        job = eng.job(tg, "dr", m, n, x0=x0, seed=4, prec="fp64", dr=dr)
        job.run(mode)
        ref = O.run(algo, "mog", w["params"], x0, n, seed=4, n_data=3, algo_params=ap)
        counts, _, _ = job.loop_counts()
        compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
        job.close()


def test_mixture_argument_checks(eng):
    from paper_2503_17405_b300 import fsmc
    d = 5
    mu = np.zeros((2, d))
    bad = [
        np.concatenate([[1.0], [1.0, 1.0], mu.ravel()]),          # rho = 1
        np.concatenate([[-0.25], [1.0, 1.0], mu.ravel()]),        # rho = -1/(d-1): singular
        np.concatenate([[0.5], [1.0, 0.0], mu.ravel()]),          # zero weight
        np.concatenate([[0.5], [1.0, 1.0], mu.ravel() + np.inf]), # non-finite mean
    ]
    for p in bad:
        with pytest.raises(fsmc.FsmcError):
            eng.target("mog", d, p, n_data=2)
    with pytest.raises(fsmc.FsmcError):
        eng.target("mog", d, np.zeros(1), n_data=0)               # no components
    tg = eng.target("mog", d, np.concatenate([[0.5], [1.0, 1.0], mu.ravel()]), n_data=2)
    with pytest.raises(fsmc.FsmcError):
        eng.job(tg, "ess", 8, 4, prec="fp32")                      # ESS needs a prior factor
