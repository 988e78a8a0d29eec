"""CUDA NUTS (iterative, FSM) vs the recursive FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W
from parity import FLIP_ALLOW, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    e = fsmc.Engine(0)
    yield e
    e.close()


def _run(eng, kind, d, params, m, n, x0, prec, nuts, mode="fsm", seed=1, n_data=0, tuning=None):
    tg = eng.target(kind, d, params, n_data=n_data)
    job = eng.job(tg, "nuts", m, n, x0=x0, seed=seed, prec=prec, nuts=nuts, tuning=tuning)
    job.run(mode)
    return job


def _oracle(kind, params, x0, n, nuts, n_data=0, chain0=0):
    return O.run("nuts", kind, params, x0, n, seed=1, n_data=n_data, chain0=chain0,
                 algo_params=[nuts["eps"], nuts["max_depth"], nuts["max_dH"]])


@pytest.mark.parametrize("mode", ["fsm", "sync"])
def test_fp64_gauss_diag_matches_oracle(eng, mode):
    w = W.gauss_diag(8)
    nuts = {"eps": 0.2, "max_depth": 10, "max_dH": 1000.0}
    m, n = 64, 200
    x0 = W.x0_gauss_diag_exact(w, m)
    job = _run(eng, "gauss_diag", 8, w["params"], m, n, x0, "fp64", nuts, mode)
    ref = _oracle("gauss_diag", w["params"], x0, n, nuts)
    counts, depth, steps = job.loop_counts()
    compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert np.array_equal(depth, ref["aux"])
    if mode == "fsm":
        assert np.array_equal(steps, counts.sum(1))   # one leapfrog per FSM step
    job.close()


@pytest.mark.parametrize("mode", ["fsm", "sync"])
def test_fp64_logreg_and_funnel_match_oracle(eng, mode):
    w = W.logreg(100, 5)
    nuts = {"eps": 0.05, "max_depth": 10, "max_dH": 1000.0}
    m, n = 32, 100
    x0 = W.x0_logreg(w, m)
    job = _run(eng, "logreg", 5, w["params"], m, n, x0, "fp64", nuts, mode, n_data=100)
    ref = _oracle("logreg", w["params"], x0, n, nuts, n_data=100)
    counts, depth, steps = job.loop_counts()
    compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert np.array_equal(depth, ref["aux"])
    if mode == "fsm":
        assert np.array_equal(steps, counts.sum(1))
    job.close()
    if mode == "sync":
        return
    nuts = {"eps": 0.2, "max_depth": 6, "max_dH": 1000.0}
    x0 = W.x0_funnel_exact(32)
    job = _run(eng, "funnel", 10, None, 32, 100, x0, "fp64", nuts)
    ref = _oracle("funnel", np.zeros(1), x0, 100, nuts)
    counts, depth, _ = job.loop_counts()
    compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    job.close()


def test_fp64_wide_logreg_three_registers_per_lane(eng):
    # d = 70 exercises the multi-element-per-lane layout
    w = W.logreg(200, 70)
    nuts = {"eps": 0.02, "max_depth": 8, "max_dH": 1000.0}
    m, n = 8, 30
    x0 = W.x0_logreg(w, m)
    job = _run(eng, "logreg", 70, w["params"], m, n, x0, "fp64", nuts, n_data=200)
    ref = _oracle("logreg", w["params"], x0, n, nuts, n_data=200)
    counts, _, _ = job.loop_counts()
    compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    job.close()


def test_fp32_logreg_matches_oracle_until_branch_flip(eng):
    w = W.logreg(1000, 25)
    nuts = {"eps": 0.05, "max_depth": 10, "max_dH": 1000.0}
    m, n = 32, 200
    x0 = W.x0_logreg(w, m)
    job = _run(eng, "logreg", 25, w["params"], m, n, x0, "fp32", nuts, n_data=1000)
    ref = _oracle("logreg", w["params"], x0, n, nuts, n_data=1000)
    counts, _, _ = job.loop_counts()
    r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp32")
    print("fp32 logreg parity", r["flipped"], "flipped of", m, "max err", r["max_err"],
          "first flips", r["first_flip"])
    assert r["flipped"] <= FLIP_ALLOW
    job.close()


def test_sync_and_fsm_identical_fp32(eng):
    # both kernels compute the logistic gradient batched over a block's chains, and a chain's
    # gradient does not depend on which chains share its block: FSM and synchronised runs give
    # the same samples, leapfrog counts and tree depths bit for bit
    w = W.logreg(1000, 25)
    nuts = {"eps": 0.05, "max_depth": 10, "max_dH": 1000.0}
    m, n = 256, 20
    x0 = W.x0_logreg(w, m)
    a = _run(eng, "logreg", 25, w["params"], m, n, x0, "fp32", nuts, "fsm", n_data=1000)
    b = _run(eng, "logreg", 25, w["params"], m, n, x0, "fp32", nuts, "sync", n_data=1000)
    ca, da, _ = a.loop_counts()
    cb, db, _ = b.loop_counts()
    assert np.array_equal(ca, cb) and np.array_equal(da, db)
    assert np.array_equal(a.samples(), b.samples())
    st = b.stats()
    # the nested synchronised loops run at least max_j N_ij leapfrog iterations per sample
    assert st["sync_iterations"] >= int(cb.max(0).sum())
    a.close()
    b.close()


def test_balanced_grid_with_more_groups_than_resident_blocks(eng):
    """5000 chains are 625 groups of eight, more than the blocks that can be resident (two per
    SM), so each block of the batched FSM launch runs several groups with balanced budgets and
    the assignment rotates from launch to launch.  Which launch runs a state must not change any
    chain: the samples equal the synchronised program's bit for bit, and a run stopped after a
    few launches and resumed from a snapshot in a fresh job equals the uninterrupted run."""
    w = W.logreg(1000, 25)
    nuts = {"eps": 0.05, "max_depth": 10, "max_dH": 1000.0}
    m, n = 5000, 12
    x0 = W.x0_logreg(w, m)
    tg = eng.target("logreg", 25, w["params"], n_data=1000)
    tu = {"steps_per_launch": 16}

    def job():
        return eng.job(tg, "nuts", m, n, x0=x0, seed=1, prec="fp32", nuts=nuts, tuning=tu)

    a = job()
    a.run("fsm")
    ca, da, sa = a.loop_counts()
    assert (sa > 16 * 4).all()  # every chain ran over several launches
    b = job()
    b.run("sync")
    cb, db, _ = b.loop_counts()
    assert np.array_equal(ca, cb) and np.array_equal(da, db)
    assert np.array_equal(a.samples(), b.samples())
    b.close()
    part = job()
    part.run("fsm", max_fsm_steps=48)
    assert not part.progress()[1]
    blob = part.snapshot()
    part.close()
    fresh = job()
    fresh.restore(blob)
    fresh.run("fsm")
    cf, df, sf = fresh.loop_counts()
    assert np.array_equal(ca, cf) and np.array_equal(da, df) and np.array_equal(sa, sf)
    assert np.array_equal(a.samples(), fresh.samples())
    fresh.close()
    a.close()


@pytest.fixture(scope="module")
def full_nuts_job(eng):
    """4096 chains x 1000 draws of NUTS on logistic regression (1000 x 25), FP32."""
    w = W.logreg(1000, 25)
    nuts = {"eps": 0.05, "max_depth": 10, "max_dH": 1000.0}
    x0 = W.x0_logreg(w, 4096)
    job = _run(eng, "logreg", 25, w["params"], 4096, 1000, x0, "fp32", nuts, n_data=1000)
    yield w, nuts, x0, job
    job.close()


SAMPLED = [0, 511, 1024, 2047, 2048, 3071, 3584, 4095]


def test_full_size_logreg_sampled_chains(full_nuts_job):
    """The oracle recomputes eight chains of the full-size run one by one (the RNG is keyed by
    chain) over all 1000 draws: within the FP32 tolerance until a flip, flips bounded."""
    w, nuts, x0, job = full_nuts_job
    nref = 1000
    counts, _, _ = job.loop_counts()
    assert counts.min() >= 1 and counts.max() <= 1023
    flipped = 0
    for chain in SAMPLED:
        ref = _oracle("logreg", w["params"], x0[chain:chain + 1], nref, nuts, n_data=1000, chain0=chain)
        r = compare(job.samples(chain, 1, 0, nref), counts[chain:chain + 1, :nref], ref["samples"],
                    ref["counts"], "fp32")
        print("chain", chain, "flip at", r["first_flip"], "max err", r["max_err"])
        flipped += r["flipped"]
    assert flipped <= FLIP_ALLOW
