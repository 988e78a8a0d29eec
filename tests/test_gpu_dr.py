"""CUDA 3-stage delayed rejection vs the FP64 oracle, through the C ABI (libfsmc.so)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_17405_b300 import workloads as W
from parity import FLIP_ALLOW, compare

pytestmark = pytest.mark.gpu

DR = {"n_stages": 3, "scale0": 1.0, "factor": 0.5}
DR_ARGS = [3, 1.0, 0.5]


@pytest.fixture(scope="module")
def eng():
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    e = fsmc.Engine(0)
    yield e
    e.close()


def _run(eng, kind, d, params, m, n, x0, prec, mode="fsm", seed=1, tuning=None, n_data=0):
    tg = eng.target(kind, d, params, n_data=n_data)
    job = eng.job(tg, "dr", m, n, x0=x0, seed=seed, prec=prec, dr=DR, tuning=tuning)
    job.run(mode)
    return job


@pytest.mark.parametrize("mode", ["fsm", "sync"])
def test_fp64_funnel_matches_oracle(eng, mode):
    m, n = 256, 500
    x0 = W.x0_funnel_exact(m)
    job = _run(eng, "funnel", 10, None, m, n, x0, "fp64", mode)
    ref = O.run("dr", "funnel", np.zeros(1), x0, n, seed=1, algo_params=DR_ARGS)
    counts, _, steps = job.loop_counts()
    compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    if mode == "fsm":
        # one PROPOSE step per stage tried
        assert np.array_equal(steps, counts.sum(1))
    else:
        assert job.stats()["sync_iterations"] == int(counts.max(0).sum())
    job.close()


def test_fp64_gauss_diag_matches_oracle(eng):
    w = W.gauss_diag(5)
    m, n = 64, 300
    x0 = W.x0_gauss_diag_exact(w, m)
    job = _run(eng, "gauss_diag", 5, w["params"], m, n, x0, "fp64")
    ref = O.run("dr", "gauss_diag", w["params"], x0, n, seed=1, algo_params=DR_ARGS)
    counts, _, _ = job.loop_counts()
    compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    job.close()


def test_fp32_funnel_matches_oracle_until_branch_flip(eng):
    m, n = 512, 1000
    x0 = W.x0_funnel_exact(m)
    job = _run(eng, "funnel", 10, None, m, n, x0, "fp32")
    ref = O.run("dr", "funnel", np.zeros(1), x0, n, seed=1, algo_params=DR_ARGS)
    counts, _, _ = job.loop_counts()
    r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp32")
    print("fp32 funnel parity", r["flipped"], "flipped of", m, "max err", r["max_err"])
    assert r["flipped"] <= FLIP_ALLOW
    job.close()


def test_sync_and_fsm_identical_fp32(eng):
    m, n = 4096, 100
    x0 = W.x0_funnel_exact(m)
    a = _run(eng, "funnel", 10, None, m, n, x0, "fp32", "fsm")
    b = _run(eng, "funnel", 10, None, m, n, x0, "fp32", "sync")
    assert np.array_equal(a.loop_counts()[0], b.loop_counts()[0])
    assert np.array_equal(a.samples(), b.samples())
    a.close()
    b.close()


@pytest.fixture(scope="module")
def full_funnel_job(eng):
    """65536 chains x 5000 samples, FP32: the delayed-rejection benchmark configuration."""
    m, n = 65536, 5000
    x0 = W.x0_funnel_exact(m)
    job = _run(eng, "funnel", 10, None, m, n, x0, "fp32")
    yield x0, job
    job.close()


def test_full_size_funnel_sampled_chains(full_funnel_job):
    """The oracle recomputes 64 chains of the full-size run over their first 1000 samples."""
    x0, job = full_funnel_job
    nref = 1000
    counts, _, _ = job.loop_counts()
    assert counts.min() >= 1 and counts.max() <= 3
    flipped = 0
    for chain in np.linspace(0, 65535, 64).astype(int):
        ref = O.run("dr", "funnel", np.zeros(1), x0[chain:chain + 1], nref, seed=1, chain0=int(chain),
                    algo_params=DR_ARGS)
        r = compare(job.samples(int(chain), 1, 0, nref), counts[chain:chain + 1, :nref], ref["samples"],
                    ref["counts"], "fp32")
        flipped += r["flipped"]
        if r["flipped"]:
            print("chain", chain, "flip at", r["first_flip"], "max err", r["max_err"])
    print("DR full size: %d of 64 sampled chains flipped in 1000 samples" % flipped)
    assert flipped <= FLIP_ALLOW


SDR = {"n_stages": 100, "scale0": 0.1, "factor": 1.0, "symmetric": 1}


@pytest.mark.parametrize("mode", ["fsm", "sync"])
def test_fp64_symmetric_dr_on_standard_normal_matches_oracle(eng, mode):
    # the paper's toy experiment (Sec. 7.1): N(0, 1), re-centred tries of sd 0.1, M = 100
    m, n = 256, 400
    params = np.array([0.0, 1.0])
    x0 = np.random.default_rng(5).standard_normal((m, 1))
    tg = eng.target("gauss_diag", 1, params)
    job = eng.job(tg, "dr", m, n, x0=x0, seed=2, prec="fp64", dr=SDR, tuning={"steps_per_launch": 40})
    job.run(mode)
    ref = O.run("sdr", "gauss_diag", params, x0, n, seed=2, algo_params=[100, 0.1])
    counts, _, steps = job.loop_counts()
    r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert r["max_err"] <= 1e-10
    assert counts.max() > 5  # some samples need many tries
    if mode == "fsm":
        assert np.array_equal(steps, counts.sum(1))
    else:
        assert job.stats()["sync_iterations"] == int(counts.max(0).sum())
    job.close()


def test_fp64_symmetric_dr_diag_gaussian_matches_oracle(eng):
    w = W.gauss_diag(3)
    m, n = 128, 300
    x0 = W.x0_gauss_diag_exact(w, m)
    sdr = {"n_stages": 20, "scale0": 0.5, "factor": 1.0, "symmetric": 1}
    tg = eng.target("gauss_diag", 3, w["params"])
    job = eng.job(tg, "dr", m, n, x0=x0, seed=4, prec="fp64", dr=sdr)
    job.run("fsm")
    ref = O.run("sdr", "gauss_diag", w["params"], x0, n, seed=4, algo_params=[20, 0.5])
    counts, _, _ = job.loop_counts()
    r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert r["max_err"] <= 1e-10
    job.close()


def test_fp32_symmetric_dr_sync_and_fsm_identical(eng):
    m, n = 2048, 300
    params = np.array([0.0, 1.0])
    x0 = np.random.default_rng(6).standard_normal((m, 1))
    tg = eng.target("gauss_diag", 1, params)
    out = []
    for mode in ("fsm", "sync"):
        job = eng.job(tg, "dr", m, n, x0=x0, seed=3, prec="fp32", dr=SDR)
        job.run(mode)
        out.append((job.samples(), job.loop_counts()[0]))
        job.close()
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_moments_only_mode_matches_stored_samples(eng, prec, rtol):
    # moments-only DR jobs keep each chain's compensated sums in shared memory during a launch
    # (one device-memory read and write per chain and launch); short launches make the sums
    # cross many launches
    m, n = 512, 400
    x0 = W.x0_funnel_exact(m)
    tg = eng.target("funnel", 10)
    a = eng.job(tg, "dr", m, n, x0=x0, seed=5, prec=prec, dr=DR, tuning={"steps_per_launch": 64})
    b = eng.job(tg, "dr", m, n, x0=x0, seed=5, prec=prec, dr=DR, store=False, tuning={"steps_per_launch": 64})
    a.run("fsm")
    b.run("fsm")
    xs = a.samples()
    sx, sx2, nk = b.moments()
    assert np.all(nk == n)
    assert np.allclose(sx, xs.sum(1), rtol=rtol, atol=rtol * n)
    assert np.allclose(sx2, (xs ** 2).sum(1), rtol=rtol, atol=rtol * n)
    a.close()
    b.close()


# ---- a chain per warp (d > 32) ------------------------------------------------------------------
WIDE = {
    "gauss_diag_d100": lambda: (W.gauss_diag(100), None),
    "funnel_d50": lambda: (W.funnel(50), None),
    "mog_d100": lambda: (W.mog(100, rho=0.5, offsets=(-3.0, 0.0, 3.0), weights=(1.0, 2.0, 1.0)), 3),
}


def _wide_x0(name, w, m):
    if name.startswith("gauss_diag"):
        return W.x0_gauss_diag_exact(w, m)
    if name.startswith("funnel"):
        return W.x0_funnel_exact(m, d=w["d"])
    return W.x0_mog_exact(w, m)


@pytest.mark.parametrize("mode", ["fsm", "sync"])
@pytest.mark.parametrize("name", list(WIDE))
def test_fp64_chain_per_warp_matches_oracle(eng, name, mode):
    # d > 32 runs a chain per warp (the density's sums across the warp); FP64 reproduces the oracle
    # to 1e-10 with identical stage counts; 100 chains leave the last block ragged
    w, n_data = WIDE[name]()
    n_data = n_data or 0
    m, n = 100, 120
    x0 = _wide_x0(name, w, m)
    tg = eng.target(w["kind"], w["d"], w["params"] if w["params"].size else None, n_data=n_data)
    job = eng.job(tg, "dr", m, n, x0=x0, seed=2, prec="fp64", dr=DR, tuning={"steps_per_launch": 40})
    assert job.tuning()["lanes_per_chain"] == 32
    job.run(mode)
    ref = O.run("dr", w["kind"], w["params"], x0, n, seed=2, n_data=n_data, algo_params=DR_ARGS)
    counts, _, steps = job.loop_counts()
    r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert r["max_err"] <= 1e-10
    assert counts.max() == 3  # every stage is exercised
    if mode == "fsm":
        assert np.array_equal(steps, counts.sum(1))
    else:
        assert job.stats()["sync_iterations"] == int(counts.max(0).sum())
    job.close()


@pytest.mark.parametrize("mode", ["fsm", "sync"])
def test_fp64_symmetric_dr_chain_per_warp_matches_oracle(eng, mode):
    w = W.gauss_diag(100)
    m, n = 64, 80
    x0 = W.x0_gauss_diag_exact(w, m)
    sdr = {"n_stages": 30, "scale0": 0.05, "factor": 1.0, "symmetric": 1}
    tg = eng.target("gauss_diag", 100, w["params"])
    job = eng.job(tg, "dr", m, n, x0=x0, seed=6, prec="fp64", dr=sdr)
    job.run(mode)
    ref = O.run("sdr", "gauss_diag", w["params"], x0, n, seed=6, algo_params=[30, 0.05])
    counts, _, _ = job.loop_counts()
    r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert r["max_err"] <= 1e-10
    assert counts.max() > 2
    job.close()


def test_fp32_chain_per_warp_fsm_equals_sync_and_follows_oracle(eng):
    w = W.gauss_diag(64)
    m, n = 256, 300
    x0 = W.x0_gauss_diag_exact(w, m)
    tg = eng.target("gauss_diag", 64, w["params"])
    a = eng.job(tg, "dr", m, n, x0=x0, seed=3, prec="fp32", dr=DR)
    b = eng.job(tg, "dr", m, n, x0=x0, seed=3, prec="fp32", dr=DR)
    a.run("fsm")
    b.run("sync")
    ca, cb = a.loop_counts()[0], b.loop_counts()[0]
    assert np.array_equal(ca, cb) and np.array_equal(a.samples(), b.samples())
    ref = O.run("dr", "gauss_diag", w["params"], x0, n, seed=3, algo_params=DR_ARGS)
    r = compare(a.samples(), ca, ref["samples"], ref["counts"], "fp32")
    print("fp32 DR chain per warp d=64:", r["flipped"], "flipped of", m, "max err", r["max_err"])
    assert r["flipped"] <= FLIP_ALLOW
    a.close()
    b.close()


def test_chain_per_warp_moments_only_matches_stored_samples(eng):
    w = W.funnel(40)
    m, n = 96, 200
    x0 = W.x0_funnel_exact(m, d=40)
    tg = eng.target("funnel", 40)
    a = eng.job(tg, "dr", m, n, x0=x0, seed=5, prec="fp64", dr=DR)
    b = eng.job(tg, "dr", m, n, x0=x0, seed=5, prec="fp64", dr=DR, store=False)
    a.run("fsm")
    b.run("fsm")
    xs = a.samples()
    sx, sx2, nk = b.moments()
    assert np.all(nk == n)
    assert np.allclose(sx, xs.sum(1), rtol=1e-12, atol=1e-10)
    assert np.allclose(sx2, (xs ** 2).sum(1), rtol=1e-12, atol=1e-10)
    a.close()
    b.close()


def test_chain_per_warp_shape_checks(eng):
    from paper_2503_17405_b300 import fsmc
    w = W.gauss_diag(40)
    tg = eng.target("gauss_diag", 40, w["params"])
    for bad in ({"lanes_per_chain": 1}, {"step_form": 2}, {"lanes_per_chain": 16}):
        with pytest.raises(fsmc.FsmcError):
            eng.job(tg, "dr", 8, 4, dr=DR, tuning=bad)
