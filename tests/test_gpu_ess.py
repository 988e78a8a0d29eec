"""CUDA elliptical slice sampling vs the FP64 oracle, through the C ABI (libfsmc.so)."""
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


def _run(eng, w, m, n, x0, prec, mode="fsm", seed=1, tuning=None, store=True):
    tg = eng.target(w["kind"], w["d"], w["params"])
    job = eng.job(tg, "ess", m, n, x0=x0, seed=seed, prec=prec, tuning=tuning, store=store)
    job.run(mode)
    return job


@pytest.mark.parametrize("lanes", [1, 32])
@pytest.mark.parametrize("mode", ["fsm", "sync"])
def test_fp64_conjugate_gaussian_matches_oracle(eng, lanes, mode):
    # ESS on the conjugate Gaussian, d = 16, 128 chains x 1000 samples, FP64
    w = W.gauss_conj(16)
    m, n = 128, 1000
    x0 = W.x0_zeros(m, 16)
    job = _run(eng, w, m, n, x0, "fp64", mode, tuning={"lanes_per_chain": lanes})
    ref = O.run("ess", "gauss_conj", w["params"], x0, n, seed=1)
    counts, _, steps = job.loop_counts()
    r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert r["max_err"] <= 1e-10
    st = job.stats()
    if mode == "fsm":
        # every FSM step runs exactly one likelihood evaluation: N + 1 per sample
        assert np.array_equal(steps, (counts + 1).sum(1))
    else:
        # the synchronised loop runs max_j N_ij body iterations per sample (Sec. 2.2)
        assert st["sync_iterations"] == int(counts.max(0).sum())
    job.close()


@pytest.mark.parametrize("mode", ["fsm", "sync"])
def test_fp64_long_shrink_sequences_match_oracle(eng, mode):
    # A likelihood 250 times narrower than the prior (noise sd 0.002) makes most samples shrink
    # the bracket more than 15 times, so chain-per-warp runs take their random numbers from
    # the lane cache's wide layout (draws 16 and beyond of a sample) as well as the two-sample
    # narrow one.
    w = W.gauss_conj(16, noise_sd=0.002)
    m, n = 64, 100
    x0 = np.tile(w["post_mean"][None, :], (m, 1))
    job = _run(eng, w, m, n, x0, "fp64", mode, tuning={"lanes_per_chain": 32})
    ref = O.run("ess", "gauss_conj", w["params"], x0, n, seed=1)
    counts, _, _ = job.loop_counts()
    assert (ref["counts"] >= 16).mean() > 0.25
    r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert r["max_err"] <= 1e-10
    job.close()


def test_fp32_gp_logit_matches_oracle_until_branch_flip(eng):
    w = W.gp_logit(256)
    m, n = 48, 400
    x0 = W.x0_zeros(m, 256)
    job = _run(eng, w, m, n, x0, "fp32")
    ref = O.run("ess", "gp_logit", w["params"], x0, n, seed=1)
    counts, _, _ = job.loop_counts()
    r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp32")
    print("fp32 gp-logit parity", r["flipped"], "flipped of", m, "max err", r["max_err"])
    assert r["flipped"] <= FLIP_ALLOW
    job.close()


def test_fp32_gp_logit_overflowing_group_products_match_oracle(eng):
    # Chains start at x = -20 s: every coordinate has t' = 20 log2(e) ~ 28.9, so each lane's
    # group of eight factors 1 + 2^t' (coordinates l, l + 32, ..., l + 224) exceeds 2^126 in single
    # precision and the likelihood takes its per-coordinate form until the chains move inwards.
    w = W.gp_logit(256)
    m, n = 32, 60
    x0 = np.tile(-20.0 * w["s"][None, :], (m, 1))
    t = (-w["s"] * x0[0] * np.log2(np.e)).astype(np.float32)
    with np.errstate(over="ignore"):
        groups = (1.0 + np.exp2(t)).reshape(8, 32).prod(axis=0, dtype=np.float32)
    assert (groups > np.float32(2.0 ** 126)).all()
    a = _run(eng, w, m, n, x0, "fp32", "fsm")
    b = _run(eng, w, m, n, x0, "fp32", "sync")
    ref = O.run("ess", "gp_logit", w["params"], x0, n, seed=1)
    ca, _, _ = a.loop_counts()
    cb, _, _ = b.loop_counts()
    assert np.array_equal(ca, cb) and np.array_equal(a.samples(), b.samples())
    r = compare(a.samples(), ca, ref["samples"], ref["counts"], "fp32")
    print("overflowing products: flipped", r["flipped"], "of", m, "max err", r["max_err"])
    assert r["flipped"] <= FLIP_ALLOW
    a.close()
    b.close()


@pytest.mark.parametrize("d", [100, 200, 256])
def test_tensor_core_generator_matches_oracle(eng, d):
    """The tcgen05 direction generator (FP16 hi/lo splits, FP32 accumulation) and the CUDA-core
    generator both follow the oracle to the FP32 tolerance."""
    w = W.gp_logit(d)
    m, n = 96, 150
    x0 = W.x0_zeros(m, d)
    ref = O.run("ess", "gp_logit", w["params"], x0, n, seed=1)
    for gen in (2, 1):
        job = _run(eng, w, m, n, x0, "fp32", tuning={"generator": gen})
        assert job.tuning()["generator"] == gen
        counts, _, _ = job.loop_counts()
        r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp32")
        print("generator", gen, "d", d, "flipped", r["flipped"], "max err", r["max_err"])
        assert r["flipped"] <= FLIP_ALLOW
        job.close()


@pytest.mark.parametrize("lanes", [8, 16])
@pytest.mark.parametrize("mode", ["fsm", "sync"])
def test_several_chains_per_warp_fp64_matches_oracle(eng, mode, lanes):
    # 8 or 16 lanes per chain (four or two chains share a warp), d = 48 (ragged lanes),
    # 100 chains (ragged last warp); FP64 gives the oracle's loop counts exactly
    w = W.gauss_conj(48)
    m, n = 100, 300
    x0 = W.x0_normal(m, 48, scale=0.3)
    job = _run(eng, w, m, n, x0, "fp64", mode, tuning={"lanes_per_chain": lanes, "steps_per_launch": 24})
    assert job.tuning()["lanes_per_chain"] == lanes
    ref = O.run("ess", "gauss_conj", w["params"], x0, n, seed=1)
    counts, _, steps = job.loop_counts()
    r = compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    assert r["max_err"] <= 1e-10
    if mode == "fsm":
        assert np.array_equal(steps, (counts + 1).sum(1))
    job.close()


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_fp32_gp_logit_lanes_match_oracle_and_sync(eng, lanes):
    # the single-precision base-2 GP-logit likelihood: FSM and synchronised kernels agree bit
    # for bit, and both follow the oracle to the FP32 tolerance (d = 200: ragged rows)
    w = W.gp_logit(200)
    m, n = 72, 150
    x0 = W.x0_normal(m, 200, scale=0.1)
    tu = {"lanes_per_chain": lanes, "generator": 2}
    a = _run(eng, w, m, n, x0, "fp32", "fsm", tuning=tu)
    b = _run(eng, w, m, n, x0, "fp32", "sync", tuning=tu)
    ca, _, steps = a.loop_counts()
    cb, _, _ = b.loop_counts()
    assert np.array_equal(ca, cb)
    assert np.array_equal(a.samples(), b.samples())
    # states counted one likelihood evaluation each, whatever the step evaluates ahead
    assert np.array_equal(steps, (ca + 1).sum(1))
    ref = O.run("ess", "gp_logit", w["params"], x0, n, seed=1)
    r = compare(a.samples(), ca, ref["samples"], ref["counts"], "fp32")
    print("lanes", lanes, "flipped", r["flipped"], "max err", r["max_err"])
    assert r["flipped"] <= FLIP_ALLOW
    a.close()
    b.close()


def test_gp_logit_labels_must_be_signs(eng):
    from paper_2503_17405_b300 import fsmc
    w = W.gp_logit(8)
    p = np.array(w["params"], dtype=np.float64)
    p[8 * 8 + 3] = 0.5
    with pytest.raises(fsmc.FsmcError):
        eng.target("gp_logit", 8, p)


def test_sync_and_fsm_give_identical_samples(eng):
    w = W.gp_logit(256)
    m, n = 300, 64
    x0 = W.x0_normal(m, 256, scale=0.1)
    a = _run(eng, w, m, n, x0, "fp32", "fsm")
    b = _run(eng, w, m, n, x0, "fp32", "sync")
    ca, _, _ = a.loop_counts()
    cb, _, _ = b.loop_counts()
    assert np.array_equal(ca, cb)
    assert np.array_equal(a.samples(), b.samples())
    assert b.stats()["sync_iterations"] == int(cb.max(0).sum())
    a.close()
    b.close()


def test_flat_likelihood_never_shrinks(eng):
    w = W.flat(8)
    m = 64
    x0 = W.x0_normal(m, 8) @ w["L"].T
    job = _run(eng, w, m, 50, x0, "fp64", tuning={"lanes_per_chain": 1})
    counts, _, _ = job.loop_counts()
    assert np.all(counts == 0)
    ref = O.run("ess", "flat", w["params"], x0, 50, seed=1)
    compare(job.samples(), counts, ref["samples"], ref["counts"], "fp64")
    job.close()


def test_resume_from_snapshot_is_bit_exact(eng):
    w = W.gauss_conj(16)
    m, n = 96, 300
    x0 = W.x0_normal(m, 16)
    whole = _run(eng, w, m, n, x0, "fp32", tuning={"lanes_per_chain": 32, "steps_per_launch": 16})
    tg = eng.target("gauss_conj", 16, w["params"])
    part = eng.job(tg, "ess", m, n, x0=x0, seed=1, prec="fp32",
                   tuning={"lanes_per_chain": 32, "steps_per_launch": 16})
    part.run("fsm", max_fsm_steps=100)
    mn, done = part.progress()
    assert not done and mn > 0
    blob = part.snapshot()
    part.close()
    fresh = eng.job(tg, "ess", m, n, x0=x0, seed=1, prec="fp32",
                    tuning={"lanes_per_chain": 32, "steps_per_launch": 16})
    fresh.restore(blob)
    fresh.run("fsm")
    assert np.array_equal(fresh.samples(), whole.samples())
    assert np.array_equal(fresh.loop_counts()[0], whole.loop_counts()[0])
    whole.close()
    fresh.close()


def test_moments_only_mode_matches_stored_samples(eng):
    w = W.gauss_conj(16)
    m, n = 64, 200
    x0 = W.x0_normal(m, 16)
    a = _run(eng, w, m, n, x0, "fp64", store=True)
    b = _run(eng, w, m, n, x0, "fp64", store=False)
    xs = a.samples()
    sx, sx2, nk = b.moments()
    assert np.all(nk == n)
    assert np.allclose(sx, xs.sum(1), rtol=1e-12, atol=1e-10)
    assert np.allclose(sx2, (xs ** 2).sum(1), rtol=1e-12, atol=1e-10)
    with pytest.raises(Exception):
        b.samples(0, 1, 0, 1)
    a.close()
    b.close()


def test_fp32_gp_logit_moments_only_matches_stored_samples(eng):
    # full 32-lane rows (d = 256): the moments-only FSM kernel keeps each lane's sums in shared
    # memory for the length of a launch; short launches make the sums cross many of them
    w = W.gp_logit(256)
    m, n = 128, 150
    x0 = W.x0_normal(m, 256, scale=0.3)
    tu = {"steps_per_launch": 32}
    a = _run(eng, w, m, n, x0, "fp32", store=True, tuning=tu)
    b = _run(eng, w, m, n, x0, "fp32", store=False, tuning=tu)
    xs = a.samples()
    sx, sx2, nk = b.moments()
    assert np.all(nk == n)
    assert np.allclose(sx, xs.sum(1), rtol=2e-5, atol=2e-5 * n)
    assert np.allclose(sx2, (xs ** 2).sum(1), rtol=2e-5, atol=2e-5 * n)
    a.close()
    b.close()


def test_admission_and_argument_errors(eng):
    from paper_2503_17405_b300 import fsmc
    small = fsmc.Engine(0, hbm_budget_bytes=1 << 20)
    w = W.gp_logit(256)
    tg = small.target("gp_logit", 256, w["params"])
    job = small.job(tg, "ess", 4096, 1000)
    with pytest.raises(fsmc.FsmcError) as ei:
        job.run()
    assert ei.value.status == fsmc.EADMIT
    with pytest.raises(fsmc.FsmcError) as ei:
        small.job(tg, "dr", 4, 10)
    assert ei.value.status == fsmc.EINVAL
    with pytest.raises(fsmc.FsmcError) as ei:
        small.target("gp_logit", 256, w["params"][:-1])
    assert ei.value.status == fsmc.EINVAL
    small.close()


@pytest.fixture(scope="module")
def full_gp_job(eng):
    """16384 chains x 2000 samples, FP32: the benchmark configuration."""
    w = W.gp_logit(256)
    job = _run(eng, w, 16384, 2000, W.x0_zeros(16384, 256), "fp32")
    yield w, job
    job.close()


def test_full_size_gp_logit_sampled_chains(full_gp_job):
    """The oracle recomputes eight chains of the full-size run one by one (the RNG is keyed by
    chain) over the first 1000 samples: within the FP32 tolerance until a flip, flips bounded."""
    w, job = full_gp_job
    nref = 1000
    counts, _, _ = job.loop_counts()
    assert np.all(counts >= 0)
    flipped = 0
    for chain in [0, 2047, 4096, 8191, 8192, 12287, 15000, 16383]:
        ref = O.run("ess", "gp_logit", w["params"], np.zeros((1, 256)), nref, seed=1, chain0=chain)
        x = job.samples(chain, 1, 0, nref)
        r = compare(x, counts[chain:chain + 1, :nref], ref["samples"], ref["counts"], "fp32")
        print("chain", chain, "flip at", r["first_flip"], "max err", r["max_err"])
        flipped += r["flipped"]
    assert flipped <= FLIP_ALLOW


@pytest.mark.parametrize("form", [1, 2, 3])
@pytest.mark.parametrize("case", ["gp_fp32", "gauss_fp64_lanes1", "gauss_fp64_lanes32"])
def test_synchronised_forms_equal_the_fsm(eng, form, case):
    # the three forms of the synchronised program (sweep, compacted list with a grid barrier, graph
    # with conditional while nodes) run the same visits: samples and loop counts equal the FSM
    # run's bit for bit, and the loop ran max_j N_ij iterations per sample
    if case == "gp_fp32":
        w, m, n, prec, tu = W.gp_logit(256), 300, 64, "fp32", {}
        x0 = W.x0_normal(m, 256, scale=0.1)
    else:
        lanes = 1 if case.endswith("1") else 32
        w, m, n, prec, tu = W.gauss_conj(16), 200, 150, "fp64", {"lanes_per_chain": lanes}
        x0 = W.x0_normal(m, 16)
    a = _run(eng, w, m, n, x0, prec, "fsm", tuning=tu)
    b = _run(eng, w, m, n, x0, prec, "sync", tuning={**tu, "sync_form": form})
    assert b.tuning()["sync_form"] == form
    ca, _, _ = a.loop_counts()
    cb, _, _ = b.loop_counts()
    assert np.array_equal(ca, cb)
    assert np.array_equal(a.samples(), b.samples())
    st = b.stats()
    assert st["sync_iterations"] == int(cb.max(0).sum())
    assert st["error_word"] == 0
    a.close()
    b.close()


@pytest.mark.parametrize("d,m,n", [(256, 300, 64), (256, 16384, 12), (64, 1000, 40)])
def test_resident_synchronised_form_equals_the_fsm(eng, d, m, n):
    # the resident sweep (sync_form 4: every chain's state and current direction on chip for the
    # launch) runs the sweep's visits: the FSM's samples and loop counts bit for bit, max_j N_ij
    # iterations per sample; 16384 chains fill seven of the eight slots of every warp of the grid
    w = W.gp_logit(d)
    x0 = W.x0_normal(m, d, scale=0.1)
    tu = {"lanes_per_chain": 32}
    a = _run(eng, w, m, n, x0, "fp32", "fsm", tuning=tu)
    b = _run(eng, w, m, n, x0, "fp32", "sync", tuning={**tu, "sync_form": 4})
    ca, _, _ = a.loop_counts()
    cb, _, _ = b.loop_counts()
    assert np.array_equal(ca, cb)
    assert np.array_equal(a.samples(), b.samples())
    st = b.stats()
    assert st["sync_iterations"] == int(cb.max(0).sum())
    assert st["error_word"] == 0
    a.close()
    b.close()


def test_resident_synchronised_form_refuses_other_jobs(eng):
    from paper_2503_17405_b300 import fsmc
    w = W.gauss_conj(16)
    tg = eng.target("gauss_conj", 16, w["params"])
    with pytest.raises(fsmc.FsmcError, match="sync_form 4"):
        eng.job(tg, "ess", 64, 10, x0=W.x0_normal(64, 16), prec="fp64", tuning={"sync_form": 4})
    g = W.gp_logit(256)
    tg2 = eng.target("gp_logit", 256, g["params"])
    with pytest.raises(fsmc.FsmcError, match="sync_form 4"):
        eng.job(tg2, "ess", 64, 10, x0=W.x0_normal(64, 256), prec="fp64", tuning={"sync_form": 4})


def test_synchronised_sweep_with_more_chains_than_its_live_masks_cover(eng):
    # the sweep form keeps a 32-bit mask of live chains per chain group while groups have at most
    # 32 chains; 120 000 chains at 32 lanes exceed that (about 3 600 resident groups), so the kernel
    # reads each chain's state id instead -- still the FSM's samples, bit for bit
    w = W.gauss_conj(16)
    m, n = 120_000, 12
    x0 = W.x0_normal(m, 16)
    tu = {"lanes_per_chain": 32}
    a = _run(eng, w, m, n, x0, "fp32", "fsm", tuning=tu)
    b = _run(eng, w, m, n, x0, "fp32", "sync", tuning={**tu, "sync_form": 1})
    ca, cb = a.loop_counts()[0], b.loop_counts()[0]
    assert np.array_equal(ca, cb)
    assert np.array_equal(a.samples(), b.samples())
    assert b.stats()["sync_iterations"] == int(cb.max(0).sum())
    a.close()
    b.close()
