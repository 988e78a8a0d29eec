"""The allocation-free ESS entry point (fsmc_ess_run_static) against fsmc_job_run.

Some callers cannot allocate device memory (a memory planner owns the device, a plugin is
handed buffers but no allocator, or cudaMalloc's implicit synchronisation is not allowed).
fsmc_ess_run_static serves them from a fixed array inside the library.  This test calls it
through the C ABI twice in a row and checks both outputs against the regular job API on
the same inputs, with the FP32 parity tolerance the other tests use.
"""
import numpy as np
import pytest

from paper_2503_17405_b300 import workloads as W
from parity import FP32_TOL, sample_errors

pytestmark = pytest.mark.gpu


def test_static_scratch_run_matches_job_api_twice():
    import torch
    from paper_2503_17405_b300 import build, fsmc

    build.build()
    torch.cuda.set_device(0)
    w = W.gp_logit(256)
    m, n, d = 384, 120, 256
    x0 = W.x0_normal(m, d, scale=0.1)

    eng = fsmc.Engine(0)
    tg = eng.target("gp_logit", d, w["params"])
    # the static-scratch run uses the CUDA-core direction generator: compare like with like
    job = eng.job(tg, "ess", m, n, x0=x0, seed=7, prec="fp32",
                  tuning={"lanes_per_chain": 32, "generator": 1})
    job.run("fsm")
    ref_x = job.samples()
    ref_c, _, _ = job.loop_counts()
    eng.close()

    dev = torch.device("cuda", 0)
    L = torch.tensor(w["L"], dtype=torch.float32, device=dev).contiguous()
    s = torch.tensor(w["s"], dtype=torch.float32, device=dev).contiguous()
    x0_d = torch.tensor(x0, dtype=torch.float32, device=dev).contiguous()
    for call in range(2):
        out = torch.full((m, n, d), float("nan"), dtype=torch.float32, device=dev)
        counts = torch.full((m, n), -7, dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream(dev)
        fsmc.ess_run_static("gp_logit", d, L.data_ptr(), s.data_ptr(), 0.0, m, n, x0_d.data_ptr(),
                            7, 32, out.data_ptr(), counts.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got_c = counts.cpu().numpy()
        got_x = out.cpu().numpy().astype(np.float64)
        assert np.array_equal(got_c, ref_c), f"call {call}: loop counts differ"
        err = sample_errors(got_x, ref_x)
        assert np.isfinite(err).all() and err.max() <= FP32_TOL, (call, err.max())


def _job_api_run(kind, w, m, n, x0, seed, lanes):
    from paper_2503_17405_b300 import fsmc
    eng = fsmc.Engine(0)
    tg = eng.target(kind, w["d"], w["params"])
    job = eng.job(tg, "ess", m, n, x0=x0, seed=seed, prec="fp32",
                  tuning={"lanes_per_chain": lanes, "generator": 1})
    job.run("fsm")
    x, (c, _, _) = job.samples(), job.loop_counts()
    eng.close()
    return x, c


def _static_run(kind, w, m, n, x0, seed, lanes):
    import torch
    from paper_2503_17405_b300 import fsmc
    dev = torch.device("cuda", 0)
    d = w["d"]
    L = torch.tensor(w["L"], dtype=torch.float32, device=dev).contiguous()
    vec = torch.tensor(w["y"] if kind == "gauss_conj" else w["s"], dtype=torch.float32, device=dev)
    x0_d = torch.tensor(x0, dtype=torch.float32, device=dev).contiguous()
    out = torch.full((m, n, d), float("nan"), dtype=torch.float32, device=dev)
    counts = torch.full((m, n), -7, dtype=torch.int32, device=dev)
    noise = float(w.get("s2", 0.0))
    fsmc.ess_run_static(kind, d, L.data_ptr(), vec.data_ptr(), noise, m, n, x0_d.data_ptr(), seed,
                        lanes, out.data_ptr(), counts.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), counts.cpu().numpy()


def test_static_scratch_large_run_then_small_run_of_another_shape():
    """A run that only fits with a ring of 4 directions per chain (5000 chains at d = 256 need
    about 5.2 KB each; 16 or 8 slots would not fit 32 MiB), then a chain-per-thread run on the
    conjugate Gaussian at d = 16, which must not see anything the larger run left behind."""
    import torch
    from paper_2503_17405_b300 import build
    build.build()
    torch.cuda.set_device(0)
    gp = W.gp_logit(256)
    m1, n1 = 5000, 40
    x1 = W.x0_normal(m1, 256, scale=0.1)
    got_x, got_c = _static_run("gp_logit", gp, m1, n1, x1, 11, 32)
    ref_x, ref_c = _job_api_run("gp_logit", gp, m1, n1, x1, 11, 32)
    assert np.array_equal(got_c, ref_c), "large run: loop counts differ"
    err = sample_errors(got_x, ref_x)
    assert np.isfinite(err).all() and err.max() <= FP32_TOL, err.max()

    gc = W.gauss_conj(16)
    m2, n2 = 200, 150
    x2 = W.x0_normal(m2, 16)
    got_x, got_c = _static_run("gauss_conj", gc, m2, n2, x2, 3, 1)
    ref_x, ref_c = _job_api_run("gauss_conj", gc, m2, n2, x2, 3, 1)
    assert np.array_equal(got_c, ref_c), "small run after the large one: loop counts differ"
    err = sample_errors(got_x, ref_x)
    assert np.isfinite(err).all() and err.max() <= FP32_TOL, err.max()


def test_static_scratch_rejects_runs_that_do_not_fit():
    import torch
    from paper_2503_17405_b300 import fsmc

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    d = 256
    buf = torch.zeros(d * d, dtype=torch.float32, device=dev)
    with pytest.raises(fsmc.FsmcError) as ei:
        fsmc.ess_run_static("gp_logit", d, buf.data_ptr(), buf.data_ptr(), 0.0, 1 << 20, 10,
                            buf.data_ptr(), 1, 32, buf.data_ptr(), buf.data_ptr(), None)
    assert ei.value.status == fsmc.EINVAL
    assert "static scratch" in str(ei.value)
