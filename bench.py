"""Benchmark: samples/s of the FSM engine vs the synchronised kernel on one B300.

Default workload (the headline configuration): elliptical slice sampling on latent GP
classification, d = 256, 16384 chains x 2000 samples, FP32, every sample stored on the
device.  One step = one whole job (all chains to n samples) through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config ess_gp|ess_gauss|dr_funnel|nuts_logreg]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Prints one JSON line (rank 0).  Under torchrun each rank runs its own job on its own GPU
(chains are independent: weak scaling, no collective on the data path); value is the
total over ranks divided by the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2503_17405_b300 import workloads as W  # noqa: E402

METRIC = "samples/s FSM vs synchronized kernel on 1 B300 at oracle tolerance; p50/p99 job latency"
SM_COUNT = 148
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2032.0
# ncu --set full of one FSM-step launch of the headline workload's kernel (ESS-GP, d = 256, 32 lanes
# per chain) on a small case; the summary and its command are in profiles/
ESS_GP_STEP_NCU = {"chains": 4096, "states": 512, "dram_bytes": 402.5e6 + 354.6e6, "issue_active": 0.714,
                   # whole job (4096 chains x 400 samples): smsp__inst_executed of every FSM-step launch
                   # over the job's FSM states
                   "warp_instructions_per_state": 108.35,
                   "source": "profiles/ess_gp_d256_m4096_n400_kernels.md (ncu --set full, 4096 chains x 512 states)"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def probe_rates(device):
    """Measured peak rates of this device (libfsmc_probe.so, built beside libfsmc.so): FP32 and
    FP64 multiply-add TFLOP/s, ex2.approx and lg2.approx tera-operations/s."""
    import ctypes
    from paper_2503_17405_b300 import build
    lib = ctypes.CDLL(build.PROBE_LIB)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.fsmc_bench_probe.argtypes = [ctypes.c_int, dp, dp, dp, dp]
    lib.fsmc_bench_probe.restype = ctypes.c_int
    r = [ctypes.c_double(0.0) for _ in range(4)]
    rc = lib.fsmc_bench_probe(device, *[ctypes.byref(x) for x in r])
    if rc != 0:
        raise RuntimeError("fsmc_bench_probe returned %d" % rc)
    return {"fp32_ffma_tflops": r[0].value, "fp64_dfma_tflops": r[1].value,
            "mufu_ex2_tops": r[2].value, "mufu_lg2_tops": r[3].value}


# ---- workloads ------------------------------------------------------------------------------
def make_config(name, scale=1.0, samples=None):
    """Returns (spec dict) for a named configuration (scale/samples shrink it for profiling)."""
    cfg = _make_config(name, scale)
    if samples:
        cfg["n"] = samples
        cfg["name"] += f"_n{samples}"
    if scale != 1.0:
        cfg["name"] += f"_scale{scale:g}"
    return cfg


def _make_config(name, scale):
    if name == "ess_gp":
        w = W.gp_logit(256)
        m, n = int(16384 * scale), 2000
        return dict(name="ess_gp_logit_d256_m16384_n2000", algo="ess", w=w, m=m, n=n, prec="fp32",
                    x0=W.x0_zeros(m, 256), algo_params=None,
                    flops_per_column=256 * 257)   # nu = L z: d(d+1)/2 FMA = d(d+1) flops
    if name == "ess_gauss":
        w = W.gauss_conj(16)
        m, n = 128, 1000
        return dict(name="ess_gauss_conj_d16_m128_n1000", algo="ess", w=w, m=m, n=n, prec="fp64",
                    x0=W.x0_zeros(m, 16), algo_params=None, flops_per_column=16 * 17)
    if name == "dr_funnel":
        w = W.funnel(10)
        m, n = int(65536 * scale), 5000
        return dict(name="dr3_funnel_d10_m65536_n5000", algo="dr", w=w, m=m, n=n, prec="fp32",
                    x0=W.x0_funnel_exact(m), algo_params=[3, 1.0, 0.5])
    if name == "dr_gauss100":
        # 3-stage DR with a chain per warp (d > 32): N(mu, diag sigma^2) in d = 100, proposal scales
        # 0.2, 0.1, 0.05 (stage-1 acceptance ~0.3)
        w = W.gauss_diag(100)
        m, n = int(16384 * scale), 1000
        return dict(name="dr3_gauss_diag_d100_m16384_n1000", algo="dr", w=w, m=m, n=n, prec="fp32",
                    x0=W.x0_gauss_diag_exact(w, m), algo_params=[3, 0.2, 0.5])
    if name == "dr_sym":
        # the paper's delayed-rejection toy (Sec. 7.1): symmetric DR on N(0, 1), re-centred tries of
        # sd 0.1, at most M = 100 tries per sample
        w = W.std_normal(1)
        m, n = int(65536 * scale), 2000
        return dict(name="sdr_std_normal_d1_M100_m65536_n2000", algo="dr", w=w, m=m, n=n, prec="fp32",
                    x0=W.x0_gauss_diag_exact(w, m), algo_params=[100, 0.1, 1.0], dr_symmetric=1,
                    oracle_algo="sdr", oracle_params=[100, 0.1])
    if name in ("ess_gpreg", "ess_gpreg400"):
        # Sec. 7.2: ESS on GP-regression hyperparameters, n = 100 points with 6 features (the
        # middle of the paper's 25 / 100 / 400; ess_gpreg400: the largest, 100 samples per chain),
        # 1024 chains; the likelihood is an n x n factorisation per evaluation
        nd, n = (100, 1000) if name == "ess_gpreg" else (400, 100)
        w = W.gp_reg(nd)
        m = int(1024 * scale)
        return dict(name=f"ess_gpreg_n{nd}_m1024_n{n}", algo="ess", w=w, m=m, n=n, prec="fp32",
                    x0=W.x0_gp_reg(w, m), algo_params=None, flops_per_column=0)
    if name == "slice_funnel":
        # Fig. 2's slice sampler (stepping out, then shrinkage) on the 10-d funnel: interval
        # widths needed range over orders of magnitude, so both loops' counts are heavy-tailed
        w = W.funnel(10)
        m, n = int(65536 * scale), 2000
        return dict(name="slice_funnel_d10_w1_m100_m65536_n2000", algo="slice", w=w, m=m, n=n, prec="fp32",
                    x0=W.x0_funnel_exact(m), algo_params=[1.0, 100])
    if name == "slice_gauss100":
        # the slice sampler with a chain per warp (d > 32): N(mu, diag sigma^2) in d = 100
        w = W.gauss_diag(100)
        m, n = int(16384 * scale), 1000
        return dict(name="slice_gauss_diag_d100_w1_m100_m16384_n1000", algo="slice", w=w, m=m, n=n,
                    prec="fp32", x0=W.x0_gauss_diag_exact(w, m), algo_params=[1.0, 100])
    if name == "nuts_mog":
        # Sec. 7.3: NUTS on the 100-d mixture of Gaussians with correlation 0.99, modes at
        # -10 * 1, 0, 10 * 1, identity mass, step 0.044 (acceptance statistic ~0.87), depth <= 10
        w = W.mog(100)
        m, n = int(4096 * scale), 1000
        return dict(name="nuts_mog_d100_rho0.99_m4096_n1000", algo="nuts", w=w, m=m, n=n,
                    prec="fp32", x0=W.x0_mog_exact(w, m), algo_params=[0.044, 10, 1000.0])
    if name == "nuts_logreg":
        w = W.logreg(1000, 25)
        m, n = int(4096 * scale), 1000
        return dict(name="nuts_logreg_n1000_d25_m4096_n1000", algo="nuts", w=w, m=m, n=n,
                    prec="fp32", x0=W.x0_logreg(w, m), algo_params=[0.05, 10, 1000.0])
    raise SystemExit(f"unknown config {name}")


# ---- clocks during the timed region ----------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None
        self.skip = 0

    def _lines(self):
        with open(self.path) as f:
            return sum(1 for _ in f)

    def start(self):
        """Starts nvidia-smi (a sample every 50 ms) and returns once it has written its first
        sample, so that the timed region that follows is sampled; samples written before the
        region starts are left out (mark)."""
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t0 = time.perf_counter()
        while self._lines() == 0 and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def mark(self):
        """The timed region starts: later samples only."""
        if self.proc is not None:
            self.skip = self._lines()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        # the samples of the timed region (all of them if it was shorter than one interval)
        rows = rows[self.skip:] or rows[-1:]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        load = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---- the oracle on the host cores --------------------------------------------------------------
def oracle_throughput(cfg, target_s=10.0):
    from oracle import oracle as O
    w = cfg["w"]
    cores = os.cpu_count() or 1
    n_s = min(cfg["n"], 200)
    m = max(cores, 8)
    t = 0.0
    while True:
        x0 = cfg["x0"][:m] if len(cfg["x0"]) >= m else np.resize(cfg["x0"], (m, w["d"]))
        t0 = time.perf_counter()
        O.run(cfg.get("oracle_algo", cfg["algo"]), w["kind"], w["params"], x0, n_s, seed=1, n_data=w["n_data"],
              algo_params=cfg.get("oracle_params", cfg["algo_params"]), n_threads=cores, store=False)
        t = time.perf_counter() - t0
        if t >= target_s / 4 or m >= 65536:
            break
        m = min(65536, int(m * max(2.0, target_s / max(t, 1e-3) / 2)))
    return {"value": m * n_s / t, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{m} chains x {n_s} samples of {cfg['name']} (FP64, {t:.1f} s)"}


def oracle_branch_flips(cfg, chains, x_gpu, c_gpu, tol=1e-4, flip_err=1e-2):
    """Part of the CPU-baseline leg: the oracle recomputes the sampled chains of the timed job (the
    RNG is keyed by chain, so one chain can be rerun alone) and each GPU trajectory is compared
    with it up to its first branch flip -- the first sample whose loop count differs or whose
    norm-wise relative error exceeds flip_err (a decision taken the other way moves a chain by a
    proposal's size, rounding by ~1e-6).  Errors before the flip must stay within tol."""
    from oracle import oracle as O
    w = cfg["w"]
    nref = x_gpu.shape[1]
    firsts, mx = [], 0.0
    for k, c in enumerate(chains):
        ref = O.run(cfg.get("oracle_algo", cfg["algo"]), w["kind"], w["params"], cfg["x0"][c:c + 1], nref, seed=1,
                    chain0=int(c), n_data=w["n_data"], algo_params=cfg.get("oracle_params", cfg["algo_params"]))
        xo, co = ref["samples"][0], ref["counts"][0]
        err = np.abs(x_gpu[k] - xo).max(-1) / np.maximum(1.0, np.abs(xo).max(-1))
        bad = np.nonzero((c_gpu[k] != co) | (err > flip_err))[0]
        end = int(bad[0]) if bad.size else nref
        if bad.size:
            firsts.append([int(c), end])
        if end:
            mx = max(mx, float(err[:end].max()))
    return {"chains_checked": len(chains), "samples_per_chain": nref, "flipped_chains": len(firsts),
            "first_flip_sample": firsts, "max_rel_err_before_flip": mx, "tolerance": tol,
            "within_tolerance": mx <= tol,
            "definition": "first sample whose loop count differs from the FP64 oracle's or whose norm-wise "
                          "relative error exceeds %g" % flip_err}


# ---- multi-GPU aggregation (independent chains per rank: weak scaling) -----------------------------
def max_over_ranks(value, dist=None, device="cpu"):
    """Slowest rank's time for a timed region (an all-reduce MAX, the only kind of collective of the run)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, chains, samples, total_ms):
    """Samples of all ranks' jobs divided by the slowest rank's time."""
    return world * steps * chains * samples / (total_ms / 1e3)


# ---- our arm ---------------------------------------------------------------------------------------
def parse_tuning(spec):
    """'lanes_per_chain=16,steps_per_launch=64' -> dict of launch-shape overrides."""
    out = {}
    for item in filter(None, (spec or "").split(",")):
        k, v = item.split("=")
        out[k.strip()] = int(v)
    return out


def run_ours(args, rank, world):
    import torch
    from paper_2503_17405_b300 import fsmc

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    cfg = make_config(args.config, args.scale, args.samples)
    w, m, n = cfg["w"], cfg["m"], cfg["n"]
    eng = fsmc.Engine(dev)
    tg = eng.target(w["kind"], w["d"], w["params"], n_data=w["n_data"])
    dr = nuts = None
    if cfg["algo"] == "dr":
        dr = dict(zip(["n_stages", "scale0", "factor"], cfg["algo_params"]), symmetric=cfg.get("dr_symmetric", 0))
    if cfg["algo"] == "nuts":
        nuts = dict(zip(["eps", "max_depth", "max_dH"], cfg["algo_params"]))
    sl = dict(zip(["w", "m"], cfg["algo_params"])) if cfg["algo"] == "slice" else None
    tuning = {"profile_kernels": 1, **parse_tuning(args.tuning)}
    job = eng.job(tg, cfg["algo"], m, n, x0=cfg["x0"], seed=1 + rank, prec=cfg["prec"], store=True,
                  dr=dr, nuts=nuts, tuning=tuning, slice=sl)
    stream = torch.cuda.Stream()          # a real stream: graph capture needs one
    torch.cuda.set_stream(stream)
    sp = stream.cuda_stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one(mode):
        job.reset()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        job.run(mode, stream=sp)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), job.stats()

    for _ in range(args.warmup):
        one("fsm")
    clocks = ClockSampler(dev)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    fsm_ms, stats = [], []
    for _ in range(args.steps):
        ms, st = one("fsm")
        fsm_ms.append(ms)
        stats.append(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    clk_mhz = clk.get("sm_mhz")
    # sampled chains of the last timed job, kept for the branch-flip check of the CPU-baseline leg
    flip_chains = sorted({int(c) for c in np.linspace(0, m - 1, 8)})
    nflip = min(n, 1000)
    flip_x = np.stack([job.samples(c, 1, 0, nflip)[0] for c in flip_chains])
    flip_c = job.loop_counts()[0][flip_chains, :nflip]
    total_ms = max_over_ranks(sum(fsm_ms), dist, "cuda")
    value = job_throughput(world, args.steps, m, n, total_ms)

    # synchronised program (Alg. 6) on the same workload, fewer steps: it is the slow baseline.
    # ESS runs each of its forms (sweep, compacted list, conditional graph, and for single-precision
    # GP-logit jobs the resident sweep) on a job of its own and the fastest is the baseline; the
    # others run their one (sweep) form.
    sync = None
    if not args.no_sync:
        forms = [1, 2, 3] if cfg["algo"] == "ess" and w["kind"] != "gp_reg" else [0]
        if cfg["algo"] == "ess" and w["kind"] == "gp_logit" and cfg["prec"] == "fp32" and w["d"] in (32, 64, 128, 256):
            forms.append(4)  # the resident sweep
        per_form = {}
        for f in forms:
            if f:
                sj = eng.job(tg, cfg["algo"], m, n, x0=cfg["x0"], seed=1 + rank, prec=cfg["prec"], store=True,
                             dr=dr, nuts=nuts, tuning={**tuning, "sync_form": f}, slice=sl)
            else:
                sj = job

            def one_sync():
                sj.reset()
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sj.run("sync", stream=sp)
                b.record(stream)
                b.synchronize()
                return a.elapsed_time(b), sj.stats()

            one_sync()  # warm-up (builds the graph form's executable graph)
            sms, sst = [], None
            for _ in range(args.sync_steps):
                ms, sst = one_sync()
                sms.append(ms)
            ms = sum(sms) / len(sms)
            iters = sst["sync_iterations"]
            per_form[{0: "sweep", 1: "sweep", 2: "list", 3: "graph", 4: "resident"}[f]] = {
                "value": m * n / (ms / 1e3), "ms_per_step": ms, "sync_iterations": iters,
                "sync_kernel_ms": sst["kernel_ms"][2], "refill_ms": sst["kernel_ms"][0],
                # the synchronised kernels' time per loop step (the loop-body iterations plus the
                # INIT pass of every sample), refills excluded
                "us_per_loop_step": sst["kernel_ms"][2] * 1e3 / max(1, iters + n),
                "launches": sst["launches"]}
            if f:
                sj.close()
        best = min(per_form, key=lambda k: per_form[k]["ms_per_step"])
        sync = {**per_form[best], "form": best, "forms": per_form, "mean_max_N": sst["mean_max_N"]}

    # moments-only mode (store = 0): the same job with every sample folded into per-chain
    # compensated sums of x and x^2 as it is drawn instead of stored; timed like the store-all
    # steps above (L2 flushed, CUDA events), after them, with one warm-up
    mom_only = None
    if not args.no_moments:
        mjob = eng.job(tg, cfg["algo"], m, n, x0=cfg["x0"], seed=1 + rank, prec=cfg["prec"], store=False,
                       dr=dr, nuts=nuts, tuning=tuning, slice=sl)

        def mone():
            mjob.reset()
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mjob.run("fsm", stream=sp)
            b.record(stream)
            b.synchronize()
            return a.elapsed_time(b)

        mone()
        mms = [mone() for _ in range(args.steps)]
        mms_total = max_over_ranks(sum(mms), dist, "cuda")
        mom_only = {"value": job_throughput(world, args.steps, m, n, mms_total), "unit": "samples/s",
                    "ms_per_step": mms_total / args.steps,
                    "store": "per-chain compensated sums of x and x^2 only"}
        mjob.close()

    # Pipelined ESS refills run on a second stream and overlap the FSM kernel, so their event
    # times include waiting for SMs.  One extra job (outside the timed region) with the refills
    # serialised gives each kernel's own time, which the roofline and E(m) use.
    serial_stats = None
    if cfg["algo"] == "ess" and job.tuning().get("pipelined", 0) == 1:
        sjob = eng.job(tg, cfg["algo"], m, n, x0=cfg["x0"], seed=1 + rank, prec=cfg["prec"], store=True,
                       tuning={**tuning, "pipelined": 2})
        flush.zero_()
        sjob.run("fsm", stream=sp)
        torch.cuda.synchronize()
        serial_stats = sjob.stats()
        sjob.close()

    st = stats[-1]
    kms = [sum(s["kernel_ms"][k] for s in stats) for k in range(4)]
    # per-kernel times with nothing overlapping (the serialised job, scaled to the timed steps)
    kms_own = [k * args.steps for k in serial_stats["kernel_ms"]] if serial_stats else kms
    kl = [sum(s["kernel_launches"][k] for s in stats) for k in range(4)]
    launches = sum(s["launches"] for s in stats)
    # predicted E(m) (Sec. 4.2, K = 1 after bundling, alpha = 1): per-sample cost of the
    # state-independent part c_gen plus one evaluation per loop-body iteration
    steps_total = sum(s["fsm_steps"] for s in stats)
    c_step = kms_own[1] / max(1, steps_total)
    cols = sum(s["columns_generated"] for s in stats)
    c_gen = kms_own[0] / max(1, cols) if cols else 0.0
    E_pred = (c_gen + c_step * (1 + st["mean_max_N"])) / (c_gen + c_step * (1 + st["mean_N"])) \
        if cfg["algo"] == "ess" else st["mean_max_N"] / max(st["mean_N"], 1e-9)

    peaks = _peaks()
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    tun = job.tuning()
    gen = tun.get("generator", 0)
    d = w["d"]
    if cfg["algo"] == "ess" and kms_own[0] >= kms_own[1]:
        achieved = cols * cfg["flops_per_column"] / (kms_own[0] / 1e3) / 1e12
        if gen == 2:
            # kind::f16 tensor cores (FP16 splits, FP32 accumulate): measured dense bf16 peak,
            # the same nominal rate as fp16; algorithmic flops d(d+1) per direction
            tp = peaks.get("bf16_tflops", 1800.0)
            roof = {"kernel": "ess_nu_gen_tc_kernel", "bound": "tensor", "achieved": achieved,
                    "peak": tp, "unit": "TFLOP/s", "frac": achieved / tp, "traffic": None,
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), fp16 has the same nominal rate",
                    "limiter": "Philox z generation on the CUDA cores (tensor pipe ~6% busy in ncu)",
                    "fp32_equivalent_frac": achieved / fp32_peak}
        else:
            roof = {"kernel": "ess_nu_gen_kernel", "bound": "alu", "achieved": achieved,
                    "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                    "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz (nominal)"}
    else:
        # FSM step kernel: algorithmic work per step (one log-density evaluation) as the hot-path
        # scope table counts it -- ESS-GP: x' = x cos + nu sin and the softplus sum, 3 d flops plus
        # 2 d multi-function operations (an exp and a log per coordinate); NUTS: one logistic
        # gradient, 4 n d flops; DR: the stage's density, ~40 flops (+ 5 Philox blocks for its
        # normals); the slice sampler: the point x + theta u and the density (~20 d)
        mufu = None
        if cfg["algo"] == "ess" and w["kind"] == "gp_reg":
            # the covariance (n^2 / 2 exponentials, counted as 2 flops each), the LDL^T sweep with
            # y folded in (n^3 / 3 + n^2 multiply-adds, 2 flops each)
            nd = w["n_data"]
            per = nd * nd + 2 * (nd ** 3 / 3 + nd * nd)
        elif cfg["algo"] == "ess":
            per = 3 * d
            if w["kind"] == "gp_logit":
                mufu = {"algorithmic_per_step": 2 * d,
                        "issued_per_step": d + d // 8,
                        "issued_note": "one ex2 per coordinate, one lg2 per group of eight (grouped-product softplus)"}
        elif cfg["algo"] == "nuts":
            # logistic regression: 4 n d; mixture: (7 K + 1) d (residual, its square, the gradient)
            per = 4 * w["n_data"] * d if w["kind"] == "logreg" else (7 * w["n_data"] + 1) * d
        elif cfg["algo"] == "dr":
            # the stage's density: funnel 2 d + ~20 (its exponential and constants; ~40 at d = 10),
            # diagonal Gaussian 3 d
            per = 2 * d + 20 if w["kind"] == "funnel" else 3 * d
        else:
            per = 20 * d
        achieved = steps_total * per / (kms_own[1] / 1e3) / 1e12 if kms_own[1] else None
        kname = {"ess": "ess_block_fsm_kernel" if w["kind"] == "gp_reg" else "ess_fsm_kernel",
                 "dr": "dr_fsm_kernel", "slice": "slice_fsm_kernel",
                 "nuts": "nuts_fsm_batched_kernel" if w["kind"] == "logreg" else "nuts_fsm_kernel"}[cfg["algo"]]
        traffic, traffic_src, issue = None, None, None
        if cfg["algo"] == "ess" and w["kind"] == "gp_logit" and d == 256 and tun.get("lanes_per_chain") == 32:
            prof = ESS_GP_STEP_NCU
            # DRAM bytes of one FSM-step launch in the ncu capture, scaled by chains and states per launch
            traffic = prof["dram_bytes"] * (m / prof["chains"]) * (tun.get("steps_per_launch", prof["states"]) / prof["states"])
            traffic_src = ("bytes per launch: ncu capture on %d chains x %d states, scaled by chains and "
                           "states per launch" % (prof["chains"], prof["states"]))
            # instruction issue: a chain is one warp, so a state costs warp_instructions_per_state issue
            # slots of one of the 4 x 148 schedulers
            clk_hz = (clk_mhz or SM_MAX_MHZ) * 1e6
            floor_ms = steps_total * prof["warp_instructions_per_state"] / (4 * SM_COUNT * clk_hz) * 1e3
            issue = {"issue_active": prof["issue_active"], "warp_instructions_per_state": prof["warp_instructions_per_state"],
                     "issue_floor_ms_per_step": floor_ms / args.steps,
                     "kernel_ms_per_step": kms_own[1] / args.steps,
                     "source": prof["source"]}
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved,
                "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": (achieved / fp32_peak) if achieved else None, "traffic": traffic,
                "traffic_source": traffic_src,
                "ncu_issue": issue,
                "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz (nominal)",
                "flops_per_step": per,
                "limiter": {"ess": "a warp per chain: length-j dot products per covariance column, shared-memory bound" if w["kind"] == "gp_reg"
                            else "instruction issue (warp instructions per state in ncu_issue), then the multi-function unit"
                            if w["kind"] == "gp_logit" else "latency: few chains (one warp each), short rows",
                            "dr": "latency: one chain per thread, ~14 resident warps per SM at 65536 chains",
                            "slice": "latency: one chain per thread, 65536 chains",
                            "nuts": "latency and occupancy of the block-batched gradient" if w["kind"] == "logreg"
                            else "latency: one chain per warp, shuffle reductions per component and U-turn test"}[cfg["algo"]]}
        if mufu and kms_own[1]:
            mufu["achieved_issued_tops"] = steps_total * mufu["issued_per_step"] / (kms_own[1] / 1e3) / 1e12
            roof["mufu"] = mufu

    # measured peak rates of this device (outside the timed regions): context for the nominal
    # FP32 peak the roofline fraction is taken against
    try:
        rates = probe_rates(dev)
        roof["measured_rates"] = rates
        if roof.get("unit") == "TFLOP/s" and roof.get("bound") == "alu" and roof.get("achieved"):
            roof["frac_of_measured_ffma"] = roof["achieved"] / rates["fp32_ffma_tflops"]
        if roof.get("mufu", {}).get("achieved_issued_tops"):
            roof["mufu"]["frac_of_measured_ex2"] = roof["mufu"]["achieved_issued_tops"] / rates["mufu_ex2_tops"]
    except (OSError, RuntimeError) as ex:
        roof["probe"] = str(ex)

    # end to end through the public API: host params and x0 in, posterior moments out.  Every
    # step: target and job created from pinned host arrays (params, x0), the whole run as a
    # moments-only job (each sample folded into per-chain sums of x and x^2 as it is drawn, the
    # job's declared result), those sums read back into pinned host arrays, the job closed; one
    # untimed warm-up.  (Reading back every stored sample instead would move m n d values per step,
    # 33.5 GB at the headline size, and time the host link rather than the sampler.)
    e2e = None
    if not args.no_e2e:
        params_h = torch.from_numpy(np.ascontiguousarray(w["params"], dtype=np.float64)).pin_memory()
        x0_h = torch.from_numpy(np.ascontiguousarray(cfg["x0"], dtype=np.float64)).pin_memory()
        sx = torch.empty((m, w["d"]), dtype=torch.float64).pin_memory().numpy()
        sx2 = torch.empty((m, w["d"]), dtype=torch.float64).pin_memory().numpy()
        nk = torch.empty((m,), dtype=torch.int64).pin_memory().numpy()

        def e2e_step():
            tg2 = eng.target(w["kind"], w["d"], params_h.numpy(), n_data=w["n_data"])
            job2 = eng.job(tg2, cfg["algo"], m, n, x0=x0_h.numpy(), seed=1 + rank, prec=cfg["prec"],
                           store=False, dr=dr, nuts=nuts, tuning=parse_tuning(args.tuning) or None, slice=sl)
            job2.run("fsm", stream=sp)
            job2.moments(sx, sx2, nk)
            job2.close()
            tg2.close()

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        t1 = time.perf_counter()
        e2e = {"value": m * n * args.steps / (t1 - t0), "unit": "samples/s",
               "result": "per-chain sums of x and x^2 over all samples (moments-only job), read to host",
               "h2d_bytes_per_step": int(params_h.numel() * 8 + x0_h.numel() * 8),
               "d2h_bytes_per_step": int(sx.nbytes + sx2.nbytes + nk.nbytes)}
    out = None
    if rank == 0:
        cpu = flips = None
        if not (args.no_cpu or world > 1):
            cpu = oracle_throughput(cfg)
            flips = oracle_branch_flips(cfg, flip_chains, flip_x, flip_c)
        out = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if cfg["prec"] == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "chains_per_gpu": m, "samples_per_chain": n,
                       "d": w["d"], "algo": cfg.get("oracle_algo", cfg["algo"]), "store": "all samples on device",
                       "l2": "flushed between steps (256 MiB write); outputs exceed L2",
                       "parallelism": f"replicas x{world} (independent chains)"},
            "fsm": {"value": value, "R_hat": st["R_hat"], "mean_N": st["mean_N"],
                    "mean_max_N": st["mean_max_N"], "E_pred": E_pred,
                    "kernel_ms_per_step": [k / args.steps for k in kms],
                    "kernel_ms_per_step_unoverlapped": [k / args.steps for k in kms_own],
                    "kernel_launches_per_step": [k / args.steps for k in kl],
                    "columns_generated_per_step": cols / max(1, len(stats)),
                    "tuning": {k: tun[k] for k in ("lanes_per_chain", "steps_per_launch", "ring_slots",
                                                   "threads_per_block", "generator", "pipelined")}},
            "sync": sync,
            "speedup_fsm_over_sync": (value / world / sync["value"]) if sync else None,
            # the paper's cost model (Sec. 4.1): a synchronised loop step costs one evaluation of every
            # chain; here that is the FSM step kernel's time for one state of every chain
            "cost_model": ({"us_per_all_chain_evaluation": kms_own[1] / args.steps * 1e3 / max(1.0, steps_total / args.steps / m),
                            "sync_model_ms": (kms_own[1] / args.steps / max(1.0, steps_total / args.steps / m))
                            * (sync["sync_iterations"] + n) + kms_own[0] / args.steps}
                           if sync and kms_own[1] else None),
            "moments_only": mom_only,
            "roofline": roof,
            "cpu_baseline": cpu,
            "branch_flips": flips,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")},
        }
    eng.close()
    # the mixed request stream (continuous batching) at a stated scale, after the job's engine is
    # closed: p50 / p99 job latency beside throughput (the full-size stream: --config serving)
    if out is not None and world == 1 and not args.no_serve and cfg["name"].startswith("ess_gp_logit"):
        try:
            out["serving"] = serve_stream(args.serve_jobs, args.serve_scale, sync_jobs=0, device=dev)
        except Exception as ex:  # noqa: BLE001 -- reported, not fatal to the headline line
            out["serving"] = {"error": str(ex)}
    if dist:
        dist.destroy_process_group()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    cfg = make_config(args.config, args.scale, args.samples)
    times, vals = [], []
    cpu = None
    for _ in range(args.warmup + args.steps):
        cpu = oracle_throughput(cfg, target_s=max(2.0, 20.0 / max(1, args.steps + args.warmup)))
        vals.append(cpu["value"])
    vals = vals[args.warmup:]
    value = statistics.mean(vals)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cfg["m"] * cfg["n"] / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "chains_per_gpu": cfg["m"],
                       "samples_per_chain": cfg["n"], "d": cfg["w"]["d"], "algo": cfg.get("oracle_algo", cfg["algo"])},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ---- step-form ablations ------------------------------------------------------------------------------
def run_ablations(args):
    """The paper's step-form ablations on the CUDA kernels (tuning.step_form = 2 against the
    default 1): ESS as the bundled step without amortisation (both states' log-density calls every
    step, one masked), with one chain per thread
    and one chain per warp; DR with its PROPOSE body unrolled into four states run one per step
    (not condensed).  The two forms give identical samples (tests/test_gpu_ablation.py); this
    reports their device time."""
    import torch
    from paper_2503_17405_b300 import fsmc

    torch.cuda.set_device(0)
    eng = fsmc.Engine(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sp = stream.cuda_stream
    scale = args.scale

    def timed(tg, algo, m, n, x0, tuning, dr=None, reps=3):
        job = eng.job(tg, algo, m, n, x0=x0, seed=1, prec="fp32", store=True, dr=dr, tuning=tuning)
        ms = []
        for r in range(reps + 1):
            job.reset()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            job.run("fsm", stream=sp)
            b.record(stream)
            b.synchronize()
            if r:
                ms.append(a.elapsed_time(b))
        st = job.stats()
        job.close()
        return {"ms_per_job": sum(ms) / len(ms), "fsm_states": st["fsm_steps"],
                "samples_per_s": m * n / (sum(ms) / len(ms) / 1e3), "mean_N": st["mean_N"]}

    out = {"metric": "step-form ablations: device ms per job, form 2 (paper's ablation) / form 1 (default)",
           "unit": "ms", "data": "synthetic", "rows": []}
    # ESS on the conjugate Gaussian: a cheap log-density (d = 16) and a dearer one (d = 256)
    for d, lanes_list, n in ((16, (1, 32), 500), (256, (32,), 200)):
        w = W.gauss_conj(d)
        tg = eng.target("gauss_conj", d, w["params"])
        m = int(16384 * scale)
        x0 = W.x0_normal(m, d, scale=0.5)
        for lanes in lanes_list:
            a = timed(tg, "ess", m, n, x0, {"lanes_per_chain": lanes, "step_form": 1})
            b = timed(tg, "ess", m, n, x0, {"lanes_per_chain": lanes, "step_form": 2})
            out["rows"].append({"ablation": "ESS log-density not amortised", "workload":
                                f"ess_gauss_conj_d{d}_m{m}_n{n}_fp32", "lanes_per_chain": lanes,
                                "default": a, "ablation_form": b, "ratio": b["ms_per_job"] / a["ms_per_job"]})
    w = W.funnel(10)
    tg = eng.target("funnel", 10, w["params"])
    m, n = int(65536 * scale), 1000
    x0 = W.x0_funnel_exact(m)
    dr = {"n_stages": 3, "scale0": 1.0, "factor": 0.5}
    a = timed(tg, "dr", m, n, x0, {"step_form": 1}, dr=dr)
    b = timed(tg, "dr", m, n, x0, {"step_form": 2}, dr=dr)
    out["rows"].append({"ablation": "DR PROPOSE body as 4 states (not condensed)",
                        "workload": f"dr3_funnel_d10_m{m}_n{n}_fp32",
                        "default": a, "ablation_form": b, "ratio": b["ms_per_job"] / a["ms_per_job"],
                        "states_per_sample": [a["fsm_states"] / (m * n), b["fsm_states"] / (m * n)]})
    # the paper's own ablation workload (Sec. 7.1): symmetric DR on N(0, 1), sd 0.1, M = 100
    w = W.std_normal(1)
    tg = eng.target(w["kind"], 1, w["params"])
    x0 = W.x0_gauss_diag_exact(w, m)
    dr = {"n_stages": 100, "scale0": 0.1, "factor": 1.0, "symmetric": 1}
    a = timed(tg, "dr", m, n, x0, {"step_form": 1}, dr=dr)
    b = timed(tg, "dr", m, n, x0, {"step_form": 2}, dr=dr)
    out["rows"].append({"ablation": "symmetric DR try as 4 states (not condensed)",
                        "workload": f"sdr_std_normal_d1_M100_m{m}_n{n}_fp32",
                        "default": a, "ablation_form": b, "ratio": b["ms_per_job"] / a["ms_per_job"],
                        "states_per_sample": [a["fsm_states"] / (m * n), b["fsm_states"] / (m * n)]})
    eng.close()
    return out


# ---- serving stream (C5) ------------------------------------------------------------------------------
def serve_stream(n_jobs, scale, sync_jobs=0, device=0):
    """Poisson-arriving mixed jobs through fsmc_submit (ESS-GP and NUTS-logistic, sizes log-uniform
    as workloads.serving_jobs draws them, times `scale` chains and draws).  A capacity pass submits
    every job at t = 0; the measured pass offers 0.8 of that capacity as Poisson arrivals; the
    synchronised kernel then serves the first `sync_jobs` jobs of the same stream one at a time.
    Latency = completion - submit, as the library records it."""
    import torch
    from paper_2503_17405_b300 import fsmc

    torch.cuda.set_device(device)
    base = W.serving_jobs(n_jobs, rate_hz=1.0, scale=scale)
    cache = {}

    def target(eng, j):
        key = (j["kind"], j["d"], j["n_data"], j["data_seed"])
        if key not in cache:
            if j["kind"] == "ess_gp":
                cache[key] = W.gp_logit(j["d"], seed=j["data_seed"])
            else:
                cache[key] = W.logreg(j["n_data"], j["d"], seed=j["data_seed"])
        w = cache[key]
        return w, eng.target(w["kind"], w["d"], w["params"], n_data=w["n_data"])

    def one_pass(mode, rate_hz, jobs_in):
        eng = fsmc.Engine(device)
        jobs = [dict(j) for j in jobs_in]
        t = 0.0
        rng = np.random.default_rng(7)
        for j in jobs:
            if rate_hz:
                t += rng.exponential(1.0 / rate_hz)
            j["arrival"] = t
        live, lat, samples = [], [], 0
        t0 = time.perf_counter()
        k = 0
        while k < len(jobs) or live:
            now = time.perf_counter() - t0
            while k < len(jobs) and jobs[k]["arrival"] <= now:
                j = jobs[k]
                w, tg = target(eng, j)
                x0 = W.x0_zeros(j["chains"], j["d"]) if j["kind"] == "ess_gp" else W.x0_logreg(w, j["chains"])
                job = eng.job(tg, "ess" if j["kind"] == "ess_gp" else "nuts", j["chains"], j["draws"],
                              x0=x0, seed=1 + k, prec="fp32", store=False,
                              nuts={"eps": 0.05, "max_depth": 10, "max_dH": 1000.0})
                job.submit(mode)
                live.append(job)
                samples += j["chains"] * j["draws"]
                k += 1
            for job in list(live):
                done, latency = job.poll()
                if done:
                    job.moments()
                    lat.append(latency)
                    job.close()
                    live.remove(job)
            time.sleep(0.0005)
        makespan = time.perf_counter() - t0
        eng.close()
        return {"makespan_s": makespan, "samples_per_s": samples / makespan,
                "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "jobs": len(lat)}

    cap = one_pass("fsm", 0.0, base)                 # all jobs at t = 0: capacity
    rate = 0.8 * cap["jobs"] / cap["makespan_s"]
    fsm = one_pass("fsm", rate, base)
    sync = one_pass("sync", rate, base[:sync_jobs]) if sync_jobs else None
    return {"scale": scale, "jobs": n_jobs, "rate_jobs_per_s": rate, "arrivals": "Poisson",
            "offered_load": "0.8 x measured FSM capacity",
            "p50_latency_s": fsm["p50_latency_s"], "p99_latency_s": fsm["p99_latency_s"],
            "samples_per_s": fsm["samples_per_s"], "fsm": fsm, "capacity_pass": cap,
            "sync_one_at_a_time": sync,
            "sync_subset": "first %d jobs of the same stream and arrival times" % sync_jobs if sync_jobs else None}


def run_serving(args):
    """--config serving: the mixed request stream on its own line (default: the full stream of 200
    jobs at full sizes, the synchronised baseline on the first --serve-sync-jobs of them)."""
    from paper_2503_17405_b300 import build
    build.build()
    sj = args.serve_sync_jobs if args.serve_sync_jobs is not None else args.serve_jobs
    r = serve_stream(args.serve_jobs, args.serve_scale, sync_jobs=0 if args.no_sync else sj)
    return {"metric": METRIC, "value": r["samples_per_s"], "unit": "samples/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving_{args.serve_jobs}_jobs_scale{args.serve_scale:g}",
                       "arrivals": "Poisson", "offered_load": "0.8 x measured FSM capacity",
                       "rate_jobs_per_s": r["rate_jobs_per_s"]},
            "p50_latency_s": r["p50_latency_s"], "p99_latency_s": r["p99_latency_s"],
            "fsm": r["fsm"], "sync_one_at_a_time": r["sync_one_at_a_time"], "sync_subset": r["sync_subset"],
            "capacity_pass": r["capacity_pass"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="ess_gp")
    ap.add_argument("--sync-steps", type=int, default=1)
    ap.add_argument("--no-sync", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-moments", action="store_true", help="skip the moments-only (store = 0) leg")
    ap.add_argument("--scale", type=float, default=1.0, help="chains x scale (profiling only)")
    ap.add_argument("--samples", type=int, default=None, help="samples per chain (profiling only)")
    ap.add_argument("--serve-jobs", type=int, default=None,
                    help="jobs of the serving stream (default: 200 for --config serving, 40 for the "
                         "serving sub-object of the default line)")
    ap.add_argument("--serve-scale", type=float, default=None,
                    help="chains and draws scale of the serving stream (default: 1 for --config serving, "
                         "0.25 for the default line's sub-object)")
    ap.add_argument("--serve-sync-jobs", type=int, default=None,
                    help="--config serving: jobs the synchronised one-at-a-time baseline serves (default 20)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving sub-object of the default line")
    ap.add_argument("--tuning", default="", help="launch-shape overrides, e.g. lanes_per_chain=16")
    args = ap.parse_args()
    full_stream = args.config == "serving"
    if args.serve_jobs is None:
        args.serve_jobs = 200 if full_stream else 40
    if args.serve_scale is None:
        args.serve_scale = 1.0 if full_stream else 0.25
    if args.serve_sync_jobs is None and full_stream:
        args.serve_sync_jobs = 20
    if args.config == "serving":
        print(json.dumps(run_serving(args)))
        return
    if args.config == "ablations":
        from paper_2503_17405_b300 import build
        build.build()
        print(json.dumps(run_ablations(args)))
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if args.impl == "reference" else 1))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        from paper_2503_17405_b300 import build
        if rank == 0:
            build.build()
        out = run_ours(args, rank, world)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
