"""ctypes binding of the FP64 CPU oracle (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg import this module.  The CUDA product path never does.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = ["rng_targets.cpp", "samplers.cpp", "api.cpp"]
_lock = threading.Lock()
_lib = None

ALGO = {"ess": 0, "dr": 1, "nuts": 2, "sdr": 3, "slice": 4}
TARGET = {"gauss_conj": 0, "gp_logit": 1, "funnel": 2, "logreg": 3, "gauss_diag": 4, "flat": 5, "mog": 6,
          "gp_reg": 7}


def build(force=False):
    """Compile liboracle.so with the host C++ compiler (plain -O2, IEEE math)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES + ["oracle.h"]]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", _LIB_PATH]
    cmd += [os.path.join(_HERE, s) for s in _SOURCES]
    subprocess.run(cmd, check=True)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            dp, ip, up = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_uint32))
            L.ora_philox4x32_10.argtypes = [up, up, up]
            L.ora_uniform.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.ora_uniform.restype = ctypes.c_double
            L.ora_uniform32.argtypes = [ctypes.c_uint32]
            L.ora_uniform32.restype = ctypes.c_double
            L.ora_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, dp]
            L.ora_logp.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.ora_logp.restype = ctypes.c_double
            L.ora_leapfrog.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                       ctypes.c_double, ctypes.c_int]
            L.ora_log1mexp.argtypes = [ctypes.c_double]
            L.ora_log1mexp.restype = ctypes.c_double
            L.ora_dr_log_alpha1.argtypes = [ctypes.c_double] * 2
            L.ora_dr_log_alpha1.restype = ctypes.c_double
            L.ora_dr_log_alpha2.argtypes = [ctypes.c_double] * 5
            L.ora_dr_log_alpha2.restype = ctypes.c_double
            L.ora_dr_log_alpha3.argtypes = [ctypes.c_double] * 9
            L.ora_dr_log_alpha3.restype = ctypes.c_double
            L.ora_dr_stage_log_alpha.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            L.ora_dr_stage_log_alpha.restype = ctypes.c_double
            L.ora_sdr_log_alpha.argtypes = [ctypes.c_double] * 3
            L.ora_sdr_log_alpha.restype = ctypes.c_double
            L.ora_ess_trace.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                        ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, dp,
                                        ctypes.c_int]
            L.ora_ess_trace.restype = ctypes.c_int
            L.ora_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, dp,
                                  ctypes.c_uint64, ctypes.c_int, dp, ip, ip, dp]
            L.ora_run.restype = ctypes.c_int
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.ora_transitions.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                          ctypes.c_int64, u32p, u32p, dp, ctypes.c_uint64, ctypes.c_int,
                                          dp, ip, ip, dp]
            L.ora_transitions.restype = ctypes.c_int
            L.ora_R_hat.argtypes = [ip, ctypes.c_int64, ctypes.c_int64]
            L.ora_R_hat.restype = ctypes.c_double
            _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().ora_philox4x32_10(c, k, o)
    return list(o)


def uniform(hi, lo):
    return lib().ora_uniform(hi, lo)


def uniform32(w):
    return lib().ora_uniform32(w)


def normals(seed, chain, sample, tag, draw0, d):
    z = np.zeros(d)
    lib().ora_normals(seed, chain, sample, tag, draw0, d, _dp(z))
    return z


def _params(params):
    p = _f64(params if params is not None else np.zeros(1))
    return p if p.size else np.zeros(1)


def logp(kind, params, x, n_data=0, grad=False):
    x = _f64(x)
    params = _params(params)
    g = np.zeros_like(x) if grad else None
    v = lib().ora_logp(TARGET[kind], x.size, n_data, _dp(params), _dp(x), _dp(g))
    return (v, g) if grad else v


def leapfrog(kind, params, x, p, eps, n_steps, n_data=0):
    x = _f64(x).copy()
    p = _f64(p).copy()
    params = _params(params)
    lib().ora_leapfrog(TARGET[kind], x.size, n_data, _dp(params), _dp(x), _dp(p), eps, n_steps)
    return x, p


def ess_trace(kind, params, x, seed, chain, sample, cap=256, n_data=0):
    x = _f64(x).copy()
    params = _f64(params)
    tr = np.zeros(3 * cap)
    n = lib().ora_ess_trace(TARGET[kind], x.size, n_data, _dp(params), _dp(x), seed, chain,
                            sample, _dp(tr), cap)
    return x, n, tr[:3 * min(n, cap)].reshape(-1, 3)


def run(algo, kind, params, x0, n_samples, seed, chain0=0, n_data=0, algo_params=None,
        n_threads=None, store=True):
    """Run the sequential oracle on chains chain0..chain0+len(x0)-1.

    Returns dict(samples[m,n,d] | None, counts[m,n], aux[m,n], x_final[m,d]).
    """
    x0 = _f64(x0)
    m, d = x0.shape
    params = _params(params)
    ap = None if algo_params is None else _f64(algo_params)
    samples = np.zeros((m, n_samples, d)) if store else None
    counts = np.zeros((m, n_samples), dtype=np.int32)
    aux = np.zeros((m, n_samples), dtype=np.int32)
    xf = np.zeros((m, d))
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    rc = lib().ora_run(ALGO[algo], TARGET[kind], d, n_data, _dp(params), _dp(ap), chain0, m,
                       n_samples, _dp(x0), seed, n_threads, _dp(samples), _ip(counts), _ip(aux),
                       _dp(xf))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return {"samples": samples, "counts": counts, "aux": aux, "x_final": xf}


def transitions(algo, kind, params, x_in, chains, samples, seed, n_data=0, algo_params=None,
                n_threads=None):
    """One transition per item: item i starts at x_in[i] as sample samples[i] of chain chains[i],
    with the random numbers a run uses there.  Returns dict(x[k,d], counts[k], aux[k], margin[k]):
    margin is the smallest relative distance between a compared value and its threshold over the
    transition's decisions (accept/reject, stop/shrink, merge, U-turn; see oracle.h)."""
    x_in = _f64(x_in)
    k, d = x_in.shape
    params = _params(params)
    ap = None if algo_params is None else _f64(algo_params)
    ch = np.ascontiguousarray(chains, dtype=np.uint32)
    sm = np.ascontiguousarray(samples, dtype=np.uint32)
    assert ch.shape == (k,) and sm.shape == (k,)
    xo = np.zeros((k, d))
    counts = np.zeros(k, dtype=np.int32)
    aux = np.zeros(k, dtype=np.int32)
    margin = np.zeros(k)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    rc = lib().ora_transitions(ALGO[algo], TARGET[kind], d, n_data, _dp(params), _dp(ap), k,
                               ch.ctypes.data_as(u32p), sm.ctypes.data_as(u32p), _dp(x_in), seed,
                               n_threads or os.cpu_count() or 1, _dp(xo), _ip(counts), _ip(aux),
                               _dp(margin))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return {"x": xo, "counts": counts, "aux": aux, "margin": margin}


def R_hat(counts):
    c = np.ascontiguousarray(counts, dtype=np.int32)
    m, n = c.shape
    return lib().ora_R_hat(_ip(c), m, n)


def dr_log_alpha1(a, b):
    return lib().ora_dr_log_alpha1(a, b)


def dr_log_alpha2(*a):
    return lib().ora_dr_log_alpha2(*a)


def dr_log_alpha3(*a):
    return lib().ora_dr_log_alpha3(*a)


def log1mexp(a):
    return lib().ora_log1mexp(a)


def sdr_log_alpha(lp_x, lp_star, lp_y):
    """log acceptance of a symmetric re-centred delayed-rejection try (oracle's function)."""
    return lib().ora_sdr_log_alpha(lp_x, lp_star, lp_y)


def dr_stage_log_alpha(k, x, ys, lps, sig):
    """log alpha of stage k (0-based) exactly as the oracle's DR transition wires it."""
    x = _f64(x)
    ys = _f64(ys)
    lps = _f64(lps)
    sig = _f64(sig)
    return lib().ora_dr_stage_log_alpha(k, x.size, _dp(x), _dp(ys), _dp(lps), _dp(sig))
