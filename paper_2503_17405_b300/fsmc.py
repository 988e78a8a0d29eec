"""Thin ctypes binding of libfsmc.so (include/fsmc.h): argument marshalling only.

Every computation of the sampling path runs in the library's CUDA kernels.  If the
library is missing, importing the binding raises; there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfsmc.so")

OK, EINVAL, ENOMEM, EADMIT, ECUDA, ETIMEOUT, ESTATE, EDEVICE, ECANCELED = 0, -1, -2, -3, -4, -5, -6, -7, -8
_STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "EADMIT", -4: "ECUDA", -5: "ETIMEOUT",
           -6: "ESTATE", -7: "EDEVICE", -8: "ECANCELED"}
TARGET = {"gauss_conj": 0, "gp_logit": 1, "funnel": 2, "logreg": 3, "gauss_diag": 4, "flat": 5, "mog": 6,
          "gp_reg": 7}
ALGO = {"ess": 0, "dr": 1, "nuts": 2, "slice": 3}
PREC = {"fp64": 0, "fp32": 1}
MODE = {"fsm": 0, "sync": 1}


class FsmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class DRParams(ctypes.Structure):
    _fields_ = [("n_stages", ctypes.c_int), ("scale0", ctypes.c_double), ("factor", ctypes.c_double),
                ("symmetric", ctypes.c_int)]


class NUTSParams(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("max_depth", ctypes.c_int), ("max_dH", ctypes.c_double)]


class SliceParams(ctypes.Structure):
    _fields_ = [("w", ctypes.c_double), ("m", ctypes.c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [("lanes_per_chain", ctypes.c_int), ("steps_per_launch", ctypes.c_int),
                ("ring_slots", ctypes.c_int), ("threads_per_block", ctypes.c_int),
                ("profile_kernels", ctypes.c_int), ("generator", ctypes.c_int),
                ("pipelined", ctypes.c_int), ("step_form", ctypes.c_int),
                ("barrier_spin_limit", ctypes.c_int), ("barrier_test_missing", ctypes.c_int),
                ("sync_form", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("R_hat", ctypes.c_double), ("mean_N", ctypes.c_double),
                ("mean_max_N", ctypes.c_double), ("samples_done", ctypes.c_int64),
                ("fsm_steps", ctypes.c_int64), ("sync_iterations", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("device_ms", ctypes.c_double),
                ("error_word", ctypes.c_int64), ("kernel_ms", ctypes.c_double * 4),
                ("kernel_launches", ctypes.c_int64 * 4), ("columns_generated", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if hasattr(v, "__len__") else v
        return out


_vp, _dp, _ip, _lp = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64))

# (name, restype, argtypes) for every entry point of include/fsmc.h
SIGNATURES = [
    ("fsmc_engine_create", ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    ("fsmc_engine_destroy", None, [_vp]),
    ("fsmc_engine_bytes_in_use", ctypes.c_size_t, [_vp]),
    ("fsmc_target_create", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                          ctypes.c_size_t, ctypes.POINTER(_vp)]),
    ("fsmc_target_destroy", None, [_vp]),
    ("fsmc_job_create", ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int64,
                                       ctypes.c_int64, _dp, ctypes.c_uint64, ctypes.c_int,
                                       ctypes.POINTER(_vp)]),
    ("fsmc_autotune", ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int64,
                                     ctypes.c_char_p, ctypes.POINTER(Tuning)]),
    ("fsmc_job_set_tuning", ctypes.c_int, [_vp, ctypes.POINTER(Tuning)]),
    ("fsmc_job_get_tuning", ctypes.c_int, [_vp, ctypes.POINTER(Tuning)]),
    ("fsmc_job_bytes", ctypes.c_size_t, [_vp]),
    ("fsmc_job_run", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64, _vp]),
    ("fsmc_job_reset", ctypes.c_int, [_vp]),
    ("fsmc_job_progress", ctypes.c_int, [_vp, _lp, ctypes.POINTER(ctypes.c_int)]),
    ("fsmc_read_samples", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, _dp]),
    ("fsmc_read_samples_dev", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, _vp, _vp]),
    ("fsmc_read_loop_counts", ctypes.c_int, [_vp, _ip, _ip, _lp]),
    ("fsmc_read_state", ctypes.c_int, [_vp, _dp]),
    ("fsmc_read_moments", ctypes.c_int, [_vp, _dp, _dp, _lp]),
    ("fsmc_read_stats", ctypes.c_int, [_vp, ctypes.POINTER(Stats)]),
    ("fsmc_job_snapshot", ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_size_t)]),
    ("fsmc_job_restore", ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    ("fsmc_job_destroy", None, [_vp]),
    ("fsmc_submit", ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    ("fsmc_poll", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), _dp]),
    ("fsmc_cancel", ctypes.c_int, [_vp]),
    ("fsmc_wait_all", ctypes.c_int, [_vp, ctypes.c_double]),
    ("fsmc_ess_run_static", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_float,
                                           ctypes.c_int64, ctypes.c_int64, _vp, ctypes.c_uint64,
                                           ctypes.c_int, _vp, _vp, _vp]),
    ("fsmc_last_error", ctypes.c_char_p, []),
]

_lib = None


def load(path=LIB_PATH):
    """Load libfsmc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2503_17405_b300/build.py "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st):
    if st != OK:
        raise FsmcError(st, load().fsmc_last_error().decode())


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


class Engine:
    def __init__(self, device=0, hbm_budget_bytes=0):
        self._h = _vp()
        _check(load().fsmc_engine_create(device, hbm_budget_bytes, ctypes.byref(self._h)))
        self._objs = []   # jobs / targets whose handles die with the engine

    @property
    def handle(self):
        return self._h

    def bytes_in_use(self):
        return load().fsmc_engine_bytes_in_use(self._h)

    def target(self, kind, d, params=None, n_data=0):
        return Target(self, kind, d, params, n_data)

    def job(self, target, algo, n_chains, n_samples, x0=None, seed=1, prec="fp32", store=True,
            dr=None, nuts=None, tuning=None, slice=None):
        return Job(self, target, algo, n_chains, n_samples, x0, seed, prec, store, dr, nuts, tuning,
                   slice)

    def autotune(self, target, algo, n_chains, prec="fp32", dr=None, nuts=None, cache_path=None, slice=None):
        """fsmc_autotune: the fastest launch shape for such jobs, as a tuning dict."""
        ap = None
        if algo == "dr":
            dr = dr or {}
            keep = DRParams(dr.get("n_stages", 3), dr.get("scale0", 1.0), dr.get("factor", 0.5),
                            int(dr.get("symmetric", 0)))
            ap = ctypes.cast(ctypes.byref(keep), _vp)
        elif algo == "nuts":
            nuts = nuts or {}
            keep = NUTSParams(nuts.get("eps", 0.05), nuts.get("max_depth", 10), nuts.get("max_dH", 1000.0))
            ap = ctypes.cast(ctypes.byref(keep), _vp)
        elif algo == "slice":
            sl = slice or {}
            keep = SliceParams(sl.get("w", 1.0), int(sl.get("m", 100)))
            ap = ctypes.cast(ctypes.byref(keep), _vp)
        t = Tuning()
        _check(load().fsmc_autotune(self._h, target._h, ALGO[algo], ap, PREC[prec], n_chains,
                                    cache_path.encode() if cache_path else None, ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def wait_all(self, timeout_s=600.0):
        _check(load().fsmc_wait_all(self._h, timeout_s))

    def close(self):
        if self._h:
            load().fsmc_engine_destroy(self._h)
            self._h = _vp()
            for o in self._objs:
                o._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Target:
    def __init__(self, engine, kind, d, params, n_data=0):
        self.engine = engine
        self.d = d
        p = _f64(params if params is not None else np.zeros(0))
        self._params = p
        self._h = _vp()
        _check(load().fsmc_target_create(engine.handle, TARGET[kind], d, n_data,
                                         _p(p) if p.size else None, p.size, ctypes.byref(self._h)))
        engine._objs.append(self)

    def close(self):
        """Frees the target's device copies (jobs on it must be closed first)."""
        if self._h:
            load().fsmc_target_destroy(self._h)
            self._h = _vp()
            if self in self.engine._objs:
                self.engine._objs.remove(self)


class Job:
    def __init__(self, engine, target, algo, n_chains, n_samples, x0, seed, prec, store, dr, nuts,
                 tuning, slice=None):
        self.engine, self.target = engine, target
        self.m, self.n, self.d = n_chains, n_samples, target.d
        self.prec = prec
        ap = None
        if algo == "dr":
            dr = dr or {}
            self._ap = DRParams(dr.get("n_stages", 3), dr.get("scale0", 1.0), dr.get("factor", 0.5),
                                int(dr.get("symmetric", 0)))
            ap = ctypes.cast(ctypes.byref(self._ap), _vp)
        elif algo == "nuts":
            nuts = nuts or {}
            self._ap = NUTSParams(nuts.get("eps", 0.05), nuts.get("max_depth", 10),
                                  nuts.get("max_dH", 1000.0))
            ap = ctypes.cast(ctypes.byref(self._ap), _vp)
        elif algo == "slice":
            sl = slice or {}
            self._ap = SliceParams(sl.get("w", 1.0), int(sl.get("m", 100)))
            ap = ctypes.cast(ctypes.byref(self._ap), _vp)
        x0a = None if x0 is None else _f64(x0).reshape(n_chains, target.d)
        self._h = _vp()
        _check(load().fsmc_job_create(engine.handle, target._h, ALGO[algo], ap, PREC[prec],
                                      n_chains, n_samples, _p(x0a), seed, 1 if store else 0,
                                      ctypes.byref(self._h)))
        engine._objs.append(self)
        if tuning:
            t = Tuning(*(int(tuning.get(name, 0)) for name, _ in Tuning._fields_))
            _check(load().fsmc_job_set_tuning(self._h, ctypes.byref(t)))

    @property
    def handle(self):
        return self._h

    def tuning(self):
        t = Tuning()
        _check(load().fsmc_job_get_tuning(self._h, ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def bytes(self):
        return load().fsmc_job_bytes(self._h)

    def run(self, mode="fsm", max_fsm_steps=0, stream=None):
        _check(load().fsmc_job_run(self._h, MODE[mode], max_fsm_steps, stream))

    def reset(self):
        _check(load().fsmc_job_reset(self._h))

    def progress(self):
        mn = ctypes.c_int64()
        done = ctypes.c_int()
        _check(load().fsmc_job_progress(self._h, ctypes.byref(mn), ctypes.byref(done)))
        return mn.value, bool(done.value)

    def samples(self, chain0=0, n_chains=None, sample0=0, n_samp=None):
        n_chains = self.m - chain0 if n_chains is None else n_chains
        n_samp = self.n - sample0 if n_samp is None else n_samp
        out = np.zeros((n_chains, n_samp, self.d))
        _check(load().fsmc_read_samples(self._h, chain0, n_chains, sample0, n_samp, _p(out)))
        return out

    def samples_dev(self, dst_ptr, chain0, n_chains, sample0, n_samp, stream=None):
        _check(load().fsmc_read_samples_dev(self._h, chain0, n_chains, sample0, n_samp, dst_ptr,
                                            stream))

    def loop_counts(self):
        c = np.zeros((self.m, self.n), dtype=np.int32)
        a = np.zeros((self.m, self.n), dtype=np.int32)
        s = np.zeros(self.m, dtype=np.int64)
        _check(load().fsmc_read_loop_counts(self._h, _p(c, _ip), _p(a, _ip), _p(s, _lp)))
        return c, a, s

    def state(self):
        x = np.zeros((self.m, self.d))
        _check(load().fsmc_read_state(self._h, _p(x)))
        return x

    def moments(self, sx=None, sx2=None, nk=None):
        """Per-chain sums of x and x^2 over the samples so far, and the sample counts.  Callers
        may pass their own (e.g. pinned) float64 / int64 arrays of shapes [m, d], [m, d], [m]."""
        sx = np.zeros((self.m, self.d)) if sx is None else sx
        sx2 = np.zeros((self.m, self.d)) if sx2 is None else sx2
        nk = np.zeros(self.m, dtype=np.int64) if nk is None else nk
        for a, shape, dt in ((sx, (self.m, self.d), np.float64), (sx2, (self.m, self.d), np.float64),
                             (nk, (self.m,), np.int64)):
            if a.shape != shape or a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("moments: output arrays must be C-contiguous %s of shape %s" % (dt, shape))
        _check(load().fsmc_read_moments(self._h, _p(sx), _p(sx2), _p(nk, _lp)))
        return sx, sx2, nk

    def stats(self):
        s = Stats()
        _check(load().fsmc_read_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def snapshot(self):
        n = ctypes.c_size_t(0)
        _check(load().fsmc_job_snapshot(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(load().fsmc_job_snapshot(self._h, buf, ctypes.byref(n)))
        return bytes(buf.raw)

    def restore(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(load().fsmc_job_restore(self._h, buf, len(blob)))

    def submit(self, mode="fsm"):
        _check(load().fsmc_submit(self.engine.handle, self._h, MODE[mode]))

    def cancel(self):
        _check(load().fsmc_cancel(self._h))

    def poll(self):
        done = ctypes.c_int()
        lat = ctypes.c_double()
        _check(load().fsmc_poll(self._h, ctypes.byref(done), ctypes.byref(lat)))
        return bool(done.value), lat.value

    def close(self):
        if self._h:
            load().fsmc_job_destroy(self._h)
            self._h = _vp()
            if self in self.engine._objs:
                self.engine._objs.remove(self)


def ess_run_static(kind, d, L_ptr, vec_ptr, noise_var, n_chains, n_samples, x0_ptr, seed,
                   lanes_per_chain, samples_ptr, counts_ptr, stream=None):
    """fsmc_ess_run_static: every argument ending in _ptr is a device address (int)."""
    _check(load().fsmc_ess_run_static(TARGET[kind], d, L_ptr, vec_ptr, noise_var, n_chains,
                                      n_samples, x0_ptr, seed, lanes_per_chain, samples_ptr,
                                      counts_ptr, stream))
