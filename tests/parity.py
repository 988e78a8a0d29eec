"""Trajectory comparison between the CUDA path and the FP64 oracle.

Tolerances:
  * FP64 jobs: every sample within 1e-10 norm-wise relative error
    |x_gpu - x_ora|_inf / max(1, |x_ora|_inf), and identical loop counts N_ij.
  * FP32 jobs: samples agree within 1e-4 (same norm) up to the first branch flip, i.e.
    the first sample whose loop count differs or whose error exceeds 1e-2 (a different
    accept/reject outcome moves the chain by O(step size), rounding moves it by ~1e-6).
    Errors between 1e-4 and 1e-2 are neither and fail the comparison.
"""
import numpy as np

FP64_TOL = 1e-10
FP32_TOL = 1e-4
FLIP_ERR = 1e-2


def sample_errors(x_gpu, x_ora):
    num = np.abs(x_gpu - x_ora).max(axis=-1)
    den = np.maximum(1.0, np.abs(x_ora).max(axis=-1))
    return num / den


def compare(x_gpu, c_gpu, x_ora, c_ora, prec):
    """Returns dict(flipped=#chains with a flip, first_flip=[...], max_err=before flips)."""
    m, n = c_ora.shape
    err = sample_errors(x_gpu, x_ora)
    if prec == "fp64":
        assert np.array_equal(c_gpu, c_ora), "loop counts differ in FP64"
        mx = float(err.max()) if err.size else 0.0
        assert mx <= FP64_TOL, mx
        return {"flipped": 0, "first_flip": [], "max_err": mx}
    flipped = 0
    firsts = []
    mx = 0.0
    for j in range(m):
        bad = np.nonzero((c_gpu[j] != c_ora[j]) | (err[j] > FLIP_ERR))[0]
        end = int(bad[0]) if bad.size else n
        if bad.size:
            flipped += 1
            firsts.append(end)
        if end:
            e = float(err[j, :end].max())
            mx = max(mx, e)
    assert mx <= FP32_TOL, mx
    return {"flipped": flipped, "first_flip": firsts, "max_err": mx}
