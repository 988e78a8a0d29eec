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
# Branch flips allowed per FP32 trajectory test: max(2, 3 x the count measured on B300).  Every
# FP32 trajectory test of the current kernels measured 0 flipped chains (ESS GP-logit 48 x 400 at
# d = 100..256 and 8/16/32 lanes, DR funnel 512 x 1000, NUTS logistic regression 32 x 200, and the
# sampled chains of the full-size runs over their first 1000 samples).
FLIP_ALLOW = 2
# A transition that disagrees with the oracle's from the same state must have met a decision
# whose compared value lay within this relative distance of its threshold (the oracle's smallest
# decision margin, oracle.transitions); anything else is an error, not a rounding-induced flip.
NEAR_TIE = 1e-4


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


def transitions_agree(x_gpu, c_gpu, ref, what):
    """Per-transition comparison with the oracle (ref = oracle.transitions(...) from the same
    states): every transition agrees within FP32_TOL with an equal loop count, or is a near tie
    (the oracle met a decision within NEAR_TIE of its threshold).  Returns the agreeing mask."""
    err = sample_errors(x_gpu, ref["x"])
    ok = (ref["counts"] == c_gpu) & (err <= FP32_TOL)
    ties = ref["margin"] < NEAR_TIE
    bad = ~ok & ~ties
    print("%s: %d of %d transitions agree (max err %.3g); %d disagree, all near ties: %s; "
          "near ties among all transitions: %d" % (what, ok.sum(), ok.size, err[ok].max() if ok.any() else 0,
                                                   (~ok).sum(), not bad.any(), ties.sum()))
    assert not bad.any(), (what, np.nonzero(bad)[0][:8], err[bad][:8], ref["margin"][bad][:8])
    assert (~ok).sum() <= max(FLIP_ALLOW, ok.size // 200)
    return ok
