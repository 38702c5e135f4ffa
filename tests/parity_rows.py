"""Row-sequence comparison of an FP32 GPU run against the FP64 oracle.

The oracle records, for every decision k, the relative margin of its admission
test (min_i |r_i - t| / t) and of its pick (distance of u S_J to the nearest
prefix boundary, relative to S_J).  An FP32 residual resolves a decision only
when that margin exceeds its own rounding.  The kept residual's absolute
rounding error stays near 2^-24 ||R^0|| (times a slowly growing factor), so its
relative error in the row norms at step k is about 2^-24 sqrt(S_0 / S_k):

    eps_k = max(1e-6, 64 * 2^-24 * sqrt(S_0 / S_k))

* the runs must select the same rows up to their first disagreement, and that
  disagreement may only happen at a decision whose oracle margin is below
  max(1e-5, 10 eps_k) (otherwise the GPU took a decision that FP32 resolves,
  differently from FP64: a bug);
* every system must agree at least up to its first decision with margin below
  eps_k, so each system contributes a minimum number of compared decisions,
  fixed by the oracle alone.

compare_rows returns the number of agreeing leading decisions."""
import numpy as np


def decision_margins(orc):
    adm = np.where(np.isnan(orc["margin_adm"]), np.inf, orc["margin_adm"])
    return np.minimum(orc["margin_pick"], adm)


def resolution(orc, K):
    S = np.asarray(orc["S"][:K], dtype=np.float64)
    return np.maximum(1e-6, 64 * 2.0 ** -24 * np.sqrt(S[0] / np.maximum(S, 1e-300)))


def compare_rows(gpu_rows, orc, K):
    K = min(K, len(orc["rows"]))
    rows = np.asarray(gpu_rows[:K])
    ref = np.asarray(orc["rows"][:K])
    margins = decision_margins(orc)[:K]
    eps = resolution(orc, K)
    diff = np.nonzero(rows != ref)[0]
    agreed = int(diff[0]) if len(diff) else K
    if agreed < K:
        lim = max(1e-5, 10 * eps[agreed])
        assert margins[agreed] < lim, (
            f"decision {agreed}: GPU picked {rows[agreed]}, oracle {ref[agreed]} at relative margin "
            f"{margins[agreed]:.3g} (resolved by FP32 down to {lim:.3g})")
    near = np.nonzero(margins < eps)[0]
    floor = int(near[0]) if len(near) else K
    assert agreed >= floor, (agreed, floor)
    return agreed
