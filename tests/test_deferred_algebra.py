"""The deferred update's bookkeeping, replayed in FP64 numpy against the oracle.

The FP32 solver can keep a chunk's rank-1 updates as terms instead of applying them to
R (grbk_opts.deferred).  R stays at its value R^0 from the chunk's start, and the
current residual is R^0 - sum_j U'_j v_j^T, with U'_j = c_j A A_{i_j}^T and
v_j = (R_{i_j} B^T) B.  The solver then
  - assembles the selected row as R^0_{i_k} - sum_{j<k} U'_{i_k j} v_j;
  - forms d_i = R^0_i . v_k - sum_{j<k} U'_{ij} (v_j . v_k);
  - updates s_i <- s_i - 2 U'_{ik} d_i + U'_{ik}^2 ||v_k||^2.
These identities are what the kernel computes in FP32/double-float.  The test replays
them in FP64 on the rows the oracle picked and checks the results against the oracle's
own trajectory:
  - the traced ||R^k||_F^2 of every iteration (the oracle computes it from the updated
    R);
  - the final R (the write-back, R^0 - sum_j U'_j v_j^T).
Any dropped term, wrong sign or wrong index in the identities moves these far past
rounding.  No CUDA code is involved; this pins the reformulation, not the kernel.
"""
import numpy as np
import pytest

import oracle
import workloads


def _replay(A, B, C, rows, alpha):
    m = A.shape[0]
    R0 = C.copy()
    a = np.einsum("ij,ij->i", A, A)
    G = A @ A.T
    s = np.einsum("ij,ij->i", R0, R0)
    Us, Vs, S = [], [], []
    for k, ik in enumerate(rows):
        S.append(s.sum())
        # the selected row from R^0 and the kept terms
        Rik = R0[ik].copy()
        for U, V in zip(Us, Vs):
            Rik -= U[ik] * V
        v = (Rik @ B.T) @ B
        U = (alpha / a[ik]) * G[:, ik]
        # d_i = R_i . v with R_i the current row, from R^0 and the Gram column v_j . v
        d = R0 @ v
        for Uj, Vj in zip(Us, Vs):
            d -= Uj * (Vj @ v)
        s = s - 2.0 * U * d + U * U * (v @ v)
        Us.append(U)
        Vs.append(v)
    R = R0.copy()
    for U, V in zip(Us, Vs):
        R -= np.outer(U, V)
    return np.array(S), R, s


@pytest.mark.parametrize("variant,theta", [("grbk", 0.5), ("rgrbk", 0.8), ("mwrbk", 1.0)])
def test_deferred_bookkeeping_reproduces_the_oracle(variant, theta):
    A, B, C, _ = workloads.gaussian(60, 12, 9, 40, seed=41)
    alpha = 1.0 / np.linalg.norm(B, 2) ** 2
    T = 64
    orc = oracle.solve(A, B, C, variant, theta=theta, alpha=alpha, seed=7, maxit=T, mode=oracle.MODE_FACTORED,
                       want_R=True)
    S, R, s = _replay(A, B, C, orc["rows"], alpha)
    assert np.max(np.abs(S - orc["S"]) / orc["S"]) < 1e-12
    scale = np.abs(C).max()
    assert np.max(np.abs(R - orc["R"])) < 1e-12 * scale
    # the carried row norms equal the norms of the written-back R
    s_direct = np.einsum("ij,ij->i", R, R)
    assert np.max(np.abs(s - s_direct)) < 1e-10 * s_direct.max()


def test_dropping_the_gram_correction_is_detected():
    """Without the v_j . v_k correction the carried norms leave the oracle's at once."""
    A, B, C, _ = workloads.gaussian(60, 12, 9, 40, seed=42)
    alpha = 1.0 / np.linalg.norm(B, 2) ** 2
    orc = oracle.solve(A, B, C, "grbk", alpha=alpha, seed=3, maxit=16, mode=oracle.MODE_FACTORED)
    rows = orc["rows"]
    R0 = C.copy()
    a = np.einsum("ij,ij->i", A, A)
    G = A @ A.T
    s = np.einsum("ij,ij->i", R0, R0)
    Us, Vs, S = [], [], []
    for ik in rows:
        S.append(s.sum())
        Rik = R0[ik].copy()
        for U, V in zip(Us, Vs):
            Rik -= U[ik] * V
        v = (Rik @ B.T) @ B
        U = (alpha / a[ik]) * G[:, ik]
        d = R0 @ v  # the correction by the earlier terms left out
        s = s - 2.0 * U * d + U * U * (v @ v)
        Us.append(U)
        Vs.append(v)
    assert np.max(np.abs(np.array(S) - orc["S"]) / orc["S"]) > 1e-6
