"""The plain form at scale: A 4000x1000 = U diag(sigma) V^T and B 800x3000 built
the same way (Haar U, V; sigma log-spaced from 1 to 1e-2), X* N(0,1),
C = A X* B, and its rank-deficient variant (rank 600 for A, 500 for B), with
the relaxation theta in {0.3, 0.5, 0.8} (Algorithm 4; theta = 1/2 is
Algorithm 3).

* FP64: the first 200 selected rows identical to the FP64 oracle's (FACTORED
  mode: the same rank-1 update of R re-associated), and X^200, the kept R^200
  and its row norms within 1e-9 relative.  This system needs about 3e11
  iterations to reach RSE 1e-6 (its condition number is 100 on each side), so
  it is checked at a fixed budget.
* Rank-deficient: the same parity, and the Lemma 3.2 invariant at the full
  size: from X^0 = 0 every iterate stays in the range where
  X = A^+ A X B B^+ (the limit of Theorem 3.3 with X^0 = 0 is A^+ C B^+).
* FP32 with the split-BF16 refresh every 64 iterations (the precision form):
  the rows agree with the FP64 oracle's up to the first decision FP32 cannot
  resolve (tests/parity_rows.py), and at the fixed budget of 200 iterations
  the FP32 iterate's distance to the FP64 oracle's iterate is stated against
  FP32's own resolution: within 1e-4 relative when every row agreed.
"""
import numpy as np
import pytest

import oracle
import workloads
from parity_rows import compare_rows

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2408_05444_gb300 as g  # noqa: E402

K = 200
_CACHE = {}


def _system(rank_deficient):
    if rank_deficient not in _CACHE:
        A, B, C, Xs = workloads.config_scale(rank_deficient=rank_deficient)
        _CACHE[rank_deficient] = (A, B, C, Xs, 1.0 / np.linalg.norm(B, 2) ** 2)
    return _CACHE[rank_deficient]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _oracle(rank_deficient, variant, theta):
    key = ("orc", rank_deficient, variant, theta)
    if key not in _CACHE:
        A, B, C, Xs, al = _system(rank_deficient)
        _CACHE[key] = oracle.solve(A, B, C, variant, theta=theta, alpha=al, seed=17, maxit=K,
                                   mode=oracle.MODE_FACTORED, want_R=True)
    return _CACHE[key]


def _gpu(rank_deficient, variant, theta, precision, **kw):
    A, B, C, Xs, al = _system(rank_deficient)
    ctx = g.grbk_create(A, B, C, precision=precision, alpha=al, trace_len=K, **kw)
    X = np.zeros((A.shape[1], B.shape[0]))
    st, res = g.grbk_solve(ctx, variant, theta=theta, maxit=K, seed=17, X_out=X)
    assert st == g.GRBK_OK and res["iters"] == K
    out = dict(X=X, rows=ctx.row_trace[:K].astype(np.int64).copy(), S=ctx.s_trace[:K].copy())
    if precision == "f64":
        R = np.zeros((A.shape[0], B.shape[1]))
        g.grbk_get_residual(ctx, R)
        s = np.zeros(A.shape[0])
        g.grbk_get_rownorms(ctx, s)
        out.update(R=R, s=s)
    g.grbk_destroy(ctx)
    return out


CASES = [(False, "rgrbk", 0.3), (False, "grbk", 0.5), (False, "rgrbk", 0.8), (True, "rgrbk", 0.3),
         (True, "grbk", 0.5), (True, "rgrbk", 0.8)]


@pytest.mark.parametrize("rank_deficient,variant,theta", CASES)
def test_fp64_matches_oracle_at_scale(rank_deficient, variant, theta):
    A, B, C, Xs, al = _system(rank_deficient)
    orc = _oracle(rank_deficient, variant, theta)
    got = _gpu(rank_deficient, variant, theta, "f64")
    assert np.array_equal(got["rows"], orc["rows"][:K]), np.nonzero(got["rows"] != orc["rows"][:K])[0][:3]
    assert np.max(np.abs(got["S"] - orc["S"][:K]) / orc["S"][:K]) < 1e-9
    assert _rel(got["X"], orc["X"]) < 1e-9
    assert np.max(np.abs(got["R"] - orc["R"])) <= 1e-9 * np.max(np.abs(C))
    assert np.max(np.abs(got["s"] - orc["s"]) / np.maximum(orc["s"], 1e-300)) < 1e-9
    if rank_deficient:
        # Lemma 3.2 with X^0 = 0: X^k - A^+ A X^k B B^+ stays 0.  A^+ A and B B^+ are the
        # projectors onto the row space of A and the column space of B, formed from the
        # singular vectors of the singular values above 1e-10 sigma_max (A and B have
        # exactly 600 and 500 such values; the others are at the rounding level)
        def proj(V, sv):
            r = int(np.sum(sv > 1e-10 * sv[0]))
            return V[:, :r] @ V[:, :r].T, r
        _, sa, Vta = np.linalg.svd(A, full_matrices=False)
        Ub, sb, _ = np.linalg.svd(B, full_matrices=False)
        Pa, ra = proj(Vta.T, sa)
        Pb, rb = proj(Ub, sb)
        assert (ra, rb) == (600, 500)
        X = got["X"]
        assert np.linalg.norm(X - Pa @ X @ Pb) <= 1e-9 * np.linalg.norm(X)


@pytest.mark.parametrize("rank_deficient,variant,theta", [(False, "rgrbk", 0.3), (False, "grbk", 0.5),
                                                          (False, "rgrbk", 0.8), (True, "grbk", 0.5)])
def test_fp32_precision_form_against_fp64_oracle_at_scale(rank_deficient, variant, theta):
    A, B, C, Xs, al = _system(rank_deficient)
    orc = _oracle(rank_deficient, variant, theta)
    got = _gpu(rank_deficient, variant, theta, "f32", refresh_T=64, check_every=64)
    kk = compare_rows(got["rows"], orc, K)
    err = _rel(got["X"], orc["X"])
    print(f"\nFP32 vs FP64 oracle, {'rank-deficient' if rank_deficient else 'full rank'} {variant} "
          f"theta={theta}: rows agree for {kk}/{K}, ||X32 - X64|| / ||X64|| = {err:.3e}")
    if kk == K:
        assert err < 1e-4
    # ||R^k||^2 traced in FP64 sums of the FP32 residual, against the FP64 oracle while the rows agree
    assert np.max(np.abs(got["S"][:kk] - orc["S"][:kk]) / orc["S"][:kk]) < 1e-4
