"""GPU parity of the row-space residual form against the FP64 CPU oracle.

The row-space form keeps Z = R Bt^T (m x r, Bt an orthonormal basis of the
row space of B) and the fixed row offsets ||Rperp_i||^2 instead of R.  It is an
exact rewriting of Algorithm 3's residual bookkeeping, so the oracle, which
keeps the full R, is the reference: in FP64 the selected rows must be the same
for 1000 iterations, the traced ||R^k||_F^2 and X must agree to 1e-9, on
consistent and inconsistent systems, full-rank and rank-deficient B.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2408_05444_gb300 as g  # noqa: E402

g.lib()


def _alpha(B):
    return 1.0 / np.linalg.norm(B, 2) ** 2


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _run(A, B, C, variant, theta=0.5, maxit=1000, seed=0, X0=None, precision="f64", alpha=None, trace=True,
         **kw):
    ctx = g.grbk_create(A, B, C, precision=precision, alpha=alpha if alpha is not None else 0.0,
                        trace_len=maxit if trace else 0, form="rowspace", **kw)
    X = np.zeros((A.shape[1], B.shape[0]))
    st, res = g.grbk_solve(ctx, variant, theta=theta, X0=X0, maxit=maxit, seed=seed, X_out=X)
    s = np.zeros(A.shape[0])
    g.grbk_get_rownorms(ctx, s)
    out = dict(X=X, s=s, st=st, res=res, form=g.grbk_form_info(ctx), dims=g.grbk_info(ctx)[0])
    if trace:
        out["rows"] = ctx.row_trace[:res["iters"]].astype(np.int64).copy()
        out["S"] = ctx.s_trace[:res["iters"]].copy()
    g.grbk_destroy(ctx)
    return out


def _same_rows(gpu_rows, orc, floor=1e-20):
    rows, S = orc["rows"], orc["S"]
    live = np.nonzero(S <= floor * S[0])[0] if len(S) else []
    if len(live):
        rows, gpu_rows = rows[:int(live[0])], gpu_rows[:int(live[0])]
    n = min(len(rows), len(gpu_rows))
    bad = np.nonzero(gpu_rows[:n] != rows[:n])[0]
    if len(bad):
        k = int(bad[0])
        pytest.fail(f"row sequence differs first at k={k}: gpu {gpu_rows[k]} oracle {rows[k]}; "
                    f"oracle margins adm={orc['margin_adm'][k]:.3e} pick={orc['margin_pick'][k]:.3e}")
    assert len(gpu_rows) == len(rows)


CASES = [("grbk", 0.5), ("rgrbk", 0.3), ("rgrbk", 0.8), ("mwrbk", 1.0), ("rbk", 0.5), ("bk", 0.5)]


@pytest.mark.parametrize("variant,theta", CASES)
def test_rowspace_rows_match_oracle_small_config(variant, theta):
    """A 200x100, B 80x150 (r = 80 < n = 150), consistent C: 1000 iterations."""
    A, B, C, Xs = workloads.config_small()
    al = _alpha(B)
    X0 = np.random.default_rng(3).standard_normal((100, 80)) if variant == "bk" else None
    orc = oracle.solve(A, B, C, variant, theta=theta, alpha=al, X0=X0, seed=7, maxit=1000,
                       mode=oracle.MODE_FACTORED)
    gpu = _run(A, B, C, variant, theta=theta, alpha=al, X0=X0, seed=7, maxit=1000)
    assert gpu["form"] == ("rowspace", 80) and gpu["dims"] == (200, 100, 80, 150)
    assert gpu["st"] == g.GRBK_OK and gpu["res"]["iters"] == 1000
    _same_rows(gpu["rows"], orc)
    assert np.max(np.abs(gpu["S"] - orc["S"]) / orc["S"]) < 1e-9
    assert _rel(gpu["X"], orc["X"]) < 1e-9


def test_rowspace_inconsistent_system_offsets():
    """C = A X* B + E with E outside the row space of B: the part of R that the
    updates never touch enters s_i through the fixed offsets, so the traced
    ||R^k||^2, the final row norms and the rows still match the oracle."""
    A, B, C, _ = workloads.gaussian(150, 30, 20, 90, seed=11)
    C = C + 0.3 * np.random.default_rng(5).standard_normal(C.shape)
    al = _alpha(B)
    for variant in ("grbk", "mwrbk"):
        orc = oracle.solve(A, B, C, variant, alpha=al, seed=2, maxit=800, mode=oracle.MODE_FACTORED, want_R=True)
        gpu = _run(A, B, C, variant, alpha=al, seed=2, maxit=800)
        assert gpu["form"] == ("rowspace", 20)
        _same_rows(gpu["rows"], orc)
        assert np.max(np.abs(gpu["S"] - orc["S"]) / orc["S"]) < 1e-9
        assert np.max(np.abs(gpu["s"] - orc["s"]) / np.maximum(orc["s"], 1e-300)) < 1e-8
        assert _rel(gpu["X"], orc["X"]) < 1e-9
    # the floor of ||R||^2 is the part outside the row space: ||C - C B^+ B||^2
    Cperp = C - C @ np.linalg.pinv(B) @ B
    assert np.sum(gpu["s"]) >= np.sum(Cperp ** 2) * (1 - 1e-9)


@pytest.mark.parametrize("m,p,q,n", [(37, 5, 7, 29), (1, 3, 2, 5), (300, 17, 3, 1), (129, 64, 33, 257),
                                     (2100, 40, 30, 1030), (90, 12, 40, 25)])
def test_rowspace_ragged_shapes(m, p, q, n):
    """Ragged sizes, one row, one column, q > n (r = n, no reduction)."""
    A, B, C, _ = workloads.gaussian(m, p, q, n, seed=m + n)
    al = _alpha(B)
    for variant in ("grbk", "mwrbk"):
        orc = oracle.solve(A, B, C, variant, alpha=al, seed=5, maxit=150, mode=oracle.MODE_FACTORED)
        gpu = _run(A, B, C, variant, alpha=al, seed=5, maxit=150, grid_ctas=4 if m > 8 else 0)
        assert gpu["form"] == ("rowspace", min(q, n))
        _same_rows(gpu["rows"], orc)
        assert _rel(gpu["X"], orc["X"]) < 1e-9


def test_rowspace_rank_deficient_b_and_bk_limit():
    """B of rank 6 with 10 rows (4 are combinations of the others): the pivoted
    factorisation finds r = 6, and ME-BK from X0 != 0 tends to the limit of
    Theorem 3.3, A^+ C B^+ + X0 - A^+ A X0 B B^+, as in the full form."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((14, 12)) @ np.diag([1.0] * 9 + [0.0] * 3) @ rng.standard_normal((12, 12))
    B = rng.standard_normal((10, 6)) @ rng.standard_normal((6, 17))
    Xs = rng.standard_normal((12, 10))
    C = A @ Xs @ B
    X0 = rng.standard_normal((12, 10))
    pinv = np.linalg.pinv
    lim = pinv(A) @ C @ pinv(B) + X0 - pinv(A) @ A @ X0 @ B @ pinv(B)
    ctx = g.grbk_create(A, B, C, precision="f64", stop_kind="relres", form="rowspace")
    assert g.grbk_form_info(ctx) == ("rowspace", int(np.linalg.matrix_rank(B))) == ("rowspace", 6)
    X = np.zeros((12, 10))
    st, res = g.grbk_solve(ctx, "bk", X0=X0, tol=1e-13, maxit=2_000_000, X_out=X)
    assert st == g.GRBK_OK
    assert _rel(X, lim) < 1e-9
    orc = oracle.solve(A, B, C, "grbk", X0=X0, seed=4, maxit=500, mode=oracle.MODE_FACTORED)
    gpu = _run(A, B, C, "grbk", X0=X0, seed=4, maxit=500, alpha=orc["alpha"])
    _same_rows(gpu["rows"], orc)
    assert _rel(gpu["X"], orc["X"]) < 1e-9


def test_rowspace_fp64_converges_to_rse_1e6():
    A, B, C, Xs = workloads.config_small()
    ctx = g.grbk_create(A, B, C, precision="f64", stop_kind="rse", x_ref=Xs, check_every=2048, form="rowspace")
    X = np.zeros((100, 80))
    st, res = g.grbk_solve(ctx, "grbk", tol=1e-6, maxit=3_000_000, seed=1, X_out=X)
    assert st == g.GRBK_OK, res
    assert _rel(X, Xs) <= 1e-6


def test_rowspace_fp32_precision_slice_rse():
    """2000x200 / 200x2000 slice (r = 200, a tenth of n): FP32 bulk with the
    split-BF16 refresh every 64 iterations reaches RSE <= 1e-4, and the first
    300 ME-MWRBK iterates stay within 1e-4 of the FP64 oracle's."""
    A, B, C, Xs = workloads.config_precision(2000, 200, 200, 2000)
    al = _alpha(B)
    ctx = g.grbk_create(A, B, C, precision="f32", alpha=al, stop_kind="rse", x_ref=Xs, refresh_T=64,
                        form="rowspace")
    assert g.grbk_form_info(ctx) == ("rowspace", 200)
    X = np.zeros((200, 200))
    st, res = g.grbk_solve(ctx, "grbk", tol=1e-4, maxit=2_000_000, seed=1, X_out=X)
    assert st == g.GRBK_OK, res
    assert _rel(X, Xs) <= 1e-4
    orc = oracle.solve(A, B, C, "mwrbk", alpha=al, maxit=300, mode=oracle.MODE_FACTORED, trace=False)
    gpu = _run(A, B, C, "mwrbk", alpha=al, maxit=300, precision="f32", trace=False, refresh_T=64)
    assert _rel(gpu["X"], orc["X"]) < 1e-4


def test_rowspace_keeps_no_full_residual():
    A, B, C, _ = workloads.gaussian(40, 6, 5, 30, seed=1)
    ctx = g.grbk_create(A, B, C, form="rowspace")
    with pytest.raises(g.GrbkError):
        g.grbk_get_residual(ctx, np.zeros((40, 30)))
    with pytest.raises(g.GrbkError):
        g.grbk_residual(ctx, np.zeros((6, 5)), np.zeros((40, 30)))
    g.grbk_destroy(ctx)


def test_rowspace_fp32_three_terms_from_nonzero_x0():
    """FP32 row-space form with the 3-term split refresh, started from X0 != 0 (its
    first residual is the transformed refresh Chat - A X0 Lt): RSE <= 1e-4."""
    A, B, C, Xs = workloads.config_precision(2000, 200, 200, 2000)
    X0 = Xs + 0.1 * np.random.default_rng(4).standard_normal(Xs.shape)
    ctx = g.grbk_create(A, B, C, precision="f32", stop_kind="rse", x_ref=Xs, refresh_T=64, split_terms=3,
                        form="rowspace")
    X = np.zeros_like(Xs)
    st, res = g.grbk_solve(ctx, "rgrbk", theta=0.5, X0=X0, tol=1e-4, maxit=2_000_000, seed=3, X_out=X)
    assert st == g.GRBK_OK, res
    assert _rel(X, Xs) <= 1e-4
    assert res["iters"] > 0
