"""The FP32 solver's deferred update (grbk_opts.deferred) against its in-place update.

Both run the same iterates of Algorithms 1-5; the deferred one applies the rank-1
updates of a chunk later.  During a chunk R stays at its value R^0 from the chunk's
start: an iteration reads R^0 once, assembles the selected row R_{i_k} from R^0 and the
kept terms U'_j v_j^T (the same fused multiply-adds, in the same order, as the in-place
update), and carries the row norms by ||R_i - U'_i v||^2 = s_i - 2 U'_i (R_i . v) +
U'_i^2 ||v||^2.  After the chunk R is written back with the terms in iteration order,
or recomputed by the refresh.

So w, v, u and X are bitwise the in-place update's as long as the same rows are picked,
and so is R after each write-back.  Only the row norms inside a chunk differ: the
recurrence follows the unrounded sequence, while the in-place update stores every
updated element in FP32 (unit roundoff u = 2^-24), which moves ||R||_F^2 by at most
2 k u relative after k updates (7.6e-6 at k = 64, all errors aligned) and by about
2 u sqrt(k / (m n)) with random signs (about 1e-9 on these systems).  The traced
||R^k||_F^2 must agree to 1e-7: far above that rounding, far below what a wrong or
missing term of the recurrence gives.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2408_05444_gb300 as g  # noqa: E402

g.lib()


def _run(A, B, C, variant, deferred, theta=0.5, maxit=300, seed=3, **kw):
    al = 1.0 / np.linalg.norm(B, 2) ** 2
    ctx = g.grbk_create(A, B, C, precision="f32", alpha=al, trace_len=maxit, deferred=deferred, **kw)
    X = np.zeros((A.shape[1], B.shape[0]))
    st, res = g.grbk_solve(ctx, variant, theta=theta, maxit=maxit, seed=seed, X_out=X)
    out = dict(X=X, st=st, res=res)
    if kw.get("form", "full") == "full":
        R = np.zeros((A.shape[0], B.shape[1]), dtype=np.float32)
        g.grbk_get_residual(ctx, R)
        out["R"] = R
    s = np.zeros(A.shape[0])
    g.grbk_get_rownorms(ctx, s)
    out["s"] = s
    out["rows"] = ctx.row_trace[:res["iters"]].astype(np.int64).copy()
    out["S"] = ctx.s_trace[:res["iters"]].copy()
    g.grbk_destroy(ctx)
    return out


def _compare(d, e, s_exact=True):
    assert d["res"]["deferred"] == 1 and e["res"]["deferred"] == 0
    assert d["res"]["iters"] == e["res"]["iters"]
    assert np.array_equal(d["rows"], e["rows"])
    assert np.array_equal(d["X"], e["X"])
    if "R" in d:
        assert np.array_equal(d["R"], e["R"])
    if s_exact:  # the row norms of the written-back R are recomputed
        assert np.array_equal(d["s"], e["s"])
    rel = np.abs(d["S"] - e["S"]) / np.maximum(e["S"], 1e-300)
    assert rel.max() < 1e-7, rel.max()


@pytest.mark.parametrize("variant,theta", [("grbk", 0.5), ("rgrbk", 0.8), ("mwrbk", 1.0), ("rbk", 0.5)])
def test_deferred_chunks_with_write_back(variant, theta):
    """No refresh: every chunk of 64 iterations ends with a write-back (the last one
    after 44 iterations); several CTAs, each with a slab of two vectors of R_{i_k}."""
    A, B, C, _ = workloads.gaussian(4000, 60, 50, 800, seed=31)
    d = _run(A, B, C, variant, True, theta=theta, check_every=64)
    e = _run(A, B, C, variant, False, theta=theta, check_every=64)
    _compare(d, e)


def test_deferred_with_refresh_and_ragged_slabs():
    """The periodic refresh replaces the write-back; n = 100 gives 32 vectors of R_{i_k}
    over more CTAs than that, so most CTAs have no slab."""
    A, B, C, _ = workloads.gaussian(4000, 40, 30, 100, seed=32)
    d = _run(A, B, C, "grbk", True, refresh_T=64, check_every=64, maxit=330)
    e = _run(A, B, C, "grbk", False, refresh_T=64, check_every=64, maxit=330)
    _compare(d, e)


def test_deferred_stop_inside_a_chunk():
    """A relative-residual stop in the middle of a chunk: the partial chunk is
    written back and both updates stop after the same iteration."""
    A, B, C, _ = workloads.gaussian(1500, 30, 20, 400, seed=33)
    runs = []
    for deferred in (True, False):
        al = 1.0 / np.linalg.norm(B, 2) ** 2
        ctx = g.grbk_create(A, B, C, precision="f32", alpha=al, check_every=48, stop_kind="relres",
                            deferred=deferred)
        X = np.zeros((A.shape[1], B.shape[0]))
        st, res = g.grbk_solve(ctx, "grbk", maxit=5000, tol=0.3, X_out=X)
        R = np.zeros((A.shape[0], B.shape[1]), dtype=np.float32)
        g.grbk_get_residual(ctx, R)
        g.grbk_destroy(ctx)
        runs.append((res, X, R))
    (rd, Xd, Rd), (re, Xe, Re) = runs
    assert rd["deferred"] == 1 and re["deferred"] == 0
    assert rd["iters"] == re["iters"] and rd["iters"] < 5000
    assert np.array_equal(Xd, Xe) and np.array_equal(Rd, Re)


def test_deferred_row_space_form():
    """The row-space form (Z = R Bt^T kept) with the deferred update: same rows and X."""
    A, B, C, _ = workloads.gaussian(3000, 40, 30, 500, seed=34)
    d = _run(A, B, C, "rgrbk", True, theta=0.7, refresh_T=64, check_every=64, form="rowspace")
    e = _run(A, B, C, "rgrbk", False, theta=0.7, refresh_T=64, check_every=64, form="rowspace")
    _compare(d, e, s_exact=False)


def test_deferred_only_for_short_chunks():
    """Chunks longer than 64 iterations keep the in-place update."""
    A, B, C, _ = workloads.gaussian(500, 20, 10, 60, seed=35)
    r = _run(A, B, C, "grbk", True, check_every=100, maxit=120)
    assert r["res"]["deferred"] == 0
