"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs.

FP64 mode: the selected-row sequence must be identical for the first 1000
iterations of every variant (the random ones on the same Philox stream); the
traced ||R^k||_F^2, the iterate X and the kept residual must agree to 1e-9
relative (both sides compute in FP64 with different summation orders, so only
rounding separates them).  FP32 mode: RSE <= 1e-4 against the exact solution.
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


def _gpu_run(A, B, C, variant, theta=0.5, maxit=1000, seed=0, X0=None, precision="f64", alpha=None,
             trace=True, **kw):
    ctx = g.grbk_create(A, B, C, precision=precision, alpha=alpha if alpha is not None else 0.0,
                        trace_len=maxit if trace else 0, **kw)
    X = np.zeros((A.shape[1], B.shape[0]))
    st, res = g.grbk_solve(ctx, variant, theta=theta, X0=X0, maxit=maxit, seed=seed, X_out=X)
    R = np.zeros((A.shape[0], B.shape[1]), dtype=np.float64 if precision == "f64" else np.float32)
    g.grbk_get_residual(ctx, R)
    s = np.zeros(A.shape[0])
    g.grbk_get_rownorms(ctx, s)
    out = dict(X=X, R=R.astype(np.float64), s=s, st=st, res=res)
    if trace:
        out["rows"] = ctx.row_trace[:res["iters"]].astype(np.int64).copy()
        out["S"] = ctx.s_trace[:res["iters"]].copy()
    g.grbk_destroy(ctx)
    return out


def _assert_same_rows(gpu_rows, orc, floor=1e-20):
    """Rows must agree while the residual is above the rounding floor: once
    ||R^k||^2 <= floor * ||R^0||^2 the row residuals are rounding noise and the
    oracle's own residual modes (Gram / factored / literal) disagree too."""
    rows = orc["rows"]
    S = orc["S"]
    live = np.nonzero(S <= floor * S[0])[0] if len(S) else []
    if len(live):
        rows = rows[:int(live[0])]
        gpu_rows = gpu_rows[:int(live[0])]
    n = min(len(rows), len(gpu_rows))
    bad = np.nonzero(gpu_rows[:n] != rows[:n])[0]
    if len(bad):
        k = int(bad[0])
        pytest.fail(f"row sequence differs first at k={k}: gpu {gpu_rows[k]} oracle {rows[k]}; "
                    f"oracle margins adm={orc['margin_adm'][k]:.3e} pick={orc['margin_pick'][k]:.3e}")
    assert len(gpu_rows) == len(rows)


CASES = [("grbk", 0.5), ("rgrbk", 0.3), ("rgrbk", 0.8), ("mwrbk", 1.0), ("rbk", 0.5), ("bk", 0.5)]


@pytest.mark.parametrize("variant,theta", CASES)
def test_fp64_row_sequence_small_config(variant, theta):
    """A 200x100, B 80x150, X* 100x80 (all N(0,1)), C = A X* B: 1000 iterations."""
    A, B, C, Xs = workloads.config_small()
    al = _alpha(B)
    X0 = None
    if variant == "bk":
        X0 = np.random.default_rng(3).standard_normal((100, 80))
    orc = oracle.solve(A, B, C, variant, theta=theta, alpha=al, X0=X0, seed=7, maxit=1000,
                       mode=oracle.MODE_FACTORED, want_R=True)
    gpu = _gpu_run(A, B, C, variant, theta=theta, alpha=al, X0=X0, seed=7, maxit=1000)
    assert gpu["st"] == g.GRBK_OK and gpu["res"]["iters"] == 1000
    _assert_same_rows(gpu["rows"], orc)
    assert np.max(np.abs(gpu["S"] - orc["S"]) / orc["S"]) < 1e-9
    assert _rel(gpu["X"], orc["X"]) < 1e-9
    assert np.max(np.abs(gpu["R"] - orc["R"])) < 1e-9 * np.max(np.abs(C))
    assert np.max(np.abs(gpu["s"] - orc["s"]) / np.maximum(orc["s"], 1e-300)) < 1e-8


@pytest.mark.parametrize("m,p,q,n", [(37, 5, 7, 29), (1, 3, 2, 5), (300, 17, 3, 1), (129, 64, 33, 257),
                                     (2100, 40, 30, 1030)])
def test_fp64_ragged_shapes(m, p, q, n):
    """Sizes that are not multiples of anything (ragged tails of every tile),
    a single row, a single column, several CTAs."""
    A, B, C, _ = workloads.gaussian(m, p, q, n, seed=m + n)
    al = _alpha(B)
    for variant in ("grbk", "mwrbk"):
        orc = oracle.solve(A, B, C, variant, alpha=al, seed=5, maxit=150, mode=oracle.MODE_FACTORED, want_R=True)
        gpu = _gpu_run(A, B, C, variant, alpha=al, seed=5, maxit=150, grid_ctas=4 if m > 8 else 0)
        _assert_same_rows(gpu["rows"], orc)
        assert _rel(gpu["X"], orc["X"]) < 1e-9
        assert np.max(np.abs(gpu["R"] - orc["R"])) < 1e-9 * max(np.max(np.abs(C)), 1e-300)


def test_fp64_chunks_and_grids_do_not_change_the_result():
    """The chunk length between host checks and the number of CTAs change the
    summation order only: same rows, X equal to 1e-12."""
    A, B, C, _ = workloads.gaussian(300, 20, 15, 200, seed=2)
    al = _alpha(B)
    runs = [_gpu_run(A, B, C, "grbk", alpha=al, seed=3, maxit=700, grid_ctas=gc, check_every=ce)
            for gc, ce in ((1, 0), (3, 17), (8, 256), (0, 1))]
    for r in runs[1:]:
        assert np.array_equal(r["rows"], runs[0]["rows"])
        assert _rel(r["X"], runs[0]["X"]) < 1e-12


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_gram_and_gemv_paths_agree(precision):
    """u = (A A^T)_{:,i} from the precomputed Gram matrix (the practice note after
    Algorithm 3) and u = A A_i^T streamed every iteration give the same rows, and
    iterates equal to rounding (FP64) or to FP32 accuracy."""
    A, B, C, _ = workloads.gaussian(333, 41, 29, 211, seed=14)
    al = _alpha(B)
    runs = [_gpu_run(A, B, C, "rgrbk", theta=0.6, alpha=al, seed=4, maxit=400, precision=precision,
                     use_gram=ug, refresh_T=(64 if precision == "f32" else 0)) for ug in (1, -1)]
    assert runs[0]["res"]["gram"] == 1 and runs[1]["res"]["gram"] == 0
    if precision == "f64":
        assert np.array_equal(runs[0]["rows"], runs[1]["rows"])
        assert _rel(runs[0]["X"], runs[1]["X"]) < 1e-12
    else:
        assert _rel(runs[0]["X"], runs[1]["X"]) < 1e-4


@pytest.mark.parametrize("terms", [2, 3])
def test_fp32_gram_with_several_tiles_per_cta(terms):
    """A A^T from the persistent tensor-core GEMM when the tile count exceeds the
    SM count (each CTA reuses both of its TMEM accumulators): the solve with the
    precomputed Gram matrix matches the one that streams A A_i^T."""
    A, B, C, _ = workloads.gaussian(3000, 40, 20, 60, seed=21)
    al = _alpha(B)
    runs = [_gpu_run(A, B, C, "rgrbk", theta=0.5, alpha=al, seed=5, maxit=300, precision="f32",
                     use_gram=ug, refresh_T=64, split_terms=terms, trace=False) for ug in (1, -1)]
    assert runs[0]["res"]["gram"] == 1 and runs[1]["res"]["gram"] == 0
    assert _rel(runs[0]["X"], runs[1]["X"]) < 1e-4


def test_fp64_refresh_keeps_parity():
    """Refreshing R = C - A X B every 64 iterations (FP64 GEMMs) keeps the row
    sequence and the iterate."""
    A, B, C, _ = workloads.gaussian(120, 30, 20, 90, seed=4)
    al = _alpha(B)
    orc = oracle.solve(A, B, C, "rgrbk", theta=0.8, alpha=al, seed=2, maxit=600, mode=oracle.MODE_FACTORED)
    gpu = _gpu_run(A, B, C, "rgrbk", theta=0.8, alpha=al, seed=2, maxit=600, refresh_T=64)
    _assert_same_rows(gpu["rows"], orc)
    assert _rel(gpu["X"], orc["X"]) < 1e-9


def test_fp64_converges_to_rse_1e6_small_config():
    """Config A 200x100 / B 80x150: ME-GRBK in FP64 reaches ||X - X*|| <= 1e-6 ||X*||."""
    A, B, C, Xs = workloads.config_small()
    ctx = g.grbk_create(A, B, C, precision="f64", stop_kind="rse", x_ref=Xs, check_every=2048)
    X = np.zeros((100, 80))
    st, res = g.grbk_solve(ctx, "grbk", tol=1e-6, maxit=3_000_000, seed=1, X_out=X)
    assert st == g.GRBK_OK, res
    assert _rel(X, Xs) <= 1e-6
    assert res["rse"] <= 1e-6


def test_fp32_converges_to_rse_1e4_small_config():
    A, B, C, Xs = workloads.config_small()
    ctx = g.grbk_create(A, B, C, precision="f32", stop_kind="rse", x_ref=Xs, refresh_T=64)
    X = np.zeros((100, 80))
    st, res = g.grbk_solve(ctx, "grbk", tol=1e-4, maxit=3_000_000, seed=1, X_out=X)
    assert st == g.GRBK_OK, res
    assert _rel(X, Xs) <= 1e-4


def test_fp32_precision_slice_rse():
    """2000x200 / 200x2000 slice of the precision configuration: FP32 bulk +
    refresh every 64 iterations reaches RSE <= 1e-4 against X* and stays within
    1e-4 of the FP64 oracle's iterate after the same iterations of ME-MWRBK."""
    A, B, C, Xs = workloads.config_precision(2000, 200, 200, 2000)
    al = _alpha(B)
    ctx = g.grbk_create(A, B, C, precision="f32", alpha=al, stop_kind="rse", x_ref=Xs, refresh_T=64)
    X = np.zeros((200, 200))
    st, res = g.grbk_solve(ctx, "grbk", tol=1e-4, maxit=2_000_000, seed=1, X_out=X)
    assert st == g.GRBK_OK, res
    assert _rel(X, Xs) <= 1e-4
    orc = oracle.solve(A, B, C, "mwrbk", alpha=al, maxit=300, mode=oracle.MODE_FACTORED, trace=False)
    gpu = _gpu_run(A, B, C, "mwrbk", alpha=al, maxit=300, precision="f32", trace=False, refresh_T=64)
    assert _rel(gpu["X"], orc["X"]) < 1e-4


def test_nonzero_x0_and_limit():
    """ME-BK from X0 != 0 on a rank-deficient pair tends to A^+CB^+ + X0 - A^+AX0BB^+
    (Theorem 3.3); the GPU needs the residual GEMM for R^0."""
    A, B, C, _ = workloads.duplicated(30, 12, 10, 25, seed=3, how="rows")
    X0 = np.random.default_rng(4).standard_normal((12, 10))
    pinv = np.linalg.pinv
    lim = pinv(A) @ C @ pinv(B) + X0 - pinv(A) @ A @ X0 @ B @ pinv(B)
    ctx = g.grbk_create(A, B, C, precision="f64", stop_kind="relres")
    X = np.zeros((12, 10))
    st, res = g.grbk_solve(ctx, "bk", X0=X0, tol=1e-13, maxit=2_000_000, X_out=X)
    assert st == g.GRBK_OK
    assert _rel(X, lim) < 1e-9


@pytest.mark.parametrize("terms,bound", [(3, 2e-6), (2, 6e-5)])
@pytest.mark.parametrize("m,p,q,n", [(700, 130, 300, 517), (129, 64, 256, 256), (9000, 64, 300, 1300)])
def test_fp32_split_bf16_refresh(terms, bound, m, p, q, n):
    """The tensor-core refresh R = C - (A X) B with split-BF16 operands: every
    entry within `bound` of |A||X||B| + |C| (3 terms ~ FP32 rounding of the
    inputs, 2 terms ~ 2^-16 per product), on shapes with several M, N and K
    tiles and ragged tails."""
    A, B, C, _ = workloads.gaussian(m, p, q, n, seed=m + q)
    X = np.random.default_rng(2).standard_normal((p, q))
    ref = oracle.residual(A, X, B, C)
    ctx = g.grbk_create(A, B, C, precision="f32", split_terms=terms)
    R32 = np.zeros(C.shape, dtype=np.float32)
    g.grbk_residual(ctx, X, R32)
    scale = np.abs(A) @ np.abs(X) @ np.abs(B) + np.abs(C)
    err = np.abs(R32 - ref) / scale
    assert np.max(err) < bound, np.max(err)


def test_residual_entry_point():
    A, B, C, _ = workloads.gaussian(257, 33, 19, 131, seed=6)
    X = np.random.default_rng(1).standard_normal((33, 19))
    ref = oracle.residual(A, X, B, C)
    ctx = g.grbk_create(A, B, C, precision="f64")
    R = np.zeros_like(C)
    g.grbk_residual(ctx, X, R)
    assert np.max(np.abs(R - ref)) < 1e-12 * np.max(np.abs(C))
    ctx32 = g.grbk_create(A, B, C, precision="f32", split_terms=3)
    R32 = np.zeros(C.shape, dtype=np.float32)
    g.grbk_residual(ctx32, X, R32)
    # 3 split terms and FP32 inputs: entries of A, B, C and X rounded to 2^-24; products of depth p and q
    scale = np.abs(A) @ np.abs(X) @ np.abs(B) + np.abs(C)
    assert np.max(np.abs(R32 - ref) / scale) < 2e-6


def test_torch_device_buffers_and_stream():
    A, B, C, Xs = workloads.gaussian(64, 10, 8, 40, seed=9)
    dev = torch.device("cuda")
    At, Bt, Ct = (torch.from_numpy(x).to(dev) for x in (A, B, C))
    s = torch.cuda.Stream()
    ctx = g.grbk_create(At, Bt, Ct, precision="f64", stream=s, stop_kind="relres")
    Xt = torch.zeros(10, 8, dtype=torch.float64, device=dev)
    st, res = g.grbk_solve(ctx, "mwrbk", tol=1e-12, maxit=200000, X_out=Xt)
    assert st == g.GRBK_OK
    assert _rel(Xt.cpu().numpy(), Xs) < 1e-9


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(37, 5, 7, 29), (200, 100, 80, 150), (2000, 200, 200, 2000), (60, 4, 1, 9),
                                   "rank_deficient"])
def test_default_step_is_inverse_squared_spectral_norm(precision, shape):
    """alpha = 1/||B||_2^2 (Section 5) from the library's Lanczos estimate of the
    largest eigenvalue of B B^T, against numpy's SVD (also for a B whose 40 rows
    span only 12 dimensions: the recurrence ends early)."""
    if shape == "rank_deficient":
        rng = np.random.default_rng(3)
        B = rng.standard_normal((40, 12)) @ rng.standard_normal((12, 70))
        A = rng.standard_normal((30, 9))
        C = A @ rng.standard_normal((9, 40)) @ B
    else:
        m, p, q, n = shape
        A, B, C, _ = workloads.gaussian(m, p, q, n, seed=q + n)
    ctx = g.grbk_create(A, B, C, precision=precision)
    _, al = g.grbk_info(ctx)
    ref = 1.0 / np.linalg.norm(B, 2) ** 2
    assert abs(al - ref) <= (1e-9 if precision == "f64" else 2e-6) * ref, (al, ref)
    g.grbk_destroy(ctx)


def test_edge_cases_and_errors():
    A, B, C, Xs = workloads.gaussian(20, 6, 5, 15, seed=11)
    ctx = g.grbk_create(A, B, C)
    X = np.zeros((6, 5))
    # maxit = 0: nothing happens
    st, res = g.grbk_solve(ctx, "grbk", maxit=0, X_out=X)
    assert st == g.GRBK_OK and res["iters"] == 0 and np.all(X == 0)
    # exact solution: R = 0 at once
    ctx0 = g.grbk_create(A, B, np.zeros_like(C))
    st, res = g.grbk_solve(ctx0, "grbk", maxit=10, X_out=X)
    assert st == g.GRBK_OK and res["iters"] == 0
    # X0 = X*: R^0 = 0 (to rounding) -> converged immediately under RELRES
    ctxr = g.grbk_create(A, B, C, stop_kind="relres")
    st, res = g.grbk_solve(ctxr, "grbk", X0=Xs, tol=1e-10, maxit=10, X_out=X)
    assert st == g.GRBK_OK and res["iters"] == 0
    # not converged within maxit
    st, res = g.grbk_solve(ctxr, "grbk", tol=1e-14, maxit=5, X_out=X)
    assert st == g.GRBK_ENOTCONV and res["iters"] == 5
    # invalid arguments
    with pytest.raises(g.GrbkError) as e:
        g.grbk_create(A, B, C[:-1])
    assert e.value.status == g.GRBK_EINVAL
    with pytest.raises(g.GrbkError) as e:
        g.grbk_solve(ctx, "rgrbk", theta=0.0, maxit=3, X_out=X)
    assert e.value.status == g.GRBK_EINVAL
    with pytest.raises(g.GrbkError) as e:
        g.grbk_create(A, B, C, alpha=2.5 * _alpha(B))
    assert e.value.status == g.GRBK_EINVAL
    Cn = C.copy()
    Cn[3, 4] = np.nan
    with pytest.raises(g.GrbkError) as e:
        g.grbk_create(A, B, Cn)
    assert e.value.status == g.GRBK_ENONFINITE
    with pytest.raises(g.GrbkError) as e:
        g.grbk_create(np.zeros_like(A), B, C)
    assert e.value.status == g.GRBK_EINVAL


def test_zero_rows_of_A_are_skipped():
    A, B, _, _ = workloads.gaussian(40, 6, 5, 30, seed=12)
    A[[0, 7, 39]] = 0.0
    C = A @ np.ones((6, 5)) @ B
    al = _alpha(B)
    for variant in ("grbk", "rgrbk", "mwrbk", "rbk", "bk"):
        orc = oracle.solve(A, B, C, variant, theta=0.4, alpha=al, seed=1, maxit=200, mode=oracle.MODE_FACTORED)
        gpu = _gpu_run(A, B, C, variant, theta=0.4, alpha=al, seed=1, maxit=200)
        _assert_same_rows(gpu["rows"], orc)
        if variant != "bk":
            assert not set(gpu["rows"].tolist()) & {0, 7, 39}


def test_block_cache_reuse_and_trim():
    """A destroyed context's device blocks serve the next create of the same sizes
    (same results), and grbk_trim_cache returns them to the driver."""
    A, B, C, _ = workloads.gaussian(3000, 60, 50, 900, seed=12)
    al = _alpha(B)
    free0 = torch.cuda.mem_get_info()[0]
    r1 = _gpu_run(A, B, C, "grbk", alpha=al, seed=2, maxit=200, precision="f32", refresh_T=64, trace=False)
    held = free0 - torch.cuda.mem_get_info()[0]
    r2 = _gpu_run(A, B, C, "grbk", alpha=al, seed=2, maxit=200, precision="f32", refresh_T=64, trace=False)
    assert np.array_equal(r1["X"], r2["X"])
    assert free0 - torch.cuda.mem_get_info()[0] <= held + (8 << 20)   # the second create reused the blocks
    g.grbk_trim_cache()
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)
