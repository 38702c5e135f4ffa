"""Batched solver (many uneven systems in one persistent launch, FP32 bulk with
FP64 row-norm sums, threshold and pick) against the FP64 oracle run per system
with the same Philox counter layout (k, system)."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _systems():
    return workloads.blur_systems(n_images=3, min_side=48, max_side=112, noise=0.0, mild=True, seed=21)


def _alphas(Bs):
    """alpha_s = 1 / ||B_s||_2^2 from numpy's SVD (Section 5's step), given to
    both the library and the oracle so neither side takes the other's step."""
    return np.array([1.0 / np.linalg.norm(B, 2) ** 2 for B in Bs])


def _band(M):
    i, c = np.nonzero(M)
    return int(np.max(np.abs(c - i))) if len(i) else 0


@pytest.mark.parametrize("band_limit", [0, -1])
def test_batch_converges_to_clean_images(band_limit):
    sy = _systems()
    As, Bs, Cs = [s["A"] for s in sy], [s["B"] for s in sy], [s["C"] for s in sy]
    b = g.grbk_batch_create(As, Bs, Cs, stop_kind="relres", band_limit=band_limit)
    Xo = [np.zeros_like(s["X"]) for s in sy]
    st, res = g.grbk_batch_solve(b, "grbk", tol=1e-6, maxit=2_000_000, seed=3, X_outs=Xo)
    assert st == g.GRBK_OK
    for s, X, r in zip(sy, Xo, res):
        assert r["relres"] <= 1e-6
        assert _rel(X, s["X"]) <= 1e-4


@pytest.mark.parametrize("band_limit", [0, -1])
@pytest.mark.parametrize("variant", ["mwrbk", "grbk", "rgrbk", "rbk", "bk"])
def test_batch_matches_oracle_per_system(variant, band_limit):
    """Fixed 120 iterations per system: the selected rows agree with the FP64
    oracle's up to the first decision the oracle marks as closer than FP32
    resolves (relative margin 1e-5), and every system agrees at least up to
    its first decision within 1e-6; where all 120 agree X agrees to 1e-4."""
    sy = _systems()
    As, Bs, Cs = [s["A"] for s in sy], [s["B"] for s in sy], [s["C"] for s in sy]
    alphas = _alphas(Bs)
    b = g.grbk_batch_create(As, Bs, Cs, trace_len=120, band_limit=band_limit, alphas=alphas)
    for sid, s in enumerate(sy):
        want = (_band(s["A"]), _band(s["B"])) if band_limit == 0 else (-1, -1)
        assert g.grbk_batch_info(b, sid) == want
    Xo = [np.zeros_like(s["X"]) for s in sy]
    st, res = g.grbk_batch_solve(b, variant, theta=0.7, maxit=120, seed=11, X_outs=Xo)
    assert st == g.GRBK_OK
    compared = []
    for sid, (s, X, r) in enumerate(zip(sy, Xo, res)):
        assert r["iters"] == 120
        assert r["alpha"] == alphas[sid]
        orc = oracle.solve(s["A"], s["B"], s["C"], variant, theta=0.7, alpha=alphas[sid], seed=11, sys=sid,
                           maxit=120, mode=oracle.MODE_FACTORED)
        kk = compare_rows(b.row_trace[sid], orc, 120)
        if kk == 120:
            assert _rel(X, orc["X"]) < 1e-4
        compared.append(kk)
    assert sum(compared) >= 0.9 * 120 * len(sy), compared


def test_banded_and_dense_paths_agree():
    """The banded path skips only exact zeros (rows of R with u_i = 0 are left as
    they are, which the dense path reproduces bit for bit), so both paths select
    the same rows while the decisions are wider than FP32 rounding and reach the
    same X to FP32 accuracy; a matrix with a wide band stays dense."""
    sy = workloads.blur_systems(n_images=2, min_side=64, max_side=160, noise=0.0, mild=True, seed=5)
    As, Bs, Cs = [s["A"] for s in sy], [s["B"] for s in sy], [s["C"] for s in sy]
    out = {}
    for bl in (0, -1):
        b = g.grbk_batch_create(As, Bs, Cs, trace_len=400, band_limit=bl)
        Xo = [np.zeros_like(s["X"]) for s in sy]
        st, res = g.grbk_batch_solve(b, "rgrbk", theta=0.8, maxit=400, seed=2, X_outs=Xo)
        assert st == g.GRBK_OK
        out[bl] = (b.row_trace.copy(), Xo)
    for sid in range(len(sy)):
        r0, r1 = out[0][0][sid], out[-1][0][sid]
        diff = np.nonzero(r0 != r1)[0]
        first = int(diff[0]) if len(diff) else 400
        assert first >= 50, first
        if first == 400:
            assert _rel(out[0][1][sid], out[-1][1][sid]) < 1e-4
    # a full A (band m - 1) keeps the dense path under the default limit
    A = np.random.default_rng(1).standard_normal((40, 40))
    b = g.grbk_batch_create([A, As[0]], [A, Bs[0]], [A @ A, Cs[0]])
    assert g.grbk_batch_info(b, 0) == (-1, -1)
    assert g.grbk_batch_info(b, 1)[0] >= 0


def test_banded_path_on_rectangular_banded_systems():
    """Rectangular A (m x p) and B (q x n) with nonzeros only within a band of the
    diagonal take the banded path and match the oracle like the dense path."""
    rng = np.random.default_rng(8)

    def banded(r, c, b):
        M = rng.standard_normal((r, c))
        i, j = np.indices((r, c))
        M[np.abs(j - i) > b] = 0.0
        return M

    sy = []
    for (m, p, q, n, ba, bb) in [(90, 70, 60, 80, 3, 5), (64, 64, 48, 100, 1, 2)]:
        A, B = banded(m, p, ba), banded(q, n, bb)
        Xs = rng.standard_normal((p, q))
        sy.append(dict(A=A, B=B, C=A @ Xs @ B, X=Xs, ba=ba, bb=bb))
    As, Bs, Cs = [s["A"] for s in sy], [s["B"] for s in sy], [s["C"] for s in sy]
    alphas = _alphas(Bs)
    b = g.grbk_batch_create(As, Bs, Cs, trace_len=150, alphas=alphas)
    for sid, s in enumerate(sy):
        assert g.grbk_batch_info(b, sid) == (_band(s["A"]), _band(s["B"]))
    Xo = [np.zeros_like(s["X"]) for s in sy]
    st, res = g.grbk_batch_solve(b, "grbk", maxit=150, seed=4, X_outs=Xo)
    assert st == g.GRBK_OK
    for sid, (s, X, r) in enumerate(zip(sy, Xo, res)):
        orc = oracle.solve(s["A"], s["B"], s["C"], "grbk", alpha=alphas[sid], seed=4, sys=sid, maxit=150,
                           mode=oracle.MODE_FACTORED)
        kk = compare_rows(b.row_trace[sid], orc, 150)
        if kk == 150:
            assert _rel(X, orc["X"]) < 1e-4


@pytest.mark.parametrize("band_limit", [0, -1])
def test_batch_from_nonzero_x0_matches_oracle(band_limit):
    """R^0 = C - A X0 B formed on the device (from the bands of A and B on the
    banded path) and the iteration from there agree with the oracle."""
    sy = _systems()[:2]
    As, Bs, Cs = [s["A"] for s in sy], [s["B"] for s in sy], [s["C"] for s in sy]
    rng = np.random.default_rng(6)
    X0s = [s["X"] + 0.05 * rng.standard_normal(s["X"].shape) for s in sy]
    alphas = _alphas(Bs)
    b = g.grbk_batch_create(As, Bs, Cs, trace_len=100, band_limit=band_limit, alphas=alphas)
    Xo = [np.zeros_like(s["X"]) for s in sy]
    st, res = g.grbk_batch_solve(b, "grbk", X0s=X0s, maxit=100, seed=5, X_outs=Xo)
    assert st == g.GRBK_OK
    for sid, (s, X, r) in enumerate(zip(sy, Xo, res)):
        assert r["x0_rejected"] == 0
        orc = oracle.solve(s["A"], s["B"], s["C"], "grbk", alpha=alphas[sid], X0=X0s[sid], seed=5, sys=sid,
                           maxit=100, mode=oracle.MODE_FACTORED)
        kk = compare_rows(b.row_trace[sid], orc, 100)
        if kk == 100:
            assert _rel(X, orc["X"]) < 1e-4


@pytest.mark.parametrize("band_limit", [0, -1])
def test_autotuned_batch_matches_oracle(band_limit):
    """With the autotuner on, each system runs the variant timed fastest on its
    class (possibly different variants side by side on separate streams); the
    rows still follow the FP64 oracle's and every system's variant is recorded
    and cached."""
    g.grbk_tune_clear()
    sy = _systems()
    As, Bs, Cs = [s["A"] for s in sy], [s["B"] for s in sy], [s["C"] for s in sy]
    alphas = _alphas(Bs)
    b = g.grbk_batch_create(As, Bs, Cs, trace_len=120, band_limit=band_limit, alphas=alphas, tune=True)
    nv = len(g.grbk_tune_variants())
    chosen = []
    for sid, s in enumerate(sy):
        v, secs = g.grbk_batch_variant(b, sid)
        assert 0 <= v < nv and secs > 0
        bA, bB = g.grbk_batch_info(b, sid)
        m, p = s["A"].shape
        q, n = s["B"].shape
        assert g.grbk_tune_lookup(m, p, q, n, bA, bB) == v
        chosen.append(v)
    Xo = [np.zeros_like(s["X"]) for s in sy]
    st, res = g.grbk_batch_solve(b, "grbk", maxit=120, seed=11, X_outs=Xo)
    assert st == g.GRBK_OK
    compared = []
    for sid, (s, X, r) in enumerate(zip(sy, Xo, res)):
        assert r["iters"] == 120
        orc = oracle.solve(s["A"], s["B"], s["C"], "grbk", alpha=alphas[sid], seed=11, sys=sid, maxit=120,
                           mode=oracle.MODE_FACTORED)
        kk = compare_rows(b.row_trace[sid], orc, 120)
        if kk == 120:
            assert _rel(X, orc["X"]) < 1e-4
        compared.append(kk)
    assert sum(compared) >= 0.9 * 120 * len(sy), compared
    # a second batch of the same shapes takes every choice from the cache
    b2 = g.grbk_batch_create(As, Bs, Cs, band_limit=band_limit, tune=True)
    assert [g.grbk_batch_variant(b2, sid)[0] for sid in range(len(sy))] == chosen
    g.grbk_tune_clear()


def _banded(n, b, rng, diag=2.0):
    """n x n with half-bandwidth b: a symmetric Toeplitz Gaussian band plus a
    small random banded perturbation, diagonally weighted (well conditioned)."""
    i, j = np.indices((n, n))
    d = np.abs(i - j)
    M = np.where(d <= b, np.exp(-(d / (0.5 * b + 1.0)) ** 2), 0.0)
    M += np.where(d <= b, 0.05 * rng.standard_normal((n, n)), 0.0)
    M[d == 0] += diag
    return M


@pytest.mark.parametrize("variant", ["grbk", "mwrbk"])
def test_wide_band_reads_bands_from_global_memory(variant):
    """Two banded systems in one launch: half-bandwidths 40 at side 600, whose
    band copies ((2 * 40 + 1) * 600 * 2 floats = 389 KB) exceed the 150 KB the
    kernel keeps in shared memory, so its w, u, v and X update read the bands
    from global memory; and half-bandwidth 5 at side 200, read from shared
    memory.  Both against the FP64 oracle as in the per-system test."""
    rng = np.random.default_rng(31)
    sy = []
    for n, bw in ((600, 40), (200, 5)):
        A = _banded(n, bw, rng)
        B = _banded(n, bw, rng)
        Xs = rng.standard_normal((n, n))
        sy.append(dict(A=A, B=B, C=A @ Xs @ B, X=Xs, bw=bw))
    As, Bs, Cs = [s["A"] for s in sy], [s["B"] for s in sy], [s["C"] for s in sy]
    alphas = _alphas(Bs)
    K = 120
    b = g.grbk_batch_create(As, Bs, Cs, trace_len=K, alphas=alphas)
    for sid, s in enumerate(sy):
        assert g.grbk_batch_info(b, sid) == (_band(s["A"]), _band(s["B"])) == (s["bw"], s["bw"])
    Xo = [np.zeros_like(s["X"]) for s in sy]
    st, res = g.grbk_batch_solve(b, variant, maxit=K, seed=5, X_outs=Xo)
    assert st == g.GRBK_OK
    for sid, (s, X, r) in enumerate(zip(sy, Xo, res)):
        assert r["iters"] == K
        orc = oracle.solve(s["A"], s["B"], s["C"], variant, alpha=alphas[sid], seed=5, sys=sid, maxit=K,
                           mode=oracle.MODE_FACTORED)
        kk = compare_rows(b.row_trace[sid], orc, K)
        assert kk >= 0.9 * K, (sid, kk)
        if kk == K:
            assert _rel(X, orc["X"]) < 1e-4
    g.grbk_batch_destroy(b)
