"""Failure detection without a GPU fault: a device-side wait that can never be
satisfied (a CTA that never arrives at the grid barrier) must end by its own
spin budget with GRBK_ETIMEOUT, and the context must stay usable."""
import time

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2408_05444_gb300 as g  # noqa: E402


def test_barrier_completes_when_everyone_arrives():
    assert g.grbk_barrier_selftest(-1) == g.GRBK_OK


def test_barrier_times_out_and_context_survives():
    t0 = time.time()
    assert g.grbk_barrier_selftest(0) == g.GRBK_ETIMEOUT
    assert time.time() - t0 < 10.0
    # the same process keeps working: a solve after the timeout converges
    A, B, C, Xs = workloads.gaussian(40, 8, 6, 30, seed=5)
    ctx = g.grbk_create(A, B, C, stop_kind="relres")
    X = np.zeros((8, 6))
    st, res = g.grbk_solve(ctx, "mwrbk", tol=1e-12, maxit=100000, X_out=X)
    assert st == g.GRBK_OK
    assert np.linalg.norm(X - Xs) / np.linalg.norm(Xs) < 1e-9
    assert g.grbk_barrier_selftest(-1) == g.GRBK_OK


def test_invalid_inputs_are_reported_not_crashed():
    A, B, C, _ = workloads.gaussian(10, 4, 3, 8, seed=6)
    with pytest.raises(g.GrbkError) as e:
        g.grbk_create(A, B, C, refresh_T=-1)
    assert e.value.status == g.GRBK_EINVAL
    nan = float("nan")
    for kw in (dict(alpha=nan), dict(alpha=float("inf")), dict(rank_tol=nan)):
        with pytest.raises(g.GrbkError) as e:
            g.grbk_create(A, B, C, **kw)
        assert e.value.status == g.GRBK_EINVAL, kw
    for kw in (dict(alpha=nan), dict(alphas=[nan]), dict(alphas=[-1.0]), dict(alphas=[1e6])):
        with pytest.raises(g.GrbkError) as e:
            g.grbk_batch_create([A], [B], [C], **kw)
        assert e.value.status == g.GRBK_EINVAL, kw
    ctx = g.grbk_create(A, B, C)
    X = np.zeros((4, 3))
    with pytest.raises(g.GrbkError) as e:
        g.grbk_solve(ctx, "grbk", tol=nan, maxit=5, X_out=X)
    assert e.value.status == g.GRBK_EINVAL
    with pytest.raises(g.GrbkError) as e:
        g.grbk_solve(ctx, "rgrbk", theta=nan, maxit=5, X_out=X)
    assert e.value.status == g.GRBK_EINVAL
    g.grbk_destroy(ctx)
    b = g.grbk_batch_create([A], [B], [C])
    for kw in (dict(tol=nan), dict(targets=[nan])):
        with pytest.raises(g.GrbkError) as e:
            g.grbk_batch_solve(b, "grbk", maxit=5, X_outs=[X], **kw)
        assert e.value.status == g.GRBK_EINVAL, kw
    g.grbk_batch_destroy(b)
    Cinf = C.copy()
    Cinf[0, 0] = np.inf
    with pytest.raises(g.GrbkError) as e:
        g.grbk_batch_create([A], [B], [Cinf])
    assert e.value.status == g.GRBK_ENONFINITE
