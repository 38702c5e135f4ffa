"""grbk_solve_small_noalloc: the entry point for callers that cannot allocate
(a process whose device memory is handed out by a fixed pool it does not own,
loops that cannot afford cudaMalloc/cudaFree and the synchronisation cudaFree
implies).  It must give what the allocating
batched entry point gives for the same single system, on two calls in a row
(the second call reuses the static working array the first one left behind).

This file is named to be collected last."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2408_05444_gb300 as g  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _system(seed):
    s = workloads.blur_systems(n_images=1, min_side=64, max_side=144, noise=0.0, mild=True, seed=seed)[0]
    return s["A"], s["B"], s["C"]


@pytest.mark.parametrize("variant,tol", [("grbk", 0.0), ("mwrbk", 0.0), ("rgrbk", 1e-5)])
def test_noalloc_matches_batch_entry_point_twice(variant, tol):
    A, B, C = _system(31)
    alpha = 1.0 / np.linalg.norm(B, 2) ** 2
    maxit = 400 if tol == 0.0 else 200000
    # the existing (allocating) entry point on the same single system, on the same (dense) path
    bt = g.grbk_batch_create([A], [B], [C], alpha=alpha, stop_kind="relres" if tol > 0 else "none", band_limit=-1)
    Xref = np.zeros((A.shape[1], B.shape[0]))
    st, res = g.grbk_batch_solve(bt, variant, theta=0.6, tol=tol, maxit=maxit, seed=9, X_outs=[Xref])
    assert st == g.GRBK_OK
    dev = torch.device("cuda")
    At, Bt, Ct = (torch.from_numpy(x.astype(np.float32)).to(dev) for x in (A, B, C))
    for call in range(2):
        X = torch.full((A.shape[1], B.shape[0]), float("nan"), dtype=torch.float32, device=dev)
        st2, it2, rr2 = g.grbk_solve_small_noalloc(At, Bt, Ct, X, variant, theta=0.6, alpha=alpha, tol=tol,
                                                   maxit=maxit, seed=9)
        assert st2 == g.GRBK_OK, (call, g.grbk_strerror(st2))
        assert it2 == res[0]["iters"]
        assert abs(rr2 - res[0]["relres"]) <= 1e-4 * max(res[0]["relres"], 1e-12)
        assert _rel(X.cpu().numpy().astype(np.float64), Xref) < 1e-4, call


def test_noalloc_default_step_and_limits():
    A, B, C = _system(32)
    dev = torch.device("cuda")
    At, Bt, Ct = (torch.from_numpy(x.astype(np.float32)).to(dev) for x in (A, B, C))
    X = torch.zeros(A.shape[1], B.shape[0], dtype=torch.float32, device=dev)
    st, it, rr = g.grbk_solve_small_noalloc(At, Bt, Ct, X, "grbk", alpha=0.0, tol=1e-4, maxit=100000, seed=1)
    assert st == g.GRBK_OK and rr <= 1e-4
    big = torch.zeros(g.GRBK_NOALLOC_MAX_SIDE + 1, 4, dtype=torch.float32, device=dev)
    Bs = torch.zeros(4, 4, dtype=torch.float32, device=dev)
    Cs = torch.zeros(g.GRBK_NOALLOC_MAX_SIDE + 1, 4, dtype=torch.float32, device=dev)
    Xs = torch.zeros(4, 4, dtype=torch.float32, device=dev)
    st, _, _ = g.grbk_solve_small_noalloc(big, Bs, Cs, Xs, "grbk", maxit=5)
    assert st == g.GRBK_EINVAL
    # non-finite step, tolerance or relaxation: rejected on the host before any work
    nan = float("nan")
    for kw in (dict(alpha=nan), dict(alpha=float("inf")), dict(tol=nan), dict(variant="rgrbk", theta=nan)):
        args = dict(variant="grbk", maxit=5)
        args.update(kw)
        st, _, _ = g.grbk_solve_small_noalloc(At, Bt, Ct, X, **args)
        assert st == g.GRBK_EINVAL, kw
