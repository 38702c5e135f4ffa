"""The seeded input generators shared by the oracle tests and the GPU tests
produce the workloads they are documented to produce (shapes, value
distributions, spectra, blur structure), and are deterministic."""
import numpy as np

import workloads


def test_small_and_gaussian_systems_are_consistent():
    A, B, C, Xs = workloads.config_small()
    assert A.shape == (200, 100) and B.shape == (80, 150) and Xs.shape == (100, 80) and C.shape == (200, 150)
    np.testing.assert_allclose(C, A @ Xs @ B, rtol=0, atol=1e-10 * np.abs(C).max())
    A2, B2, C2, X2 = workloads.config_small()
    assert all(np.array_equal(u, v) for u, v in ((A, A2), (B, B2), (C, C2), (Xs, X2)))
    A, B, C, Xs = workloads.gaussian(30, 7, 5, 20, seed=3, noise=0.5)
    assert np.linalg.norm(C - A @ Xs @ B) > 0.1 * np.sqrt(C.size) * 0.5


def test_precision_recipe_variances():
    """Entries of A and B are N(0, 1/cols): sample variances within 5 %."""
    A, B, C, Xs = workloads.config_precision(2000, 200, 200, 2000)
    assert abs(A.var() * 200 - 1) < 0.05 and abs(B.var() * 2000 - 1) < 0.05 and abs(Xs.var() - 1) < 0.05
    np.testing.assert_allclose(C, (A @ Xs) @ B, rtol=0, atol=1e-12 * np.abs(C).max())
    A32 = workloads.config_precision(200, 20, 20, 200, dtype=np.float32)[0]
    assert A32.dtype == np.float32


def test_haar_columns_are_orthonormal():
    Q = workloads.haar(workloads.rng(5), 60, 20)
    np.testing.assert_allclose(Q.T @ Q, np.eye(20), atol=1e-12)


def test_scale_recipe_spectra():
    """A = U diag(sigma) V^T with sigma log-spaced from 1 to 1e-2; the
    rank-deficient variant has rank 600 (A) and 500 (B)."""
    A, B, C, Xs = workloads.config_scale()
    assert A.shape == (4000, 1000) and B.shape == (800, 3000)
    sa = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(sa, np.logspace(0, -2, 1000), rtol=1e-8)
    sb = np.linalg.svd(B, compute_uv=False)
    np.testing.assert_allclose(sb, np.logspace(0, -2, 800), rtol=1e-8)
    Ad, Bd, _, _ = workloads.config_scale(rank_deficient=True)
    assert np.linalg.matrix_rank(Ad) == 600 and np.linalg.matrix_rank(Bd) == 500


def test_duplicated_pairs_are_rank_deficient():
    A, B, C, _ = workloads.duplicated(10, 4, 3, 8)
    assert A.shape[0] == 20 and np.array_equal(A[:10], A[10:])
    assert np.linalg.matrix_rank(A) == 4


def test_gaussian_toeplitz_blur():
    """Symmetric banded Toeplitz: taps exp(-k^2 / (2 sigma^2)) for |k| <= band // 2,
    normalised to sum 1 (interior rows), zero boundary (edge rows sum to less)."""
    T = workloads.gaussian_toeplitz(40, 9, 2.0)
    assert np.array_equal(T, T.T)
    i, j = np.nonzero(T)
    assert np.max(np.abs(i - j)) == 4
    np.testing.assert_allclose(T[20].sum(), 1.0, rtol=1e-14)
    assert T[0].sum() < 1.0
    k = np.arange(-4, 5)
    taps = np.exp(-k ** 2 / 8.0)
    np.testing.assert_allclose(T[20, 16:25], taps / taps.sum(), rtol=1e-14)


def test_blur_image_systems():
    """Per image: sides multiples of 16 in [min, max], one blur per side with
    band in {7, ..., 15}, three channel systems C = A X B + E with X in [0, 1]
    and E ~ N(0, noise^2); drawing in a spawn pool gives the same systems."""
    sy = workloads.blur_systems(n_images=4, min_side=32, max_side=64, seed=2, noise=1e-3)
    assert len(sy) == 12
    for q in sy:
        h, w = q["X"].shape
        assert h % 16 == 0 and w % 16 == 0 and 32 <= h <= 64 and 32 <= w <= 64
        for M in (q["A"], q["B"]):
            i, j = np.nonzero(M)
            assert np.max(np.abs(i - j)) in (3, 4, 5, 6, 7) and np.array_equal(M, M.T)
        assert 0.0 <= q["X"].min() and q["X"].max() <= 1.0
        np.testing.assert_allclose(q["C"], q["A"] @ q["X"] @ q["B"] + q["E"], atol=1e-12)
        assert abs(q["E"].std() / 1e-3 - 1) < 0.1
    again = workloads.blur_systems(n_images=4, min_side=32, max_side=64, seed=2, noise=1e-3, processes=2)
    assert all(np.array_equal(u["C"], v["C"]) for u, v in zip(sy, again))
    mild = workloads.blur_image_systems(0, seed=2, min_side=32, max_side=64, mild=True)
    assert np.linalg.cond(mild[0]["A"]) < 10
