"""The oracle against its stored trajectory on the 200x100 / 80x150 system.

tests/golden/oracle_rows_small.json holds the selected row i_k and ||R^k||_F^2
for the first 200 iterations of each variant (ME-GRBK, ME-RGRBK at two theta,
ME-MWRBK, ME-RBK, ME-BK from a nonzero X^0), written by
tests/golden/make_oracle_rows.py from the oracle alone.  This is a regression
guard: a change to the oracle's arithmetic that moves a pick or a residual shows
up here and has to be justified by the passage of Sections 3-4 it follows (the
oracle's correctness itself is pinned by the closed-form and brute-force tests).
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = os.path.join(HERE, "golden", "oracle_rows_small.json")


def _load():
    with open(FIXTURE) as f:
        return json.load(f)


def _cases():
    return [(c["variant"], c["theta"]) for c in _load()["cases"]]


@pytest.mark.parametrize("variant,theta", _cases())
def test_oracle_matches_stored_trajectory(variant, theta):
    d = _load()
    case = next(c for c in d["cases"] if c["variant"] == variant and c["theta"] == theta)
    A, B, C, _ = workloads.config_small()
    X0 = workloads.rng(77).standard_normal((100, 80)) if case["x0"] != "0" else None
    r = oracle.solve(A, B, C, variant, theta=theta, alpha=float.fromhex(d["alpha"]), X0=X0,
                     seed=d["seed"], maxit=d["maxit"], mode=oracle.MODE_FACTORED)
    assert r["iters"] == d["maxit"]
    assert [int(i) for i in r["rows"]] == case["rows"]
    S_ref = np.array([float.fromhex(v) for v in case["S"]])
    np.testing.assert_allclose(r["S"], S_ref, rtol=1e-10, atol=0)


def test_fixture_alpha_is_inverse_spectral_norm():
    """The stored alpha is 1/||B||_2^2 of the system (checked against LAPACK's SVD)."""
    _, B, _, _ = workloads.config_small()
    alpha = float.fromhex(_load()["alpha"])
    assert alpha == pytest.approx(1.0 / np.linalg.norm(B, 2) ** 2, rel=1e-10)


def test_fixture_cyclic_rows():
    """ME-BK visits the rows in order 0, 1, ..., m-1, 0, ... (Section 3)."""
    case = next(c for c in _load()["cases"] if c["variant"] == "bk")
    assert case["rows"] == [k % 200 for k in range(200)]


def test_openmp_timing_build_gives_the_same_bits():
    """The OpenMP build that times the oracle on every host core splits only
    loops whose elements are independent and keeps every sum over rows serial,
    so it must reproduce the single-thread build exactly."""
    import numpy as np
    import workloads
    A, B, C, Xs = workloads.config_small()
    alpha = 1.0 / np.linalg.norm(B, 2) ** 2
    for variant in ("grbk", "mwrbk"):
        one = oracle.solve(A, B, C, variant, alpha=alpha, seed=3, maxit=150, mode=oracle.MODE_FACTORED, want_R=True)
        allc = oracle.solve(A, B, C, variant, alpha=alpha, seed=3, maxit=150, mode=oracle.MODE_FACTORED,
                            want_R=True, omp=True)
        assert np.array_equal(one["rows"], allc["rows"])
        assert np.array_equal(one["X"], allc["X"]) and np.array_equal(one["R"], allc["R"])
        assert np.array_equal(one["S"], allc["S"])
    assert oracle.threads(False) == 1
