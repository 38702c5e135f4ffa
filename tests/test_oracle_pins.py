"""Pins for the FP64 CPU oracle: each test ties an oracle function to something
other than itself -- a closed form from the paper, an invariant or identity the
paper proves, a library routine, a hand-built case or brute-force statistics.

Paper references: Eq. (2.2) least-norm solution and the full-rank formulas of
Section 2; Lemma 3.2 / Eq. (3.1) invariant; Theorem 3.3 ME-BK limit;
Eqs. (3.4)-(3.6) per-step error identity; Remark 4.1 non-empty admitted set;
Remark 4.4 theta = 1/2; Theorem 4.8 / Eq. (4.18) MWRBK contraction;
Lemma 2.2 / Eq. (2.3), Theorem 4.2 / Eq. (4.3) and Theorem 4.5 / Eqs. (4.13),
(4.15) expected-rate bounds;
Algorithms 1-5 for the selection rules.
"""
import numpy as np
import pytest

import oracle
import workloads

pinv = np.linalg.pinv


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _alpha(B):
    return 1.0 / np.linalg.norm(B, 2) ** 2


# ---------------------------------------------------------------- Philox / RNG

@pytest.mark.parametrize("key,ctr", [((7, 0), (0, 0, 0, 0)), ((123456789, 0), (5, 3, 0, 0)),
                                     ((2**63 + 11, 99), (2**64 - 1, 17, 2**40, 3)),
                                     ((0, 0), (1, 0, 0, 0))])
def test_philox_matches_numpy(key, ctr):
    # numpy's Philox increments its 256-bit counter before each block, so the
    # block for counter c is what numpy emits when started from c - 1.
    c = sum(int(v) << (64 * i) for i, v in enumerate(ctr))
    prev = (c - 1) % (1 << 256)
    words = np.array([(prev >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=words)
    expect = bg.random_raw(4)
    got = oracle.philox4x64_10(ctr, key)
    assert np.array_equal(got, expect)


@pytest.mark.parametrize("seed,k,sys", [(0, 0, 0), (42, 999, 0), (7, 123456, 191)])
def test_uniform_matches_numpy_random(seed, k, sys):
    c = (k | (sys << 64)) - 1
    c %= 1 << 256
    words = np.array([(c >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    gen = np.random.Generator(np.random.Philox(key=np.array([seed, 0], dtype=np.uint64),
                                               counter=words))
    assert oracle.uniform(seed, k, sys) == gen.random()


# ---------------------------------------------------------------- dense helpers

def test_residual_rownorms_specnorm_vs_numpy():
    g = np.random.default_rng(5)
    A, B = g.standard_normal((7, 4)), g.standard_normal((3, 9))
    X, C = g.standard_normal((4, 3)), g.standard_normal((7, 9))
    assert _rel(oracle.residual(A, X, B, C), C - A @ X @ B) < 1e-14
    assert _rel(oracle.row_sqnorms(A), np.einsum("ij,ij->i", A, A)) < 1e-15
    assert abs(oracle.spectral_norm_sq(B, 400) / np.linalg.norm(B, 2) ** 2 - 1) < 1e-12


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("variant,theta", [("grbk", 0.5), ("rgrbk", 0.3), ("rgrbk", 0.8),
                                           ("mwrbk", 1.0), ("rbk", 0.5)])
def test_converges_to_unique_solution(variant, theta):
    """Full column rank A, full row rank B: the limit is
    (A^T A)^{-1} A^T C B^T (B B^T)^{-1} = A^+ C B^+ (Section 2 / Eq. 2.2)."""
    A, B, C, Xs = workloads.gaussian(14, 5, 4, 11, seed=1)
    Xu = np.linalg.solve(A.T @ A, A.T @ C @ B.T) @ np.linalg.inv(B @ B.T)
    assert _rel(Xu, pinv(A) @ C @ pinv(B)) < 1e-10
    r = oracle.solve(A, B, C, variant, theta=theta, alpha=_alpha(B), seed=3, maxit=6000,
                     mode=oracle.MODE_FACTORED, trace=False)
    assert _rel(r["X"], Xu) < 1e-10


@pytest.mark.parametrize("variant", ["grbk", "mwrbk"])
def test_converges_to_least_norm_full_row_rank(variant):
    """A full row rank, B full column rank: from X^0 = 0 the greedy methods
    reach A^T (A A^T)^{-1} C (B^T B)^{-1} B^T (Section 2), the least-norm one."""
    A, B, C, _ = workloads.gaussian(4, 9, 10, 5, seed=2)
    Xln = A.T @ np.linalg.inv(A @ A.T) @ C @ np.linalg.inv(B.T @ B) @ B.T
    assert _rel(Xln, pinv(A) @ C @ pinv(B)) < 1e-10
    r = oracle.solve(A, B, C, variant, alpha=_alpha(B), seed=4, maxit=6000,
                     mode=oracle.MODE_FACTORED, trace=False)
    assert _rel(r["X"], Xln) < 1e-9


@pytest.mark.parametrize("variant", ["bk", "grbk", "rbk", "mwrbk"])
def test_limit_with_nonzero_x0_rank_deficient(variant):
    """Theorem 3.3: from any X^0 the ME-BK iterates tend to
    A^+ C B^+ + X^0 - A^+ A X^0 B B^+.  Lemma 3.2's proof never uses the row
    rule, so the other variants share that limit."""
    A, B, C, _ = workloads.duplicated(5, 7, 6, 4, seed=1, how="rows")  # A 10x7 rank 5, B 6x8 rank 4
    g = np.random.default_rng(9)
    X0 = g.standard_normal((7, 6))
    X0lim = pinv(A) @ C @ pinv(B) + X0 - pinv(A) @ A @ X0 @ B @ pinv(B)
    r = oracle.solve(A, B, C, variant, alpha=_alpha(B), X0=X0, seed=5, maxit=20000,
                     mode=oracle.MODE_FACTORED, trace=False)
    assert _rel(r["X"], X0lim) < 1e-9


@pytest.mark.parametrize("variant", ["grbk", "rgrbk", "mwrbk", "rbk", "bk"])
def test_lemma_invariant(variant):
    """Lemma 3.2 / Eq. (3.1): X^k - A^+ A X^k B B^+ is the same for every k."""
    A, B, C, _ = workloads.duplicated(4, 6, 5, 3, seed=2, how="cols")  # A 4x12, B 10x3
    g = np.random.default_rng(1)
    X0 = g.standard_normal((12, 10))
    P = lambda X: X - pinv(A) @ A @ X @ B @ pinv(B)
    for k in (1, 7, 40):
        r = oracle.solve(A, B, C, variant, theta=0.7, alpha=_alpha(B), X0=X0, seed=2, maxit=k,
                         mode=oracle.MODE_GRAM, trace=False)
        assert _rel(P(r["X"]), P(X0)) < 1e-11


def test_recursive_residual_equals_definition():
    """R^k kept by the rank-1 recursion (Gram form of Algorithm 3 and its
    re-associated form) equals C - A X^k B computed from the iterate."""
    A, B, C, _ = workloads.gaussian(30, 8, 6, 20, seed=3)
    for mode in (oracle.MODE_GRAM, oracle.MODE_FACTORED):
        for variant in ("grbk", "mwrbk", "bk"):
            r = oracle.solve(A, B, C, variant, alpha=_alpha(B), seed=1, maxit=300, mode=mode,
                             want_R=True)
            Rdef = C - A @ r["X"] @ B
            assert _rel(r["R"], Rdef) < 1e-11 * np.linalg.norm(C) / np.linalg.norm(Rdef)
            assert _rel(r["s"], np.einsum("ij,ij->i", Rdef, Rdef)) < 1e-9
    # the three residual modes pick the same rows
    rows = [oracle.solve(A, B, C, "grbk", alpha=_alpha(B), seed=8, maxit=200, mode=md)["rows"]
            for md in (oracle.MODE_GRAM, oracle.MODE_FACTORED, oracle.MODE_LITERAL)]
    assert np.array_equal(rows[0], rows[1]) and np.array_equal(rows[0], rows[2])


def test_per_step_error_identity():
    """Eqs. (3.4)-(3.6) with X_* any solution of a consistent system:
    ||E^{k+1}||^2 - ||E^k||^2 = (alpha^2 ||R_i B^T||^2 - 2 alpha ||R_i||^2) / a_i."""
    A, B, C, Xs = workloads.gaussian(12, 6, 5, 9, seed=4)
    alpha = 1.3 * _alpha(B)
    X = np.zeros((6, 5))
    for k in range(60):
        R = C - A @ X @ B
        r = oracle.solve(A, B, C, "grbk", alpha=alpha, X0=X, seed=100 + k, maxit=1, trace=True)
        i = int(r["rows"][0])
        a_i = A[i] @ A[i]
        pred = (alpha ** 2 * np.sum((R[i] @ B.T) ** 2) - 2 * alpha * R[i] @ R[i]) / a_i
        diff = np.sum((r["X"] - Xs) ** 2) - np.sum((X - Xs) ** 2)
        assert abs(diff - pred) <= 1e-10 * np.sum((X - Xs) ** 2)
        X = r["X"]


def test_mwrbk_contraction():
    """Theorem 4.8 / Eq. (4.18): every ME-MWRBK step contracts the error by at
    least 1 - (2 alpha - alpha^2 ||B||_2^2) sigma_min^2(A) sigma_min^2(B) / gamma_k."""
    A, B, C, _ = workloads.gaussian(25, 6, 5, 18, seed=5)
    Xs = pinv(A) @ C @ pinv(B)
    alpha = _alpha(B)
    sa = np.linalg.svd(A, compute_uv=False)[-1]
    sb = np.linalg.svd(B, compute_uv=False)[-1]
    nb2 = np.linalg.norm(B, 2) ** 2
    r = oracle.solve(A, B, C, "mwrbk", alpha=alpha, maxit=400, Xref=Xs, mode=oracle.MODE_GRAM)
    e = r["err2"]
    gamma = np.sum(A * A)  # no zero-residual rows occur on this input
    rho = 1 - (2 * alpha - alpha ** 2 * nb2) * sa ** 2 * sb ** 2 / gamma
    assert np.all(e[1:] <= rho * e[:-1] * (1 + 1e-12))
    assert e[-1] < 0.5 * e[0]


# ---------------------------------------------------------------- selection rules

def _diag_problem(r_target, a_diag):
    """A = diag(d), B = I, C chosen so that row i of R^0 = C has ||R_i||^2 =
    r_i a_i: the weighted residuals r_i = s_i / a_i are r_target exactly."""
    m = len(r_target)
    d = np.sqrt(np.asarray(a_diag, dtype=float))
    A = np.diag(d)
    B = np.eye(3)
    C = np.zeros((m, 3))
    s = np.asarray(r_target, dtype=float) * d ** 2
    C[:, 0] = np.sqrt(s)
    return A, B, C, s


def _pick_counts(A, B, C, variant, theta, nseeds):
    counts = np.zeros(A.shape[0], dtype=np.int64)
    for sd in range(nseeds):
        r = oracle.solve(A, B, C, variant, theta=theta, alpha=1.0, seed=sd, maxit=1)
        counts[r["rows"][0]] += 1
    return counts


def _chi2_ok(counts, probs):
    from scipy.stats import chisquare
    nz = probs > 0
    assert counts[~nz].sum() == 0, "picked a row outside the admitted set"
    if nz.sum() == 1:
        return True
    stat = chisquare(counts[nz], probs[nz] * counts.sum())
    return stat.pvalue > 1e-4


def test_admitted_set_hand_built():
    """r = (4, 5, 6, 9) with a = (1, 4, 0.25, 2): S = sum r_i a_i, F = sum a_i.
    The threshold theta r_max + (1 - theta) S / F (Algorithms 3, 4) admits
    only the last row for theta = 1/2 and rows {2, 3} for theta = 0.01; the
    pick is proportional to ||R_i||^2 (not to r_i) over the admitted rows."""
    r_t = np.array([4.0, 5.0, 6.0, 9.0])
    a = np.array([1.0, 4.0, 0.25, 2.0])
    A, B, C, s = _diag_problem(r_t, a)
    S, F = s.sum(), a.sum()
    # S/F = (4 + 20 + 1.5 + 18) / 7.25 = 6.0
    assert abs(S / F - 6.0) < 1e-15
    r = oracle.solve(A, B, C, "grbk", alpha=1.0, seed=0, maxit=1)
    assert r["t"][0] == 0.5 * 9 + 0.5 * 6.0 and r["rows"][0] == 3
    # theta = 0.01: t = 6.03 -> only row 3 (r=9) ... and rows with r >= 6.03
    counts = _pick_counts(A, B, C, "rgrbk", 0.01, 400)
    assert counts[3] == 400
    # raise row 2 just above the small-theta threshold: r = (4, 5, 6.5, 9)
    r_t2 = np.array([4.0, 5.0, 6.5, 9.0])
    A, B, C, s = _diag_problem(r_t2, a)
    counts = _pick_counts(A, B, C, "rgrbk", 0.01, 3000)
    probs = np.array([0, 0, s[2], s[3]]) / (s[2] + s[3])
    assert _chi2_ok(counts, probs)
    # s-weights differ strongly from r-weights here: 6.5*0.25 vs 9*2
    assert counts[3] > 5 * counts[2]


def test_admission_is_inclusive_and_nonempty():
    """Equal weighted residuals: t equals every r_i, and ">=" admits all rows
    (Algorithm 3's set definition; Remark 4.1).  The pick is then ∝ s_i."""
    d = np.array([1.0, 2.0, 0.5, 3.0, 1.5])  # a_i = d_i^2 and sqrt(4 a_i) = 2 d_i are exact
    A, B, C, s = _diag_problem(np.full(5, 4.0), d ** 2)
    assert np.array_equal(C[:, 0], 2 * d)
    counts = _pick_counts(A, B, C, "grbk", 0.5, 4000)
    assert _chi2_ok(counts, s / s.sum())
    assert np.all(counts > 0)


def test_theta_one_is_mwrbk_and_half_is_grbk():
    """Remark 4.4: theta = 1/2 gives ME-GRBK; at theta = 1 the admitted set is
    the set of maximisers, i.e. the ME-MWRBK choice when the max is unique."""
    A, B, C, _ = workloads.gaussian(40, 7, 6, 25, seed=6)
    al = _alpha(B)
    g = oracle.solve(A, B, C, "grbk", alpha=al, seed=11, maxit=300)["rows"]
    h = oracle.solve(A, B, C, "rgrbk", theta=0.5, alpha=al, seed=11, maxit=300)["rows"]
    assert np.array_equal(g, h)
    t1 = oracle.solve(A, B, C, "rgrbk", theta=1.0, alpha=al, seed=11, maxit=300)["rows"]
    mw = oracle.solve(A, B, C, "mwrbk", alpha=al, seed=11, maxit=300)
    assert np.all(mw["margin_pick"] > 0)
    assert np.array_equal(t1, mw["rows"])


def test_admitted_sets_shrink_with_theta():
    """For fixed residuals the admitted set for a larger theta is a subset:
    over many draws the rows picked at theta=0.9 are a subset of those at 0.2,
    and the maximiser of r_i is always admissible (Remark 4.1)."""
    A, B, C, _ = workloads.gaussian(30, 6, 5, 12, seed=7)
    R = C
    s = np.einsum("ij,ij->i", R, R)
    r = s / np.einsum("ij,ij->i", A, A)
    lo = set(np.nonzero(_pick_counts(A, B, C, "rgrbk", 0.2, 600))[0])
    hi = set(np.nonzero(_pick_counts(A, B, C, "rgrbk", 0.9, 600))[0])
    assert hi <= lo
    assert int(np.argmax(r)) in lo and int(np.argmax(r)) in hi


def test_rbk_and_bk_rules():
    """Algorithm 1 picks row i with probability a_i / F; Algorithm 2 cycles."""
    a = np.array([1.0, 4.0, 0.25, 2.0, 3.0])
    A, B, C, _ = _diag_problem(np.array([1.0, 2, 3, 4, 5]), a)
    counts = _pick_counts(A, B, C, "rbk", 0.5, 4000)
    assert _chi2_ok(counts, a / a.sum())
    rows = oracle.solve(A, B, C, "bk", alpha=0.5, maxit=12)["rows"]
    assert np.array_equal(rows, np.arange(12) % 5)


def test_zero_row_of_A_is_never_selected():
    A, B, C, _ = workloads.gaussian(10, 4, 3, 7, seed=8)
    A[3] = 0.0
    C = A @ np.ones((4, 3)) @ B
    for v in ("grbk", "rgrbk", "mwrbk", "rbk"):
        rows = oracle.solve(A, B, C, v, theta=0.3, alpha=_alpha(B), seed=1, maxit=200)["rows"]
        assert 3 not in set(rows.tolist())


# ---------------------------------------------------------------- statistics

def test_expected_rate_bounds():
    """Lemma 2.2 / Eq. (2.3) for ME-RBK and Theorem 4.2 / Eq. (4.3) for ME-GRBK:
    the mean of ||X^k - X_*||^2 over seeds stays below the product of the
    per-step factors times ||X^0 - X_*||^2."""
    A, B, C, _ = workloads.gaussian(16, 5, 4, 12, seed=9)
    Xs = pinv(A) @ C @ pinv(B)
    alpha = _alpha(B)
    sa = np.linalg.svd(A, compute_uv=False)[-1]
    sb = np.linalg.svd(B, compute_uv=False)[-1]
    nb2 = np.linalg.norm(B, 2) ** 2
    FA, FB = np.sum(A * A), np.sum(B * B)
    rho = 1 - (2 * alpha - alpha ** 2 * nb2) / FA * sa ** 2 * sb ** 2
    kappa2 = FA * FB / (sa ** 2 * sb ** 2)
    rho0 = 1 - (2 * alpha - alpha ** 2 * nb2) * FB / kappa2
    K = 60
    for variant, bound in (("rbk", rho ** np.arange(K + 1)),
                           ("grbk", np.concatenate([[1.0], rho0 * rho ** np.arange(K)]))):
        errs = np.array([oracle.solve(A, B, C, variant, alpha=alpha, seed=sd, maxit=K, Xref=Xs,
                                      mode=oracle.MODE_FACTORED)["err2"] for sd in range(200)])
        mean = errs.mean(axis=0)
        assert np.all(mean <= bound * mean[0] * (1 + 1e-9))


def _rate_constants(A, B, alpha):
    sa = np.linalg.svd(A, compute_uv=False)[-1]
    sb = np.linalg.svd(B, compute_uv=False)[-1]
    nb2 = np.linalg.norm(B, 2) ** 2
    FA = np.sum(A * A)
    # kappa_{F,2}^2(B^T (x) A) = ||A||_F^2 ||B||_F^2 / (sigma_min(A) sigma_min(B))^2, so
    # rho_0 = 1 - (2 alpha - alpha^2 ||B||_2^2) ||B||_F^2 / kappa^2 = 1 - (...) sigma^2 sigma^2 / ||A||_F^2
    return 1 - (2 * alpha - alpha ** 2 * nb2) * sa ** 2 * sb ** 2 / FA


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.8])
def test_rgrbk_first_step_expectation_exact(theta):
    """Theorem 4.5 / Eq. (4.13) for ME-RGRBK, with the expectation taken
    exactly: the oracle's X^1 for every row it picks (seeds 0..599), weighted by
    Algorithm 4's probabilities s_i / S_J over the admitted set built here from
    R^0 = C; every admitted row must occur, no other row may, and the expected
    error must not exceed rho_0 ||X^0 - X_*||^2."""
    A, B, C, _ = workloads.gaussian(12, 4, 3, 10, seed=21)
    Xs = pinv(A) @ C @ pinv(B)
    alpha = _alpha(B)
    a = np.sum(A * A, axis=1)
    s = np.sum(C * C, axis=1)
    r = s / a
    t = min(theta * r.max() + (1 - theta) * s.sum() / a.sum(), r.max())
    J = np.nonzero(r >= t)[0]
    X1 = {}
    for sd in range(600):
        out = oracle.solve(A, B, C, "rgrbk", theta=theta, alpha=alpha, seed=sd, maxit=1)
        X1.setdefault(int(out["rows"][0]), out["X"])
    assert sorted(X1) == sorted(int(i) for i in J)
    E = sum(s[i] / s[J].sum() * np.sum((X1[int(i)] - Xs) ** 2) for i in J)
    assert E <= _rate_constants(A, B, alpha) * np.sum(Xs ** 2)


@pytest.mark.parametrize("theta", [0.3, 0.8])
def test_rgrbk_expected_rate_bound(theta):
    """Theorem 4.5 / Eq. (4.15) for ME-RGRBK: every factor rho_{l,theta} is at
    most rho_0 (Remark 4.6; equal to it while no residual row vanishes, when
    phi_l = ||B||_F^2), so the mean of ||X^k - X_*||^2 over 200 seeds stays
    below rho_0^k ||X^0 - X_*||^2."""
    A, B, C, _ = workloads.gaussian(16, 5, 4, 12, seed=9)
    Xs = pinv(A) @ C @ pinv(B)
    alpha = _alpha(B)
    rho = _rate_constants(A, B, alpha)
    K = 60
    errs = []
    for sd in range(200):
        out = oracle.solve(A, B, C, "rgrbk", theta=theta, alpha=alpha, seed=sd, maxit=K, Xref=Xs,
                           mode=oracle.MODE_FACTORED)
        errs.append(out["err2"])
    mean = np.mean(errs, axis=0)
    assert np.all(mean <= rho ** np.arange(K + 1) * mean[0] * (1 + 1e-9))


def test_greedy_needs_fewer_iterations_than_rbk_loose():
    """Loose sanity on a Table 3 shape (randn 140x30, 70x160): ME-GRBK and
    ME-MWRBK need fewer iterations than ME-RBK to RRN <= 1e-6 (squared ratio,
    i.e. RSE <= 1e-3).  The paper's exact counts are not reproducible (MATLAB
    random streams), so only the ordering is checked."""
    A, B, C, Xs = workloads.gaussian(140, 30, 70, 160, seed=10)
    al = _alpha(B)
    it = {}
    for v in ("rbk", "grbk", "mwrbk"):
        r = oracle.solve(A, B, C, v, alpha=al, seed=1, maxit=200000, Xref=Xs,
                         stop=oracle.STOP_RSE, tol=1e-3, mode=oracle.MODE_FACTORED, trace=False)
        assert r["status"] == oracle.TOL_MET
        it[v] = r["iters"]
    assert it["grbk"] < it["rbk"] and it["mwrbk"] <= it["grbk"] * 1.2


def test_stop_rules():
    A, B, C, Xs = workloads.gaussian(20, 6, 5, 15, seed=11)
    r = oracle.solve(A, B, C, "mwrbk", alpha=_alpha(B), maxit=100000, stop=oracle.STOP_RELRES,
                     tol=1e-8, trace=False, mode=oracle.MODE_FACTORED)
    assert r["status"] == oracle.TOL_MET
    assert np.linalg.norm(C - A @ r["X"] @ B) <= 1e-8 * np.linalg.norm(C) * (1 + 1e-6)
    r0 = oracle.solve(A, B, np.zeros_like(C), "grbk", alpha=_alpha(B), maxit=10)
    assert r0["status"] == oracle.EXACT and r0["iters"] == 0


# ------------------------------------------- least-squares extension (Eq. 2.1)

def _ls_system(seed=0, noise=0.1):
    """A 60x20 (full column rank), B 30x10 (full column rank, so B^+ B = I),
    C = A X* B + noise E with E generic: inconsistent on the side of A."""
    g = np.random.default_rng(700 + seed)
    A = g.standard_normal((60, 20))
    B = g.standard_normal((30, 10))
    Xs = g.standard_normal((20, 30))
    C = A @ Xs @ B + noise * g.standard_normal((60, 10))
    return A, B, C


def test_column_draw_matches_numpy_random():
    """The extended method's column draw is numpy's Philox block for counter
    (k, sys, 1, 0) -- word 2 of the counter selects the second stream."""
    for seed, k, sys in [(5, 0, 0), (99, 1234, 7), (2**40 + 3, 77, 191)]:
        c = k | (sys << 64) | (1 << 128)
        prev = (c - 1) % (1 << 256)
        words = np.array([(prev >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
        bg = np.random.Philox(counter=words, key=np.array([seed, 0], dtype=np.uint64))
        want = (int(bg.random_raw(4)[0]) >> 11) * 2.0 ** -53
        assert oracle.uniform_column(seed, k, sys) == want


@pytest.mark.parametrize("variant,theta", [("grbk", 0.5), ("rgrbk", 0.8), ("mwrbk", 1.0), ("rbk", 0.5)])
def test_extended_reaches_least_squares_solution(variant, theta):
    """Eq. 2.1: with B of full column rank the extended iteration tends to the
    least-squares solution of least norm A^+ C B^+ (numpy's pinv), while the
    plain iteration on the same inconsistent system stalls at an error floor."""
    A, B, C = _ls_system()
    Xls = pinv(A) @ C @ pinv(B)
    ext = oracle.solve(A, B, C, variant, theta=theta, alpha=_alpha(B), seed=3, maxit=60000,
                       mode=oracle.MODE_FACTORED, extended=True, trace=False, want_R=True)
    assert _rel(ext["X"], Xls) < 1e-8
    # the auxiliary matrix is the part of C outside the range of A: (I - A A^+) C
    assert _rel(ext["Y"], C - A @ pinv(A) @ C) < 1e-8
    plain = oracle.solve(A, B, C, variant, theta=theta, alpha=_alpha(B), seed=3, maxit=60000,
                         mode=oracle.MODE_FACTORED, trace=False)
    assert _rel(plain["X"], Xls) > 1e-3


def test_extended_residual_definition_and_consistent_case():
    """The kept residual of the extended iteration is C - Y - A X B (recursive
    and literal modes agree row for row); on a consistent system it reaches the
    solution like the plain method and Y tends to zero."""
    A, B, C = _ls_system(seed=1)
    for maxit in (1, 7, 300):
        f = oracle.solve(A, B, C, "grbk", alpha=_alpha(B), seed=4, maxit=maxit, mode=oracle.MODE_FACTORED,
                         extended=True, want_R=True)
        lit = oracle.solve(A, B, C, "grbk", alpha=_alpha(B), seed=4, maxit=maxit, mode=oracle.MODE_LITERAL,
                           extended=True, want_R=True)
        assert np.array_equal(f["rows"], lit["rows"])
        assert np.max(np.abs(f["R"] - (C - f["Y"] - A @ f["X"] @ B))) < 1e-12 * np.max(np.abs(C))
        assert np.max(np.abs(f["R"] - lit["R"])) < 1e-12 * np.max(np.abs(C))
    A, B, C0 = _ls_system(seed=2, noise=0.0)
    Xs = pinv(A) @ C0 @ pinv(B)
    ext = oracle.solve(A, B, C0, "grbk", alpha=_alpha(B), seed=5, maxit=60000, mode=oracle.MODE_FACTORED,
                       extended=True, want_R=True, trace=False)
    assert _rel(ext["X"], Xs) < 1e-8
    assert np.linalg.norm(ext["Y"]) < 1e-8 * np.linalg.norm(C0)
