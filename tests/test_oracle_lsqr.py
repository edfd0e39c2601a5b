"""CPU pins of the oracle's LSQR (Paige & Saunders, the solver of Sec. 2.1)."""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

import oracle
from paper_2503_22863_b300 import synth
from dense_ref import columns, dense, sparse


def rhs(sys, consistent=False):
    b = np.zeros(sys["n_rows"])
    oracle.aprod1(sys, sys["x_star"], b)
    if not consistent:
        b += sys["noise"]
    return b


SMALL = dict(n_stars=60, n_knots=40, n_instr=15, n_glob=1, obs=20, poisson=True, seed=31)


def test_lsqr_vs_dense_qr():
    # The LSQR result is argmin ||A x - b||; LAPACK's QR/SVD least squares is the pin.
    sys = synth.make_system(**SMALL)
    b = rhs(sys)
    A = dense(sys)
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    for scale in ("colnorm", None):
        res = oracle.lsqr(sys, b, atol=1e-15, btol=1e-15, scale=scale)
        assert res["istop"] in (1, 2, 4, 5), res["istop"]
        err = np.linalg.norm(res["x"] - x_ls) / np.linalg.norm(x_ls)
        assert err < 1e-11, (scale, err)
        # normal-equation residual: A^T (b - A x) ~ 0 relative to ||A|| ||r||
        r = b - A @ res["x"]
        assert np.linalg.norm(A.T @ r) / (np.linalg.norm(A) * np.linalg.norm(r)) < 1e-12


def test_planted_solution_recovered():
    # "identity solution" of Sec. 3: a consistent b = A x* is solved exactly.
    sys = synth.make_system(n_stars=200, n_knots=60, n_instr=20, n_glob=1, obs=25, seed=32,
                            x_star="ones")
    b = rhs(sys, consistent=True)
    res = oracle.lsqr(sys, b, atol=1e-15, btol=1e-15)
    assert res["istop"] in (1, 4)
    assert np.max(np.abs(res["x"] - 1.0)) < 1e-10
    sys2 = synth.make_system(n_stars=200, n_knots=60, n_instr=20, n_glob=0, obs=25, seed=33)
    b2 = rhs(sys2, consistent=True)
    res2 = oracle.lsqr(sys2, b2, atol=1e-15, btol=1e-15)
    assert np.linalg.norm(res2["x"] - sys2["x_star"]) / np.linalg.norm(sys2["x_star"]) < 1e-10


@pytest.mark.parametrize("scale", [None, "colnorm"])
def test_iterates_match_scipy(scale):
    # scipy's LSQR is an independent textbook implementation of the same recurrence:
    # with the stopping tests disabled, x_k must agree for every k.
    sys = synth.make_system(**SMALL)
    b = rhs(sys)
    A = sparse(sys)
    if scale == "colnorm":
        c = np.sqrt(np.asarray(A.multiply(A).sum(axis=0))).ravel()
        d = 1.0 / c
    else:
        d = np.ones(A.shape[1])
    Ad = A @ sps.diags(d)
    # Unscaled, the iteration is ill-conditioned enough that a 1e-15 change of b moves
    # x_17 by ~1e-6 (intrinsic to the recurrence), so only early iterates are compared.
    ks = (1, 2, 5, 8) if scale is None else (1, 2, 5, 17, 40)
    for k in ks:
        res = oracle.lsqr(sys, b, atol=0.0, btol=0.0, conlim=0.0, itnlim=k, scale=scale)
        assert res["itn"] == k and res["istop"] == 7
        z = spla.lsqr(Ad, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=k)[0]
        ref = d * z
        tol = 1e-12 if scale is not None else 1e-10
        assert np.linalg.norm(res["x"] - ref) <= tol * np.linalg.norm(ref), k


def test_stopping_rule_matches_scipy():
    sys = synth.make_system(**SMALL)
    b = rhs(sys)
    A = sparse(sys)
    res = oracle.lsqr(sys, b, atol=1e-8, btol=1e-8, conlim=1e8, scale=None)
    out = spla.lsqr(A, b, atol=1e-8, btol=1e-8, conlim=1e8, iter_lim=10000)
    istop, itn = out[1], out[2]
    assert res["istop"] == istop
    # scipy estimates ||x|| by a recurrence; the oracle uses the exact norm, so the
    # stopping iteration may differ by one.
    assert abs(res["itn"] - itn) <= 1
    assert abs(res["rnorm"] - out[3]) <= 1e-10 * out[3]


def test_stopping_rule_on_the_preconditioned_system():
    # The loop runs on A D (Sec. 2, solver step 2) and de-preconditions after it
    # (step 5): its stopping tests use ||A D|| and the norm of the iterate z of
    # A D z = b, as scipy's LSQR does when given A D. Columns spread over 1e-8 ..
    # 1e8 make ||x|| = ||D z|| and ||z|| differ by orders of magnitude, so a test
    # on ||x|| would stop at a different iteration (here: at the first).
    sys = synth.make_system(**SMALL)
    C = 10.0 ** np.random.default_rng(8).uniform(-8, 8, oracle.n_unknowns(sys))
    cols = columns(sys)
    sys = dict(sys, vals=sys["vals"] * np.where(cols >= 0, C[np.maximum(cols, 0)], 0.0))
    b = rhs(sys)
    A = sparse(sys)
    c = np.sqrt(np.asarray(A.multiply(A).sum(axis=0))).ravel()
    Ad = A @ sps.diags(1.0 / c)
    for tol in (1e-6, 1e-10):
        res = oracle.lsqr(sys, b, atol=tol, btol=tol, conlim=1e8)
        out = spla.lsqr(Ad, b, atol=tol, btol=tol, conlim=1e8, iter_lim=10000)
        assert res["istop"] == out[1], tol
        assert abs(res["itn"] - out[2]) <= 1, (tol, res["itn"], out[2])
        assert res["itn"] > 10


def test_residual_estimates_and_monotonicity():
    sys = synth.make_system(**SMALL)
    b = rhs(sys)
    A = dense(sys)
    res = oracle.lsqr(sys, b, atol=0.0, btol=0.0, conlim=0.0, itnlim=30, want_rnorm_hist=True)
    h = res["rnorm_hist"]
    assert (np.diff(h) <= 1e-12 * h[0]).all()  # ||r_k|| is non-increasing
    r = b - A @ res["x"]
    assert abs(np.linalg.norm(r) - res["rnorm"]) <= 1e-10 * np.linalg.norm(b)
    arn = np.linalg.norm(res["scale"] * (A.T @ r))
    assert abs(arn - res["arnorm"]) <= 1e-8 * arn + 1e-14


def test_scaled_and_unscaled_agree():
    # Column scaling changes the iteration, never the least-squares answer.
    sys = synth.make_system(**SMALL)
    b = rhs(sys)
    a = oracle.lsqr(sys, b, atol=1e-15, btol=1e-15, scale=None)["x"]
    c = oracle.lsqr(sys, b, atol=1e-15, btol=1e-15, scale="colnorm")["x"]
    rng = np.random.default_rng(0)
    d = np.exp(rng.uniform(-1, 1, sys["n_unk"]))
    e = oracle.lsqr(sys, b, atol=1e-15, btol=1e-15, scale=d)["x"]
    assert np.linalg.norm(a - c) / np.linalg.norm(a) < 1e-11
    assert np.linalg.norm(a - e) / np.linalg.norm(a) < 1e-11


@pytest.mark.parametrize("params", [
    dict(n_stars=1, n_knots=4, n_instr=6, n_glob=1, obs=60, poisson=False, seed=42),
    dict(n_stars=2, n_knots=5, n_instr=6, n_glob=0, obs=100, poisson=False, seed=43),
])
def test_variance_vs_dense_inverse(params):
    # After n = N_unk steps the summed directions d_k = w_k/rho_k give
    # diag((A^T A)^{-1}) in exact arithmetic (Paige & Saunders' standard errors).
    # In FP64 the Golub-Kahan vectors lose orthogonality, so on these tiny
    # well-conditioned systems agreement is ~1e-4; a wrong term is O(1).
    sys = synth.make_system(**params)
    b = rhs(sys)
    A = dense(sys)
    n = A.shape[1]
    res = oracle.lsqr(sys, b, atol=0.0, btol=0.0, conlim=0.0, itnlim=n, want_var=True)
    ref = np.diag(np.linalg.inv(A.T @ A))
    np.testing.assert_allclose(res["var"], ref, rtol=1e-3)


def test_zero_rhs_and_zero_column():
    sys = synth.make_system(**SMALL)
    res = oracle.lsqr(sys, np.zeros(sys["n_rows"]))
    assert res["istop"] == 0 and res["itn"] == 0 and not res["x"].any()
    # an instrumental column that no row uses: scale 1, component stays 0
    sys2 = synth.make_system(n_stars=30, n_knots=20, n_instr=400, n_glob=1, obs=10, seed=5)
    used = np.zeros(400, bool)
    used[np.asarray(sys2["instr"]).ravel()] = True
    assert not used.all()
    b = rhs(sys2)
    r = oracle.lsqr(sys2, b, atol=1e-12, btol=1e-12)
    unused_cols = 5 * 30 + 3 * 20 + np.nonzero(~used)[0]
    assert np.all(r["x"][unused_cols] == 0.0)
    assert np.all(r["scale"][unused_cols] == 1.0)


def test_tiny_config_solution_vs_dense():
    # The 100,000-row workload: LSQR at tol 1e-12 vs the dense QR solution.
    sys = synth.make_config("tiny")
    b = rhs(sys)
    res = oracle.lsqr(sys, b, atol=1e-14, btol=1e-14)
    A = sparse(sys)
    # normal equations solved densely (13,501 unknowns) as the independent pin
    AtA = (A.T @ A).toarray()
    x_ne = np.linalg.solve(AtA, A.T @ b)
    err = np.linalg.norm(res["x"] - x_ne) / np.linalg.norm(x_ne)
    assert err < 1e-10, err


def test_rank_deficient_minimum_norm():
    # Rank-deficient A (stars with 1-4 rows, empty knot and instrumental
    # columns): LSQR from x0 = 0 on A D converges to the minimum-norm solution
    # of the scaled problem, x = D pinv(A D) b, with x_j = 0 on empty columns.
    sys = synth.rank_deficient_system()
    b = rhs(sys)
    A = dense(sys)
    c = np.sqrt((A ** 2).sum(axis=0))
    assert (c == 0).sum() > 100 and np.linalg.matrix_rank(A) < A.shape[1] - (c == 0).sum()
    d = np.where(c > 0, 1.0 / np.where(c > 0, c, 1.0), 1.0)
    x_pin = d * (np.linalg.pinv(A * d[None, :], rcond=1e-12) @ b)
    res = oracle.lsqr(sys, b, atol=1e-14, btol=1e-14)
    assert res["istop"] in (1, 2)
    assert np.linalg.norm(res["x"] - x_pin) / np.linalg.norm(x_pin) < 1e-12
    assert not res["x"][c == 0].any()


@pytest.mark.parametrize("params", [
    dict(n_stars=1, n_knots=4, n_instr=6, n_glob=1, obs=60, poisson=False, seed=42),
    dict(n_stars=2, n_knots=5, n_instr=6, n_glob=0, obs=100, poisson=False, seed=43),
])
def test_covariance_pairs_vs_dense_inverse(params):
    # Sec. 2.2, Eq. 4 read with the variance's direction vectors: after exactly
    # n = N_unk steps, sum_k d_k d_k^T = (A^T A)^{-1} in exact arithmetic, so
    # each pair's estimate is the (j1, j2) entry of the dense inverse. As for
    # the variance, only tiny systems whose run takes all n steps pin it (LSQR
    # that stops early at machine precision has explored less than the whole
    # space); the tolerance is the variance's, relative to sqrt(var_j1 var_j2)
    # because a covariance can be near zero. The run is column-scaled (as the
    # solver's is), so a missing de-preconditioning factor d_j1 d_j2 would be an
    # O(1) error. Every pair j1 <= j2 is checked; a
    # pair (j, j) must equal the variance exactly (the same sum), and swapping
    # the two indexes must change nothing.
    sys = synth.make_system(**params)
    b = rhs(sys)
    A = dense(sys)
    n = A.shape[1]
    inv = np.linalg.inv(A.T @ A)
    j1, j2 = np.triu_indices(n)
    pairs = np.stack([j1, j2], axis=1)
    res = oracle.lsqr(sys, b, atol=0.0, btol=0.0, conlim=0.0, itnlim=n, want_var=True,
                      cov_pairs=pairs)
    assert res["itn"] == n
    ref = inv[j1, j2]
    den = np.sqrt(np.diag(inv)[j1] * np.diag(inv)[j2])
    assert np.max(np.abs(res["cov"] - ref) / den) < 1e-3
    diag = j1 == j2
    np.testing.assert_array_equal(res["cov"][diag], res["var"][j1[diag]])
    sw = oracle.lsqr(sys, b, atol=0.0, btol=0.0, conlim=0.0, itnlim=n, cov_pairs=pairs[:, ::-1])
    np.testing.assert_array_equal(sw["cov"], res["cov"])
