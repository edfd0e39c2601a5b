"""GPU parity of the products and solves on inputs far outside FP32's range.

The coefficients of Eq. 2 / Eq. 3 and the vectors are FP64 (Sec. 2); the
library's float-pair kernels carry FP32's exponent range, so it rescales the
problem by exact powers of two and falls back to FP64 kernels for inputs it
cannot rescale into range. These tests check that no valid FP64 input gives a
wrong answer: rows and columns of A, x and y spanning 1e-30 .. 1e30, values
beyond FP32 (1e-150 .. 1e150) and products in FP64's subnormal range, each
against the FP64 oracle element by element (aprod 1e-12 scaled by |A||x|,
LSQR 1e-9 relative), and the documented error codes where a call is refused.
"""
import numpy as np
import pytest
import torch

import oracle
from dense_ref import columns
from paper_2503_22863_b300 import synth
from gpu_util import APROD_TOL, LSQR_TOL, aprod1_ref, aprod2_ref, scaled_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsr():
    from paper_2503_22863_b300 import gsr as g
    return g


def rescaled(base, row_dec=0.0, col_dec=0.0, factor=1.0, seed=0):
    """base with A_ij -> factor * R_i A_ij C_j, R and C log-uniform over
    10^[-dec, dec]; returns the system and C."""
    rng = np.random.default_rng(seed)
    cols = columns(base)
    n_unk = oracle.n_unknowns(base)
    R = 10.0 ** rng.uniform(-row_dec, row_dec, base["n_rows"]) if row_dec else np.ones(base["n_rows"])
    C = 10.0 ** rng.uniform(-col_dec, col_dec, n_unk) if col_dec else np.ones(n_unk)
    cmul = np.where(cols >= 0, C[np.maximum(cols, 0)], 0.0)
    vals = factor * base["vals"] * R[:, None] * cmul
    return dict(base, vals=vals), C


def wide_vector(rng, n, dec):
    return rng.standard_normal(n) * 10.0 ** rng.uniform(-dec, dec, n)


def base_system(seed, n_glob=1):
    return synth.make_system(n_stars=300, n_knots=60, n_instr=40, n_glob=n_glob, obs=20,
                             seed=seed)


def aprod_errors(gsr, sys, x, y0, u, x0):
    with gsr.System(sys) as S:
        ref, scale = aprod1_ref(sys, x, y0)
        y = to_dev(y0)
        S.aprod1(to_dev(x), y)
        e1 = scaled_err(to_host(y), ref, scale)
        ref2, scale2 = aprod2_ref(sys, u, x0)
        xo = to_dev(x0)
        S.aprod2(to_dev(u), xo)
        e2 = scaled_err(to_host(xo), ref2, scale2)
    return e1, e2


@pytest.mark.parametrize("case", [
    dict(row_dec=30, col_dec=30, x_dec=30, seed=41),   # rows, columns and vectors 1e-30..1e30
    dict(row_dec=0, col_dec=30, x_dec=0, seed=42),     # columns only (LSQR-compatible)
    dict(row_dec=30, col_dec=0, x_dec=0, seed=43),     # rows only
    dict(row_dec=0, col_dec=0, x_dec=30, seed=44),     # vectors only, A unscaled
    dict(row_dec=150, col_dec=0, x_dec=150, seed=45),  # beyond FP32: 1e-150 .. 1e150
], ids=lambda c: "r%d_c%d_x%d" % (c["row_dec"], c["col_dec"], c["x_dec"]))
def test_aprod_wide_magnitudes(gsr, case):
    base = base_system(case["seed"])
    sys, _ = rescaled(base, case["row_dec"], case["col_dec"], seed=case["seed"])
    rng = np.random.default_rng(case["seed"] + 100)
    n, m = sys["n_rows"], oracle.n_unknowns(sys)
    dec = case["x_dec"]
    x = wide_vector(rng, m, dec) if dec else rng.standard_normal(m)
    y0 = wide_vector(rng, n, dec) if dec else rng.standard_normal(n)
    u = wide_vector(rng, n, dec) if dec else rng.standard_normal(n)
    x0 = wide_vector(rng, m, dec) if dec else rng.standard_normal(m)
    e1, e2 = aprod_errors(gsr, sys, x, y0, u, x0)
    assert e1 <= APROD_TOL, e1
    assert e2 <= APROD_TOL, e2


def test_aprod_column_rescaled_float_pair_path(gsr):
    """Columns spread over 1e-30..1e30 with x = N(0,1)/C: the rescaled x lies in
    the float-pair band, so the float-pair kernels (with the column and output
    exponents) run, not the FP64 ones."""
    base = base_system(46)
    sys, C = rescaled(base, col_dec=30, seed=46)
    rng = np.random.default_rng(146)
    n, m = sys["n_rows"], oracle.n_unknowns(sys)
    x = rng.standard_normal(m) / C
    u = rng.standard_normal(n)
    e1, e2 = aprod_errors(gsr, sys, x, rng.standard_normal(n), u, rng.standard_normal(m) / C)
    assert e1 <= APROD_TOL and e2 <= APROD_TOL, (e1, e2)


def test_aprod_subnormal_products(gsr):
    """A at 1e-300 times x at 1e-10: products and results in FP64's subnormal
    range, as the oracle computes them."""
    base = base_system(47)
    sys, _ = rescaled(base, factor=1e-300, seed=47)
    rng = np.random.default_rng(147)
    n, m = sys["n_rows"], oracle.n_unknowns(sys)
    x = 1e-10 * rng.standard_normal(m)
    u = 1e-10 * rng.standard_normal(n)
    e1, e2 = aprod_errors(gsr, sys, x, np.zeros(n), u, np.zeros(m))
    assert e1 <= APROD_TOL and e2 <= APROD_TOL, (e1, e2)


def test_aprod_no_global_column_wide(gsr):
    base = base_system(48, n_glob=0)
    sys, _ = rescaled(base, row_dec=30, col_dec=30, seed=48)
    rng = np.random.default_rng(148)
    n, m = sys["n_rows"], oracle.n_unknowns(sys)
    e1, e2 = aprod_errors(gsr, sys, wide_vector(rng, m, 30), wide_vector(rng, n, 30),
                          wide_vector(rng, n, 30), wide_vector(rng, m, 30))
    assert e1 <= APROD_TOL and e2 <= APROD_TOL, (e1, e2)


@pytest.mark.parametrize("dec", [0, 30])
def test_batched_aprod_wide_magnitudes(gsr, dec):
    """k = 3 columns of very different magnitude through the batched products."""
    base = base_system(49)
    sys, C = rescaled(base, row_dec=30 if dec else 0, col_dec=30, seed=49)
    rng = np.random.default_rng(149)
    n, m, k = sys["n_rows"], oracle.n_unknowns(sys), 3
    X = np.stack([wide_vector(rng, m, 30), 1e20 * rng.standard_normal(m) / C,
                  rng.standard_normal(m) / C], axis=1) if dec else \
        np.stack([rng.standard_normal(m) / C * s for s in (1e-20, 1.0, 1e20)], axis=1)
    Y0 = rng.standard_normal((n, k))
    U = np.stack([wide_vector(rng, n, 30), rng.standard_normal(n), 1e-25 * rng.standard_normal(n)],
                 axis=1)
    with gsr.System(sys) as S:
        Yd = to_dev(Y0)
        S.aprod1_batch(to_dev(X), Yd)
        Xd = torch.zeros((m, k), dtype=torch.float64, device="cuda")
        S.aprod2_batch(to_dev(U), Xd)
        Yg, Xg = to_host(Yd), to_host(Xd)
    for j in range(k):
        ref, scale = aprod1_ref(sys, X[:, j], Y0[:, j])
        assert scaled_err(Yg[:, j], ref, scale) <= APROD_TOL, j
        ref2, scale2 = aprod2_ref(sys, U[:, j], np.zeros(m))
        assert scaled_err(Xg[:, j], ref2, scale2) <= APROD_TOL, j


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def lsqr_case(seed, factor, b_scale):
    """A = factor * A0 * C (columns over 1e-30..1e30), b = b_scale (A x* + noise)
    with x* = N(0,1)/C, so x spans 1e-30..1e30 too."""
    base = synth.make_system(n_stars=400, n_knots=80, n_instr=30, n_glob=1, obs=25, seed=seed)
    sys, C = rescaled(base, col_dec=30, factor=factor, seed=seed)
    rng = np.random.default_rng(seed + 7)
    xs = rng.standard_normal(oracle.n_unknowns(sys)) / C
    b = np.zeros(sys["n_rows"])
    oracle.aprod1(sys, xs, b)
    b = b_scale * (b + 1e-3 * factor * rng.standard_normal(sys["n_rows"]))
    return sys, b


@pytest.mark.parametrize("factor,b_scale", [(1e-30, 1.0), (1.0, 1e-35), (1e30, 1e40)],
                         ids=["A1e-30", "b1e-35", "A1e30_b1e40"])
def test_lsqr_wide_magnitudes(gsr, factor, b_scale):
    sys, b = lsqr_case(51, factor, b_scale)
    ref = oracle.lsqr(sys, b, atol=1e-14, btol=1e-14)
    with gsr.System(sys) as S:
        r = S.lsqr(to_dev(b), atol=1e-14, btol=1e-14, itnlim=5000, x_ref=to_dev(ref["x"]),
                   err_hist=True)
        x = to_host(r["x"])
    # the stopping tests run on the preconditioned system, so the spread of x
    # does not end the run early: both sides iterate to convergence
    assert ref["itn"] > 10 and r["itn"] > 10, (ref["itn"], r["itn"])
    assert relerr(x, ref["x"]) <= LSQR_TOL
    assert r["err_hist"][-1] <= LSQR_TOL
    assert abs(r["rnorm"] - ref["rnorm"]) <= 1e-6 * ref["rnorm"]
    assert abs(r["xnorm"] - ref["xnorm"]) <= 1e-9 * ref["xnorm"]


def test_lsqr_wide_mixed_and_variance(gsr):
    sys, b = lsqr_case(52, 1e-30, 1e-5)
    ref = oracle.lsqr(sys, b, atol=1e-14, btol=1e-14)
    assert ref["itn"] > 10
    # the variance (a sum over the run) over the same 15 iterations on both sides,
    # before convergence (past it the added terms are rounding noise and the two
    # runs' sums part), so the two sums have the same terms; it spans ~1e40 ..
    # 1e110 here
    ref_v = oracle.lsqr(sys, b, atol=0.0, btol=0.0, conlim=0.0, itnlim=15, want_var=True)
    with gsr.System(sys, storage="f32+f64") as S:
        r = S.lsqr(to_dev(b), atol=1e-14, btol=1e-14, precision="mixed", itnlim=5000)
        assert r["phase2_itn"] > 0 and r["itn"] - r["phase2_itn"] > 10
        assert relerr(to_host(r["x"]), ref["x"]) <= LSQR_TOL
        r = S.lsqr(to_dev(b), atol=0.0, btol=0.0, conlim=0.0, itnlim=15, want_var=True)
        var = to_host(r["var"])
    assert r["itn"] == 15
    assert np.max(np.abs(var - ref_v["var"]) / ref_v["var"]) < 1e-6


def test_lsqr_batch_wide_magnitudes(gsr):
    sys, b1 = lsqr_case(53, 1.0, 1e-30)
    _, b2 = lsqr_case(53, 1.0, 1e30)
    rng = np.random.default_rng(5)
    b3 = b1 * 1e32 + 1e-3 * rng.standard_normal(b1.size)
    B = np.stack([b1, b2, b3], axis=1)
    with gsr.System(sys) as S:
        r = S.lsqr_batch(to_dev(B), atol=1e-14, btol=1e-14, itnlim=5000)
        X = to_host(r["x"])
    for j in range(3):
        ref = oracle.lsqr(sys, B[:, j], atol=1e-14, btol=1e-14)
        assert relerr(X[:, j], ref["x"]) <= LSQR_TOL, j
        assert abs(r["rnorm"][j] - ref["rnorm"]) <= 1e-6 * ref["rnorm"], j


def test_lsqr_refuses_row_rescaled_system(gsr):
    """Rows that need different exponents: the products work, LSQR says
    GSR_E_UNSUPPORTED (the row rescaling is not folded into the solve)."""
    base = base_system(54)
    sys, _ = rescaled(base, row_dec=30, seed=54)
    with gsr.System(sys) as S:
        with pytest.raises(gsr.GsrError) as e:
            S.lsqr(to_dev(np.ones(sys["n_rows"])))
        assert e.value.code == 8
        with pytest.raises(gsr.GsrError) as e:
            S.lsqr_batch(to_dev(np.ones((sys["n_rows"], 2))))
        assert e.value.code == 8


def test_lsqr_rejects_nonfinite_rhs_and_bad_scale(gsr):
    sys = base_system(55)
    b = np.ones(sys["n_rows"])
    b[17] = np.nan
    with gsr.System(sys) as S:
        with pytest.raises(gsr.GsrError) as e:
            S.lsqr(to_dev(b))
        assert e.value.code == 4
        with pytest.raises(gsr.GsrError) as e:
            S.lsqr_batch(to_dev(np.stack([np.ones_like(b), b], axis=1)))
        assert e.value.code == 4
        d = np.ones(sys["n_unk"])
        d[3] = -1.0
        with pytest.raises(gsr.GsrError) as e:
            S.lsqr(to_dev(np.ones_like(b)), precond="user", scale=to_dev(d))
        assert e.value.code == 1
        # the system is still usable afterwards
        r = S.lsqr(to_dev(np.ones_like(b)), itnlim=3)
        assert r["itn"] == 3
