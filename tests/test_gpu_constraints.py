"""GPU parity with constraint equations (Sec. 2: a set of constraint equations
makes the solution unique; Sec. 2.1: about 1% of the system, replicated on
every process). Constraint rows are generic sparse rows after the
observations; the library computes them in FP64. Checked against the FP64
oracle: aprod 1 / aprod 2 element by element (1e-12 scaled by |A||x|),
including rows longer than one segment and coefficients far outside FP32's
range; LSQR (FP64-accurate and mixed precision, with variances and
covariances) on a rank-deficient system that the constraints make full rank
(1e-9); argument validation; replacing and removing the constraints."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_22863_b300 import synth
from gpu_util import APROD_TOL, LSQR_TOL, aprod1_ref, aprod2_ref, scaled_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsr():
    from paper_2503_22863_b300 import gsr as g
    return g


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def aprod_pair(gsr, sys, seed=0, storage="f64"):
    rng = np.random.default_rng(seed)
    m, n = oracle.n_equations(sys), oracle.n_unknowns(sys)
    x, y0, u, x0 = (rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(m),
                    rng.standard_normal(n))
    with gsr.System(sys, storage=storage) as S:
        assert S.n_eq == m
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
    dict(n_con=6, per_row=200),     # a few rows, one segment each
    dict(n_con=3, per_row=5000),    # rows of several 1024-entry segments
    dict(n_con=40, per_row=8),      # many short rows
    dict(n_con=1, per_row=1),       # one single-entry row
], ids=lambda c: "c%d_nnz%d" % (c["n_con"], c["per_row"]))
def test_constraint_aprods(gsr, case):
    base = synth.make_system(n_stars=2000, n_knots=300, n_instr=100, n_glob=1, obs=20, seed=81)
    sys = synth.add_constraints(base, seed=82, **case)
    e1, e2 = aprod_pair(gsr, sys, seed=3)
    assert e1 <= APROD_TOL and e2 <= APROD_TOL, (e1, e2)


def test_constraint_aprods_wide_values(gsr):
    # constraint coefficients over 1e-100 .. 1e100 (FP64 rows: no rescaling needed)
    base = synth.make_system(n_stars=500, n_knots=80, n_instr=30, n_glob=1, obs=20, seed=83)
    sys = synth.add_constraints(base, n_con=8, per_row=300, seed=84)
    rng = np.random.default_rng(4)
    sys["con_val"] = sys["con_val"] * 10.0 ** rng.uniform(-100, 100, sys["con_val"].size)
    e1, e2 = aprod_pair(gsr, sys, seed=5)
    assert e1 <= APROD_TOL and e2 <= APROD_TOL, (e1, e2)


@pytest.fixture(scope="module")
def constrained():
    """A rank-deficient system (four stars with 2 rows) made full rank by 16
    constraint rows, b = A x* + noise over all equations."""
    counts = np.array([25] * 300 + [2] * 4)
    base = synth.make_system(n_stars=304, n_knots=60, n_instr=20, n_glob=1, counts=counts, seed=85)
    sys = synth.add_constraints(base, n_con=16, per_row=120, seed=86,
                                must_cols=np.arange(5 * 300, 5 * 304))
    b = np.zeros(oracle.n_equations(sys))
    oracle.aprod1(sys, sys["x_star"], b)
    b += 1e-3 * np.random.default_rng(6).standard_normal(b.size)
    return sys, b


def test_constraint_lsqr(gsr, constrained):
    sys, b = constrained
    n = oracle.n_unknowns(sys)
    pairs = np.array([[0, 1], [5 * 300, 5 * 300 + 1], [5 * 301, 5 * 302], [n - 1, 7], [9, 9]],
                     dtype=np.int64)
    ref = oracle.lsqr(sys, b, atol=1e-14, btol=1e-14)
    # variances and covariances are sums over the run: compared over the same 15
    # iterations (before convergence, where both runs add the same terms)
    ref15 = oracle.lsqr(sys, b, atol=0.0, btol=0.0, conlim=0.0, itnlim=15, want_var=True,
                        cov_pairs=pairs)
    with gsr.System(sys, storage="f32+f64") as S:
        r = S.lsqr(to_dev(b), atol=1e-14, btol=1e-14, itnlim=5000)
        assert relerr(to_host(r["x"]), ref["x"]) <= LSQR_TOL
        assert abs(r["itn"] - ref["itn"]) <= 3
        assert abs(r["rnorm"] - ref["rnorm"]) <= 1e-9 * ref["rnorm"]
        r15 = S.lsqr(to_dev(b), atol=0.0, btol=0.0, conlim=0.0, itnlim=15, want_var=True,
                     cov_pairs=torch.from_numpy(pairs).cuda())
        var, cov = to_host(r15["var"]), to_host(r15["cov"])
        assert np.max(np.abs(var - ref15["var"]) / ref15["var"]) < 1e-6
        den = np.sqrt(ref15["var"][pairs[:, 0]] * ref15["var"][pairs[:, 1]])
        assert np.max(np.abs(cov - ref15["cov"]) / den) < 1e-6
        rm = S.lsqr(to_dev(b), atol=1e-14, btol=1e-14, itnlim=5000, precision="mixed")
        assert relerr(to_host(rm["x"]), ref["x"]) <= LSQR_TOL


def test_constraint_validation_replace_and_remove(gsr, constrained):
    sys, b = constrained
    base = {k: v for k, v in sys.items() if not k.startswith("con_")}
    with gsr.System(base) as S:
        assert S.n_eq == S.n_rows
        ptr, col, val = sys["con_ptr"], sys["con_col"].copy(), sys["con_val"].copy()
        col[3] = S.n_unk
        with pytest.raises(gsr.GsrError) as e:
            S.set_constraints(ptr, col, val)
        assert e.value.code == 2                      # GSR_E_INDEX
        col[3] = 0
        val[5] = np.inf
        with pytest.raises(gsr.GsrError) as e:
            S.set_constraints(ptr, col, val)
        assert e.value.code == 4                      # GSR_E_NONFINITE
        bad = ptr.copy()
        bad[2], bad[3] = bad[3], bad[2]
        with pytest.raises(gsr.GsrError) as e:
            S.set_constraints(bad, sys["con_col"], sys["con_val"])
        assert e.value.code == 1                      # GSR_E_ARG
        # set, replace by the same, solve; then remove and match the plain system
        S.set_constraints(ptr, sys["con_col"], sys["con_val"])
        S.set_constraints(ptr, sys["con_col"], sys["con_val"])
        assert S.n_eq == S.n_rows + 16
        ref = oracle.lsqr(sys, b, atol=1e-14, btol=1e-14)
        r = S.lsqr(to_dev(b), atol=1e-14, btol=1e-14, itnlim=5000)
        assert relerr(to_host(r["x"]), ref["x"]) <= LSQR_TOL
        with pytest.raises(gsr.GsrError) as e:
            S.lsqr_batch(to_dev(np.stack([b, b], axis=1)))
        assert e.value.code == 8                      # batched forms: no constraint rows
        S.set_constraints(np.zeros(1, np.int64), np.zeros(0, np.int64), np.zeros(0))
        assert S.n_eq == S.n_rows
        bo = b[:S.n_rows].copy()
        c_gpu = to_host(S.column_norms())
        np.testing.assert_allclose(c_gpu, np.sqrt(oracle.colnorm2(base)), rtol=1e-13)
        ref0 = oracle.lsqr(base, bo, atol=1e-14, btol=1e-14, itnlim=5000)
        r0 = S.lsqr(to_dev(bo), atol=1e-14, btol=1e-14, itnlim=5000)
        # rank-deficient without the constraints: both give the minimum-norm solution
        assert relerr(to_host(r0["x"]), ref0["x"]) <= LSQR_TOL
