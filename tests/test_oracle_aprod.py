"""CPU pins of the oracle's aprod 1 / aprod 2 / column norms (Eq. 2, Eq. 3)."""
import numpy as np
import pytest

import oracle
from paper_2503_22863_b300 import synth
from dense_ref import dense, load_probe_system, n_unk, sparse


def small_cases():
    return [
        dict(n_stars=40, n_knots=30, n_instr=12, n_glob=1, obs=9, poisson=True, seed=1),
        dict(n_stars=25, n_knots=4, n_instr=6, n_glob=1, obs=5, poisson=False, seed=2),
        dict(n_stars=1, n_knots=8, n_instr=6, n_glob=0, obs=40, poisson=False, seed=3),
        dict(n_stars=60, n_knots=100, n_instr=80, n_glob=0, obs=7, poisson=True, seed=4),
    ]


def test_golden_unit_probes():
    sys, probes = load_probe_system()
    assert oracle.n_unknowns(sys) == 33
    seen = set()
    for lhs, expect in probes:
        kind = lhs[0]
        seen.add(kind)
        if kind == "aprod1":
            x = np.zeros(33)
            x[int(lhs[1])] = 1.0
            y = np.zeros(3)
            oracle.aprod1(sys, x, y)
            assert y.tolist() == expect, lhs
        elif kind == "accum1":
            x = np.zeros(33)
            x[int(lhs[1])] = 1.0
            y = np.array([float(t) for t in lhs[2:]])
            oracle.aprod1(sys, x, y)
            assert y.tolist() == expect, lhs
        elif kind == "aprod2":
            y = np.zeros(3)
            y[int(lhs[1])] = 1.0
            x = np.zeros(33)
            oracle.aprod2(sys, y, x)
            assert x.tolist() == expect, lhs
    assert seen == {"aprod1", "accum1", "aprod2"}


@pytest.mark.parametrize("case", small_cases())
def test_aprod_vs_dense(case):
    sys = synth.make_system(**case)
    A = dense(sys)
    rng = np.random.default_rng(7)
    x = rng.standard_normal(A.shape[1])
    y0 = rng.standard_normal(A.shape[0])
    y = y0.copy()
    oracle.aprod1(sys, x, y)
    ref = y0 + A @ x
    scale = np.abs(A) @ np.abs(x) + np.abs(y0)
    assert np.max(np.abs(y - ref) / scale) < 1e-14
    u = rng.standard_normal(A.shape[0])
    x0 = rng.standard_normal(A.shape[1])
    xo = x0.copy()
    oracle.aprod2(sys, u, xo)
    ref2 = x0 + A.T @ u
    scale2 = np.abs(A.T) @ np.abs(u) + np.abs(x0)
    assert np.max(np.abs(xo - ref2) / scale2) < 1e-14


def test_colnorm_vs_dense():
    sys = synth.make_system(**small_cases()[0])
    A = dense(sys)
    c2 = oracle.colnorm2(sys)
    np.testing.assert_allclose(c2, (A * A).sum(axis=0), rtol=1e-14, atol=0)


def test_adjoint_identity_medium():
    # <A x, y> = <x, A^T y> on a 200k-row system (no dense matrix needed).
    sys = synth.make_system(n_stars=5000, n_knots=2000, n_instr=300, n_glob=1, obs=40, seed=11)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(sys["n_unk"])
    y = rng.standard_normal(sys["n_rows"])
    ax = np.zeros(sys["n_rows"])
    oracle.aprod1(sys, x, ax)
    aty = np.zeros(sys["n_unk"])
    oracle.aprod2(sys, y, aty)
    lhs, rhs = ax @ y, x @ aty
    A = sparse(sys)
    bound = abs(A) @ np.abs(x) @ np.abs(y)
    assert abs(lhs - rhs) <= 1e-13 * bound


def test_linearity():
    sys = synth.make_system(n_stars=300, n_knots=50, n_instr=20, obs=12, seed=5)
    rng = np.random.default_rng(9)
    x1, x2 = rng.standard_normal((2, sys["n_unk"]))
    y1, y2, y12 = (np.zeros(sys["n_rows"]) for _ in range(3))
    oracle.aprod1(sys, x1, y1)
    oracle.aprod1(sys, x2, y2)
    oracle.aprod1(sys, 2.0 * x1 - 3.0 * x2, y12)
    np.testing.assert_allclose(y12, 2.0 * y1 - 3.0 * y2, rtol=0, atol=1e-12)


def test_generator_shapes_and_ranges():
    sys = synth.make_system(n_stars=500, n_knots=40, n_instr=9, n_glob=1, obs=30, seed=21)
    n = sys["n_rows"]
    assert sys["vals"].shape == (n, 24) and sys["instr"].shape == (n, 6)
    assert (np.diff(sys["astro_off"]) >= 0).all()
    s = sys["att_off"] - 5 * sys["n_stars"]
    assert s.min() >= 0 and s.max() <= sys["n_knots"] - 4
    ins = np.asarray(sys["instr"])
    assert (np.diff(ins, axis=1) > 0).all() and ins.min() >= 0 and ins.max() < 9
    assert (sys["counts"] >= 5).all()
    assert n_unk(sys) == sys["n_unk"]
    # deterministic in the seed, independent of the thread count
    again = synth.make_system(n_stars=500, n_knots=40, n_instr=9, n_glob=1, obs=30, seed=21,
                              threads=1)
    assert np.array_equal(again["vals"], sys["vals"])
    assert np.array_equal(again["instr"], sys["instr"])
