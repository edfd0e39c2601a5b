"""CPU pins of the oracle's constraint rows (Sec. 2: the system needs a set of
constraint equations for a unique solution; Sec. 2.1: they are part of A).

The constraint rows are generic sparse rows after the observations: the
oracle's aprods must equal the dense [A; C] built independently, the adjoint
identity must hold, and LSQR on a rank-deficient A made full rank by the
constraints must give the unique least-squares solution of [A; C] x = [b; c]
(LAPACK)."""
import numpy as np

import oracle
from paper_2503_22863_b300 import synth
from dense_ref import dense


def test_constraint_aprods_vs_dense():
    base = synth.make_system(n_stars=40, n_knots=20, n_instr=12, n_glob=1, obs=15, seed=71)
    sys = synth.add_constraints(base, n_con=5, per_row=60, seed=72)
    A = dense(sys)
    m, n = A.shape
    assert m == sys["n_rows"] + 5 and oracle.n_equations(sys) == m
    rng = np.random.default_rng(1)
    x, y0, y, x0 = (rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(m),
                    rng.standard_normal(n))
    y1 = y0.copy()
    oracle.aprod1(sys, x, y1)
    np.testing.assert_allclose(y1, y0 + A @ x, rtol=0, atol=1e-12 * (np.abs(A) @ np.abs(x)).max())
    x1 = x0.copy()
    oracle.aprod2(sys, y, x1)
    np.testing.assert_allclose(x1, x0 + A.T @ y, rtol=0, atol=1e-12 * (np.abs(A).T @ np.abs(y)).max())
    # adjoint identity <A x, y> = <x, A^T y>
    ax = np.zeros(m)
    oracle.aprod1(sys, x, ax)
    aty = np.zeros(n)
    oracle.aprod2(sys, y, aty)
    assert abs(ax @ y - x @ aty) <= 1e-13 * np.abs(ax) @ np.abs(y)
    # column norms include the constraint rows
    np.testing.assert_allclose(oracle.colnorm2(sys), (A ** 2).sum(axis=0), rtol=1e-14)


def test_constraints_make_rank_deficient_system_unique():
    counts = np.array([25] * 60 + [2] * 4)   # the last four stars have 2 rows: rank-deficient
    base = synth.make_system(n_stars=64, n_knots=30, n_instr=10, n_glob=1, counts=counts,
                             seed=73)
    A0 = dense(base)
    assert np.linalg.matrix_rank(A0) < A0.shape[1]
    deficient = np.arange(5 * 60, 5 * 64)
    sys = synth.add_constraints(base, n_con=16, per_row=40, seed=74, must_cols=deficient)
    A = dense(sys)
    assert np.linalg.matrix_rank(A) == A.shape[1]
    rng = np.random.default_rng(2)
    b = A @ sys["x_star"] + 1e-3 * rng.standard_normal(A.shape[0])
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    res = oracle.lsqr(sys, b, atol=1e-15, btol=1e-15)
    assert res["istop"] in (1, 2, 4, 5)
    assert np.linalg.norm(res["x"] - x_ls) / np.linalg.norm(x_ls) < 1e-11
