"""The all-core CPU baseline's products agree with the oracle (so that the
benchmark times a correct CPU implementation)."""
import numpy as np

import cpu_baseline
import oracle
from paper_2503_22863_b300 import synth


def test_openmp_aprods_match_oracle():
    counts = np.array([0, 1, 2, 7, 30, 3, 0, 55] * 40)
    sys = synth.make_system(n_stars=counts.size, n_knots=50, n_instr=30, n_glob=1, counts=counts,
                            seed=91)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(sys["n_unk"]), rng.standard_normal(sys["n_rows"])
    for glob in (1, 0):
        s = dict(sys, n_glob=glob, n_unk=sys["n_unk"] - 1 + glob,
                 vals=sys["vals"] if glob else np.where(np.arange(24) == 23, 0.0, sys["vals"]))
        xs = x[:s["n_unk"]]
        ya, yb = np.zeros(s["n_rows"]), np.zeros(s["n_rows"])
        oracle.aprod1(s, xs, ya)
        cpu_baseline.aprod1(s, xs, yb)
        assert np.max(np.abs(ya - yb)) <= 1e-13 * np.max(np.abs(ya))
        xa, xb = np.zeros(s["n_unk"]), np.zeros(s["n_unk"])
        oracle.aprod2(s, y, xa)
        cpu_baseline.aprod2(s, y, xb)
        assert np.max(np.abs(xa - xb)) <= 1e-13 * np.max(np.abs(xa))
    assert cpu_baseline.threads() >= 1
