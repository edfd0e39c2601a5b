"""GPU parity of aprod 1 / aprod 2 (Eq. 2, Eq. 3) against the FP64 CPU oracle.

Element by element on seeded systems: the tiny 100,000-row workload, ragged
small shapes (partial last tile, single star, minimum knots and instrumental
columns, no global column, stars spanning lanes, tiles and warp ranges; the
knot-order copy of u blocked by rows, up to 32 blocks with a partial last
one, or not blocked), and
the full 30M-row workload in the bench's launch configuration. The bar:
max |gpu - oracle| / max (|A||x|) <= 1e-12 (aprod 1) and the
same with |A|^T|y| (aprod 2)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_22863_b300 import synth
from gpu_util import APROD_TOL, aprod1_ref, aprod2_ref, scaled_err, to_dev, to_host

pytestmark = pytest.mark.gpu

SHAPES = [
    dict(n_stars=2000, obs=50, poisson=False, n_knots=1000, n_instr=500, n_glob=1, seed=2503),
    dict(n_stars=37, obs=9, poisson=True, n_knots=30, n_instr=12, n_glob=1, seed=1),
    dict(n_stars=1, obs=300, poisson=False, n_knots=4, n_instr=6, n_glob=1, seed=2),
    dict(n_stars=50, obs=7, poisson=True, n_knots=4, n_instr=6, n_glob=0, seed=3),
    dict(n_stars=3000, obs=30, poisson=True, n_knots=200, n_instr=64, n_glob=1, seed=4),
    dict(n_stars=400, obs=1, poisson=False, n_knots=9, n_instr=7, n_glob=1, seed=5),
    dict(n_stars=5, obs=3000, poisson=False, n_knots=5000, n_instr=20000, n_glob=1, seed=6),
    # the most instrumental columns (split into two column groups), many tiles
    dict(n_stars=20000, obs=30, poisson=True, n_knots=3000, n_instr=24576, n_glob=1, seed=7),
    # few knots: the float-pair copy of u in the most row blocks (32, the last partial)
    dict(n_stars=5000, obs=40, poisson=True, n_knots=50, n_instr=100, n_glob=1, seed=8),
]


@pytest.fixture(scope="module")
def gsr():
    from paper_2503_22863_b300 import gsr as g
    return g


def _check_pair(gsr, sys, storage="f64", values="f64", rng_seed=0):
    rng = np.random.default_rng(rng_seed)
    with gsr.System(sys, storage=storage) as S:
        x = rng.standard_normal(S.n_unk)
        y0 = rng.standard_normal(S.n_rows)
        sysv = sys if values == "f64" else dict(sys, vals=sys["vals"].astype(np.float32).astype(np.float64))
        ref, scale = aprod1_ref(sysv, x, y0)
        y = to_dev(y0)
        S.aprod1(to_dev(x), y, values=values)
        e1 = scaled_err(to_host(y), ref, scale)
        u = rng.standard_normal(S.n_rows)
        x0 = rng.standard_normal(S.n_unk)
        ref2, scale2 = aprod2_ref(sysv, u, x0)
        xo = to_dev(x0)
        S.aprod2(to_dev(u), xo, values=values)
        e2 = scaled_err(to_host(xo), ref2, scale2)
    return e1, e2


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "s%d_k%d_i%d_g%d" % (
    s["n_stars"], s["n_knots"], s["n_instr"], s["n_glob"]))
def test_aprod_parity_shapes(gsr, shape):
    sys = synth.make_system(**shape)
    e1, e2 = _check_pair(gsr, sys)
    assert e1 <= APROD_TOL, e1
    assert e2 <= APROD_TOL, e2


def test_aprod_explicit_star_sizes(gsr):
    # stars of 0, 1, 2, ... rows: runs inside one lane, runs of one row, empty stars
    counts = np.array([0, 1, 2, 3, 0, 4, 5, 1, 1, 7, 128, 0, 129, 2, 255, 1, 1, 1, 3, 64] * 20)
    sys = synth.make_system(n_stars=counts.size, n_knots=17, n_instr=9, n_glob=1, counts=counts,
                            seed=8)
    e1, e2 = _check_pair(gsr, sys)
    assert e1 <= APROD_TOL and e2 <= APROD_TOL, (e1, e2)


def test_aprod_golden_probes(gsr):
    # the hand-worked 3-row system: exact small integers must come back exactly
    from dense_ref import load_probe_system
    sys, probes = load_probe_system()
    with gsr.System(sys) as S:
        for lhs, expect in probes:
            if lhs[0] == "aprod1":
                x = np.zeros(33)
                x[int(lhs[1])] = 1.0
                y = to_dev(np.zeros(3))
                S.aprod1(to_dev(x), y)
                assert to_host(y).tolist() == expect, lhs
            elif lhs[0] == "aprod2":
                y = np.zeros(3)
                y[int(lhs[1])] = 1.0
                xo = to_dev(np.zeros(33))
                S.aprod2(to_dev(y), xo)
                assert to_host(xo).tolist() == expect, lhs


def test_aprod_accumulates_and_is_repeatable(gsr):
    sys = synth.make_system(n_stars=500, n_knots=60, n_instr=40, n_glob=1, obs=20, seed=9)
    rng = np.random.default_rng(1)
    with gsr.System(sys) as S:
        x = to_dev(rng.standard_normal(S.n_unk))
        y = to_dev(np.zeros(S.n_rows))
        S.aprod1(x, y)
        S.aprod1(x, y)  # += twice
        y1 = to_dev(np.zeros(S.n_rows))
        S.aprod1(x, y1)
        np.testing.assert_allclose(to_host(y), 2 * to_host(y1), rtol=1e-14, atol=0)
        y2 = to_dev(np.zeros(S.n_rows))
        S.aprod1(x, y2)
        assert np.array_equal(to_host(y1), to_host(y2))  # aprod 1 is deterministic


def test_aprod_empty_system(gsr):
    sys = synth.make_system(n_stars=3, n_knots=4, n_instr=6, n_glob=1, counts=np.zeros(3, int),
                            seed=1)
    with gsr.System(sys) as S:
        assert S.n_rows == 0
        x = to_dev(np.ones(S.n_unk))
        y = torch.zeros(0, dtype=torch.float64, device="cuda")
        S.aprod1(x, y)
        xo = to_dev(np.full(S.n_unk, 2.0))
        S.aprod2(y, xo)
        assert (to_host(xo) == 2.0).all()


def test_aprod_adjoint_on_gpu(gsr):
    sys = synth.make_system(n_stars=20000, n_knots=3000, n_instr=800, n_glob=1, obs=30, seed=12)
    rng = np.random.default_rng(5)
    with gsr.System(sys) as S:
        x = rng.standard_normal(S.n_unk)
        y = rng.standard_normal(S.n_rows)
        ax = to_dev(np.zeros(S.n_rows))
        S.aprod1(to_dev(x), ax)
        aty = to_dev(np.zeros(S.n_unk))
        S.aprod2(to_dev(y), aty)
        lhs = float(to_host(ax) @ y)
        rhs = float(x @ to_host(aty))
        sabs = np.zeros(S.n_rows)
        oracle.aprod1(dict(sys, vals=np.abs(sys["vals"])), np.abs(x), sabs)
        assert abs(lhs - rhs) <= 1e-13 * float(sabs @ np.abs(y))


@pytest.mark.parametrize("values", ["f64", "f32"])
def test_aprod_f32_storage(gsr, values):
    # With F32_PLUS_F64 storage both copies are kept: the FP64 one must still
    # match A, the FP32 one must match the FP32-rounded matrix.
    sys = synth.make_system(n_stars=3000, n_knots=400, n_instr=300, n_glob=1, obs=25, seed=13)
    e1, e2 = _check_pair(gsr, sys, storage="f32+f64", values=values)
    assert e1 <= APROD_TOL and e2 <= APROD_TOL, (e1, e2)


@pytest.mark.parametrize("values", ["f64", "f32"])
@pytest.mark.parametrize("n_instr", [6145, 10000, 20000, 24576])
def test_aprod_instr_beyond_shared_memory(gsr, values, n_instr):
    # more instrumental unknowns than aprod 1 stages in shared memory beside its
    # record buffers (6,144): they are gathered through L1/L2 instead; one past
    # the limit up to the maximum, both value precisions, ragged last record
    sys = synth.make_system(n_stars=1500, n_knots=200, n_instr=n_instr, n_glob=1, obs=21,
                            poisson=True, seed=n_instr)
    e1, e2 = _check_pair(gsr, sys, storage="f32+f64", values=values, rng_seed=5)
    assert e1 <= APROD_TOL and e2 <= APROD_TOL, (e1, e2)


def test_aprod_parity_medium_full_size(gsr):
    """The 30M-row workload (the benchmark's), every element against the oracle."""
    sys = synth.make_config("medium")
    e1, e2 = _check_pair(gsr, sys, rng_seed=77)
    assert e1 <= APROD_TOL, e1
    assert e2 <= APROD_TOL, e2
