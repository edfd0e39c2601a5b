"""GPU parity of the multi-right-hand-side forms (k systems sharing A).

Batched aprods against the oracle column by column (1e-12 scaled), and the
batched LSQR against k single-right-hand-side solves and the FP64 oracle
(1e-9); k = 1 equals the plain path; a right-hand side that has stopped keeps
its answer while the others continue."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_22863_b300 import synth
from gpu_util import (APROD_TOL, LSQR_TOL, abs_system, aprod1_ref, aprod2_ref, scaled_err, to_dev,
                      to_host)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsr():
    from paper_2503_22863_b300 import gsr as g
    return g


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("k", [1, 3, 8, 32])
def test_batched_aprod_parity(gsr, k):
    sys = synth.make_system(n_stars=3000, n_knots=300, n_instr=200, n_glob=1, obs=20, seed=71 + k)
    rng = np.random.default_rng(k)
    with gsr.System(sys) as S:
        X = rng.standard_normal((S.n_unk, k))
        Y0 = rng.standard_normal((S.n_rows, k))
        Y = to_dev(Y0)
        S.aprod1_batch(to_dev(X), Y)
        Yg = to_host(Y)
        U = rng.standard_normal((S.n_rows, k))
        X0 = rng.standard_normal((S.n_unk, k))
        Xo = to_dev(X0)
        S.aprod2_batch(to_dev(U), Xo)
        Xg = to_host(Xo)
    for j in range(k):
        ref, scale = aprod1_ref(sys, X[:, j], Y0[:, j])
        assert scaled_err(Yg[:, j], ref, scale) <= APROD_TOL, ("aprod1", j)
        ref2, scale2 = aprod2_ref(sys, U[:, j], X0[:, j])
        assert scaled_err(Xg[:, j], ref2, scale2) <= APROD_TOL, ("aprod2", j)


@pytest.mark.parametrize("k,n_stars", [(32, 10000), (5, 20000)])
def test_batched_aprod_multi_tile(gsr, k, n_stars):
    # more rows than one instrumental row tile (2^17 rows at k = 32, 2^19 at
    # k <= 8), with a ragged last tile
    sys = synth.make_system(n_stars=n_stars, n_knots=2000, n_instr=700, n_glob=1, obs=30,
                            seed=91 + k)
    rng = np.random.default_rng(100 + k)
    with gsr.System(sys) as S:
        assert S.n_rows > (1 << 17 if k > 8 else 1 << 19)
        X = rng.standard_normal((S.n_unk, k))
        Y0 = rng.standard_normal((S.n_rows, k))
        Y = to_dev(Y0)
        S.aprod1_batch(to_dev(X), Y)
        Yg = to_host(Y)
        U = rng.standard_normal((S.n_rows, k))
        X0 = rng.standard_normal((S.n_unk, k))
        Xo = to_dev(X0)
        S.aprod2_batch(to_dev(U), Xo)
        Xg = to_host(Xo)
    for j in (0, k // 2, k - 1):
        ref, scale = aprod1_ref(sys, X[:, j], Y0[:, j])
        assert scaled_err(Yg[:, j], ref, scale) <= APROD_TOL, ("aprod1", j)
        ref2, scale2 = aprod2_ref(sys, U[:, j], X0[:, j])
        assert scaled_err(Xg[:, j], ref2, scale2) <= APROD_TOL, ("aprod2", j)


@pytest.fixture(scope="module")
def tiny_batch():
    sys = synth.make_system(n_rhs=5, **synth.CONFIGS["tiny"])
    b0 = np.zeros(sys["n_rows"])
    oracle.aprod1(sys, sys["x_star"], b0)
    B = b0[:, None] + sys["noise"]
    return sys, B


def test_batched_lsqr_matches_oracle_and_single(gsr, tiny_batch):
    sys, B = tiny_batch
    k = B.shape[1]
    with gsr.System(sys) as S:
        r = S.lsqr_batch(to_dev(B), atol=1e-14, btol=1e-14)
        X = to_host(r["x"])
        tun = S.batch_tuning()
        assert tun["threads"] in (128, 256)
        assert tun["tile_rows"] >= 1 and tun["tile_rows"] & (tun["tile_rows"] - 1) == 0
        for j in (0, k - 1):
            single = S.lsqr(to_dev(B[:, j]), atol=1e-14, btol=1e-14)
            assert relerr(X[:, j], to_host(single["x"])) <= LSQR_TOL
            assert abs(r["itn"][j] - single["itn"]) <= 3
    for j in range(k):
        ref = oracle.lsqr(sys, B[:, j], atol=1e-14, btol=1e-14)
        assert relerr(X[:, j], ref["x"]) <= LSQR_TOL, j
        assert r["istop"][j] in (1, 2, 4, 5)


def test_batched_k1_equals_plain(gsr, tiny_batch):
    sys, B = tiny_batch
    b = B[:, :1].copy()
    with gsr.System(sys) as S:
        rb = S.lsqr_batch(to_dev(b), atol=1e-13, btol=1e-13)
        rs = S.lsqr(to_dev(b[:, 0]), atol=1e-13, btol=1e-13)
    assert relerr(to_host(rb["x"])[:, 0], to_host(rs["x"])) <= 1e-10
    assert abs(rb["itn"][0] - rs["itn"]) <= 1


def test_batched_masks_freeze_converged(gsr, tiny_batch):
    # one right-hand side is zero (stops at the start), one is consistent
    # (converges early); the others run on. Every answer must still be right.
    sys, B = tiny_batch
    B2 = B[:, :4].copy()
    B2[:, 1] = 0.0
    b0 = np.zeros(sys["n_rows"])
    oracle.aprod1(sys, sys["x_star"], b0)
    B2[:, 2] = b0
    with gsr.System(sys) as S:
        r = S.lsqr_batch(to_dev(B2), atol=1e-12, btol=1e-12)
        X = to_host(r["x"])
    assert r["istop"][1] == 0 and r["itn"][1] == 0 and not X[:, 1].any()
    assert relerr(X[:, 2], sys["x_star"]) <= 1e-9
    for j in (0, 3):
        ref = oracle.lsqr(sys, B2[:, j], atol=1e-12, btol=1e-12)
        assert relerr(X[:, j], ref["x"]) <= LSQR_TOL


def test_batched_error_history(gsr, tiny_batch):
    sys, B = tiny_batch
    with gsr.System(sys) as S:
        ref = S.lsqr_batch(to_dev(B), atol=1e-15, btol=1e-15)
        xr = ref["x"].clone()
        r = S.lsqr_batch(to_dev(B), atol=0.0, btol=0.0, conlim=0.0, itnlim=30, x_ref=xr,
                         err_hist=True)
    eh = r["err_hist"]
    assert eh.shape == (30, B.shape[1])
    assert (eh[-1] < 1e-6).all() and (eh[0] > eh[-1]).all()


def test_batched_aprod_medium_k32_sampled_columns(gsr):
    """The 30M-row workload with k = 32 right-hand sides (the benchmark's batched
    configuration): three whole columns of each product against the oracle."""
    sys = synth.make_config("medium")
    k = 32
    rng = np.random.default_rng(2532)
    with gsr.System(sys) as S:
        X = rng.standard_normal((S.n_unk, k))
        Y = torch.zeros((S.n_rows, k), dtype=torch.float64, device="cuda")
        S.aprod1_batch(to_dev(X), Y)
        cols = (0, 17, k - 1)
        Yg = {j: to_host(Y[:, j].contiguous()) for j in cols}
        del Y
        U = rng.standard_normal((S.n_rows, k))
        Xo = torch.zeros((S.n_unk, k), dtype=torch.float64, device="cuda")
        S.aprod2_batch(to_dev(U), Xo)
        Xg = {j: to_host(Xo[:, j].contiguous()) for j in cols}
    asys = abs_system(sys)
    for j in cols:
        xj, uj = np.ascontiguousarray(X[:, j]), np.ascontiguousarray(U[:, j])
        ref, scale = np.zeros(sys["n_rows"]), np.zeros(sys["n_rows"])
        oracle.aprod1(sys, xj, ref)
        oracle.aprod1(asys, np.abs(xj), scale)
        assert scaled_err(Yg[j], ref, scale) <= APROD_TOL, ("aprod1", j)
        ref2, scale2 = np.zeros(S.n_unk), np.zeros(S.n_unk)
        oracle.aprod2(sys, uj, ref2)
        oracle.aprod2(asys, np.abs(uj), scale2)
        assert scaled_err(Xg[j], ref2, scale2) <= APROD_TOL, ("aprod2", j)


def test_batched_mixed_matches_oracle(gsr, tiny_batch):
    """Mixed precision for k right-hand sides: an FP32-value phase (FP32
    products) and a float-pair correction phase on the residual; every column
    must meet the same 1e-9 bar against the FP64 oracle. A zero right-hand side
    and a consistent one exercise the masks in both phases."""
    sys, B = tiny_batch
    B2 = B.copy()
    B2[:, 1] = 0.0
    b0 = np.zeros(sys["n_rows"])
    oracle.aprod1(sys, sys["x_star"], b0)
    B2[:, 3] = b0
    refs = [oracle.lsqr(sys, B2[:, j], atol=1e-14, btol=1e-14) for j in range(B2.shape[1])]
    with gsr.System(sys, storage="f32+f64") as S:
        r = S.lsqr_batch(to_dev(B2), atol=1e-14, btol=1e-14, precision="mixed")
        X = to_host(r["x"])
        # a fixed first phase and the error history over both phases
        xr = to_dev(np.stack([ref["x"] for ref in refs], axis=1))
        r2 = S.lsqr_batch(to_dev(B2), atol=1e-14, btol=1e-14, precision="mixed",
                          mixed_switch_itn=25, x_ref=xr, err_hist=True)
    assert r["istop"][1] == 0 and not X[:, 1].any()
    for j in (0, 2, 3, 4):
        assert relerr(X[:, j], refs[j]["x"]) <= LSQR_TOL, j
        assert r["phase2_itn"][j] > 0 and r["itn"][j] > r["phase2_itn"][j], j
    assert relerr(X[:, 3], sys["x_star"]) <= 1e-9
    eh = r2["err_hist"]
    for j in (0, 2, 4):
        assert eh[24, j] > 1e-8          # the FP32 phase alone stops short of 1e-9
        assert np.nanmin(eh[:, j]) <= LSQR_TOL, j
