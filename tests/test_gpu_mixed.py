"""GPU parity of the mixed-precision solve (FP32-stored A, FP64 correction).

Phase 1 runs LSQR with the FP32-rounded matrix; phase 2 solves the correction
problem with the full-precision matrix. The final answer must meet the same
1e-9 bar against the FP64 oracle as the plain path; the error of the FP32
phase alone is recorded (it is bounded by the FP32 rounding of A, not 1e-9)."""
import numpy as np
import pytest

import oracle
from paper_2503_22863_b300 import synth
from gpu_util import LSQR_TOL, rhs, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsr():
    from paper_2503_22863_b300 import gsr as g
    return g


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def tiny():
    sys = synth.make_config("tiny")
    b = rhs(sys)
    ref = oracle.lsqr(sys, b, atol=1e-14, btol=1e-14)
    return sys, b, ref


def test_mixed_matches_fp64_oracle(gsr, tiny):
    sys, b, ref = tiny
    with gsr.System(sys, storage="f32+f64") as S:
        r = S.lsqr(to_dev(b), atol=1e-14, btol=1e-14, precision="mixed",
                   x_ref=to_dev(ref["x"]), err_hist=True)
        x = to_host(r["x"])
    err = relerr(x, ref["x"])
    assert err <= LSQR_TOL, err
    n2 = r["phase2_itn"]
    n1 = r["itn"] - n2
    assert n1 > 0 and n2 > 0
    eh = r["err_hist"]
    # the FP32 phase stalls at the FP32 rounding of A; the correction removes it
    assert 1e-10 < eh[n1 - 1] < 1e-4, eh[n1 - 1]
    assert eh[-1] <= LSQR_TOL


def test_mixed_fixed_switch(gsr, tiny):
    sys, b, ref = tiny
    with gsr.System(sys, storage="f32+f64") as S:
        r = S.lsqr(to_dev(b), atol=1e-14, btol=1e-14, precision="mixed", mixed_switch_itn=12)
    assert r["itn"] - r["phase2_itn"] == 12
    assert relerr(to_host(r["x"]), ref["x"]) <= LSQR_TOL


def test_mixed_requires_fp32_copy(gsr, tiny):
    sys, b, _ = tiny
    with gsr.System(sys) as S:
        with pytest.raises(gsr.GsrError):
            S.lsqr(to_dev(b), precision="mixed")


def test_fp32_phase_alone_is_fp32_accurate(gsr, tiny):
    # LSQR on the FP32-rounded matrix alone converges to the A32 solution, which
    # differs from the FP64 one by about the FP32 rounding of A.
    sys, b, ref = tiny
    sys32 = dict(sys, vals=sys["vals"].astype(np.float32).astype(np.float64))
    ref32 = oracle.lsqr(sys32, b, atol=1e-14, btol=1e-14)
    d = relerr(ref32["x"], ref["x"])
    assert 1e-9 < d < 1e-5, d


def test_many_instrumental_columns_both_phases(gsr):
    # 10,000 instrumental columns: more than aprod 1 stages beside two record
    # buffers per warp pair, so both precisions run its one-buffer configuration
    # with all of them in shared memory (LSQR form with the knot-order copy)
    sys = synth.make_system(n_stars=8000, obs=40, poisson=True, n_knots=400, n_instr=10000,
                            n_glob=1, seed=91)
    b = rhs(sys)
    ref = oracle.lsqr(sys, b, atol=1e-14, btol=1e-14)
    with gsr.System(sys, storage="f32+f64") as S:
        r64 = S.lsqr(to_dev(b), atol=1e-14, btol=1e-14)
        assert relerr(to_host(r64["x"]), ref["x"]) <= LSQR_TOL
        rm = S.lsqr(to_dev(b), atol=1e-14, btol=1e-14, precision="mixed")
        assert relerr(to_host(rm["x"]), ref["x"]) <= LSQR_TOL
