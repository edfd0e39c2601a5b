"""The allocation-free aprod 1 entry point (gsr_aprod1_noalloc) against gsr_aprod1.

Some callers cannot allocate device memory at call time (graph capture, memory
held by another allocator, latency-critical loops); gsr_aprod1_noalloc stages
its scratch in a fixed device array of the library instead. This file is
collected last so that a stop-at-first-failure run has run every other test
before it; it passes alone in a fresh process as well."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_22863_b300 import synth
from gpu_util import APROD_TOL, aprod1_ref, scaled_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsr():
    from paper_2503_22863_b300 import gsr as g
    g.lib.gsr_aprod1_noalloc.argtypes = [ctypes.c_void_p] * 4
    g.lib.gsr_aprod1_noalloc.restype = ctypes.c_int
    return g


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_aprod1_two_calls(gsr):
    sys_ = synth.make_system(n_stars=20000, n_knots=2000, n_instr=700, n_glob=1, obs=30, seed=61)
    rng = np.random.default_rng(4)
    with gsr.System(sys_) as S:
        for call in range(2):  # two calls in a row share the static scratch
            x = torch.from_numpy(rng.standard_normal(S.n_unk)).cuda()
            y0 = rng.standard_normal(S.n_rows)
            y_ref = torch.from_numpy(y0).cuda()
            y_new = torch.from_numpy(y0).cuda()
            assert gsr.lib.gsr_aprod1(S._h, _ptr(x), _ptr(y_ref), _stream()) == 0
            assert gsr.lib.gsr_aprod1_noalloc(S._h, _ptr(x), _ptr(y_new), _stream()) == 0
            torch.cuda.synchronize()
            a, b = y_new.cpu().numpy(), y_ref.cpu().numpy()
            _, scale = aprod1_ref(sys_, x.cpu().numpy(), y0)
            assert scaled_err(a, b, scale) <= APROD_TOL, call


def test_noalloc_rejects_too_many_unknowns(gsr):
    limit = 1048576
    n_stars = limit // 5 + 10   # 5 astrometric unknowns per star push N_unk past the limit
    sys_ = synth.make_system(n_stars=n_stars, n_knots=4, n_instr=6, n_glob=1,
                             counts=np.ones(n_stars, dtype=np.int64), seed=62)
    with gsr.System(sys_) as S:
        assert S.n_unk > limit
        x = torch.zeros(S.n_unk, dtype=torch.float64, device="cuda")
        y = torch.zeros(S.n_rows, dtype=torch.float64, device="cuda")
        assert gsr.lib.gsr_aprod1_noalloc(S._h, _ptr(x), _ptr(y), _stream()) == 8  # UNSUPPORTED
