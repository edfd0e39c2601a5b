"""CPU checks of the C-ABI library: it loads, exports every declared symbol, and
its host-side validation returns the documented codes (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsr_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def gsr():
    from paper_2503_22863_b300 import build
    build.build()
    from paper_2503_22863_b300 import gsr as g
    return g


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("gsr_create", "gsr_aprod1", "gsr_aprod2", "gsr_lsqr_solve", "gsr_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(gsr):
    lib = ctypes.CDLL(gsr._build.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_defaults(gsr):
    assert gsr.strerror(0) == "ok"
    assert "sorted" in gsr.strerror(3)
    o = gsr.LsqrOpts()
    gsr.lib.gsr_lsqr_default_opts(ctypes.byref(o))
    assert o.atol == 1e-12 and o.btol == 1e-12 and o.precond == 1 and o.precision == 0


def _tiny(n_glob=1):
    from paper_2503_22863_b300 import synth
    return synth.make_system(n_stars=10, n_knots=8, n_instr=7, n_glob=n_glob, obs=6,
                             poisson=False, seed=3)


def _create(gsr, sys, **over):
    d = gsr.Dims(sys["n_rows"], sys["n_stars"], sys["n_knots"], sys["n_instr"], sys["n_glob"], 0)
    for k, v in over.items():
        setattr(d, k, v)
    vals = np.ascontiguousarray(sys["vals"])
    ao = np.ascontiguousarray(sys["astro_off"])
    at = np.ascontiguousarray(sys["att_off"])
    ins = np.ascontiguousarray(sys["instr"])
    h = ctypes.c_void_p()
    code = gsr.lib.gsr_create(ctypes.byref(d), vals.ctypes.data_as(ctypes.c_void_p),
                              ao.ctypes.data_as(ctypes.c_void_p), at.ctypes.data_as(ctypes.c_void_p),
                              ins.ctypes.data_as(ctypes.c_void_p), 0, None, ctypes.byref(h))
    if code == 0:
        gsr.lib.gsr_destroy(h)
    return code


def test_create_rejects_bad_inputs_on_host(gsr):
    base = _tiny()
    assert _create(gsr, base, n_knots=3) == 1          # GSR_E_ARG
    assert _create(gsr, base, n_instr=5) == 1
    assert _create(gsr, base, n_glob=2) == 1
    assert _create(gsr, base, n_instr=70000) == 8       # GSR_E_UNSUPPORTED
    s = dict(base, astro_off=base["astro_off"].copy())
    s["astro_off"][3] = 7                               # not a multiple of 5
    assert _create(gsr, s) == 2
    s = dict(base, astro_off=base["astro_off"][::-1].copy())
    assert _create(gsr, s) == 3                         # GSR_E_UNSORTED
    s = dict(base, att_off=base["att_off"].copy())
    s["att_off"][0] = 5 * 10 + 5                        # s = 5 > K - 4 = 4
    assert _create(gsr, s) == 2
    s = dict(base, instr=base["instr"].copy())
    s["instr"][1, 2] = s["instr"][1, 1]                 # repeated instrumental column
    assert _create(gsr, s) == 2
    s = dict(base, instr=base["instr"].copy())
    s["instr"][0, 5] = 7                                # outside [0, n_instr)
    assert _create(gsr, s) == 2
    s = dict(base, vals=base["vals"].copy())
    s["vals"][4, 9] = np.nan
    assert _create(gsr, s) == 4                         # GSR_E_NONFINITE
    # an ignored global slot may hold anything when n_glob = 0
    s0 = _tiny(n_glob=0)
    s0 = dict(s0, vals=s0["vals"].copy())
    s0["vals"][:, 23] = np.inf
    s0["vals"][0, 0] = np.nan
    assert _create(gsr, s0) == 4


def test_learned_entry_points_validate_arguments(gsr):
    """The MLP / feature entry points reject bad arguments before touching a device."""
    lib = gsr.lib
    p = ctypes.c_void_p(8)  # never dereferenced: validation fails first
    E_ARG = 1
    assert lib.gsr_mlp_forward(p, -1, p, p, p, None) == E_ARG
    assert lib.gsr_mlp_forward(None, 5, p, p, p, None) == E_ARG
    assert lib.gsr_mlp_forward(None, 0, None, None, None, None) == 0  # nothing to do
    assert lib.gsr_mlp_grad(p, p, 0, p, p, p, p, None, None) == E_ARG
    assert lib.gsr_mlp_grad(p, None, 10, p, p, p, p, None, None) == E_ARG
    assert lib.gsr_mlp_adam(p, p, p, p, 0, ctypes.c_float(1e-3), ctypes.c_float(0.9),
                            ctypes.c_float(0.999), ctypes.c_float(1e-8), None) == E_ARG
    assert lib.gsr_mlp_adam(p, p, p, p, 1, ctypes.c_float(0.0), ctypes.c_float(0.9),
                            ctypes.c_float(0.999), ctypes.c_float(1e-8), None) == E_ARG
    assert lib.gsr_mlp_adam(p, p, p, p, 1, ctypes.c_float(1e-3), ctypes.c_float(1.0),
                            ctypes.c_float(0.999), ctypes.c_float(1e-8), None) == E_ARG
    assert lib.gsr_feature_moments(p, -3, p, None) == E_ARG
    assert lib.gsr_feature_moments(None, 0, p, None) == 0
    assert lib.gsr_feature_standardisation(None, 10, p, None) == E_ARG
    assert lib.gsr_feature_standardisation(p, 0, p, None) == E_ARG
    assert lib.gsr_column_features(None, p, None) == E_ARG
    assert lib.gsr_learned_scaling(None, None, ctypes.c_float(3.0), p, None) == E_ARG
    assert lib.gsr_n_learned_cols(None) == 0


def test_batch_entry_points_validate_arguments(gsr):
    lib = gsr.lib
    p = ctypes.c_void_p(8)
    E_ARG = 1
    for k in (0, 33):
        assert lib.gsr_aprod1_batch(None, k, p, p, None) == E_ARG
        assert lib.gsr_aprod2_batch(None, k, p, p, None) == E_ARG
    t = ctypes.c_int()
    assert lib.gsr_batch_tuning(None, ctypes.byref(t), ctypes.byref(t)) == E_ARG


def test_binding_refuses_host_tensors(gsr):
    # the binding marshals device pointers only: a host tensor is an error, not
    # a silent copy or a CPU path
    import torch
    with pytest.raises(TypeError):
        gsr._dptr(torch.zeros(3, dtype=torch.float64), 3, "x")
    with pytest.raises(TypeError):
        gsr._dptr2(torch.zeros((3, 2), dtype=torch.float64), 3, 2, "X")
    with pytest.raises(TypeError):
        gsr._dptr(np.zeros(3), 3, "x")


def test_create_rescaling_decision_on_host(gsr):
    """gsr_create's range check runs on the host before the device: a spread that
    no power-of-two row and column scaling removes is GSR_E_UNSUPPORTED; a row
    scaled far beyond FP32's range is accepted (rescaled exactly)."""
    base = _tiny()
    # rows 0 and 1 share star 0's astrometric columns 0 and 1; the 2 x 2 minor
    # a00 a11 / (a01 a10) = 1e70 is the same under every diagonal scaling, so
    # one of a01, a10 stays below 2^-100 of its row and column maxima
    s = dict(base, vals=base["vals"].copy())
    s["vals"][0, 0], s["vals"][0, 1] = 1.0, 1e-70
    s["vals"][1, 0], s["vals"][1, 1] = 1.0, 1.0
    assert _create(gsr, s) == 8                          # GSR_E_UNSUPPORTED
    # a diagonal scaling of an N(0,1) matrix is removable, however wide: row 3
    # times 1e200 and the global column (slot 23 of every row) times 1e-250
    s = dict(base, vals=base["vals"].copy())
    s["vals"][3, :] *= 1e200
    s["vals"][:, 23] *= 1e-250
    code = _create(gsr, s)
    assert code != 8 and code in (0, 6), code            # 6: no device on this host
    # subnormal FP64 coefficients are finite values: accepted
    s = dict(base, vals=base["vals"] * 1e-310)
    code = _create(gsr, s)
    assert code in (0, 6), code
