"""ctypes shim over ``gsr_oracle.c`` (test infrastructure only).

The C file is compiled with ``-O2 -ffp-contract=off`` into ``oracle/_build``.
Arrays are numpy; every function copies nothing it does not have to.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_p = ctypes.c_void_p


def build_oracle(force=False):
    """Compile the C oracle (plain gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(_SO)
        dims = [_i64, _i64, _i64, _i64, _i32]
        lib.oracle_n_unknowns.argtypes = dims
        lib.oracle_n_unknowns.restype = _i64
        cons = [_i64, _p, _p, _p]
        for name in ("oracle_aprod1", "oracle_aprod2"):
            getattr(lib, name).argtypes = dims + [_p] * 4 + cons + [_p] * 2
            getattr(lib, name).restype = None
        lib.oracle_colnorm2.argtypes = dims + [_p] * 4 + cons + [_p]
        lib.oracle_colnorm2.restype = None
        lib.oracle_lsqr.argtypes = (dims + [_p] * 4 + cons + [_p] * 3 + [_i64] + [_p] * 5 +
                                    [_i64, _p, _p, _p])
        lib.oracle_lsqr.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_p) if a is not None else None


def _dims(sys):
    return (int(sys["n_rows"]), int(sys["n_stars"]), int(sys["n_knots"]),
            int(sys["n_instr"]), int(sys["n_glob"]))


def _arrays(sys):
    vals = np.ascontiguousarray(sys["vals"], dtype=np.float64)
    ao = np.ascontiguousarray(sys["astro_off"], dtype=np.int64)
    at = np.ascontiguousarray(sys["att_off"], dtype=np.int64)
    ins = np.ascontiguousarray(sys["instr"], dtype=np.int32)
    assert vals.shape == (sys["n_rows"], 24) and ins.shape == (sys["n_rows"], 6)
    return vals, ao, at, ins


def _cons(sys):
    """(n_con, ptr, col, val) of the system's constraint rows (CSR; none: 0)."""
    if sys.get("con_ptr") is None:
        return 0, None, None, None
    ptr = np.ascontiguousarray(sys["con_ptr"], dtype=np.int64)
    col = np.ascontiguousarray(sys["con_col"], dtype=np.int64)
    val = np.ascontiguousarray(sys["con_val"], dtype=np.float64)
    n_con = ptr.size - 1
    assert n_con >= 0 and ptr[0] == 0 and ptr[-1] == col.size == val.size
    return n_con, ptr, col, val


def _cons_args(c):
    return (c[0], _ptr(c[1]), _ptr(c[2]), _ptr(c[3]))


def n_equations(sys):
    """Rows of A: the observations and the constraint rows."""
    return int(sys["n_rows"]) + _cons(sys)[0]


def n_unknowns(sys):
    return int(_load().oracle_n_unknowns(*_dims(sys)))


def aprod1(sys, x, y):
    """Eq. 2: y += A x (in place on ``y``, which must be float64 contiguous, with
    one entry per equation: observations, then constraint rows)."""
    lib = _load()
    vals, ao, at, ins = _arrays(sys)
    c = _cons(sys)
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert y.dtype == np.float64 and y.flags.c_contiguous and y.shape == (n_equations(sys),)
    lib.oracle_aprod1(*_dims(sys), _ptr(vals), _ptr(ao), _ptr(at), _ptr(ins), *_cons_args(c),
                      _ptr(x), _ptr(y))
    return y


def aprod2(sys, y, x):
    """Eq. 3: x += A^T y (in place on ``x``)."""
    lib = _load()
    vals, ao, at, ins = _arrays(sys)
    c = _cons(sys)
    y = np.ascontiguousarray(y, dtype=np.float64)
    assert y.shape == (n_equations(sys),)
    assert x.dtype == np.float64 and x.flags.c_contiguous and x.shape == (n_unknowns(sys),)
    lib.oracle_aprod2(*_dims(sys), _ptr(vals), _ptr(ao), _ptr(at), _ptr(ins), *_cons_args(c),
                      _ptr(y), _ptr(x))
    return x


def colnorm2(sys):
    """Squared column norms of A (constraint rows included)."""
    lib = _load()
    vals, ao, at, ins = _arrays(sys)
    c2 = np.zeros(n_unknowns(sys))
    lib.oracle_colnorm2(*_dims(sys), _ptr(vals), _ptr(ao), _ptr(at), _ptr(ins),
                        *_cons_args(_cons(sys)), _ptr(c2))
    return c2


def lsqr(sys, b, atol=1e-12, btol=1e-12, conlim=1e12, itnlim=None, scale="colnorm",
         want_var=False, x_ref=None, want_rnorm_hist=False, cov_pairs=None):
    """Paige-Saunders LSQR on A D with de-preconditioning x = D z.

    ``scale`` is "colnorm" (d_j = 1/||A_:,j||, 1 for an empty column), None
    (no scaling) or an explicit array of positive d_j. Returns a dict with
    x, istop, itn, rnorm, arnorm, anorm, acond, xnorm and, if asked for,
    var, err_hist (relative error vs ``x_ref`` per iteration), rnorm_hist and
    cov (the estimate of Sec. 2.2, Eq. 4 for the index pairs ``cov_pairs``,
    an [n, 2] integer array).
    """
    lib = _load()
    vals, ao, at, ins = _arrays(sys)
    n = n_unknowns(sys)
    if itnlim is None:
        itnlim = 20 * n
    b = np.ascontiguousarray(b, dtype=np.float64)
    if isinstance(scale, str):
        assert scale == "colnorm"
        c = np.sqrt(colnorm2(sys))
        d = np.where(c > 0, 1.0 / np.where(c > 0, c, 1.0), 1.0)
    elif scale is None:
        d = None
    else:
        d = np.ascontiguousarray(scale, dtype=np.float64)
    x = np.zeros(n)
    var = np.zeros(n) if want_var else None
    xr = np.ascontiguousarray(x_ref, dtype=np.float64) if x_ref is not None else None
    eh = np.full(itnlim, np.nan) if xr is not None else None
    rh = np.full(itnlim, np.nan) if want_rnorm_hist else None
    out = np.zeros(7)
    opts = np.array([atol, btol, conlim], dtype=np.float64)
    pairs = None
    cov = None
    if cov_pairs is not None:
        pairs = np.ascontiguousarray(cov_pairs, dtype=np.int64).reshape(-1, 2)
        assert ((pairs >= 0) & (pairs < n)).all()
        cov = np.zeros(pairs.shape[0])
    assert b.shape == (n_equations(sys),)
    rc = lib.oracle_lsqr(*_dims(sys), _ptr(vals), _ptr(ao), _ptr(at), _ptr(ins),
                         *_cons_args(_cons(sys)), _ptr(b),
                         _ptr(d), _ptr(opts), int(itnlim), _ptr(x), _ptr(var), _ptr(xr),
                         _ptr(eh), _ptr(rh), int(pairs.shape[0]) if pairs is not None else 0,
                         _ptr(pairs), _ptr(cov), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle_lsqr: allocation failed")
    itn = int(out[1])
    res = dict(x=x, istop=int(out[0]), itn=itn, rnorm=out[2], arnorm=out[3], anorm=out[4],
               acond=out[5], xnorm=out[6], scale=d)
    if want_var:
        res["var"] = var
    if cov is not None:
        res["cov"] = cov
    if eh is not None:
        res["err_hist"] = eh[:itn]
    if rh is not None:
        res["rnorm_hist"] = rh[:itn]
    return res
