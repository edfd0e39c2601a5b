"""Python binding over the C ABI of libgsr (include/gsr.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libgsr.so. Device vectors are torch tensors (float64, contiguous,
on the system's device); the current torch stream is passed to every call.
There is no CPU fallback: if libgsr.so is missing or fails to load, importing
this module raises.
"""
import ctypes
import os

import numpy as np
import torch

from . import build as _build

_c_i64 = ctypes.c_int64
_c_i32 = ctypes.c_int32
_c_dbl = ctypes.c_double
_c_p = ctypes.c_void_p

STATUS = {0: "GSR_OK", 1: "GSR_E_ARG", 2: "GSR_E_INDEX", 3: "GSR_E_UNSORTED",
          4: "GSR_E_NONFINITE", 5: "GSR_E_OOM", 6: "GSR_E_CUDA", 7: "GSR_E_TIMEOUT",
          8: "GSR_E_UNSUPPORTED"}
VALUES_F64, VALUES_F32 = 0, 1
STORE_F64, STORE_F32_PLUS_F64 = 0, 1
PRECOND = {"none": 0, "colnorm": 1, "user": 2}
PRECISION = {"f64": 0, "mixed": 1}


class GsrError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%s)" % (where, STATUS.get(code, code), strerror(code)))


class Dims(ctypes.Structure):
    _fields_ = [("n_rows", _c_i64), ("n_stars", _c_i64), ("n_knots", _c_i64),
                ("n_instr", _c_i64), ("n_glob", _c_i32), ("storage", _c_i32)]


class LsqrOpts(ctypes.Structure):
    _fields_ = [("atol", _c_dbl), ("btol", _c_dbl), ("conlim", _c_dbl), ("itnlim", _c_i64),
                ("precond", _c_i32), ("precision", _c_i32), ("scale", _c_p), ("var", _c_p),
                ("x_ref", _c_p), ("err_hist", _c_p), ("rnorm_hist", _c_p),
                ("mixed_switch_itn", _c_i32), ("profile", _c_i32),
                ("n_cov", _c_i64), ("cov_pairs", _c_p), ("cov", _c_p)]


class LsqrResult(ctypes.Structure):
    _fields_ = [("istop", _c_i32), ("phase2_itn", _c_i32), ("itn", _c_i64), ("rnorm", _c_dbl),
                ("arnorm", _c_dbl), ("anorm", _c_dbl), ("acond", _c_dbl), ("xnorm", _c_dbl),
                ("n_launches", _c_i64), ("n_timed_itn", _c_i64), ("t_aprod1_ms", _c_dbl),
                ("t_aprod2_ms", _c_dbl), ("t_vector_ms", _c_dbl)]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("libgsr.so not built (%s); run paper_2503_22863_b300/build.py or "
                          "__graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    lib.gsr_create.argtypes = [ctypes.POINTER(Dims), _c_p, _c_p, _c_p, _c_p, ctypes.c_int, _c_p,
                               ctypes.POINTER(_c_p)]
    lib.gsr_create.restype = ctypes.c_int
    lib.gsr_destroy.argtypes = [_c_p]
    lib.gsr_destroy.restype = None
    lib.gsr_strerror.argtypes = [ctypes.c_int]
    lib.gsr_strerror.restype = ctypes.c_char_p
    lib.gsr_n_unknowns.argtypes = [_c_p]
    lib.gsr_n_unknowns.restype = _c_i64
    lib.gsr_n_rows.argtypes = [_c_p]
    lib.gsr_n_rows.restype = _c_i64
    lib.gsr_n_equations.argtypes = [_c_p]
    lib.gsr_n_equations.restype = _c_i64
    lib.gsr_set_constraints.argtypes = [_c_p, _c_i64, _c_p, _c_p, _c_p, _c_p]
    lib.gsr_set_constraints.restype = ctypes.c_int
    for name in ("gsr_aprod1", "gsr_aprod2"):
        getattr(lib, name).argtypes = [_c_p, _c_p, _c_p, _c_p]
        getattr(lib, name).restype = ctypes.c_int
    for name in ("gsr_aprod1_values", "gsr_aprod2_values"):
        getattr(lib, name).argtypes = [_c_p, ctypes.c_int, _c_p, _c_p, _c_p]
        getattr(lib, name).restype = ctypes.c_int
    lib.gsr_column_norms.argtypes = [_c_p, _c_p, _c_p]
    lib.gsr_column_norms.restype = ctypes.c_int
    lib.gsr_lsqr_default_opts.argtypes = [ctypes.POINTER(LsqrOpts)]
    lib.gsr_lsqr_default_opts.restype = None
    lib.gsr_lsqr_solve.argtypes = [_c_p, _c_p, _c_p, ctypes.POINTER(LsqrOpts),
                                   ctypes.POINTER(LsqrResult), _c_p]
    lib.gsr_lsqr_solve.restype = ctypes.c_int
    for name in ("gsr_aprod1_batch", "gsr_aprod2_batch"):
        getattr(lib, name).argtypes = [_c_p, ctypes.c_int, _c_p, _c_p, _c_p]
        getattr(lib, name).restype = ctypes.c_int
    lib.gsr_lsqr_solve_batch.argtypes = [_c_p, ctypes.c_int, _c_p, _c_p,
                                         ctypes.POINTER(LsqrOpts), ctypes.POINTER(LsqrResult),
                                         _c_p]
    lib.gsr_lsqr_solve_batch.restype = ctypes.c_int
    lib.gsr_batch_tuning.argtypes = [_c_p, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]
    lib.gsr_batch_tuning.restype = ctypes.c_int
    lib.gsr_n_learned_cols.argtypes = [_c_p]
    lib.gsr_n_learned_cols.restype = _c_i64
    lib.gsr_column_features.argtypes = [_c_p, _c_p, _c_p]
    lib.gsr_feature_moments.argtypes = [_c_p, _c_i64, _c_p, _c_p]
    lib.gsr_feature_standardisation.argtypes = [_c_p, _c_i64, _c_p, _c_p]
    lib.gsr_mlp_forward.argtypes = [_c_p, _c_i64, _c_p, _c_p, _c_p, _c_p]
    lib.gsr_mlp_grad.argtypes = [_c_p, _c_p, _c_i64, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p]
    lib.gsr_mlp_adam.argtypes = [_c_p, _c_p, _c_p, _c_p, _c_i64, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, ctypes.c_float, _c_p]
    lib.gsr_learned_scaling.argtypes = [_c_p, _c_p, ctypes.c_float, _c_p, _c_p]
    for name in ("gsr_column_features", "gsr_feature_moments", "gsr_feature_standardisation",
                 "gsr_mlp_forward", "gsr_mlp_grad", "gsr_mlp_adam", "gsr_learned_scaling"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()


def strerror(code):
    return lib.gsr_strerror(int(code)).decode()


def _check(code, where):
    if code != 0:
        raise GsrError(code, where)


def _stream():
    return _c_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t, n, name, dtype=torch.float64):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError("%s must be a contiguous %s tensor with %d elements" % (name, dtype, n))
    return _c_p(t.data_ptr())


class System:
    """A packed AVU-GSR system resident on one GPU (wraps gsr_create/gsr_destroy)."""

    def __init__(self, sys, device=0, storage="f64"):
        vals = np.ascontiguousarray(sys["vals"], dtype=np.float64)
        ao = np.ascontiguousarray(sys["astro_off"], dtype=np.int64)
        at = np.ascontiguousarray(sys["att_off"], dtype=np.int64)
        ins = np.ascontiguousarray(sys["instr"], dtype=np.int32)
        self.device = torch.device("cuda", device)
        d = Dims(int(sys["n_rows"]), int(sys["n_stars"]), int(sys["n_knots"]),
                 int(sys["n_instr"]), int(sys["n_glob"]),
                 STORE_F32_PLUS_F64 if storage == "f32+f64" else STORE_F64)
        h = _c_p()
        with torch.cuda.device(self.device):
            code = lib.gsr_create(ctypes.byref(d), vals.ctypes.data_as(_c_p),
                                  ao.ctypes.data_as(_c_p), at.ctypes.data_as(_c_p),
                                  ins.ctypes.data_as(_c_p), int(device), _stream(),
                                  ctypes.byref(h))
        _check(code, "gsr_create")
        self._h = h
        self.n_rows = int(lib.gsr_n_rows(h))
        self.n_unk = int(lib.gsr_n_unknowns(h))
        self.n_eq = self.n_rows
        if sys.get("con_ptr") is not None:
            self.set_constraints(sys["con_ptr"], sys["con_col"], sys["con_val"])
        self.n_stars, self.n_knots = int(sys["n_stars"]), int(sys["n_knots"])
        self.n_instr, self.n_glob = int(sys["n_instr"]), int(sys["n_glob"])
        self.storage = storage

    def set_constraints(self, con_ptr, con_col, con_val):
        """Constraint rows in CSR form (host arrays; gsr_set_constraints). Vectors
        over the equations then have n_eq = n_rows + n_con entries."""
        ptr = np.ascontiguousarray(con_ptr, dtype=np.int64)
        col = np.ascontiguousarray(con_col, dtype=np.int64)
        val = np.ascontiguousarray(con_val, dtype=np.float64)
        if ptr.ndim != 1 or ptr.size < 1 or col.shape != val.shape or ptr[-1] != col.size:
            raise ValueError("constraints must be CSR arrays: ptr[n_con + 1], col[nnz], val[nnz]")
        with torch.cuda.device(self.device):
            _check(lib.gsr_set_constraints(self._h, ptr.size - 1, ptr.ctypes.data_as(_c_p),
                                           col.ctypes.data_as(_c_p), val.ctypes.data_as(_c_p),
                                           _stream()), "gsr_set_constraints")
        self.n_eq = int(lib.gsr_n_equations(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib.gsr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def aprod1(self, x, y, values="f64"):
        """Eq. 2: y += A x (in place on the tensor y)."""
        code = lib.gsr_aprod1_values(self._h, VALUES_F32 if values == "f32" else VALUES_F64,
                                     _dptr(x, self.n_unk, "x"), _dptr(y, self.n_eq, "y"),
                                     _stream())
        _check(code, "gsr_aprod1")
        return y

    def aprod2(self, y, x, values="f64"):
        """Eq. 3: x += A^T y (in place on the tensor x)."""
        code = lib.gsr_aprod2_values(self._h, VALUES_F32 if values == "f32" else VALUES_F64,
                                     _dptr(y, self.n_eq, "y"), _dptr(x, self.n_unk, "x"),
                                     _stream())
        _check(code, "gsr_aprod2")
        return x

    def column_norms(self):
        c = torch.empty(self.n_unk, dtype=torch.float64, device=self.device)
        _check(lib.gsr_column_norms(self._h, _c_p(c.data_ptr()), _stream()), "gsr_column_norms")
        return c

    def lsqr(self, b, x=None, atol=1e-12, btol=1e-12, conlim=1e12, itnlim=0, precond="colnorm",
             precision="f64", scale=None, want_var=False, x_ref=None, err_hist=False,
             rnorm_hist=False, mixed_switch_itn=0, profile=False, cov_pairs=None):
        """Preconditioned LSQR (gsr_lsqr_solve). Returns a dict with x and the result fields;
        cov_pairs (a CUDA int64 tensor [n, 2]) adds "cov", the covariance estimates."""
        o = LsqrOpts()
        lib.gsr_lsqr_default_opts(ctypes.byref(o))
        o.atol, o.btol, o.conlim, o.itnlim = atol, btol, conlim, int(itnlim)
        o.precond = PRECOND[precond]
        o.precision = PRECISION[precision]
        o.mixed_switch_itn = int(mixed_switch_itn)
        o.profile = 1 if profile else 0
        if scale is not None:
            o.scale = _dptr(scale, self.n_unk, "scale").value
        var = None
        if want_var:
            var = torch.zeros(self.n_unk, dtype=torch.float64, device=self.device)
            o.var = var.data_ptr()
        if x_ref is not None:
            o.x_ref = _dptr(x_ref, self.n_unk, "x_ref").value
        cov = None
        if cov_pairs is not None:
            if not isinstance(cov_pairs, torch.Tensor) or cov_pairs.dim() != 2 or \
                    cov_pairs.shape[1] != 2:
                raise ValueError("cov_pairs must be a tensor of shape (n, 2)")
            npair = int(cov_pairs.shape[0])
            o.cov_pairs = _dptr(cov_pairs, 2 * npair, "cov_pairs", dtype=torch.int64).value
            cov = torch.zeros(npair, dtype=torch.float64, device=self.device)
            o.n_cov = npair
            o.cov = cov.data_ptr() if npair > 0 else None
        lim = int(itnlim) if itnlim else 20 * max(1, self.n_unk)
        eh = rh = None
        if err_hist:
            if x_ref is None:
                raise ValueError("err_hist needs x_ref")
            eh = np.full(lim, np.nan)
            o.err_hist = eh.ctypes.data
        if rnorm_hist:
            rh = np.full(lim, np.nan)
            o.rnorm_hist = rh.ctypes.data
        if x is None:
            x = torch.empty(self.n_unk, dtype=torch.float64, device=self.device)
        r = LsqrResult()
        code = lib.gsr_lsqr_solve(self._h, _dptr(b, self.n_eq, "b"), _dptr(x, self.n_unk, "x"),
                                  ctypes.byref(o), ctypes.byref(r), _stream())
        _check(code, "gsr_lsqr_solve")
        out = dict(x=x, istop=r.istop, itn=r.itn, phase2_itn=r.phase2_itn, rnorm=r.rnorm,
                   arnorm=r.arnorm, anorm=r.anorm, acond=r.acond, xnorm=r.xnorm,
                   n_launches=r.n_launches, n_timed_itn=r.n_timed_itn,
                   t_aprod1_ms=r.t_aprod1_ms, t_aprod2_ms=r.t_aprod2_ms,
                   t_vector_ms=r.t_vector_ms)
        if var is not None:
            out["var"] = var
        if cov is not None:
            out["cov"] = cov
        if eh is not None:
            out["err_hist"] = eh[:r.itn]
        if rh is not None:
            out["rnorm_hist"] = rh[:r.itn]
        return out


def _dptr2(t, n, k, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != (n, k):
        raise ValueError("%s must be a contiguous float64 tensor of shape (%d, %d)" % (name, n, k))
    return _c_p(t.data_ptr())


def _batch_methods():
    def aprod1_batch(self, X, Y):
        """Eq. 2 for k columns: Y[n_rows, k] += A X[N_unk, k]."""
        k = int(X.shape[1])
        _check(lib.gsr_aprod1_batch(self._h, k, _dptr2(X, self.n_unk, k, "X"),
                                    _dptr2(Y, self.n_eq, k, "Y"), _stream()), "gsr_aprod1_batch")
        return Y

    def aprod2_batch(self, Y, X):
        """Eq. 3 for k columns: X[N_unk, k] += A^T Y[n_rows, k]."""
        k = int(Y.shape[1])
        _check(lib.gsr_aprod2_batch(self._h, k, _dptr2(Y, self.n_eq, k, "Y"),
                                    _dptr2(X, self.n_unk, k, "X"), _stream()), "gsr_aprod2_batch")
        return X

    def lsqr_batch(self, B, X=None, atol=1e-12, btol=1e-12, conlim=1e12, itnlim=0,
                   precond="colnorm", scale=None, x_ref=None, err_hist=False, precision="f64",
                   mixed_switch_itn=0):
        """LSQR on k right-hand sides B[n_rows, k] at once (gsr_lsqr_solve_batch)."""
        k = int(B.shape[1])
        o = LsqrOpts()
        lib.gsr_lsqr_default_opts(ctypes.byref(o))
        o.atol, o.btol, o.conlim, o.itnlim = atol, btol, conlim, int(itnlim)
        o.precond = PRECOND[precond]
        o.precision = PRECISION[precision]
        o.mixed_switch_itn = int(mixed_switch_itn)
        if scale is not None:
            o.scale = _dptr(scale, self.n_unk, "scale").value
        eh = None
        lim = int(itnlim) if itnlim else 20 * max(1, self.n_unk)
        if x_ref is not None:
            o.x_ref = _dptr2(x_ref, self.n_unk, k, "x_ref").value
        if err_hist:
            if x_ref is None:
                raise ValueError("err_hist needs x_ref")
            eh = np.full((lim + 1) * k, np.nan)
            o.err_hist = eh.ctypes.data
        if X is None:
            X = torch.empty((self.n_unk, k), dtype=torch.float64, device=self.device)
        res = (LsqrResult * k)()
        _check(lib.gsr_lsqr_solve_batch(self._h, k, _dptr2(B, self.n_eq, k, "B"),
                                        _dptr2(X, self.n_unk, k, "X"), ctypes.byref(o), res,
                                        _stream()), "gsr_lsqr_solve_batch")
        out = dict(x=X, istop=[r.istop for r in res], itn=[r.itn for r in res],
                   phase2_itn=[r.phase2_itn for r in res],
                   rnorm=[r.rnorm for r in res], anorm=[r.anorm for r in res],
                   iterations=res[0].n_timed_itn, n_launches=res[0].n_launches)
        if eh is not None:
            it = res[0].n_timed_itn
            out["err_hist"] = eh[:it * k].reshape(it, k)
        return out

    def batch_tuning(self):
        t, c = ctypes.c_int(), ctypes.c_int()
        _check(lib.gsr_batch_tuning(self._h, ctypes.byref(t), ctypes.byref(c)), "gsr_batch_tuning")
        return dict(threads=t.value, tile_rows=c.value)

    System.aprod1_batch = aprod1_batch
    System.aprod2_batch = aprod2_batch
    System.lsqr_batch = lsqr_batch
    System.batch_tuning = batch_tuning


_batch_methods()


# ---------------------------------------------------------------------------
# Learned column preconditioner: the MLP kernels (current device, current
# stream). Tensors are float32 CUDA tensors; theta has MLP_NPARAM entries.
# ---------------------------------------------------------------------------
MLP_NFEAT, MLP_HIDDEN, MLP_NPARAM, MLP_GRID = 8, 64, 4801, 296
MLP_WORK_FLOATS = MLP_GRID * (MLP_NPARAM + 1)


def _fptr(t, n, name):
    return _dptr(t, n, name, dtype=torch.float32)


def feature_moments(feats, acc):
    """acc[16] (float64) += column sums of feats and of feats**2."""
    n = int(feats.shape[0])
    _check(lib.gsr_feature_moments(_fptr(feats, n * MLP_NFEAT, "feats"), n,
                                   _dptr(acc, 2 * MLP_NFEAT, "acc"), _stream()),
           "gsr_feature_moments")
    return acc


def feature_standardisation(acc, n, norm=None):
    """norm[16] (float32) = mean, 1/std of n feature rows from their moments acc."""
    if norm is None:
        norm = torch.empty(2 * MLP_NFEAT, dtype=torch.float32, device=acc.device)
    _check(lib.gsr_feature_standardisation(_dptr(acc, 2 * MLP_NFEAT, "acc"), int(n),
                                           _fptr(norm, 2 * MLP_NFEAT, "norm"), _stream()),
           "gsr_feature_standardisation")
    return norm


def mlp_forward(feats, norm, theta, out=None):
    """Network outputs m[n] for raw features feats[n, 8]."""
    n = int(feats.shape[0])
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=feats.device)
    _check(lib.gsr_mlp_forward(_fptr(feats, n * MLP_NFEAT, "feats"), n,
                               _fptr(norm, 2 * MLP_NFEAT, "norm"), _fptr(theta, MLP_NPARAM, "theta"),
                               _fptr(out, n, "out"), _stream()), "gsr_mlp_forward")
    return out


def mlp_grad(feats, target, norm, theta, work, grad, loss=None):
    """grad = dL/dtheta of the mean squared error; loss[1] = L if given."""
    n = int(feats.shape[0])
    _check(lib.gsr_mlp_grad(_fptr(feats, n * MLP_NFEAT, "feats"), _fptr(target, n, "target"), n,
                            _fptr(norm, 2 * MLP_NFEAT, "norm"), _fptr(theta, MLP_NPARAM, "theta"),
                            _fptr(work, MLP_WORK_FLOATS, "work"), _fptr(grad, MLP_NPARAM, "grad"),
                            _fptr(loss, 1, "loss") if loss is not None else None, _stream()),
           "gsr_mlp_grad")
    return grad


def mlp_adam(theta, grad, mom, vel, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step on theta (in place)."""
    _check(lib.gsr_mlp_adam(_fptr(theta, MLP_NPARAM, "theta"), _fptr(grad, MLP_NPARAM, "grad"),
                            _fptr(mom, MLP_NPARAM, "mom"), _fptr(vel, MLP_NPARAM, "vel"), int(step),
                            lr, beta1, beta2, eps, _stream()), "gsr_mlp_adam")
    return theta


def _learned_methods():
    def n_learned_cols(self):
        return int(lib.gsr_n_learned_cols(self._h))

    def column_features(self):
        """Features [3K + n_instr, 8] (float32) of the attitude + instrumental columns."""
        nq = self.n_learned_cols()
        f = torch.empty((nq, MLP_NFEAT), dtype=torch.float32, device=self.device)
        _check(lib.gsr_column_features(self._h, _fptr(f, nq * MLP_NFEAT, "feats"), _stream()),
               "gsr_column_features")
        return f

    def learned_scaling(self, m=None, clamp=3.0):
        """Column scaling d [N_unk] (float64): exp(m_q) / ||A_:,j|| on the learned columns."""
        d = torch.empty(self.n_unk, dtype=torch.float64, device=self.device)
        mp = _fptr(m, self.n_learned_cols(), "m") if m is not None else None
        _check(lib.gsr_learned_scaling(self._h, mp, float(clamp), _c_p(d.data_ptr()), _stream()),
               "gsr_learned_scaling")
        return d

    System.n_learned_cols = n_learned_cols
    System.column_features = column_features
    System.learned_scaling = learned_scaling


_learned_methods()
