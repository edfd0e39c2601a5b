"""Helpers shared by the GPU parity tests (tolerances and oracle-side references)."""
import numpy as np
import torch

import oracle

# Parity tolerances: aprod 1e-12 in the infinity norm scaled by |A||x|
# (resp. |A|^T|y|); LSQR solutions 1e-9 relative in the 2-norm.
APROD_TOL = 1e-12
LSQR_TOL = 1e-9


def abs_system(sys):
    """|A| (constraint rows included) for the accuracy scale |A||x|."""
    out = dict(sys, vals=np.abs(sys["vals"]))
    if sys.get("con_val") is not None:
        out["con_val"] = np.abs(sys["con_val"])
    return out


def aprod1_ref(sys, x, y0):
    """(y0 + A x, |y0| + |A||x|) from the oracle."""
    y = np.array(y0, dtype=np.float64, copy=True)
    oracle.aprod1(sys, x, y)
    s = np.abs(np.asarray(y0, dtype=np.float64)).copy()
    oracle.aprod1(abs_system(sys), np.abs(x), s)
    return y, s


def aprod2_ref(sys, y, x0):
    x = np.array(x0, dtype=np.float64, copy=True)
    oracle.aprod2(sys, y, x)
    s = np.abs(np.asarray(x0, dtype=np.float64)).copy()
    oracle.aprod2(abs_system(sys), np.abs(y), s)
    return x, s


def scaled_err(got, ref, scale):
    """max_i |got - ref| / max_i scale_i (the aprod accuracy measure)."""
    den = float(np.max(scale)) if scale.size else 1.0
    if den == 0.0:
        den = 1.0
    return float(np.max(np.abs(got - ref))) / den if got.size else 0.0


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def to_host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rhs(sys):
    b = np.zeros(sys["n_rows"])
    oracle.aprod1(sys, sys["x_star"], b)
    noise = sys["noise"]
    if noise.ndim == 2:
        noise = noise[:, 0]
    return b + noise
