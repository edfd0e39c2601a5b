"""Learned column preconditioner: labels from solve histories, BF16 MLP training
on the GPU, evaluation, and the fallback to plain column scaling.

Every numerical step runs in libgsr's kernels (features, MLP forward/gradient,
Adam, the scaling, LSQR); this module only marshals tensors and makes the
host-side decisions (which candidate scaling won, whether the trained model
is used at all).

Method (an extension of the paper's column-norm preconditioning, Sec. 2):
  * each attitude / instrumental column q gets 8 features (gsr_column_features);
  * for a training system, candidate scalings d = gamma_B / ||A_:,j|| with one
    multiplier gamma_B per block B (attitude, instrumental) are scored by the
    solver's own error history: log10 of the relative error at the iteration
    just before column scaling reaches the tolerance (lower is better). A
    coordinate search over log2(gamma) in {-1/2, -1/4, 0, 1/4, 1/2} per block,
    refined by the vertex of a parabola through the best point and its two
    neighbours, gives the label m_q = log(gamma_B*) of every column of block B;
  * the MLP 8 -> 64 -> 64 -> 1 (BF16 weights/activations, FP32 accumulation)
    is fit to the labels by full-batch Adam on the mean squared error;
  * at solve time d_q = exp(m_q) / ||A_:,q|| on the learned columns;
  * the model is used only if, on validation systems it was not trained on,
    it lowers the median iteration count to the tolerance; otherwise (and for
    any caller that disables it) the scaling is plain column scaling.
"""
import math

import numpy as np
import torch

from . import gsr
from . import synth

LOG2_GAMMAS = (-0.5, -0.25, 0.0, 0.25, 0.5)


def iterations_to(err_hist, tol):
    """1-based index of the first iterate with relative error <= tol (None if never)."""
    idx = np.nonzero(np.asarray(err_hist) <= tol)[0]
    return int(idx[0]) + 1 if idx.size else None


def make_rhs(S, sys_):
    """b = A x* + noise through the library's aprod 1 (Eq. 2)."""
    b = torch.as_tensor(np.asarray(sys_["noise"], dtype=np.float64)).to(S.device)
    x = torch.as_tensor(np.asarray(sys_["x_star"], dtype=np.float64)).to(S.device)
    S.aprod1(x, b)
    return b


class SolveProbe:
    """Error histories of LSQR on one system under a given column scaling."""

    def __init__(self, S, b, tol=1e-9, ref_tol=1e-15):
        self.S, self.b, self.tol = S, b, tol
        ref = S.lsqr(b, atol=ref_tol, btol=ref_tol, itnlim=20000)
        self.x_ref = ref["x"].clone()
        base = self.history(S.learned_scaling(None), itnlim=ref["itn"] + 5)
        self.n_colnorm = iterations_to(base, tol)
        if self.n_colnorm is None:
            raise RuntimeError("column-scaled LSQR did not reach %g" % tol)
        # the iterate scored: one before column scaling reaches the tolerance
        self.k_score = max(1, self.n_colnorm - 1)

    def history(self, d, itnlim):
        r = self.S.lsqr(self.b, atol=0.0, btol=0.0, conlim=0.0, itnlim=itnlim,
                        precond="user", scale=d, x_ref=self.x_ref, err_hist=True)
        return r["err_hist"]

    def score(self, d):
        eh = self.history(d, self.k_score)
        return float(np.log10(max(eh[self.k_score - 1], 1e-300)))

    def iterations(self, d, cap_factor=3):
        eh = self.history(d, cap_factor * self.n_colnorm)
        n = iterations_to(eh, self.tol)
        return n if n is not None else cap_factor * self.n_colnorm


def _vertex(xs, ys):
    """Abscissa of the minimum of the parabola through three points (the middle
    one must be the smallest); falls back to the middle point when flat."""
    (x0, x1, x2), (y0, y1, y2) = xs, ys
    den = (x0 - x1) * (x0 - x2) * (x1 - x2)
    a = (x2 * (y1 - y0) + x1 * (y0 - y2) + x0 * (y2 - y1)) / den
    b = (x2 * x2 * (y0 - y1) + x1 * x1 * (y2 - y0) + x0 * x0 * (y1 - y2)) / den
    if a <= 0:
        return x1
    return min(max(-b / (2 * a), x0), x2)


def block_labels(S, probe, log2_gammas=LOG2_GAMMAS):
    """Coordinate search of the per-block multipliers; returns (labels [nq] float32
    tensor, dict with gamma_att, gamma_instr and the scores)."""
    K = S.n_knots
    nq = S.n_learned_cols()
    best = {"att": 0.0, "ins": 0.0}
    table = {}
    for blk in ("att", "ins"):
        ys = []
        for lg in log2_gammas:
            trial = dict(best)
            trial[blk] = lg
            m = torch.empty(nq, dtype=torch.float32, device=S.device)
            m[:3 * K] = trial["att"] * math.log(2.0)
            m[3 * K:] = trial["ins"] * math.log(2.0)
            ys.append(probe.score(S.learned_scaling(m)))
        table[blk] = ys
        i = int(np.argmin(ys))
        if 0 < i < len(ys) - 1:
            best[blk] = _vertex(log2_gammas[i - 1:i + 2], ys[i - 1:i + 2])
        else:
            best[blk] = log2_gammas[i]
    lab = torch.empty(nq, dtype=torch.float32, device=S.device)
    lab[:3 * K] = best["att"] * math.log(2.0)
    lab[3 * K:] = best["ins"] * math.log(2.0)
    return lab, dict(log2_gamma_att=best["att"], log2_gamma_instr=best["ins"], scores=table)


class Model:
    """Parameters (FP32 master copy, device) and feature standardisation."""

    def __init__(self, theta, norm):
        self.theta, self.norm = theta, norm

    def predict(self, feats):
        return gsr.mlp_forward(feats, self.norm, self.theta)

    def state(self):
        return dict(theta=self.theta.cpu().numpy().tolist(), norm=self.norm.cpu().numpy().tolist())


def standardisation(feats_list, device):
    """mean and 1/std of the features over all training rows (moments and the
    standardisation by kernels)."""
    acc = torch.zeros(16, dtype=torch.float64, device=device)
    n = 0
    for f in feats_list:
        gsr.feature_moments(f, acc)
        n += int(f.shape[0])
    return gsr.feature_standardisation(acc, n)


def train(feats_list, labels_list, steps=1500, lr=2e-3, seed=2503, device=None):
    """Full-batch Adam on the MSE between network output and labels; returns
    (Model, loss history)."""
    device = device or feats_list[0].device
    feats = torch.cat(feats_list).contiguous()
    labels = torch.cat(labels_list).contiguous()
    norm = standardisation(feats_list, device)
    theta = torch.tensor(synth.mlp_init_params(seed), dtype=torch.float32, device=device)
    mom = torch.zeros_like(theta)
    vel = torch.zeros_like(theta)
    grad = torch.empty_like(theta)
    work = torch.empty(gsr.MLP_WORK_FLOATS, dtype=torch.float32, device=device)
    loss = torch.empty(1, dtype=torch.float32, device=device)
    hist = torch.empty(steps, dtype=torch.float32, device=device)
    for step in range(1, steps + 1):
        gsr.mlp_grad(feats, labels, norm, theta, work, grad, loss)
        hist[step - 1:step].copy_(loss)
        gsr.mlp_adam(theta, grad, mom, vel, step, lr)
    return Model(theta, norm), hist.cpu().numpy()


class LearnedPreconditioner:
    """A trained model plus the fallback decision."""

    def __init__(self, model, clamp=3.0, enabled=True):
        self.model, self.clamp, self.enabled = model, clamp, enabled
        self.validation = None

    def scaling(self, S):
        """Column scaling for system S: learned if enabled, else plain column scaling."""
        if not self.enabled or self.model is None:
            return S.learned_scaling(None)
        m = self.model.predict(S.column_features())
        return S.learned_scaling(m, clamp=self.clamp)

    def validate(self, pairs):
        """pairs: iterable of (System, SolveProbe). Keeps the model only if it
        lowers the median iterations-to-tolerance over these systems."""
        learned, base = [], []
        was = self.enabled
        self.enabled = True
        for S, probe in pairs:
            learned.append(probe.iterations(self.scaling(S)))
            base.append(probe.n_colnorm)
        self.enabled = was and float(np.median(learned)) < float(np.median(base))
        self.validation = dict(learned=learned, colnorm=base, enabled=self.enabled)
        return self.validation
