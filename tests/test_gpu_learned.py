"""GPU parity of the learned column preconditioner against the CPU oracle.

Features against oracle/mlp.column_features; the BF16 tensor-core MLP forward
pass and gradient against the oracle network with BF16 rounding at the same
points (the remaining differences come from FP32 accumulation order and the
occasional BF16 rounding it flips); Adam against the FP64 update; the scaling
against its definition; the LSQR answer unchanged under a learned scaling;
the fallback equal to plain column scaling; and a small end-to-end training
run that reports what the model gains over column scaling."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as omlp
from paper_2503_22863_b300 import synth
from gpu_util import LSQR_TOL, rhs, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsr():
    from paper_2503_22863_b300 import gsr as g
    return g


def f32(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def standardised(feats, norm):
    """What the kernels feed the first layer: (f - mean) * (1/std) with FP32 inputs."""
    f = np.asarray(feats, dtype=np.float32).astype(np.float64)
    nrm = np.asarray(norm, dtype=np.float32).astype(np.float64)
    return (f - nrm[:8]) * nrm[8:]


def make_inputs(seed, n):
    rng = np.random.default_rng(seed)
    feats = (rng.standard_normal((n, 8)) * 2.0 + 1.0).astype(np.float32)
    norm = np.concatenate([rng.standard_normal(8) * 0.5, 0.5 + rng.random(8)]).astype(np.float32)
    theta = synth.mlp_init_params(seed).astype(np.float32)
    theta[512:576] = (rng.standard_normal(64) * 0.1).astype(np.float32)   # b1
    theta[4672:4736] = (rng.standard_normal(64) * 0.1).astype(np.float32)  # b2
    theta[4800] = 0.2
    t = (rng.standard_normal(n) * 0.3).astype(np.float32)
    return feats, norm, theta, t


@pytest.mark.parametrize("seed,n", [(1, 1), (2, 15), (3, 64), (4, 1000), (5, 4103)])
def test_mlp_forward_parity(gsr, seed, n):
    feats, norm, theta, _ = make_inputs(seed, n)
    m = gsr.mlp_forward(f32(feats), f32(norm), f32(theta)).cpu().numpy()
    ref, _ = omlp.forward(theta.astype(np.float64), standardised(feats, norm), bf16=True)
    scale = np.abs(ref).max() + 1e-30
    assert np.abs(m - ref).max() <= 5e-3 * scale, np.abs(m - ref).max() / scale
    # the bulk agrees to FP32 accumulation order
    assert np.median(np.abs(m - ref)) <= 1e-5 * scale


@pytest.mark.parametrize("seed,n", [(6, 7), (7, 64), (8, 3000), (9, 70001)])
def test_mlp_grad_parity(gsr, seed, n):
    feats, norm, theta, t = make_inputs(seed, n)
    work = torch.empty(gsr.MLP_WORK_FLOATS, dtype=torch.float32, device="cuda")
    grad = torch.empty(gsr.MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    gsr.mlp_grad(f32(feats), f32(t), f32(norm), f32(theta), work, grad, loss)
    g = grad.cpu().numpy().astype(np.float64)
    x = standardised(feats, norm)
    ref = omlp.grad(theta.astype(np.float64), x, t.astype(np.float64), bf16=True)
    L = omlp.loss(theta.astype(np.float64), x, t.astype(np.float64), bf16=True)
    assert abs(float(loss.item()) - L) <= 1e-4 * L
    for name, sl in [("W1", slice(0, 512)), ("b1", slice(512, 576)), ("W2", slice(576, 4672)),
                     ("b2", slice(4672, 4736)), ("w3", slice(4736, 4800)),
                     ("b3", slice(4800, 4801))]:
        d = np.linalg.norm(g[sl] - ref[sl])
        assert d <= 2e-2 * np.linalg.norm(ref[sl]) + 1e-12, (name, d, np.linalg.norm(ref[sl]))
    # deterministic: same inputs, same bits
    grad2 = torch.empty_like(grad)
    gsr.mlp_grad(f32(feats), f32(t), f32(norm), f32(theta), work, grad2, None)
    assert torch.equal(grad, grad2)


def test_adam_parity(gsr):
    rng = np.random.default_rng(10)
    th = rng.standard_normal(gsr.MLP_NPARAM).astype(np.float32)
    mo = np.zeros(gsr.MLP_NPARAM, dtype=np.float32)
    ve = np.zeros(gsr.MLP_NPARAM, dtype=np.float32)
    T, M, V = f32(th), f32(mo), f32(ve)
    ref = (th.astype(np.float64), mo.astype(np.float64), ve.astype(np.float64))
    for step in range(1, 4):
        g = rng.standard_normal(gsr.MLP_NPARAM).astype(np.float32)
        gsr.mlp_adam(T, f32(g), M, V, step, 1e-2)
        ref = omlp.adam_step(ref[0], g.astype(np.float64), ref[1], ref[2], step, 1e-2)
    assert np.abs(T.cpu().numpy() - ref[0]).max() <= 1e-5
    assert np.abs(M.cpu().numpy() - ref[1]).max() <= 1e-6


@pytest.mark.parametrize("cfg", [
    dict(n_stars=300, n_knots=40, n_instr=30, n_glob=1, obs=12, poisson=True, seed=31),
    dict(n_stars=2000, n_knots=1000, n_instr=500, n_glob=0, obs=50, poisson=False, seed=32),
])
def test_column_features_parity(gsr, cfg):
    sys = synth.make_system(**cfg)
    ref = omlp.column_features(sys)
    with gsr.System(sys) as S:
        f = S.column_features().cpu().numpy().astype(np.float64)
    assert f.shape == ref.shape
    assert np.abs(f - ref).max() <= 2e-6 * (1 + np.abs(ref).max())
    # counts are integers: exp of feature 1 recovers them exactly (after rounding)
    assert np.array_equal(np.rint(np.expm1(f[:, 1].astype(np.float64))),
                          np.rint(np.expm1(ref[:, 1])))


def test_learned_scaling_definition(gsr):
    sys = synth.make_config("tiny")
    c = np.sqrt(oracle.colnorm2(sys))
    with gsr.System(sys) as S:
        nq = S.n_learned_cols()
        rng = np.random.default_rng(12)
        m = rng.standard_normal(nq).astype(np.float32) * 2.0
        d = to_host(S.learned_scaling(f32(m), clamp=1.5))
        d0 = to_host(S.learned_scaling(None))
    q0 = 5 * sys["n_stars"]
    want = np.where(c > 0, 1.0 / np.where(c > 0, c, 1.0), 1.0)
    assert np.allclose(d0, want, rtol=1e-12, atol=0)
    want2 = want.copy()
    want2[q0:q0 + nq] = np.exp(np.clip(m.astype(np.float64), -1.5, 1.5)) / c[q0:q0 + nq]
    assert np.allclose(d, want2, rtol=1e-12, atol=0)


def test_solution_unchanged_under_learned_scaling(gsr):
    sys = synth.make_config("tiny")
    b = rhs(sys)
    ref = oracle.lsqr(sys, b, atol=1e-14, btol=1e-14)
    with gsr.System(sys) as S:
        rng = np.random.default_rng(13)
        m = (rng.standard_normal(S.n_learned_cols()) * 0.5).astype(np.float32)
        d = S.learned_scaling(f32(m))
        r = S.lsqr(to_dev(b), atol=1e-14, btol=1e-14, precond="user", scale=d)
    assert relerr(to_host(r["x"]), ref["x"]) <= LSQR_TOL


def _family(n, seed0):
    """Small systems shaped like the learned-preconditioner family (obs/star,
    attitude knots and instrumental columns varied log-uniformly)."""
    out = []
    for s in range(n):
        g = np.random.default_rng(seed0 + s)
        K = int(round(math.exp(g.uniform(math.log(200), math.log(2000)))))
        ni = int(round(math.exp(g.uniform(math.log(20), math.log(200)))))
        out.append(synth.make_system(n_stars=6000, n_knots=K, n_instr=ni, n_glob=1, obs=30,
                                     poisson=True, seed=seed0 + s))
    return out


def test_train_and_fallback_end_to_end(gsr):
    from paper_2503_22863_b300 import learned
    systems = _family(6, 4100)
    feats, labels, probes = [], [], []
    handles = []
    for sys_ in systems:
        S = gsr.System(sys_)
        handles.append(S)
        b = learned.make_rhs(S, sys_)
        p = learned.SolveProbe(S, b)
        lab, info = learned.block_labels(S, p)
        assert abs(info["log2_gamma_att"]) <= 0.5 and abs(info["log2_gamma_instr"]) <= 0.5
        feats.append(S.column_features())
        labels.append(lab)
        probes.append(p)
    model, hist = learned.train(feats[:4], labels[:4], steps=300, lr=3e-3)
    assert hist[-1] < hist[0] and np.isfinite(hist).all()
    pre = learned.LearnedPreconditioner(model)
    val = pre.validate(list(zip(handles[4:], probes[4:])))
    # the gate keeps the model only if it cuts the median iteration count
    assert pre.enabled == (np.median(val["learned"]) < np.median(val["colnorm"]))
    # fallback: plain column scaling, the same iteration count as COLNORM
    pre.enabled = False
    for S, p in zip(handles[4:], probes[4:]):
        assert p.iterations(pre.scaling(S)) == p.n_colnorm
    # whatever scaling is used, the answer is the least-squares solution
    pre.enabled = True
    S, p = handles[5], probes[5]
    r = S.lsqr(p.b, atol=1e-14, btol=1e-14, precond="user", scale=pre.scaling(S))
    assert relerr(to_host(r["x"]), to_host(p.x_ref)) <= LSQR_TOL
    for S in handles:
        S.close()


def test_feature_standardisation_kernel():
    """mean and 1/std of the features (moments kernel + standardisation kernel)
    against numpy's, a constant feature getting 1/std = 1."""
    from paper_2503_22863_b300 import gsr
    rng = np.random.default_rng(12)
    f = (rng.standard_normal((5000, 8)) * np.arange(1, 9) + np.arange(8)).astype(np.float32)
    f[:, 3] = 2.5
    parts = [torch.from_numpy(f[:1200]).cuda(), torch.from_numpy(f[1200:]).cuda()]
    acc = torch.zeros(16, dtype=torch.float64, device="cuda")
    for p in parts:
        gsr.feature_moments(p.contiguous(), acc)
    norm = gsr.feature_standardisation(acc, f.shape[0]).cpu().numpy()
    fd = f.astype(np.float64)
    mean = fd.mean(axis=0)
    std = fd.std(axis=0)
    np.testing.assert_allclose(norm[:8], mean, rtol=1e-6, atol=1e-6)
    istd = np.where(std > 1e-6, 1.0 / np.where(std > 1e-6, std, 1.0), 1.0)
    np.testing.assert_allclose(norm[8:], istd, rtol=1e-5)
    assert norm[8 + 3] == 1.0
