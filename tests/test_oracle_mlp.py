"""CPU pins of the learned-preconditioner oracle (oracle/mlp.py).

The network gradient is pinned by central finite differences of the FP64
loss, BF16 rounding by hand-worked ties and exact values, Adam by its
closed-form first step, and the column features by brute force over the rows
of small systems."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2503_22863_b300 import synth
from dense_ref import dense as dense_matrix


def test_bf16_round_hand_values():
    # BF16 keeps 8 significant bits: the spacing just above 1 is 2^-7.
    u = 2.0 ** -7
    cases = [
        (1.0, 1.0),
        (1.0 + u / 2, 1.0),                   # tie -> even (1.0)
        (1.0 + 3 * u / 2, 1.0 + 2 * u),        # tie -> even (mantissa 2)
        (1.0 + u / 2 + 2.0 ** -20, 1.0 + u),  # just above the tie
        (-(1.0 + 3 * u / 2), -(1.0 + 2 * u)),
        (3.0, 3.0),
        (0.0, 0.0),
        (2.0 ** -130, 2.0 ** -130),           # FP32 subnormal, exact in BF16
    ]
    for x, want in cases:
        assert mlp.bf16_round(np.array([x]))[0] == want, x
    # BF16 values are fixed points; every rounding is within half a spacing
    rng = np.random.default_rng(0)
    x = rng.standard_normal(10000) * 10.0
    r = mlp.bf16_round(x)
    assert np.array_equal(mlp.bf16_round(r), r)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 * (1 + 1e-12))


def _problem(seed, n=37):
    rng = np.random.default_rng(seed)
    theta = synth.mlp_init_params(seed)
    theta[mlp.N_H * mlp.N_IN:mlp.N_H * mlp.N_IN + mlp.N_H] = rng.standard_normal(mlp.N_H) * 0.1
    f = rng.standard_normal((n, mlp.N_IN))
    t = rng.standard_normal(n) * 0.3
    return theta, f, t


def test_grad_matches_finite_differences():
    theta, f, t = _problem(1)
    g = mlp.grad(theta, f, t)
    rng = np.random.default_rng(2)
    # every bias and the output layer, plus random weights of W1 and W2
    idx = np.concatenate([np.arange(512, 576), np.arange(4672, 4801),
                          rng.choice(512, 40, replace=False),
                          576 + rng.choice(4096, 60, replace=False)])
    h = 1e-6
    for i in idx:
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, f, t) - mlp.loss(tm, f, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_grad_is_zero_at_exact_fit():
    theta, f, _ = _problem(3)
    m, _ = mlp.forward(theta, f)
    assert np.abs(mlp.grad(theta, f, m)).max() == 0.0


def test_bf16_mode_close_to_exact():
    theta, f, t = _problem(4, n=500)
    m64, _ = mlp.forward(theta, f)
    m16, _ = mlp.forward(theta, f, bf16=True)
    assert np.abs(m16 - m64).max() <= 0.05 * np.abs(m64).max()
    g64 = mlp.grad(theta, f, t)
    g16 = mlp.grad(theta, f, t, bf16=True)
    assert np.linalg.norm(g16 - g64) <= 0.05 * np.linalg.norm(g64)


def test_adam_first_step_closed_form():
    # step 1: bias-corrected moments are g and g^2, so the update is
    # -lr * g / (|g| + eps)
    rng = np.random.default_rng(5)
    th = rng.standard_normal(mlp.N_PARAMS)
    g = rng.standard_normal(mlp.N_PARAMS)
    z = np.zeros(mlp.N_PARAMS)
    th1, m1, v1 = mlp.adam_step(th, g, z, z, 1, 1e-3)
    assert np.allclose(th1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    # step 2 by hand
    g2 = rng.standard_normal(mlp.N_PARAMS)
    th2, m2, v2 = mlp.adam_step(th1, g2, m1, v1, 2, 1e-3)
    mh = (0.9 * 0.1 * g + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g * g + 0.001 * g2 * g2) / (1 - 0.999 ** 2)
    assert np.allclose(th2, th1 - 1e-3 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-12, atol=1e-15)


def test_training_loop_fits_a_simple_map():
    # Adam + gradient together drive the loss down on a learnable target
    rng = np.random.default_rng(6)
    f = rng.standard_normal((256, mlp.N_IN))
    t = 0.5 * f[:, 0] - 0.25 * np.abs(f[:, 1])
    th = synth.mlp_init_params(6)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    l0 = mlp.loss(th, f, t)
    for step in range(1, 301):
        th, m, v = mlp.adam_step(th, mlp.grad(th, f, t), m, v, step, 3e-3)
    assert mlp.loss(th, f, t) < 0.05 * l0


def _features_brute(sys):
    """Counts and norms from an explicit dense A, positions by their definition."""
    A = dense_matrix(sys)
    K, ni, ns = sys["n_knots"], sys["n_instr"], sys["n_stars"]
    n_rows = A.shape[0]
    cols = range(5 * ns, 5 * ns + 3 * K + ni)
    out = []
    s = np.asarray(sys["att_off"]) - 5 * ns
    for q, j in enumerate(cols):
        if q < 3 * K:
            kn = q % K
            n = sum(1 for i in range(n_rows) if s[i] <= kn <= s[i] + 3)
            pos, axis, ins, mean = kn / (K - 1), (q // K) / 2, 0.0, 4.0 * n_rows / K
        else:
            i_ = q - 3 * K
            n = sum(1 for i in range(n_rows) if i_ in sys["instr"][i])
            pos, axis, ins, mean = i_ / (ni - 1), 0.0, 1.0, 6.0 * n_rows / ni
        c = np.sqrt(np.sum(A[:, j] ** 2))
        lc = np.log(c) if c > 0 else 0.0
        out.append([lc, np.log1p(n), ins, axis, pos, np.log(mean), np.log1p(n) - np.log1p(mean),
                    lc - 0.5 * np.log(max(n, 1))])
    return np.array(out)


@pytest.mark.parametrize("seed", [11, 12])
def test_column_features_brute_force(seed):
    sys = synth.make_system(n_stars=12, n_knots=9, n_instr=8, n_glob=1, obs=6, poisson=False,
                            seed=seed)
    f = mlp.column_features(sys)
    assert f.shape == (3 * 9 + 8, 8)
    assert np.allclose(f, _features_brute(sys), rtol=0, atol=1e-12)


def test_column_features_edge_knots():
    # every row starts at knot 0 of a 5-knot axis: knots 0..3 are covered by
    # all rows, knot 4 by none (zero column: log-norm feature 0)
    sys = synth.make_system(n_stars=3, n_knots=5, n_instr=6, n_glob=0, obs=7, poisson=False,
                            seed=13)
    sys["att_off"][:] = 5 * 3
    f = mlp.column_features(sys)
    n = 21
    for a in range(3):
        assert np.allclose(f[a * 5:a * 5 + 4, 1], np.log1p(n))
        assert f[a * 5 + 4, 1] == 0.0 and f[a * 5 + 4, 0] == 0.0
    # 6 instrumental columns and 6 distinct per row: every row touches all
    assert np.allclose(f[15:, 1], np.log1p(n))
    assert np.allclose(f[15:, 4], np.arange(6) / 5)
