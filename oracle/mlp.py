"""FP64 CPU oracle of the learned column preconditioner (test infrastructure only).

The network is the one the CUDA library trains and evaluates:

    h1 = relu(W1 f + b1)      W1: 64 x 8
    h2 = relu(W2 h1 + b2)     W2: 64 x 64
    m  = w3 . h2 + b3         w3: 64

mapping the standardised features f of an attitude or instrumental column to
a log multiplier m of its column scaling, d_j = exp(m_j) / ||A_:,j||. The loss
is the mean squared error against the labels t, L = (1/n) sum_i (m_i - t_i)^2,
and the optimiser is Adam (Kingma & Ba, 2015, Algorithm 1).

With ``bf16=True`` every value the CUDA kernels hold in BF16 is rounded to
BF16 here at the same point (inputs, weights, h1, h2 and the activation
gradients dz2, dz1; round-to-nearest-even from FP32); all sums stay FP64, so
the two sides differ only by the FP32 accumulation order of the kernels and
by the rare BF16 rounding decision that order flips. With ``bf16=False`` it is
the exact FP64 network, pinned by central finite differences of ``loss``.

Parameter vector layout (shared with the library's ABI description, not its
code): W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3.
"""
import numpy as np

N_IN, N_H = 8, 64
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("w3", (N_H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    """Split the flat parameter vector into named arrays (views)."""
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[n], dtype=np.float64).ravel() for n, _ in SHAPES])


def bf16_round(a):
    """Round to the nearest BF16 (ties to even) through FP32, returned as FP64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    finite = np.isfinite(f)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    r = np.where(finite, r, u & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _r(a, on):
    return bf16_round(a) if on else a


def forward(theta, f, bf16=False):
    """Network output m[n] for standardised features f[n][8]; also the
    activations (f, h1, h2) the backward pass uses."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    W1, W2, w3 = _r(p["W1"], bf16), _r(p["W2"], bf16), _r(p["w3"], bf16)
    x = _r(np.asarray(f, dtype=np.float64), bf16)
    h1 = _r(np.maximum(x @ W1.T + p["b1"], 0.0), bf16)
    h2 = _r(np.maximum(h1 @ W2.T + p["b2"], 0.0), bf16)
    m = h2 @ w3 + p["b3"][0]
    return m, (x, h1, h2)


def loss(theta, f, t, bf16=False):
    m, _ = forward(theta, f, bf16)
    return float(np.mean((m - np.asarray(t, dtype=np.float64)) ** 2))


def grad(theta, f, t, bf16=False):
    """Gradient of ``loss`` by the chain rule through the three layers."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    W2, w3 = _r(p["W2"], bf16), _r(p["w3"], bf16)
    m, (x, h1, h2) = forward(theta, f, bf16)
    n = len(m)
    g = 2.0 * (m - np.asarray(t, dtype=np.float64)) / n          # dL/dm
    dz2 = _r(np.outer(g, w3) * (h2 > 0), bf16)                   # dL/dz2
    dz1 = _r((dz2 @ W2) * (h1 > 0), bf16)                        # dL/dz1
    return pack({"W1": dz1.T @ x, "b1": dz1.sum(0), "W2": dz2.T @ h1, "b2": dz2.sum(0),
                 "w3": h2.T @ g, "b3": np.array([g.sum()])})


def adam_step(theta, gr, mom, vel, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments); ``step`` counts from 1.
    Returns new (theta, mom, vel)."""
    mom = beta1 * mom + (1.0 - beta1) * gr
    vel = beta2 * vel + (1.0 - beta2) * gr * gr
    mh = mom / (1.0 - beta1 ** step)
    vh = vel / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), mom, vel


def column_features(sys):
    """Features [3K + n_instr, 8] of the attitude and instrumental columns, from
    their definitions: with n_q the number of rows having a coefficient slot in
    column q (a row with start knot s covers knots s..s+3 of every axis and its
    6 instrumental columns) and c_q the column norm,
      0 log c_q      1 log(1+n_q)    2 instrumental flag   3 axis / 2
      4 knot / (K-1) or instrument / (n_instr-1)           5 log(block mean count)
      6 log(1+n_q) - log(1+block mean count)               7 log c_q - log(max(n_q,1)) / 2
    Block mean counts: 4 n_rows / K (attitude), 6 n_rows / n_instr (instrumental)."""
    from .core import colnorm2
    K, ni, ns = int(sys["n_knots"]), int(sys["n_instr"]), int(sys["n_stars"])
    n_rows = len(sys["astro_off"])
    s = np.asarray(sys["att_off"], dtype=np.int64) - 5 * ns
    cnt_att = np.bincount(np.concatenate([s + o for o in range(4)]), minlength=K)[:K]
    cnt_ins = np.bincount(np.asarray(sys["instr"]).ravel(), minlength=ni)[:ni]
    c = np.sqrt(colnorm2(sys))[5 * ns:5 * ns + 3 * K + ni]
    n = np.concatenate([np.tile(cnt_att, 3), cnt_ins]).astype(np.float64)
    ins = np.concatenate([np.zeros(3 * K), np.ones(ni)])
    axis = np.concatenate([np.repeat([0.0, 0.5, 1.0], K), np.zeros(ni)])
    pos = np.concatenate([np.tile(np.arange(K) / max(K - 1, 1), 3),
                          np.arange(ni) / max(ni - 1, 1)])
    mean = np.concatenate([np.full(3 * K, 4.0 * n_rows / K), np.full(ni, 6.0 * n_rows / ni)])
    lc = np.where(c > 0, np.log(np.where(c > 0, c, 1.0)), 0.0)
    f = np.stack([lc, np.log1p(n), ins, axis, pos, np.log(mean), np.log1p(n) - np.log1p(mean),
                  lc - 0.5 * np.log(np.maximum(n, 1.0))], axis=1)
    return f
