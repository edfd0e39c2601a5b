"""Seeded synthetic AVU-GSR systems (shared by the tests, the benchmark and the oracle checks).

This module only draws random numbers and lays them out in the packed row
format; it performs none of the method's arithmetic (no products with A).
The right-hand side b = A x* + noise is formed by whichever side needs it,
from the x* and noise drawn here.

Row format (Sec. 2: at most 24 coefficients per row; 5 astrometric, 12
attitude, 6 instrumental, 1 global):
  vals      float64 [n_rows, 24]  slot order: astro 0..4 | att axis0 t0..3,
                                  axis1 t0..3, axis2 t0..3 | instr 0..5 | glob
  astro_off int64   [n_rows]      5 * star(i), rows sorted by star
  att_off   int64   [n_rows]      5 * n_stars + s_i, s_i uniform on [0, K-4]
  instr     int32   [n_rows, 6]   6 distinct uniform columns of [0, n_instr), sorted
Column layout of x: [astro 5*n_stars | att 3*K | instr n_instr | glob n_glob].

The recipe stands in for the paper's own synthetic generator (Sec. 3): values
N(0,1), obs per star max(Poisson(lambda), 5) (or fixed), x* ~ N(0,1),
noise N(0, sigma^2).
"""
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

NSLOT = 24
CHUNK_ROWS = 1 << 20

# The benchmark workloads (sizes from the paper-shaped configurations).
CONFIGS = {
    "tiny": dict(n_stars=2000, obs=50, poisson=False, n_knots=1000, n_instr=500, n_glob=1,
                 seed=2503),
    "medium": dict(n_stars=1_000_000, obs=30, poisson=True, n_knots=50_000, n_instr=5_000,
                   n_glob=1, seed=2504),
    "large": dict(n_stars=4_000_000, obs=40, poisson=True, n_knots=200_000, n_instr=20_000,
                  n_glob=1, seed=2505),
    # profiling case: the medium shape at 1/10 of the rows (~1 GB on the device,
    # still well above the 126 MB L2)
    "small": dict(n_stars=100_000, obs=30, poisson=True, n_knots=20_000, n_instr=2_000,
                  n_glob=1, seed=2510),
    # profiling case: the large shape (200,000 knots, 20,000 instrumental columns)
    # at 300,000 stars (~12M rows, ~2.6 GB of records)
    "large_small": dict(n_stars=300_000, obs=40, poisson=True, n_knots=200_000,
                        n_instr=20_000, n_glob=1, seed=2511),
}
NOISE_SIGMA = 1e-3


def n_unknowns(n_stars, n_knots, n_instr, n_glob):
    return 5 * n_stars + 3 * n_knots + n_instr + n_glob


def _draw_instr(rng, n, n_instr):
    if n_instr < 6:
        raise ValueError("n_instr must be >= 6 (6 distinct instrumental columns per row)")
    if n_instr <= 64:
        keys = rng.random((n, n_instr))
        idx = np.argsort(keys, axis=1)[:, :6]
    else:
        idx = rng.integers(0, n_instr, size=(n, 6))
        while True:
            idx.sort(axis=1)
            bad = np.nonzero((idx[:, 1:] == idx[:, :-1]).any(axis=1))[0]
            if bad.size == 0:
                break
            idx[bad] = rng.integers(0, n_instr, size=(bad.size, 6))
    idx = np.sort(idx, axis=1)
    return idx.astype(np.int32)


def make_system(n_stars, n_knots, n_instr, n_glob=1, obs=30, poisson=True, min_obs=5, seed=0,
                noise_sigma=NOISE_SIGMA, n_rhs=1, threads=None, counts=None, x_star="normal"):
    """Draw one system. Returns a dict with the packed arrays, x_star and noise.

    counts: optional explicit observations per star (overrides obs/poisson).
    x_star: "normal" (N(0,1)) or "ones" (the all-ones planted solution).
    n_rhs:  number of independent noise vectors (noise has shape [n_rows] or [n_rows, n_rhs]).
    """
    if n_knots < 4:
        raise ValueError("n_knots must be >= 4 (4 consecutive spline knots per axis)")
    if n_glob not in (0, 1):
        raise ValueError("n_glob must be 0 or 1")
    ss = np.random.SeedSequence(seed)
    s_counts, s_rows, s_x, s_noise = ss.spawn(4)
    if counts is None:
        rng = np.random.Generator(np.random.PCG64(s_counts))
        if poisson:
            counts = np.maximum(rng.poisson(obs, n_stars), min_obs)
        else:
            counts = np.full(n_stars, obs)
    counts = np.asarray(counts, dtype=np.int64)
    assert counts.shape == (n_stars,) and (counts >= 0).all()
    n_rows = int(counts.sum())
    n_unk = n_unknowns(n_stars, n_knots, n_instr, n_glob)

    vals = np.empty((n_rows, NSLOT), dtype=np.float64)
    att_off = np.empty(n_rows, dtype=np.int64)
    instr = np.empty((n_rows, 6), dtype=np.int32)
    astro_off = np.repeat(np.arange(n_stars, dtype=np.int64) * 5, counts)

    n_chunks = max(1, (n_rows + CHUNK_ROWS - 1) // CHUNK_ROWS)
    seeds = s_rows.spawn(n_chunks)

    def work(c):
        r0 = c * CHUNK_ROWS
        r1 = min(n_rows, r0 + CHUNK_ROWS)
        if r1 <= r0:
            return
        g = np.random.Generator(np.random.PCG64(seeds[c]))
        g.standard_normal(out=vals[r0:r1])
        if n_glob == 0:
            vals[r0:r1, 23] = 0.0
        att_off[r0:r1] = 5 * n_stars + g.integers(0, n_knots - 3, size=r1 - r0)
        instr[r0:r1] = _draw_instr(g, r1 - r0, n_instr)

    nt = threads or min(16, os.cpu_count() or 1)
    if n_chunks == 1 or nt == 1:
        for c in range(n_chunks):
            work(c)
    else:
        with ThreadPoolExecutor(nt) as ex:
            list(ex.map(work, range(n_chunks)))

    gx = np.random.Generator(np.random.PCG64(s_x))
    xs = np.ones(n_unk) if x_star == "ones" else gx.standard_normal(n_unk)
    gn = np.random.Generator(np.random.PCG64(s_noise))
    shape = (n_rows,) if n_rhs == 1 else (n_rows, n_rhs)
    noise = gn.standard_normal(shape) * noise_sigma
    return dict(n_rows=n_rows, n_stars=n_stars, n_knots=n_knots, n_instr=n_instr, n_glob=n_glob,
                n_unk=n_unk, vals=vals, astro_off=astro_off, att_off=att_off, instr=instr,
                x_star=xs, noise=noise, counts=counts, seed=seed)


def make_config(name, n_rhs=1, threads=None):
    """One of the named workloads ("tiny", "medium", "large")."""
    cfg = dict(CONFIGS[name])
    return make_system(n_rhs=n_rhs, threads=threads, **cfg)


def learned_system_params(s):
    """Shape of system s (0..63) of the learned-preconditioner family.

    200,000 stars x max(Poisson(30), 5) obs; attitude knots per axis and
    instrumental columns log-uniform on [5k, 50k] and [500, 5000].
    """
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(25030400 + s)))
    k = int(round(math.exp(g.uniform(math.log(5000), math.log(50000)))))
    ni = int(round(math.exp(g.uniform(math.log(500), math.log(5000)))))
    return dict(n_stars=200_000, obs=30, poisson=True, n_knots=k, n_instr=ni, n_glob=1,
                seed=25030400 + s)



def mlp_init_params(seed):
    """Initial parameters of the learned-preconditioner MLP (8 -> 64 -> 64 -> 1),
    flat float64 in the order W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3:
    normal weights with standard deviations sqrt(2/8), sqrt(2/64), sqrt(1/64)
    (He initialisation) and zero biases, from a seeded PCG64 stream."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    return np.concatenate([g.normal(0.0, math.sqrt(2.0 / 8), 64 * 8), np.zeros(64),
                           g.normal(0.0, math.sqrt(2.0 / 64), 64 * 64), np.zeros(64),
                           g.normal(0.0, math.sqrt(1.0 / 64), 64), np.zeros(1)])


def rank_deficient_system(seed=35):
    """An overdetermined, rank-deficient system (for the minimum-norm checks).

    120 stars of 1, 2, 3, 4 or 40 observations (a star with fewer than 5 rows
    leaves its 5 astrometric columns rank-deficient), attitude start knots
    restricted to [0, 45] of 100 (knots 49..99 have no rows: empty columns),
    and the coefficients of instrumental columns 0..4 set to zero (empty
    columns as well). About 2,200 rows, 951 unknowns.
    """
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed + 1)))
    counts = rng.choice([1, 2, 3, 4, 40], size=120, p=[0.15, 0.15, 0.15, 0.15, 0.4])
    s = make_system(n_stars=120, n_knots=100, n_instr=50, n_glob=1, counts=counts, seed=seed)
    att = 5 * 120 + (s["att_off"] - 5 * 120) % 46
    vals = s["vals"].copy()
    vals[:, 17:23][s["instr"] < 5] = 0.0
    return dict(s, vals=vals, att_off=att)


def add_constraints(sys, n_con=6, per_row=200, seed=0, must_cols=None):
    """The system with n_con constraint rows appended (CSR arrays con_ptr,
    con_col, con_val): each row has per_row distinct columns, four fifths
    astrometric columns of random stars and the rest attitude, instrumental
    or global columns, coefficients N(0, 1). must_cols (optional) are columns
    every row also includes (e.g. those of rank-deficient stars). The
    right-hand side's constraint part is formed by whichever side uses it."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    n_unk = n_unknowns(sys["n_stars"], sys["n_knots"], sys["n_instr"], sys["n_glob"])
    n_astro = 5 * sys["n_stars"]
    ptr, cols, vals = [0], [], []
    for _ in range(n_con):
        na = min(n_astro, (4 * per_row) // 5)
        c = set(rng.choice(n_astro, size=na, replace=False).tolist())
        if n_unk > n_astro:
            c |= set((n_astro + rng.choice(n_unk - n_astro, size=min(n_unk - n_astro,
                                                                      per_row - na),
                                           replace=False)).tolist())
        if must_cols is not None:
            c |= set(int(j) for j in must_cols)
        c = np.array(sorted(c), dtype=np.int64)
        cols.append(c)
        vals.append(rng.standard_normal(c.size))
        ptr.append(ptr[-1] + c.size)
    return dict(sys, con_ptr=np.array(ptr, dtype=np.int64),
                con_col=np.concatenate(cols) if cols else np.zeros(0, np.int64),
                con_val=np.concatenate(vals) if vals else np.zeros(0))
