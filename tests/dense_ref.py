"""Independent dense/sparse builders of A for the CPU pins.

Written from the row layout alone (5 astrometric | 3 axes x 4 consecutive
attitude knots | 6 instrumental | 1 global, Sec. 2) without reusing the
oracle's or the CUDA library's indexing code.
"""
import os

import numpy as np
import scipy.sparse as sp

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def columns(sys):
    """[n_rows, 24] int64 column of every slot (-1 where the global slot is absent)."""
    n = sys["n_rows"]
    K = sys["n_knots"]
    cols = np.empty((n, 24), dtype=np.int64)
    ao = np.asarray(sys["astro_off"], dtype=np.int64)
    at = np.asarray(sys["att_off"], dtype=np.int64)
    cols[:, 0:5] = ao[:, None] + np.arange(5)[None, :]
    for axis in range(3):
        cols[:, 5 + 4 * axis:9 + 4 * axis] = at[:, None] + axis * K + np.arange(4)[None, :]
    ibase = 5 * sys["n_stars"] + 3 * K
    cols[:, 17:23] = ibase + np.asarray(sys["instr"], dtype=np.int64)
    cols[:, 23] = ibase + sys["n_instr"] if sys["n_glob"] == 1 else -1
    return cols


def n_unk(sys):
    return 5 * sys["n_stars"] + 3 * sys["n_knots"] + sys["n_instr"] + sys["n_glob"]


def n_con(sys):
    return 0 if sys.get("con_ptr") is None else len(sys["con_ptr"]) - 1


def sparse(sys):
    """A as a sparse matrix: the observation rows, then any constraint rows
    (CSR con_ptr / con_col / con_val, repeated columns summed)."""
    cols = columns(sys)
    rows = np.repeat(np.arange(sys["n_rows"]), 24).reshape(-1, 24)
    keep = cols >= 0
    r, c, v = rows[keep], cols[keep], np.asarray(sys["vals"])[keep]
    nc = n_con(sys)
    if nc:
        ptr = np.asarray(sys["con_ptr"])
        crow = sys["n_rows"] + np.repeat(np.arange(nc), np.diff(ptr))
        r = np.concatenate([r, crow])
        c = np.concatenate([c, np.asarray(sys["con_col"])])
        v = np.concatenate([v, np.asarray(sys["con_val"])])
    return sp.csr_matrix((v, (r, c)), shape=(sys["n_rows"] + nc, n_unk(sys)))


def dense(sys):
    return sparse(sys).toarray()


def load_probe_system():
    """The hand-worked 3-row system of golden/aprod_unit_probes.txt and its probes."""
    rows, probes = [], []
    with open(os.path.join(GOLDEN, "aprod_unit_probes.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "row":
                rows.append([int(t) for t in tok[1:]])
            else:
                lhs, rhs = line.split(":")
                probes.append((lhs.split(), [float(t) for t in rhs.split()]))
    n_rows = len(rows)
    vals = np.array([[100.0 * (i + 1) + t for t in range(24)] for i in range(n_rows)])
    sys = dict(n_rows=n_rows, n_stars=2, n_knots=5, n_instr=7, n_glob=1,
               vals=vals,
               astro_off=np.array([5 * r[1] for r in rows], dtype=np.int64),
               att_off=np.array([10 + r[2] for r in rows], dtype=np.int64),
               instr=np.array([r[3:9] for r in rows], dtype=np.int32))
    return sys, probes
