import json
import multiprocessing as mp
import os
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300)")
    config.addinivalue_line("markers", "slow: larger CPU cases")


# ---------------------------------------------------------------------------
# The oracle's answer on the 30M-row workload. One single-core FP64 LSQR run
# to atol = btol = 1e-14 takes minutes, so when a selected test asks for it
# the run starts in a separate (spawned, CPU-only) process as soon as
# collection is done and overlaps the other tests; the test waits for it.
# ---------------------------------------------------------------------------
_MEDIUM = {}


def medium_oracle_job(out_prefix):
    """Child process: the medium workload from its seed, b = A x* + noise, and
    the oracle's LSQR solution at atol = btol = 1e-14 (saved as .npy + .json)."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import oracle
    from paper_2503_22863_b300 import synth
    s = synth.make_config("medium")
    b = np.zeros(s["n_rows"])
    oracle.aprod1(s, s["x_star"], b)
    b += s["noise"]
    r = oracle.lsqr(s, b, atol=1e-14, btol=1e-14)
    np.save(out_prefix + ".npy", r["x"])
    with open(out_prefix + ".json", "w") as f:
        json.dump({k: r[k] for k in ("istop", "itn", "rnorm", "anorm", "xnorm")}, f)


def pytest_collection_finish(session):
    if session.config.option.collectonly:
        return
    if any("medium_oracle" in getattr(it, "fixturenames", ()) for it in session.items):
        d = tempfile.mkdtemp(prefix="gsr_medium_oracle_")
        prefix = os.path.join(d, "x")
        p = mp.get_context("spawn").Process(target=medium_oracle_job, args=(prefix,),
                                            daemon=True)
        p.start()
        _MEDIUM.update(proc=p, prefix=prefix)


def pytest_sessionfinish(session, exitstatus):
    p = _MEDIUM.get("proc")
    if p is not None and p.is_alive():
        p.terminate()  # the child this session started, by its own handle
        p.join(10)


@pytest.fixture(scope="session")
def medium_oracle():
    """(x, result fields) of the oracle on the medium workload."""
    import numpy as np
    p = _MEDIUM.get("proc")
    if p is None:  # the fixture was requested late (e.g. by -k): run it here
        d = tempfile.mkdtemp(prefix="gsr_medium_oracle_")
        prefix = os.path.join(d, "x")
        p = mp.get_context("spawn").Process(target=medium_oracle_job, args=(prefix,))
        p.start()
        _MEDIUM.update(proc=p, prefix=prefix)
    p.join(3600)
    assert p.exitcode == 0, "oracle run on the medium workload failed (%s)" % p.exitcode
    prefix = _MEDIUM["prefix"]
    with open(prefix + ".json") as f:
        info = json.load(f)
    return np.load(prefix + ".npy"), info
