#!/usr/bin/env python3
"""Benchmark of the AVU-GSR hot path on one B300: LSQR time to 1e-9 relative
error on the 30M-row synthetic system, with the aprod kernels' HBM roofline.

One step = one complete preconditioned LSQR solve of A x = b (every aprod 1,
aprod 2 and vector update of the path) from b resident in HBM to x, for the N*
iterations that first bring ||x_k - x_ref|| / ||x_ref|| to 1e-9 (N* and x_ref
are found before the timed region; x_ref is the same solver run to its
attainable floor and is verified against the normal equations by the tests).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank solves its own
replica; the reported time is the max over ranks. --impl reference times the
FP64 CPU oracle as it stands on the host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LSQR time-to-1e-9 and aprod1/aprod2 HBM GB/s vs peak: FP64 vs mixed/batched"
TARGET_ERR = 1e-9
# Iterations to 1e-9 per workload, measured by this benchmark's own N* search
# on the GPU (used by the CPU reference arm, which cannot afford to find N*).
ITERS_TO_1E9 = {"tiny": 25, "small": 51, "medium": 68, "large_small": 40, "large": 45}
FALLBACK_HBM_GBS = 6400.0
# Algorithmic bytes of one launch group, per row and per unknown, for the
# FP64 method: a row is 24 FP64 values + 8 B star offset + 8 B attitude offset
# + 6 x 4 B instrumental columns = 232 B.
#   aprod 1 (u = A v - alpha u): 232 A + 8 u read + 8 u write = 248 B/row;
#            v read once = 8 B/unknown
#   aprod 2 (v = A^T u - beta v): 232 A + 8 u = 240 B/row; v read + write
#            = 16 B/unknown
# (The device layout moves 240 B/row in aprod 1 and 244 B/row in aprod 2:
# float-pair values are 8 B like FP64, indices are narrower, and the row order
# and knot order copies add a u scatter and a second u read.)
BYTES = {"aprod1": (248, 8), "aprod2": (240, 16)}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("gsr_aprod.cu", "gsr_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2503_22863_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, n_rows):
    """DRAM bytes per launch (read + write) of the kernel group from the ncu
    figures in profiles/traffic.json, taken on the current kernel source (else
    None): a capture of this very workload when there is one, otherwise a
    smaller workload's bytes per row scaled to n_rows (the traffic of these
    row-streaming kernels grows about in proportion to the rows processed).
    A workload with a capture of its own taken on an older source gets None:
    its own figures showed that the scaled ones do not hold for it."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        entries = json.load(f).get("entries", [])
    h = kernel_source_hash()
    cur = [e for e in entries if e.get("kernel") == kernel and e.get("kernel_source_hash") == h]
    for e in cur:
        if e.get("n_rows") == n_rows and "bytes_per_launch" in e:
            return float(e["bytes_per_launch"])
    if any(e.get("kernel") == kernel and e.get("n_rows") == n_rows for e in entries):
        return None
    for e in cur:
        if "bytes_per_row" in e:
            return float(e["bytes_per_row"]) * n_rows
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "gsr_bench_clocks_%d_%d.csv" % (
            gpu_index, os.getpid()))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
def cpu_oracle_estimate(sys, b, iters):
    """Time the FP64 oracle (as it stands, one host core) on a bounded sample of
    the workload: LSQR with 1 and with 2 iterations; extrapolate to `iters`."""
    import oracle
    t0 = time.perf_counter()
    oracle.lsqr(sys, b, atol=0.0, btol=0.0, conlim=0.0, itnlim=1)
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.lsqr(sys, b, atol=0.0, btol=0.0, conlim=0.0, itnlim=2)
    t2 = time.perf_counter() - t0
    per_iter = max(t2 - t1, 1e-9)
    return t1 + (iters - 1) * per_iter, per_iter, t1


def cpu_aprod_times(sys_, n_threads_note=None):
    """Seconds per aprod 1 and aprod 2 of the single-core oracle and of the
    all-core OpenMP baseline on `sys_` (median of a few runs; inputs seeded)."""
    import cpu_baseline
    import oracle
    rng = np.random.default_rng(0)
    x = rng.standard_normal(sys_["n_unk"])
    y = rng.standard_normal(sys_["n_rows"])
    out = {}
    for name, a1, a2, reps in (("oracle", oracle.aprod1, oracle.aprod2, 1),
                               ("openmp", cpu_baseline.aprod1, cpu_baseline.aprod2, 3)):
        t1, t2 = [], []
        for _ in range(reps):
            yy = np.zeros(sys_["n_rows"])
            t0 = time.perf_counter()
            a1(sys_, x, yy)
            t1.append(time.perf_counter() - t0)
            xx = np.zeros(sys_["n_unk"])
            t0 = time.perf_counter()
            a2(sys_, y, xx)
            t2.append(time.perf_counter() - t0)
        out[name] = {"aprod1_s": statistics.median(t1), "aprod2_s": statistics.median(t2)}
    out["openmp"]["threads"] = cpu_baseline.threads()
    out["oracle"]["threads"] = 1
    return out


def make_workload(name):
    from paper_2503_22863_b300 import synth
    t0 = time.perf_counter()
    sys_ = synth.make_config(name)
    log("workload %s: %d rows, %d unknowns (generated in %.1f s)" % (
        name, sys_["n_rows"], sys_["n_unk"], time.perf_counter() - t0))
    return sys_


def workload_desc(name, sys_):
    from paper_2503_22863_b300 import synth
    c = synth.CONFIGS[name]
    obs = ("max(Poisson(%d),5)" % c["obs"]) if c["poisson"] else str(c["obs"])
    return ("%s: %d stars x %s obs = %d rows; 3 x %d attitude knots, %d instrumental, %d global; "
            "N(0,1) values, x* ~ N(0,1), b = A x* + noise of sigma 1e-3; seed %d" % (
                name, c["n_stars"], obs, sys_["n_rows"], c["n_knots"], c["n_instr"], c["n_glob"],
                c["seed"]))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    sys_ = make_workload(args.workload)
    b = np.zeros(sys_["n_rows"])
    oracle.aprod1(sys_, sys_["x_star"], b)
    b += sys_["noise"]
    iters = ITERS_TO_1E9[args.workload]
    t0 = time.perf_counter()
    oracle.lsqr(sys_, b, atol=0.0, btol=0.0, conlim=0.0, itnlim=1)
    t1 = time.perf_counter() - t0
    samples = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.lsqr(sys_, b, atol=0.0, btol=0.0, conlim=0.0, itnlim=2)
        t2 = time.perf_counter() - t0
        if k >= args.warmup:
            samples.append(t2 - t1)
    per_iter = statistics.median(samples)
    value = t1 + (iters - 1) * per_iter
    sample = ("oracle LSQR with 1 iteration (%.2f s, includes column norms and start) and %d "
              "runs with 2 iterations; per-iteration %.2f s extrapolated to %d iterations" % (
                  t1, len(samples), per_iter, iters))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_iter * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, sys_), "iterations_to_1e9": iters},
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_solves(S, b, x, steps, stream, **solve):
    """Run `steps` solves back to back; per-step device time (CUDA events on the
    solve stream) and the per-solve results."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    res = []
    ev[0].record(stream)
    for k in range(steps):
        res.append(S.lsqr(b, x=x, **solve))
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    return [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)], res


def bench_mixed(S, b, x_ref, args, stream, dev):
    """Mixed precision (FP32-stored A + FP64 correction): find the phase-1 length
    and the phase-2 iterations to 1e-9, then time solves of exactly that shape."""
    import torch
    probe = S.lsqr(b, atol=1e-15, btol=1e-15, precision="mixed", itnlim=5000, x_ref=x_ref,
                   err_hist=True)
    eh = probe["err_hist"]
    n1 = probe["itn"] - probe["phase2_itn"]
    ok = np.nonzero(eh[n1:] <= TARGET_ERR)[0]
    n2 = int(ok[0]) + 1 if ok.size else int(probe["phase2_itn"])
    x = torch.empty(S.n_unk, dtype=torch.float64, device=dev)
    solve = dict(atol=0.0, btol=0.0, conlim=0.0, precision="mixed", mixed_switch_itn=n1,
                 itnlim=n1 + n2)
    for _ in range(args.warmup):
        S.lsqr(b, x=x, **solve)
    ms, res = timed_solves(S, b, x, args.steps, stream, profile=True, **solve)
    err = float(torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref))
    nt = sum(r["n_timed_itn"] for r in res)
    log("mixed: phase 1 %d + phase 2 %d iterations, %.1f ms, err %.2e" % (n1, n2, np.mean(ms), err))
    return {"value": float(np.mean(ms)) / 1e3, "unit": "s", "phase1_itn_fp32": n1,
            "phase2_itn_fp64": n2, "fp32_phase_rel_err": float(eh[n1 - 1]),
            "final_rel_err": err,
            "aprod1_ms_mean": sum(r["t_aprod1_ms"] for r in res) / max(nt, 1),
            "aprod2_ms_mean": sum(r["t_aprod2_ms"] for r in res) / max(nt, 1),
            "gpu_launches": int(sum(r["n_launches"] for r in res))}


def bench_batched(S, sys_, k, ms_single, args, stream, dev):
    """k right-hand sides b_j = A x* + noise_j (noise drawn on the device from a
    fixed seed) solved at once: time until every one reaches 1e-9."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(2504 * 100 + k)
    xs = torch.from_numpy(sys_["x_star"]).to(dev)
    Xs = xs[:, None].repeat(1, k).contiguous()
    B = torch.randn((S.n_rows, k), generator=g, dtype=torch.float64, device=dev) * 1e-3
    S.aprod1_batch(Xs, B)
    ref = S.lsqr_batch(B, atol=1e-15, btol=1e-15, itnlim=5000)
    x_ref = ref["x"].clone()
    probe = S.lsqr_batch(B, atol=0.0, btol=0.0, conlim=0.0, itnlim=max(ref["itn"]) + 20,
                         x_ref=x_ref, err_hist=True)
    worst = probe["err_hist"].max(axis=1)
    ok = np.nonzero(worst <= TARGET_ERR)[0]
    n_star = int(ok[0]) + 1 if ok.size else int(max(ref["itn"]))
    X = torch.empty((S.n_unk, k), dtype=torch.float64, device=dev)
    solve = dict(atol=0.0, btol=0.0, conlim=0.0, itnlim=n_star)
    S.lsqr_batch(B, X=X, **solve)
    torch.cuda.synchronize(dev)
    steps = max(1, min(args.steps, 3))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    res = None
    for i in range(steps):
        res = S.lsqr_batch(B, X=X, **solve)
        ev[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    ms = float(np.mean([ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]))
    err = float((torch.linalg.norm(X - x_ref, dim=0) / torch.linalg.norm(x_ref, dim=0)).max())
    log("batched k=%d: %d iterations, %.1f ms (%.1f ms per right-hand side), worst err %.2e"
        % (k, n_star, ms, ms / k, err))
    out = {"value": ms / 1e3, "unit": "s", "k": k, "iterations_to_1e9": n_star,
           "s_per_rhs": ms / 1e3 / k, "speedup_vs_k_single_solves": k * ms_single / ms,
           "worst_final_rel_err": err, "tuning": S.batch_tuning(),
           "gpu_launches": int(res["n_launches"]) * steps}
    if S.storage == "f32+f64":
        out["mixed"] = bench_batched_mixed(S, B, x_ref, k, ms_single, steps, stream, dev)
    return out


def bench_batched_mixed(S, B, x_ref, k, ms_single, steps, stream, dev):
    """The k right-hand sides with mixed precision (FP32-value phase, then the
    float-pair correction phase): find the first phase's length and the second
    phase's iterations to 1e-9 for the worst right-hand side, then time solves
    of exactly that shape."""
    import torch
    probe = S.lsqr_batch(B, atol=1e-15, btol=1e-15, precision="mixed", itnlim=5000, x_ref=x_ref,
                         err_hist=True)
    n1 = max(i - p for i, p in zip(probe["itn"], probe["phase2_itn"]))
    worst = probe["err_hist"].max(axis=1)
    ok = np.nonzero(worst[n1:] <= TARGET_ERR)[0]
    n2 = int(ok[0]) + 1 if ok.size else int(max(probe["phase2_itn"]))
    X = torch.empty((S.n_unk, k), dtype=torch.float64, device=dev)
    solve = dict(atol=0.0, btol=0.0, conlim=0.0, precision="mixed", mixed_switch_itn=n1,
                 itnlim=n1 + n2)
    S.lsqr_batch(B, X=X, **solve)
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    res = None
    for i in range(steps):
        res = S.lsqr_batch(B, X=X, **solve)
        ev[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    ms = float(np.mean([ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]))
    err = float((torch.linalg.norm(X - x_ref, dim=0) / torch.linalg.norm(x_ref, dim=0)).max())
    log("batched k=%d mixed: %d FP32 + %d float-pair iterations, %.1f ms (%.1f ms per "
        "right-hand side), worst err %.2e" % (k, n1, n2, ms, ms / k, err))
    return {"value": ms / 1e3, "unit": "s", "phase1_itn_fp32": n1, "phase2_itn": n2,
            "s_per_rhs": ms / 1e3 / k, "speedup_vs_k_single_solves": k * ms_single / ms,
            "worst_final_rel_err": err, "gpu_launches": int(res["n_launches"]) * steps}


def bench_learned(args, dev):
    """Learned column preconditioner on its family of 64 seeded systems
    (200,000 stars x max(Poisson(30), 5) obs, K log-uniform on [5k, 50k],
    n_instr on [500, 5000]): labels from solve histories on systems 0-39,
    the fallback gate on 40-47, iterations to 1e-9 on the held-out 48-63,
    learned vs plain column scaling. Systems are generated one ahead on a
    host thread while the GPU works on the current one."""
    import threading
    import torch
    from paper_2503_22863_b300 import gsr, learned, synth

    def gen(s, out):
        out[s] = synth.make_system(**synth.learned_system_params(s))

    n_sys = args.learned_systems
    n_train, n_val = (n_sys * 40) // 64, (n_sys * 8) // 64
    pending = {}
    th = threading.Thread(target=gen, args=(0, pending))
    th.start()
    feats, labels, val, held = [], [], [], []
    t_lab = t_eval = 0.0
    gam = []
    for s in range(n_sys):
        th.join()
        sys_ = pending.pop(s)
        if s + 1 < n_sys:
            th = threading.Thread(target=gen, args=(s + 1, pending))
            th.start()
        S = gsr.System(sys_, device=dev.index or 0)
        b = learned.make_rhs(S, sys_)
        del sys_
        t0 = time.perf_counter()
        probe = learned.SolveProbe(S, b, tol=TARGET_ERR)
        if s < n_train:
            lab, info = learned.block_labels(S, probe)
            feats.append(S.column_features())
            labels.append(lab)
            gam.append((info["log2_gamma_att"], info["log2_gamma_instr"]))
            S.close()
            t_lab += time.perf_counter() - t0
        elif s < n_train + n_val:
            val.append((S, probe))
        else:
            held.append((S, probe))
    t0 = time.perf_counter()
    model, hist = learned.train(feats, labels, steps=1500, lr=2e-3)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    pre = learned.LearnedPreconditioner(model)
    pre.validate(val)
    t0 = time.perf_counter()
    base, raw, used = [], [], []
    was = pre.enabled
    for S, probe in held:
        base.append(probe.n_colnorm)
        pre.enabled = True
        raw.append(probe.iterations(pre.scaling(S)))
        pre.enabled = was
        used.append(probe.iterations(pre.scaling(S)))
    t_eval = time.perf_counter() - t0
    for S, _ in val + held:
        S.close()
    med = lambda v: float(np.median(v))
    log("learned: held-out median iterations colnorm %.1f, learned %.1f, with fallback %.1f "
        "(model %s); labels %.1f s, training %.1f s (loss %.3g -> %.3g)"
        % (med(base), med(raw), med(used), "kept" if was else "rejected by the gate", t_lab,
           t_train, hist[0], hist[-1]))
    return {"value": med(used), "unit": "iterations to 1e-9 (median, held-out)",
            "systems": {"train": n_train, "validate": n_val, "held_out": len(held)},
            "median_itn_colnorm": med(base), "median_itn_learned": med(raw),
            "median_itn_with_fallback": med(used), "model_enabled": bool(was),
            "validation": pre.validation, "held_out_itn_colnorm": base,
            "held_out_itn_learned": raw,
            "label_log2_gamma_att_range": [min(g[0] for g in gam), max(g[0] for g in gam)],
            "label_log2_gamma_instr_range": [min(g[1] for g in gam), max(g[1] for g in gam)],
            "train_loss_first_last": [float(hist[0]), float(hist[-1])],
            "train_s": t_train, "label_search_s": t_lab, "eval_s": t_eval}


def max_over_ranks(vals, dist, device):
    """Element-wise maximum of per-rank values over all ranks (identity for one
    process): with independent replicas the job takes as long as its slowest rank."""
    if dist is None:
        return [float(v) for v in vals]
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2503_22863_b300 import gsr

    sys_ = make_workload(args.workload)
    t0 = time.perf_counter()
    free0 = torch.cuda.mem_get_info(local)[0]
    S = gsr.System(sys_, device=local, storage="f32+f64" if args.variants else "f64")
    # device memory the system took (its layout, copies and solver vectors)
    resident_gb = (free0 - torch.cuda.mem_get_info(local)[0]) / 1e9
    log("gsr_create: %.1f s, %.1f GB on the device" % (time.perf_counter() - t0, resident_gb))
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    with torch.cuda.stream(stream):
        xs = torch.from_numpy(sys_["x_star"]).to(dev)
        b = torch.from_numpy(np.ascontiguousarray(sys_["noise"])).to(dev)
        S.aprod1(xs, b)  # b = A x* + noise
        # reference solution: the same solver run to its attainable floor
        ref = S.lsqr(b, atol=1e-15, btol=1e-15, itnlim=5000)
        x_ref = ref["x"].clone()
        log("x_ref: istop %d after %d iterations" % (ref["istop"], ref["itn"]))
        probe = S.lsqr(b, atol=0.0, btol=0.0, conlim=0.0, itnlim=min(5000, ref["itn"] + 50),
                       x_ref=x_ref, err_hist=True)
        eh = probe["err_hist"]
        ok = np.nonzero(eh <= TARGET_ERR)[0]
        n_star = int(ok[0]) + 1 if ok.size else int(ref["itn"])
        log("N* = %d iterations to %.0e (err %.3e)" % (n_star, TARGET_ERR, eh[n_star - 1]))
        x = torch.empty(S.n_unk, dtype=torch.float64, device=dev)
        solve = dict(atol=0.0, btol=0.0, conlim=0.0, itnlim=n_star)
        for _ in range(args.warmup):
            S.lsqr(b, x=x, **solve)
        torch.cuda.synchronize(dev)

        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.2)
        barrier()
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        results = []
        ev[0].record(stream)
        for k in range(args.steps):
            r = S.lsqr(b, x=x, profile=True, **solve)
            ev[k + 1].record(stream)
            results.append(r)
        torch.cuda.synchronize(dev)
        barrier()
        clk = clocks.stop()
        step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
        err = float(torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref))

        # end to end through the public API with host buffers
        b_host = torch.empty(S.n_rows, dtype=torch.float64, pin_memory=True)
        b_host.copy_(b)
        x_host = torch.empty(S.n_unk, dtype=torch.float64, pin_memory=True)
        b_dev = torch.empty_like(b)
        torch.cuda.synchronize(dev)
        barrier()
        e2e = []
        for k in range(max(1, min(args.steps, 5))):
            t0 = time.perf_counter()
            b_dev.copy_(b_host, non_blocking=True)
            S.lsqr(b_dev, x=x, **solve)
            x_host.copy_(x, non_blocking=True)
            torch.cuda.synchronize(dev)
            e2e.append(time.perf_counter() - t0)
        barrier()

        # iterations per second over the paper's 100-iteration run (Sec. 3): one
        # solve that cannot stop before itnlim = 100
        ev100 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        x100 = torch.empty_like(x)
        ev100[0].record(stream)
        r100 = S.lsqr(b, x=x100, atol=0.0, btol=0.0, conlim=0.0, itnlim=100)
        ev100[1].record(stream)
        torch.cuda.synchronize(dev)
        t100 = ev100[0].elapsed_time(ev100[1]) / 1e3
        its_100 = r100["itn"] / t100
        log("100-iteration solve: %.1f ms (%.0f iterations/s)" % (t100 * 1e3, its_100))

        variants = {}
        if args.variants:
            variants["mixed"] = bench_mixed(S, b, x_ref, args, stream, dev)
            for kk in args.batch_k:
                variants["batched_k%d" % kk] = bench_batched(S, sys_, kk, ms_single=float(
                    np.mean(step_ms)), args=args, stream=stream, dev=dev)
            if args.learned_systems > 0:
                variants["learned"] = bench_learned(args, dev)

    # replicas: the job's time is that of its slowest rank
    ms, e2e_s = max_over_ranks([float(np.mean(step_ms)), float(np.median(e2e))], dist, dev)

    nt = sum(r["n_timed_itn"] for r in results)
    t_a1 = sum(r["t_aprod1_ms"] for r in results) / max(nt, 1)
    t_a2 = sum(r["t_aprod2_ms"] for r in results) / max(nt, 1)
    t_vec = sum(r["t_vector_ms"] for r in results) / max(nt, 1)
    n_rows, n_unk = S.n_rows, S.n_unk
    by1 = BYTES["aprod1"][0] * n_rows + BYTES["aprod1"][1] * n_unk
    by2 = BYTES["aprod2"][0] * n_rows + BYTES["aprod2"][1] * n_unk
    peak, peak_kind = measured_peaks()
    gbs1 = by1 / (t_a1 * 1e-3) / 1e9 if t_a1 > 0 else 0.0
    gbs2 = by2 / (t_a2 * 1e-3) / 1e9 if t_a2 > 0 else 0.0
    dom = "aprod1" if t_a1 >= t_a2 else "aprod2"
    ach = gbs1 if dom == "aprod1" else gbs2
    launches = int(sum(r["n_launches"] for r in results))

    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2+f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload, sys_), "n_rows": n_rows,
                   "n_unk": n_unk, "iterations_to_1e9": n_star, "final_rel_err": err,
                   "l2": ("inputs larger than L2 (system %.1f GB resident in HBM)" if resident_gb > 0.126
                          else "system of %.1f GB: fits in L2 (timings not HBM-bound)") % resident_gb,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak,
                     "unit": "GB/s", "frac": ach / peak, "peak_kind": peak_kind,
                     "traffic": profiled_traffic(dom, n_rows)},
        "aprod": {"aprod1_ms": t_a1, "aprod1_GBps": gbs1, "aprod2_ms": t_a2, "aprod2_GBps": gbs2,
                  "vector_ms": t_vec, "iterations_per_s": its_100,
                  "iterations_per_s_how": "one solve of exactly 100 iterations (the paper's "
                                          "run length, Sec. 3), CUDA events around it",
                  "iterations_per_s_kernels_only": 1e3 / (t_a1 + t_a2 + t_vec),
                  "bytes_per_launch": {"aprod1": by1, "aprod2": by2}},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * n_rows,
                "d2h_bytes_per_step": 8 * n_unk},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if variants:
        line["variants"] = variants
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        bh = b.detach().cpu().numpy()
        log("timing the CPU oracle on a bounded sample ...")
        est, per_iter, t1 = cpu_oracle_estimate(sys_, bh, n_star)
        line["cpu_baseline"] = {
            "value": est, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": "oracle LSQR with 1 and 2 iterations on the same system (%.1f s and %.1f s); "
                      "per-iteration %.2f s extrapolated to %d iterations" % (
                          t1, t1 + per_iter, per_iter, n_star)}
        log("timing the oracle and the all-core OpenMP products ...")
        cpu = cpu_aprod_times(sys_)
        tiny = make_workload("tiny")
        cpu_tiny = cpu_aprod_times(tiny)
        omp = cpu["openmp"]
        line["cpu_openmp"] = {
            "kind": "all-core OpenMP aprod (independent of the oracle and the CUDA library)",
            "cores": omp["threads"], "aprod1_s": omp["aprod1_s"], "aprod2_s": omp["aprod2_s"],
            "lsqr_time_to_1e9_s_lower_bound": n_star * (omp["aprod1_s"] + omp["aprod2_s"]),
            "lower_bound_how": "%d iterations x (aprod 1 + aprod 2), vector updates not counted"
                               % n_star,
            "gpu_speedup_per_aprod": {"aprod1": omp["aprod1_s"] / (t_a1 * 1e-3),
                                      "aprod2": omp["aprod2_s"] / (t_a2 * 1e-3)}}
        line["cpu_baseline"]["oracle_aprod_s"] = {
            args.workload: cpu["oracle"], "tiny": cpu_tiny["oracle"]}
        line["cpu_openmp"]["tiny"] = cpu_tiny["openmp"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    S.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="medium", choices=["tiny", "small", "medium", "large", "large_small"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the mixed-precision / batched variants")
    ap.add_argument("--learned-systems", type=int, default=64,
                    help="systems of the learned-preconditioner family (40/64 train, 8/64 "
                         "validate, the rest held out); 0 skips the variant")
    ap.add_argument("--batch-k", type=int, nargs="*", default=[8, 32],
                    help="right-hand-side counts of the batched variant")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
