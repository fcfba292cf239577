#!/usr/bin/env python3
"""Benchmark of the fixed-pattern KKT refactorization path on GB300.

Workload (default): the 2,000-bus sequence, plain FP64 plus adjoint (KKT
dimension 14,000, 140,400 stored entries, 30 value sets whose D_x, D_s widen
to [1e-8, 1e8]).  One step is one KKT system of the sequence through the
whole path: refactorization, solve, iterative refinement to scaled residual
1e-14, transposed solve with its refinement, and the adjoint gather (the
backward of x = A^-1 b).  All value sets, right-hand sides and upstream
gradients are resident in HBM before the timed region; L2 is flushed between
timed steps (a 256 MiB write, outside the per-step events).

Metric: microseconds per KKT system (lower is better) and HBM GB/s.  The
``e2e`` figure runs the same step from pinned host buffers through the C
interface, copies included.  ``--impl reference`` times the CPU oracle on the
host cores on the same workload (a bounded sample per step).

Multi-GPU (torchrun): every rank runs its own replica of the sequence on its
own GPU (independent systems, no collective on the data path); the reported
value divides the slowest rank's time by all systems processed.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

METRIC = "refactor+solve µs per KKT system and HBM GB/s on 1 GB300; batched/FP32 vs plain"
UNIT = "us/system"
WORKLOADS = {
    "2000bus_fp64_adjoint": dict(cfg=1, fp32=False),
    "200bus_fp64": dict(cfg=0, fp32=False),
}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25      # GB300 FP64 (non-tensor and tensor), nominal
HBM_FALLBACK_GBS = 6800.0


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _init_dist(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(value: float, ws: int, device=None) -> float:
    """Max of a float over all ranks (identity when not distributed)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_us_per_system(max_rank_seconds: float, systems_per_rank: int, ws: int) -> float:
    """Whole-job time per system: the slowest rank's time over all systems."""
    return max_rank_seconds * 1e6 / (systems_per_rank * ws)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- peaks
def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def source_hash():
    h = hashlib.sha256()
    for f in ("kkt.cu", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2306_14337_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, or
    None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        for ln in open(path):
            if ln.startswith("#") or not ln.strip():
                continue
            k, w, sha, b = ln.split()[:4]
            if k == kernel and w == workload and sha == source_hash():
                return float(b)
    except OSError:
        pass
    return None


# ----------------------------------------------------------------- oracle leg
def oracle_sample(seq, step_ids, budget_s: float):
    """Time the oracle (as it stands, single-threaded) on whole steps of the
    workload until ``budget_s`` seconds of CPU work are spent; returns
    (us per system, systems timed)."""
    import oracle
    perm = oracle.min_degree(seq.n, seq.indptr, seq.indices)   # ordering: outside, like analyze
    rng = np.random.default_rng(7)
    done, t_total = 0, 0.0
    for k in step_ids:
        v, b = seq.values(k), seq.rhs(k)
        g = rng.standard_normal(seq.n)
        t0 = time.perf_counter()
        o = oracle.Oracle(seq.n, seq.indptr, seq.indices, v, perm)
        x = o.solve(b)
        x, *_ = o.refine(b, x0=x)
        o.adjoint(x, g)
        t_total += time.perf_counter() - t0
        done += 1
        if t_total >= budget_s:
            break
    return t_total * 1e6 / max(done, 1), done


def run_reference(args, ws, rank):
    """--impl reference: the CPU oracle on the host cores, same metric."""
    if rank != 0:
        return 0
    from kktgen import config_sequence
    wl = WORKLOADS[args.workload]
    seq = config_sequence(wl["cfg"])
    ids = [k % seq.steps for k in range(args.warmup + args.steps)]
    oracle_sample(seq, ids[: args.warmup], 1e9)
    us, done = oracle_sample(seq, ids[args.warmup:], 1e9)
    cores = 1
    line = {
        "impl": "reference", "metric": METRIC, "value": us, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": us / 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": seq.n, "nnz": seq.nnz, "value_sets": seq.steps,
                   "l2": "host cores (no GPU cache)", "parallelism": "one host core"},
        "cpu_baseline": {"value": us, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{done} whole steps (refactor, solve, refine, transposed solve, adjoint) "
                                   f"of the {args.workload} sequence, single-threaded"},
        "e2e": {"value": us, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU leg
def run_native(args, ws, rank, local):
    import torch
    from kktgen import config_sequence
    from paper_2306_14337_gb300 import KKTSolver

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        _init_dist(ws, "nccl")
    wl = WORKLOADS[args.workload]
    seq = config_sequence(wl["cfg"])
    n, nnz, K = seq.n, seq.nnz, seq.steps
    S = KKTSolver(n, seq.indptr, seq.indices, fp32=wl["fp32"], device=local)
    st0 = S.stats()
    rng = np.random.default_rng(1234 + rank)
    vals = [torch.tensor(seq.values(k), device=dev) for k in range(K)]
    bs = [torch.tensor(seq.rhs(k), device=dev) for k in range(K)]
    gs = [torch.tensor(rng.standard_normal(n), device=dev) for k in range(K)]
    x = torch.empty(n, dtype=torch.float64, device=dev)
    lam = torch.empty_like(x)
    dA = torch.empty(nnz, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(k, ev=None):
        """One KKT system: refactor, solve, refine, transposed solve + refine, adjoint."""
        if ev is not None:
            ev[0].record(stream)
        S.refactor(vals[k])
        if ev is not None:
            ev[1].record(stream)
        S.solve(bs[k], out=x)
        if ev is not None:
            ev[2].record(stream)
        r1 = S.refine(bs[k], x, 1e-14, 20)
        if ev is not None:
            ev[3].record(stream)
        S.solve_transpose(gs[k], out=lam)
        r2 = S.refine_transpose(gs[k], lam, 1e-14, 20)
        if ev is not None:
            ev[4].record(stream)
        S.adjoint_gather(lam, x, out=dA)
        if ev is not None:
            ev[5].record(stream)
        return r1, r2

    for w in range(args.warmup):
        step(w % K)
    torch.cuda.synchronize()
    launches0 = S.stats()["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    phase = {"refactor": [], "solve": [], "refine": [], "transpose": [], "adjoint": []}
    step_ms, iters, omegas = [], [], []
    for it in range(args.steps):
        k = (args.warmup + it) % K
        flush.zero_()                               # L2 flush, outside the step's events
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        r1, r2 = step(k, ev)
        torch.cuda.synchronize()
        names = list(phase)
        for j, nm in enumerate(names):
            phase[nm].append(ev[j].elapsed_time(ev[j + 1]))
        step_ms.append(ev[0].elapsed_time(ev[5]))
        iters.append((r1["iters"], r2["iters"]))
        omegas.append(max(r1["omega"], r2["omega"]))
        if not (r1["converged"] and r2["converged"]):
            raise SystemExit(f"refinement did not converge at step {k}: {r1} {r2}")
    torch.cuda.synchronize()
    barrier(ws)
    launches = S.stats()["kernel_launches"] - launches0 - 0
    total_s = sum(step_ms) / 1e3
    total_s = reduce_max(total_s, ws, dev)
    clk = clocks.stop()
    st_code, npert = S.status()

    # e2e: the same step from pinned host buffers, copies inside the timed region
    hv = [v.cpu().pin_memory() for v in vals]
    hb = [b.cpu().pin_memory() for b in bs]
    hg = [g.cpu().pin_memory() for g in gs]
    dv = torch.empty(nnz, dtype=torch.float64, device=dev)
    db_ = torch.empty(n, dtype=torch.float64, device=dev)
    dg = torch.empty(n, dtype=torch.float64, device=dev)
    hx = torch.empty(n, dtype=torch.float64).pin_memory()
    hl = torch.empty(n, dtype=torch.float64).pin_memory()
    hdA = torch.empty(nnz, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for it in range(args.steps):
        k = (args.warmup + it) % K
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dv.copy_(hv[k], non_blocking=True)
        db_.copy_(hb[k], non_blocking=True)
        dg.copy_(hg[k], non_blocking=True)
        S.refactor(dv)
        S.solve(db_, out=x)
        S.refine(db_, x, 1e-14, 20)
        S.solve_transpose(dg, out=lam)
        S.refine_transpose(dg, lam, 1e-14, 20)
        S.adjoint_gather(lam, x, out=dA)
        hx.copy_(x, non_blocking=True)
        hl.copy_(lam, non_blocking=True)
        hdA.copy_(dA, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_s = reduce_max(sum(e2e_ms) / 1e3, ws, dev)

    # CPU baseline (rank 0, N = 1 only): the oracle on a bounded sample
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        us_cpu, done = oracle_sample(seq, list(range(K)), args.cpu_budget)
        cpu = {"value": us_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{done} whole steps of the {args.workload} sequence, single-threaded, "
                         f"ordering computed once outside the timing"}

    variants = {}
    if rank == 0 and not args.no_variants:
        variants = run_variants(dev)

    if rank != 0:
        return 0
    us = whole_job_us_per_system(total_s, args.steps, ws)
    ph_ms = {k: statistics.mean(v) for k, v in phase.items()}
    # dominant phase and its roofline
    st = S.stats()
    peak_hbm, peak_kind = load_peaks()
    flops = st["flops_refactor"]
    dom = max(ph_ms, key=ph_ms.get)
    fp64_peak_tflops = FP64_NOMINAL_TFLOPS
    if dom == "refactor":
        # FP64 FMA work dominates bytes by ~15x on this workload: ALU-bound roofline
        achieved = flops / (ph_ms["refactor"] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_refactor<double> (+k_scale, k_amax)",
                "achieved": achieved, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak_tflops,
                "peak_source": "nominal GB300 FP64 rate (a DFMA probe measured 1.2 TFLOP/s)",
                "algorithmic_flops_per_launch": flops,
                "traffic": committed_traffic("k_refactor_f64", args.workload)}
    else:
        # triangular solves: bytes of the factor read once per solve
        nsolves = {"solve": 1, "refine": max(1, statistics.mean(i[0] for i in iters)),
                   "transpose": 1 + statistics.mean(i[1] for i in iters)}.get(dom, 1)
        by = st["bytes_solve"] * nsolves
        achieved = by / (ph_ms[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": f"{dom} (k_trisolve)", "achieved": achieved,
                "peak": peak_hbm, "unit": "GB/s", "frac": achieved / peak_hbm,
                "peak_source": peak_kind, "algorithmic_bytes_per_launch": by,
                "traffic": committed_traffic("k_trisolve_f64", args.workload)}
    ref_bytes = st["bytes_refactor"]
    line = {
        "metric": METRIC, "value": us, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if wl["fp32"] else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "nnz": nnz, "nnz_lu": st["nnz_lu"],
                   "levels": st["n_levels"], "value_sets": K,
                   "l2": "flushed between timed steps (256 MiB write, outside the step events)",
                   "parallelism": f"replicas x{ws}"},
        "breakdown_ms": ph_ms,
        "refactor_hbm_gbs": ref_bytes / (ph_ms["refactor"] * 1e-3) / 1e9,
        "refine_iters": {"solve": statistics.mean(i[0] for i in iters),
                         "transpose": statistics.mean(i[1] for i in iters)},
        "omega_max": max(omegas), "status": int(st_code), "perturbed_pivots": npert,
        "roofline": roof,
        # Why the fraction is low: the refactorization is a chain of dependent
        # rows, one hand-off per level of the elimination DAG.
        "critical_path": {"refactor_levels": st["n_levels"],
                          "refactor_us_per_level": ph_ms["refactor"] * 1e3 / st["n_levels"],
                          "solve_levels": {"forward": st["n_levels"], "backward": st["n_levels_u"]},
                          "solve_tasks": st["n_tasks"], "longest_task_rows": st["max_task"]},
        "cpu_baseline": cpu,
        "e2e": {"value": whole_job_us_per_system(e2e_s, args.steps, ws), "unit": UNIT,
                "h2d_bytes_per_step": 8 * (nnz + 2 * n), "d2h_bytes_per_step": 8 * (nnz + 2 * n)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "variants": variants,
    }
    print(json.dumps(line), flush=True)
    return 0


def _time_ms(fn, reps=3):
    """Median device time (ms) of fn() over reps runs after one warm-up, CUDA
    events on the current stream, L2 flushed before each run."""
    import torch
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=torch.cuda.current_device())
    out = []
    fn()
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def run_uneven(dev):
    """48 systems with different patterns (16 x 500, 16 x 2,000, 12 x 5,000,
    4 x 20,000 buses): FP32 factors, one work queue and one CUDA graph per
    phase sequence (refactor, solve, 8 classic refinement steps), launch shape
    from the autotuner; systems the in-graph steps leave above 1e-14 finish
    with FGMRES on their context; then one transposed solve per system.
    Compared with the plain FP64 path run system by system."""
    import torch
    from kktgen.acopf import uneven_sequences
    from paper_2306_14337_gb300 import KKTQueue, KKTSolver
    from paper_2306_14337_gb300.tune import autotune_queue
    seqs = uneven_sequences()
    sols = [KKTSolver(s.n, s.indptr, s.indices, fp32=True, refine_mode="auto") for s in seqs]
    Q = KKTQueue(sols)
    vals = [torch.tensor(s.values(0), device=dev) for s in seqs]
    bs = [torch.tensor(s.rhs(0), device=dev) for s in seqs]
    gs = [torch.tensor(np.random.default_rng(k).standard_normal(s.n), device=dev) for k, s in enumerate(seqs)]
    xs = [torch.zeros_like(b) for b in bs]
    lams = [torch.zeros_like(g) for g in gs]
    om = torch.zeros(len(seqs), dtype=torch.float64, device=dev)
    state = {}

    def run():
        Q.run(vals, bs, xs, n_refine=8, omega=om)
        Q.solve_transpose(gs, lams)
        torch.cuda.synchronize()
        late = [k for k in range(len(seqs)) if not (om[k].item() <= 1e-14)]
        for k in late:
            sols[k].refine(bs[k], xs[k], 1e-14, 20)
        state["late"] = len(late)

    def once():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3
    best, table = autotune_queue(Q, once, [(s.n, s.indptr, s.indices) for s in seqs], reps=2)
    tq = _time_ms(run)
    worst = 0.0
    for k in range(len(seqs)):
        r = sols[k].refine(bs[k], xs[k], 1e-14, 0)
        worst = max(worst, r["omega"])
    # plain FP64, one system at a time
    plain = [KKTSolver(s.n, s.indptr, s.indices) for s in seqs]
    xp = [torch.zeros_like(b) for b in bs]

    def run_plain():
        for k, S in enumerate(plain):
            S.refactor(vals[k])
            S.solve(bs[k], out=xp[k])
            S.refine(bs[k], xp[k], 1e-14, 20)
            S.solve_transpose(gs[k], out=lams[k])
    tp = _time_ms(run_plain, reps=2)
    return {"us_per_system": tq * 1e3 / len(seqs), "plain_fp64_us_per_system": tp * 1e3 / len(seqs),
            "speedup_vs_plain": tp / tq, "systems": len(seqs), "omega_max": worst,
            "finished_outside_graph": state.get("late"), "launch_shape": list(best),
            "tuning_ms": {f"{w}x{c}": t * 1e3 for (w, c), t in (table or {}).items()}}


def run_variants(dev):
    """The batched and FP32 forms against the plain FP64 path on the same GPU,
    all refined to scaled residual <= 1e-14 (per system, microseconds):
      batched: 64 scenario systems of the 10,000-bus grid (loads scaled by
               U(0.8, 1.2)), one batched refactor + solve + refine;
      fp32:    the 70,000-bus late-IPM system, FP32 factors + FP64 refinement."""
    import torch
    from kktgen import config_sequence
    from paper_2306_14337_gb300 import KKTSolver
    res = {}
    # batched, 10,000-bus x 64
    s = config_sequence(2)
    k, B = 2, 64
    vals = torch.tensor(np.stack([s.values(k, sc) for sc in range(1, B + 1)], axis=1), device=dev)
    bs = torch.tensor(np.stack([s.csr(k, sc) @ s.x_true(k, sc) for sc in range(1, B + 1)], axis=1),
                      device=dev)
    Sb = KKTSolver(s.n, s.indptr, s.indices, max_batch=B)
    xb = torch.empty_like(bs)
    info = {}

    def batched():
        Sb.batch_refactor(vals)
        Sb.batch_solve(bs, out=xb)
        info["r"] = Sb.batch_refine(bs, xb, 1e-14, 40)
    tb = _time_ms(batched)
    S1 = KKTSolver(s.n, s.indptr, s.indices)
    v1 = vals[:, 0].contiguous()
    b1 = bs[:, 0].contiguous()
    x1 = torch.empty_like(b1)
    info1 = {}

    def plain():
        S1.refactor(v1)
        S1.solve(b1, out=x1)
        info1["r"] = S1.refine(b1, x1, 1e-14, 20)
    tp = _time_ms(plain)
    res["batched_10000bus_x64_fp64"] = {
        "us_per_system": tb * 1e3 / B, "plain_fp64_us_per_system": tp * 1e3,
        "speedup_vs_plain": tp * B / tb, "omega_max": float(np.max(info["r"]["omega"])),
        "refine_iters": info["r"]["iters"], "n": s.n, "batch": B}
    del Sb, S1, vals, bs
    # FP32 factors + FP64 refinement, 70,000-bus
    s = config_sequence(3)
    v = torch.tensor(s.values(0), device=dev)
    b = torch.tensor(s.rhs(0), device=dev)
    out = {}
    for fp32 in (True, False):
        S = KKTSolver(s.n, s.indptr, s.indices, fp32=fp32, refine_mode="auto")
        x = torch.empty_like(b)
        inf = {}

        def run():
            S.refactor(v)
            S.solve(b, out=x)
            inf["r"] = S.refine(b, x, 1e-14, 20)
        t = _time_ms(run, reps=2)
        out["fp32" if fp32 else "fp64"] = (t, inf["r"], S.stats())
        del S
    t32, r32, st = out["fp32"]
    t64, r64, _ = out["fp64"]
    res["uneven_48_fp32_queue"] = run_uneven(dev)
    res["fp32_refined_70000bus"] = {
        "us_per_system": t32 * 1e3, "plain_fp64_us_per_system": t64 * 1e3,
        "speedup_vs_plain": t64 / t32, "omega": r32["omega"], "refine_iters": r32["iters"],
        "fp64_omega": r64["omega"], "n": s.n, "nnz_lu": st["nnz_lu"], "levels": st["n_levels"],
        "hbm_gbs_refactor_solve_fp32": (st["bytes_refactor"] + st["bytes_solve"]) / (t32 * 1e-3) / 1e9}
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="2000bus_fp64_adjoint")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the batched and FP32 comparisons (about a minute)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    ws, rank, local = _dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_native(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
