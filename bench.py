#!/usr/bin/env python3
"""Benchmark of the fixed-pattern KKT refactorization path on GB300.

Workload (default): the 70,000-bus late-IPM system with FP32 factors and FP64
refinement (KKT dimension 490,000, 4,914,000 stored entries, 4 value sets with
D_x, D_s log-uniform in [1e-8, 1e8]), the largest single-GPU configuration.
The values are symmetric (Eq. 4), so the FP32 factors are computed in the
LDL^T form (same storage and solves as LU, half the refactorization's
arithmetic), with the dense root block factored by k_dense_lu.
``--workload 2000bus_fp64_adjoint`` runs the 2,000-bus plain FP64 sequence
(n = 14,000, 30 value sets).  One step is one KKT system through the whole
path: refactorization, solve, iterative refinement to scaled residual 1e-14,
transposed solve with its refinement, and the adjoint gather (the backward of
x = A^-1 b).  All value sets, right-hand sides and upstream gradients are
resident in HBM before the timed region; L2 is flushed between timed steps
(a 256 MiB write, outside the per-step events).

Metric: microseconds per KKT system (lower is better) and HBM GB/s.  The
``e2e`` figure runs the same step from pinned host buffers through the C
interface, copies included.  ``--impl reference`` times the CPU oracle on the
host cores on the same workload (a bounded sample: whole systems until a CPU
time budget is spent).

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
    # the KKT values are symmetric (Eq. 4): the FP32 factors are the LDL^T form
    # (the same L and U storage; half the refactorization's arithmetic);
    # refinement by FGMRES with the factors as preconditioner (Sec. 5.1), which
    # needs fewer solves than classic refinement with these FP32 factors
    "70000bus_fp32_refined": dict(cfg=3, fp32=True, refine="fgmres", symmetric=True),
    # the same form on the 10,000-bus grid (a smaller case of the same kernels)
    "10000bus_fp32_refined": dict(cfg=2, fp32=True, refine="fgmres", symmetric=True),
    "2000bus_fp64_adjoint": dict(cfg=1, fp32=False, refine="classic"),
    "200bus_fp64": dict(cfg=0, fp32=False, refine="classic"),
    # 64 scenario systems of the 10,000-bus grid, batched; sharded across
    # ranks by contiguous slices (total work fixed: strong scaling)
    "10000bus_x64_batched": dict(cfg=2, fp32=False, refine="classic", batched=64),
}
DEFAULT_WORKLOAD = "70000bus_fp32_refined"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
HBM_FALLBACK_GBS = 6800.0
# nominal non-tensor FMA rates of GB300 (152 SMs at 2.07 GHz): FP32 128 lanes
# per SM, FP64 2 lanes per SM (x 2 flops per FMA); the bench measures its own
FMA_NOMINAL_TFLOPS = {"f32": 152 * 128 * 2 * 2.07e9 / 1e12, "f64": 152 * 2 * 2 * 2.07e9 / 1e12}


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
    for f in ("kkt.cu", "kernels.cuh", "dense.cu"):
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
def oracle_sample(seq, step_ids, budget_s: float, refine_mode: str = "auto", keep_first=False, perm=None):
    """Time the oracle (as it stands, single-threaded) on whole steps of the
    workload -- factorization, solve, refinement, transposed solve with its
    refinement, adjoint -- until ``budget_s`` seconds of CPU work are spent.
    The ordering is computed once outside the timing (the symbolic phase, as
    for the GPU).  Returns (us per system, systems timed, results of the first
    step: x and lambda, refined to 1e-14, or None)."""
    import oracle
    if perm is None:
        perm = oracle.min_degree(seq.n, seq.indptr, seq.indices)
    done, t_total, first = 0, 0.0, None
    for k in step_ids:
        v, b = seq.values(k), seq.rhs(k)
        g = np.random.default_rng(1234 + k).standard_normal(seq.n)
        t0 = time.perf_counter()
        o = oracle.Oracle(seq.n, seq.indptr, seq.indices, v, perm)
        x, *_ = o.refine(b, x0=o.solve(b), mode=refine_mode)
        # transposed solve, refined classically with the same factors
        At = seq.csr(k).T.tocsr()
        lam = o.solve_t(g)
        for _ in range(20):
            if oracle.omega(seq.n, At.indptr, At.indices, At.data, g, lam) <= 1e-14:
                break
            lam = lam + o.solve_t(oracle.residual(seq.n, At.indptr, At.indices, At.data, g, lam))
        o.adjoint(x, g)
        t_total += time.perf_counter() - t0
        if keep_first and first is None:
            first = {"k": k, "x": x, "lam": lam}
        done += 1
        if t_total >= budget_s:
            break
    return t_total * 1e6 / max(done, 1), done, first


def _oracle_omega_pool(args_list):
    """Worker of the all-cores oracle timing (one system per task, spawn pool)."""
    import oracle
    n, rp, ci, v, b, perm = args_list
    t0 = time.perf_counter()
    o = oracle.Oracle(n, rp, ci, v, perm)
    x, *_ = o.refine(b, x0=o.solve(b))
    return time.perf_counter() - t0


def oracle_all_cores(systems, budget_s: float):
    """Independent systems (n, rp, ci, values, b) through the oracle (factor,
    solve, refine) on every host core with a spawn process pool, until about
    ``budget_s`` of wall time: (us per system of wall time, systems, cores)."""
    import multiprocessing as mp
    import oracle
    cores = len(os.sched_getaffinity(0))
    perms = {}
    tasks = []
    for (n, rp, ci, v, b) in systems:
        key = (n, len(ci), int(rp[-1]), int(ci[:64].sum()))
        if key not in perms:
            perms[key] = oracle.min_degree(n, rp, ci)
        tasks.append((n, rp, ci, v, b, perms[key]))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    done = 0
    with ctx.Pool(cores) as pool:
        for _ in pool.imap_unordered(_oracle_omega_pool, tasks):
            done += 1
            if time.perf_counter() - t0 > budget_s:
                pool.terminate()
                break
    wall = time.perf_counter() - t0
    return wall * 1e6 / max(done, 1), done, cores


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args, ws, rank):
    """--impl reference: the CPU oracle on the host cores, same metric and
    workload.  A step is one whole system; warm-up steps and timed steps each
    stop at a CPU-time budget (one system at least), so the run ends within a
    few minutes also on the 490,000-row workload (about 20-40 s per system)."""
    if rank != 0:
        return 0
    from kktgen import config_sequence
    wl = WORKLOADS[args.workload]
    seq = config_sequence(wl["cfg"])
    import oracle
    ids = [k % seq.steps for k in range(args.warmup + args.steps)]
    perm = oracle.min_degree(seq.n, seq.indptr, seq.indices)       # symbolic: outside the timing
    if wl.get("batched"):
        # a step is the scenarios of one IPM value set: factor, solve, refine each
        def scen_sample(budget):
            t_tot, done = 0.0, 0
            for it in range(args.warmup + args.steps):
                k = it % seq.steps
                for sc in range(1, wl["batched"] + 1):
                    v, rhs = seq.values(k, sc), seq.csr(k, sc) @ seq.x_true(k, sc)
                    t0 = time.perf_counter()
                    o = oracle.Oracle(seq.n, seq.indptr, seq.indices, v, perm)
                    o.refine(rhs, x0=o.solve(rhs))
                    t_tot += time.perf_counter() - t0
                    done += 1
                    if t_tot >= budget:
                        return t_tot * 1e6 / done, done
            return t_tot * 1e6 / max(done, 1), done
        scen_sample(min(args.cpu_budget, 10.0))
        us, done = scen_sample(args.ref_budget)
        sample = (f"{done} scenario systems (factor, solve, refine) of the {args.workload} sequence, "
                  f"single-threaded, bounded at {args.ref_budget:.0f} s of CPU time; warm-up bounded at 10 s")
    else:
        oracle_sample(seq, ids[: args.warmup], min(args.cpu_budget, 10.0), wl["refine"], perm=perm)
        us, done, _ = oracle_sample(seq, ids[args.warmup:], args.ref_budget, wl["refine"], perm=perm)
        sample = (f"{done} of the {args.steps} requested steps (whole systems: refactor, solve, refine, "
                  f"transposed solve + refine, adjoint) of the {args.workload} sequence, single-threaded, "
                  f"bounded at {args.ref_budget:.0f} s of CPU time; warm-up bounded at 10 s")
    cores = 1
    line = {
        "impl": "reference", "metric": METRIC, "value": us, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": us / 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": seq.n, "nnz": seq.nnz, "value_sets": seq.steps,
                   "l2": "host cores (no GPU cache)", "parallelism": "one host core"},
        "cpu_baseline": {"value": us, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model()},
        "e2e": {"value": us, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def probe_fma(dev_index):
    """Measured FMA rates (TFLOP/s) of this GPU from the library's probe."""
    import ctypes as C
    from paper_2306_14337_gb300 import _capi
    L = _capi.load()
    out = {}
    for key, fp64 in (("f32", 0), ("f64", 1)):
        v = C.c_double(0.0)
        if L.kkt_probe_fma_tflops(int(dev_index), fp64, C.byref(v)) == 0:
            out[key] = v.value
    return out


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ----------------------------------------------------------------- GPU leg, batched
def run_native_batched(args, ws, rank, local):
    """The 64 scenarios of the 10,000-bus grid, this rank's contiguous slice
    as one batch (batch innermost): per step one IPM value set through
    batched refactorization, solve and refinement to 1e-14.  No collective on
    the data path; between steps the ranks meet at a host step barrier on the
    rendezvous store (a rank that left is reported before the next launch)."""
    import torch
    from kktgen import config_sequence
    from paper_2306_14337_gb300 import KKTSolver
    from paper_2306_14337_gb300.shard import contiguous_slice, step_barrier

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    store = None
    if ws > 1:
        dist = _init_dist(ws, "nccl")
        try:
            store = dist.distributed_c10d._get_default_store()
        except Exception:
            store = None
    wl = WORKLOADS[args.workload]
    total = wl["batched"]
    a, b = contiguous_slice(total, rank, ws)
    B = b - a
    seq = config_sequence(wl["cfg"])
    n, nnz, K = seq.n, seq.nnz, seq.steps
    scen = list(range(a + 1, b + 1))          # scenario 0 is the unscaled base case
    vals = [torch.tensor(np.stack([seq.values(k, sc) for sc in scen], axis=1), device=dev) for k in range(K)]
    bs = [torch.tensor(np.stack([seq.csr(k, sc) @ seq.x_true(k, sc) for sc in scen], axis=1), device=dev)
          for k in range(K)]
    S = KKTSolver(n, seq.indptr, seq.indices, max_batch=B, device=local)
    x = torch.empty_like(bs[0])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(k, ev=None):
        if ev is not None:
            ev[0].record(stream)
        S.batch_refactor(vals[k])
        if ev is not None:
            ev[1].record(stream)
        S.batch_solve(bs[k], out=x)
        r = S.batch_refine(bs[k], x, 1e-14, 40)
        if ev is not None:
            ev[2].record(stream)
        return r

    for w in range(args.warmup):
        step(w % K)
    torch.cuda.synchronize()
    launches0 = S.stats()["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    ref_ms, step_ms, omega = [], [], 0.0
    for it in range(args.steps):
        k = (args.warmup + it) % K
        if store is not None:
            step_barrier(store, rank, ws, it)
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        r = step(k, ev)
        torch.cuda.synchronize()
        ref_ms.append(ev[0].elapsed_time(ev[1]))
        step_ms.append(ev[0].elapsed_time(ev[2]))
        omega = max(omega, float(np.max(r["omega"])))
        if not r["converged"]:
            raise SystemExit(f"batched refinement did not converge at step {k}")
    torch.cuda.synchronize()
    barrier(ws)
    launches = S.stats()["kernel_launches"] - launches0
    total_s = reduce_max(sum(step_ms) / 1e3, ws, dev)
    clk = clocks.stop()
    # e2e: this rank's slice from pinned host memory, x back
    hv = [v.cpu().pin_memory() for v in vals]
    hb = [t.cpu().pin_memory() for t in bs]
    dv, db_ = torch.empty_like(vals[0]), torch.empty_like(bs[0])
    hx = torch.empty(x.shape, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for it in range(args.steps):
        k = (args.warmup + it) % K
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dv.copy_(hv[k], non_blocking=True)
        db_.copy_(hb[k], non_blocking=True)
        S.batch_refactor(dv)
        S.batch_solve(db_, out=x)
        S.batch_refine(db_, x, 1e-14, 40)
        hx.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_s = reduce_max(sum(e2e_ms) / 1e3, ws, dev)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        perm = oracle.min_degree(n, seq.indptr, seq.indices)
        t_tot, done = 0.0, 0
        for sc in scen:
            v, rhs = seq.values(0, sc), seq.csr(0, sc) @ seq.x_true(0, sc)
            t0 = time.perf_counter()
            o = oracle.Oracle(n, seq.indptr, seq.indices, v, perm)
            o.refine(rhs, x0=o.solve(rhs))
            t_tot += time.perf_counter() - t0
            done += 1
            if t_tot >= args.cpu_budget:
                break
        cpu = {"value": t_tot * 1e6 / done, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": cpu_model(),
               "sample": f"{done} scenario systems (factor, solve, refine), single-threaded, ordering "
                         f"computed once outside the timing"}
    if rank != 0:
        return 0
    st = S.stats()
    peak_hbm, peak_kind = load_peaks()
    fma = probe_fma(local)
    t_ref = statistics.mean(ref_ms) * 1e-3
    by = st["bytes_refactor"] * B
    achieved = by / t_ref / 1e9
    line = {
        "metric": METRIC, "value": total_s * 1e6 / (args.steps * total), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
        "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "nnz": nnz, "systems_per_step": total,
                   "systems_per_rank": [contiguous_slice(total, r, ws)[1] - contiguous_slice(total, r, ws)[0]
                                        for r in range(ws)],
                   "value_sets": K, "l2": "flushed between timed steps (256 MiB write, outside the step events)",
                   "parallelism": f"scenario shards x{ws} (contiguous slices, no collective on the data path)"},
        "breakdown_ms": {"refactor": statistics.mean(ref_ms), "step": statistics.mean(step_ms)},
        "omega_max": omega,
        "roofline": {"bound": "hbm", "kernel": "k_brefactor<double> (+k_bscale, k_bamax)",
                     "achieved": achieved, "peak": peak_hbm, "unit": "GB/s", "frac": achieved / peak_hbm,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                     "algorithmic_bytes_per_launch": by, "traffic": None,
                     "alu_achieved_tflops": st["flops_refactor"] * B / t_ref / 1e12,
                     "alu_peak_tflops": fma.get("f64", FMA_NOMINAL_TFLOPS["f64"]),
                     "alu_frac": st["flops_refactor"] * B / t_ref / 1e12 / fma.get("f64", FMA_NOMINAL_TFLOPS["f64"])},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_s * 1e6 / (args.steps * total), "unit": UNIT,
                "h2d_bytes_per_step": 8 * B * (nnz + n), "d2h_bytes_per_step": 8 * B * n},
        "gpu_launches": int(launches),
        "clocks": clk,
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
    S = KKTSolver(n, seq.indptr, seq.indices, fp32=wl["fp32"], refine_mode=wl["refine"],
                  symmetric=wl.get("symmetric", False), solve_far_blocks=args.solve_far_blocks,
                  solve_far_ctas=args.solve_far_ctas, device=local)
    dname = "f32" if wl["fp32"] else "f64"
    rng = np.random.default_rng(1234 + rank)
    vals = [torch.tensor(seq.values(k), device=dev) for k in range(K)]
    bs = [torch.tensor(seq.rhs(k), device=dev) for k in range(K)]
    gs = [torch.tensor(np.random.default_rng(1234 + k).standard_normal(n), device=dev) for k in range(K)]
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
    launches = S.stats()["kernel_launches"] - launches0
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

    # the GPU's results for value set 0, kept for the FP64-oracle comparison
    step(0)
    torch.cuda.synchronize()
    x0, lam0 = x.cpu().numpy().copy(), lam.cpu().numpy().copy()

    # CPU baseline (rank 0, N = 1 only): the oracle on a bounded sample, whose
    # first system (value set 0) is also the FP64 reference of the results
    cpu, oracle_err = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        us_cpu, done, first = oracle_sample(seq, list(range(K)), args.cpu_budget, wl["refine"], keep_first=True)
        cpu = {"value": us_cpu, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": cpu_model(),
               "sample": f"{done} whole system(s) (refactor, solve, refine, transposed solve + refine, "
                         f"adjoint) of the {args.workload} sequence, single-threaded, ordering computed "
                         f"once outside the timing, bounded at {args.cpu_budget:.0f} s of CPU time"}
        At = seq.csr(0).T.tocsr()
        oracle_err = {
            "value_set": 0,
            "x_rel_err_inf": _relerr(x0, first["x"]), "lambda_rel_err_inf": _relerr(lam0, first["lam"]),
            "omega_x_by_oracle": oracle.omega(n, seq.indptr, seq.indices, seq.values(0), seq.rhs(0), x0),
            "omega_lambda_by_oracle": oracle.omega(n, At.indptr, At.indices, At.data,
                                                   np.random.default_rng(1234).standard_normal(n), lam0),
            "note": "both solutions are refined to omega <= 1e-14 (the backward error both methods "
                    "control); their distance is bounded only by cond(A) * 1e-14, and with D over 16 "
                    "decades cond(A) * 1e-14 exceeds 1 on this system, so x itself is not fixed by FP64"}

    variants = {}
    if rank == 0 and not args.no_variants:
        variants = run_variants(dev, with_oracle=not args.no_cpu_baseline, budget=args.cpu_budget)

    if rank != 0:
        return 0
    us = whole_job_us_per_system(total_s, args.steps, ws)
    ph_ms = {k: statistics.mean(v) for k, v in phase.items()}
    st = S.stats()
    peak_hbm, peak_kind = load_peaks()
    fma = probe_fma(local)
    alu_peak = fma.get(dname, FMA_NOMINAL_TFLOPS[dname])
    # dominant kernel: the refactorization (k_refactor; k_scale, k_amax and
    # k_pack_tiles share its events and are a few percent of it)
    t_ref = ph_ms["refactor"] * 1e-3
    by_ref = st["bytes_refactor"]
    achieved = by_ref / t_ref / 1e9
    tname = 'float' if wl['fp32'] else 'double'
    roof = {"bound": "hbm", "kernel": f"k_refactor<{tname}>"
                                      + (f" + k_dense_lu<{tname}>" if st["dense_rows"] else "")
                                      + " (+k_scale, k_amax, k_pack_tiles in the same events)",
            "achieved": achieved, "peak": peak_hbm, "unit": "GB/s", "frac": achieved / peak_hbm,
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_launch": by_ref,
            "traffic": committed_traffic(f"k_refactor_{dname}", args.workload),
            "alu_achieved_tflops": st["flops_refactor"] / t_ref / 1e12, "alu_peak_tflops": alu_peak,
            "alu_frac": st["flops_refactor"] / t_ref / 1e12 / alu_peak,
            "alu_peak_source": ("measured by kkt_probe_fma_tflops on this GPU" if dname in fma
                                else "nominal")}
    rs_s = (ph_ms["refactor"] + ph_ms["solve"]) * 1e-3
    rs_bytes = st["bytes_refactor"] + st["bytes_solve"]
    line = {
        "metric": METRIC, "value": us, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": dname, "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "nnz": nnz, "nnz_lu": st["nnz_lu"],
                   "levels": st["n_levels"], "value_sets": K, "dense_rows": st["dense_rows"],
                   "solve_partner_ctas": st["solve_far_ctas"], "solve_far_rows": st["solve_far_rows"],
                   "factors": ("FP32, FP64 residual/refinement/pivot test" if wl["fp32"] else "FP64")
                              + (", LDL^T of the symmetric values" if wl.get("symmetric") else ", LU"),
                   "refine": wl["refine"],
                   "l2": "flushed between timed steps (256 MiB write, outside the step events)",
                   "parallelism": f"replicas x{ws}"},
        "breakdown_ms": ph_ms,
        "refactor_solve_us": rs_s * 1e6,
        "refactor_solve_hbm_gbs": rs_bytes / rs_s / 1e9,
        "refactor_solve_hbm_frac": rs_bytes / rs_s / 1e9 / peak_hbm,
        "refine_iters": {"solve": statistics.mean(i[0] for i in iters),
                         "transpose": statistics.mean(i[1] for i in iters)},
        "omega_max": max(omegas), "status": int(st_code), "perturbed_pivots": npert,
        "roofline": roof,
        "fma_probe_tflops": fma,
        # Why the fraction is low: the refactorization is a chain of dependent
        # rows, one hand-off per level of the elimination DAG.
        "critical_path": {"refactor_levels": st["n_levels"],
                          "refactor_us_per_level": ph_ms["refactor"] * 1e3 / st["n_levels"],
                          "solve_levels": {"forward": st["n_levels"], "backward": st["n_levels_u"]},
                          "solve_tasks": st["n_tasks"], "longest_task_rows": st["max_task"]},
        "oracle_error": oracle_err,
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


def run_uneven(dev, with_oracle=True, budget=15.0):
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
    sols = [KKTSolver(s.n, s.indptr, s.indices, fp32=True, refine_mode="fgmres") for s in seqs]
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
    out = {"us_per_system": tq * 1e3 / len(seqs), "plain_fp64_us_per_system": tp * 1e3 / len(seqs),
           "speedup_vs_plain": tp / tq, "systems": len(seqs), "omega_max": worst,
           "finished_outside_graph": state.get("late"), "launch_shape": list(best),
           "tuning_ms": {"x".join(str(v) for v in cand): t * 1e3 for cand, t in (table or {}).items()}}
    if with_oracle:
        import oracle
        # FP64-oracle error of the solution of one system of each size
        errs = {}
        run()
        for k in (0, 16, 32, 44):
            q = seqs[k]
            sols[k].refine(bs[k], xs[k], 1e-14, 20)
            o = oracle.Oracle(q.n, q.indptr, q.indices, q.values(0), oracle.min_degree(q.n, q.indptr, q.indices))
            xo, *_ = o.refine(q.rhs(0))
            xh = xs[k].cpu().numpy()
            errs[f"n{q.n}"] = {"x_rel_err_inf": _relerr(xh, xo),
                               "omega_x_by_oracle": oracle.omega(q.n, q.indptr, q.indices, q.values(0),
                                                                 q.rhs(0), xh)}
        out["oracle_error"] = errs
        us_all, done, cores = oracle_all_cores(
            [(q.n, q.indptr, q.indices, q.values(0), q.rhs(0)) for q in seqs], budget)
        out["cpu_baseline_all_cores"] = {
            "value": us_all, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{done} of the 48 systems (factor, solve, refine), one per process, spawn pool, "
                      f"wall time per system"}
    return out


def run_variants(dev, with_oracle=True, budget=15.0):
    """The batched and FP32 forms against the plain FP64 path on the same GPU,
    all refined to scaled residual <= 1e-14 (per system, microseconds):
      batched: 64 scenario systems of the 10,000-bus grid (loads scaled by
               U(0.8, 1.2)), one batched refactor + solve + refine per IPM step,
               5 steps;
      fp32:    the 70,000-bus late-IPM system, FP32 factors + FP64 refinement,
               against plain FP64 factors;
      uneven:  the 48 systems of different patterns in one work queue;
      2000bus: the 2,000-bus plain FP64 step of the adjoint workload.
    With the oracle: the FP64-oracle error of sampled results and the oracle
    timed on all host cores for the batched and uneven forms."""
    import torch
    from kktgen import config_sequence
    from paper_2306_14337_gb300 import KKTSolver
    res = {}
    # batched, 10,000-bus x 64, all 5 IPM steps of the sequence
    s = config_sequence(2)
    B = 64
    steps = list(range(s.steps))
    vals = [torch.tensor(np.stack([s.values(k, sc) for sc in range(1, B + 1)], axis=1), device=dev)
            for k in steps]
    bs = [torch.tensor(np.stack([s.csr(k, sc) @ s.x_true(k, sc) for sc in range(1, B + 1)], axis=1),
                       device=dev) for k in steps]
    Sb = KKTSolver(s.n, s.indptr, s.indices, max_batch=B)
    xb = torch.empty_like(bs[0])
    info = {"omega": 0.0, "iters": []}

    def batched():
        for k in steps:
            Sb.batch_refactor(vals[k])
            Sb.batch_solve(bs[k], out=xb)
            r = Sb.batch_refine(bs[k], xb, 1e-14, 40)
            info["omega"] = max(info["omega"], float(np.max(r["omega"])))
            info["iters"].append(r["iters"])
    tb = _time_ms(batched)
    S1 = KKTSolver(s.n, s.indptr, s.indices)
    x1 = torch.empty(s.n, dtype=torch.float64, device=dev)
    v1 = [vals[k][:, 0].contiguous() for k in steps]
    b1 = [bs[k][:, 0].contiguous() for k in steps]
    info1 = {}

    def plain():
        for k in steps:
            S1.refactor(v1[k])
            S1.solve(b1[k], out=x1)
            info1["r"] = S1.refine(b1[k], x1, 1e-14, 20)
    tp = _time_ms(plain)
    nsys = B * len(steps)
    bat = {"us_per_system": tb * 1e3 / nsys, "plain_fp64_us_per_system": tp * 1e3 / len(steps),
           "speedup_vs_plain": (tp / len(steps)) / (tb / nsys), "omega_max": info["omega"],
           "refine_iters": info["iters"][-len(steps):], "n": s.n, "batch": B, "ipm_steps": len(steps)}
    if with_oracle:
        import oracle
        k = steps[-1]
        xh = xb.cpu().numpy()
        v0, b0 = vals[k][:, 0].cpu().numpy(), bs[k][:, 0].cpu().numpy()
        o = oracle.Oracle(s.n, s.indptr, s.indices, v0, oracle.min_degree(s.n, s.indptr, s.indices))
        xo, *_ = o.refine(b0)
        bat["oracle_error"] = {"scenario": 0, "ipm_step": k, "x_rel_err_inf": _relerr(xh[:, 0], xo),
                               "omega_x_by_oracle": oracle.omega(s.n, s.indptr, s.indices, v0, b0, xh[:, 0])}
        us_all, done, cores = oracle_all_cores(
            [(s.n, s.indptr, s.indices, vals[k][:, j].cpu().numpy(), bs[k][:, j].cpu().numpy())
             for j in range(B)], budget)
        bat["cpu_baseline_all_cores"] = {
            "value": us_all, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{done} of the 64 scenario systems of the last IPM step (factor, solve, refine), "
                      f"one per process, spawn pool, wall time per system"}
    res["batched_10000bus_x64_fp64"] = bat
    del Sb, S1, vals, bs
    # FP32 factors + FP64 refinement against plain FP64, 70,000-bus
    s = config_sequence(3)
    v = torch.tensor(s.values(0), device=dev)
    b = torch.tensor(s.rhs(0), device=dev)
    out = {}
    for fp32 in (True, False):
        S = KKTSolver(s.n, s.indptr, s.indices, fp32=fp32, refine_mode="fgmres")
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
    res["fp32_refined_70000bus"] = {
        "us_per_system": t32 * 1e3, "plain_fp64_us_per_system": t64 * 1e3,
        "speedup_vs_plain": t64 / t32, "omega": r32["omega"], "refine_iters": r32["iters"],
        "fp64_omega": r64["omega"], "n": s.n, "nnz_lu": st["nnz_lu"], "levels": st["n_levels"]}
    # symmetric values: LDL^T refactorization (same storage and solves) with inertia
    ld = {}
    for fp32 in (False, True):
        S = KKTSolver(s.n, s.indptr, s.indices, fp32=fp32, refine_mode="fgmres", symmetric=True)
        x = torch.empty_like(b)
        inf = {}

        def run_ld():
            S.refactor(v)
            S.solve(b, out=x)
            inf["r"] = S.refine(b, x, 1e-14, 20)
        t = _time_ms(run_ld, reps=2)
        tr = _time_ms(lambda: S.refactor(v), reps=3)
        pos, neg, pert = S.inertia()
        ld["fp32" if fp32 else "fp64"] = {
            "us_per_system": t * 1e3, "refactor_us": tr * 1e3, "omega": inf["r"]["omega"],
            "refine_iters": inf["r"]["iters"], "inertia": {"positive": pos, "negative": neg,
                                                           "perturbed": pert}}
        del S
    ld["speedup_vs_plain_fp64_lu"] = t64 / (ld["fp64"]["us_per_system"] / 1e3)
    ld["n_x"] = 2 * s.grid.nb + 2 * s.grid.ng
    res["ldlt_symmetric_70000bus"] = ld
    del v, b
    res["uneven_48_fp32_queue"] = run_uneven(dev, with_oracle, budget)
    # the 2,000-bus FP64 step (refactor, solve, refine, transposed solve + refine, adjoint)
    s = config_sequence(1)
    S = KKTSolver(s.n, s.indptr, s.indices)
    v = torch.tensor(s.values(29), device=dev)
    b = torch.tensor(s.rhs(29), device=dev)
    g = torch.tensor(np.random.default_rng(5).standard_normal(s.n), device=dev)
    x, lam = torch.empty_like(b), torch.empty_like(b)
    dA = torch.empty(s.nnz, dtype=torch.float64, device=dev)

    def step2k():
        S.refactor(v)
        S.solve(b, out=x)
        S.refine(b, x, 1e-14, 20)
        S.solve_transpose(g, out=lam)
        S.refine_transpose(g, lam, 1e-14, 20)
        S.adjoint_gather(lam, x, out=dA)
    res["fp64_adjoint_2000bus"] = {"us_per_system": _time_ms(step2k, reps=10) * 1e3, "n": s.n}
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work per CPU leg")
    ap.add_argument("--ref-budget", type=float, default=60.0,
                    help="--impl reference: seconds of oracle work over the timed steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the batched and FP32 comparisons (about a minute)")
    ap.add_argument("--solve-far-blocks", type=int, default=0,
                    help="single-system workloads: the library option solve_far_blocks (0: its default, "
                         "-1: no partner CTAs)")
    ap.add_argument("--solve-far-ctas", type=int, default=0,
                    help="single-system workloads: the library option solve_far_ctas (0: its default)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    ws, rank, local = _dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if WORKLOADS[args.workload].get("batched"):
        return run_native_batched(args, ws, rank, local)
    return run_native(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
