"""Benchmark of the learned-preconditioner PCG hot path on one GB300.

Metric: ms to a 1e-6 relative residual per system, learned-L PCG (graph
network factor + PCG, the paper's "precompute + solve" total, Sec. 5.1
"Evaluation Metrics") next to IC(0)-PCG on the same GPU; secondary: SpTRSV
bandwidth against the HBM roofline.

Default workload (one step = one system): 3-D variable-coefficient
diffusion, 7-point finite differences on a 128^3 grid (n = 2,097,152,
nnz = 14,581,760), log k a GRF (sigma 1.5, correlation 0.05), b ~ N(0,1);
6-layer hidden-64 network on the BF16 tensor cores; FP64 PCG to 1e-6 with
FP32 triangular solves.  Inputs are resident in HBM when the timed region
starts (the pattern is analysed once: a fixed mesh, as in the paper's
environments; the analysis is timed separately as analyse_ms); L2 is flushed
between steps.  Other workloads: --workload fem2d_256 (2-D FEM, n = 64,516),
batched_256 (256 uneven systems in one batched solve), heat2d_256 (implicit
heat step), train_32 (one training step).

--impl reference times the CPU oracle (the method's plain FP64 restatement)
on the host cores on a bounded sample of the same workload.
Multi-GPU (torchrun): a single-system workload runs one replica per rank
(independent systems seeded by rank, no collective on the data path: weak
scaling); batched_256 splits its one fixed batch of 256 systems over the
ranks by a greedy bin-pack on the nonzeros (strong scaling) and gathers the
per-system statistics to rank 0 in the batch's order.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WEIGHTS_DIR = os.path.join(ROOT, "paper_2305_16432_gb300", "weights")
METRIC = "ms to 1e-6 rel. residual per system (learned vs IC(0) PCG); SpTRSV HBM GB/s"
RTOL = 1e-6
WORKLOAD_LABEL = {"fem2d_256": "fem2d_256_learned_pcg", "fd3d_128": "fd3d_128_learned_pcg",
                  "batched_256": "batched_256_learned_pcg", "heat2d_256": "heat2d_256_learned_pcg"}
SOLVE_WORKLOADS = tuple(WORKLOAD_LABEL)
L2_FLUSH = "flushed between steps (256 MB write)"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1906.5)), "measured"
    return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# the network trained for each workload's family (the paper trains one per
# task); the mixed 2-D / 3-D network serves the uneven batch and is the fallback
TASK_WEIGHTS = {"fem2d_256": "gnn_6x64_fem2d.npy", "fd3d_128": "gnn_6x64_fd3d.npy", "batched_256": "gnn_6x64.npy",
                "heat2d_256": "gnn_6x64_heat2d.npy"}


def weights_for(workload, x0=False):
    name = TASK_WEIGHTS.get(workload, "gnn_6x64.npy")
    if x0:
        # the same network with a trained initial-guess head
        name = name.replace(".npy", "_x0.npy")
    p = os.path.join(WEIGHTS_DIR, name)
    return p if os.path.exists(p) else os.path.join(WEIGHTS_DIR, "gnn_6x64.npy")


def _load_weights(cfg, path):
    from paper_2305_16432_gb300 import inputs as I
    if path and os.path.exists(path):
        w = np.load(path).astype(np.float32)
        meta = {}
        mp = os.path.splitext(path)[0] + ".json"
        if os.path.exists(mp):
            meta = json.load(open(mp))
        if meta.get("config"):
            cfg = I.GnnConfig(**meta["config"])
        if len(w) == cfg.nparams:
            return w, "trained", meta, cfg
    return I.gnn_weights(cfg, 1), "random-init", {}, cfg


# ------------------------------------------------------------------ sharding
def nnz_estimate(prob) -> int:
    """Nonzeros of a synthetic system from its shape alone (no assembly):
    exact for the FD stencils, 7 per unknown for the FEM lattices (six
    neighbours and the diagonal of an interior lattice node)."""
    from paper_2305_16432_gb300 import inputs as I
    if prob.kind == I.FD:
        nx, ny, nz = prob.nx, prob.ny, (prob.nz if prob.dim == 3 else 1)
        faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + (nx * ny * (nz - 1) if prob.dim == 3 else 0)
        return prob.n + 2 * faces
    return 7 * prob.n


def partition_by_nnz(weights, world):
    """Greedy bin-pack of systems onto ranks: the heaviest system first, each
    into the currently lightest shard (ties to the lower rank).  Returns the
    sorted system indices of every rank's shard."""
    order = sorted(range(len(weights)), key=lambda k: (-weights[k], k))
    load = [0] * world
    shards = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        shards[r].append(k)
        load[r] += weights[k]
    return [sorted(s) for s in shards]


def gather_stats(local, shard, nsys, world):
    """Per-system statistics of every rank's shard, back in batch order (on
    every rank; the one collective of the batched path, after the timing)."""
    if world <= 1:
        return list(local)
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, (list(shard), list(local)))
    out = [None] * nsys
    for sh, st in parts:
        for k, s in zip(sh, st):
            out[k] = s
    return out


def _problems(I, workload, rank, world):
    """(systems this rank solves, their indices in the workload's batch).
    A single-system workload gives every rank its own system seeded by rank
    (independent replicas); the batch is one fixed set of 256 systems split
    by partition_by_nnz."""
    if workload == "fem2d_256":
        return [I.fem2d_256(seed=rank)], [0]
    if workload == "fd3d_128":
        return [I.fd3d_128(seed=rank)], [0]
    if workload == "heat2d_256":
        return [I.heat2d(256, seed=rank)], [0]
    batch = I.batched_mix(256, seed=0)
    shard = partition_by_nnz([nnz_estimate(p) for p in batch], world)[rank] if world > 1 else list(range(len(batch)))
    return [batch[k] for k in shard], shard


def job_ms_per_step(local_ms, world, device=None):
    """Slowest rank's ms per step (the job ends when the last rank ends)."""
    if world <= 1:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(ms_per_step, systems_per_rank, world):
    """Whole-job metric: ms per system over the systems all ranks solved."""
    return ms_per_step / (systems_per_rank * world)


def host_cpu():
    """The host the oracle ran on: logical cores and CPU model."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def grad_allreduce_mean_(g, world):
    """Data-parallel training: the gradient averaged over the ranks (each
    rank's gradient is already the mean over its own systems and pairs), in
    place, so every rank takes the same Adam step.  The one collective on
    the training path (about 0.2 M FP32 values per step)."""
    if world > 1:
        import torch
        torch.distributed.all_reduce(g, op=torch.distributed.ReduceOp.SUM)
        g.div_(world)
    return g


def pcg_launch_mode(args, n, nsys, design=None):
    """How the library launches the PCG iterations of a triangular-solve
    preconditioner here: one launch at a time for a single system of 2^18
    rows or more whose tuned solve is level-ordered (it then runs in row
    blocks; the library's default), else the device-side loop graph.
    design: the tuned design's name, None when not yet known."""
    if getattr(args, "eager_pcg", False):
        return "iterations launched one by one (forced, for profiling)"
    if nsys == 1 and n >= (1 << 18) and design != "syncfree":
        return "iterations launched one by one (row-block solves)"
    return "iterations in a device-side loop graph"


def solve_config(args, cfg, wkind, n, nnz, nnz_L, levels, nsys):
    """The config block of the JSON line (identical on both arms)."""
    return {"workload": WORKLOAD_LABEL[args.workload], "systems_per_step": nsys, "n": int(n), "nnz": int(nnz),
            "nnz_L": int(nnz_L), "levels": int(levels),
            "gnn": f"n_mp={cfg.n_mp},l={cfg.l},l_mp={cfg.l_mp},h={cfg.h},diag_mode={cfg.diag_mode},"
                   + args.precision + (",x0_head" if args.x0 else ""),
            "weights": wkind, "pcg": "fp64 recurrences, " + args.apply + " L L^T solves, "
                                     + pcg_launch_mode(args, n, nsys),
            "rtol": RTOL, "l2": L2_FLUSH}


# ------------------------------------------------------------------ oracle legs
def _strip(Ao, frac):
    """Leading principal block (the first rows of the lexicographic order)."""
    import oracle as O
    m = max(2, int(Ao.n * frac))
    e = int(Ao.row_ptr[m])
    rows = np.repeat(np.arange(m), np.diff(Ao.row_ptr[:m + 1]))
    keep = Ao.col_idx[:e] < m
    rp = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=m))])
    return O.CSR(rp, Ao.col_idx[:e][keep], Ao.val[:e][keep])


def oracle_sample(Ao, cfg, w, b, learned_iters, L_pcg, strip_nnz=6000, k_iter=3, threads=1):
    """One bounded sample of the oracle's cost for the learned path on one
    system (CPU, FP64): the network forward timed on a leading strip of
    about strip_nnz nonzeros and scaled by nnz, plus k_iter PCG iterations on
    the full system with a factor of the same pattern (L_pcg), scaled to
    learned_iters.  With threads > 1 the SpMV and vector updates of PCG run
    on that many host threads (the network forward and the triangular solves
    stay sequential).  Returns (ms per system, wall ms of the sample,
    description)."""
    import oracle as O
    t_start = time.perf_counter()
    S = _strip(Ao, min(1.0, strip_nnz / max(1, Ao.nnz)))
    t0 = time.perf_counter()
    O.gnn_forward(cfg, S, b[:S.n], w)
    t_gnn = (time.perf_counter() - t0) * Ao.nnz / S.nnz
    used = O.set_threads(threads)
    t0 = time.perf_counter()
    O.pcg(Ao, b, O.PREC_LLT, L_pcg, rtol=0.0, max_iter=k_iter)
    t_it = (time.perf_counter() - t0) / k_iter
    O.set_threads(1)
    ms = 1e3 * (t_gnn + t_it * learned_iters)
    wall = 1e3 * (time.perf_counter() - t_start)
    desc = (f"oracle network forward on the first {S.n} of {Ao.n} rows (nnz {S.nnz}) scaled by nnz to the "
            f"full system, plus {k_iter} oracle PCG iterations on the full system ({used} thread(s) for SpMV "
            f"and vector updates) scaled to {learned_iters} iterations")
    return ms, wall, desc, used


def _oracle_system(I, workload):
    """The workload's first system assembled by the oracle (host), its b,
    its IC(0) factor (the PCG sample's factor of the same pattern) and its
    level count."""
    import oracle as O
    if workload == "fem2d_256":
        prob = I.fem2d_256(seed=0)
    elif workload == "fd3d_128":
        prob = I.fd3d_128(seed=0)
    elif workload == "heat2d_256":
        prob = I.heat2d(256, seed=0)
    else:
        raise ValueError(workload)
    Ao = O.assemble(prob)
    b = I.rhs(prob.n, 0)
    Lo, _ = O.ic0(Ao)
    _, nlev, _, _ = O.levels(Lo)
    return prob, Ao, b, Lo, nlev


def learned_iters_of(meta, workload):
    """Learned-path PCG iterations of the GPU arm on the workload's system,
    recorded beside the weights by the benchmark of the committed network."""
    return int(meta.get("bench_iters", {}).get(workload, 0)) or None


def run_reference(args):
    """The oracle as it stands, timed on the host cores on a bounded sample of
    the same workload (rank 0 only): every step is one oracle_sample."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle as O
    from paper_2305_16432_gb300 import inputs as I
    O.build()
    if args.workload not in ("fem2d_256", "fd3d_128", "heat2d_256"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm covers the single-system "
                          "workloads (fd3d_128, fem2d_256, heat2d_256)"}))
        return
    w, wkind, meta, cfg = _load_weights(I.GnnConfig(n_mp=6, l=2, l_mp=2, h=64), args.weights)
    prob, Ao, b, Lo, nlev = _oracle_system(I, args.workload)
    iters = learned_iters_of(meta, args.workload) or 200
    vals, walls = [], []
    desc, used = "", 1
    for s in range(args.warmup + args.steps):
        ms, wall, desc, used = oracle_sample(Ao, cfg, w, b, iters, Lo)
        if s >= args.warmup:
            vals.append(ms)
            walls.append(wall)
    v = float(np.mean(vals))
    config = solve_config(args, cfg, wkind, Ao.n, Ao.nnz, Lo.nnz, nlev, 1)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms/system", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(walls)),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": v, "unit": "ms/system", "cores": used, "kind": "oracle",
                             "sample": desc + f"; ms_per_step is the wall time of one such sample, value the "
                                              f"per-system cost it extrapolates to", "host": host_cpu()},
            "e2e": {"value": v, "unit": "ms/system", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def validate_oracle_estimate(args):
    """Runs the oracle's full learned path once on the 256^2 FEM system (the
    network forward over every row, then FP64 PCG with that factor to
    1e-6) and the sampled estimate beside it, so the extrapolation of
    oracle_sample is checked against a measurement.  Prints one JSON line."""
    import oracle as O
    from paper_2305_16432_gb300 import inputs as I
    O.build()
    cfg0 = I.GnnConfig(n_mp=6, l=2, l_mp=2, h=64)
    w, wkind, meta, cfg = _load_weights(cfg0, weights_for("fem2d_256"))
    prob, Ao, b, Lo, nlev = _oracle_system(I, "fem2d_256")
    t0 = time.perf_counter()
    Lg = O.gnn_forward(cfg, Ao, b, w.astype(np.float64))
    t_gnn = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, it, rel, st = O.pcg(Ao, b, O.PREC_LLT, Lg, rtol=RTOL)
    t_pcg = time.perf_counter() - t0
    full_ms = 1e3 * (t_gnn + t_pcg)
    est, wall, desc, _ = oracle_sample(Ao, cfg, w, b, it, Lo)
    print(json.dumps({"workload": "fem2d_256", "oracle_full_ms": full_ms, "oracle_gnn_ms": 1e3 * t_gnn,
                      "oracle_pcg_ms": 1e3 * t_pcg, "oracle_iters": it, "status": st,
                      "estimate_ms": est, "estimate_over_full": est / full_ms, "sample_wall_ms": wall,
                      "sample": desc, "host": host_cpu()}), flush=True)


# ------------------------------------------------------------------ GPU arm
def _assemble(N, I, probs, rank):
    """Assemble every system on the GPU; one concatenated pattern."""
    import torch
    rps, cis, vs, bs, sys_ptr = [], [], [], [], [0]
    off_n = off_nnz = 0
    for k, p in enumerate(probs):
        rp, ci, v = N.assemble_system(p)
        n = rp.numel() - 1
        rps.append(rp[:-1] + off_nnz)
        cis.append(ci + off_n)
        vs.append(v)
        bs.append(I.rhs(n, 1000 * rank + k))
        off_n += n
        off_nnz += ci.numel()
        sys_ptr.append(off_n)
    rp_cat = torch.cat(rps + [torch.tensor([off_nnz], dtype=torch.int32, device=rps[0].device)])
    ci_cat, v_cat = torch.cat(cis), torch.cat(vs)
    b = torch.as_tensor(np.concatenate(bs), device=v_cat.device)
    return rp_cat, ci_cat, v_cat, b, sys_ptr


def _timed(fn, k, stream, flush):
    """k runs of fn, each between CUDA events on the launching stream, L2
    flushed before each.  Returns (ms list, last result)."""
    import torch
    ms, last = [], None
    for _ in range(k):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last = fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms, last


def _spmv_roofline(N, P, v, hbm, flush, reps=20):
    """SpMV y = A x, one launch between CUDA events after each L2 flush (a
    cold-cache DRAM number at every size; the kernel is HBM-bound)."""
    import torch
    x = torch.randn(P.n, dtype=torch.float64, device=v.device)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        N.spmv(P, v, x, out=y)
    ms, _ = _timed(lambda: N.spmv(P, v, x, out=y), reps, stream, flush)
    t = float(np.mean(ms))
    byts = 12 * P.nnz + 4 * (P.n + 1) + 16 * P.n
    ach = byts / (t * 1e-3) / 1e9
    kname = "k_spmv_rows" if P.max_row <= 16 else "k_spmv_plain"
    return {"kernel": kname + " (SpMV, FP64)", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "bytes_per_launch": byts, "ms_per_launch": t,
            "timing": "one launch per event pair, L2 flushed before each"}


def run_solve(args, rank, world, local):
    import torch
    from paper_2305_16432_gb300 import inputs as I
    from paper_2305_16432_gb300 import npcg as N

    prec = N.BF16 if args.precision == "bf16" else N.FP32
    cfg0 = I.GnnConfig(n_mp=6, l=2, l_mp=2, h=64)
    w_np, wkind, wmeta, cfg = _load_weights(cfg0, args.weights)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    probs, shard = _problems(I, args.workload, rank, world)
    rp, ci, v, b, sys_ptr = _assemble(N, I, probs, rank)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P = N.analyse(rp, ci, sys_ptr if len(probs) > 1 else None)
    torch.cuda.synchronize()
    analyse_ms = 1e3 * (time.perf_counter() - t0)
    nsys = P.nsys
    w = torch.as_tensor(w_np, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    apply32 = args.apply == "fp32"
    pc = N.PREC_LLT32 if apply32 else N.PREC_LLT

    use_x0 = bool(args.x0)
    if use_x0 and not cfg.x0_head:
        raise SystemExit("--x0 needs weights with an initial-guess head")
    Lbuf = torch.empty(P.nnz_L, dtype=torch.float64, device=dev)

    def factor():
        if use_x0:
            return N.gnn_factor_x0(P, v, b, cfg, w, precision=prec)
        return N.gnn_factor(P, v, b, cfg, w, precision=prec, out=Lbuf), None

    def learned_step():
        L, x0 = factor()
        x, st = N.pcg_solve(P, v, b, pc, L, rtol=RTOL, x0=x0)
        return st

    def ic0_step():
        L, _ = N.ic0_factor(P, v, out=Lbuf)
        x, st = N.pcg_solve(P, v, b, pc, L, rtol=RTOL)
        return st

    def sgs_step():
        x, st = N.pcg_solve(P, v, b, pc, N.sgs_factor(P, v, out=Lbuf), rtol=RTOL)
        return st

    def jacobi_step():
        x, st = N.pcg_solve(P, v, b, N.PREC_JACOBI, None, rtol=RTOL)
        return st

    for _ in range(args.warmup):
        learned_step()
        ic0_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    ms_l, st_l = _timed(learned_step, args.steps, stream, flush)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = job_ms_per_step(float(np.sum(ms_l)) / args.steps, world, dev)
    total_sys = 256 if args.workload == "batched_256" else nsys * world
    value = ms_per_step / total_sys
    st_all = gather_stats(st_l, shard, 256, world) if args.workload == "batched_256" else st_l
    it_l = [s["iters"] for s in st_l]
    assert all(s["status"] == 0 for s in st_l), "a system did not converge"

    # the comparison preconditioners on the same systems
    ms_i, st_i = _timed(ic0_step, args.steps, stream, flush)
    sgs_step()
    ms_g, st_g = _timed(sgs_step, args.steps, stream, flush)
    jacobi_step()
    ms_j, st_j = _timed(jacobi_step, args.steps, stream, flush)
    it_i = [s["iters"] for s in st_i]

    # phases of the two totals (precompute and solve), each from CUDA events
    ms_gnn, _ = _timed(lambda: factor(), args.steps, stream, flush)
    Lg = factor()[0].clone()
    x0g = factor()[1]
    ms_lp, _ = _timed(lambda: N.pcg_solve(P, v, b, pc, Lg, rtol=RTOL, x0=x0g), args.steps, stream, flush)
    ms_ic, _ = _timed(lambda: N.ic0_factor(P, v, out=Lbuf), args.steps, stream, flush)
    Li = Lbuf.clone()
    ms_ip, _ = _timed(lambda: N.pcg_solve(P, v, b, pc, Li, rtol=RTOL), args.steps, stream, flush)

    # dominant kernel: the triangular solve of the tuned design, timed alone
    hbm, bf16, peak_kind = _peaks()
    N.factor_load(P, Li)
    r = torch.randn(P.n, dtype=torch.float64, device=dev)
    trsv_ms, _ = N.sptrsv_timed(P, r, transpose=False, reps=args.trsv_reps, f32=apply32)
    # SpTRSV bytes per launch: index + value per L entry, row pointer, rhs + solution
    trsv_bytes = (8 if apply32 else 12) * P.nnz_L + 4 * (P.n + 1) + 16 * P.n
    achieved = trsv_bytes / (trsv_ms * 1e-3) / 1e9
    design = {N.TRSV_LEVELSYNC: "levelsync", N.TRSV_LEVELFLAG: "levelflag", N.TRSV_LEVELSPLIT: "levelsplit",
              N.TRSV_LEVELMERGE: "levelmerge"}.get(P.trsv_mode, "syncfree")
    trsv_kernel = {"levelsync": "k_trsv_cta", "levelsplit": "k_trsv_split", "levelmerge": "k_trsv_cta",
                   "levelflag": "k_trsv_flag" if apply32 else "k_trsv_cta"}.get(design, "k_trsv")
    # DRAM bytes of one forward launch from an ncu capture of this kernel
    traffic = None
    prof = os.path.join(ROOT, "profiles", "trsv_traffic.json")
    if os.path.exists(prof):
        traffic = json.load(open(prof)).get(f"{args.workload}_{trsv_kernel}_{design}_fwd_bytes")
    spmv_rl = _spmv_roofline(N, P, v, hbm, flush)

    # end to end through the C ABI with host buffers (pinned)
    a_host = torch.empty(P.nnz, dtype=torch.float64, pin_memory=True)
    a_host.copy_(v.cpu())
    b_host = torch.empty(P.n, dtype=torch.float64, pin_memory=True)
    b_host.copy_(b.cpu())
    x_host = torch.empty(P.n, dtype=torch.float64, pin_memory=True)
    ts = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        N.solve_host(P, a_host.numpy(), b_host.numpy(), method=N.METHOD_GNN, cfg=cfg, weights=w,
                     precision=prec, rtol=RTOL, x_host=x_host.numpy(), f32_apply=apply32)
        ts.append(time.perf_counter() - t0)
    e2e_ms = job_ms_per_step(1e3 * float(np.mean(ts[args.warmup:])), world, dev) / total_sys
    h2d = 8 * (P.nnz + P.n)
    d2h = 8 * P.n

    # kernel launches per learned step (counted from the launch structure):
    # network: scales, 2 encoders, 2 per layer, decoder, L assembly
    gnn_launches = 1 + 2 + 2 * cfg.n_mp + 1 + 1
    # PCG: factor loads, init, preconditioner apply, r^T z, then per graph
    # trip 2 iterations (p update, SpMV, update, r^T z and the apply) + the
    # loop condition, or one by one in batches of 16 iterations, and the stats
    apply = {"levelsync": 4, "levelflag": 4, "levelsplit": 4, "levelmerge": 5}.get(design, 2)
    loads = 2 + (2 * P.merge_levels if design == "levelmerge" else 0) + 2
    if "one by one" in pcg_launch_mode(args, P.n, nsys, design):
        loop = (4 + apply) * 16 * max(1, math.ceil(max(it_l) / 16))
    else:
        loop = (2 * (4 + apply) + 1) * max(1, math.ceil(max(it_l) / 2))
    pcg_launches = loads + 1 + apply + 1 + loop + 1
    launches = (gnn_launches + pcg_launches) * args.steps

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(I, cfg, w_np, rp, ci, v, b, sys_ptr, nsys, it_l, P)

    if rank == 0:
        med = lambda a: float(np.median(a)) / nsys   # noqa: E731
        line = {
            "metric": METRIC, "value": value, "unit": "ms/system", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
            "scaling": "strong" if (args.workload == "batched_256" and world > 1) else "weak",
            "vs_baseline": None, "dtype": "f64+" + args.precision, "data": "synthetic",
            "config": solve_config(args, cfg, wkind, P.n, P.nnz, P.nnz_L, P.nlev_fwd, nsys),
            "compare": {"learned_iters": [s["iters"] for s in st_all] if len(st_all) > 1 else it_l[0],
                        "learned_ms_median": med(ms_l),
                        # the paper's statistic: mean of the fastest 5 timed runs
                        "learned_ms_fastest5_mean": float(np.mean(np.sort(ms_l)[:5])) / nsys,
                        "gnn_ms": med(ms_gnn), "learned_pcg_ms": med(ms_lp),
                        "ic0_ms_per_system": float(np.mean(ms_i)) / nsys,
                        "ic0_ms_fastest5_mean": float(np.mean(np.sort(ms_i)[:5])) / nsys,
                        "ic0_factor_ms": med(ms_ic), "ic0_pcg_ms": med(ms_ip),
                        "ic0_iters": it_i if nsys > 1 else it_i[0],
                        "jacobi_ms_per_system": float(np.mean(ms_j)) / nsys,
                        "jacobi_iters": [x["iters"] for x in st_j] if nsys > 1 else st_j[0]["iters"],
                        "sgs_ms_per_system": float(np.mean(ms_g)) / nsys,
                        "sgs_iters": [x["iters"] for x in st_g] if nsys > 1 else st_g[0]["iters"],
                        "analyse_ms": analyse_ms,
                        "wall_s_timed": wall, "trsv_design": design,
                        "merge_levels": P.merge_levels if design == "levelmerge" else 0,
                        "block_units": P.block_units,
                        "trsv_tuned_ms_fwd_bwd": P.tuned_ms},
            "roofline": {"kernel": trsv_kernel + " (forward SpTRSV, " + args.apply + ", " + design + ")",
                         "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "peak_kind": peak_kind, "traffic": traffic, "bytes_per_launch": trsv_bytes,
                         "ms_per_launch": trsv_ms, "levels": P.nlev_fwd},
            "roofline_spmv": dict(spmv_rl, peak_kind=peak_kind),
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms, "unit": "ms/system", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if args.workload == "batched_256" and world > 1:
            line["config"]["parallelism"] = f"{world} shards of one batch of 256 (greedy bin-pack on nnz)"
        print(json.dumps(line), flush=True)


def _cpu_baseline(I, cfg, w_np, rp, ci, v, b, sys_ptr, nsys, it_l, P):
    """The oracle on the host cores, on a bounded sample of the same systems:
    one core (the oracle as it stands) and all cores (OpenMP SpMV and vector
    updates).  The PCG sample uses the oracle's own IC(0) factor (the same
    pattern as the learned one; values do not change the cost)."""
    import oracle as O
    O.build()
    bh = b.cpu().numpy()
    rph, cih, vh = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy()
    members = list(range(nsys)) if nsys <= 3 else [0, nsys // 2, nsys - 1]
    sysm = {}
    for k in members:
        r0, r1 = sys_ptr[k], sys_ptr[k + 1]
        e0, e1 = int(rph[r0]), int(rph[r1])
        Ao = O.CSR(rph[r0:r1 + 1] - e0, cih[e0:e1] - r0, vh[e0:e1])
        sysm[k] = (Ao, O.ic0(Ao)[0], bh[r0:r1])
    res = {}
    for threads in (1, os.cpu_count() or 1):
        tot_ms, nnz_s, desc, used = 0.0, 0, "", 1
        for k in members:
            Ao, Lo, bk = sysm[k]
            ms_k, _, desc, used = oracle_sample(Ao, cfg, w_np, bk, it_l[k], Lo, threads=threads)
            tot_ms += ms_k
            nnz_s += Ao.nnz
        ms_cpu = tot_ms * (P.nnz / nnz_s) / nsys
        smp = desc if nsys == 1 else (f"{len(members)} of {nsys} members, each: " + desc +
                                      "; scaled by nnz to the batch, per system")
        res[threads] = {"value": ms_cpu, "unit": "ms/system", "cores": used, "kind": "oracle", "sample": smp}
    one = res[1]
    allc = res[max(res)]
    return dict(one, host=host_cpu(), all_cores=allc if allc is not one else None)


def run_train(args, rank, world, local):
    """One training step of the method: loss Eq. (loss_Ab) over 32 systems x
    8 (x, b) pairs through the network (BF16 tensor-core forward, FP32
    adjoint) and one Adam step on the FP32 master weights.  Under torchrun
    each rank takes its own 32 systems and the gradient is averaged over the
    ranks before the step (data parallelism)."""
    import torch
    from paper_2305_16432_gb300 import inputs as I
    from paper_2305_16432_gb300 import npcg as N
    prec = N.BF16 if args.precision == "bf16" else N.FP32
    cfg = I.GnnConfig(n_mp=6, l=2, l_mp=2, h=64, loss=N.LOSS_FROB if args.loss == "frob" else N.LOSS_AB)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    probs = I.training_mix(32, seed=1000 + 100 * rank)
    rp, ci, v, _, sys_ptr = _assemble(N, I, probs, rank)
    P = N.analyse(rp, ci, sys_ptr)
    pairs = 8
    Bm = torch.as_tensor(np.stack([I.rhs(P.n, 5000 + 37 * rank + q) for q in range(pairs)]), device=dev)
    Xm = torch.empty_like(Bm)
    Lic, _ = N.ic0_factor(P, v)
    for q in range(pairs):
        Xm[q], _ = N.pcg_solve(P, v, Bm[q], N.PREC_LLT, Lic, rtol=1e-12, raise_on_fail=True)
    w = torch.as_tensor(I.gnn_weights(cfg, 2023), device=dev)
    m = torch.zeros_like(w)
    vv = torch.zeros_like(w)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    state = {"t": 0}

    def step():
        loss, g = N.loss_and_grad(P, v, Xm, Bm, cfg, w, precision=prec)
        grad_allreduce_mean_(g, world)
        state["t"] += 1
        N.adam_step(w, g, m, vv, state["t"])
        return loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    ms, loss = _timed(step, args.steps, stream, flush)
    clk = clocks.stop()
    ms_per_step = job_ms_per_step(float(np.mean(ms)), world, dev)
    # the step's dense contractions: per pair one network forward (encoders,
    # n_mp node and edge MLPs, decoder) and its adjoint (input gradients and
    # weight gradients: twice the forward), i.e. 3x the forward's flops
    h, n, nnz = cfg.h, P.n, P.nnz
    fwd = (2 * n * (h + 2 * h * h) + 2 * nnz * (h + 2 * h * h)
           + cfg.n_mp * (2 * n * (2 * h * h + 2 * h * h) + 2 * nnz * (3 * h * h + 2 * h * h))
           + 2 * nnz * (2 * h * h + h))
    flops = 3.0 * fwd * pairs
    achieved = flops / (ms_per_step * 1e-3) / 1e12
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    roofline = {"kernel": "whole training step (tensor-core MLP forward and adjoint, k_mlp_bf16 / "
                          "k_mlp_bwd_tc / k_wgrad_tc)", "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None, "flops_per_step": flops,
                "peak_kind": "measured sustained" if peaks else "fallback"}
    if rank == 0:
        line = {"metric": "ms per training step (32 systems x 8 pairs, loss + adjoint + Adam)",
                "value": ms_per_step, "unit": "ms/step", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+" + args.precision, "data": "synthetic",
                "config": {"workload": "train_32x8" + ("_frobenius" if args.loss == "frob" else ""), "n": P.n,
                           "nnz": P.nnz, "systems": 32, "pairs": pairs,
                           "loss": "Eq. loss_A (Frobenius)" if args.loss == "frob" else "Eq. loss_Ab",
                           "parallelism": f"dp{world} (gradient all-reduce)" if world > 1 else "dp1",
                           "gnn": "n_mp=6,l=2,l_mp=2,h=64", "l2": L2_FLUSH},
                "loss_last": loss, "roofline": roofline, "cpu_baseline": None, "e2e": None, "clocks": clk}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fd3d_128", choices=list(SOLVE_WORKLOADS) + ["train_32"],
                    help="fd3d_128 (the headline line), fem2d_256, batched_256, heat2d_256 or train_32")
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"],
                    help="network arithmetic: BF16 tensor cores (default) or FP32")
    ap.add_argument("--apply", default="fp32", choices=["fp32", "fp64"],
                    help="arithmetic of the L L^T solves inside the FP64 PCG")
    ap.add_argument("--weights", default=None, help="network weights (.npy); default: the workload's own")
    ap.add_argument("--loss", default="ab", choices=["ab", "frob"],
                    help="train_32: the method's loss Eq. (loss_Ab) or the Frobenius ablation Eq. (loss_A)")
    ap.add_argument("--x0", action="store_true",
                    help="start PCG from the network's initial guess (weights with an initial-guess head)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--validate-oracle-estimate", action="store_true",
                    help="run the oracle's full learned path on the 256^2 FEM system beside its sampled estimate")
    ap.add_argument("--trsv-reps", type=int, default=50)
    ap.add_argument("--eager-pcg", action="store_true",
                    help="launch each PCG iteration's kernels one by one instead of the device-side loop graph "
                         "(kernel profilers do not see kernels inside a conditional graph node; results are "
                         "identical, the timing is not the benchmark's)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.weights is None:
        args.weights = weights_for(args.workload, args.x0)
    if args.validate_oracle_estimate:
        validate_oracle_estimate(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2305_16432_gb300 import build as B
    B.build()
    if args.eager_pcg:
        from paper_2305_16432_gb300 import npcg as N
        N.handle().set_pcg_eager(True)
    if args.workload == "train_32":
        run_train(args, rank, world, local)
    else:
        run_solve(args, rank, world, local)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
