"""Benchmark of the learned-preconditioner PCG hot path on one GB300.

Metric: ms to a 1e-6 relative residual per system, learned-L PCG (graph
network factor + PCG, the paper's "precompute + solve" total, Sec. 5.1
"Evaluation Metrics") next to IC(0)-PCG on the same GPU; secondary: SpTRSV
bandwidth against the HBM roofline.

Workload (one step = one system): 2-D variable-coefficient diffusion,
P1 FEM on the Delaunay triangulation of a seeded jittered 256 x 256 lattice
(n = 64,516, nnz = 449,582), log k a GRF (sigma 1, correlation 0.1),
b ~ N(0,1); 6-layer hidden-64 network; FP64 PCG to 1e-6.  Inputs are
resident in HBM when the timed region starts (pattern analysed once: a fixed
mesh, as in the paper's environments); L2 is flushed between steps.

--impl reference times the CPU oracle (the method's plain FP64 restatement)
on the host cores for the same metric; see cpu_baseline below.
Multi-GPU (torchrun): every rank solves its own systems (independent
problems, no collective on the data path); value = systems of all ranks per
unit time, expressed as ms per system.
"""
from __future__ import annotations

import argparse
import json
import math
import os
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


def _load_weights(cfg, path):
    from paper_2305_16432_gb300 import inputs as I
    if path and os.path.exists(path):
        w = np.load(path).astype(np.float32)
        if len(w) == cfg.nparams:
            meta = {}
            mp = os.path.splitext(path)[0] + ".json"
            if os.path.exists(mp):
                meta = json.load(open(mp))
            return w, "trained", meta
    return I.gnn_weights(cfg, 1), "random-init", {}


def _strip(Ao, frac):
    """Leading principal block (the first rows of the lexicographic lattice)."""
    import oracle as O
    m = max(2, int(Ao.n * frac))
    rp, ci, v = [0], [], []
    for i in range(m):
        s, e = Ao.row_ptr[i], Ao.row_ptr[i + 1]
        cols = Ao.col_idx[s:e]
        keep = cols < m
        ci.extend(cols[keep].tolist())
        v.extend(Ao.val[s:e][keep].tolist())
        rp.append(len(ci))
    return O.CSR(rp, ci, v)


def oracle_estimate(prob, cfg, w, b, learned_iters, budget_frac=1.0 / 16):
    """Oracle (CPU, FP64, 1 thread) cost of the learned path on the full
    system: network forward timed on a strip of the mesh (budget_frac of the
    rows) scaled by nnz, plus PCG: per-iteration oracle cost on the full
    system (same factor pattern) times the learned path's iteration count."""
    import oracle as O
    Ao = O.assemble(prob)
    S = _strip(Ao, budget_frac)
    t0 = time.perf_counter()
    O.gnn_forward(cfg, S, b[:S.n], w)
    t_gnn = (time.perf_counter() - t0) * Ao.nnz / S.nnz
    L, _ = O.ic0(Ao)
    k = 30
    t0 = time.perf_counter()
    O.pcg(Ao, b, O.PREC_LLT, L, rtol=0.0, max_iter=k)
    t_it = (time.perf_counter() - t0) / k
    ms = 1e3 * (t_gnn + t_it * learned_iters)
    sample = (f"oracle network forward on the first {S.n} of {Ao.n} rows (nnz {S.nnz}) scaled by nnz "
              f"to the full system, plus oracle PCG cost per iteration over {k} iterations on the full "
              f"system times {learned_iters} learned-path iterations")
    return ms, sample


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle as O
    from paper_2305_16432_gb300 import inputs as I
    O.build()
    prob = I.fem2d_256(seed=0)
    cfg = I.GnnConfig(n_mp=6, l=2, l_mp=2, h=64)
    w, kind, meta = _load_weights(cfg, os.path.join(WEIGHTS_DIR, "fem2d_6x64.npy"))
    b = I.rhs(prob.n, 0)
    iters = int(meta.get("learned_iters_fem256", 0)) or 191
    vals = []
    sample = ""
    for s in range(args.warmup + args.steps):
        ms, sample = oracle_estimate(prob, cfg, w, b, iters, budget_frac=1.0 / 64)
        if s >= args.warmup:
            vals.append(ms)
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms/system", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fem2d_256_learned_pcg", "n": prob.n, "rtol": RTOL},
            "cpu_baseline": {"value": v, "unit": "ms/system", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "ms/system", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"],
                    help="network arithmetic: BF16 tensor cores (default) or FP32")
    ap.add_argument("--apply", default="fp32", choices=["fp32", "fp64"],
                    help="arithmetic of the L L^T solves inside the FP64 PCG")
    ap.add_argument("--weights", default=os.path.join(WEIGHTS_DIR, "fem2d_6x64.npy"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--trsv-reps", type=int, default=50)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
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
    from paper_2305_16432_gb300 import inputs as I
    B.build()
    from paper_2305_16432_gb300 import npcg as N

    prec = N.BF16 if args.precision == "bf16" else N.FP32
    prob = I.fem2d_256(seed=rank)
    cfg = I.GnnConfig(n_mp=6, l=2, l_mp=2, h=64)
    w_np, wkind, wmeta = _load_weights(cfg, args.weights)
    if wmeta.get("config", {}).get("diag_mode", 0):
        cfg = I.GnnConfig(n_mp=6, l=2, l_mp=2, h=64, diag_mode=int(wmeta["config"]["diag_mode"]))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    rp, ci, v = N.assemble_system(prob)
    P = N.analyse(rp, ci)
    b = torch.as_tensor(I.rhs(P.n, rank), device=dev)
    w = torch.as_tensor(w_np, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    apply32 = args.apply == "fp32"
    pc = N.PREC_LLT32 if apply32 else N.PREC_LLT

    def learned_step():
        L = N.gnn_factor(P, v, b, cfg, w, precision=prec)
        x, st = N.pcg_solve(P, v, b, pc, L, rtol=RTOL)
        return st[0]

    def ic0_step():
        L, _ = N.ic0_factor(P, v)
        x, st = N.pcg_solve(P, v, b, pc, L, rtol=RTOL)
        return st[0]

    def timed(fn, k):
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
    ms_l, st_l = timed(learned_step, args.steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms_i, st_i = timed(ic0_step, args.steps)
    ms_per_step = float(np.sum(ms_l)) / args.steps
    if world > 1:
        t = torch.tensor([ms_per_step], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_per_step = float(t.item())
    value = ms_per_step / world

    # dominant kernel: the level-ordered triangular solve, timed alone
    hbm, bf16, peak_kind = _peaks()
    Lic, _ = N.ic0_factor(P, v)
    N.factor_load(P, Lic)
    r = torch.randn(P.n, dtype=torch.float64, device=dev)
    trsv_ms, _ = N.sptrsv_timed(P, r, transpose=False, reps=args.trsv_reps, f32=apply32)
    # SpTRSV bytes per launch: index + value per L entry, row pointer, rhs + solution
    trsv_bytes = (8 if apply32 else 12) * P.nnz_L + 4 * (P.n + 1) + 16 * P.n
    achieved = trsv_bytes / (trsv_ms * 1e-3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "trsv_traffic.json")
    if os.path.exists(prof):
        traffic = json.load(open(prof)).get("fem2d_256_fwd_bytes")

    # end to end through the C ABI with host buffers
    e2e_ms = None
    h2d = d2h = 0
    if True:
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
        e2e_ms = 1e3 * float(np.mean(ts[args.warmup:])) / world
        h2d = 8 * (P.nnz + P.n)
        d2h = 8 * P.n

    # kernel launches per learned step (counted from the launch structure)
    it = st_l["iters"]
    # network: scales, 2 encoders, 2 per layer, decoder, L assembly
    gnn_launches = 1 + 2 + 2 * cfg.n_mp + 1 + 1
    # PCG: 4 factor loads, init, 2 solves, r^T z, 11 per graph trip (2 iterations
    # of 5 kernels + the loop condition), stats
    trips = max(1, math.ceil(it / 2))
    pcg_launches = 4 + 1 + 2 + 1 + 11 * trips + 1
    launches = (gnn_launches + pcg_launches) * args.steps

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        ms_cpu, sample = oracle_estimate(prob, cfg, w_np, I.rhs(P.n, 0), it, budget_frac=1.0 / 64)
        cpu = {"value": ms_cpu, "unit": "ms/system", "cores": 1, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ms/system", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+" + args.precision, "data": "synthetic",
            "config": {"workload": "fem2d_256_learned_pcg", "n": P.n, "nnz": P.nnz, "nnz_L": P.nnz_L,
                       "levels": P.nlev_fwd, "gnn": "n_mp=6,l=2,l_mp=2,h=64," + args.precision,
                       "weights": wkind, "pcg": "fp64 recurrences, " + args.apply + " L L^T solves",
                       "rtol": RTOL, "l2": "flushed between steps (256 MB write)"},
            "compare": {"learned_iters": st_l["iters"], "learned_ms_median": float(np.median(ms_l)),
                        "ic0_ms": float(np.mean(ms_i)), "ic0_iters": st_i["iters"],
                        "learned_relres": st_l["relres"], "wall_s_timed": wall,
                        "trsv_design": "levelsync" if P.trsv_mode == N.TRSV_LEVELSYNC else "syncfree",
                        "trsv_tuned_ms_fwd_bwd": P.tuned_ms},
            "roofline": {"kernel": ("k_trsv_cta" if P.trsv_mode == N.TRSV_LEVELSYNC else "k_trsv")
                         + " (forward SpTRSV, " + args.apply + ")", "bound": "hbm",
                         "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "peak_kind": peak_kind, "traffic": traffic, "bytes_per_launch": trsv_bytes,
                         "ms_per_launch": trsv_ms, "levels": P.nlev_fwd},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms, "unit": "ms/system", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
