"""A small, self-contained run of one hot-path operation for profilers.

Builds one 3-D variable-coefficient diffusion system (7-point FD on an
N^3 grid, log k a GRF with sigma 1.5 and the 128^3 workload's correlation of
6.4 grid cells), analyses its pattern and repeats one operation a few times
after a warm-up, so that a kernel profiler can capture a handful of launches
of a case that is larger than L2 but holds only a few GB on the device:

    python -m paper_2305_16432_gb300.profile_case --case gnn --grid 64 --reps 3

Cases: gnn (BF16 network forward with the 3-D task network: encoders, the
message-passing node and edge MLPs, the decoder), trsv (forward triangular
solve of the tuned design, FP32), spmv (y = A x), ic0 (IC(0) factorisation),
pcg (learned-factor PCG to 1e-6).  Prints the CUDA-event time per repetition;
--profile-range limits a profiler started with --profile-from-start off to
the timed repetitions.
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np
import torch

from . import inputs as I

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "gnn_6x64_fd3d.npy")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", required=True, choices=["gnn", "trsv", "spmv", "ic0", "pcg"])
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--trsv", default="auto", choices=["auto", "syncfree", "levelsync", "levelmerge"],
                    help="triangular-solve design (default: the one the analysis tuned; a profiler's slowdown "
                         "of the analysis' trial solves can change that choice)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed repetitions with cudaProfilerStart/Stop (for a profiler started "
                         "with --profile-from-start off)")
    args = ap.parse_args()
    from . import build as B
    B.build()
    from . import npcg as N
    torch.cuda.set_device(0)
    side = args.grid
    prob = I.fd3d(side, sigma=1.5, corr_len=6.4 / (side + 1), seed=11)
    rp, ci, v = N.assemble_system(prob)
    P = N.analyse(rp, ci)
    if args.trsv != "auto":
        P.set_trsv(getattr(N, "TRSV_" + args.trsv.upper()))
    b = torch.as_tensor(I.rhs(P.n, 11), device="cuda")
    meta = json.load(open(os.path.splitext(WEIGHTS)[0] + ".json"))
    cfg = I.GnnConfig(**meta["config"])
    w = torch.as_tensor(np.load(WEIGHTS), device="cuda")
    L = torch.empty(P.nnz_L, dtype=torch.float64, device="cuda")
    y = torch.empty_like(b)
    if args.case in ("trsv", "pcg"):
        N.gnn_factor(P, v, b, cfg, w, precision=N.BF16, out=L)
        N.factor_load(P, L)

    def op():
        if args.case == "gnn":
            N.gnn_factor(P, v, b, cfg, w, precision=N.BF16, out=L)
        elif args.case == "trsv":
            N.sptrsv_timed(P, b, transpose=False, reps=1, out=y, f32=True)
        elif args.case == "spmv":
            N.spmv(P, v, b, out=y)
        elif args.case == "ic0":
            N.ic0_factor(P, v, out=L)
        else:
            N.pcg_solve(P, v, b, N.PREC_LLT32, L, rtol=1e-6)

    for _ in range(args.warmup):
        op()
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.cudart().cudaProfilerStart()
    times = []
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        op()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    if args.profile_range:
        torch.cuda.cudart().cudaProfilerStop()
    print(json.dumps({"case": args.case, "grid": side, "n": P.n, "nnz": P.nnz, "nnz_L": P.nnz_L,
                      "trsv_mode": P.trsv_mode, "block_units": P.block_units, "merge_levels": P.merge_levels,
                      "tuned_ms": P.tuned_ms, "ms": times}))


if __name__ == "__main__":
    main()
