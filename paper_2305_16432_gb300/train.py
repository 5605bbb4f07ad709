"""Training of the graph-network preconditioner on the GPU.

Data (Sec. 4.3, App. A.2 describe (A_i, x_i, b_i) tuples from simulations;
the paper's datasets are not available, so the tuples are synthetic): groups
of 8 seeded systems, 2-D P1 FEM diffusion on jittered lattices and 3-D 7-point
FD diffusion (log k a GRF, sigma 1, correlation 0.1), right-hand sides
b ~ N(0, 1), and x = A^-1 b computed by this library's own IC(0)-PCG to a
1e-10 relative residual.  Loss Eq. (loss_Ab), mean over a batch of 8 systems
x 2 pairs (the paper's batch size 16 for 2-D problems), Adam with lr 1e-3
(App. A.4) decayed by a cosine to 1e-4.  Every forward, adjoint and
optimiser step runs in the library's kernels (BF16 tensor-core forward with
the FP32 adjoint, or FP32 throughout).

On this data the loss keeps falling long after PCG iterations stop improving
(with the softplus diagonal a network reaches 20x less loss than IC(0) while
needing several times IC(0)'s iterations), so the run keeps the checkpoint
with the fewest PCG iterations on held-out systems of the training family
(model selection by validation; the paper trains to convergence).  The
committed network uses the App. A.3 factorisation L D L^T with D = diag(A):

    python -m paper_2305_16432_gb300.train --steps 720 --val_every 40 --diag_mode 1 \
        --sizes 96,128,160 --sizes3d 20,26,32 --precision bf16 --out weights/gnn_6x64.npy
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import sys
import time

import numpy as np
import torch

from . import inputs as I


# a checkpoint whose PCG has not converged by then counts as failed
VAL_MAX_ITER = 5000


def _np(t):
    return t.detach().cpu().numpy()


def make_group(N, probs, pairs, seed, rtol=1e-10):
    """One batched pattern of several systems with `pairs` (x, b) tuples each."""
    rps, cis, vs, sys_ptr = [], [], [], [0]
    Xs, Bs = [], []
    off_n, off_nnz = 0, 0
    for k, p in enumerate(probs):
        rp, ci, v = N.assemble_system(p)
        P1 = N.analyse(rp, ci)
        L, _ = N.ic0_factor(P1, v)
        B = torch.as_tensor(I.rhs(P1.n, seed * 1000 + k, count=pairs), device="cuda")
        X = torch.empty_like(B)
        for q in range(pairs):
            X[q], st = N.pcg_solve(P1, v, B[q], N.PREC_LLT, L, rtol=rtol, raise_on_fail=True)
        rps.append(rp[:-1] + off_nnz)
        cis.append(ci + off_n)
        vs.append(v)
        Xs.append(X)
        Bs.append(B)
        off_n += P1.n
        off_nnz += P1.nnz
        sys_ptr.append(off_n)
        del P1
    rp_cat = torch.cat(rps + [torch.tensor([off_nnz], dtype=torch.int32, device="cuda")])
    P = N.analyse(rp_cat, torch.cat(cis), sys_ptr)
    return P, torch.cat(vs), torch.cat(Xs, dim=1).contiguous(), torch.cat(Bs, dim=1).contiguous()


def evaluate(N, cfg, w, probs, rtol=1e-6, seed=77, precision=None):
    """Iterations to rtol of learned-L, IC(0) and Jacobi PCG on held-out systems."""
    out = []
    for k, p in enumerate(probs):
        rp, ci, v = N.assemble_system(p)
        P = N.analyse(rp, ci)
        b = torch.as_tensor(I.rhs(P.n, seed + k), device="cuda")
        L = N.gnn_factor(P, v, b, cfg, w, precision=N.FP32 if precision is None else precision)
        _, sl = N.pcg_solve(P, v, b, N.PREC_LLT, L, rtol=rtol, max_iter=VAL_MAX_ITER)
        Li, _ = N.ic0_factor(P, v)
        _, si = N.pcg_solve(P, v, b, N.PREC_LLT, Li, rtol=rtol)
        _, sj = N.pcg_solve(P, v, b, N.PREC_JACOBI, None, rtol=rtol)
        rec = {"n": P.n, "learned": sl[0]["iters"], "ic0": si[0]["iters"], "jacobi": sj[0]["iters"],
               "learned_status": sl[0]["status"]}
        if cfg.x0_head:
            # the same factor, PCG started from the head's initial guess
            L2, x0 = N.gnn_factor_x0(P, v, b, cfg, w, precision=N.FP32 if precision is None else precision)
            _, sx = N.pcg_solve(P, v, b, N.PREC_LLT, L2, rtol=rtol, max_iter=VAL_MAX_ITER, x0=x0)
            rec["learned_x0"] = sx[0]["iters"]
            rec["x0_relres"] = float(torch.linalg.norm(b - N.spmv(P, v, x0)) / torch.linalg.norm(b))
        out.append(rec)
    return out


def save_checkpoint(path, cfg, w, mom, vel, step, hist):
    """Weights and Adam state as one file (resumable)."""
    np.savez(path, w=_np(w), m=_np(mom), v=_np(vel), step=step, hist=np.asarray(hist),
             config=np.asarray([cfg.n_mp, cfg.l, cfg.l_mp, cfg.h], np.int64))


def train(cfg: I.GnnConfig, steps=600, groups=4, per_group=8, pairs=8, m=128, lr=1e-3, lr_final=1e-4,
          seed=2023, log_every=25, w0=None, ckpt=None, resume=None, val_every=50, precision=None, sizes=None,
          sizes3d=None, sigma3d=1.0, corr3d=0.1, head_only=False, heat=False, corr3d_cells=None, val3d=None):
    """Adam at lr (App. A.4), cosine-decayed to lr_final over the run; returns
    the weights with the fewest validation PCG iterations.  precision: the
    network forward's arithmetic (FP32, or BF16 tensor cores with the FP32
    adjoint); sizes: lattice size of each 2-D FEM group (default m for
    all, [] for none); sizes3d: grid side of each 3-D FD group (none by
    default), with log k a GRF of sigma3d and correlation length corr3d.
    head_only: train the initial-guess head alone (the trunk's gradient is
    zeroed, so Adam leaves it unchanged) and validate PCG started from x0.
    heat: the 2-D groups and validation systems are implicit heat steps
    M + tau K with Dirichlet arcs (inputs.heat2d) instead of stiffness
    matrices.  corr3d_cells: the 3-D correlation length in grid cells
    instead (corr = cells / (side + 1)), so that grids of every side see the
    local coefficient statistics of the target grid; val3d: side of the 3-D
    validation system (default: the middle training side)."""
    from . import build as B
    B.build()
    from . import npcg as N
    prec = N.FP32 if precision is None else precision
    if sizes is None:
        sizes = [m] * groups
    specs = [("fem", x) for x in sizes] + [("fd3", x) for x in (sizes3d or [])]
    family2d = (lambda mm, sd: I.heat2d(mm, seed=sd)) if heat else \
        (lambda mm, sd: I.fem2d(mm, sigma=1.0, corr_len=0.1, seed=sd))
    groups = len(specs)
    def corr_of(side):
        return corr3d_cells / (side + 1) if corr3d_cells else corr3d

    t0 = time.time()
    data = []
    for g, (kind, mg) in enumerate(specs):
        if kind == "fem":
            probs = [family2d(mg, seed + 100 * g + k) for k in range(per_group)]
        else:
            probs = [I.fd3d(mg, sigma=sigma3d, corr_len=corr_of(mg), seed=seed + 100 * g + k)
                     for k in range(per_group)]
        data.append(make_group(N, probs, pairs, seed + g))
    t_data = time.time() - t0
    w = torch.as_tensor(I.gnn_weights(cfg, seed) if w0 is None else w0, device="cuda")
    mom = torch.zeros_like(w)
    vel = torch.zeros_like(w)
    hist = []
    start = 1
    if resume and os.path.exists(resume):
        ck = np.load(resume)
        assert list(ck["config"]) == [cfg.n_mp, cfg.l, cfg.l_mp, cfg.h], "checkpoint of another network"
        w.copy_(torch.as_tensor(ck["w"]))
        mom.copy_(torch.as_tensor(ck["m"]))
        vel.copy_(torch.as_tensor(ck["v"]))
        start = int(ck["step"]) + 1
        hist = list(ck["hist"])
    # validation: PCG iterations on held-out systems of the training family;
    # the checkpoint with the fewest mean iterations is kept
    vals = []
    vprobs = [family2d(m, 8000 + k) for k in range(2)] if sizes else []
    if sizes3d:
        sv = val3d or sizes3d[len(sizes3d) // 2]
        v3 = I.fd3d(sv, sigma=sigma3d, corr_len=corr_of(sv), seed=8000)
        vprobs = [vprobs[0], v3] if vprobs else [v3]
    for k, pv in enumerate(vprobs):
        rp, ci, v = N.assemble_system(pv)
        Pv = N.analyse(rp, ci)
        vals.append((Pv, v, torch.as_tensor(I.rhs(Pv.n, 8000 + k), device="cuda")))

    n_trunk = N.gnn_nparams(dataclasses.replace(cfg, x0_head=0))

    def val_iters():
        its = []
        for Pv, v, bv in vals:
            # the deployed configuration: FP32 triangular solves with a BF16 network
            if cfg.x0_head:
                L, x0 = N.gnn_factor_x0(Pv, v, bv, cfg, w, precision=prec)
            else:
                L, x0 = N.gnn_factor(Pv, v, bv, cfg, w, precision=prec), None
            _, st = N.pcg_solve(Pv, v, bv, N.PREC_LLT32 if prec == N.BF16 else N.PREC_LLT, L, rtol=1e-6,
                                max_iter=VAL_MAX_ITER, x0=x0)
            its.append(st[0]["iters"] if st[0]["status"] == 0 else 2 * VAL_MAX_ITER)
        return float(np.mean(its))

    best = (val_iters(), 0, w.clone())
    curve = [(0, best[0], float("nan"))]
    t1 = time.time()
    for t in range(start, steps + 1):
        P, A, X, Bb = data[(t - 1) % groups]
        q = ((t - 1) // groups) % (pairs // 2)
        loss, g = N.loss_and_grad(P, A, X[2 * q:2 * q + 2].contiguous(), Bb[2 * q:2 * q + 2].contiguous(), cfg, w,
                                  precision=prec)
        if head_only:
            g[:n_trunk] = 0
        lr_t = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * (t - 1) / max(1, steps - 1)))
        N.adam_step(w, g, mom, vel, t, lr=float(lr_t))
        hist.append(loss)
        if log_every and (t % log_every == 0 or t == 1):
            print(f"step {t:5d} loss {loss:.6e} lr {lr_t:.2e} ({time.time() - t1:.1f} s)", flush=True)
        if ckpt and t % 250 == 0:
            save_checkpoint(ckpt, cfg, w, mom, vel, t, hist)
        if val_every and t % val_every == 0:
            vi = val_iters()
            curve.append((t, vi, float(np.mean(hist[-val_every:]))))
            if vi < best[0]:
                best = (vi, t, w.clone())
            if log_every:
                print(f"  validation at step {t}: {vi:.1f} iterations (best {best[0]:.1f} at {best[1]})", flush=True)
    torch.cuda.synchronize()
    return best[2], hist, {"data_s": t_data, "train_s": time.time() - t1, "best_step": best[1],
                           "best_val_iters": best[0], "val_curve": curve, "final_weights_val_iters": curve[-1][1]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--h", type=int, default=64)
    ap.add_argument("--n_mp", type=int, default=6)
    ap.add_argument("--m", type=int, default=128)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr_final", type=float, default=1e-4)
    ap.add_argument("--ckpt", default=None)
    ap.add_argument("--resume", default=None)
    ap.add_argument("--val_every", type=int, default=50)
    ap.add_argument("--diag_mode", type=int, default=0,
                    help="0: softplus diagonal; 1: L = L' D^1/2 (App. A.3, D = diag(A)); 2: L = D^1/2 L~ (rows scaled)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--sizes", default="", help="comma-separated lattice sizes of the 2-D FEM training groups")
    ap.add_argument("--sizes3d", default="", help="comma-separated grid sides of the 3-D FD training groups")
    ap.add_argument("--per_group", type=int, default=8,
                    help="systems per training group (the adjoint's workspace grows with the group's nonzeros)")
    ap.add_argument("--sigma3d", type=float, default=1.0, help="GRF sigma of the 3-D groups")
    ap.add_argument("--corr3d", type=float, default=0.1, help="GRF correlation length of the 3-D groups")
    ap.add_argument("--corr3d_cells", type=float, default=None,
                    help="3-D correlation length in grid cells instead (6.4 = the 128^3 workload's 0.05)")
    ap.add_argument("--val3d", type=int, default=None, help="side of the 3-D validation grid")
    ap.add_argument("--eval128", action="store_true",
                    help="also evaluate on the 128^3 benchmark system (sigma 1.5, corr 0.05) and record the "
                         "deployed configuration's iterations as the benchmark's learned iterations")
    ap.add_argument("--loss", default="ab", choices=["ab", "frob"],
                    help="Eq. (loss_Ab) (the method) or the Frobenius loss Eq. (loss_A) (ablation)")
    ap.add_argument("--init", default=None, help="start from these weights (same network shape)")
    ap.add_argument("--heat", action="store_true",
                    help="2-D systems are implicit heat steps M + tau K with Dirichlet arcs")
    ap.add_argument("--x0_from", default=None,
                    help="weights of a trained network: add the initial-guess head and train it alone")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "weights", "gnn_6x64.npy"))
    args = ap.parse_args()
    cfg = I.GnnConfig(n_mp=args.n_mp, l=2, l_mp=2, h=args.h, diag_mode=args.diag_mode,
                      loss=1 if args.loss == "frob" else 0)
    from . import build as B
    B.build()
    from . import npcg as N
    w_init = None
    if args.init:
        w_init = np.load(args.init).astype(np.float32)
        assert w_init.size == cfg.nparams, "initial weights of another network"
    if args.x0_from:
        # trained trunk + a freshly initialised head (the tail of the flat layout)
        trunk = np.load(args.x0_from).astype(np.float32)
        cfg = dataclasses.replace(cfg, x0_head=1)
        w_init = I.gnn_weights(cfg, 2023)
        assert trunk.size == N.gnn_nparams(dataclasses.replace(cfg, x0_head=0)), "trunk of another network"
        w_init[:trunk.size] = trunk
    prec = N.BF16 if args.precision == "bf16" else N.FP32
    sizes = [] if args.sizes == "none" else ([int(x) for x in args.sizes.split(",") if x] or None)
    sizes3d = [int(x) for x in args.sizes3d.split(",") if x] or None
    w, hist, tm = train(cfg, steps=args.steps, per_group=args.per_group, m=args.m, lr=args.lr,
                        lr_final=args.lr_final, ckpt=args.ckpt,
                        resume=args.resume, val_every=args.val_every, precision=prec, sizes=sizes,
                        sizes3d=sizes3d, sigma3d=args.sigma3d, corr3d=args.corr3d, w0=w_init,
                        head_only=bool(args.x0_from), heat=args.heat, corr3d_cells=args.corr3d_cells,
                        val3d=args.val3d)
    w0 = torch.as_tensor(I.gnn_weights(cfg, 2023), device="cuda")
    fam = (lambda mm, sd: I.heat2d(mm, seed=sd)) if args.heat else \
        (lambda mm, sd: I.fem2d(mm, sigma=1.0, corr_len=0.1, seed=sd))
    held = [fam(args.m, 9000 + k) for k in range(3)]
    fam_name = "heat" if args.heat else "fem"
    ev = evaluate(N, cfg, w, held, precision=prec)
    ev0 = evaluate(N, cfg, w0, held[:1], precision=prec)
    small = evaluate(N, cfg, w, [fam(96, 9200)], precision=prec)
    big = evaluate(N, cfg, w, [I.heat2d(256, seed=0) if args.heat else I.fem2d_256(seed=0)], precision=prec)
    fd3 = evaluate(N, cfg, w, [I.fd3d(32, sigma=1.0, corr_len=0.1, seed=9300),
                               I.fd3d(64, sigma=1.5, corr_len=0.05, seed=9301)], precision=prec)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, _np(w).astype(np.float32))
    meta = {"config": {"n_mp": cfg.n_mp, "l": cfg.l, "l_mp": cfg.l_mp, "h": cfg.h, "diag_mode": cfg.diag_mode,
                       "x0_head": cfg.x0_head},
            "loss": "Eq. loss_A (Frobenius)" if cfg.loss else "Eq. loss_Ab",
            "train": {"steps": args.steps, "lr": args.lr, "lr_final": args.lr_final, "schedule": "cosine",
                      "batch": f"{args.per_group} systems x 2 pairs",
                      "selection": "checkpoint with the fewest validation PCG iterations",
                      "systems": f"groups of {args.per_group}: 2-D FEM {'heat steps (inputs.heat2d) ' if args.heat else ''}"
                                 f"lattices {sizes if sizes is not None else [args.m]} "
                                 f"(sigma 1, corr 0.1), 3-D FD sides {sizes3d or []} (sigma {args.sigma3d}, "
                                 + (f"corr {args.corr3d_cells} cells = {args.corr3d_cells} / (side + 1)"
                                    if args.corr3d_cells else f"corr {args.corr3d}") + ")",
                      "precision": args.precision, "head_only_from": os.path.basename(args.x0_from) if args.x0_from else None,
                      "initialised_from": os.path.basename(args.init) if args.init else None, **tm},
            "loss_first": hist[0], "loss_last": float(np.mean(hist[-20:])),
            f"heldout_{fam_name}{args.m}": ev, f"untrained_{fam_name}{args.m}": ev0, f"heldout_{fam_name}96": small,
            f"{fam_name}256_seed0": big,
            "heldout_fd3d": fd3,
            f"learned_iters_{fam_name}256": big[0]["learned"]}
    if args.eval128:
        # the benchmark system, and its deployed configuration (the network's
        # precision, FP32 triangular solves inside FP64 PCG)
        p128 = I.fd3d_128(seed=0)
        meta["fd3d_128_seed0"] = evaluate(N, cfg, w, [p128], precision=prec)
        rp, ci, v = N.assemble_system(p128)
        P128 = N.analyse(rp, ci)
        b128 = torch.as_tensor(I.rhs(P128.n, 0), device="cuda")
        L128 = N.gnn_factor(P128, v, b128, cfg, w, precision=prec)
        _, s128 = N.pcg_solve(P128, v, b128, N.PREC_LLT32, L128, rtol=1e-6, max_iter=VAL_MAX_ITER)
        meta["bench_iters"] = {"fd3d_128": s128[0]["iters"]}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    sys.exit(main())
