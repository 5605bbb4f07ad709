"""Writes tests/golden/poisson2d_32_oracle.json from the oracle alone: the
32 x 32 Poisson configuration (k = 1, b ~ N(0,1) seed 0, a 2-layer width-16
network with seeded weights, softplus diagonal), its IC(0), learned-L and
plain-CG PCG iteration counts at 1e-8 and summaries of the factors and
solutions.  A regression fixture of the oracle, not a value from the paper:
a change of the oracle's arithmetic shows up as a mismatch and needs the
passage that justifies it."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2305_16432_gb300 import inputs as I  # noqa: E402


def compute():
    prob = I.poisson2d_32()
    A = O.assemble(prob)
    b = I.rhs(A.n, 0)
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=16)
    w = I.gnn_weights(cfg, 1).astype(np.float64)
    Ll = O.gnn_forward(cfg, A, b, w)
    Li, alpha = O.ic0(A)
    xl, itl, _, _ = O.pcg(A, b, O.PREC_LLT, Ll, rtol=1e-8)
    xi, iti, _, _ = O.pcg(A, b, O.PREC_LLT, Li, rtol=1e-8)
    xc, itc, _, _ = O.pcg(A, b, O.PREC_NONE, rtol=1e-8)
    xs, its, _, _ = O.pcg(A, b, O.PREC_LLT, O.sgs(A), rtol=1e-8)
    lev, nf, _, nb = O.levels(Li)
    return {
        "n": int(A.n), "nnz": int(A.nnz), "levels_fwd": int(nf), "levels_bwd": int(nb),
        "iters": {"learned_random_L": int(itl), "ic0": int(iti), "cg": int(itc), "sgs": int(its)},
        "ic0_shift": float(alpha),
        "sum_L_learned": float(Ll.val.sum()), "sum_L_ic0": float(Li.val.sum()),
        "norm_x_learned": float(np.linalg.norm(xl)), "norm_x_ic0": float(np.linalg.norm(xi)),
    }


if __name__ == "__main__":
    O.build()
    out = os.path.join(HERE, "poisson2d_32_oracle.json")
    with open(out, "w") as f:
        json.dump(compute(), f, indent=1)
    print(out)
