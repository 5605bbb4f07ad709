"""What training gains (behavioural, not parity): the committed 6 x 64
network (L D L^T with D = diag(A), App. A.3), trained on the GPU by this
library's own forward, adjoint and Adam kernels
(paper_2305_16432_gb300/train.py) on 2-D FEM and 3-D FD systems, needs fewer
PCG iterations than the same network untrained and than Jacobi on held-out
systems, and stays within 1.5x of IC(0)'s iterations there."""
import json
import os

import numpy as np
import pytest
import torch

from paper_2305_16432_gb300 import inputs as I

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2305_16432_gb300", "weights", "gnn_6x64.npy")


@pytest.fixture(scope="module")
def N():
    from paper_2305_16432_gb300 import build
    build.build()
    from paper_2305_16432_gb300 import npcg
    return npcg


@pytest.mark.parametrize("prob", [I.fem2d(128, sigma=1.0, corr_len=0.1, seed=9100),
                                  I.fem2d(96, sigma=1.0, corr_len=0.1, seed=9200),
                                  I.fem2d(200, sigma=1.0, corr_len=0.1, seed=9400),
                                  I.fd3d(28, sigma=1.0, corr_len=0.1, seed=9500)])
def test_trained_beats_untrained_and_jacobi(N, prob):
    meta = json.load(open(os.path.splitext(WEIGHTS)[0] + ".json"))
    cfg = I.GnnConfig(**meta["config"])
    w = torch.as_tensor(np.load(WEIGHTS), device="cuda")
    w0 = torch.as_tensor(I.gnn_weights(cfg, 2023), device="cuda")
    rp, ci, v = N.assemble_system(prob)
    P = N.analyse(rp, ci)
    b = torch.as_tensor(I.rhs(P.n, prob.seed), device="cuda")
    it = {}
    for name, ww in (("trained", w), ("untrained", w0)):
        L = N.gnn_factor(P, v, b, cfg, ww)
        _, st = N.pcg_solve(P, v, b, N.PREC_LLT, L, rtol=1e-6)
        assert st[0]["status"] == 0
        it[name] = st[0]["iters"]
    _, sj = N.pcg_solve(P, v, b, N.PREC_JACOBI, None, rtol=1e-6)
    Lic, _ = N.ic0_factor(P, v)
    _, si = N.pcg_solve(P, v, b, N.PREC_LLT, Lic, rtol=1e-6)
    assert it["trained"] < it["untrained"]
    assert it["trained"] < sj[0]["iters"]
    assert it["trained"] <= 1.5 * si[0]["iters"]
