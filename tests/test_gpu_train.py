"""GPU parity of the training path: the loss Eq. (loss_Ab) and its
hand-written adjoint through the network (FP32) against the FP64 oracle, and
Adam against the oracle's step.

Tolerance: the adjoint runs in FP32 (unit roundoff 6e-8) through chains of
about ten MLP layers and reductions of up to a few hundred terms, so the
loss is compared at 1e-5 relative and the gradient at 1e-4 relative in the
2-norm of EVERY Linear's weight matrix and, separately, of its bias (a
whole-vector norm would let a small block be entirely wrong).

BF16 forward (mixed precision): the loss at 4e-2 (quadratic in L, whose bar
is 2e-2), the whole gradient at 4e-2 in the 2-norm, and every block at 8e-2.
A block's gradient is a sum over rows of products of two forward states;
where the inputs carry signs (the node encoder's input b / ||b||_inf with
b ~ N(0,1)) the sum cancels, |sum| << sum |.|, and the forward's relative
rounding is amplified by that ratio (5.9 % measured on the node encoder's
input layer).  A wrong block (a dropped term, a transposed operand, a
missing bias) is off by O(1) and fails either bar.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2305_16432_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_2305_16432_gb300 import build
    build.build()
    from paper_2305_16432_gb300 import npcg
    return npcg


def _gpu(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def grad_block_errors(cfg, gg, go):
    """Relative 2-norm error of the gradient of every Linear's W and b, in
    the flat layout (per Linear: W[out][in], then b[out])."""
    errs, k = [], 0
    for q, (fi, fo) in enumerate(cfg.linears()):
        for name, size in (("W", fi * fo), ("b", fo)):
            a, r = gg[k:k + size], go[k:k + size]
            nr = np.linalg.norm(r)
            e = np.linalg.norm(a - r) / nr if nr > 0 else np.linalg.norm(a)
            errs.append((e, f"linear {q} {name} ({fo}x{fi})"))
            k += size
    assert k == len(go) == len(gg)
    return errs


def assert_grad_blocks(cfg, gg, go, tol):
    bad = [(e, name) for e, name in grad_block_errors(cfg, gg, go) if not e <= tol]
    assert not bad, f"gradient blocks above {tol}: {bad[:6]}"


def assert_grad_bf16(cfg, gg, go):
    # the mixed-precision bars (module docstring)
    assert np.linalg.norm(gg - go) / np.linalg.norm(go) <= 4e-2
    assert_grad_blocks(cfg, gg, go, 8e-2)


def _pairs(A, k, seed):
    B = I.rhs(A.n, seed, count=k)
    X = np.linalg.solve(A.dense(), B.T).T
    return X, B


@pytest.mark.parametrize("cfg,prob", [
    (I.GnnConfig(n_mp=2, l=2, l_mp=2, h=16), I.fem2d(7, sigma=1.0, seed=3)),
    (I.GnnConfig(n_mp=3, l=1, l_mp=2, h=32), I.fd2d(6, 5, sigma=1.0, seed=4)),
    (I.GnnConfig(n_mp=2, l=2, l_mp=2, h=64), I.fem2d(12, sigma=1.0, seed=5)),
    (I.GnnConfig(n_mp=0, l=2, l_mp=2, h=16), I.fd3d(4, 3, 3, sigma=1.0, seed=6)),
    (I.GnnConfig(n_mp=2, l=2, l_mp=2, h=32, diag_mode=1), I.fem2d(9, sigma=1.0, seed=7)),
    (I.GnnConfig(n_mp=2, l=2, l_mp=2, h=64, diag_mode=2), I.fd3d(5, 4, 4, sigma=1.5, corr_len=0.2, seed=8)),
])
def test_loss_and_grad_parity(N, cfg, prob):
    om, ph = I.grf_features(prob)
    Ao = O.assemble(prob, om, ph)
    rp, ci, v = N.assemble_system(prob, om, ph)
    P = N.analyse(rp, ci)
    X, B = _pairs(Ao, 3, 17)
    w = I.gnn_weights(cfg, 2, scale=1.5)
    lo, go = O.loss_and_grad(cfg, Ao, X, B, w.astype(np.float64))
    lg, gg = N.loss_and_grad(P, v, _gpu(X), _gpu(B), cfg, _gpu(w, torch.float32))
    gg = gg.cpu().numpy().astype(np.float64)
    assert abs(lg - lo) <= 1e-5 * abs(lo)
    assert_grad_blocks(cfg, gg, go, 1e-4)


def test_loss_and_grad_batched_is_mean_over_systems(N):
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=16)
    probs = [I.fem2d(8, sigma=1.0, seed=8), I.fd2d(7, 5, sigma=1.0, seed=9)]
    w = I.gnn_weights(cfg, 3)
    As, cis, vs, Xs, Bs = [], [], [], [], []
    off, sys_ptr = 0, [0]
    for k, p in enumerate(probs):
        om, ph = I.grf_features(p)
        Ao = O.assemble(p, om, ph)
        rp, ci, v = N.assemble_system(p, om, ph)
        As.append(Ao)
        cis.append(ci.cpu().numpy() + off)
        vs.append(v.cpu().numpy())
        X, B = _pairs(Ao, 2, 30 + k)
        Xs.append(X)
        Bs.append(B)
        off += Ao.n
        sys_ptr.append(off)
    nnz_off = np.cumsum([0] + [a.nnz for a in As])
    rp_cat = np.concatenate([a.row_ptr[:-1] + nnz_off[k] for k, a in enumerate(As)] + [[nnz_off[-1]]])
    P = N.analyse(_gpu(rp_cat, torch.int32), _gpu(np.concatenate(cis), torch.int32), sys_ptr)
    Xc = np.concatenate(Xs, axis=1)
    Bc = np.concatenate(Bs, axis=1)
    lg, gg = N.loss_and_grad(P, _gpu(np.concatenate(vs)), _gpu(Xc), _gpu(Bc), cfg, _gpu(w, torch.float32))
    ref = [O.loss_and_grad(cfg, As[k], Xs[k], Bs[k], w.astype(np.float64)) for k in range(2)]
    lo = np.mean([r[0] for r in ref])
    go = np.mean([r[1] for r in ref], axis=0)
    assert abs(lg - lo) <= 1e-5 * abs(lo)
    gg = gg.cpu().numpy().astype(np.float64)
    assert_grad_blocks(cfg, gg, go, 1e-4)


def test_adam_matches_oracle(N):
    g = np.random.default_rng(0)
    w = g.standard_normal(1000).astype(np.float32)
    wo = w.astype(np.float64)
    m, v = np.zeros(1000), np.zeros(1000)
    wg = _gpu(w, torch.float32)
    mg = torch.zeros_like(wg)
    vg = torch.zeros_like(wg)
    for t in range(1, 6):
        grad = g.standard_normal(1000).astype(np.float32)
        O.adam(wo, grad.astype(np.float64), m, v, t)
        N.adam_step(wg, _gpu(grad, torch.float32), mg, vg, t)
    torch.cuda.synchronize()
    assert np.abs(wg.cpu().numpy() - wo).max() <= 1e-6


def test_autograd_function_matches_oracle_gradient(N):
    """The adjoint behind torch.autograd: backward() leaves the oracle's FP64
    gradient (scaled by the incoming gradient) in w.grad."""
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=32)
    prob = I.fem2d(10, sigma=1.0, seed=11)
    om, ph = I.grf_features(prob)
    Ao = O.assemble(prob, om, ph)
    rp, ci, v = N.assemble_system(prob, om, ph)
    P = N.analyse(rp, ci)
    X, B = _pairs(Ao, 2, 23)
    w = I.gnn_weights(cfg, 4, scale=1.5)
    lo, go = O.loss_and_grad(cfg, Ao, X, B, w.astype(np.float64))
    wt = _gpu(w, torch.float32).requires_grad_(True)
    loss = N.llt_loss(wt, P, v, _gpu(X), _gpu(B), cfg)
    (3.0 * loss).backward()
    assert abs(loss.item() - lo) <= 1e-5 * abs(lo)
    gg = wt.grad.cpu().numpy().astype(np.float64)
    assert_grad_blocks(cfg, gg, 3.0 * go, 1e-4)


@pytest.mark.parametrize("diag_mode", [0, 1, 2])
def test_loss_and_grad_bf16_forward(N, diag_mode):
    """Mixed precision: BF16 tensor-core forward, FP32 adjoint at its states.
    Bars derived from the BF16 bar on L (2e-2): the loss is quadratic in L
    (2 x 2e-2), and the gradient is bilinear in the residual and the
    network's states (again 2 x 2e-2, on every Linear's W and b)."""
    cfg = I.GnnConfig(n_mp=3, l=2, l_mp=2, h=64, diag_mode=diag_mode)
    prob = I.fem2d(14, sigma=1.0, seed=12)
    om, ph = I.grf_features(prob)
    Ao = O.assemble(prob, om, ph)
    rp, ci, v = N.assemble_system(prob, om, ph)
    P = N.analyse(rp, ci)
    X, B = _pairs(Ao, 2, 41)
    w = I.gnn_weights(cfg, 6, scale=1.5)
    lo, go = O.loss_and_grad(cfg, Ao, X, B, w.astype(np.float64))
    lg, gg = N.loss_and_grad(P, v, _gpu(X), _gpu(B), cfg, _gpu(w, torch.float32), precision=N.BF16)
    gg = gg.cpu().numpy().astype(np.float64)
    assert abs(lg - lo) <= 4e-2 * abs(lo)
    assert_grad_bf16(cfg, gg, go)


@pytest.mark.parametrize("prec,tl,tg", [("fp32", 1e-5, 1e-4), ("bf16", 4e-2, 4e-2)])
def test_loss_and_grad_x0_head(N, prec, tl, tg):
    """The loss with the initial-guess head's regression term and the
    gradient (head by its regression, trunk by Eq. (loss_Ab) alone) against
    the oracle; FP32 and the BF16 bars of the tests above."""
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=64, diag_mode=1, x0_head=1)
    prob = I.fem2d(12, sigma=1.0, seed=13)
    om, ph = I.grf_features(prob)
    Ao = O.assemble(prob, om, ph)
    rp, ci, v = N.assemble_system(prob, om, ph)
    P = N.analyse(rp, ci)
    X, B = _pairs(Ao, 2, 51)
    w = I.gnn_weights(cfg, 9, scale=1.5)
    lo, go = O.loss_and_grad(cfg, Ao, X, B, w.astype(np.float64))
    lg, gg = N.loss_and_grad(P, v, _gpu(X), _gpu(B), cfg, _gpu(w, torch.float32),
                             precision=N.FP32 if prec == "fp32" else N.BF16)
    gg = gg.cpu().numpy().astype(np.float64)
    assert abs(lg - lo) <= tl * abs(lo)
    if prec == "bf16":
        assert_grad_bf16(cfg, gg, go)
    else:
        assert_grad_blocks(cfg, gg, go, tg)


@pytest.mark.parametrize("cfg,prob", [
    (I.GnnConfig(n_mp=2, l=2, l_mp=2, h=16, diag_mode=1, loss=1), I.fem2d(9, sigma=1.0, seed=21)),
    (I.GnnConfig(n_mp=2, l=2, l_mp=2, h=32, diag_mode=0, loss=1), I.fd2d(8, 7, sigma=1.0, seed=22)),
    (I.GnnConfig(n_mp=1, l=2, l_mp=2, h=64, diag_mode=1, loss=1), I.heat2d(12, seed=23)),
])
def test_frobenius_loss_and_grad_parity(N, cfg, prob):
    """The Frobenius loss Eq. (loss_A), fill-in of L L^T included, and its
    gradient through the network against the oracle (the FP32 bars)."""
    om, ph = I.grf_features(prob)
    Ao = O.assemble(prob, om, ph)
    rp, ci, v = N.assemble_system(prob, om, ph)
    P = N.analyse(rp, ci)
    X, B = _pairs(Ao, 2, 61)
    w = I.gnn_weights(cfg, 4, scale=1.5)
    lo, go = O.loss_and_grad(cfg, Ao, X, B, w.astype(np.float64))
    lg, gg = N.loss_and_grad(P, v, _gpu(X), _gpu(B), cfg, _gpu(w, torch.float32))
    gg = gg.cpu().numpy().astype(np.float64)
    assert abs(lg - lo) <= 1e-5 * abs(lo)
    assert_grad_blocks(cfg, gg, go, 1e-4)


def test_frobenius_loss_batched_is_mean_over_systems(N):
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=16, diag_mode=1, loss=1)
    probs = [I.fem2d(8, sigma=1.0, seed=24), I.fd2d(7, 5, sigma=1.0, seed=25)]
    As, rps, cis, vs = [], [], [], []
    for p in probs:
        Ao = O.assemble(p)
        As.append(Ao)
    off, sys_ptr = 0, [0]
    for Ao in As:
        cis.append(Ao.col_idx + off)
        vs.append(Ao.val)
        off += Ao.n
        sys_ptr.append(off)
    nnz_off = np.cumsum([0] + [a.nnz for a in As])
    rp_cat = np.concatenate([a.row_ptr[:-1] + nnz_off[k] for k, a in enumerate(As)] + [[nnz_off[-1]]])
    P = N.analyse(_gpu(rp_cat, torch.int32), _gpu(np.concatenate(cis), torch.int32), sys_ptr)
    B = np.concatenate([I.rhs(a.n, 70 + k, count=2) for k, a in enumerate(As)], axis=1)
    X = np.zeros_like(B)
    w = I.gnn_weights(cfg, 5, scale=1.5)
    lg, gg = N.loss_and_grad(P, _gpu(np.concatenate(vs)), _gpu(X), _gpu(B), cfg, _gpu(w, torch.float32))
    los, gos = [], []
    for k, Ao in enumerate(As):
        Bk = B[:, sys_ptr[k]:sys_ptr[k + 1]]
        l, g = O.loss_and_grad(cfg, Ao, np.zeros_like(Bk), Bk, w.astype(np.float64))
        los.append(l)
        gos.append(g)
    lo, go = np.mean(los), np.mean(gos, axis=0)
    assert abs(lg - lo) <= 1e-5 * abs(lo)
    assert_grad_blocks(cfg, gg.cpu().numpy().astype(np.float64), go, 1e-4)


_C4 = {}


def _c4_member():
    """One member of the training workload's size: a 128 x 128 lattice FEM
    system (n = 15,876, about 110 k edges), the 6 x 64 network, one (x, b)
    pair; the oracle's FP64 loss and gradient computed once."""
    if not _C4:
        cfg = I.GnnConfig(n_mp=6, l=2, l_mp=2, h=64, diag_mode=1)
        prob = I.fem2d(128, sigma=1.0, corr_len=0.1, seed=1000)
        om, ph = I.grf_features(prob)
        Ao = O.assemble(prob, om, ph)
        B = I.rhs(Ao.n, 91, count=1)
        L, _ = O.ic0(Ao)
        x, _, _, st = O.pcg(Ao, B[0], O.PREC_LLT, L, rtol=1e-12)
        assert st == 0
        X = x[None, :]
        w = I.gnn_weights(cfg, 12)
        lo, go = O.loss_and_grad(cfg, Ao, X, B, w.astype(np.float64))
        _C4.update(cfg=cfg, prob=prob, om=om, ph=ph, X=X, B=B, w=w, lo=lo, go=go)
    return _C4


@pytest.mark.parametrize("prec,tl,tg", [("fp32", 1e-5, 1e-4), ("bf16", 4e-2, 4e-2)])
def test_loss_and_grad_training_size_member(N, prec, tl, tg):
    """A training-sized member against the oracle: many tiles of every
    kernel, and the many-CTA split of the tensor-core weight gradient with its
    partial sums, per Linear block at the FP32 and BF16 bars."""
    c = _c4_member()
    rp, ci, v = N.assemble_system(c["prob"], c["om"], c["ph"])
    P = N.analyse(rp, ci)
    lg, gg = N.loss_and_grad(P, v, _gpu(c["X"]), _gpu(c["B"]), c["cfg"], _gpu(c["w"], torch.float32),
                             precision=N.FP32 if prec == "fp32" else N.BF16)
    gg = gg.cpu().numpy().astype(np.float64)
    assert abs(lg - c["lo"]) <= tl * abs(c["lo"])
    if prec == "bf16":
        assert_grad_bf16(c["cfg"], gg, c["go"])
    else:
        assert_grad_blocks(c["cfg"], gg, c["go"], tg)
