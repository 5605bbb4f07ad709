"""Pins of the oracle's GNN (Sec. 4.2 "Architecture", App. A.3), the loss
Eq. (loss_Ab) with its gradient, and Adam (App. A.4)."""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from paper_2305_16432_gb300 import inputs as I


def _unpack(cfg, w):
    """Flat weights -> list of MLPs, each a list of (W, b)."""
    w = np.asarray(w, np.float64)
    lin = cfg.linears()
    mats, k = [], 0
    for fi, fo in lin:
        W = w[k:k + fi * fo].reshape(fo, fi)
        k += fi * fo
        b = w[k:k + fo]
        k += fo
        mats.append((W, b))
    sizes = [cfg.l + 1] * 2 + [cfg.l_mp + 1, cfg.l_mp + 1] * cfg.n_mp + [cfg.l + 1]
    if cfg.x0_head:
        sizes += [cfg.l + 1]
    out, k = [], 0
    for s in sizes:
        out.append(mats[k:k + s])
        k += s
    assert k == len(mats)
    return out


def _mlp(layers, X):
    """Batched MLP over the last axis: ReLU between Linears, none at the end."""
    for q, (W, b) in enumerate(layers):
        X = X @ W.T + b
        if q < len(layers) - 1:
            X = np.maximum(X, 0)
    return X


def _dense_gnn(cfg, D, b, w):
    return _dense_gnn_impl(cfg, D, b, w)


def _dense_gnn_impl(cfg, D, b, w):
    """Independent dense-tensor formulation: node features V [n, h], edge
    features E [n, n, h] on the nonzeros of D; message passing as a masked
    einsum.  Returns the lower-triangular L as a dense matrix."""
    n = D.shape[0]
    mask = D != 0
    mlps = _unpack(cfg, w)
    s = np.max(np.diag(D))
    binf = np.max(np.abs(b)) or 1.0
    V = _mlp(mlps[0], (b / binf)[:, None])
    if cfg.diag_mode == 2:
        # edge input: the Jacobi-scaled matrix D^-1/2 A D^-1/2
        dsq = np.sqrt(np.diag(D))
        Ein = D / np.outer(dsq, dsq)
    else:
        Ein = D / s
    E = _mlp(mlps[1], Ein[:, :, None]) * mask[:, :, None]
    for t in range(cfg.n_mp):
        agg = np.einsum("ijh,jh->ih", E, V)                 # sum_j e_ij (.) v_j
        V = _mlp(mlps[2 + 2 * t], np.concatenate([V, agg], 1))
        X = np.concatenate([E, np.broadcast_to(V[:, None, :], E.shape),
                            np.broadcast_to(V[None, :, :], E.shape)], 2)
        E = _mlp(mlps[3 + 2 * t], X) * mask[:, :, None]
    S = _mlp(mlps[2 + 2 * cfg.n_mp], E)[:, :, 0] * mask
    sym = 0.5 * (S + S.T)
    L = np.tril(sym, -1)
    if cfg.diag_mode == 1:
        # L' unit lower triangular, P = L' D L'^T with D = diag(A): L = L' D^1/2
        L[np.diag_indices(n)] = 1.0
        return (L @ np.diag(np.sqrt(np.diag(D)))) * np.tril(mask)
    if cfg.diag_mode == 2:
        # the rows scaled instead: L = D^1/2 L~, P = D^1/2 L~ L~^T D^1/2
        L[np.diag_indices(n)] = 1.0
        return (np.diag(np.sqrt(np.diag(D))) @ L) * np.tril(mask)
    sp = np.maximum(np.diag(S), 0) + np.log1p(np.exp(-np.abs(np.diag(S))))
    L[np.diag_indices(n)] = sp
    return math.sqrt(s) * L * np.tril(mask)


@pytest.mark.parametrize("cfg", [I.GnnConfig(n_mp=2, l=2, l_mp=2, h=4),
                                 I.GnnConfig(n_mp=3, l=1, l_mp=2, h=5),
                                 I.GnnConfig(n_mp=0, l=2, l_mp=2, h=3),
                                 I.GnnConfig(n_mp=2, l=2, l_mp=1, h=4, diag_mode=1),
                                 I.GnnConfig(n_mp=2, l=2, l_mp=2, h=4, diag_mode=2)])
def test_gnn_matches_dense_formulation(cfg):
    A = O.assemble(I.fem2d(6, sigma=1.0, seed=2))
    b = I.rhs(A.n, 3)
    w = I.gnn_weights(cfg, 7, scale=2.0)
    L = O.gnn_forward(cfg, A, b, w)
    Ld = _dense_gnn(cfg, A.dense(), b, w)
    assert np.allclose(L.dense(), Ld, rtol=1e-12, atol=1e-12 * np.abs(Ld).max())
    assert O.gnn_nparams(cfg) == cfg.nparams == len(w)


def test_gnn_zero_weights():
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=8)
    A = O.assemble(I.fd2d(5, 4, sigma=1.0, seed=1))
    L = O.gnn_forward(cfg, A, I.rhs(A.n, 1), np.zeros(cfg.nparams))
    D = L.dense()
    s = A.dense().diagonal().max()
    assert np.allclose(np.diag(D), math.sqrt(s) * math.log(2.0), rtol=1e-15)
    assert np.all(np.tril(D, -1) == 0)


def test_ldlt_mode_zero_weights_is_jacobi():
    # App. A.3 variant: with zero weights L' = I, so P = diag(A) (Jacobi)
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=8, diag_mode=1)
    A = O.assemble(I.fem2d(9, sigma=1.0, seed=4))
    L = O.gnn_forward(cfg, A, I.rhs(A.n, 1), np.zeros(cfg.nparams))
    assert np.allclose(L.dense() @ L.dense().T, np.diag(np.diag(A.dense())), rtol=1e-15, atol=0)
    b = I.rhs(A.n, 2)
    _, it_l, _, _ = O.pcg(A, b, O.PREC_LLT, L, rtol=1e-8)
    _, it_j, _, _ = O.pcg(A, b, O.PREC_JACOBI, rtol=1e-8)
    assert it_l == it_j


def test_scaled_mode_zero_weights_is_jacobi():
    # rows scaled: with zero weights L~ = I, so P = diag(A) again
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=8, diag_mode=2)
    A = O.assemble(I.fd3d(6, 5, 4, sigma=1.5, seed=4))
    L = O.gnn_forward(cfg, A, I.rhs(A.n, 1), np.zeros(cfg.nparams))
    assert np.allclose(L.dense() @ L.dense().T, np.diag(np.diag(A.dense())), rtol=1e-15, atol=0)


def _ssor_weights(cfg, omega):
    # n_mp = 0, l = 1, h = 2: the edge encoder splits its input x into
    # (relu(x), relu(-x)) and passes them on, the decoder returns
    # omega (relu(x) - relu(-x)) = omega x, so s_ij = omega * input_ij
    assert (cfg.n_mp, cfg.l, cfg.h) == (0, 1, 2)
    parts = []
    for fi, fo in cfg.linears():
        parts.append(np.zeros(fi * fo + fo))
    enc_e1, enc_e2, dec1, dec2 = 2, 3, 4, 5
    parts[enc_e1][:2] = [1.0, -1.0]                      # W [2][1]
    parts[enc_e2][:4] = [1.0, 0.0, 0.0, 1.0]             # identity [2][2]
    parts[dec1][:4] = [1.0, 0.0, 0.0, 1.0]
    parts[dec2][:2] = [omega, -omega]                    # W [1][2]
    return np.concatenate(parts)


@pytest.mark.parametrize("omega", [1.0, 1.6])
def test_scaled_mode_represents_ssor(omega):
    # rows scaled with L~_ij = omega (D^-1/2 A D^-1/2)_ij gives the SSOR
    # factor L = (D + omega L_A) D^-1/2, and at omega = 1 symmetric
    # Gauss-Seidel, the oracle's own sgs factor
    cfg = I.GnnConfig(n_mp=0, l=1, l_mp=1, h=2, diag_mode=2)
    A = O.assemble(I.fd3d(6, 5, 4, sigma=1.5, seed=7))
    w = _ssor_weights(cfg, omega)
    L = O.gnn_forward(cfg, A, I.rhs(A.n, 2), w)
    D = A.dense()
    d = np.diag(D)
    ref = (np.diag(d) + omega * np.tril(D, -1)) @ np.diag(1.0 / np.sqrt(d))
    assert np.allclose(L.dense(), ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())
    if omega == 1.0:
        assert np.allclose(L.val, O.sgs(A).val, rtol=1e-14, atol=0)


def test_gnn_no_message_passing_is_elementwise():
    # n_mp = 0: L_ij depends on A_ij only (A symmetric), L_ii on A_ii only
    cfg = I.GnnConfig(n_mp=0, l=2, l_mp=2, h=6)
    w = I.gnn_weights(cfg, 3)
    A = O.assemble(I.fd2d(6, 6, sigma=1.0, seed=4))
    L1 = O.gnn_forward(cfg, A, I.rhs(A.n, 1), w)
    L2 = O.gnn_forward(cfg, A, I.rhs(A.n, 2), w)      # b does not reach L
    assert np.array_equal(L1.val, L2.val)
    _, a2l = O.tril(A)
    vals = {}
    for k in range(A.nnz):
        if a2l[k] >= 0:
            vals.setdefault(round(A.val[k], 15), set()).add(round(L1.val[a2l[k]], 12))
    assert all(len(v) == 1 for v in vals.values())


def test_gnn_permutation_equivariance():
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=6)
    w = I.gnn_weights(cfg, 5, scale=1.5)
    A = O.assemble(I.fem2d(7, sigma=1.0, seed=9))
    b = I.rhs(A.n, 9)
    D = A.dense()
    perm = np.random.default_rng(0).permutation(A.n)
    Dp = D[np.ix_(perm, perm)]
    rp, ci, v = [0], [], []
    for i in range(A.n):
        nz = np.nonzero(Dp[i])[0]
        ci += list(nz)
        v += list(Dp[i, nz])
        rp.append(len(ci))
    Ap = O.CSR(rp, ci, v)
    _, s = O.gnn_forward(cfg, A, b, w, return_s=True)
    _, sp = O.gnn_forward(cfg, Ap, b[perm], w, return_s=True)
    S = np.zeros_like(D)
    Sp = np.zeros_like(D)
    for M, AA, ss in ((S, A, s), (Sp, Ap, sp)):
        for i in range(AA.n):
            for k in range(AA.row_ptr[i], AA.row_ptr[i + 1]):
                M[i, AA.col_idx[k]] = ss[k]
    assert np.allclose(Sp, S[np.ix_(perm, perm)], rtol=1e-12, atol=1e-12)


def test_gnn_preconditioner_is_spd():
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=8)
    A = O.assemble(I.fem2d(8, sigma=1.0, seed=5))
    L = O.gnn_forward(cfg, A, I.rhs(A.n, 0), I.gnn_weights(cfg, 1))
    P = L.dense() @ L.dense().T
    assert np.allclose(P, P.T) and np.linalg.eigvalsh(P).min() > 0


# ----------------------------------------------------------------- loss
def _tiny_system():
    A = O.assemble(I.fem2d(5, sigma=1.0, seed=3))          # n = 9
    return A


def test_loss_zero_for_exact_factor_and_solution():
    n = 12
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    rp, ci, v = [0], [], []
    for i in range(n):
        nz = np.nonzero(T[i])[0]
        ci += list(nz)
        v += list(T[i, nz])
        rp.append(len(ci))
    A = O.CSR(rp, ci, v)
    L, _ = O.ic0(A)                                          # exact on a tridiagonal
    B = I.rhs(n, 4, count=3)
    X = np.linalg.solve(T, B.T).T
    loss, dL = O.llt_loss(L, X, B)
    assert loss < 1e-25 and np.abs(dL).max() < 1e-12


def test_loss_gradient_wrt_L_by_finite_differences():
    A = _tiny_system()
    L, _ = O.ic0(A)
    g = np.random.default_rng(0)
    L = O.CSR(L.row_ptr, L.col_idx, L.val + 0.1 * g.standard_normal(L.nnz))
    X = g.standard_normal((3, A.n))
    B = g.standard_normal((3, A.n))
    loss, dL = O.llt_loss(L, X, B)
    # loss definition by dense matrices
    Ld = L.dense()
    dense = np.mean([np.sum((Ld @ Ld.T @ X[p] - B[p]) ** 2) for p in range(3)])
    assert math.isclose(loss, dense, rel_tol=1e-13)
    eps = 1e-6
    for k in range(L.nnz):
        vp, vm = L.val.copy(), L.val.copy()
        vp[k] += eps
        vm[k] -= eps
        fp = O.llt_loss(O.CSR(L.row_ptr, L.col_idx, vp), X, B, False)[0]
        fm = O.llt_loss(O.CSR(L.row_ptr, L.col_idx, vm), X, B, False)[0]
        fd = (fp - fm) / (2 * eps)
        assert abs(fd - dL[k]) <= 1e-6 * max(1.0, abs(dL[k]))


@pytest.mark.parametrize("cfg", [I.GnnConfig(n_mp=2, l=2, l_mp=2, h=3),
                                 I.GnnConfig(n_mp=1, l=1, l_mp=1, h=4),
                                 I.GnnConfig(n_mp=1, l=2, l_mp=1, h=3, diag_mode=1),
                                 I.GnnConfig(n_mp=1, l=2, l_mp=1, h=3, diag_mode=2)])
def test_loss_and_grad_central_differences(cfg):
    # central differences, eps = 1e-6, FP64, on every weight
    A = _tiny_system()
    g = np.random.default_rng(1)
    B = g.standard_normal((2, A.n))
    X = np.linalg.solve(A.dense(), B.T).T
    w = I.gnn_weights(cfg, 2, scale=1.5).astype(np.float64)
    loss, grad = O.loss_and_grad(cfg, A, X, B, w)
    # relative error per weight; components far below the largest one are
    # measured against 1e-3 of it, because there the rounding noise of the
    # difference quotient (~ 1e-16 * loss / eps) dominates
    eps = 1e-6
    floor = 1e-3 * np.abs(grad).max()
    err = 0.0
    for k in range(len(w)):
        wp, wm = w.copy(), w.copy()
        wp[k] += eps
        wm[k] -= eps
        fd = (O.loss_and_grad(cfg, A, X, B, wp, False)[0] -
              O.loss_and_grad(cfg, A, X, B, wm, False)[0]) / (2 * eps)
        err = max(err, abs(fd - grad[k]) / max(floor, abs(grad[k])))
    assert err < 1e-6, err
    # loss equals the mean over pairs of ||L L^T x - b||^2 of the forward L
    lp = []
    for p in range(2):
        L = O.gnn_forward(cfg, A, B[p], w).dense()
        lp.append(np.sum((L @ L.T @ X[p] - B[p]) ** 2))
    assert math.isclose(loss, np.mean(lp), rel_tol=1e-12)


def test_adam_single_step_by_hand():
    # w = [1, -2], g = [0.5, -0.1], first step: m_hat = g, v_hat = g^2,
    # update = lr * g / (|g| + eps)
    w = np.array([1.0, -2.0])
    g = np.array([0.5, -0.1])
    m, v = np.zeros(2), np.zeros(2)
    O.adam(w, g, m, v, 1)
    expect = np.array([1.0 - 1e-3 * 0.5 / (0.5 + 1e-8), -2.0 + 1e-3 * 0.1 / (0.1 + 1e-8)])
    assert np.allclose(w, expect, rtol=0, atol=1e-15)
    assert np.allclose(m, [0.05, -0.01]) and np.allclose(v, [0.00025, 0.00001])
    # second step with the same gradient: m = 0.19 g, v = 0.001999 g^2
    O.adam(w, g, m, v, 2)
    mh = 0.19 * g / (1 - 0.81)
    vh = 0.001999 * g * g / (1 - 0.998001)
    expect2 = expect - 1e-3 * mh / (np.sqrt(vh) + 1e-8)
    assert np.allclose(w, expect2, rtol=0, atol=1e-15)


@pytest.mark.parametrize("prob", [I.fem2d(16, sigma=1.0, seed=21), I.fd3d(7, 6, 5, sigma=1.0, seed=22)])
def test_gnn_rows_on_neighbourhood_balls(prob):
    """Sampled rows of a large system's L (the full-size parity harness): the
    rows computed on the (n_mp + 1)-hop ball with the parent's scales equal the
    full forward's rows bit for bit, and a ball one hop smaller does not."""
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=8)
    A = O.assemble(prob)
    b = I.rhs(A.n, 4)
    w = I.gnn_weights(cfg, 9, scale=2.0)
    L = O.gnn_forward(cfg, A, b, w)
    rows = [0, A.n // 3, A.n // 2 + 1, A.n - 1]
    got = O.gnn_rows(cfg, A, b, w, rows)
    for r in rows:
        s, e = L.row_ptr[r], L.row_ptr[r + 1]
        cols, vals = got[r]
        assert np.array_equal(cols, L.col_idx[s:e])
        assert np.array_equal(vals, L.val[s:e])
    # one hop short: an interior row sees truncated neighbourhoods
    r = A.n // 2 + 1
    nodes = O.ball(A, [r], cfg.n_mp)
    rows_of = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    s_max = float(A.val[A.col_idx == rows_of].max())
    Ls = O.gnn_forward_scaled(cfg, O.induced(A, nodes), b[nodes], w, s_max, float(np.abs(b).max()))
    k = int(np.searchsorted(nodes, r))
    s, e = L.row_ptr[r], L.row_ptr[r + 1]
    assert not np.allclose(Ls.val[Ls.row_ptr[k]:Ls.row_ptr[k + 1]], L.val[s:e], rtol=1e-9, atol=0)


def _dense_x0(cfg, D, b, w):
    """Initial guess of the head in the dense formulation: the final node
    features V through the head MLP, scaled by ||b||_inf / s."""
    n = D.shape[0]
    mask = D != 0
    mlps = _unpack(cfg, w)
    s = np.max(np.diag(D))
    binf = np.max(np.abs(b)) or 1.0
    V = _mlp(mlps[0], (b / binf)[:, None])
    E = _mlp(mlps[1], (D / s)[:, :, None]) * mask[:, :, None]
    for t in range(cfg.n_mp):
        agg = np.einsum("ijh,jh->ih", E, V)
        V = _mlp(mlps[2 + 2 * t], np.concatenate([V, agg], 1))
        X = np.concatenate([E, np.broadcast_to(V[:, None, :], E.shape),
                            np.broadcast_to(V[None, :, :], E.shape)], 2)
        E = _mlp(mlps[3 + 2 * t], X) * mask[:, :, None]
    return binf / s * _mlp(mlps[-1], V)[:, 0]


@pytest.mark.parametrize("cfg", [I.GnnConfig(n_mp=2, l=2, l_mp=2, h=4, diag_mode=1, x0_head=1),
                                 I.GnnConfig(n_mp=0, l=1, l_mp=2, h=3, x0_head=1)])
def test_x0_head_matches_dense_formulation(cfg):
    A = _tiny_system()
    b = np.random.default_rng(3).standard_normal(A.n)
    w = I.gnn_weights(cfg, 5, scale=1.5).astype(np.float64)
    assert np.allclose(O.gnn_x0(cfg, A, b, w), _dense_x0(cfg, A.dense(), b, w), rtol=1e-12, atol=1e-13)
    # the factor does not depend on the head
    base = dataclasses.replace(cfg, x0_head=0)
    nb = base.nparams
    assert np.array_equal(O.gnn_forward(cfg, A, b, w).val, O.gnn_forward(base, A, b, w[:nb]).val)


def test_x0_head_constant_output():
    # head weights zero except the last bias c: x0 = (||b||_inf / s) c everywhere
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=1, h=4, x0_head=1)
    A = _tiny_system()
    b = np.random.default_rng(4).standard_normal(A.n)
    w = I.gnn_weights(cfg, 6).astype(np.float64)
    nb = dataclasses.replace(cfg, x0_head=0).nparams
    w[nb:] = 0.0
    w[-1] = 0.75
    s = np.max(np.diag(A.dense()))
    assert np.allclose(O.gnn_x0(cfg, A, b, w), np.max(np.abs(b)) / s * 0.75, rtol=1e-14)


def test_x0_head_gradient():
    # the head is trained by regression to x in its output units; the trunk
    # is not differentiated through it: head weights match central
    # differences of the total loss, trunk weights match the gradient of the
    # network without the head
    cfg = I.GnnConfig(n_mp=1, l=2, l_mp=1, h=3, diag_mode=1, x0_head=1)
    base = dataclasses.replace(cfg, x0_head=0)
    nb = base.nparams
    A = _tiny_system()
    g = np.random.default_rng(7)
    B = g.standard_normal((2, A.n))
    X = np.linalg.solve(A.dense(), B.T).T
    w = I.gnn_weights(cfg, 8, scale=1.5).astype(np.float64)
    loss, grad = O.loss_and_grad(cfg, A, X, B, w)
    lb, gb = O.loss_and_grad(base, A, X, B, w[:nb])
    assert np.allclose(grad[:nb], gb, rtol=1e-12, atol=1e-14 * np.abs(gb).max())
    s = np.max(np.diag(A.dense()))
    lx = np.mean([np.sum((_dense_x0(cfg, A.dense(), B[p], w) - X[p]) ** 2) * (s / np.max(np.abs(B[p]))) ** 2
                  for p in range(2)])
    assert math.isclose(loss, lb + lx, rel_tol=1e-10)
    eps = 1e-6
    floor = 1e-3 * np.abs(grad[nb:]).max()
    err = 0.0
    for k in range(nb, len(w)):
        wp, wm = w.copy(), w.copy()
        wp[k] += eps
        wm[k] -= eps
        fd = (O.loss_and_grad(cfg, A, X, B, wp, False)[0] - O.loss_and_grad(cfg, A, X, B, wm, False)[0]) / (2 * eps)
        err = max(err, abs(fd - grad[k]) / max(floor, abs(grad[k])))
    assert err < 1e-6, err


# ------------------------------------------------------------------ Frobenius loss Eq. (loss_A)
def _csr(D):
    rp, ci, v = [0], [], []
    for i in range(D.shape[0]):
        nz = np.nonzero(D[i])[0]
        ci += list(nz)
        v += list(D[i, nz])
        rp.append(len(ci))
    return O.CSR(rp, ci, v)


def test_frob_loss_zero_at_exact_factor():
    # tridiagonal A has a fill-free Cholesky factor on tril(A): L L^T = A,
    # so the loss and its gradient vanish
    n = 9
    D = 2.5 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    A = _csr(D)
    Lc = np.linalg.cholesky(D)
    L = _csr(np.where(np.tril(D) != 0, Lc, 0.0))
    loss, dL = O.frob_loss(A, L)
    assert loss < 1e-26 and np.abs(dL).max() < 1e-13


def test_frob_loss_closed_form_diagonal_factor():
    # L = c I: ||c^2 I - A||_F^2 = sum_i (c^2 - a_ii)^2 + sum_{i != j} a_ij^2,
    # dl/dL_ii = 4 ((c^2 I - A) c I)_ii = 4 c (c^2 - a_ii)
    A = O.assemble(I.fem2d(7, sigma=1.0, seed=2))
    D = A.dense()
    c = 1.7
    L = _csr(np.diag(np.full(A.n, c)))
    loss, dL = O.frob_loss(A, L)
    d = np.diag(D)
    expect = np.sum((c * c - d) ** 2) + np.sum(D ** 2) - np.sum(d ** 2)
    assert math.isclose(loss, expect, rel_tol=1e-13)
    assert np.allclose(dL, 4 * c * (c * c - d), rtol=1e-13)


def test_frob_loss_includes_fill_in():
    # the product L L^T of a 2-D FEM factor has entries outside pattern(A)
    # (two-hop fill); the loss counts them: against the same loss taken on
    # pattern(A) only it is strictly larger
    A = O.assemble(I.fem2d(8, sigma=1.0, seed=3))
    Lic, _ = O.ic0(A)
    loss, _ = O.frob_loss(A, Lic)
    P = Lic.dense() @ Lic.dense().T - A.dense()
    on_pattern = np.sum((P * (A.dense() != 0)) ** 2)
    assert math.isclose(loss, np.sum(P ** 2), rel_tol=1e-12) and loss > on_pattern * (1 + 1e-6)


def test_frob_loss_gradient_central_differences():
    A = O.assemble(I.fd2d(5, 4, sigma=1.0, seed=4))
    L0, _ = O.ic0(A)
    g = np.random.default_rng(2)
    L = O.CSR(L0.row_ptr, L0.col_idx, L0.val * (1 + 0.2 * g.standard_normal(L0.nnz)))
    loss, dL = O.frob_loss(A, L)
    eps = 1e-6
    for k in range(L.nnz):
        vp, vm = L.val.copy(), L.val.copy()
        vp[k] += eps
        vm[k] -= eps
        fd = (O.frob_loss(A, O.CSR(L.row_ptr, L.col_idx, vp), False)[0] -
              O.frob_loss(A, O.CSR(L.row_ptr, L.col_idx, vm), False)[0]) / (2 * eps)
        assert abs(fd - dL[k]) <= 1e-6 * max(1.0, abs(dL[k]))


def test_frob_network_gradient_central_differences():
    # through the network: the weights' gradient of the mean Frobenius loss
    # over two pairs (each pair has its own L = f(A, b_p)) matches central
    # differences; with cfg.loss = 1 the (x, b) data enter only as the input b
    cfg = I.GnnConfig(n_mp=1, l=2, l_mp=1, h=3, diag_mode=1, loss=1)
    A = _tiny_system()
    g = np.random.default_rng(9)
    B = g.standard_normal((2, A.n))
    X = g.standard_normal((2, A.n))
    w = I.gnn_weights(cfg, 3, scale=1.5).astype(np.float64)
    loss, grad = O.loss_and_grad(cfg, A, X, B, w)
    Ls = [O.gnn_forward(cfg, A, B[p], w) for p in range(2)]
    assert math.isclose(loss, np.mean([O.frob_loss(A, L, False)[0] for L in Ls]), rel_tol=1e-13)
    assert O.loss_and_grad(cfg, A, X + 1.0, B, w, False)[0] == loss
    eps = 1e-6
    floor = 1e-3 * np.abs(grad).max()
    err = 0.0
    for k in range(len(w)):
        wp, wm = w.copy(), w.copy()
        wp[k] += eps
        wm[k] -= eps
        fd = (O.loss_and_grad(cfg, A, X, B, wp, False)[0] - O.loss_and_grad(cfg, A, X, B, wm, False)[0]) / (2 * eps)
        err = max(err, abs(fd - grad[k]) / max(floor, abs(grad[k])))
    assert err < 1e-6, err
