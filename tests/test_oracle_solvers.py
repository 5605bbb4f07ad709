"""Pins of the oracle's sparse kernels, level sets, IC(0) and PCG
(Algorithm 1) against dense linear algebra, closed forms and brute force."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2305_16432_gb300 import inputs as I


def _csr_from_dense(D):
    rp, ci, v = [0], [], []
    for i in range(D.shape[0]):
        nz = np.nonzero(D[i])[0]
        ci += list(nz)
        v += list(D[i, nz])
        rp.append(len(ci))
    return O.CSR(rp, ci, v)


def _random_spd_sparse(n, density, seed, positive_offdiag=False):
    g = np.random.default_rng(seed)
    M = (g.random((n, n)) < density).astype(float) * g.uniform(0.2, 1.0, (n, n))
    M = np.triu(M, 1)
    M = M + M.T
    if not positive_offdiag:
        M = -M
    D = M + np.diag(np.abs(M).sum(1) + g.uniform(0.1, 1.0, n))
    return D


def test_spmv_matches_dense():
    A = O.assemble(I.fem2d(10, seed=1))
    x = np.random.default_rng(0).standard_normal(A.n)
    assert np.allclose(O.spmv(A, x), A.dense() @ x, rtol=1e-14, atol=1e-14)


def test_tril_pattern():
    A = O.assemble(I.fem2d(11, seed=2))
    L, a2l = O.tril(A)
    assert np.array_equal(L.dense(), np.tril(A.dense()))
    # diagonal is the last entry of each row of L
    for i in range(L.n):
        assert L.col_idx[L.row_ptr[i + 1] - 1] == i
    assert np.sum(a2l >= 0) == L.nnz == (A.nnz + A.n) // 2


def test_levels_closed_form_2d_3d():
    nx, ny = 7, 5
    L, _ = O.tril(O.assemble(I.fd2d(nx, ny)))
    lev, nf, levb, nb = O.levels(L)
    x, y = np.meshgrid(np.arange(nx), np.arange(ny))
    assert np.array_equal(lev, (x + y).ravel())
    assert np.array_equal(levb, ((nx - 1 - x) + (ny - 1 - y)).ravel())
    assert nf == nb == nx + ny - 1
    L3, _ = O.tril(O.assemble(I.fd3d(4, 3, 5)))
    lev3, nf3, _, _ = O.levels(L3)
    z, y, x = np.meshgrid(np.arange(5), np.arange(3), np.arange(4), indexing="ij")
    assert np.array_equal(lev3, (x + y + z).ravel()) and nf3 == 4 + 3 + 5 - 2
    # 32 x 32 grid: 63 levels
    L1, _ = O.tril(O.assemble(I.poisson2d_32()))
    assert O.levels(L1)[1] == 63


def _longest_path_bruteforce(n, edges_to):
    """Longest dependency chain ending at each node, by enumerating every
    path (depth-first, exponential; tiny n only)."""
    best = [0] * n

    def walk(node, length):
        best[node] = max(best[node], length)
        for nxt in edges_to[node]:
            walk(nxt, length + 1)
    for s in range(n):
        walk(s, 0)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_levels_bruteforce_random_dag(seed):
    n = 11
    D = _random_spd_sparse(n, 0.3, seed)
    L, _ = O.tril(_csr_from_dense(D))
    lev, nf, levb, nb = O.levels(L)
    # forward: edge j -> i for L_ij != 0, j < i
    fwd = [[] for _ in range(n)]
    bwd = [[] for _ in range(n)]
    for i in range(n):
        for k in range(L.row_ptr[i], L.row_ptr[i + 1]):
            j = L.col_idx[k]
            if j < i:
                fwd[j].append(i)
                bwd[i].append(j)
    assert list(lev) == _longest_path_bruteforce(n, fwd)
    assert list(levb) == _longest_path_bruteforce(n, bwd)
    perm, ptr = O.level_perm(lev, nf)
    assert np.array_equal(perm, np.lexsort((np.arange(n), lev)))
    assert ptr[-1] == n and np.array_equal(np.diff(ptr), np.bincount(lev, minlength=nf))


def test_trsv_matches_library():
    A = O.assemble(I.fem2d(12, seed=3))
    Lic, _ = O.ic0(A)
    r = np.random.default_rng(1).standard_normal(A.n)
    Ld = Lic.dense()
    y = O.trsv_lower(Lic, r)
    assert np.allclose(y, sla.solve_triangular(Ld, r, lower=True), rtol=1e-12, atol=1e-12)
    z = O.trsv_upper(Lic, y)
    assert np.allclose(z, sla.solve_triangular(Ld.T, y, lower=False), rtol=1e-12, atol=1e-12)


def test_ic0_tridiagonal_closed_form():
    # tridiag(-1, 2, -1): L_kk = sqrt((k+1)/k), L_{k+1,k} = -sqrt(k/(k+1)) (1-based)
    n = 9
    D = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    L, alpha = O.ic0(_csr_from_dense(D))
    Ld = L.dense()
    k = np.arange(1, n + 1)
    assert alpha == 0.0
    assert np.allclose(np.diag(Ld), np.sqrt((k + 1) / k), rtol=1e-15)
    assert np.allclose(np.diag(Ld, -1), -np.sqrt(k[:-1] / (k[:-1] + 1)), rtol=1e-15)


def test_ic0_equals_cholesky_when_no_fill():
    # tridiagonal or full pattern: IC(0) is the exact Cholesky factor
    g = np.random.default_rng(4)
    n = 12
    T = np.diag(g.uniform(3, 4, n)) + np.diag(g.uniform(-1, 1, n - 1), 1)
    T = np.triu(T) + np.triu(T, 1).T
    for D in (T, _random_spd_sparse(8, 1.0, 5)):
        L, _ = O.ic0(_csr_from_dense(D))
        assert np.allclose(L.dense(), np.linalg.cholesky(D), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("prob", [I.poisson2d_32(), I.fem2d(16, seed=7), I.fd3d(6, sigma=1.0, seed=3)])
def test_ic0_defining_property(prob):
    # (L L^T)_ij = A_ij on pattern(tril A)
    A = O.assemble(prob)
    L, alpha = O.ic0(A)
    assert alpha == 0.0
    LL = L.dense() @ L.dense().T
    D = A.dense()
    mask = np.tril(D != 0)
    assert np.allclose(LL[mask], D[mask], rtol=1e-13, atol=1e-13 * np.abs(D).max())


def test_ic0_breakdown_shift():
    # Kershaw's 4 x 4 SPD matrix (D. S. Kershaw, J. Comput. Phys. 26, 1978):
    # IC(0) meets a negative pivot.  The shifted retry must report
    # alpha = 1e-3 * 2^t and factor A + alpha diag(A) on the pattern.
    D = np.array([[3, -2, 0, 2], [-2, 3, -2, 0], [0, -2, 3, -2], [2, 0, -2, 3.0]])
    assert np.linalg.eigvalsh(D).min() > 0
    L, alpha = O.ic0(_csr_from_dense(D))
    assert alpha > 0
    t = math.log2(alpha / 1e-3)
    assert t == int(round(t))
    Ds = D + alpha * np.diag(np.diag(D))
    mask = np.tril(D != 0)
    LL = L.dense() @ L.dense().T
    assert np.allclose(LL[mask], Ds[mask], rtol=1e-12, atol=1e-12)
    # the previous shift must still break down (smallest working shift)
    if t > 0:
        prev = alpha / 2
        Dp = D + prev * np.diag(np.diag(D))
        # plain Cholesky-like recurrence on the pattern hits a pivot <= 0
        Lp, a2 = O.ic0(_csr_from_dense(Dp))
        assert a2 > 0


def test_cg_terminates_within_n_steps():
    n = 16
    D = _random_spd_sparse(n, 1.0, 9)
    A = _csr_from_dense(D)
    b = np.random.default_rng(3).standard_normal(n)
    x, it, rr, st = O.pcg(A, b, O.PREC_NONE, rtol=1e-10, max_iter=10 * n)
    assert st == 0 and it <= n
    assert np.allclose(x, np.linalg.solve(D, b), rtol=1e-9, atol=1e-9)
    # few distinct eigenvalues: CG ends in as many steps
    Q = np.linalg.qr(np.random.default_rng(4).standard_normal((n, n)))[0]
    D3 = Q @ np.diag(np.repeat([1.0, 4.0, 9.0], [5, 5, 6])) @ Q.T
    x, it, rr, st = O.pcg(_csr_from_dense(D3), b, O.PREC_NONE, rtol=1e-10)
    assert st == 0 and it <= 3


def test_exact_factor_converges_in_one_iteration():
    n = 14
    D = _random_spd_sparse(n, 1.0, 2)         # full pattern: tril holds the exact factor
    A = _csr_from_dense(D)
    Lch = np.linalg.cholesky(D)
    L, _ = O.tril(A)
    Lex = O.CSR(L.row_ptr, L.col_idx, Lch[np.tril(D != 0)])
    b = np.random.default_rng(0).standard_normal(n)
    x, it, rr, st = O.pcg(A, b, O.PREC_LLT, Lex, rtol=1e-10)
    assert st == 0 and it == 1
    assert np.allclose(x, np.linalg.solve(D, b), rtol=1e-12)
    # tridiagonal: IC(0) is exact, so one iteration too
    T = 2 * np.eye(30) - np.eye(30, k=1) - np.eye(30, k=-1)
    AT = _csr_from_dense(T)
    LT, _ = O.ic0(AT)
    bt = np.random.default_rng(1).standard_normal(30)
    x, it, rr, st = O.pcg(AT, bt, O.PREC_LLT, LT, rtol=1e-10)
    assert it == 1


def test_pcg_solution_matches_dense_solve():
    A = O.assemble(I.fem2d(20, seed=6))
    b = I.rhs(A.n, 6)
    xs = np.linalg.solve(A.dense(), b)
    L, _ = O.ic0(A)
    for pc, LL in ((O.PREC_NONE, None), (O.PREC_JACOBI, None), (O.PREC_LLT, L)):
        x, it, rr, st = O.pcg(A, b, pc, LL, rtol=1e-12)
        assert st == 0 and rr <= 1e-12
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-10
        # the recursive residual matches the true one
        assert np.linalg.norm(b - A.dense() @ x) / np.linalg.norm(b) < 1e-11


def test_jacobi_on_constant_diagonal_equals_cg():
    A = O.assemble(I.poisson2d_32())
    b = I.rhs(A.n, 0)
    x0, it0, rr0, _ = O.pcg(A, b, O.PREC_NONE, rtol=1e-8)
    x1, it1, rr1, _ = O.pcg(A, b, O.PREC_JACOBI, rtol=1e-8)
    assert it0 == it1
    assert np.allclose(x0, x1, rtol=1e-12, atol=1e-12)


def test_ic0_beats_jacobi_beats_nothing_on_poisson():
    # the ordering of the paper's Table 1 iteration counts (IC < Jacobi)
    A = O.assemble(I.poisson2d_32())
    b = I.rhs(A.n, 0)
    L, _ = O.ic0(A)
    it_ic = O.pcg(A, b, O.PREC_LLT, L, rtol=1e-8)[1]
    it_cg = O.pcg(A, b, O.PREC_NONE, rtol=1e-8)[1]
    assert it_ic < it_cg


def test_pcg_edge_cases():
    A = O.assemble(I.fd2d(6, 5))
    x, it, rr, st = O.pcg(A, np.zeros(A.n), O.PREC_NONE)
    assert it == 0 and st == 0 and np.all(x == 0)
    b = I.rhs(A.n, 2)
    x, it, rr, st = O.pcg(A, b, O.PREC_NONE, rtol=1e-12, max_iter=3)
    assert st == 1 and it == 3
    # initial guess = solution: nothing to do
    xs = np.linalg.solve(A.dense(), b)
    x, it, rr, st = O.pcg(A, b, O.PREC_NONE, rtol=1e-6, x0=xs)
    assert it == 0
    # Algorithm 1's first update happens before the loop test: one iteration
    # is counted even when it alone converges (exact factor case above)


def test_iteration_counts_match_dense_reference_recurrence():
    # a dense-matrix PCG written with explicit inverses, checked iteration by
    # iteration: iterates of Algorithm 1 are uniquely determined
    A = O.assemble(I.fem2d(9, seed=12))
    D = A.dense()
    b = I.rhs(A.n, 12)
    L, _ = O.ic0(A)
    Pinv = np.linalg.inv(L.dense() @ L.dense().T)
    for kmax in (1, 2, 5, 9):
        x, it, rr, st = O.pcg(A, b, O.PREC_LLT, L, rtol=0.0, max_iter=kmax)
        xd = np.zeros(A.n)
        r = b.copy()
        z = Pinv @ r
        p = z.copy()
        for k in range(kmax):
            w = D @ p
            al = (r @ z) / (p @ w)
            xd = xd + al * p
            rn = r - al * w
            zn = Pinv @ rn
            be = (rn @ zn) / (r @ z)
            p = zn + be * p
            r, z = rn, zn
        assert it == kmax
        assert np.allclose(x, xd, rtol=1e-9, atol=1e-12)


def _cg_with_order(A, b, rtol, order, L=None, kmax=None):
    """Algorithm 1 (without preconditioner, or with P = L L^T from a dense
    triangular solve), dot products summed in another (equally valid) order;
    used to measure how far rounding alone moves the iteration count (the
    return value), or, with kmax, the iterate x after exactly kmax updates."""
    import scipy.linalg as sl
    D = A.dense()
    n = A.n
    Ld = L.dense() if L is not None else None

    def prec(r):
        if Ld is None:
            return r.copy()
        return sl.solve_triangular(Ld.T, sl.solve_triangular(Ld, r, lower=True), lower=False)

    def dot(u, w):
        if order == "pairwise":
            return float(np.dot(u, w))
        if order == "blocked":
            return float(sum(np.sum(u[k:k + 2048] * w[k:k + 2048]) for k in range(0, n, 2048)))
        s = 0.0
        for i in range(n - 1, -1, -1):
            s += u[i] * w[i]
        return s
    x = np.zeros(n)
    r = b.copy()
    tol = rtol * math.sqrt(dot(b, b))
    z = prec(r)
    p = z.copy()
    rz = dot(r, z)
    k = 0
    while True:
        w = D @ p
        al = rz / dot(p, w)
        x += al * p
        r -= al * w
        k += 1
        if kmax is not None:
            if k == kmax:
                return x
        elif math.sqrt(dot(r, r)) <= tol:
            return k
        z = prec(r)
        rzn = dot(r, z)
        p = z + (rzn / rz) * p
        rz = rzn


def test_cg_iteration_spread_under_summation_order():
    # Unpreconditioned CG on an ill-conditioned FEM system: the iteration
    # count to 1e-8 moves by a few under a different summation order of the
    # same recurrence, so a +-1 bar is below the arithmetic's resolution
    # there; the spread stays within 1 % of the count.
    A = O.assemble(I.fem2d(34, sigma=1.0, seed=5))
    b = I.rhs(A.n, 7)
    _, it, _, _ = O.pcg(A, b, O.PREC_NONE, rtol=1e-8)
    others = [_cg_with_order(A, b, 1e-8, o) for o in ("pairwise", "blocked", "reverse")]
    spread = max(abs(k - it) for k in others)
    assert spread > 1                      # the effect is real
    assert spread <= max(1, math.ceil(0.01 * it))


def test_pcg_iteration_spread_learned_factor():
    # PCG with a network factor that needs hundreds of iterations (a random
    # 2 x 16 network on the 34 x 34 FEM system): other summation orders of the
    # same recurrence move the count by more than one iteration, up to 3 % of
    # it.  This is the resolution of the arithmetic that an iteration-count
    # comparison of learned factors can ask for.
    A = O.assemble(I.fem2d(34, sigma=1.0, seed=5))
    b = I.rhs(A.n, 7)
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=16)
    L = O.gnn_forward(cfg, A, b, I.gnn_weights(cfg, 3))
    _, it, _, st = O.pcg(A, b, O.PREC_LLT, L, rtol=1e-6)
    assert st == 0 and it > 300
    others = [_cg_with_order(A, b, 1e-6, o, L) for o in ("pairwise", "blocked", "reverse")]
    spread = max(abs(k - it) for k in others)
    assert spread > 1
    assert spread <= math.ceil(0.03 * it)
    # the iterates after the same number of updates: the oracle's own x moves
    # by more than 1e-8 (relative) under another summation order, and by less
    # than 1e-6 (with IC(0), 28 iterations, by rounding only)
    xo, _, _, _ = O.pcg(A, b, O.PREC_LLT, L, rtol=1e-6)
    dx = max(np.linalg.norm(_cg_with_order(A, b, 1e-6, o, L, kmax=it) - xo) / np.linalg.norm(xo)
             for o in ("pairwise", "blocked", "reverse"))
    assert 1e-8 < dx <= 1e-6
    Lic, _ = O.ic0(A)
    xi, iti, _, _ = O.pcg(A, b, O.PREC_LLT, Lic, rtol=1e-6)
    dxi = np.linalg.norm(_cg_with_order(A, b, 1e-6, "reverse", Lic, kmax=iti) - xi) / np.linalg.norm(xi)
    assert dxi <= 1e-12


# ------------------------------------------------------------------ symmetric Gauss-Seidel
def test_sgs_tridiagonal_closed_form():
    # tridiag(-1, 2, -1): (D + L)(D^-1)(D + U) = A + L D^-1 U = A + diag(0, 1/2, ..., 1/2)
    n = 8
    D = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    L = O.sgs(_csr_from_dense(D)).dense()
    P = L @ L.T
    assert np.allclose(P, D + np.diag([0.0] + [0.5] * (n - 1)), rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sgs_equals_symmetric_sweep(seed):
    # the L L^T form against the sweep product assembled from A's triangles
    A = _random_spd_sparse(40, 0.15, seed)
    L = O.sgs(_csr_from_dense(A)).dense()
    Dg = np.diag(np.diag(A))
    Lo = np.tril(A, -1)
    P_sweep = (Dg + Lo) @ np.linalg.inv(Dg) @ (Dg + Lo).T
    assert np.allclose(L @ L.T, P_sweep, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("prob", [I.fd2d(9, 7, sigma=1.0, seed=1), I.fem2d(11, sigma=1.0, seed=2),
                                  I.fd3d(5, 4, 4, sigma=1.5, corr_len=0.05, seed=3)])
def test_sgs_spectrum_in_unit_interval(prob):
    # for SPD A, the symmetric Gauss-Seidel (SSOR, omega = 1) preconditioned
    # operator has its eigenvalues in (0, 1]: P - A = L_A D^-1 L_A^T >= 0
    A = O.assemble(prob)
    L = O.sgs(A).dense()
    lam = sla.eigh(A.dense(), L @ L.T, eigvals_only=True)
    assert lam.min() > 0 and lam.max() <= 1 + 1e-10
    # and the largest is 1 exactly when L_A D^-1 L_A^T is singular (n > rank
    # of L_A): here the first row of L_A is empty, so P - A has a zero row
    assert abs(lam.max() - 1.0) <= 1e-10


def test_sgs_pcg_between_jacobi_and_ic0_on_poisson():
    A = O.assemble(I.poisson2d_32())
    b = I.rhs(A.n, 0)
    _, it_j, _, _ = O.pcg(A, b, O.PREC_JACOBI, rtol=1e-8)
    _, it_s, _, st = O.pcg(A, b, O.PREC_LLT, O.sgs(A), rtol=1e-8)
    _, it_i, _, _ = O.pcg(A, b, O.PREC_LLT, O.ic0(A)[0], rtol=1e-8)
    assert st == 0 and it_i < it_s < it_j


def test_threaded_spmv_and_pcg_identical_to_single_thread():
    # the all-cores leg of the oracle's timing runs the independent rows of
    # SpMV and the elementwise PCG updates on several threads; every row and
    # element keeps the single-threaded arithmetic, so results are identical
    A = O.assemble(I.fd3d(18, sigma=1.5, corr_len=0.1, seed=2))
    b = I.rhs(A.n, 3)
    L, _ = O.ic0(A)
    x = np.random.default_rng(1).standard_normal(A.n)
    try:
        assert O.set_threads(1) == 1
        y1 = O.spmv(A, x)
        x1, it1, r1, s1 = O.pcg(A, b, O.PREC_LLT, L, rtol=1e-10)
        k = O.set_threads(4)
        y4 = O.spmv(A, x)
        x4, it4, r4, s4 = O.pcg(A, b, O.PREC_LLT, L, rtol=1e-10)
    finally:
        O.set_threads(1)
    assert k in (1, 4)
    assert np.array_equal(y1, y4) and np.array_equal(x1, x4) and (it1, r1, s1) == (it4, r4, s4)
