"""Pins of the oracle's PDE assembly (Sec. 3 "Discretization") against
closed forms, an independent element formula and brute force."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2305_16432_gb300 import inputs as I


def test_poisson2d_32_is_textbook_matrix():
    # 5-point Laplacian on a 32 x 32 interior grid, k == 1: nnz = 5n - 2(nx+ny)
    A = O.assemble(I.poisson2d_32())
    assert A.n == 1024 and A.nnz == 4992
    D = A.dense()
    assert np.all(np.diag(D) == 4.0)
    off = D - np.diag(np.diag(D))
    assert set(np.unique(off)) == {-1.0, 0.0}
    # closed-form spectrum 4 - 2cos(p pi/33) - 2cos(q pi/33)
    th = np.arange(1, 33) * np.pi / 33
    ev = np.sort((4 - 2 * np.cos(th)[:, None] - 2 * np.cos(th)[None, :]).ravel())
    assert np.allclose(np.linalg.eigvalsh(D), ev, atol=1e-12)


def test_poisson3d_closed_form():
    nx, ny, nz = 5, 4, 3
    A = O.assemble(I.fd3d(nx, ny, nz, sigma=0.0))
    n = nx * ny * nz
    assert A.nnz == 7 * n - 2 * (nx * ny + ny * nz + nx * nz)
    D = A.dense()
    ev = np.sort(np.add.outer(np.add.outer(
        2 - 2 * np.cos(np.arange(1, nz + 1) * np.pi / (nz + 1)),
        2 - 2 * np.cos(np.arange(1, ny + 1) * np.pi / (ny + 1))),
        2 - 2 * np.cos(np.arange(1, nx + 1) * np.pi / (nx + 1))).ravel())
    assert np.allclose(np.linalg.eigvalsh(D), ev, atol=1e-12)
    # natural ordering, x fastest: node (1,0,0) is index 1, (0,1,0) is nx
    assert D[0, 1] == -1 and D[0, nx] == -1 and D[0, nx * ny] == -1


@pytest.mark.parametrize("dim", [2, 3])
def test_fd_variable_k_invariants(dim):
    p = I.fd2d(9, 7, sigma=1.0, seed=5) if dim == 2 else I.fd3d(6, 5, 4, sigma=1.0, seed=5)
    A = O.assemble(p)
    D = A.dense()
    assert np.array_equal(D, D.T)
    assert np.all(D - np.diag(np.diag(D)) <= 0)          # M-matrix signs
    rs = D.sum(axis=1)
    assert np.all(rs >= -1e-12)                          # diagonal dominance
    assert np.linalg.eigvalsh(D).min() > 0                # SPD
    # rows whose stencil touches no boundary sum to zero exactly (to rounding)
    nx, ny = p.nx, p.ny
    nz = p.nz if dim == 3 else 1
    for l in range(nz):
        for j in range(ny):
            for i in range(nx):
                a = (l * ny + j) * nx + i
                inner = 0 < i < nx - 1 and 0 < j < ny - 1 and (dim == 2 or 0 < l < nz - 1)
                if inner:
                    assert abs(rs[a]) < 1e-12 * D[a, a]
                else:
                    assert rs[a] > 0


def test_fd_face_coefficient_is_harmonic_mean():
    # two interior nodes: off-diagonal = -2 k_a k_b / (k_a + k_b) with k = exp(g)
    p = I.fd2d(3, 3, sigma=0.8, seed=2)
    om, ph = I.grf_features(p)
    A = O.assemble(p, om, ph)
    pts = np.array([[1 / 4, 1 / 4], [2 / 4, 1 / 4]])
    k = np.exp(O.grf_eval(pts, om, ph, p.sigma))
    assert math.isclose(A.dense()[0, 1], -2 * k[0] * k[1] / (k[0] + k[1]), rel_tol=1e-14)


def test_grf_statistics():
    # squared-exponential covariance: Var g = sigma^2, Cov(g(p), g(p + l e1)) = sigma^2 e^{-1/2}
    sigma, ell = 1.3, 0.1
    pts = np.array([[0.3, 0.4], [0.3 + ell, 0.4], [0.9, 0.9]])
    vals = []
    for s in range(1500):
        om, ph = I.grf_features(I.fd2d(4, sigma=sigma, corr_len=ell, seed=s), M=256)
        vals.append(O.grf_eval(pts, om, ph, sigma))
    v = np.array(vals)
    assert abs(v[:, 0].mean()) < 0.15
    assert abs(v[:, 0].var() / sigma**2 - 1) < 0.12
    c = np.mean(v[:, 0] * v[:, 1]) / sigma**2
    assert abs(c - math.exp(-0.5)) < 0.12
    assert abs(np.mean(v[:, 0] * v[:, 2]) / sigma**2) < 0.12   # far apart: ~0


def _lattice(m, jitter):
    a = np.arange(m)
    X = (a[None, :] * 1024 + jitter.reshape(m, m, 2)[:, :, 0]).astype(np.int64)
    Y = (a[:, None] * 1024 + jitter.reshape(m, m, 2)[:, :, 1]).astype(np.int64)
    return X.reshape(-1), Y.reshape(-1)     # point a + m c


def _triangles(m, diag):
    tris = []
    for c in range(m - 1):
        for a in range(m - 1):
            p00 = a + m * c
            p10, p01, p11 = p00 + 1, p00 + m, p00 + m + 1
            if diag[a + (m - 1) * c] == 0:
                tris += [(p00, p10, p11), (p00, p11, p01)]
            else:
                tris += [(p00, p10, p01), (p10, p11, p01)]
    return tris


def test_fem_triangulation_is_delaunay_bruteforce():
    # empty-circumcircle property checked with exact Python integers over all points
    m = 9
    p = I.fem2d(m, sigma=1.0, seed=11)
    jit = I.fem_jitter(p)
    X, Y = _lattice(m, jit)
    tris = _triangles(m, O.fem_diagonals(m, jit))
    for (i, j, k) in tris:
        # positively oriented
        assert (X[j] - X[i]) * (Y[k] - Y[i]) - (Y[j] - Y[i]) * (X[k] - X[i]) > 0
        for q in range(m * m):
            if q in (i, j, k):
                continue
            rows = []
            for v in (i, j, k):
                dx, dy = int(X[v] - X[q]), int(Y[v] - Y[q])
                rows.append((dx, dy, dx * dx + dy * dy))
            (a1, a2, a3), (b1, b2, b3), (c1, c2, c3) = rows
            det = a1 * (b2 * c3 - b3 * c2) - a2 * (b1 * c3 - b3 * c1) + a3 * (b1 * c2 - b2 * c1)
            assert det <= 0, "a point lies strictly inside a circumcircle"


def _fem_dense_bruteforce(m, jit, g):
    """Independent P1 stiffness: barycentric gradients from a 3x3 solve."""
    X, Y = _lattice(m, jit)
    x, y = X / (1024.0 * (m - 1)), Y / (1024.0 * (m - 1))
    diag = O.fem_diagonals(m, jit)
    N = (m - 2) ** 2
    K = np.zeros((N, N))

    def idx(p):
        a, c = p % m, p // m
        if a in (0, m - 1) or c in (0, m - 1):
            return -1
        return (a - 1) + (m - 2) * (c - 1)
    for t in _triangles(m, diag):
        M = np.array([[x[v], y[v], 1.0] for v in t])
        grads = np.linalg.solve(M, np.eye(3))[:2, :].T      # row s: grad of lambda_s
        area = 0.5 * abs(np.linalg.det(M))
        kT = math.exp(sum(g[v] for v in t) / 3.0)
        for s in range(3):
            for u in range(3):
                a, b = idx(t[s]), idx(t[u])
                if a >= 0 and b >= 0:
                    K[a, b] += kT * area * grads[s] @ grads[u]
    return K


@pytest.mark.parametrize("sigma", [0.0, 1.0])
def test_fem_matches_bruteforce_element_formula(sigma):
    m = 12
    p = I.fem2d(m, sigma=sigma, seed=4)
    jit = I.fem_jitter(p)
    om, ph = I.grf_features(p)
    A = O.assemble(p, om, ph, jit)
    X, Y = _lattice(m, jit)
    pts = np.stack([X / (1024.0 * (m - 1)), Y / (1024.0 * (m - 1))], 1)
    g = O.grf_eval(pts, om, ph, sigma)
    K = _fem_dense_bruteforce(m, jit, g)
    D = A.dense()
    assert np.allclose(D, K, rtol=1e-11, atol=1e-11 * np.abs(K).max())
    # pattern: every stored entry is a mesh edge (or diagonal)
    assert np.array_equal(D, D.T)
    assert np.linalg.eigvalsh(D).min() > 0


def test_fem_zero_jitter_unit_k_is_five_point_stencil():
    # right-triangle mesh, k == 1: P1 stiffness = 5-point stencil; the
    # cot(90 deg) = 0 diagonal edges are not in the pattern
    A = O.assemble(I.fem2d(18, sigma=0.0), jitter=I.zero_jitter(18))
    B = O.assemble(I.fd2d(16, sigma=0.0))
    assert A.nnz == B.nnz
    assert np.array_equal(A.row_ptr, B.row_ptr) and np.array_equal(A.col_idx, B.col_idx)
    assert np.allclose(A.val, B.val, rtol=0, atol=1e-14)


def test_fem_interior_row_sums_vanish():
    # the full Neumann stiffness has zero row sums; rows of points whose
    # neighbours are all interior keep that property after elimination
    m = 14
    p = I.fem2d(m, sigma=1.0, seed=8)
    A = O.assemble(p)
    D = A.dense()
    for c in range(2, m - 2):
        for a in range(2, m - 2):
            i = (a - 1) + (m - 2) * (c - 1)
            assert abs(D[i].sum()) < 1e-12 * D[i, i]


def test_fem_256_size():
    p = I.fem2d_256()
    A = O.assemble(p)
    assert A.n == 64516
    # interior points: 1 + 4 lattice + 2 diagonal neighbours on average
    assert 440_000 < A.nnz < 460_000


# ------------------------------------------------------------------ implicit time-step systems
def _perimeter(m):
    # boundary points counter-clockwise from (0, 0), written out edge by edge
    pts = [(a, 0) for a in range(m - 1)] + [(m - 1, c) for c in range(m - 1)]
    pts += [(a, m - 1) for a in range(m - 1, 0, -1)] + [(0, c) for c in range(m - 1, 0, -1)]
    return [a + m * c for a, c in pts]


def _unknown_ids(m, start, length):
    per = _perimeter(m)
    if length == 0:
        dirich = set(per)
    else:
        dirich = {per[(start + t) % len(per)] for t in range(length)}
    ids, k = {}, 0
    for p in range(m * m):
        if p not in dirich:
            ids[p] = k
            k += 1
    return ids, k


@pytest.mark.parametrize("start,length", [(0, 0), (5, 9), (30, 20), (0, 36), (17, 1)])
def test_fem_dirichlet_arc_numbering(start, length):
    m = 10
    ids, n = _unknown_ids(m, start, length)
    uid, n_o = O.fem_unknowns(m, start, length)
    assert n_o == n
    for p in range(m * m):
        assert uid[p] == ids.get(p, -1)
    assert I.Problem(I.FEM, 2, m, m, 0, 0.0, 0.1, 0, 0.0, start, length).n == n


def _fem_dense_heat(m, jit, g, tau, ids, n):
    """Independent M + tau K: barycentric gradients from a 3x3 solve for K,
    edge-midpoint quadrature (exact for quadratics) for M = int lambda_s lambda_t."""
    X, Y = _lattice(m, jit)
    x, y = X / (1024.0 * (m - 1)), Y / (1024.0 * (m - 1))
    A = np.zeros((n, n))
    for t in _triangles(m, O.fem_diagonals(m, jit)):
        Mt = np.array([[x[v], y[v], 1.0] for v in t])
        grads = np.linalg.solve(Mt, np.eye(3))[:2, :].T
        area = 0.5 * abs(np.linalg.det(Mt))
        kT = math.exp(sum(g[v] for v in t) / 3.0)
        lam_mid = [np.array([0.5 if q != e else 0.0 for q in range(3)]) for e in range(3)]
        for s in range(3):
            for u in range(3):
                a, b = ids.get(t[s], -1), ids.get(t[u], -1)
                if a < 0 or b < 0:
                    continue
                mass = area / 3.0 * sum(lm[s] * lm[u] for lm in lam_mid)
                A[a, b] += tau * kT * area * grads[s] @ grads[u] + mass
    return A


@pytest.mark.parametrize("start,length", [(0, 0), (5, 9), (30, 20)])
def test_heat_fem_matches_bruteforce(start, length):
    m = 10
    p = I.Problem(I.FEM, 2, m, m, 0, 1.0, 0.1, 6, 0.37, start, length)
    jit = I.fem_jitter(p)
    om, ph = I.grf_features(p)
    A = O.assemble(p, om, ph, jit)
    X, Y = _lattice(m, jit)
    g = O.grf_eval(np.stack([X / (1024.0 * (m - 1)), Y / (1024.0 * (m - 1))], 1), om, ph, 1.0)
    ids, n = _unknown_ids(m, start, length)
    B = _fem_dense_heat(m, jit, g, 0.37, ids, n)
    D = A.dense()
    assert A.n == n and np.allclose(D, B, rtol=1e-11, atol=1e-11 * np.abs(B).max())
    # every element pair is stored (the mass entries are positive)
    assert A.nnz == np.count_nonzero(B)
    assert np.array_equal(D, D.T) and np.linalg.eigvalsh(D).min() > 0


def test_heat_fem_uniform_lattice_mass():
    # zero jitter, right triangles of legs h: M_ii = h^2/2 (six incident
    # triangles), M_ij = h^2/12 on every element edge; tau = 0 part is K
    m = 12
    h = 1.0 / (m - 1)
    tau = 1e-3
    P = I.Problem(I.FEM, 2, m, m, 0, 0.0, 0.1, 0, tau)
    A = O.assemble(P, jitter=I.zero_jitter(m)).dense()
    K = O.assemble(I.fem2d(m, sigma=0.0), jitter=I.zero_jitter(m)).dense()
    M = A - tau * K
    mi = m - 2
    for c in range(mi):
        for a in range(mi):
            i = a + mi * c
            assert abs(M[i, i] - h * h / 2) < 1e-15
            for (da, dc) in [(1, 0), (0, 1), (1, 1)]:       # axis edges and the (a,c)-(a+1,c+1) diagonal
                if a + da < mi and c + dc < mi:
                    j = (a + da) + mi * (c + dc)
                    assert abs(M[i, j] - h * h / 12) < 1e-15 and abs(M[j, i] - h * h / 12) < 1e-15
            if a + 1 < mi and c >= 1:                       # the other diagonal is not an edge
                assert M[i, (a + 1) + mi * (c - 1)] == 0.0


def test_heat_fd_lumped_mass():
    p0 = I.fd3d(5, 4, 3, sigma=1.0, seed=2)
    p1 = I.Problem(I.FD, 3, 5, 4, 3, 1.0, 0.1, 2, 0.25)
    K = O.assemble(p0)
    A = O.assemble(p1)
    assert np.array_equal(A.row_ptr, K.row_ptr) and np.array_equal(A.col_idx, K.col_idx)
    expect = 0.25 * K.dense() + np.eye(K.n) / 36.0          # h = 1 / (nx + 1)
    assert np.allclose(A.dense(), expect, rtol=1e-14, atol=1e-15)


def test_stiffness_with_dirichlet_arc():
    # pure stiffness, only an arc Dirichlet: rows of points with no
    # Dirichlet element neighbour keep zero row sums (the Neumann operator
    # annihilates constants); the matrix stays SPD
    m = 12
    p = I.Problem(I.FEM, 2, m, m, 0, 1.0, 0.1, 3, 0.0, 7, 10)
    A = O.assemble(p)
    D = A.dense()
    ids, n = _unknown_ids(m, 7, 10)
    dirich = {q for q in range(m * m) if q not in ids}
    tris = _triangles(m, O.fem_diagonals(m, I.fem_jitter(p)))
    touches = set()
    for t in tris:
        if any(v in dirich for v in t):
            touches.update(t)
    for q, i in ids.items():
        if q not in touches:
            assert abs(D[i].sum()) < 1e-12 * D[i, i]
        else:
            assert D[i].sum() > 0
    assert np.linalg.eigvalsh(D).min() > 0
