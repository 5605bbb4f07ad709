"""Python access to the FP64 CPU oracle (oracle/oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference legs, never by the product package.  It
shares no code with the CUDA path; both sides meet only in the seeded inputs
of ``paper_2305_16432_gb300.inputs``.

Every function takes and returns numpy arrays (int32 indices, float64 values)
and documents the passage of the paper it restates; see oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain C11, no contraction, no -march), with
    OpenMP where the compiler has it (used only by set_threads)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    tmp = _OUT + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    r = subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True)
    if r.returncode != 0:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _OUT)
    return _OUT


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
            i8p = np.ctypeslib.ndpointer(np.int8, flags="C")
            vp = C.c_void_p
            lib.or_grf_eval.argtypes = [C.c_int, C.c_int64, f64p, C.c_int, f64p, f64p, C.c_double, f64p]
            lib.or_assemble_fd.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, f64p, f64p,
                                           C.c_double, C.c_double, vp, vp, vp]
            lib.or_assemble_fd.restype = C.c_int64
            lib.or_assemble_fem.argtypes = [C.c_int, i32p, C.c_int, f64p, f64p, C.c_double, C.c_double,
                                            C.c_int32, C.c_int32, vp, vp, vp]
            lib.or_fem_unknowns.argtypes = [C.c_int, C.c_int32, C.c_int32, i32p]
            lib.or_fem_unknowns.restype = C.c_int32
            lib.or_assemble_fem.restype = C.c_int64
            lib.or_fem_diagonals.argtypes = [C.c_int, i32p, i8p]
            lib.or_spmv.argtypes = [C.c_int32, i32p, i32p, f64p, f64p, f64p]
            lib.or_set_threads.argtypes = [C.c_int]
            lib.or_set_threads.restype = C.c_int
            lib.or_tril.argtypes = [C.c_int32, i32p, i32p, vp, vp, vp, vp, vp]
            lib.or_tril.restype = C.c_int64
            lib.or_levels_lower.argtypes = [C.c_int32, i32p, i32p, i32p]
            lib.or_levels_lower.restype = C.c_int32
            lib.or_levels_upper.argtypes = [C.c_int32, i32p, i32p, i32p]
            lib.or_levels_upper.restype = C.c_int32
            lib.or_level_perm.argtypes = [C.c_int32, i32p, C.c_int32, i32p, i32p]
            lib.or_trsv_lower.argtypes = [C.c_int32, i32p, i32p, f64p, f64p, f64p]
            lib.or_trsv_upper.argtypes = [C.c_int32, i32p, i32p, f64p, f64p, f64p]
            lib.or_ic0.argtypes = [C.c_int32, i32p, i32p, f64p, f64p, C.POINTER(C.c_double)]
            lib.or_ic0.restype = C.c_int
            lib.or_sgs_factor.argtypes = [C.c_int32, i32p, i32p, f64p, f64p]
            lib.or_sgs_factor.restype = None
            lib.or_pcg.argtypes = [C.c_int32, i32p, i32p, f64p, f64p, f64p, C.c_int, vp, vp, vp,
                                   C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]
            lib.or_pcg.restype = C.c_int
            lib.or_gnn_nparams.argtypes = [vp]
            lib.or_gnn_nparams.restype = C.c_int64
            lib.or_gnn_forward.argtypes = [vp, C.c_int32, i32p, i32p, f64p, f64p, f64p, i32p, i32p, f64p, vp]
            lib.or_gnn_forward_scaled.argtypes = [vp, C.c_int32, i32p, i32p, f64p, f64p, f64p, i32p, i32p, f64p,
                                                  f64p]
            lib.or_gnn_x0.argtypes = [vp, C.c_int32, i32p, i32p, f64p, f64p, f64p, i32p, i32p, f64p, f64p]
            lib.or_llt_loss.argtypes = [C.c_int32, i32p, i32p, f64p, C.c_int, f64p, f64p, vp]
            lib.or_llt_loss.restype = C.c_double
            lib.or_frob_loss.argtypes = [C.c_int32, i32p, i32p, f64p, i32p, i32p, f64p, vp]
            lib.or_frob_loss.restype = C.c_double
            lib.or_loss_and_grad.argtypes = [vp, C.c_int32, i32p, i32p, f64p, C.c_int, f64p, f64p, f64p, vp]
            lib.or_loss_and_grad.restype = C.c_double
            lib.or_adam.argtypes = [C.c_int64, f64p, f64p, f64p, f64p, C.c_int, C.c_double, C.c_double,
                                    C.c_double, C.c_double]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class CSR:
    """Plain CSR (int32 row_ptr / col_idx, float64 val), sorted columns."""

    def __init__(self, row_ptr, col_idx, val):
        self.row_ptr, self.col_idx, self.val = _i32(row_ptr), _i32(col_idx), _f64(val)

    @property
    def n(self):
        return len(self.row_ptr) - 1

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def dense(self):
        d = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            d[i, self.col_idx[s:e]] = self.val[s:e]
        return d


# ------------------------------------------------------------------ assembly
def grf_eval(points, omega, phase, sigma):
    """g(p) = sigma sqrt(2/M) sum_m cos(omega_m . p + phi_m) at points [N, dim]."""
    points = _f64(points)
    omega, phase = _f64(omega), _f64(phase)
    g = np.empty(points.shape[0])
    _L().or_grf_eval(points.shape[1], points.shape[0], points.reshape(-1), len(phase),
                     omega.reshape(-1), phase, float(sigma), g)
    return g


def assemble(problem, omega=None, phase=None, jitter=None) -> CSR:
    """Stiffness matrix of -div(k grad u) (Sec. 3 Discretization) for a
    ``paper_2305_16432_gb300.inputs.Problem`` and its random inputs; with
    problem.tau > 0 the implicit time-step matrix M + tau K (FEM: consistent
    mass; FD: h^2 I), with problem.dir_len > 0 only an arc of the FEM
    boundary Dirichlet (see oracle.c)."""
    from paper_2305_16432_gb300 import inputs as I
    if omega is None:
        omega, phase = I.grf_features(problem)
    omega, phase = _f64(omega), _f64(phase)
    M = len(phase)
    lib = _L()
    if problem.kind == I.FD:
        args = (problem.dim, problem.nx, problem.ny, problem.nz, M, omega.reshape(-1), phase,
                float(problem.sigma), float(problem.tau))
        nnz = lib.or_assemble_fd(*args, None, None, None)
        n = problem.n
        rp, ci, v = np.zeros(n + 1, np.int32), np.zeros(nnz, np.int32), np.zeros(nnz)
        lib.or_assemble_fd(*args, _ptr(rp), _ptr(ci), _ptr(v))
    else:
        if jitter is None:
            jitter = I.fem_jitter(problem)
        jitter = _i32(jitter)
        args = (problem.nx, jitter, M, omega.reshape(-1), phase, float(problem.sigma), float(problem.tau),
                int(problem.dir_start), int(problem.dir_len))
        nnz = lib.or_assemble_fem(*args, None, None, None)
        n = problem.n
        rp, ci, v = np.zeros(n + 1, np.int32), np.zeros(nnz, np.int32), np.zeros(nnz)
        lib.or_assemble_fem(*args, _ptr(rp), _ptr(ci), _ptr(v))
    return CSR(rp, ci, v)


def fem_unknowns(m, dir_start=0, dir_len=0):
    """(unknown index of every lattice point, -1 for Dirichlet; n)."""
    uid = np.zeros(m * m, np.int32)
    n = _L().or_fem_unknowns(m, dir_start, dir_len, uid)
    return uid, n


def fem_diagonals(m, jitter):
    d = np.zeros((m - 1) * (m - 1), np.int8)
    _L().or_fem_diagonals(m, _i32(jitter), d)
    return d


def set_threads(k: int) -> int:
    """Host threads for SpMV and the PCG vector updates (1 = the plain
    single-threaded oracle); results are identical for every count.  Returns
    the count in effect (1 when the build has no OpenMP)."""
    return int(_L().or_set_threads(int(k)))


# ------------------------------------------------------------------ sparse
def spmv(A: CSR, x):
    y = np.empty(A.n)
    _L().or_spmv(A.n, A.row_ptr, A.col_idx, A.val, _f64(x), y)
    return y


def tril(A: CSR, with_values=True):
    """(L CSR on tril(A), a2l map [nnz] -> L position or -1)."""
    lib = _L()
    nnzL = lib.or_tril(A.n, A.row_ptr, A.col_idx, None, None, None, None, None)
    Lrp, Lci, Lv = np.zeros(A.n + 1, np.int32), np.zeros(nnzL, np.int32), np.zeros(nnzL)
    a2l = np.zeros(A.nnz, np.int32)
    lib.or_tril(A.n, A.row_ptr, A.col_idx, _ptr(A.val) if with_values else None,
                _ptr(Lrp), _ptr(Lci), _ptr(Lv), _ptr(a2l))
    return CSR(Lrp, Lci, Lv), a2l


def levels(L: CSR):
    """(forward levels, backward levels) of L y = r and L^T z = y."""
    lev = np.zeros(L.n, np.int32)
    levb = np.zeros(L.n, np.int32)
    nf = _L().or_levels_lower(L.n, L.row_ptr, L.col_idx, lev)
    nb = _L().or_levels_upper(L.n, L.row_ptr, L.col_idx, levb)
    return lev, nf, levb, nb


def level_perm(lev, nlev):
    perm = np.zeros(len(lev), np.int32)
    ptr = np.zeros(nlev + 1, np.int32)
    _L().or_level_perm(len(lev), _i32(lev), nlev, perm, ptr)
    return perm, ptr


def trsv_lower(L: CSR, r):
    y = np.empty(L.n)
    _L().or_trsv_lower(L.n, L.row_ptr, L.col_idx, L.val, _f64(r), y)
    return y


def trsv_upper(L: CSR, y):
    z = np.empty(L.n)
    _L().or_trsv_upper(L.n, L.row_ptr, L.col_idx, L.val, _f64(y), z)
    return z


def ic0(A: CSR):
    """IC(0) on tril(A) with the shifted retry; returns (L, alpha)."""
    L, _ = tril(A)
    Lv = np.zeros(L.nnz)
    alpha = C.c_double(0.0)
    rc = _L().or_ic0(L.n, L.row_ptr, L.col_idx, L.val, Lv, C.byref(alpha))
    if rc != 0:
        raise RuntimeError("IC(0) failed for every shift")
    return CSR(L.row_ptr, L.col_idx, Lv), alpha.value


def sgs(A: CSR):
    """Symmetric Gauss-Seidel (Sec. 5.1 baseline, read as the symmetric
    sweep): L = (D + L_A) D^{-1/2} on tril(A), so that L L^T =
    (D + L_A) D^-1 (D + L_A)^T."""
    L, _ = tril(A)
    Lv = np.zeros(L.nnz)
    _L().or_sgs_factor(L.n, L.row_ptr, L.col_idx, L.val, Lv)
    return CSR(L.row_ptr, L.col_idx, Lv)


PREC_NONE, PREC_JACOBI, PREC_LLT = 0, 1, 2


def pcg(A: CSR, b, precond=PREC_NONE, L: CSR | None = None, rtol=1e-8, max_iter=None, x0=None):
    """Algorithm 1.  Returns (x, iters, relres, status)."""
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    it, rr = C.c_int(0), C.c_double(0.0)
    if max_iter is None:
        max_iter = 10 * A.n
    st = _L().or_pcg(A.n, A.row_ptr, A.col_idx, A.val, b, x, precond,
                     _ptr(L.row_ptr) if L is not None else None,
                     _ptr(L.col_idx) if L is not None else None,
                     _ptr(L.val) if L is not None else None,
                     float(rtol), int(max_iter), C.byref(it), C.byref(rr))
    return x, it.value, rr.value, st


# ------------------------------------------------------------------ GNN
class _Cfg(C.Structure):
    _fields_ = [("n_mp", C.c_int), ("l", C.c_int), ("l_mp", C.c_int), ("h", C.c_int), ("diag_mode", C.c_int),
                ("x0_head", C.c_int), ("loss", C.c_int)]


def _cfg(cfg):
    return _Cfg(cfg.n_mp, cfg.l, cfg.l_mp, cfg.h, cfg.diag_mode, int(getattr(cfg, "x0_head", 0)),
                int(getattr(cfg, "loss", 0)))


def gnn_nparams(cfg):
    c = _cfg(cfg)
    return int(_L().or_gnn_nparams(C.byref(c)))


def gnn_forward(cfg, A: CSR, b, w, return_s=False):
    """L on tril(A) from the GNN (Sec. 4.2, App. A.3); FP64."""
    L, _ = tril(A, with_values=False)
    Lv = np.zeros(L.nnz)
    s = np.zeros(A.nnz) if return_s else None
    c = _cfg(cfg)
    _L().or_gnn_forward(C.byref(c), A.n, A.row_ptr, A.col_idx, A.val, _f64(b), _f64(w),
                        L.row_ptr, L.col_idx, Lv, _ptr(s))
    out = CSR(L.row_ptr, L.col_idx, Lv)
    return (out, s) if return_s else out


def gnn_x0(cfg, A: CSR, b, w):
    """Initial guess of the x0 head (Sec. 4.4, cfg.x0_head): x0_i = (||b||_inf / s) MLP_x(v_i)."""
    L, _ = tril(A, with_values=False)
    Lv = np.zeros(L.nnz)
    x0 = np.zeros(A.n)
    c = _cfg(cfg)
    _L().or_gnn_x0(C.byref(c), A.n, A.row_ptr, A.col_idx, A.val, _f64(b), _f64(w), L.row_ptr, L.col_idx, Lv, x0)
    return x0


def gnn_forward_scaled(cfg, A: CSR, b, w, s_max_diag, b_inf):
    """L on tril(A) with the input scales of a parent system given (max
    diagonal s and ||b||_inf); A is then a subgraph cut from that system."""
    L, _ = tril(A, with_values=False)
    Lv = np.zeros(L.nnz)
    c = _cfg(cfg)
    _L().or_gnn_forward_scaled(C.byref(c), A.n, A.row_ptr, A.col_idx, A.val, _f64(b), _f64(w),
                               L.row_ptr, L.col_idx, Lv, np.array([s_max_diag, b_inf], dtype=np.float64))
    return CSR(L.row_ptr, L.col_idx, Lv)


def ball(A: CSR, centres, radius):
    """Sorted node ids within `radius` hops of any centre (breadth-first)."""
    seen = set(int(c) for c in centres)
    front = list(seen)
    for _ in range(radius):
        nxt = []
        for i in front:
            for j in A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]:
                j = int(j)
                if j not in seen:
                    seen.add(j)
                    nxt.append(j)
        front = nxt
    return np.array(sorted(seen), dtype=np.int64)


def induced(A: CSR, nodes):
    """Subgraph of A on sorted `nodes` (relabelled in the same order)."""
    pos = {int(v): k for k, v in enumerate(nodes)}
    rp, ci, val = [0], [], []
    for i in nodes:
        s, e = A.row_ptr[i], A.row_ptr[i + 1]
        for k in range(s, e):
            j = int(A.col_idx[k])
            if j in pos:
                ci.append(pos[j])
                val.append(A.val[k])
        rp.append(len(ci))
    return CSR(rp, ci, val)


def gnn_rows(cfg, A: CSR, b, w, rows):
    """Rows `rows` of the network's L on the full system A, evaluated one
    neighbourhood at a time: a node's state after n_mp rounds depends only on
    nodes within n_mp hops (App. A.3), so the rows at the centre of the
    (n_mp + 1)-hop ball, computed with the full system's input scales, are the
    full system's rows.  Returns {row: (cols, values)}."""
    b = _f64(b)
    rows_of = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    s_max = float(A.val[A.col_idx == rows_of].max())
    b_inf = float(np.max(np.abs(b))) or 1.0
    out = {}
    for r in rows:
        nodes = ball(A, [r], cfg.n_mp + 1)
        S = induced(A, nodes)
        Ls = gnn_forward_scaled(cfg, S, b[nodes], w, s_max, b_inf)
        k = int(np.searchsorted(nodes, r))
        s, e = Ls.row_ptr[k], Ls.row_ptr[k + 1]
        out[int(r)] = (nodes[Ls.col_idx[s:e]], Ls.val[s:e].copy())
    return out


def llt_loss(L: CSR, X, B, with_grad=True):
    """(1/B) sum_p ||L L^T x_p - b_p||^2 and d/dL on the pattern (Eq. loss_Ab)."""
    X, B = np.atleast_2d(_f64(X)), np.atleast_2d(_f64(B))
    dL = np.zeros(L.nnz) if with_grad else None
    loss = _L().or_llt_loss(L.n, L.row_ptr, L.col_idx, L.val, X.shape[0], X.reshape(-1),
                            B.reshape(-1), _ptr(dL))
    return loss, dL


def frob_loss(A: CSR, L: CSR, with_grad=True):
    """||L L^T - A||_F^2 (Eq. loss_A for one L) and d/dL on the pattern of L."""
    dL = np.zeros(L.nnz) if with_grad else None
    loss = _L().or_frob_loss(A.n, A.row_ptr, A.col_idx, A.val, L.row_ptr, L.col_idx, L.val, _ptr(dL))
    return loss, dL


def loss_and_grad(cfg, A: CSR, X, B, w, with_grad=True):
    """Loss through the GNN (Eq. loss_Ab, or Eq. loss_A when cfg.loss == 1)
    and its gradient w.r.t. the weights."""
    X, B = np.atleast_2d(_f64(X)), np.atleast_2d(_f64(B))
    w = _f64(w)
    g = np.zeros(len(w)) if with_grad else None
    c = _cfg(cfg)
    loss = _L().or_loss_and_grad(C.byref(c), A.n, A.row_ptr, A.col_idx, A.val, X.shape[0],
                                 X.reshape(-1), B.reshape(-1), w, _ptr(g))
    return loss, g


def adam(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step (float64 arrays)."""
    _L().or_adam(len(w), w, _f64(g), m, v, int(t), lr, b1, b2, eps)
