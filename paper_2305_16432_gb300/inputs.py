"""Seeded synthetic inputs shared by the CUDA path and by the tests' oracle.

This module only draws random numbers and states workload shapes; it holds
none of the method's arithmetic (no assembly, no GNN, no solver).  Every
random quantity the method consumes is drawn here and passed to both sides as
an input, so the two sides see the same bytes:

* Gaussian-random-field features for ``log k`` (random Fourier features of a
  squared-exponential covariance: frequencies ``omega ~ N(0, corr_len^-2 I)``,
  phases ``phi ~ U[0, 2 pi)``).  The paper's PDE coefficients come from its
  own simulator (Sec. 5.1, App. A.2); a GRF is the synthetic stand-in.
* integer lattice jitter for the P1 FEM point set (units of 1/1024 of the
  lattice spacing, |jitter| <= 204, i.e. just under 0.2 h; boundary points
  are not jittered).
* right-hand sides ``b ~ N(0, 1)`` (the node input of the GNN, Sec. 4.1).
* for the implicit time-step systems, the position and length of the
  Dirichlet arc on the FEM boundary.
* GNN weights, PyTorch-style ``U(-1/sqrt(fan_in), 1/sqrt(fan_in))`` for W and
  bias, in the flat layout documented in ``include/npcg.h``.

Every generator is ``numpy.random.default_rng(seed)`` (PCG64) with a fixed
stream offset per quantity so that two quantities drawn from one seed do not
share random numbers.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GRF_FEATURES = 1024          # number of random Fourier features M
JITTER_UNITS = 1024          # lattice spacing in integer units
JITTER_MAX = 204             # max |jitter| in integer units (< 0.2 * 1024)

# stream offsets so different quantities drawn from one seed are independent
_S_GRF, _S_JIT, _S_RHS, _S_W, _S_MIX, _S_ARC = 0x1000, 0x2000, 0x3000, 0x4000, 0x5000, 0x6000


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


# --------------------------------------------------------------------------
# problems
# --------------------------------------------------------------------------
FD = 0      # finite-difference 5-point (2-D) / 7-point (3-D) stencil
FEM = 1     # P1 FEM on the Delaunay triangulation of a jittered lattice (2-D)


@dataclasses.dataclass(frozen=True)
class Problem:
    """Shape of one synthetic diffusion system -div(k grad u) = f.

    kind FD:  interior grid nx x ny (x nz when dim == 3), Dirichlet boundary.
    kind FEM: m x m lattice points on the unit square, (m-2)^2 unknowns.
    sigma / corr_len: GRF standard deviation and correlation length of log k
    (sigma == 0 gives k == 1).
    tau > 0: the implicit time-step matrix M + tau K of the heat / wave
    equation instead of K.
    dir_start / dir_len (FEM): with dir_len > 0 only dir_len consecutive
    boundary points from perimeter index dir_start are Dirichlet; the other
    boundary points are unknowns.
    """
    kind: int
    dim: int
    nx: int
    ny: int = 0
    nz: int = 0
    sigma: float = 0.0
    corr_len: float = 0.1
    seed: int = 0
    tau: float = 0.0
    dir_start: int = 0
    dir_len: int = 0

    @property
    def n(self) -> int:
        if self.kind == FEM:
            per = 4 * (self.nx - 1)
            free = per - min(self.dir_len, per) if self.dir_len > 0 else 0
            return (self.nx - 2) ** 2 + free
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)


def fd2d(nx, ny=None, sigma=0.0, corr_len=0.1, seed=0) -> Problem:
    return Problem(FD, 2, nx, ny if ny is not None else nx, 0, sigma, corr_len, seed)


def fd3d(nx, ny=None, nz=None, sigma=0.0, corr_len=0.1, seed=0) -> Problem:
    ny = ny if ny is not None else nx
    nz = nz if nz is not None else nx
    return Problem(FD, 3, nx, ny, nz, sigma, corr_len, seed)


def fem2d(m, sigma=1.0, corr_len=0.1, seed=0) -> Problem:
    return Problem(FEM, 2, m, m, 0, sigma, corr_len, seed)


def grf_features(p: Problem, M: int = GRF_FEATURES):
    """(omega [M, dim], phase [M]) for the GRF of problem ``p`` (float64)."""
    g = _rng(p.seed, _S_GRF)
    omega = g.standard_normal((M, p.dim)) / float(p.corr_len)
    phase = g.uniform(0.0, 2.0 * math.pi, M)
    return np.ascontiguousarray(omega, dtype=np.float64), np.ascontiguousarray(phase, dtype=np.float64)


def fem_jitter(p: Problem) -> np.ndarray:
    """int32 [m*m*2] integer jitter (x, y) per lattice point, point index a + m*c.

    Boundary points (a or c in {0, m-1}) get zero jitter.
    """
    assert p.kind == FEM
    m = p.nx
    g = _rng(p.seed, _S_JIT)
    j = g.integers(-JITTER_MAX, JITTER_MAX + 1, size=(m, m, 2), dtype=np.int64)
    j[0, :, :] = 0
    j[m - 1, :, :] = 0
    j[:, 0, :] = 0
    j[:, m - 1, :] = 0
    # array index [c, a, xy] -> point a + m*c
    return np.ascontiguousarray(j.reshape(-1), dtype=np.int32)


def heat2d(m, seed=0, steps_over_explicit=100.0, sigma=1.0, corr_len=0.1) -> Problem:
    """Implicit time step of the heat equation on the jittered-lattice FEM
    mesh: A = M + tau K with tau = steps_over_explicit * h^2 / 4 (h = 1/(m-1),
    a step that many times the explicit stability limit), and a Dirichlet
    arc whose position and length (1/8 to 1/2 of the boundary) are drawn from
    the seed, as in the paper's varying-boundary heat / wave environments."""
    g = _rng(seed, _S_ARC)
    per = 4 * (m - 1)
    start = int(g.integers(0, per))
    length = int(g.integers(per // 8, per // 2 + 1))
    h = 1.0 / (m - 1)
    return Problem(FEM, 2, m, m, 0, sigma, corr_len, seed, steps_over_explicit * h * h / 4.0, start, length)


def zero_jitter(m: int) -> np.ndarray:
    return np.zeros(m * m * 2, dtype=np.int32)


def rhs(n: int, seed: int, count: int | None = None) -> np.ndarray:
    """b ~ N(0,1) of length n (or [count, n])."""
    g = _rng(seed, _S_RHS)
    shape = (n,) if count is None else (count, n)
    return np.ascontiguousarray(g.standard_normal(shape), dtype=np.float64)


# --------------------------------------------------------------------------
# GNN weights
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class GnnConfig:
    """Encoder-processor-decoder shape (App. A.3).

    n_mp: message-passing layers; l: depth of encoders/decoder; l_mp: depth of
    the processor MLPs; h: hidden width (also the latent width).  An MLP of
    depth l is Linear(in,h) ReLU [Linear(h,h) ReLU] x (l-1) Linear(h,out).
    """
    n_mp: int = 2
    l: int = 2
    l_mp: int = 2
    h: int = 16
    diag_mode: int = 0     # 0: L_ii = softplus(s_ii); 1: L = L' D^1/2; 2: L = D^1/2 L~ (D = diag A)
    x0_head: int = 0       # 1: initial-guess head (node MLP of depth l after the decoder)
    loss: int = 0          # training loss: 0 Eq. (loss_Ab), 1 the Frobenius loss Eq. (loss_A)

    def linears(self):
        """(fan_in, fan_out) of every Linear in flat-layout order."""
        h = self.h

        def mlp(i, o, depth):
            dims = [i] + [h] * depth + [o]
            return [(dims[k], dims[k + 1]) for k in range(len(dims) - 1)]
        out = []
        out += mlp(1, h, self.l)              # node encoder
        out += mlp(1, h, self.l)              # edge encoder
        for _ in range(self.n_mp):
            out += mlp(2 * h, h, self.l_mp)   # node update
            out += mlp(3 * h, h, self.l_mp)   # edge update
        out += mlp(h, 1, self.l)              # decoder
        if self.x0_head:
            out += mlp(h, 1, self.l)          # initial-guess head
        return out

    @property
    def nparams(self) -> int:
        return sum(i * o + o for i, o in self.linears())


def gnn_weights(cfg: GnnConfig, seed: int, scale: float = 1.0) -> np.ndarray:
    """Flat float32 weights: per Linear, W[out][in] row-major then b[out]."""
    g = _rng(seed, _S_W)
    parts = []
    for fan_in, fan_out in cfg.linears():
        bound = scale / math.sqrt(fan_in)
        parts.append(g.uniform(-bound, bound, fan_in * fan_out))
        parts.append(g.uniform(-bound, bound, fan_out))
    return np.ascontiguousarray(np.concatenate(parts), dtype=np.float32)


# --------------------------------------------------------------------------
# workloads (sizes of the paper-shaped synthetic configurations)
# --------------------------------------------------------------------------
def poisson2d_32() -> Problem:
    """32 x 32 interior FD Poisson, k == 1 (n = 1024, nnz = 4992)."""
    return fd2d(32, 32, sigma=0.0, seed=0)


def fem2d_256(seed: int = 0) -> Problem:
    """256 x 256 jittered-lattice P1 FEM, log k GRF sigma 1, corr 0.1 (n = 64516)."""
    return fem2d(256, sigma=1.0, corr_len=0.1, seed=seed)


def fd3d_128(seed: int = 0) -> Problem:
    """128^3 7-point FD, log k GRF sigma 1.5, corr 0.05 (n = 2,097,152)."""
    return fd3d(128, sigma=1.5, corr_len=0.05, seed=seed)


def batched_mix(nsys: int = 256, seed: int = 0, n_lo: int = 4000, n_hi: int = 260000,
                s_lo: int = 16, s_hi: int = 64):
    """Uneven batch: even members 2-D FEM with n ~ U[n_lo, n_hi], odd members
    3-D FD with side ~ U{s_lo..s_hi}; log k GRF sigma 1, corr 0.1."""
    g = _rng(seed, _S_MIX)
    out = []
    for s in range(nsys):
        if s % 2 == 0:
            n = int(g.integers(n_lo, n_hi + 1))
            m = int(round(math.sqrt(n))) + 2
            out.append(fem2d(m, sigma=1.0, corr_len=0.1, seed=seed * 100003 + s))
        else:
            side = int(g.integers(s_lo, s_hi + 1))
            out.append(fd3d(side, sigma=1.0, corr_len=0.1, seed=seed * 100003 + s))
    return out


def training_mix(nsys: int = 32, seed: int = 1000):
    """Training set: half 2-D FEM m = 128 (n = 15876), half 3-D FD 25^3 (n = 15625)."""
    out = []
    for s in range(nsys):
        if s % 2 == 0:
            out.append(fem2d(128, sigma=1.0, corr_len=0.1, seed=seed + s))
        else:
            out.append(fd3d(25, sigma=1.0, corr_len=0.1, seed=seed + s))
    return out
