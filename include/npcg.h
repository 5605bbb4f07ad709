/*
 * npcg.h -- C ABI of the GB300 learned-preconditioner PCG library
 * (Li, Chen, Du, Matusik, "Learning Preconditioners for Conjugate Gradient
 * PDE Solvers", ICML 2023).
 *
 * The library solves A x = b for sparse SPD A from a discretised linear
 * second-order PDE (Sec. 3, "Discretization") with PCG (Algorithm 1) and the
 * preconditioner P = L L^T, where L lives on the lower-triangular pattern of
 * A and is written by a graph network over the sparsity graph of A
 * (Sec. 4.1-4.2, App. A.3).  IC(0), Jacobi and plain CG are the comparison
 * preconditioners (Sec. 5.1, "Baseline Methods").
 *
 * Conventions for every call:
 *   - All array arguments are DEVICE pointers on the handle's device unless
 *     a parameter says "host".  The caller allocates and owns every array
 *     it passes; the library never frees caller memory.  Objects the library
 *     creates (handles, patterns) are freed by their own destroy call.
 *   - Work is enqueued on the handle's stream.  A call returns after
 *     enqueueing unless it returns host data (documented per call), in which
 *     case it synchronises that stream.
 *   - Indices are int32, row-major CSR with strictly ascending columns; the
 *     pattern of A must be structurally symmetric with every diagonal entry
 *     present (a matrix of an undirected mesh graph with self-loops).
 *   - The return code is the only error channel.  On error, npcg_last_error()
 *     gives a one-line description.  Calls never abort the process.
 *   - Device-side waits (on rows, levels or copies that other threads of
 *     the same launch produce: the triangular solves, IC(0), the level
 *     analysis) have an iteration limit (npcg_set_wait_limit); reaching it
 *     returns NPCG_ETIMEOUT and leaves the context usable.
 */
#ifndef NPCG_H
#define NPCG_H

#include <stdint.h>

#if defined(__GNUC__)
#define NPCG_API __attribute__((visibility("default")))
#else
#define NPCG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NPCG_OK = 0,
    NPCG_EINVAL = 1,       /* malformed argument or matrix pattern           */
    NPCG_ENOMEM = 2,       /* device allocation failed                       */
    NPCG_ECUDA = 3,        /* CUDA runtime error                             */
    NPCG_ENOTSPD = 4,      /* IC(0) failed for every shift; L_ii <= 0        */
    NPCG_EBREAKDOWN = 5,   /* PCG: p^T A p <= 0, r^T z <= 0, or non-finite   */
    NPCG_EMAXITER = 6,     /* PCG: max_iter updates without reaching rtol    */
    NPCG_ETIMEOUT = 7,     /* a device spin-wait reached its iteration limit */
    NPCG_ESTALL = 8        /* PCG: ||r|| not below its best for stall_iters
                              updates (npcg_pcg_solve_ex)                   */
} npcg_status;

typedef struct npcg_handle_s* npcg_handle;     /* stream, workspace, error text */
typedef struct npcg_pattern_s* npcg_pattern;   /* analysed sparsity pattern     */

/* --------------------------------------------------------------------------
 * Handle.
 * ------------------------------------------------------------------------ */
/* Creates a handle bound to the current CUDA device and to `stream`
 * (a cudaStream_t; NULL = legacy default stream).  *out is owned by the
 * caller and released with npcg_destroy. */
NPCG_API npcg_status npcg_create(npcg_handle* out, void* stream);
/* Destroys the handle.  Patterns analysed with it should be freed first;
 * any left are detached (calls with them return NPCG_EINVAL) and must
 * still be released with npcg_pattern_free. */
NPCG_API npcg_status npcg_destroy(npcg_handle h);
/* Last error message of the handle (static storage owned by the handle). */
NPCG_API const char* npcg_last_error(npcg_handle h);
/* Polls after which every device wait of later calls on this handle gives
 * up (the sync-free and level-ordered triangular solves, IC(0), the level
 * analysis): the kernel records a timeout, stops, and the call returns
 * NPCG_ETIMEOUT with the context still usable.  polls <= 0 restores the
 * default of 2^22 (about one to two seconds of polling).  A short limit
 * (e.g. 2^10) lets a failure-detection test make a wait run out quickly; a
 * limit too short for a real workload makes its solves time out. */
NPCG_API npcg_status npcg_set_wait_limit(npcg_handle h, int64_t polls);
/* How later PCG calls on this handle launch their iterations (Algorithm 1's
 * loop).  eager = 0: the loop body is a CUDA graph with a device-side while
 * node, launched once per solve.  eager > 0: the same kernels in the same
 * order are enqueued one launch at a time, with the handle's stream
 * synchronised every 16 iterations to test whether any system is still
 * iterating.  eager < 0 (the default): one launch at a time for the
 * triangular-solve preconditioners of a single system solved in row blocks
 * (2^18 rows or more), where it measured faster (on the 128^3 grid, 176
 * IC(0)-PCG iterations with FP32 solves: 175.6 against 180.2 ms), the graph
 * otherwise (on a 256^2 FEM system the graph is faster: 39.3 against 41.1
 * ms for the learned solve).
 * Results are bit-identical in every mode.  Kernel profilers do not see the
 * kernels inside a conditional graph node, so eager > 0 also serves to
 * profile a solve's iterations. */
NPCG_API npcg_status npcg_set_pcg_eager(npcg_handle h, int32_t eager);
NPCG_API const char* npcg_status_string(npcg_status s);

/* --------------------------------------------------------------------------
 * Assembly of A (Sec. 3 "Discretization": Galerkin stiffness matrix of
 * -div(k grad u) = f with homogeneous Dirichlet boundary).  The paper's own
 * meshes are not available; the problems are synthetic stand-ins:
 *   NPCG_FD : 5-point (dim 2) / 7-point (dim 3) finite differences on the
 *             nx x ny (x nz) interior grid of the unit square / cube, natural
 *             order (x fastest); face coefficient = harmonic mean of the
 *             nodal k; h factors dropped.
 *   NPCG_FEM: P1 elements on the Delaunay triangulation of an m x m lattice
 *             (m = nx) on [0,1]^2 with integer jitter (units of 1/1024 of the
 *             spacing); boundary points are eliminated, (m-2)^2 unknowns,
 *             index (a-1) + (m-2)(c-1).  The cell diagonal is chosen by the
 *             exact in-circle predicate (ties: (a,c)-(a+1,c+1)); an edge
 *             whose every cotangent numerator is exactly zero is dropped.
 * log k is a Gaussian random field by random Fourier features:
 *   g(p) = sigma sqrt(2/M) sum_m cos(omega_m . p + phase_m),  k = exp(g),
 * k at the nodes (FD) or k_T = exp(mean of the three nodal g) (FEM).
 * ------------------------------------------------------------------------ */
enum { NPCG_FD = 0, NPCG_FEM = 1 };

typedef struct {
    int32_t kind;             /* NPCG_FD or NPCG_FEM                            */
    int32_t dim;              /* 2 or 3 (FEM: 2)                                */
    int32_t nx, ny, nz;       /* FD: interior grid; FEM: nx = m lattice points  */
    int32_t n_features;       /* M, number of random Fourier features           */
    double sigma;             /* GRF standard deviation (0: k == 1)             */
    const double* omega;      /* device [M * dim] frequencies                   */
    const double* phase;      /* device [M] phases                              */
    const int32_t* jitter;    /* device [m * m * 2] (FEM only; NULL for FD)     */
    /* Implicit time step of the heat / wave equation (Sec. 5.1 environments):
     * tau > 0 assembles A = M + tau K instead of K, M the consistent P1 mass
     * matrix (FEM, M_T[s][t] = area (1 + [s == t]) / 12) or h^2 I (FD, in the
     * units of the h-free stencil, h = 1 / (nx + 1)).  tau = 0: A = K.     */
    double tau;
    /* FEM boundary: dir_len = 0 makes every boundary point Dirichlet; with
     * dir_len > 0 only dir_len consecutive points from perimeter index
     * dir_start are, and the other boundary points are unknowns (natural
     * boundary).  Perimeter index k runs counter-clockwise from (0,0):
     * bottom (k, 0), right (m-1, k-(m-1)), top (m-1-(k-2(m-1)), m-1), left
     * (0, m-1-(k-3(m-1))).  Unknowns are numbered in point order a + m c.
     * FD: both must be 0.                                                   */
    int32_t dir_start, dir_len;
} npcg_problem;

/* Size of the assembled system: *n_out, *nnz_out (host).  Synchronises. */
NPCG_API npcg_status npcg_assemble_count(npcg_handle h, const npcg_problem* p,
                                int64_t* n_out, int64_t* nnz_out);
/* Assembles A into caller arrays row_ptr [n+1], col_idx [nnz], val [nnz]
 * (sizes from npcg_assemble_count). */
NPCG_API npcg_status npcg_assemble_system(npcg_handle h, const npcg_problem* p,
                                 int32_t* row_ptr, int32_t* col_idx, double* val);

/* --------------------------------------------------------------------------
 * Pattern analysis (the sparsity graph of A, Sec. 4.2, and the triangular
 * structure of "Solve P z = r", Algorithm 1): validation, L = tril(A) pattern,
 * mirror edges e_ij <-> e_ji, forward/backward level sets of L y = r and
 * L^T z = y (computed on the device), and the level-ordered layouts used by
 * the solvers.  A pattern may hold nsys independent systems concatenated
 * block-diagonally (row offsets sys_ptr, host [nsys+1], sys_ptr[0] = 0,
 * sys_ptr[nsys] = n; NULL when nsys == 1).  The row_ptr / col_idx arrays are
 * copied; the caller may free them afterwards.  Synchronises.
 * ------------------------------------------------------------------------ */
NPCG_API npcg_status npcg_analyse(npcg_handle h, int64_t n, int64_t nnz, const int32_t* row_ptr,
                         const int32_t* col_idx, int32_t nsys, const int64_t* sys_ptr,
                         npcg_pattern* out);
NPCG_API npcg_status npcg_pattern_free(npcg_pattern p);

/* Triangular-solve designs (all exact, same result up to rounding):
 *   NPCG_TRSV_SYNCFREE: every SM; rows claimed in level order by warps, each
 *     row waits on its dependencies' values (flag-free, bounded waits);
 *   NPCG_TRSV_LEVELSYNC: one CTA per system walks the levels with one
 *     barrier per level, dependencies in a shared-memory window, each level's
 *     data prefetched by TMA bulk copies;
 *   NPCG_TRSV_LEVELFLAG: the same layout and prefetch without the barrier:
 *     each window slot carries its row's position next to the value and a
 *     row polls its dependencies' slots (FP32 solves, NPCG_PREC_LLT32; FP64
 *     solves use NPCG_TRSV_LEVELSYNC).  Available when the window also
 *     covers how far one warp can run ahead of another;
 *   NPCG_TRSV_LEVELSPLIT: the level-synchronous design with the step
 *     bookkeeping on separate warps: operand warps stage step k+1 while
 *     compute warps solve step k (one system per SM).
 * npcg_analyse times the sync-free, level-synchronous and merged-level
 * designs on the pattern and keeps the fastest (the flag and split-role
 * variants measured slower everywhere and are only selected explicitly). */
enum { NPCG_TRSV_AUTO = 0, NPCG_TRSV_SYNCFREE = 1, NPCG_TRSV_LEVELSYNC = 2, NPCG_TRSV_LEVELFLAG = 3,
       NPCG_TRSV_LEVELSPLIT = 4,
       /* the level-synchronous design over groups of G consecutive levels:
        * substituting the dependencies inside a group gives
        *   y_i = sum_a C_ia r_a - sum_b M_ib y_b
        * (a in the row's group, b in earlier groups), so one step solves a
        * group; C and M are evaluated from each loaded factor.  Single
        * systems below 2^18 rows and patterns up to 2^22 rows; G = 2, 4 or 8
        * as tuned (4 when set before tuning found one)                    */
       NPCG_TRSV_LEVELMERGE = 5 };

typedef struct {
    int64_t n, nnz, nnz_L;
    int32_t nsys;
    int32_t nlev_fwd, nlev_bwd;   /* number of levels of L y = r / L^T z = y */
    int32_t trsv_mode;            /* design in use (NPCG_TRSV_SYNCFREE / _LEVELSYNC / _LEVELFLAG) */
    float tuned_ms_syncfree;      /* measured forward + backward FP32 solve, ms */
    float tuned_ms_levelsync;     /* (0 when the design does not apply)         */
    float tuned_ms_levelflag;
    float tuned_ms_levelsplit;
    int32_t max_row;              /* entries of the longest row of A (rows of at most
                                     16 take the one-thread-per-row SpMV)          */
    float tuned_ms_levelmerge;    /* merged levels at the tuned group size (0: not timed) */
    int32_t merge_levels;         /* levels per step of the built merged layouts (0: none) */
    int32_t block_units;          /* row blocks of one large system's level-ordered layouts
                                     (tuned: one per SM or fewer, thicker ones; 0: not blocked) */
} npcg_pattern_info;
NPCG_API npcg_status npcg_pattern_get_info(npcg_pattern p, npcg_pattern_info* out);  /* host out */
/* Overrides the tuned design (NPCG_TRSV_AUTO restores the tuned choice).
 * NPCG_TRSV_LEVELSYNC / _LEVELFLAG / _LEVELSPLIT return NPCG_EINVAL when the
 * layout does not fit (for _LEVELFLAG: its window does not cover the drift;
 * for _LEVELSPLIT: no ring of two stages fits beside the staging slots). */
NPCG_API npcg_status npcg_pattern_set_trsv(npcg_pattern p, int32_t mode);

/* Copies of the analysis results (device arrays, caller-allocated):
 * L_row_ptr [n+1], L_col_idx [nnz_L] (tril(A), diagonal last in each row),
 * lev_fwd / lev_bwd [n] (level of each row), perm_fwd / perm_bwd [n] (rows in
 * processing order: by level, ascending row within a level).  Any pointer
 * may be NULL. */
NPCG_API npcg_status npcg_pattern_export(npcg_handle h, npcg_pattern p, int32_t* L_row_ptr,
                                int32_t* L_col_idx, int32_t* lev_fwd, int32_t* lev_bwd,
                                int32_t* perm_fwd, int32_t* perm_bwd);

/* --------------------------------------------------------------------------
 * Graph-network factor (Sec. 4.2 "Architecture", App. A.3).
 *   MLP of depth d: Linear(in,h) ReLU [Linear(h,h) ReLU] x (d-1) Linear(h,out)
 *   node input b_i / ||b||_inf, edge input A_ij / s with s = max_i A_ii
 *   (per system), encoders of depth l to width h;
 *   n_mp times:  v_i <- MLP_v([v_i || sum_j e_ij (.) v_j])   (j over row i)
 *                e_ij <- MLP_e([e_ij || v_i || v_j])          (new v)
 *   decoder of depth l: s_ij = MLP_dec(e_ij);
 *   L_ij = sqrt(s) (s_ij + s_ji) / 2 for i > j;  L_ii = sqrt(s) softplus(s_ii)
 * Flat FP32 weights: node encoder, edge encoder, n_mp x (node MLP with input
 * 2h, edge MLP with input 3h, both of depth l_mp), decoder (output 1); each
 * Linear stored as W[out][in] row-major followed by bias[out].
 * ------------------------------------------------------------------------ */
enum { NPCG_FP32 = 0, NPCG_BF16 = 1 };
/* Diagonal rule.  NPCG_DIAG_SOFTPLUS: L_ii = sqrt(s) softplus(s_ii) (above).
 * NPCG_DIAG_LDLT_DIAGA (App. A.3): P = L' D L'^T with D = diag(A) and a
 * unit-diagonal L', L'_ij = (s_ij + s_ji)/2; returned as L = L' D^{1/2}, i.e.
 * L_ii = sqrt(A_ii), L_ij = sqrt(A_jj) (s_ij + s_ji)/2 (no sqrt(s) scaling).
 * NPCG_DIAG_LDLT_ROWS: the same L D L^T form with the scaling on the rows,
 * L = D^{1/2} L~ with a unit-diagonal L~_ij = (s_ij + s_ji)/2, i.e.
 * L_ii = sqrt(A_ii), L_ij = sqrt(A_ii) (s_ij + s_ji)/2, so that L~ factors
 * the Jacobi-scaled matrix D^{-1/2} A D^{-1/2}; the edge input is then that
 * matrix's entry A_ij / sqrt(A_ii A_jj) instead of A_ij / s.  (The network's
 * L~_ij is symmetric in the ends of the edge; scaling the rows lets it
 * express SSOR, L~ = omega times the scaled strict lower triangle, on
 * matrices whose diagonal varies.) */
enum { NPCG_DIAG_SOFTPLUS = 0, NPCG_DIAG_LDLT_DIAGA = 1, NPCG_DIAG_LDLT_ROWS = 2 };

typedef struct {
    int32_t n_mp;        /* message-passing layers                       */
    int32_t l;           /* depth of encoders and decoder                */
    int32_t l_mp;        /* depth of the node / edge update MLPs         */
    int32_t h;           /* hidden = latent width: 16, 32 or 64          */
    int32_t diag_mode;   /* NPCG_DIAG_SOFTPLUS or NPCG_DIAG_LDLT_DIAGA    */
    int32_t precision;   /* NPCG_FP32 (parity) or NPCG_BF16 (tensor cores)*/
    int32_t x0_head;     /* 1: the weights end with the initial-guess head
                            (an MLP of depth l, h -> 1, on the final node
                            features; Sec. 4.4 surrogate use), else 0     */
    int32_t loss;        /* training loss of npcg_loss_and_grad:
                            NPCG_LOSS_AB (Eq. loss_Ab, the method's) or
                            NPCG_LOSS_FROB (Eq. loss_A, the Frobenius
                            ablation); ignored by the forward calls        */
} npcg_gnn_config;
enum { NPCG_LOSS_AB = 0, NPCG_LOSS_FROB = 1 };

/* Number of FP32 parameters of the flat weight vector (host out). */
NPCG_API npcg_status npcg_gnn_nparams(const npcg_gnn_config* cfg, int64_t* out);
/* L values on the tril(A) pattern (order of npcg_pattern_export's L arrays),
 * FP64 [nnz_L].  A_val [nnz], b [n], weights [nparams]. */
NPCG_API npcg_status npcg_gnn_factor(npcg_handle h, npcg_pattern p, const double* A_val,
                            const double* b, const npcg_gnn_config* cfg,
                            const float* weights, double* L_val);
/* Factor and initial guess from one network pass (cfg->x0_head must be 1):
 * L_val as npcg_gnn_factor; x0 [n] (device, FP64) receives
 * x0_i = (||b||_inf / s) MLP_x(v_i) with s the largest diagonal of A and
 * ||b||_inf of the row's system (the head's output scale), to be passed to
 * npcg_pcg_solve as the starting iterate.  Both outputs are caller-owned
 * device buffers.  NPCG_EINVAL for a NULL argument or cfg->x0_head != 1;
 * otherwise the statuses of npcg_gnn_factor. */
NPCG_API npcg_status npcg_gnn_factor_x0(npcg_handle h, npcg_pattern p, const double* A_val, const double* b,
                                        const npcg_gnn_config* cfg, const float* weights, double* L_val,
                                        double* x0);

/* --------------------------------------------------------------------------
 * IC(0) (Sec. 5.1 baseline "IC"), textbook row-oriented form on tril(A):
 *   L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj,  L_ii = sqrt(A_ii - sum L_ik^2).
 * On a non-positive pivot a system is refactored from A + alpha diag(A),
 * alpha = 1e-3 * 2^t, t = 0..30.  alpha_out (host [nsys], may be NULL)
 * receives the shift used per system (0: none).  Synchronises.
 * ------------------------------------------------------------------------ */
NPCG_API npcg_status npcg_ic0_factor(npcg_handle h, npcg_pattern p, const double* A_val,
                            double* L_val, double* alpha_out);

/* --------------------------------------------------------------------------
 * Symmetric Gauss-Seidel (Sec. 5.1 baseline "Gauss-Seidel"; printed as
 * P = L + U, which is not SPD, and read as the symmetric sweep
 *   P = (D + L_A) D^-1 (D + L_A)^T,  L_A the strict lower triangle of A).
 * Writes L = (D + L_A) D^{-1/2} on the tril(A) pattern, so that P = L L^T:
 *   L_ii = sqrt(A_ii),  L_ij = A_ij / sqrt(A_jj)  (j < i),
 * FP64 [nnz_L] in the order of npcg_pattern_export's L arrays, for
 * npcg_pcg_solve with NPCG_PREC_LLT / _LLT32.  A_val [nnz] device, L_val
 * caller-owned device buffer.  NPCG_EINVAL for a NULL argument; A must have
 * a positive diagonal (not checked: a non-positive one gives NaN entries and
 * PCG then reports NPCG_EBREAKDOWN).  Asynchronous on the handle's stream.
 * ------------------------------------------------------------------------ */
NPCG_API npcg_status npcg_sgs_factor(npcg_handle h, npcg_pattern p, const double* A_val, double* L_val);

/* --------------------------------------------------------------------------
 * Preconditioned conjugate gradient, Algorithm 1, in FP64.
 * Stops when ||r_k||_2 <= rtol ||b||_2 (per system).  iters counts the
 * updates of x (Algorithm 1's k).  x holds x_0 on entry, the solution on
 * exit.  precond: NPCG_PREC_NONE (plain CG), NPCG_PREC_JACOBI (P = diag A),
 * NPCG_PREC_LLT (P = L L^T with L_val [nnz_L] on tril(A), FP64).
 * The iteration runs as a CUDA graph with a device-side while loop; the
 * call synchronises once at the end to return the stats (host [nsys]).
 * Returns NPCG_OK if every system converged, else the first failing
 * system's status (per-system codes are in stats).
 * ------------------------------------------------------------------------ */
enum { NPCG_PREC_NONE = 0, NPCG_PREC_JACOBI = 1, NPCG_PREC_LLT = 2, NPCG_PREC_LLT32 = 3 };
/* NPCG_PREC_LLT32: P = L' L'^T with L' = L rounded to FP32 and the two
 * triangular solves in FP32 arithmetic (right-hand side and result FP64);
 * the PCG recurrences, dot products and SpMV stay FP64. */

typedef struct {
    int32_t iters;       /* updates of x (both runs after a fallback)     */
    int32_t status;      /* npcg_status of this system                    */
    double relres;       /* ||r_k|| / ||b|| (recursive residual)          */
    int32_t fallback;    /* 1: the factored solve failed and IC(0) took
                            over (npcg_pcg_solve_ex, npcg_solve_host)     */
    int32_t fallback_iters; /* updates made with the IC(0) factor         */
} npcg_solve_stats;

NPCG_API npcg_status npcg_pcg_solve(npcg_handle h, npcg_pattern p, const double* A_val,
                           const double* b, double* x, int32_t precond,
                           const double* L_val, double rtol, int32_t max_iter,
                           npcg_solve_stats* stats);
/* Same recurrence for every system of a multi-system pattern at once, in one
 * graph of persistent-style launches over the concatenated CSR, with
 * per-system alpha, beta and convergence masks.  stats: host [nsys]. */
NPCG_API npcg_status npcg_pcg_solve_batched(npcg_handle h, npcg_pattern p, const double* A_val,
                                   const double* b, double* x, int32_t precond,
                                   const double* L_val, double rtol, int32_t max_iter,
                                   npcg_solve_stats* stats);

/* Options of npcg_pcg_solve_ex. */
typedef struct {
    int32_t stall_iters;   /* > 0: a system whose ||r|| has not fallen below
                              its smallest value so far for this many
                              consecutive updates stops with NPCG_ESTALL   */
    int32_t fallback_ic0;  /* != 0 (NPCG_PREC_LLT / _LLT32 only): a system
                              that stops with NPCG_EBREAKDOWN, NPCG_EMAXITER
                              or NPCG_ESTALL is solved again with IC(0)'s
                              factor (Sec. 5.1 baseline, npcg_ic0_factor):
                              from x_0 after a breakdown, otherwise from its
                              last iterate, with a fresh max_iter; stats
                              record the switch (fallback, fallback_iters)  */
} npcg_solve_opts;

/* npcg_pcg_solve / npcg_pcg_solve_batched (any pattern) with options; opts
 * may be NULL (the plain call).  With the fallback, L_val is left as given
 * and the IC(0) factor lives in the pattern's workspace.  Returns the status
 * of the last run (NPCG_OK when every system converged, first or after the
 * fallback).  Synchronises. */
NPCG_API npcg_status npcg_pcg_solve_ex(npcg_handle h, npcg_pattern p, const double* A_val,
                                       const double* b, double* x, int32_t precond,
                                       const double* L_val, double rtol, int32_t max_iter,
                                       const npcg_solve_opts* opts, npcg_solve_stats* stats);

/* --------------------------------------------------------------------------
 * Building blocks of the iteration (Algorithm 1), exposed for tests and
 * bandwidth measurement.  y = A x:
 * ------------------------------------------------------------------------ */
NPCG_API npcg_status npcg_spmv(npcg_handle h, npcg_pattern p, const double* A_val,
                      const double* x, double* y);
/* Loads L_val [nnz_L] into the pattern's level-ordered solve layouts. */
NPCG_API npcg_status npcg_factor_load(npcg_handle h, npcg_pattern p, const double* L_val);
/* With the loaded factor: transpose == 0 solves L y = r, transpose == 1
 * solves L^T y = r (r, y [n], distinct). */
NPCG_API npcg_status npcg_sptrsv(npcg_handle h, npcg_pattern p, int32_t transpose,
                        const double* r, double* y);
/* Failure injection for tests (host-side; nothing faults): the sync-free
 * triangular solve of npcg_sptrsv (NPCG_TRSV_SYNCFREE, whatever design is
 * tuned) with its first `skip` slices of 32 rows (in level order) never
 * claimed.  Those rows are never written, so every row that depends on
 * them waits until the handle's wait limit; the call then returns
 * NPCG_ETIMEOUT (NPCG_OK when nothing depends on them).  skip outside
 * [0, slices] returns NPCG_EINVAL.  y [n] is left partly unwritten.
 * Synchronises. */
NPCG_API npcg_status npcg_sptrsv_unclaimed(npcg_handle h, npcg_pattern p, int32_t transpose, int32_t skip,
                                           const double* r, double* y);
/* Same solve repeated reps times (f32 != 0: FP32 factor and arithmetic, as in
 * NPCG_PREC_LLT32); *ms_per_launch (host) is the mean duration of the
 * triangular-solve kernel alone, from CUDA events recorded on the handle's
 * stream around each launch.  Synchronises. */
NPCG_API npcg_status npcg_sptrsv_timed(npcg_handle h, npcg_pattern p, int32_t transpose, int32_t f32,
                              const double* r, double* y, int32_t reps, double* ms_per_launch);

/* --------------------------------------------------------------------------
 * Training loss Eq. (loss_Ab): loss = mean over pairs and systems of
 * ||L L^T x - b||^2, each pair with its own GNN forward (node input b).
 * X, B: [npairs][n] (row p holds pair p of every system of the pattern).
 * loss_out: host.  grad: device [nparams] FP32, overwritten with d loss /
 * d weights (hand-written adjoint of the loss and of the network).
 * cfg->precision NPCG_FP32: FP32 forward and adjoint.  NPCG_BF16 (h = 64):
 * the forward runs on the BF16 tensor cores with FP32 accumulation and the
 * FP32 adjoint is taken at its node / edge states (mixed-precision
 * training with FP32 master weights).
 * cfg->loss NPCG_LOSS_FROB: the Frobenius loss Eq. (loss_A) instead, mean
 * over pairs and systems of ||L L^T - A||_F^2 with L = f(A, b_p) (X unused;
 * the full matrices, fill-in of L L^T included); d/dL = 4 (L L^T - A) L on
 * the pattern of L, by a product structure built on the first call for the
 * pattern.  With cfg->x0_head the head's regression to x is added (both
 * losses).  Synchronises.
 * ------------------------------------------------------------------------ */
NPCG_API npcg_status npcg_loss_and_grad(npcg_handle h, npcg_pattern p, const double* A_val,
                               int32_t npairs, const double* X, const double* B,
                               const npcg_gnn_config* cfg, const float* weights,
                               double* loss_out, float* grad);

/* Adam step (App. A.4: Adam, lr 1e-3) on FP32 master weights, in place.
 * t is the 1-based step count; m, v are the moment buffers [n]. */
NPCG_API npcg_status npcg_adam_step(npcg_handle h, int64_t n, float* w, const float* g, float* m,
                           float* v, int32_t t, float lr, float beta1, float beta2,
                           float eps);

/* --------------------------------------------------------------------------
 * End to end from HOST buffers (the paper's timed quantity, Sec. 5.1
 * "Evaluation Metrics": precompute + solve).  Copies A_val_host [nnz] and
 * b_host [n] in, builds the preconditioner (method: NPCG_METHOD_GNN with
 * cfg + device weights, NPCG_METHOD_IC0, NPCG_METHOD_JACOBI, NPCG_METHOD_CG,
 * NPCG_METHOD_SGS),
 * runs PCG from x_0 = 0 and copies x out to x_host [n].  f32_apply != 0
 * applies the L L^T preconditioners in FP32 (NPCG_PREC_LLT32).  With
 * NPCG_METHOD_GNN a system whose learned-factor solve breaks down, reaches
 * max_iter or stagnates for 200 updates falls back to IC(0) as in
 * npcg_pcg_solve_ex (stats[s].fallback).  Host buffers should be pinned for
 * asynchronous copies.  stats: host [nsys].  Synchronises.
 * ------------------------------------------------------------------------ */
enum { NPCG_METHOD_GNN = 0, NPCG_METHOD_IC0 = 1, NPCG_METHOD_JACOBI = 2, NPCG_METHOD_CG = 3,
       NPCG_METHOD_SGS = 4 };

NPCG_API npcg_status npcg_solve_host(npcg_handle h, npcg_pattern p, int32_t method,
                            const npcg_gnn_config* cfg, const float* weights,
                            const double* A_val_host, const double* b_host, double* x_host,
                            double rtol, int32_t max_iter, int32_t f32_apply,
                            npcg_solve_stats* stats);

/* --------------------------------------------------------------------------
 * Allocation-free solve (the paper has no counterpart; this serves callers
 * that cannot allocate device memory: code running while another arena or
 * runtime owns the device memory, real-time loops where an allocation's
 * latency or failure is unacceptable).  Plain CG (NPCG_PREC_NONE) or
 * Jacobi-PCG (NPCG_PREC_JACOBI), the recurrence of npcg_pcg_solve, on a raw
 * CSR matrix (row_ptr [n+1], col_idx [nnz], A_val [nnz], b [n], x [n]:
 * device, caller-owned; x holds x_0 on entry).  No handle, no pattern, no
 * cudaMalloc / cudaFree or allocating library call: the working vectors and
 * the solver state live in one fixed device array inside the library,
 * sized for n <= NPCG_NOALLOC_MAX_N (about 10 MB), which every GPU that
 * loads the library keeps until the process exits.  Larger n, other
 * preconditioners or NULL arrays return NPCG_EINVAL before any GPU work;
 * with Jacobi, a row without a nonzero finite diagonal entry returns
 * NPCG_EINVAL after the first pass.  A CUDA error already pending on the
 * calling thread returns NPCG_ECUDA before any launch.
 * The first call on a device looks up that array's device address (and may
 * load the library's device code).  Every call synchronises its stream
 * (every 16 iterations, to test convergence), so it must never be called
 * while that stream is being captured into a CUDA graph.
 * All calls on a device share the array: calls that overlap on the GPU
 * (other streams, other host threads) race and corrupt each other; the
 * array keeps the last call's contents, which each call resets as needed.
 * Work runs on `stream` (a cudaStream_t).  stats: host, one entry.
 * ------------------------------------------------------------------------ */
#define NPCG_NOALLOC_MAX_N 262144

NPCG_API npcg_status npcg_pcg_solve_noalloc(void* stream, int64_t n, int64_t nnz,
                                            const int32_t* row_ptr, const int32_t* col_idx,
                                            const double* A_val, const double* b, double* x,
                                            int32_t precond, double rtol, int32_t max_iter,
                                            npcg_solve_stats* stats);

#ifdef __cplusplus
}
#endif
#endif /* NPCG_H */
