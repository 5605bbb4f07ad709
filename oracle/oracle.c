/*
 * oracle.c -- plain, slow, obviously-correct CPU reference of the learned
 * preconditioner hot path, in FP64, single-threaded (an OpenMP build may
 * spread the independent rows of SpMV and the vector updates of PCG over
 * host threads, with identical results: or_set_threads).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs do.  It shares no code, header, table or
 * helper with the CUDA library; the only thing both sides share is the seeded
 * random inputs (paper_2305_16432_gb300/inputs.py), passed in as arrays.
 *
 * What it restates, with the passage each part follows:
 *   - assembly of A for -div(k grad u) = f with Dirichlet boundary, Galerkin
 *     (Sec. 3 "Discretization"); FD 5/7-point and P1 FEM on a Delaunay mesh.
 *     The coefficient field and meshes are synthetic stand-ins.
 *   - the sparsity graph of A (Sec. 4.2: one node per row, one edge per
 *     nonzero) and the lower-triangular pattern tril(A) that L lives on.
 *   - level sets of the triangular solves "Solve P z = r" (Algorithm 1).
 *   - IC(0) (Sec. 5.1 baselines, "Incomplete Cholesky"), textbook form.
 *   - PCG (Algorithm 1), with relative stopping ||r_k|| <= rtol ||b||.
 *   - the GNN (Sec. 4.2 "Architecture", App. A.3): encoders, message
 *     passing, decoder, symmetrisation onto tril(A).
 *   - the loss sum ||L L^T x - b||^2 (Eq. loss_Ab, Sec. 4.3) and its exact
 *     gradient by reverse-mode differentiation through the GNN.
 *   - Adam (App. A.4, lr 1e-3).
 *
 * Parity is pinned by the tests in tests/test_oracle_*.py against dense
 * linear algebra, closed forms, brute force and finite differences.
 * Parity unpinned: nothing here pins the *quality* of a trained network.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads for the row-independent loops of the sparse matrix-vector
 * product and the elementwise vector updates of PCG (OpenMP builds only; the
 * default is one).  Each row or element is computed by exactly the
 * arithmetic of the single-threaded loop, and the dot products, triangular
 * solves and IC(0) stay sequential, so results do not depend on the thread
 * count.  Returns the count in effect. */
static int or_threads = 1;
int or_set_threads(int k) {
#ifdef _OPENMP
    or_threads = k < 1 ? 1 : k;
#else
    (void)k;
    or_threads = 1;
#endif
    return or_threads;
}

/* ======================================================================
 * Gaussian random field for log k: random Fourier features of the squared
 * exponential covariance, g(p) = sigma sqrt(2/M) sum_m cos(omega_m . p + phi_m)
 * ==================================================================== */
void or_grf_eval(int dim, int64_t npts, const double* pts, int M,
                 const double* omega, const double* phase, double sigma, double* g) {
    for (int64_t p = 0; p < npts; ++p) {
        if (sigma == 0.0) { g[p] = 0.0; continue; }
        double s = 0.0;
        for (int m = 0; m < M; ++m) {
            double arg = phase[m];
            for (int d = 0; d < dim; ++d) arg += omega[(int64_t)m * dim + d] * pts[p * dim + d];
            s += cos(arg);
        }
        g[p] = sigma * sqrt(2.0 / (double)M) * s;
    }
}

/* ======================================================================
 * COO builder: entries are merged by (row, col); duplicates summed in the
 * order they were added (ties broken by insertion sequence).
 * ==================================================================== */
typedef struct { int32_t i, j; int64_t seq; double v; int nz_flag; } coo_t;
typedef struct { coo_t* e; int64_t n, cap; } coo_list;

static void coo_add(coo_list* c, int32_t i, int32_t j, double v, int nz_flag) {
    if (c->n == c->cap) {
        c->cap = c->cap ? 2 * c->cap : 1024;
        c->e = (coo_t*)realloc(c->e, (size_t)c->cap * sizeof(coo_t));
    }
    c->e[c->n].i = i; c->e[c->n].j = j; c->e[c->n].v = v;
    c->e[c->n].seq = c->n; c->e[c->n].nz_flag = nz_flag;
    c->n++;
}

static int coo_cmp(const void* a, const void* b) {
    const coo_t* x = (const coo_t*)a; const coo_t* y = (const coo_t*)b;
    if (x->i != y->i) return x->i < y->i ? -1 : 1;
    if (x->j != y->j) return x->j < y->j ? -1 : 1;
    return x->seq < y->seq ? -1 : (x->seq > y->seq);
}

/* Sort + merge.  If drop_flagless, an off-diagonal entry none of whose
 * contributions carried nz_flag is removed.  Writes CSR if row_ptr != NULL;
 * returns nnz. */
static int64_t coo_to_csr(coo_list* c, int32_t n, int drop_flagless,
                          int32_t* row_ptr, int32_t* col_idx, double* val) {
    qsort(c->e, (size_t)c->n, sizeof(coo_t), coo_cmp);
    int64_t nnz = 0;
    if (row_ptr) for (int32_t r = 0; r <= n; ++r) row_ptr[r] = 0;
    int64_t k = 0;
    while (k < c->n) {
        int32_t i = c->e[k].i, j = c->e[k].j;
        double v = 0.0; int flag = 0;
        while (k < c->n && c->e[k].i == i && c->e[k].j == j) { v += c->e[k].v; flag |= c->e[k].nz_flag; ++k; }
        if (drop_flagless && i != j && !flag) continue;
        if (row_ptr) { col_idx[nnz] = j; val[nnz] = v; row_ptr[i + 1]++; }
        ++nnz;
    }
    if (row_ptr) for (int32_t r = 0; r < n; ++r) row_ptr[r + 1] += row_ptr[r];
    return nnz;
}

/* ======================================================================
 * FD assembly (Sec. 3, "Discretization"; grid stand-in for the paper's
 * meshes).  Interior unknowns of an nx x ny (x nz) grid on the unit square /
 * cube, natural order (x fastest).  Face coefficient between nodes a, b is
 * the harmonic mean 2 k_a k_b / (k_a + k_b); a face to a Dirichlet boundary
 * node adds to the diagonal only.  h factors dropped.  k = exp(g).
 * ==================================================================== */
static double fd_coord(int i, int nx) { return (double)(i + 1) / (double)(nx + 1); }

static double fd_k(int dim, int i, int j, int l, int nx, int ny, int nz,
                   int M, const double* omega, const double* phase, double sigma) {
    double p[3] = { fd_coord(i, nx), fd_coord(j, ny), dim == 3 ? fd_coord(l, nz) : 0.0 };
    double g;
    or_grf_eval(dim, 1, p, M, omega, phase, sigma, &g);
    return exp(g);
}

int64_t or_assemble_fd(int dim, int nx, int ny, int nz, int M, const double* omega,
                       const double* phase, double sigma, double tau,
                       int32_t* row_ptr, int32_t* col_idx, double* val) {
    /* tau > 0: implicit time step A = h^2 I + tau K (lumped mass in the units
     * of the h-free stencil, h = 1 / (nx + 1)) */
    const double ks = tau > 0.0 ? tau : 1.0;
    if (dim == 2) nz = 1;
    int32_t n = nx * ny * nz;
    /* k at every grid point including the boundary layer: index (i+1,j+1,l+1) */
    int ex = nx + 2, ey = ny + 2, ez = (dim == 3) ? nz + 2 : 1;
    double* kk = (double*)malloc(sizeof(double) * (size_t)ex * ey * ez);
    for (int l = 0; l < ez; ++l)
        for (int j = 0; j < ey; ++j)
            for (int i = 0; i < ex; ++i)
                kk[((int64_t)l * ey + j) * ex + i] =
                    fd_k(dim, i - 1, j - 1, dim == 3 ? l - 1 : 0, nx, ny, nz, M, omega, phase, sigma);
    coo_list c = {0};
    int nd = 2 * dim;
    int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dl[6] = {0, 0, 0, 0, -1, 1};
    for (int l = 0; l < nz; ++l)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int32_t a = (int32_t)(((int64_t)l * ny + j) * nx + i);
                int la = (dim == 3) ? l + 1 : 0;
                double ka = kk[((int64_t)la * ey + (j + 1)) * ex + (i + 1)];
                for (int d = 0; d < nd; ++d) {
                    int i2 = i + di[d], j2 = j + dj[d], l2 = l + dl[d];
                    int lb = (dim == 3) ? l2 + 1 : 0;
                    double kb = kk[((int64_t)lb * ey + (j2 + 1)) * ex + (i2 + 1)];
                    double kf = 2.0 * ka * kb / (ka + kb);
                    coo_add(&c, a, a, ks * kf, 1);
                    int interior = i2 >= 0 && i2 < nx && j2 >= 0 && j2 < ny && l2 >= 0 && l2 < nz;
                    if (interior) {
                        int32_t b = (int32_t)(((int64_t)l2 * ny + j2) * nx + i2);
                        coo_add(&c, a, b, -ks * kf, 1);
                    }
                }
                if (tau > 0.0) {
                    const double h = 1.0 / (double)(nx + 1);
                    coo_add(&c, a, a, h * h, 1);
                }
            }
    int64_t nnz = coo_to_csr(&c, n, 0, row_ptr, col_idx, val);
    free(c.e); free(kk);
    return nnz;
}

/* ======================================================================
 * P1 FEM assembly (Sec. 3 "Discretization", Galerkin).  Points: m x m
 * lattice on [0,1]^2 in integer units X = a*1024 + jx, Y = c*1024 + jy,
 * coordinates X / (1024 (m-1)).  Each lattice cell is split by the diagonal
 * that passes the in-circle test (exact in int64); a tie takes the
 * (a,c)-(a+1,c+1) diagonal.  Dirichlet points are eliminated: the whole
 * boundary (dir_len = 0), or an arc of dir_len consecutive boundary points
 * starting at perimeter index dir_start, the other boundary points being
 * unknowns (natural boundary).  Perimeter index k walks the boundary
 * counter-clockwise from (0,0): bottom (k, 0), right (m-1, k-(m-1)), top
 * (m-1-(k-2(m-1)), m-1), left (0, m-1-(k-3(m-1))).  Unknowns are numbered
 * in point order a + m c; with the whole boundary Dirichlet the index of
 * (a,c) is (a-1) + (m-2)(c-1).
 * tau > 0 (implicit time step of the heat / wave equation, Sec. 5.1
 * environments): A = M + tau K with the consistent P1 mass matrix
 * M_T[s][t] = area (1 + [s == t]) / 12; every vertex pair of an element is
 * then part of the pattern.
 * Element matrix K_T[s][t] = k_T (e_s . e_t) / (4 area), e_s the edge
 * opposite vertex s; k_T = exp(mean of the nodal g).  An off-diagonal entry
 * whose every contribution has an exactly-zero integer dot e_s . e_t is not
 * part of the pattern.
 * ==================================================================== */
static int64_t incircle_i64(const int64_t* a, const int64_t* b, const int64_t* c, const int64_t* d) {
    int64_t adx = a[0] - d[0], ady = a[1] - d[1];
    int64_t bdx = b[0] - d[0], bdy = b[1] - d[1];
    int64_t cdx = c[0] - d[0], cdy = c[1] - d[1];
    int64_t alift = adx * adx + ady * ady;
    int64_t blift = bdx * bdx + bdy * bdy;
    int64_t clift = cdx * cdx + cdy * cdy;
    /* 3x3 determinant by cofactor expansion along the lift column */
    return alift * (bdx * cdy - cdx * bdy)
         - blift * (adx * cdy - cdx * ady)
         + clift * (adx * bdy - bdx * ady);
}

/* diag[cell a + (m-1) c] = 0 for the (a,c)-(a+1,c+1) diagonal, 1 for (a+1,c)-(a,c+1) */
void or_fem_diagonals(int m, const int32_t* jitter, int8_t* diag) {
    for (int c = 0; c < m - 1; ++c)
        for (int a = 0; a < m - 1; ++a) {
            int64_t P[4][2];
            int pa[4] = {a, a + 1, a + 1, a}, pc[4] = {c, c, c + 1, c + 1};   /* p00 p10 p11 p01 */
            for (int q = 0; q < 4; ++q) {
                int64_t id = (int64_t)pa[q] + (int64_t)m * pc[q];
                P[q][0] = (int64_t)pa[q] * 1024 + jitter[2 * id + 0];
                P[q][1] = (int64_t)pc[q] * 1024 + jitter[2 * id + 1];
            }
            int64_t ic = incircle_i64(P[0], P[1], P[2], P[3]);
            diag[a + (int64_t)(m - 1) * c] = ic > 0 ? 1 : 0;
        }
}

/* point id a + m c of perimeter index k */
static int64_t perimeter_point(int m, int64_t k) {
    const int64_t e = m - 1;
    if (k < e) return k;
    if (k < 2 * e) return (m - 1) + (int64_t)m * (k - e);
    if (k < 3 * e) return (m - 1 - (k - 2 * e)) + (int64_t)m * (m - 1);
    return (int64_t)m * (m - 1 - (k - 3 * e));
}

/* unknown index of every lattice point (-1: Dirichlet); returns n */
int32_t or_fem_unknowns(int m, int32_t dir_start, int32_t dir_len, int32_t* uid) {
    const int64_t np = (int64_t)m * m, per = 4 * (int64_t)(m - 1);
    char* dir = (char*)calloc((size_t)np, 1);
    for (int c = 0; c < m; ++c)
        for (int a = 0; a < m; ++a)
            if (dir_len == 0 && (a == 0 || a == m - 1 || c == 0 || c == m - 1)) dir[a + (int64_t)m * c] = 1;
    for (int64_t t = 0; t < (dir_len > 0 ? dir_len : 0); ++t)
        dir[perimeter_point(m, (dir_start + t) % per)] = 1;
    int32_t n = 0;
    for (int64_t p = 0; p < np; ++p) uid[p] = dir[p] ? -1 : n++;
    free(dir);
    return n;
}

int64_t or_assemble_fem(int m, const int32_t* jitter, int M, const double* omega,
                        const double* phase, double sigma, double tau, int32_t dir_start, int32_t dir_len,
                        int32_t* row_ptr, int32_t* col_idx, double* val) {
    int64_t np = (int64_t)m * m;
    int32_t* uid = (int32_t*)malloc(sizeof(int32_t) * (size_t)np);
    const int32_t n = or_fem_unknowns(m, dir_start, dir_len, uid);
    int64_t* XY = (int64_t*)malloc(sizeof(int64_t) * 2 * np);
    double* pos = (double*)malloc(sizeof(double) * 2 * np);
    double* g = (double*)malloc(sizeof(double) * np);
    double scale = 1024.0 * (double)(m - 1);
    for (int c = 0; c < m; ++c)
        for (int a = 0; a < m; ++a) {
            int64_t id = a + (int64_t)m * c;
            XY[2 * id] = (int64_t)a * 1024 + jitter[2 * id];
            XY[2 * id + 1] = (int64_t)c * 1024 + jitter[2 * id + 1];
            pos[2 * id] = (double)XY[2 * id] / scale;
            pos[2 * id + 1] = (double)XY[2 * id + 1] / scale;
        }
    or_grf_eval(2, np, pos, M, omega, phase, sigma, g);
    int8_t* dg = (int8_t*)malloc((size_t)(m - 1) * (m - 1));
    or_fem_diagonals(m, jitter, dg);
    coo_list cl = {0};
    for (int c = 0; c < m - 1; ++c)
        for (int a = 0; a < m - 1; ++a) {
            int64_t p00 = a + (int64_t)m * c, p10 = p00 + 1, p01 = p00 + m, p11 = p01 + 1;
            int64_t tri[2][3];
            if (dg[a + (int64_t)(m - 1) * c] == 0) {
                tri[0][0] = p00; tri[0][1] = p10; tri[0][2] = p11;
                tri[1][0] = p00; tri[1][1] = p11; tri[1][2] = p01;
            } else {
                tri[0][0] = p00; tri[0][1] = p10; tri[0][2] = p01;
                tri[1][0] = p10; tri[1][1] = p11; tri[1][2] = p01;
            }
            for (int t = 0; t < 2; ++t) {
                double e[3][2]; int64_t ei[3][2];
                for (int s = 0; s < 3; ++s) {
                    int64_t q1 = tri[t][(s + 1) % 3], q2 = tri[t][(s + 2) % 3];
                    e[s][0] = pos[2 * q2] - pos[2 * q1];
                    e[s][1] = pos[2 * q2 + 1] - pos[2 * q1 + 1];
                    ei[s][0] = XY[2 * q2] - XY[2 * q1];
                    ei[s][1] = XY[2 * q2 + 1] - XY[2 * q1 + 1];
                }
                /* area from the cross product of two edges (positive for CCW) */
                double area = 0.5 * (e[2][0] * (-e[1][1]) - e[2][1] * (-e[1][0]));
                double kT = exp((g[tri[t][0]] + g[tri[t][1]] + g[tri[t][2]]) / 3.0);
                for (int s = 0; s < 3; ++s) {
                    int32_t is = uid[tri[t][s]];
                    if (is < 0) continue;
                    for (int u = 0; u < 3; ++u) {
                        int32_t iu = uid[tri[t][u]];
                        if (iu < 0) continue;
                        double dot = e[s][0] * e[u][0] + e[s][1] * e[u][1];
                        int64_t doti = ei[s][0] * ei[u][0] + ei[s][1] * ei[u][1];
                        double kst = kT * dot / (4.0 * area);
                        if (tau > 0.0)
                            coo_add(&cl, is, iu, tau * kst + area * (s == u ? 2.0 : 1.0) / 12.0, 1);
                        else
                            coo_add(&cl, is, iu, kst, doti != 0);
                    }
                }
            }
        }
    int64_t nnz = coo_to_csr(&cl, n, 1, row_ptr, col_idx, val);
    free(cl.e); free(XY); free(pos); free(g); free(dg); free(uid);
    return nnz;
}

/* ======================================================================
 * Sparse helpers: y = A x, tril(A), level sets.
 * ==================================================================== */
void or_spmv(int32_t n, const int32_t* rp, const int32_t* ci, const double* v,
             const double* x, double* y) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_threads > 1)
#endif
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
        y[i] = s;
    }
}

/* L pattern = {(i,j) in pattern(A) : j <= i} (Sec. 4.2: L on the
 * lower-triangular indices of A).  Returns nnz_L; fills if Lrp != NULL.
 * a2l[k] (optional) = position in L of A's entry k, or -1. */
int64_t or_tril(int32_t n, const int32_t* rp, const int32_t* ci, const double* v,
                int32_t* Lrp, int32_t* Lci, double* Lv, int32_t* a2l) {
    int64_t nnz = 0;
    if (Lrp) Lrp[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            if (ci[k] <= i) {
                if (Lrp) { Lci[nnz] = ci[k]; if (Lv && v) Lv[nnz] = v[k]; }
                if (a2l) a2l[k] = (int32_t)nnz;
                ++nnz;
            } else if (a2l) a2l[k] = -1;
        }
        if (Lrp) Lrp[i + 1] = (int32_t)nnz;
    }
    return nnz;
}

/* Forward levels of L y = r: lev(i) = 0 if row i has no j < i, else
 * 1 + max lev(j).  Backward levels of L^T z = y: levb(j) = 0 if no i > j has
 * L_ij != 0, else 1 + max levb(i).  Returns number of levels. */
int32_t or_levels_lower(int32_t n, const int32_t* Lrp, const int32_t* Lci, int32_t* lev) {
    int32_t nl = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t l = 0;
        for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k)
            if (Lci[k] < i && lev[Lci[k]] + 1 > l) l = lev[Lci[k]] + 1;
        lev[i] = l;
        if (l + 1 > nl) nl = l + 1;
    }
    return n ? nl : 0;
}

int32_t or_levels_upper(int32_t n, const int32_t* Lrp, const int32_t* Lci, int32_t* levb) {
    for (int32_t i = 0; i < n; ++i) levb[i] = 0;
    int32_t nl = 0;
    for (int32_t i = n - 1; i >= 0; --i) {        /* levb[i] is final here */
        if (levb[i] + 1 > nl) nl = levb[i] + 1;
        for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k) {
            int32_t j = Lci[k];
            if (j < i && levb[i] + 1 > levb[j]) levb[j] = levb[i] + 1;
        }
    }
    return nl;
}

/* rows sorted by (level, row): stable counting sort. */
void or_level_perm(int32_t n, const int32_t* lev, int32_t nlev, int32_t* perm, int32_t* level_ptr) {
    for (int32_t l = 0; l <= nlev; ++l) level_ptr[l] = 0;
    for (int32_t i = 0; i < n; ++i) level_ptr[lev[i] + 1]++;
    for (int32_t l = 0; l < nlev; ++l) level_ptr[l + 1] += level_ptr[l];
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nlev + 1));
    memcpy(fill, level_ptr, sizeof(int32_t) * (size_t)(nlev + 1));
    for (int32_t i = 0; i < n; ++i) perm[fill[lev[i]]++] = i;
    free(fill);
}

/* ======================================================================
 * Triangular solves "Solve P z = r" with P = L L^T (Algorithm 1).
 * ==================================================================== */
void or_trsv_lower(int32_t n, const int32_t* Lrp, const int32_t* Lci, const double* Lv,
                   const double* r, double* y) {
    for (int32_t i = 0; i < n; ++i) {
        double s = r[i], d = 0.0;
        for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k) {
            if (Lci[k] < i) s -= Lv[k] * y[Lci[k]];
            else d = Lv[k];
        }
        y[i] = s / d;
    }
}

/* L^T z = y by backward substitution over the rows of L (column sweep). */
void or_trsv_upper(int32_t n, const int32_t* Lrp, const int32_t* Lci, const double* Lv,
                   const double* y, double* z) {
    for (int32_t i = 0; i < n; ++i) z[i] = y[i];
    for (int32_t i = n - 1; i >= 0; --i) {
        double d = 0.0;
        for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k) if (Lci[k] == i) d = Lv[k];
        z[i] = z[i] / d;
        for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k)
            if (Lci[k] < i) z[Lci[k]] -= Lv[k] * z[i];
    }
}

/* ======================================================================
 * IC(0) (Sec. 5.1 baseline "Incomplete Cholesky"): row-oriented, on the
 * pattern of tril(A):
 *   L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj      (j < i)
 *   L_ii = sqrt(A_ii - sum_{k<i} L_ik^2)
 * sums over k in pattern(row i) and pattern(row j).  On a non-positive
 * pivot the factorisation is retried on A + alpha diag(A), alpha =
 * 1e-3 * 2^t, t = 0, 1, ...; *alpha_out reports the shift used (0: none).
 * Returns 0 on success, -1 if no shift up to 2^30 * 1e-3 worked.
 * ==================================================================== */
static int ic0_once(int32_t n, const int32_t* Lrp, const int32_t* Lci, const double* Av,
                    double alpha, double* Lv) {
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t kk = Lrp[i]; kk < Lrp[i + 1]; ++kk) {
            int32_t j = Lci[kk];
            double s = Av[kk];
            if (j == i) s += alpha * Av[kk];
            /* sum over k < j present in both row i and row j of L */
            for (int32_t a = Lrp[i]; a < Lrp[i + 1]; ++a) {
                int32_t k = Lci[a];
                if (k >= j) continue;
                for (int32_t b = Lrp[j]; b < Lrp[j + 1]; ++b)
                    if (Lci[b] == k) { s -= Lv[a] * Lv[b]; break; }
            }
            if (j < i) {
                double d = Lv[Lrp[j + 1] - 1];    /* diagonal is last in row j */
                Lv[kk] = s / d;
            } else {
                if (!(s > 0.0)) return 1;
                Lv[kk] = sqrt(s);
            }
        }
    }
    return 0;
}

int or_ic0(int32_t n, const int32_t* Lrp, const int32_t* Lci, const double* Atril_v,
           double* Lv, double* alpha_out) {
    if (ic0_once(n, Lrp, Lci, Atril_v, 0.0, Lv) == 0) { *alpha_out = 0.0; return 0; }
    for (int t = 0; t <= 30; ++t) {
        double alpha = 1e-3 * ldexp(1.0, t);
        if (ic0_once(n, Lrp, Lci, Atril_v, alpha, Lv) == 0) { *alpha_out = alpha; return 0; }
    }
    return -1;
}

/* ======================================================================
 * Symmetric Gauss-Seidel preconditioner (Sec. 5.1 baseline "Gauss-Seidel",
 * printed as P = L + U, which is not SPD; read as the symmetric sweep)
 *   P = (D + L_A) D^-1 (D + L_A)^T,  L_A the strict lower triangle of A,
 * handed to PCG as P = L L^T with L = (D + L_A) D^{-1/2} on tril(A):
 *   L_ii = sqrt(A_ii),  L_ij = A_ij / sqrt(A_jj)  (j < i).
 * Atril_v: A's values on the tril pattern (diagonal last in each row).
 * ==================================================================== */
void or_sgs_factor(int32_t n, const int32_t* Lrp, const int32_t* Lci, const double* Atril_v, double* Lv) {
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k) {
            const int32_t j = Lci[k];
            const double ajj = Atril_v[Lrp[j + 1] - 1];
            Lv[k] = j == i ? sqrt(ajj) : Atril_v[k] / sqrt(ajj);
        }
}

/* ======================================================================
 * PCG, Algorithm 1.  Stops when ||r_k||_2 <= rtol ||b||_2 (relative form of
 * the printed absolute epsilon).  iters = number of x updates (Algorithm 1's
 * k; its pre-loop update counts as 1).  If ||r_0|| is already below the
 * threshold no update is made (k = 0).
 * precond: 0 none (plain CG), 1 Jacobi P = diag(A), 2 P = L L^T.
 * Returns 0 converged, 1 max_iter reached, 2 breakdown (p^T A p <= 0,
 * r^T z <= 0 or non-finite).
 * ==================================================================== */
static double dot(int32_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static void apply_prec(int precond, int32_t n, const int32_t* rp, const int32_t* ci, const double* v,
                       const int32_t* Lrp, const int32_t* Lci, const double* Lv,
                       const double* r, double* z, double* tmp) {
    if (precond == 0) { for (int32_t i = 0; i < n; ++i) z[i] = r[i]; return; }
    if (precond == 1) {
        for (int32_t i = 0; i < n; ++i) {
            double d = 0.0;
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k) if (ci[k] == i) d = v[k];
            z[i] = r[i] / d;
        }
        return;
    }
    or_trsv_lower(n, Lrp, Lci, Lv, r, tmp);
    or_trsv_upper(n, Lrp, Lci, Lv, tmp, z);
}

int or_pcg(int32_t n, const int32_t* rp, const int32_t* ci, const double* v, const double* b,
           double* x, int precond, const int32_t* Lrp, const int32_t* Lci, const double* Lv,
           double rtol, int max_iter, int* iters_out, double* relres_out) {
    double* r = (double*)malloc(sizeof(double) * (size_t)n * 5);
    double *z = r + n, *p = z + n, *w = p + n, *tmp = w + n;
    double bnorm = sqrt(dot(n, b, b));
    double tol = rtol * bnorm;
    or_spmv(n, rp, ci, v, x, w);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_threads > 1)
#endif
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
    double rnorm = sqrt(dot(n, r, r));
    int k = 0, status = 0;
    if (rnorm <= tol) goto done;
    apply_prec(precond, n, rp, ci, v, Lrp, Lci, Lv, r, z, tmp);
    double rz = dot(n, r, z);
    if (!(rz > 0.0) || !isfinite(rz)) { status = 2; goto done; }
    for (int32_t i = 0; i < n; ++i) p[i] = z[i];
    for (;;) {
        or_spmv(n, rp, ci, v, p, w);
        double pw = dot(n, p, w);
        if (!(pw > 0.0) || !isfinite(pw)) { status = 2; break; }
        double alpha = rz / pw;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_threads > 1)
#endif
        for (int32_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * w[i]; }
        ++k;
        rnorm = sqrt(dot(n, r, r));
        if (rnorm <= tol) break;
        if (!isfinite(rnorm)) { status = 2; break; }
        if (k >= max_iter) { status = 1; break; }
        apply_prec(precond, n, rp, ci, v, Lrp, Lci, Lv, r, z, tmp);
        double rz_new = dot(n, r, z);
        if (!(rz_new > 0.0) || !isfinite(rz_new)) { status = 2; break; }
        double beta = rz_new / rz;
        rz = rz_new;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_threads > 1)
#endif
        for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
done:
    *iters_out = k;
    *relres_out = bnorm > 0.0 ? rnorm / bnorm : rnorm;
    free(r);
    return status;
}

/* ======================================================================
 * GNN (Sec. 4.2 "Architecture", App. A.3).
 *   MLP of depth l: Linear(in,h) ReLU [Linear(h,h) ReLU] x (l-1) Linear(h,out)
 *   node input b_i / ||b||_inf, edge input A_ij / s, s = max_i A_ii
 *   v_i <- MLP_v([v_i || sum_j e_ij (.) v_j])   (sum over row i incl. j = i)
 *   e_ij <- MLP_e([e_ij || v_i || v_j])         (new v; every directed edge)
 *   s_ij = MLP_dec(e_ij)
 *   diag_mode 0: L_ij = sqrt(s) (s_ij + s_ji)/2 (i > j),  L_ii = sqrt(s) softplus(s_ii)
 *   diag_mode 1 (App. A.3, L D L^T with D = diag(A)): L = L' D^{1/2} with a
 *     unit-diagonal L', L'_ij = (s_ij + s_ji)/2, i.e. L_ii = sqrt(A_ii),
 *     L_ij = sqrt(A_jj) (s_ij + s_ji)/2
 *   diag_mode 2 (the same L D L^T form with D = diag(A), the scaling taken on
 *     the rows): L = D^{1/2} L~ with a unit-diagonal L~, L~_ij = (s_ij + s_ji)/2,
 *     i.e. P = D^{1/2} L~ L~^T D^{1/2}, L~ a factor of the Jacobi-scaled
 *     matrix D^{-1/2} A D^{-1/2}; L_ii = sqrt(A_ii), L_ij = sqrt(A_ii)
 *     (s_ij + s_ji)/2, and the edge input is that matrix's entry
 *     A_ij / sqrt(A_ii A_jj) (1 on the diagonal) instead of A_ij / s
 * Flat weights: node encoder, edge encoder, n_mp x (node MLP, edge MLP),
 * decoder; each Linear W[out][in] then b[out].
 * ==================================================================== */
/* x0_head: the initial-guess head of Sec. 4.4 ("surrogate" use): an MLP of
 * depth l on the final node features, x0_i = (||b||_inf / s) MLP_x(v_i) */
/* loss: 0 Eq. (loss_Ab), 1 Eq. (loss_A) (training only; no weights) */
typedef struct { int n_mp, l, l_mp, h, diag_mode, x0_head, loss; } or_gnn_cfg;

static int64_t mlp_nparams(int in, int h, int out, int depth) {
    int64_t s = (int64_t)in * h + h;
    for (int k = 1; k < depth; ++k) s += (int64_t)h * h + h;
    s += (int64_t)h * out + out;
    return s;
}

int64_t or_gnn_nparams(const or_gnn_cfg* c) {
    int h = c->h;
    int64_t s = 2 * mlp_nparams(1, h, h, c->l);
    s += c->n_mp * (mlp_nparams(2 * h, h, h, c->l_mp) + mlp_nparams(3 * h, h, h, c->l_mp));
    s += mlp_nparams(h, h, 1, c->l);
    if (c->x0_head) s += mlp_nparams(h, h, 1, c->l);
    return s;
}

/* One MLP application.  If tape != NULL, stores the input of every Linear:
 * tape = [x0 (in) | x1 (h) | ... | x_depth (h)], followed by the pre-ReLU
 * values z_0..z_{depth-1} (h each).  Tape size: in + 2*depth*h. */
static void mlp_fwd(const double* w, int in, int h, int out, int depth,
                    const double* x, double* y, double* tape) {
    double buf_a[1024], buf_b[1024];
    const double* cur = x;
    int cur_dim = in;
    const double* wp = w;
    if (tape) memcpy(tape, x, sizeof(double) * (size_t)in);
    for (int layer = 0; layer <= depth; ++layer) {
        int od = (layer == depth) ? out : h;
        const double* W = wp; const double* bb = wp + (int64_t)od * cur_dim;
        double* dst = (layer == depth) ? y : ((layer % 2) ? buf_b : buf_a);
        for (int o = 0; o < od; ++o) {
            double s = bb[o];
            for (int q = 0; q < cur_dim; ++q) s += W[(int64_t)o * cur_dim + q] * cur[q];
            dst[o] = s;
        }
        if (layer < depth) {
            if (tape) memcpy(tape + in + (size_t)depth * h + (size_t)layer * h, dst, sizeof(double) * (size_t)h);
            for (int o = 0; o < od; ++o) dst[o] = dst[o] > 0.0 ? dst[o] : 0.0;
            if (tape) memcpy(tape + in + (size_t)layer * h, dst, sizeof(double) * (size_t)h);
        }
        wp = bb + od;
        cur = dst; cur_dim = od;
    }
}

/* Reverse of mlp_fwd: given dy, accumulates dW into gw (same layout as w)
 * and writes dx (may be NULL). */
static void mlp_bwd(const double* w, double* gw, int in, int h, int out, int depth,
                    const double* tape, const double* dy, double* dx) {
    /* offsets of each Linear */
    int64_t off[64]; int dims[66];
    dims[0] = in; for (int k = 1; k <= depth; ++k) dims[k] = h; dims[depth + 1] = out;
    int64_t o = 0;
    for (int layer = 0; layer <= depth; ++layer) { off[layer] = o; o += (int64_t)dims[layer] * dims[layer + 1] + dims[layer + 1]; }
    double g_cur[1024], g_prev[1024];
    memcpy(g_cur, dy, sizeof(double) * (size_t)out);
    for (int layer = depth; layer >= 0; --layer) {
        int id = dims[layer], od = dims[layer + 1];
        const double* xin = (layer == 0) ? tape : tape + in + (size_t)(layer - 1) * h;
        const double* W = w + off[layer];
        double* gW = gw + off[layer];
        double* gb = gW + (int64_t)od * id;
        for (int oo = 0; oo < od; ++oo) {
            gb[oo] += g_cur[oo];
            for (int q = 0; q < id; ++q) gW[(int64_t)oo * id + q] += g_cur[oo] * xin[q];
        }
        for (int q = 0; q < id; ++q) {
            double s = 0.0;
            for (int oo = 0; oo < od; ++oo) s += W[(int64_t)oo * id + q] * g_cur[oo];
            g_prev[q] = s;
        }
        if (layer > 0) {
            const double* z = tape + in + (size_t)depth * h + (size_t)(layer - 1) * h;
            for (int q = 0; q < id; ++q) g_cur[q] = z[q] > 0.0 ? g_prev[q] : 0.0;
        } else if (dx) {
            memcpy(dx, g_prev, sizeof(double) * (size_t)id);
        }
    }
}

static double softplus(double z) { return (z > 0.0 ? z : 0.0) + log1p(exp(-fabs(z))); }
static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* position of (i, j) in row i of A, or -1 */
static int32_t find_entry(const int32_t* rp, const int32_t* ci, int32_t i, int32_t j) {
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) if (ci[k] == j) return k;
    return -1;
}

typedef struct {
    int64_t nnz; int32_t n; int h, Tn, Te, Td;  /* tape sizes per node / edge MLP / decoder */
    double *v, *e;           /* [n_mp+1][n][h], [n_mp+1][nnz][h] */
    double *agg;             /* [n_mp][n][h] */
    double *tv, *te;         /* node / edge MLP tapes per layer */
    double *tev, *tee;       /* encoder tapes */
    double *td;              /* decoder tapes */
    double *s;               /* decoder outputs [nnz] */
    double *xo, *tx;         /* initial-guess head: outputs [n], tapes [n][Td] */
    double sA, binf;         /* input scales */
} gnn_tape;

static void tape_free(gnn_tape* t) {
    free(t->v); free(t->e); free(t->agg); free(t->tv); free(t->te);
    free(t->tev); free(t->tee); free(t->td); free(t->s);
    free(t->xo); free(t->tx);
}

/* forward; fills Lv on the tril pattern (Lrp/Lci from or_tril) and the tape */
static void gnn_forward_tape(const or_gnn_cfg* c, int32_t n, const int32_t* rp, const int32_t* ci,
                             const double* av, const double* b, const double* w,
                             const int32_t* Lrp, const int32_t* Lci, double* Lv, gnn_tape* T,
                             const double* scales) {
    int h = c->h, l = c->l, lm = c->l_mp;
    int64_t nnz = rp[n];
    T->nnz = nnz; T->n = n; T->h = h;
    int Tenc = 1 + 2 * l * h;
    T->Tn = 2 * h + 2 * lm * h; T->Te = 3 * h + 2 * lm * h; T->Td = h + 2 * l * h;
    T->v = (double*)calloc((size_t)(c->n_mp + 1) * n * h, sizeof(double));
    T->e = (double*)calloc((size_t)(c->n_mp + 1) * nnz * h, sizeof(double));
    T->agg = (double*)calloc((size_t)(c->n_mp ? c->n_mp : 1) * n * h, sizeof(double));
    T->tv = (double*)calloc((size_t)(c->n_mp ? c->n_mp : 1) * n * T->Tn, sizeof(double));
    T->te = (double*)calloc((size_t)(c->n_mp ? c->n_mp : 1) * nnz * T->Te, sizeof(double));
    T->tev = (double*)calloc((size_t)n * Tenc, sizeof(double));
    T->tee = (double*)calloc((size_t)nnz * Tenc, sizeof(double));
    T->td = (double*)calloc((size_t)nnz * T->Td, sizeof(double));
    T->s = (double*)calloc((size_t)nnz, sizeof(double));
    T->xo = c->x0_head ? (double*)calloc((size_t)n, sizeof(double)) : NULL;
    T->tx = c->x0_head ? (double*)calloc((size_t)n * T->Td, sizeof(double)) : NULL;

    /* input scaling */
    double sA = 0.0, binf = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t k = find_entry(rp, ci, i, i);
        if (av[k] > sA) sA = av[k];
        if (fabs(b[i]) > binf) binf = fabs(b[i]);
    }
    if (binf == 0.0) binf = 1.0;
    /* a sub-problem cut from a larger system keeps the parent's scales */
    if (scales) { sA = scales[0]; binf = scales[1]; }

    const double* w_encv = w;
    const double* w_ence = w_encv + mlp_nparams(1, h, h, l);
    const double* w_mp = w_ence + mlp_nparams(1, h, h, l);
    int64_t pn = mlp_nparams(2 * h, h, h, lm), pe = mlp_nparams(3 * h, h, h, lm);
    const double* w_dec = w_mp + c->n_mp * (pn + pe);

    for (int32_t i = 0; i < n; ++i) {
        double x = b[i] / binf;
        mlp_fwd(w_encv, 1, h, h, l, &x, T->v + (size_t)i * h, T->tev + (size_t)i * Tenc);
    }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            double x;
            if (c->diag_mode == 2) {
                const double aii = av[find_entry(rp, ci, i, i)], ajj = av[find_entry(rp, ci, ci[k], ci[k])];
                x = av[k] / sqrt(aii * ajj);
            } else {
                x = av[k] / sA;
            }
            mlp_fwd(w_ence, 1, h, h, l, &x, T->e + (size_t)k * h, T->tee + (size_t)k * Tenc);
        }
    double* in = (double*)malloc(sizeof(double) * 3 * (size_t)h);
    for (int t = 0; t < c->n_mp; ++t) {
        const double* wn = w_mp + t * (pn + pe);
        const double* we = wn + pn;
        double* v0 = T->v + (size_t)t * n * h;   double* v1 = v0 + (size_t)n * h;
        double* e0 = T->e + (size_t)t * nnz * h; double* e1 = e0 + (size_t)nnz * h;
        double* ag = T->agg + (size_t)t * n * h;
        for (int32_t i = 0; i < n; ++i) {
            for (int q = 0; q < h; ++q) ag[(size_t)i * h + q] = 0.0;
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
                for (int q = 0; q < h; ++q)
                    ag[(size_t)i * h + q] += e0[(size_t)k * h + q] * v0[(size_t)ci[k] * h + q];
            memcpy(in, v0 + (size_t)i * h, sizeof(double) * h);
            memcpy(in + h, ag + (size_t)i * h, sizeof(double) * h);
            mlp_fwd(wn, 2 * h, h, h, lm, in, v1 + (size_t)i * h, T->tv + ((size_t)t * n + i) * T->Tn);
        }
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
                memcpy(in, e0 + (size_t)k * h, sizeof(double) * h);
                memcpy(in + h, v1 + (size_t)i * h, sizeof(double) * h);
                memcpy(in + 2 * h, v1 + (size_t)ci[k] * h, sizeof(double) * h);
                mlp_fwd(we, 3 * h, h, h, lm, in, e1 + (size_t)k * h, T->te + ((size_t)t * nnz + k) * T->Te);
            }
    }
    free(in);
    double* eL = T->e + (size_t)c->n_mp * nnz * h;
    for (int64_t k = 0; k < nnz; ++k)
        mlp_fwd(w_dec, h, h, 1, l, eL + (size_t)k * h, T->s + k, T->td + (size_t)k * T->Td);
    T->sA = sA;
    T->binf = binf;
    if (c->x0_head) {
        /* initial-guess head on the final node features (weights after the decoder's) */
        const double* w_x = w_dec + mlp_nparams(h, h, 1, l);
        const double* vL = T->v + (size_t)c->n_mp * n * h;
        for (int32_t i = 0; i < n; ++i)
            mlp_fwd(w_x, h, h, 1, l, vL + (size_t)i * h, T->xo + i, T->tx + (size_t)i * T->Td);
    }
    double rs = sqrt(sA);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t kk = Lrp[i]; kk < Lrp[i + 1]; ++kk) {
            int32_t j = Lci[kk];
            int32_t kij = find_entry(rp, ci, i, j);
            if (c->diag_mode == 1) {
                /* App. A.3: P = L' D L'^T with D = diag(A) and unit-diagonal L',
                 * L'_ij = (s_ij + s_ji)/2; stored as L = L' D^{1/2} */
                double djj = av[find_entry(rp, ci, j, j)];
                if (j == i) Lv[kk] = sqrt(djj);
                else {
                    int32_t kji = find_entry(rp, ci, j, i);
                    Lv[kk] = sqrt(djj) * 0.5 * (T->s[kij] + T->s[kji]);
                }
            } else if (c->diag_mode == 2) {
                /* L = D^{1/2} L~, unit-diagonal L~_ij = (s_ij + s_ji)/2 */
                double dii = av[find_entry(rp, ci, i, i)];
                if (j == i) Lv[kk] = sqrt(dii);
                else {
                    int32_t kji = find_entry(rp, ci, j, i);
                    Lv[kk] = sqrt(dii) * 0.5 * (T->s[kij] + T->s[kji]);
                }
            } else if (j == i) {
                Lv[kk] = rs * softplus(T->s[kij]);
            } else {
                int32_t kji = find_entry(rp, ci, j, i);
                Lv[kk] = rs * 0.5 * (T->s[kij] + T->s[kji]);
            }
        }
}

/* Public forward: Lv on the tril pattern; s_out (optional) = decoder outputs [nnz]. */
void or_gnn_forward(const or_gnn_cfg* c, int32_t n, const int32_t* rp, const int32_t* ci,
                    const double* av, const double* b, const double* w,
                    const int32_t* Lrp, const int32_t* Lci, double* Lv, double* s_out) {
    gnn_tape T;
    gnn_forward_tape(c, n, rp, ci, av, b, w, Lrp, Lci, Lv, &T, NULL);
    if (s_out) memcpy(s_out, T.s, sizeof(double) * (size_t)rp[n]);
    tape_free(&T);
}

/* Forward with the input scales given: scales[0] = s (max diagonal of the
 * whole system), scales[1] = ||b||_inf of the whole system.  Used to evaluate
 * rows of a large system on a subgraph: after n_mp rounds a node's state
 * depends only on nodes within n_mp hops (App. A.3), so L_ij of a row i at the
 * centre of the ball of radius n_mp + 1 around i equals the full system's. */
/* Initial guess of the head: x0_i = (||b||_inf / s) MLP_x(v_i) (needs x0_head). */
void or_gnn_x0(const or_gnn_cfg* c, int32_t n, const int32_t* rp, const int32_t* ci, const double* av,
               const double* b, const double* w, const int32_t* Lrp, const int32_t* Lci, double* Lv, double* x0) {
    gnn_tape T;
    gnn_forward_tape(c, n, rp, ci, av, b, w, Lrp, Lci, Lv, &T, NULL);
    for (int32_t i = 0; i < n; ++i) x0[i] = c->x0_head ? T.binf / T.sA * T.xo[i] : 0.0;
    tape_free(&T);
}

void or_gnn_forward_scaled(const or_gnn_cfg* c, int32_t n, const int32_t* rp, const int32_t* ci,
                           const double* av, const double* b, const double* w,
                           const int32_t* Lrp, const int32_t* Lci, double* Lv, const double* scales) {
    gnn_tape T;
    gnn_forward_tape(c, n, rp, ci, av, b, w, Lrp, Lci, Lv, &T, scales);
    tape_free(&T);
}

/* Reverse pass: given dL on the tril pattern, accumulates dtheta into gw. */
static void gnn_backward(const or_gnn_cfg* c, int32_t n, const int32_t* rp, const int32_t* ci,
                         const double* av, const double* w, const int32_t* Lrp, const int32_t* Lci,
                         const double* dL, gnn_tape* T, double* gw) {
    int h = c->h, l = c->l, lm = c->l_mp;
    int64_t nnz = rp[n];
    int Tenc = 1 + 2 * l * h;
    double sA = 0.0;
    for (int32_t i = 0; i < n; ++i) { int32_t k = find_entry(rp, ci, i, i); if (av[k] > sA) sA = av[k]; }
    double rs = sqrt(sA);
    int64_t penc = mlp_nparams(1, h, h, l);
    int64_t pn = mlp_nparams(2 * h, h, h, lm), pe = mlp_nparams(3 * h, h, h, lm);
    int64_t off_mp = 2 * penc, off_dec = off_mp + c->n_mp * (pn + pe);

    /* dL -> ds */
    double* ds = (double*)calloc((size_t)nnz, sizeof(double));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t kk = Lrp[i]; kk < Lrp[i + 1]; ++kk) {
            int32_t j = Lci[kk];
            int32_t kij = find_entry(rp, ci, i, j);
            if (c->diag_mode == 1 || c->diag_mode == 2) {
                /* L_ii = sqrt(A_ii) is fixed; L_ij = sqrt(A_cc) (s_ij + s_ji)/2
                 * with c = j (mode 1, column scaling) or c = i (mode 2, rows) */
                if (j != i) {
                    int32_t kji = find_entry(rp, ci, j, i);
                    const int32_t cc = c->diag_mode == 1 ? j : i;
                    double g = sqrt(av[find_entry(rp, ci, cc, cc)]) * 0.5 * dL[kk];
                    ds[kij] += g;
                    ds[kji] += g;
                }
            } else if (j == i) {
                ds[kij] += rs * sigmoid(T->s[kij]) * dL[kk];
            } else {
                int32_t kji = find_entry(rp, ci, j, i);
                ds[kij] += rs * 0.5 * dL[kk];
                ds[kji] += rs * 0.5 * dL[kk];
            }
        }
    /* decoder */
    double* de = (double*)calloc((size_t)nnz * h, sizeof(double));
    double* dv = (double*)calloc((size_t)n * h, sizeof(double));
    for (int64_t k = 0; k < nnz; ++k)
        mlp_bwd(w + off_dec, gw + off_dec, h, h, 1, l, T->td + (size_t)k * T->Td, ds + k, de + (size_t)k * h);
    double* de_prev = (double*)calloc((size_t)nnz * h, sizeof(double));
    double* dv_prev = (double*)calloc((size_t)n * h, sizeof(double));
    double* dx = (double*)malloc(sizeof(double) * 3 * (size_t)h);
    for (int t = c->n_mp - 1; t >= 0; --t) {
        int64_t on = off_mp + t * (pn + pe), oe = on + pn;
        double* v0 = T->v + (size_t)t * n * h;
        double* e0 = T->e + (size_t)t * nnz * h;
        memset(de_prev, 0, sizeof(double) * (size_t)nnz * h);
        memset(dv_prev, 0, sizeof(double) * (size_t)n * h);
        /* edge MLP: de (grad of e^{t+1}) -> de_prev, dv (grad of v^{t+1}) */
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
                mlp_bwd(w + oe, gw + oe, 3 * h, h, h, lm, T->te + ((size_t)t * nnz + k) * T->Te,
                        de + (size_t)k * h, dx);
                for (int q = 0; q < h; ++q) {
                    de_prev[(size_t)k * h + q] += dx[q];
                    dv[(size_t)i * h + q] += dx[h + q];
                    dv[(size_t)ci[k] * h + q] += dx[2 * h + q];
                }
            }
        /* node MLP: dv (complete grad of v^{t+1}) -> dv_prev, dagg */
        double* ag_bar = (double*)calloc((size_t)n * h, sizeof(double));
        for (int32_t i = 0; i < n; ++i) {
            mlp_bwd(w + on, gw + on, 2 * h, h, h, lm, T->tv + ((size_t)t * n + i) * T->Tn,
                    dv + (size_t)i * h, dx);
            for (int q = 0; q < h; ++q) {
                dv_prev[(size_t)i * h + q] += dx[q];
                ag_bar[(size_t)i * h + q] = dx[h + q];
            }
        }
        /* aggregation agg_i = sum_j e_ij (.) v_j */
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
                for (int q = 0; q < h; ++q) {
                    double g = ag_bar[(size_t)i * h + q];
                    de_prev[(size_t)k * h + q] += g * v0[(size_t)ci[k] * h + q];
                    dv_prev[(size_t)ci[k] * h + q] += g * e0[(size_t)k * h + q];
                }
        free(ag_bar);
        double* tmp = de; de = de_prev; de_prev = tmp;
        tmp = dv; dv = dv_prev; dv_prev = tmp;
    }
    /* encoders (inputs are data: only weight gradients) */
    for (int32_t i = 0; i < n; ++i)
        mlp_bwd(w, gw, 1, h, h, l, T->tev + (size_t)i * Tenc, dv + (size_t)i * h, NULL);
    for (int64_t k = 0; k < nnz; ++k)
        mlp_bwd(w + penc, gw + penc, 1, h, h, l, T->tee + (size_t)k * Tenc, de + (size_t)k * h, NULL);
    free(dx); free(ds); free(de); free(dv); free(de_prev); free(dv_prev);
}

/* ======================================================================
 * Loss Eq. (loss_Ab): l = (1/B) sum_p ||L_p L_p^T x_p - b_p||^2, one GNN
 * forward per pair (its node input is b_p).  With y = L^T x, u = L y,
 * r = u - b, w = L^T r:  dl/dL_ij = (2/B)(r_i y_j + x_i w_j) on tril(A).
 * grad (optional) accumulates dl/dtheta (caller zeroes it).
 * ==================================================================== */
static void lower_mv(int32_t n, const int32_t* Lrp, const int32_t* Lci, const double* Lv,
                     const double* x, double* y) {           /* y = L x */
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k) s += Lv[k] * x[Lci[k]];
        y[i] = s;
    }
}
static void lowerT_mv(int32_t n, const int32_t* Lrp, const int32_t* Lci, const double* Lv,
                      const double* x, double* y) {          /* y = L^T x */
    for (int32_t i = 0; i < n; ++i) y[i] = 0.0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k) y[Lci[k]] += Lv[k] * x[i];
}

/* loss of a given L (no network): also returns dl/dL (scaled by 1/B) */
double or_llt_loss(int32_t n, const int32_t* Lrp, const int32_t* Lci, const double* Lv,
                   int npairs, const double* X, const double* B, double* dL) {
    double* y = (double*)malloc(sizeof(double) * 4 * (size_t)n);
    double *u = y + n, *r = u + n, *wv = r + n;
    double loss = 0.0;
    int64_t nnzL = Lrp[n];
    if (dL) for (int64_t k = 0; k < nnzL; ++k) dL[k] = 0.0;
    for (int p = 0; p < npairs; ++p) {
        const double* x = X + (size_t)p * n; const double* b = B + (size_t)p * n;
        lowerT_mv(n, Lrp, Lci, Lv, x, y);
        lower_mv(n, Lrp, Lci, Lv, y, u);
        double s = 0.0;
        for (int32_t i = 0; i < n; ++i) { r[i] = u[i] - b[i]; s += r[i] * r[i]; }
        loss += s / npairs;
        if (dL) {
            lowerT_mv(n, Lrp, Lci, Lv, r, wv);
            for (int32_t i = 0; i < n; ++i)
                for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k) {
                    int32_t j = Lci[k];
                    dL[k] += (2.0 / npairs) * (r[i] * y[j] + x[i] * wv[j]);
                }
        }
    }
    free(y);
    return loss;
}

/* Frobenius loss of Eq. (loss_A) for one L and its system A:
 *   l = ||L L^T - A||_F^2 over the full n x n matrices (the fill-in of L L^T
 *   outside the pattern of A included),
 *   dl/dL_ik = 4 ((L L^T - A) L)_ik on the pattern of L (R symmetric).
 * Written out densely: R and L as n x n arrays (test sizes only). */
double or_frob_loss(int32_t n, const int32_t* rp, const int32_t* ci, const double* av,
                    const int32_t* Lrp, const int32_t* Lci, const double* Lv, double* dL) {
    double* Ld = (double*)calloc((size_t)n * n, sizeof(double));
    double* R = (double*)calloc((size_t)n * n, sizeof(double));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k) Ld[(size_t)i * n + Lci[k]] = Lv[k];
    /* (L L^T)_ij = sum_k L_ik L_jk */
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j) {
            double sum = 0.0;
            for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k) sum += Lv[k] * Ld[(size_t)j * n + Lci[k]];
            R[(size_t)i * n + j] = sum;
        }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) R[(size_t)i * n + ci[k]] -= av[k];
    double loss = 0.0;
    for (size_t e = 0; e < (size_t)n * n; ++e) loss += R[e] * R[e];
    if (dL)
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = Lrp[i]; k < Lrp[i + 1]; ++k) {
                const int32_t col = Lci[k];
                double sum = 0.0;
                for (int32_t j = 0; j < n; ++j) sum += R[(size_t)i * n + j] * Ld[(size_t)j * n + col];
                dL[k] = 4.0 * sum;
            }
    free(Ld); free(R);
    return loss;
}

/* Loss over the (x, b) pairs of one system and its gradient in the flat
 * weights.  c->loss = 0: Eq. (loss_Ab), ||L L^T x - b||^2; 1: Eq. (loss_A),
 * ||L L^T - A||_F^2 with L = f(A, b_p) (the node input is b_p, so each
 * pair still has its own L).  Mean over the pairs. */
double or_loss_and_grad(const or_gnn_cfg* c, int32_t n, const int32_t* rp, const int32_t* ci,
                        const double* av, int npairs, const double* X, const double* B,
                        const double* w, double* grad) {
    int64_t nnzL = or_tril(n, rp, ci, NULL, NULL, NULL, NULL, NULL);
    int32_t* Lrp = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t* Lci = (int32_t*)malloc(sizeof(int32_t) * (size_t)nnzL);
    double* Lv = (double*)malloc(sizeof(double) * (size_t)nnzL);
    double* dL = (double*)malloc(sizeof(double) * (size_t)nnzL);
    or_tril(n, rp, ci, NULL, Lrp, Lci, NULL, NULL);
    double loss = 0.0;
    for (int p = 0; p < npairs; ++p) {
        gnn_tape T;
        gnn_forward_tape(c, n, rp, ci, av, B + (size_t)p * n, w, Lrp, Lci, Lv, &T, NULL);
        /* this pair's share of the mean */
        double lp = c->loss == 1 ? or_frob_loss(n, rp, ci, av, Lrp, Lci, Lv, grad ? dL : NULL)
                                 : or_llt_loss(n, Lrp, Lci, Lv, 1, X + (size_t)p * n, B + (size_t)p * n, grad ? dL : NULL);
        loss += lp / npairs;
        if (grad) {
            for (int64_t k = 0; k < nnzL; ++k) dL[k] /= npairs;
            gnn_backward(c, n, rp, ci, av, w, Lrp, Lci, dL, &T, grad);
        }
        if (c->x0_head) {
            /* regression of the head to x in its own output units,
             * sum_i (MLP_x(v_i) - x_i s / ||b||_inf)^2; the trunk is not
             * differentiated through (the preconditioner is trained by the
             * loss above alone) */
            const int h = c->h, l = c->l;
            int64_t off_x = or_gnn_nparams(c) - mlp_nparams(h, h, 1, l);
            const double t_scale = T.sA / T.binf;
            const double* xp = X + (size_t)p * n;
            double lx = 0.0;
            for (int32_t i = 0; i < n; ++i) {
                const double d = T.xo[i] - xp[i] * t_scale;
                lx += d * d;
                if (grad) {
                    const double dy = 2.0 * d / npairs;
                    mlp_bwd(w + off_x, grad + off_x, h, h, 1, l, T.tx + (size_t)i * T.Td, &dy, NULL);
                }
            }
            loss += lx / npairs;
        }
        tape_free(&T);
    }
    free(Lrp); free(Lci); free(Lv); free(dL);
    return loss;
}

/* ======================================================================
 * Adam (App. A.4 uses Adam with lr 1e-3; Kingma & Ba defaults otherwise).
 * t is the 1-based step count.
 * ==================================================================== */
void or_adam(int64_t np, double* w, const double* g, double* m, double* v, int t,
             double lr, double b1, double b2, double eps) {
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t k = 0; k < np; ++k) {
        m[k] = b1 * m[k] + (1.0 - b1) * g[k];
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
        double mh = m[k] / c1, vh = v[k] / c2;
        w[k] -= lr * mh / (sqrt(vh) + eps);
    }
}
