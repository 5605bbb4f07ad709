// Assembly of the stiffness matrix A of -div(k grad u) = f with homogeneous
// Dirichlet boundary (Sec. 3 "Discretization", standard Galerkin), or of the
// implicit time-step matrix M + tau K of the heat / wave equation with a
// Dirichlet arc of the FEM boundary (Sec. 5.1 environments).  The
// paper's meshes and simulator are not available; the problems are
// synthetic stand-ins on the unit square / cube:
//   FD : 5/7-point stencil, face coefficient = harmonic mean of nodal k.
//   FEM: P1 elements on the Delaunay triangulation of a jittered lattice,
//        assembled row by row (each interior point gathers the element
//        contributions of its incident triangles; no atomics).
// log k is a Gaussian random field given by random Fourier features.
#include <algorithm>

#include "npcg_internal.cuh"

namespace npcg {

namespace {

constexpr int kMaxFeatures = 2048;

// g(p) = sigma sqrt(2/M) sum_m cos(omega_m . p + phase_m) for npts points;
// point coordinates come from a callback-free layout: coord[p * dim + d].
__global__ void k_grf(int dim, int64_t npts, const double* pts, int M, const double* omega,
                      const double* phase, double sigma, double* g) {
    extern __shared__ double sh[];   // [M * (dim + 1)]
    for (int t = threadIdx.x; t < M * dim; t += blockDim.x) sh[t] = omega[t];
    for (int t = threadIdx.x; t < M; t += blockDim.x) sh[M * dim + t] = phase[t];
    __syncthreads();
    const double amp = sigma * sqrt(2.0 / (double)M);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (sigma == 0.0) { g[p] = 0.0; continue; }
        double x[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < dim; ++d) x[d] = pts[p * dim + d];
        double s = 0.0;
        for (int m = 0; m < M; ++m) {
            double arg = sh[M * dim + m];
            for (int d = 0; d < dim; ++d) arg = fma(sh[m * dim + d], x[d], arg);
            s += cos(arg);
        }
        g[p] = amp * s;
    }
}

// ---------------------------------------------------------------- FD
// Extended grid (nx+2) x (ny+2) (x (nz+2)) including the Dirichlet layer.
__global__ void k_fd_points(int dim, int nx, int ny, int nz, double* pts) {
    int ex = nx + 2, ey = ny + 2, ez = dim == 3 ? nz + 2 : 1;
    int64_t np = (int64_t)ex * ey * ez;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(p % ex), j = (int)((p / ex) % ey), l = (int)(p / ((int64_t)ex * ey));
        pts[p * dim + 0] = (double)i / (double)(nx + 1);
        pts[p * dim + 1] = (double)j / (double)(ny + 1);
        if (dim == 3) pts[p * dim + 2] = (double)l / (double)(nz + 1);
    }
}

__global__ void k_fd_rows(int dim, int nx, int ny, int nz, const double* g, double tau, int32_t* rp,
                          int32_t* ci, double* val, int pass) {
    // tau > 0: h^2 I + tau K (lumped mass in the units of the h-free stencil)
    const double ks = tau > 0.0 ? tau : 1.0;
    const double hh = tau > 0.0 ? 1.0 / ((double)(nx + 1) * (double)(nx + 1)) : 0.0;
    const int ex = nx + 2, ey = ny + 2;
    const int nzz = dim == 3 ? nz : 1;
    const int64_t n = (int64_t)nx * ny * nzz;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(a % nx), j = (int)((a / nx) % ny), l = (int)(a / ((int64_t)nx * ny));
        int le = dim == 3 ? l + 1 : 0;
        auto kat = [&](int ii, int jj, int ll) {
            return exp(g[((int64_t)ll * ey + jj) * ex + ii]);
        };
        const double ka = kat(i + 1, j + 1, le);
        // neighbours in ascending column order: -z, -y, -x, self, +x, +y, +z
        const int di[7] = {0, 0, -1, 0, 1, 0, 0};
        const int dj[7] = {0, -1, 0, 0, 0, 1, 0};
        const int dl[7] = {-1, 0, 0, 0, 0, 0, 1};
        double kf[7];
        double diag = 0.0;
        int cnt = 0;
        for (int d = 0; d < 7; ++d) {
            if (d == 3) continue;
            if (dim == 2 && (d == 0 || d == 6)) { kf[d] = 0.0; continue; }
            int i2 = i + di[d], j2 = j + dj[d], l2 = l + dl[d];
            double kb = kat(i2 + 1, j2 + 1, dim == 3 ? l2 + 1 : 0);
            kf[d] = 2.0 * ka * kb / (ka + kb);
            diag += kf[d];
        }
        for (int d = 0; d < 7; ++d) {
            if (dim == 2 && (d == 0 || d == 6)) continue;
            int i2 = i + di[d], j2 = j + dj[d], l2 = l + dl[d];
            bool in = i2 >= 0 && i2 < nx && j2 >= 0 && j2 < ny && l2 >= 0 && l2 < nzz;
            if (!in) continue;
            if (pass == 1) {
                int32_t pos = rp[a] + cnt;
                ci[pos] = (int32_t)(((int64_t)l2 * ny + j2) * nx + i2);
                val[pos] = d == 3 ? ks * diag + hh : -ks * kf[d];
            }
            ++cnt;
        }
        if (pass == 0) rp[a] = cnt;
    }
}

// ---------------------------------------------------------------- FEM
__device__ __forceinline__ void fem_xy(int m, const int32_t* jit, int a, int c, long long* X,
                                       long long* Y) {
    int64_t id = (int64_t)a + (int64_t)m * c;
    *X = (long long)a * 1024 + jit[2 * id];
    *Y = (long long)c * 1024 + jit[2 * id + 1];
}

__global__ void k_fem_points(int m, const int32_t* jit, double* pts) {
    int64_t np = (int64_t)m * m;
    const double scale = 1024.0 * (double)(m - 1);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        int a = (int)(p % m), c = (int)(p / m);
        long long X, Y;
        fem_xy(m, jit, a, c, &X, &Y);
        pts[2 * p] = (double)X / scale;
        pts[2 * p + 1] = (double)Y / scale;
    }
}

// in-circle determinant of (p00, p10, p11) and p01, exact in int64
__global__ void k_fem_diag(int m, const int32_t* jit, int8_t* dg) {
    int64_t nc = (int64_t)(m - 1) * (m - 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nc;
         t += (int64_t)gridDim.x * blockDim.x) {
        int a = (int)(t % (m - 1)), c = (int)(t / (m - 1));
        long long P[4][2];
        const int pa[4] = {a, a + 1, a + 1, a}, pc[4] = {c, c, c + 1, c + 1};
        for (int q = 0; q < 4; ++q) fem_xy(m, jit, pa[q], pc[q], &P[q][0], &P[q][1]);
        long long adx = P[0][0] - P[3][0], ady = P[0][1] - P[3][1];
        long long bdx = P[1][0] - P[3][0], bdy = P[1][1] - P[3][1];
        long long cdx = P[2][0] - P[3][0], cdy = P[2][1] - P[3][1];
        long long al = adx * adx + ady * ady, bl = bdx * bdx + bdy * bdy, cl = cdx * cdx + cdy * cdy;
        long long det = al * (bdx * cdy - cdx * bdy) - bl * (adx * cdy - cdx * ady) + cl * (adx * bdy - bdx * ady);
        dg[t] = det > 0 ? 1 : 0;
    }
}

// perimeter index k -> point id a + m c (counter-clockwise from (0,0))
__device__ __forceinline__ int64_t perimeter_point(int m, int64_t k) {
    const int64_t e = m - 1;
    if (k < e) return k;
    if (k < 2 * e) return (m - 1) + (int64_t)m * (k - e);
    if (k < 3 * e) return (m - 1 - (k - 2 * e)) + (int64_t)m * (m - 1);
    return (int64_t)m * (m - 1 - (k - 3 * e));
}

// free[p] = 1 for an unknown point: interior, or a boundary point outside
// the Dirichlet arc (dir_len = 0: the whole boundary is Dirichlet).  One
// block: the arc is cleared after the whole lattice is marked.
__global__ void k_fem_free(int m, int dir_start, int dir_len, int32_t* fr) {
    const int64_t np = (int64_t)m * m, per = 4 * (int64_t)(m - 1);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(p % m), c = (int)(p / m);
        const bool bnd = a == 0 || a == m - 1 || c == 0 || c == m - 1;
        fr[p] = bnd && dir_len == 0 ? 0 : 1;
    }
    __syncthreads();
    // the arc (a point may be listed once only: dir_len <= perimeter)
    const int64_t len = dir_len < per ? dir_len : per;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < len;
         t += (int64_t)gridDim.x * blockDim.x)
        fr[perimeter_point(m, (dir_start + t) % per)] = 0;
}

// uid[p] = unknown index of point p (-1: Dirichlet) and rowpt[uid] = p,
// from the exclusive scan of free[]
__global__ void k_fem_uid(int64_t np, int64_t n, const int32_t* fr, const int32_t* scan, int32_t* uid,
                          int32_t* rowpt) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int u = fr[p] ? scan[p] : -1;
        uid[p] = u < n ? u : -1;
        if (u >= 0 && u < n) rowpt[u] = (int32_t)p;
    }
}

// Row of unknown point (a, c): accumulates the 3x3 stencil slots
// (dc, da) in {-1,0,1}^2 over the two triangles of each incident cell
// (cells inside the lattice only); vertices that are Dirichlet are skipped.
// tau > 0: tau K + M, every vertex pair of an element in the pattern.
__device__ void fem_row(int m, int a, int c, const int32_t* jit, const double* pts, const double* g,
                        const int8_t* dg, const int32_t* uid, double tau, double* sv, int* sf) {
    for (int s = 0; s < 9; ++s) { sv[s] = 0.0; sf[s] = 0; }
    for (int cc = c - 1; cc <= c; ++cc)
        for (int ca = a - 1; ca <= a; ++ca) {
            if (ca < 0 || cc < 0 || ca > m - 2 || cc > m - 2) continue;
            int64_t p00 = ca + (int64_t)m * cc;
            int64_t v[2][3];
            if (dg[ca + (int64_t)(m - 1) * cc] == 0) {
                v[0][0] = p00; v[0][1] = p00 + 1; v[0][2] = p00 + m + 1;
                v[1][0] = p00; v[1][1] = p00 + m + 1; v[1][2] = p00 + m;
            } else {
                v[0][0] = p00; v[0][1] = p00 + 1; v[0][2] = p00 + m;
                v[1][0] = p00 + 1; v[1][1] = p00 + m + 1; v[1][2] = p00 + m;
            }
            const int64_t me = a + (int64_t)m * c;
            for (int t = 0; t < 2; ++t) {
                int s = -1;
                for (int q = 0; q < 3; ++q) if (v[t][q] == me) s = q;
                if (s < 0) continue;
                double ex[3], ey[3];
                long long ix[3], iy[3];
                for (int q = 0; q < 3; ++q) {
                    int64_t q1 = v[t][(q + 1) % 3], q2 = v[t][(q + 2) % 3];
                    ex[q] = pts[2 * q2] - pts[2 * q1];
                    ey[q] = pts[2 * q2 + 1] - pts[2 * q1 + 1];
                    long long X1, Y1, X2, Y2;
                    fem_xy(m, jit, (int)(q1 % m), (int)(q1 / m), &X1, &Y1);
                    fem_xy(m, jit, (int)(q2 % m), (int)(q2 / m), &X2, &Y2);
                    ix[q] = X2 - X1;
                    iy[q] = Y2 - Y1;
                }
                double area = 0.5 * (ex[2] * (-ey[1]) - ey[2] * (-ex[1]));
                double kT = exp((g[v[t][0]] + g[v[t][1]] + g[v[t][2]]) / 3.0);
                for (int u = 0; u < 3; ++u) {
                    int64_t pu = v[t][u];
                    if (uid[pu] < 0) continue;
                    int au = (int)(pu % m), cu = (int)(pu / m);
                    int slot = (cu - c + 1) * 3 + (au - a + 1);
                    double dot = ex[s] * ex[u] + ey[s] * ey[u];
                    long long doti = ix[s] * ix[u] + iy[s] * iy[u];
                    const double kst = kT * dot / (4.0 * area);
                    if (tau > 0.0) {
                        sv[slot] += tau * kst + area * (s == u ? 2.0 : 1.0) / 12.0;
                        sf[slot] = 1;
                    } else {
                        sv[slot] += kst;
                        sf[slot] |= doti != 0;
                    }
                }
            }
        }
}

__global__ void k_fem_rows(int m, int64_t n, const int32_t* rowpt, const int32_t* uid, const int32_t* jit,
                           const double* pts, const double* g, const int8_t* dg, double tau, int32_t* rp,
                           int32_t* ci, double* val, int pass) {
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = rowpt[row];
        int a = (int)(p % m), c = (int)(p / m);
        double sv[9];
        int sf[9];
        fem_row(m, a, c, jit, pts, g, dg, uid, tau, sv, sf);
        // slots in ascending point order, hence ascending unknown index
        int cnt = 0;
        for (int s = 0; s < 9; ++s) {
            if (s != 4 && !sf[s]) continue;
            int au = a + s % 3 - 1, cu = c + s / 3 - 1;
            if (au < 0 || au > m - 1 || cu < 0 || cu > m - 1) continue;
            const int32_t col = uid[au + (int64_t)m * cu];
            if (col < 0) continue;
            if (pass == 1) {
                int32_t pos = rp[row] + cnt;
                ci[pos] = col;
                val[pos] = sv[s];
            }
            ++cnt;
        }
        if (pass == 0) rp[row] = cnt;
    }
}

// number of FEM unknowns: interior points plus the boundary points off the arc
int64_t fem_unknowns(const npcg_problem* p) {
    const int64_t m = p->nx, per = 4 * (m - 1);
    if (p->dir_len == 0) return (m - 2) * (m - 2);
    return (m - 2) * (m - 2) + per - std::min<int64_t>(p->dir_len, per);
}

int grid_of(int64_t n, int cap) {
    int64_t g = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

npcg_status check_problem(Handle* h, const npcg_problem* p) {
    if (!p) return set_error(h, NPCG_EINVAL, "problem is NULL");
    if (p->n_features < 0 || p->n_features > kMaxFeatures)
        return set_error(h, NPCG_EINVAL, "n_features must be in [0, 2048]");
    if (p->sigma != 0.0 && (!p->omega || !p->phase || p->n_features == 0))
        return set_error(h, NPCG_EINVAL, "sigma != 0 needs omega and phase");
    if (!(p->tau >= 0.0) || p->tau > 1e300) return set_error(h, NPCG_EINVAL, "tau must be finite and >= 0");
    if (p->dir_len < 0 || p->dir_start < 0) return set_error(h, NPCG_EINVAL, "dir_start and dir_len must be >= 0");
    if (p->kind == NPCG_FD) {
        if (p->dir_len != 0 || p->dir_start != 0)
            return set_error(h, NPCG_EINVAL, "Dirichlet arcs are defined for FEM problems only");
        if (p->dim != 2 && p->dim != 3) return set_error(h, NPCG_EINVAL, "FD dim must be 2 or 3");
        if (p->nx < 1 || p->ny < 1 || (p->dim == 3 && p->nz < 1))
            return set_error(h, NPCG_EINVAL, "FD grid sizes must be >= 1");
        long long n = (long long)p->nx * p->ny * (p->dim == 3 ? p->nz : 1);
        if (n * 7 >= (1LL << 31)) return set_error(h, NPCG_EINVAL, "FD system too large for int32 CSR");
    } else if (p->kind == NPCG_FEM) {
        if (p->dim != 2) return set_error(h, NPCG_EINVAL, "FEM is 2-D");
        if (p->nx < 3) return set_error(h, NPCG_EINVAL, "FEM needs m >= 3");
        if (!p->jitter) return set_error(h, NPCG_EINVAL, "FEM needs the jitter array");
        if ((long long)p->nx * p->nx * 7 >= (1LL << 31)) return set_error(h, NPCG_EINVAL, "FEM system too large");
    } else {
        return set_error(h, NPCG_EINVAL, "unknown problem kind");
    }
    return NPCG_OK;
}

// Shared driver: pass 0 counts per row into rp, pass 1 fills.
npcg_status assemble_impl(Handle* h, const npcg_problem* p, int32_t* rp_counts, int32_t* rp,
                          int32_t* ci, double* val, int64_t* n_out, int64_t* nnz_out) {
    NPCG_TRY(check_problem(h, p));
    const int M = p->sigma != 0.0 ? p->n_features : 0;
    const int cap = h->num_sms * 16;
    const size_t grf_smem = (size_t)std::max(M, 1) * (p->dim + 1) * sizeof(double);
    NPCG_CUDA(h, cudaFuncSetAttribute(k_grf, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    if (p->kind == NPCG_FD) {
        const int nzz = p->dim == 3 ? p->nz : 1;
        const int64_t n = (int64_t)p->nx * p->ny * nzz;
        const int64_t np = (int64_t)(p->nx + 2) * (p->ny + 2) * (p->dim == 3 ? p->nz + 2 : 1);
        DevBuf<double> pts, g;
        NPCG_CUDA(h, pts.alloc(np * p->dim));
        NPCG_CUDA(h, g.alloc(np));
        k_fd_points<<<grid_of(np, cap), 256, 0, h->stream>>>(p->dim, p->nx, p->ny, p->nz, pts.p);
        k_grf<<<grid_of(np, cap), 256, grf_smem, h->stream>>>(p->dim, np, pts.p, M, p->omega, p->phase, p->sigma, g.p);
        k_fd_rows<<<grid_of(n, cap), 256, 0, h->stream>>>(p->dim, p->nx, p->ny, p->nz, g.p, p->tau, rp_counts,
                                                          nullptr, nullptr, 0);
        NPCG_CUDA(h, cudaGetLastError());
        if (n_out) *n_out = n;
        if (rp) {
            NPCG_TRY(scan_i32_to_i32(h, rp_counts, rp, n));
            k_fd_rows<<<grid_of(n, cap), 256, 0, h->stream>>>(p->dim, p->nx, p->ny, p->nz, g.p, p->tau, rp, ci,
                                                              val, 1);
            NPCG_CUDA(h, cudaGetLastError());
        }
        NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
        if (nnz_out) {
            int nx = p->nx, ny = p->ny;
            int64_t e = (int64_t)(nx - 1) * ny * nzz + (int64_t)nx * (ny - 1) * nzz;
            if (p->dim == 3) e += (int64_t)nx * ny * (nzz - 1);
            *nnz_out = n + 2 * e;
        }
        return NPCG_OK;
    }
    const int m = p->nx;
    const int64_t np = (int64_t)m * m, n = fem_unknowns(p);
    DevBuf<double> pts, g;
    DevBuf<int8_t> dg;
    DevBuf<int32_t> fr, scan, uid, rowpt;
    NPCG_CUDA(h, pts.alloc(np * 2));
    NPCG_CUDA(h, g.alloc(np));
    NPCG_CUDA(h, dg.alloc((size_t)(m - 1) * (m - 1)));
    NPCG_CUDA(h, fr.alloc(np));
    NPCG_CUDA(h, scan.alloc(np + 1));
    NPCG_CUDA(h, uid.alloc(np));
    NPCG_CUDA(h, rowpt.alloc(std::max<int64_t>(n, 1)));
    k_fem_free<<<1, 256, 0, h->stream>>>(m, p->dir_start, p->dir_len, fr.p);
    NPCG_TRY(scan_i32_to_i32(h, fr.p, scan.p, np));
    NPCG_CUDA(h, cudaMemsetAsync(rowpt.p, 0, std::max<int64_t>(n, 1) * sizeof(int32_t), h->stream));
    k_fem_uid<<<grid_of(np, cap), 256, 0, h->stream>>>(np, n, fr.p, scan.p, uid.p, rowpt.p);
    k_fem_points<<<grid_of(np, cap), 256, 0, h->stream>>>(m, p->jitter, pts.p);
    k_grf<<<grid_of(np, cap), 256, grf_smem, h->stream>>>(2, np, pts.p, M, p->omega, p->phase, p->sigma, g.p);
    k_fem_diag<<<grid_of((int64_t)(m - 1) * (m - 1), cap), 256, 0, h->stream>>>(m, p->jitter, dg.p);
    k_fem_rows<<<grid_of(n, cap), 256, 0, h->stream>>>(m, n, rowpt.p, uid.p, p->jitter, pts.p, g.p, dg.p, p->tau,
                                                       rp_counts, nullptr, nullptr, 0);
    NPCG_CUDA(h, cudaGetLastError());
    if (n_out) *n_out = n;
    if (rp) {
        NPCG_TRY(scan_i32_to_i32(h, rp_counts, rp, n));
        k_fem_rows<<<grid_of(n, cap), 256, 0, h->stream>>>(m, n, rowpt.p, uid.p, p->jitter, pts.p, g.p, dg.p,
                                                           p->tau, rp, ci, val, 1);
        NPCG_CUDA(h, cudaGetLastError());
    }
    if (nnz_out) {
        DevBuf<int32_t> tmp;
        NPCG_CUDA(h, tmp.alloc(n + 1));
        NPCG_TRY(scan_i32_to_i32(h, rp_counts, tmp.p, n));
        int32_t nnz = 0;
        NPCG_TRY(read_scalar(h, tmp.p + n, &nnz));
        *nnz_out = nnz;
    }
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    return NPCG_OK;
}

}  // namespace

npcg_status assemble_count_run(Handle* h, const npcg_problem* p, int64_t* n, int64_t* nnz) {
    NPCG_TRY(check_problem(h, p));
    int64_t nn = p->kind == NPCG_FD ? (int64_t)p->nx * p->ny * (p->dim == 3 ? p->nz : 1) : fem_unknowns(p);
    DevBuf<int32_t> counts;
    NPCG_CUDA(h, counts.alloc(nn + 1));
    return assemble_impl(h, p, counts.p, nullptr, nullptr, nullptr, n, nnz);
}

npcg_status assemble_run(Handle* h, const npcg_problem* p, int32_t* rp, int32_t* ci, double* v) {
    NPCG_TRY(check_problem(h, p));
    int64_t nn = p->kind == NPCG_FD ? (int64_t)p->nx * p->ny * (p->dim == 3 ? p->nz : 1) : fem_unknowns(p);
    DevBuf<int32_t> counts;
    NPCG_CUDA(h, counts.alloc(nn + 1));
    return assemble_impl(h, p, counts.p, rp, ci, v, nullptr, nullptr);
}

}  // namespace npcg
