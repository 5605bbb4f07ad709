// PCG (Algorithm 1) in FP64 on the GPU: CSR SpMV, sync-free level-ordered
// sparse triangular solves for "Solve P z = r" with P = L L^T, fused vector
// updates with deterministic per-system reductions, and the iteration as a
// CUDA graph whose while-loop runs on the device until every system of the
// pattern has converged, failed, or reached max_iter.
#include <algorithm>
#include <vector>

#include "npcg_internal.cuh"

namespace npcg {

namespace {

constexpr int kTrsvThreads = 256;
constexpr int kDepChunk = 8;

// ------------------------------------------------------------------ reduce
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double (*sh)[kChunkThreads / 32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        double x = v[j];
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[j][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double s = 0.0;
            for (int w = 0; w < kChunkThreads / 32; ++w) s += sh[j][w];
            v[j] = s;
        }
    }
}

// Publishes this chunk's partial sums; returns true (in every thread of the
// block) for the last chunk of its system to arrive, which then owns the
// finalisation.
template <int N>
__device__ __forceinline__ bool publish(const Chunk& c, const double (&v)[N], double* part,
                                        unsigned* arrive, const int32_t* sys_chunk0) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < N; ++j) part[(int64_t)c.slot * 4 + j] = v[j];
        __threadfence();
        unsigned nch = (unsigned)(sys_chunk0[c.sys + 1] - sys_chunk0[c.sys]);
        unsigned prev = atomicAdd(&arrive[c.sys], 1u);
        last = (prev == nch - 1);
    }
    __syncthreads();
    return last;
}

// Sums the system's chunk partials with the whole block (fixed assignment,
// so the result is deterministic); the total ends in thread 0.
template <int N>
__device__ __forceinline__ void gather_parts(const Chunk& c, const double* part,
                                             const int32_t* sys_chunk0, unsigned* arrive,
                                             double (&tot)[N], double (*sh)[kChunkThreads / 32]) {
    __threadfence();
#pragma unroll
    for (int j = 0; j < N; ++j) tot[j] = 0.0;
    for (int q = sys_chunk0[c.sys] + threadIdx.x; q < sys_chunk0[c.sys + 1]; q += kChunkThreads)
#pragma unroll
        for (int j = 0; j < N; ++j) tot[j] += __ldcg(part + (int64_t)q * 4 + j);
    block_sum<N>(tot, sh);
    if (threadIdx.x == 0) arrive[c.sys] = 0u;
}

__device__ __forceinline__ void deactivate(SysState& s, int status, int* n_active) {
    s.status = status;
    s.active = 0;
    atomicSub(n_active, 1);
}

// ------------------------------------------------------------------ kernels
struct PcgArgs {
    const int32_t* rp;
    const int32_t* ci;
    const double* av;
    const int32_t* adiag;
    const Chunk* chunks;
    const int32_t* sys_chunk0;
    SysState* st;
    double* part;
    unsigned* arrive;
    int* ctl;            // [0] n_active [1] flags [2] fwd ticket [3] bwd ticket
    double *x, *r, *z, *y, *w, *b;
    void* rperm;              // level-synchronous mode: r in forward processing order
    const int32_t* cposf;     //   and the forward position of each row
    int rperm_f32;            //   stored as FP32 (NPCG_PREC_LLT32) or FP64
    int precond;
    int short_rows;           // every row has <= kShortRow entries: one thread per row in the SpMV
};

__device__ __forceinline__ void store_perm(const PcgArgs& a, int row, double ri) {
    const int q = a.cposf[row];
    if (a.rperm_f32) static_cast<float*>(a.rperm)[q] = (float)ri;
    else static_cast<double*>(a.rperm)[q] = ri;
}

// sum_j A_ij * v_j for one row by a group of G lanes (row entries strided by G)
// (every lane of the warp calls this; lanes of an invalid row add nothing)
template <int G>
__device__ __forceinline__ double row_dot(const int32_t* rp, const int32_t* ci, const double* av,
                                          const double* v, int row, int g, bool valid) {
    double s = 0.0;
    const int k1 = valid ? rp[row + 1] : 0;
    for (int k = valid ? rp[row] + g : 0; k < k1; k += G) s = fma(av[k], v[ci[k]], s);
#pragma unroll
    for (int o = G / 2; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, G);
    return s;
}

// r = b - A x; partials ||b||^2, ||r||^2; finaliser sets tolerances and the
// active mask; sentinels and p buffers are reset for the first iteration.
__global__ void k_init(PcgArgs a, double rtol, int max_iter, double* p0, double* p1, int stall_k) {
    __shared__ double sh[2][kChunkThreads / 32];
    const Chunk c = a.chunks[blockIdx.x];
    const int g = threadIdx.x & 7, sub = (threadIdx.x >> 3) & 3, warp = threadIdx.x >> 5;
    double acc[2] = {0.0, 0.0};
    for (int base = c.row0 + warp * 4; base < c.row1; base += kChunkThreads / 8) {
        const int row = base + sub;
        const bool valid = row < c.row1;
        double ax = row_dot<8>(a.rp, a.ci, a.av, a.x, row, g, valid);
        if (g == 0 && valid) {
            double bi = a.b[row];
            double ri = bi - ax;
            a.r[row] = ri;
            if (a.rperm) store_perm(a, row, ri);
            p0[row] = 0.0;
            p1[row] = 0.0;
            a.y[row] = sentinel_f64();
            a.z[row] = sentinel_f64();
            acc[0] = fma(bi, bi, acc[0]);
            acc[1] = fma(ri, ri, acc[1]);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) { a.ctl[2] = 0; a.ctl[3] = 0; }
    block_sum<2>(acc, sh);
    if (publish<2>(c, acc, a.part, a.arrive, a.sys_chunk0)) {
        double tot[2];
        gather_parts<2>(c, a.part, a.sys_chunk0, a.arrive, tot, sh);
        if (threadIdx.x != 0) return;
        SysState& s = a.st[c.sys];
        s.bnorm2 = tot[0];
        s.tol2 = rtol * rtol * tot[0];
        s.rr = tot[1];
        s.iters = 0;
        s.max_iter = max_iter;
        s.beta = 0.0;
        s.alpha = 0.0;
        s.rz = 0.0;
        s.pw = 0.0;
        s.best_rr = tot[1];
        s.since_best = 0;
        s.stall_k = stall_k;
        if (!(tot[1] <= s.tol2)) {
            if (max_iter <= 0) {
                s.status = NPCG_EMAXITER;
                s.active = 0;
            } else if (isfinite(tot[1])) {
                s.status = NPCG_OK;
                s.active = 1;
                atomicAdd(&a.ctl[0], 1);
            } else {
                s.status = NPCG_EBREAKDOWN;
                s.active = 0;
            }
        } else {
            s.status = NPCG_OK;
            s.active = 0;
        }
    }
}

// elementwise preconditioners (z = r / diag or z = r) with r^T z partials;
// used for the initial z (finalise_beta = false sets rz) and, fused in
// k_update, every iteration.
__device__ __forceinline__ double elementwise_z(const PcgArgs& a, int row, double ri) {
    return a.precond == NPCG_PREC_JACOBI ? ri / a.av[a.adiag[row]] : ri;
}

// r^T z; finaliser: first call (init) stores rz, later calls compute beta.
__global__ void k_dot_rz(PcgArgs a, int init) {
    __shared__ double sh[1][kChunkThreads / 32];
    const Chunk c = a.chunks[blockIdx.x];
    if (!a.st[c.sys].active) return;
    double acc[1] = {0.0};
    for (int row = c.row0 + threadIdx.x; row < c.row1; row += kChunkThreads) {
        double ri = a.r[row];
        double zi;
        if (a.precond >= NPCG_PREC_LLT) zi = a.z[row];
        else { zi = elementwise_z(a, row, ri); a.z[row] = zi; }
        acc[0] = fma(ri, zi, acc[0]);
    }
    block_sum<1>(acc, sh);
    if (publish<1>(c, acc, a.part, a.arrive, a.sys_chunk0)) {
        double tot[1];
        gather_parts<1>(c, a.part, a.sys_chunk0, a.arrive, tot, sh);
        if (threadIdx.x != 0) return;
        SysState& s = a.st[c.sys];
        double rz = tot[0];
        if (!(rz > 0.0) || !isfinite(rz)) {
            deactivate(s, NPCG_EBREAKDOWN, &a.ctl[0]);
        } else {
            s.beta = init ? 0.0 : rz / s.rz;
            s.rz = rz;
        }
    }
}

// p_new = z + beta p_old (Algorithm 1), streamed once per iteration so the
// SpMV below gathers one vector
__global__ void k_pnew(PcgArgs a, const double* __restrict__ p_old, double* __restrict__ p_new) {
    const Chunk c = a.chunks[blockIdx.x];
    const SysState& s0 = a.st[c.sys];
    if (!s0.active) return;
    const double beta = s0.beta;
    for (int row = c.row0 + threadIdx.x; row < c.row1; row += kChunkThreads)
        p_new[row] = fma(beta, p_old[row], a.z[row]);
}

// w = A p, partial p^T w; finaliser: alpha = rz / p^T w.
__global__ void k_spmv_p(PcgArgs a, const double* __restrict__ p) {
    __shared__ double sh[1][kChunkThreads / 32];
    const Chunk c = a.chunks[blockIdx.x];
    const SysState& s0 = a.st[c.sys];
    if (!s0.active) return;
    double acc[1] = {0.0};
    if (a.short_rows) {
        // one thread per row: a warp keeps 32 rows' entries in flight (the
        // eight-lane mapping below keeps four), which is what a bandwidth-
        // bound stencil or mesh row of 7-9 entries needs
        for (int row = c.row0 + threadIdx.x; row < c.row1; row += kChunkThreads) {
            const int k0 = a.rp[row], k1 = a.rp[row + 1];
            double s = 0.0;
#pragma unroll 4
            for (int k = k0; k < k1; ++k) s = fma(a.av[k], p[a.ci[k]], s);
            a.w[row] = s;
            acc[0] = fma(p[row], s, acc[0]);
        }
    } else {
        const int g = threadIdx.x & 7, sub = (threadIdx.x >> 3) & 3, warp = threadIdx.x >> 5;
        for (int base = c.row0 + warp * 4; base < c.row1; base += kChunkThreads / 8) {
            const int row = base + sub;
            const bool valid = row < c.row1;
            double s = 0.0;
            const int k1 = valid ? a.rp[row + 1] : 0;
            for (int k = valid ? a.rp[row] + g : 0; k < k1; k += 8) s = fma(a.av[k], p[a.ci[k]], s);
#pragma unroll
            for (int o = 4; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, 8);
            if (g == 0 && valid) {
                a.w[row] = s;
                acc[0] = fma(p[row], s, acc[0]);
            }
        }
    }
    block_sum<1>(acc, sh);
    if (publish<1>(c, acc, a.part, a.arrive, a.sys_chunk0)) {
        double tot[1];
        gather_parts<1>(c, a.part, a.sys_chunk0, a.arrive, tot, sh);
        if (threadIdx.x != 0) return;
        SysState& s = a.st[c.sys];
        s.pw = tot[0];
        if (!(tot[0] > 0.0) || !isfinite(tot[0])) deactivate(s, NPCG_EBREAKDOWN, &a.ctl[0]);
        else s.alpha = s.rz / tot[0];
    }
}

// x += alpha p, r -= alpha w, ||r||^2 (and, for the elementwise
// preconditioners, z and r^T z); finaliser counts the update, tests
// convergence (||r|| <= rtol ||b||) and max_iter, and computes beta.
__global__ void k_update(PcgArgs a, const double* __restrict__ p) {
    __shared__ double sh[2][kChunkThreads / 32];
    if (blockIdx.x == 0 && threadIdx.x == 0) { a.ctl[2] = 0; a.ctl[3] = 0; }
    const Chunk c = a.chunks[blockIdx.x];
    const SysState& s0 = a.st[c.sys];
    if (!s0.active) return;
    const double alpha = s0.alpha;
    const bool llt = a.precond >= NPCG_PREC_LLT;
    double acc[2] = {0.0, 0.0};
    for (int row = c.row0 + threadIdx.x; row < c.row1; row += kChunkThreads) {
        a.x[row] = fma(alpha, p[row], a.x[row]);
        double ri = fma(-alpha, a.w[row], a.r[row]);
        a.r[row] = ri;
        if (a.rperm) store_perm(a, row, ri);
        acc[0] = fma(ri, ri, acc[0]);
        if (llt) {
            a.y[row] = sentinel_f64();
            a.z[row] = sentinel_f64();
        } else {
            double zi = elementwise_z(a, row, ri);
            a.z[row] = zi;
            acc[1] = fma(ri, zi, acc[1]);
        }
    }
    block_sum<2>(acc, sh);
    if (publish<2>(c, acc, a.part, a.arrive, a.sys_chunk0)) {
        double tot[2];
        gather_parts<2>(c, a.part, a.sys_chunk0, a.arrive, tot, sh);
        if (threadIdx.x != 0) return;
        SysState& s = a.st[c.sys];
        s.rr = tot[0];
        s.iters += 1;
        if (tot[0] < s.best_rr) {
            s.best_rr = tot[0];
            s.since_best = 0;
        } else {
            s.since_best += 1;
        }
        if (tot[0] <= s.tol2) {
            deactivate(s, NPCG_OK, &a.ctl[0]);
        } else if (!isfinite(tot[0])) {
            deactivate(s, NPCG_EBREAKDOWN, &a.ctl[0]);
        } else if (s.iters >= s.max_iter) {
            deactivate(s, NPCG_EMAXITER, &a.ctl[0]);
        } else if (s.stall_k > 0 && s.since_best > 0 && s.since_best >= s.stall_k) {
            // ||r|| has not fallen below its best for stall_k updates
            deactivate(s, NPCG_ESTALL, &a.ctl[0]);
        } else if (!llt) {
            double rz = tot[1];
            if (!(rz > 0.0) || !isfinite(rz)) deactivate(s, NPCG_EBREAKDOWN, &a.ctl[0]);
            else { s.beta = rz / s.rz; s.rz = rz; }
        }
    }
}

// ------------------------------------------------------------------ SpTRSV
struct TriDev {
    int64_t n;
    int32_t nslices;
    const int32_t* perm;
    const int64_t* soff;
    const int32_t* sw;
    const int32_t* col;
    const void* val;    // V[slots]
    const void* dinv;   // V[n] reciprocal diagonal by position
};

// One warp per 32-row slice, one lane per row, slices claimed in level order
// by a ticket counter, so every dependency belongs to an earlier-claimed
// (running) warp or to a lower lane of the same slice.  out[] holds the
// sentinel until written.  Each round, every unfinished lane polls the
// pending dependencies of its current chunk of (up to 8) off-diagonals; once
// a chunk is complete the lane folds it in slot order (so the result does
// not depend on timing), moves to its next chunk, and publishes its row the
// moment its last chunk is folded -- inside the round, because other lanes
// of the same warp may be waiting for it.
template <bool kBatched, class V>
__global__ void __launch_bounds__(kTrsvThreads) k_trsv(TriDev T, const double* __restrict__ rhs,
                                                       double* out, int* ticket, int* flags,
                                                       const int32_t* row_sys, const SysState* st,
                                                       long long spin_limit) {
    const V* tval = static_cast<const V*>(T.val);
    const V* tdinv = static_cast<const V*>(T.dinv);
    const int lane = threadIdx.x & 31;
    const unsigned long long kS = kSentinelBits;
    if (!kBatched && st && !st[0].active) return;
    for (;;) {
        int slice = 0;
        if (lane == 0) slice = atomicAdd(ticket, 1);
        slice = __shfl_sync(0xffffffffu, slice, 0);
        if (slice >= T.nslices) return;
        const int64_t q = (int64_t)slice * kSlice + lane;
        const int row = q < T.n ? T.perm[q] : -1;
        bool act = row >= 0;
        if (kBatched && act) act = st[row_sys[row]].active != 0;
        const int width = T.sw[slice];
        const int64_t off = T.soff[slice];
        V acc = act ? (V)rhs[row] : (V)0;
        const V dinv = act ? tdinv[q] : (V)1;
        int cj[kDepChunk];
        V lv[kDepChunk], yv[kDepChunk];
        unsigned pend = 0;
        int k0 = 0;
        bool done = !act;
        // first chunk
#pragma unroll
        for (int k = 0; k < kDepChunk; ++k) {
            cj[k] = -1;
            lv[k] = (V)0;
            yv[k] = (V)0;
            if (act && k < width) {
                const int64_t slot = off + (int64_t)k * kSlice + lane;
                cj[k] = T.col[slot];
                lv[k] = tval[slot];
                if (cj[k] >= 0) pend |= 1u << k;
            }
        }
        long long spins = 0;
        while (__any_sync(0xffffffffu, !done)) {
            if (!done) {
#pragma unroll
                for (int k = 0; k < kDepChunk; ++k) {
                    if (pend & (1u << k)) {
                        const unsigned long long bits = ld_relaxed_u64(out + cj[k]);
                        if (bits != kS) {
                            yv[k] = (V)__longlong_as_double((long long)bits);
                            pend &= ~(1u << k);
                        }
                    }
                }
                while (!done && pend == 0) {
#pragma unroll
                    for (int k = 0; k < kDepChunk; ++k)
                        if (cj[k] >= 0) acc = fma(-lv[k], yv[k], acc);
                    k0 += kDepChunk;
                    if (k0 >= width) {
                        st_relaxed_u64(out + row, (unsigned long long)__double_as_longlong((double)(acc * dinv)));
                        done = true;
                    } else {
#pragma unroll
                        for (int k = 0; k < kDepChunk; ++k) {
                            cj[k] = -1;
                            if (k0 + k < width) {
                                const int64_t slot = off + (int64_t)(k0 + k) * kSlice + lane;
                                cj[k] = T.col[slot];
                                lv[k] = tval[slot];
                                if (cj[k] >= 0) pend |= 1u << k;
                            }
                        }
                    }
                }
            }
            if (++spins > spin_limit) {
                if (!done) atomicOr(flags, kFlagTimeout | kFlagAbort);
                return;
            }
            if ((spins & 255) == 0) {
                const int f = lane == 0 ? ld_relaxed_s32(flags) : 0;
                if (__shfl_sync(0xffffffffu, f, 0) & kFlagAbort) return;
            }
        }
    }
}

__global__ void k_load_factor(int64_t slots, const int32_t* src, const double* L, double* val,
                              float* val32, int64_t n, const int32_t* dsrc, double* dinv, float* dinv32) {
    int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t st = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = i0; i < slots; i += st) {
        int s = src[i];
        double v = s >= 0 ? L[s] : 0.0;
        val[i] = v;
        val32[i] = (float)v;
    }
    for (int64_t i = i0; i < n; i += st) {
        double d = 1.0 / L[dsrc[i]];
        dinv[i] = d;
        dinv32[i] = (float)d;
    }
}

__global__ void k_fill_sentinel(int64_t n, double* y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = sentinel_f64();
}

// y = A x with one thread per row (rows of at most kShortRow entries)
__global__ void k_spmv_rows(int64_t n, const int32_t* rp, const int32_t* ci, const double* av,
                            const double* x, double* y) {
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int k0 = rp[row], k1 = rp[row + 1];
        double s = 0.0;
#pragma unroll 4
        for (int k = k0; k < k1; ++k) s = fma(av[k], x[ci[k]], s);
        y[row] = s;
    }
}

__global__ void k_spmv_plain(int64_t n, const int32_t* rp, const int32_t* ci, const double* av,
                             const double* x, double* y) {
    const int g = threadIdx.x & 7;
    const int64_t wbase = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 4;
    const int64_t wstride = (((int64_t)gridDim.x * blockDim.x) >> 5) * 4;
    for (int64_t base = wbase; base < n; base += wstride) {
        const int64_t row = base + ((threadIdx.x >> 3) & 3);
        const bool valid = row < n;
        double s = row_dot<8>(rp, ci, av, x, (int)row, g, valid);
        if (g == 0 && valid) y[row] = s;
    }
}

// Loop condition of the device-side while: some system still active, no
// abort, and the trip count (ctl[4]) below its bound (ctl[5], set by the
// host from max_iter; every system stops by max_iter, so reaching the bound
// means the bookkeeping failed and the loop is cut with an abort).
__global__ void k_set_cond(cudaGraphConditionalHandle hd, int* ctl) {
    if (threadIdx.x == 0) {
        int trips = ++ctl[4];
        int go = ctl[0] > 0 && !(ctl[1] & kFlagAbort);
        if (go && trips >= ctl[5]) {
            ctl[1] |= kFlagAbort | kFlagTripBound;
            go = 0;
        }
        cudaGraphSetConditional(hd, go ? 1u : 0u);
    }
}

__global__ void k_stats(int nsys, const SysState* st, npcg_solve_stats* out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsys) {
        out[s].iters = st[s].iters;
        out[s].status = st[s].status;
        double b2 = st[s].bnorm2;
        out[s].relres = b2 > 0.0 ? sqrt(st[s].rr / b2) : sqrt(st[s].rr);
        out[s].fallback = 0;
        out[s].fallback_iters = 0;
    }
}

TriDev tri_dev(const Pattern* P, const TriLayout& T, bool f32) {
    TriDev d;
    d.n = P->n;
    d.nslices = T.nslices;
    d.perm = T.perm.p;
    d.soff = T.slice_off.p;
    d.sw = T.slice_w.p;
    d.col = T.col.p;
    d.val = f32 ? (const void*)T.val32.p : (const void*)T.val.p;
    d.dinv = f32 ? (const void*)T.dinv32.p : (const void*)T.dinv.p;
    return d;
}

int trsv_grid(Handle* h, const TriLayout& T) {
    int warps_needed = T.nslices;
    int blocks = ceil_div(warps_needed, kTrsvThreads / 32);
    return std::max(1, std::min(blocks, h->num_sms * 4));
}

void launch_trsv(Handle* h, cudaStream_t s, Pattern* P, int transpose, const double* rhs, double* out,
                 int* ticket, bool batched, const SysState* st, bool f32) {
    const TriLayout& T = transpose ? P->bwd : P->fwd;
    TriDev d = tri_dev(P, T, f32);
    const int g = trsv_grid(h, T);
    int* fl = P->ctl.p + 1;
    const long long lim = h->spin_limit;
    if (f32) {
        if (batched) k_trsv<true, float><<<g, kTrsvThreads, 0, s>>>(d, rhs, out, ticket, fl, P->row_sys.p, st, lim);
        else k_trsv<false, float><<<g, kTrsvThreads, 0, s>>>(d, rhs, out, ticket, fl, P->row_sys.p, st, lim);
    } else {
        if (batched) k_trsv<true, double><<<g, kTrsvThreads, 0, s>>>(d, rhs, out, ticket, fl, P->row_sys.p, st, lim);
        else k_trsv<false, double><<<g, kTrsvThreads, 0, s>>>(d, rhs, out, ticket, fl, P->row_sys.p, st, lim);
    }
}

npcg_status ensure_pcg_workspace(Handle* h, Pattern* P) {
    const int64_t n = P->n;
    NPCG_CUDA(h, P->x.ensure(n));
    NPCG_CUDA(h, P->r.ensure(n));
    NPCG_CUDA(h, P->z.ensure(n));
    NPCG_CUDA(h, P->y.ensure(n));
    NPCG_CUDA(h, P->w.ensure(n));
    NPCG_CUDA(h, P->p0.ensure(n));
    NPCG_CUDA(h, P->p1.ensure(n));
    NPCG_CUDA(h, P->b.ensure(n));
    NPCG_CUDA(h, P->Aval_dev.ensure(P->nnz));
    NPCG_CUDA(h, P->part.ensure((size_t)P->nchunks * 4));
    if (P->arrive.n < (size_t)P->nsys) {
        NPCG_CUDA(h, P->arrive.alloc(P->nsys));
        NPCG_CUDA(h, cudaMemsetAsync(P->arrive.p, 0, P->nsys * sizeof(unsigned), h->stream));
    }
    NPCG_CUDA(h, P->st.ensure(P->nsys));
    NPCG_CUDA(h, P->stats_dev.ensure(P->nsys));
    if (P->cfwd.built) {
        NPCG_CUDA(h, P->r_cf.ensure(P->n + 4));
        NPCG_CUDA(h, P->y_cb.ensure(P->n + 4));
        NPCG_CUDA(h, P->yglob.ensure(P->n));
        NPCG_CUDA(h, P->yq.ensure(P->n + 4));
    }
    return NPCG_OK;
}

PcgArgs pcg_args(Pattern* P, int precond) {
    PcgArgs a;
    a.rp = P->rp.p;
    a.ci = P->ci.p;
    a.av = P->Aval_dev.p;
    a.adiag = P->adiag.p;
    a.chunks = P->chunks.p;
    a.sys_chunk0 = P->sys_chunk0.p;
    a.st = P->st.p;
    a.part = P->part.p;
    a.arrive = P->arrive.p;
    a.ctl = P->ctl.p;
    a.x = P->x.p;
    a.r = P->r.p;
    a.z = P->z.p;
    a.y = P->y.p;
    a.w = P->w.p;
    a.b = P->b.p;
    a.precond = precond;
    a.short_rows = P->max_row <= kShortRow;
    // the level-synchronous solve reads r in its processing order (the merged
    // solve gathers r itself)
    const bool cta = P->trsv_mode == kTrsvCta && !P->cta_merge && precond >= NPCG_PREC_LLT;
    a.rperm = cta ? (void*)P->r_cf.p : nullptr;
    a.cposf = cta ? P->cfwd.cpos.p : nullptr;
    a.rperm_f32 = precond == NPCG_PREC_LLT32;
    return a;
}

// z = L^-T L^-1 r with the tuned triangular-solve design
npcg_status apply_llt(Handle* h, cudaStream_t s, Pattern* P, bool batched, bool f32) {
    if (P->trsv_mode == kTrsvCta && P->cta_merge) return merge_apply(h, s, P, f32);
    if (P->trsv_mode == kTrsvCta) {
        if (P->cfwd.blocked) {
            // row blocks publish to y and z (natural order; the update kernel
            // resets them to the sentinel and the tickets to zero every iteration)
            NPCG_TRY(cta_trsv_launch(h, s, P, P->cfwd, P->r_cf.p, P->yq.p, P->st.p, f32, P->ctl.p + 2, P->y.p));
            NPCG_TRY(cta_permute(h, s, P, P->cfwd, P->yq.p, f32, P->cbwd.other.p, P->y_cb.p, f32));
            return cta_trsv_launch(h, s, P, P->cbwd, P->y_cb.p, P->yq.p, P->st.p, f32, P->ctl.p + 3, P->z.p);
        }
        NPCG_TRY(cta_trsv_launch(h, s, P, P->cfwd, P->r_cf.p, P->yq.p, P->st.p, f32));
        NPCG_TRY(cta_permute(h, s, P, P->cfwd, P->yq.p, f32, P->cbwd.other.p, P->y_cb.p, f32));
        NPCG_TRY(cta_trsv_launch(h, s, P, P->cbwd, P->y_cb.p, P->yq.p, P->st.p, f32));
        return cta_permute(h, s, P, P->cbwd, P->yq.p, f32, P->cbwd.cpos.p, P->z.p, false);
    }
    launch_trsv(h, s, P, 0, P->r.p, P->y.p, P->ctl.p + 2, batched, P->st.p, f32);
    launch_trsv(h, s, P, 1, P->y.p, P->z.p, P->ctl.p + 3, batched, P->st.p, f32);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

// one PCG iteration (Algorithm 1 loop body) on the stream
npcg_status enqueue_iteration(Handle* h, cudaStream_t s, Pattern* P, const PcgArgs& a, const double* p_old,
                              double* p_new) {
    const bool batched = P->nsys > 1;
    k_pnew<<<P->nchunks, kChunkThreads, 0, s>>>(a, p_old, p_new);
    k_spmv_p<<<P->nchunks, kChunkThreads, 0, s>>>(a, p_new);
    k_update<<<P->nchunks, kChunkThreads, 0, s>>>(a, p_new);
    if (a.precond >= NPCG_PREC_LLT) {
        NPCG_TRY(apply_llt(h, s, P, batched, a.precond == NPCG_PREC_LLT32));
        k_dot_rz<<<P->nchunks, kChunkThreads, 0, s>>>(a, 0);
    }
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

npcg_status build_graph(Handle* h, Pattern* P, int precond) {
    // the graph is specific to the triangular-solve design
    const int mode_key = P->trsv_mode | (P->cta_flag ? 16 : 0) | (P->cta_split ? 32 : 0) | (P->cta_merge ? 64 : 0);
    if (P->graph[precond] && P->graph_mode[precond] == mode_key && P->graph_spin[precond] == h->spin_limit)
        return NPCG_OK;
    if (P->graph[precond]) { cudaGraphExecDestroy(P->graph[precond]); P->graph[precond] = nullptr; }
    PcgArgs a = pcg_args(P, precond);
    cudaGraph_t g = nullptr;
    NPCG_CUDA(h, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hd;
    cudaError_t e = cudaGraphConditionalHandleCreate(&hd, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(h, e, "cudaGraphConditionalHandleCreate"); }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(h, e, "cudaGraphAddNode(conditional)"); }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // captured on the handle's private stream (the caller's stream may be the
    // legacy default stream, which cannot capture)
    cudaStream_t cs = h->capture_stream;
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(h, e, "cudaStreamBeginCaptureToGraph"); }
    // two iterations per trip so the p ping-pong is static
    npcg_status st = enqueue_iteration(h, cs, P, a, P->p0.p, P->p1.p);
    if (st == NPCG_OK) st = enqueue_iteration(h, cs, P, a, P->p1.p, P->p0.p);
    if (st == NPCG_OK) k_set_cond<<<1, 32, 0, cs>>>(hd, P->ctl.p);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    if (st != NPCG_OK) {
        // a refused layout or a failed launch inside the capture: the status
        // and its message are already recorded on the handle
        cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(h, e, "cudaStreamEndCapture"); }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    P->graph[precond] = ex;
    P->graph_mode[precond] = mode_key;
    P->graph_spin[precond] = h->spin_limit;
    return NPCG_OK;
}

}  // namespace

npcg_status factor_load(Handle* h, Pattern* P, const double* L_val) {
    if (P->cfwd.built) {
        NPCG_TRY(cta_factor_load(h, &P->cfwd, L_val));
        NPCG_TRY(cta_factor_load(h, &P->cbwd, L_val));
    }
    if (P->cta_merge) NPCG_TRY(merge_factor_load(h, P, L_val));
    int blocks = h->num_sms * 4;
    for (TriLayout* T : {&P->fwd, &P->bwd})
        k_load_factor<<<blocks, 256, 0, h->stream>>>(T->slots, T->src.p, L_val, T->val.p, T->val32.p, P->n,
                                                     T->diag_src.p, T->dinv.p, T->dinv32.p);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

npcg_status sptrsv_run(Handle* h, Pattern* P, int transpose, const double* r, double* y,
                       const int32_t*) {
    NPCG_CUDA(h, cudaMemsetAsync(P->ctl.p + 1, 0, 3 * sizeof(int), h->stream));
    if (P->trsv_mode == kTrsvCta && P->cta_merge) {
        NPCG_TRY(ensure_pcg_workspace(h, P));
        return merge_sptrsv(h, h->stream, P, transpose, r, y, false, nullptr, nullptr);
    }
    if (P->trsv_mode == kTrsvCta) {
        NPCG_TRY(ensure_pcg_workspace(h, P));
        const CtaLayout& C = transpose ? P->cbwd : P->cfwd;
        NPCG_TRY(cta_gather(h, h->stream, C, P->n, r, P->r_cf.p, false));
        if (C.blocked) k_fill_sentinel<<<h->num_sms * 4, 256, 0, h->stream>>>(P->n, P->y.p);
        NPCG_TRY(cta_trsv_launch(h, h->stream, P, C, P->r_cf.p, P->yq.p, nullptr, false,
                                 P->ctl.p + 2 + (transpose ? 1 : 0), P->y.p));
        return cta_permute(h, h->stream, P, C, P->yq.p, false, C.cpos.p, y, false);
    }
    k_fill_sentinel<<<h->num_sms * 4, 256, 0, h->stream>>>(P->n, y);
    launch_trsv(h, h->stream, P, transpose, r, y, P->ctl.p + 2 + (transpose ? 1 : 0), false, nullptr, false);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

npcg_status sptrsv_unclaimed_run(Handle* h, Pattern* P, int transpose, int skip, const double* r, double* y) {
    const TriLayout& T = transpose ? P->bwd : P->fwd;
    if (skip < 0 || skip > T.nslices) return set_error(h, NPCG_EINVAL, "skip must be in [0, number of slices]");
    // flags and both tickets cleared, then this direction's ticket set past
    // the skipped slices: no warp ever claims them, so their rows stay at
    // the sentinel and their dependants wait until the wait limit
    NPCG_CUDA(h, cudaMemsetAsync(P->ctl.p + 1, 0, 3 * sizeof(int), h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(P->ctl.p + 2 + (transpose ? 1 : 0), &skip, sizeof(int), cudaMemcpyHostToDevice,
                                 h->stream));
    k_fill_sentinel<<<h->num_sms * 4, 256, 0, h->stream>>>(P->n, y);
    launch_trsv(h, h->stream, P, transpose, r, y, P->ctl.p + 2 + (transpose ? 1 : 0), false, nullptr, false);
    NPCG_CUDA(h, cudaGetLastError());
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    return NPCG_OK;
}

npcg_status sptrsv_timed_run(Handle* h, Pattern* P, int transpose, const double* r, double* y, int reps,
                             double* ms_per_launch, bool f32) {
    NPCG_TRY(ensure_pcg_workspace(h, P));
    cudaEvent_t e0, e1;
    NPCG_CUDA(h, cudaEventCreate(&e0));
    NPCG_CUDA(h, cudaEventCreate(&e1));
    double total = 0.0;
    npcg_status st = NPCG_OK;
    for (int k = 0; k < reps && st == NPCG_OK; ++k) {
        cudaMemsetAsync(P->ctl.p + 1, 0, 3 * sizeof(int), h->stream);
        if (P->trsv_mode == kTrsvCta && P->cta_merge) {
            st = merge_sptrsv(h, h->stream, P, transpose, r, y, f32, e0, e1);
        } else if (P->trsv_mode == kTrsvCta) {
            const CtaLayout& C = transpose ? P->cbwd : P->cfwd;
            cta_gather(h, h->stream, C, P->n, r, P->r_cf.p, f32);
            if (C.blocked) k_fill_sentinel<<<h->num_sms * 4, 256, 0, h->stream>>>(P->n, P->y.p);
            cudaEventRecord(e0, h->stream);
            cta_trsv_launch(h, h->stream, P, C, P->r_cf.p, P->yq.p, nullptr, f32, P->ctl.p + 2 + (transpose ? 1 : 0),
                            P->y.p);
            cudaEventRecord(e1, h->stream);
            cta_permute(h, h->stream, P, C, P->yq.p, f32, C.cpos.p, y, false);
        } else {
            k_fill_sentinel<<<h->num_sms * 4, 256, 0, h->stream>>>(P->n, y);
            cudaEventRecord(e0, h->stream);
            launch_trsv(h, h->stream, P, transpose, r, y, P->ctl.p + 2 + (transpose ? 1 : 0), false, nullptr, f32);
            cudaEventRecord(e1, h->stream);
        }
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { st = cuda_fail(h, e, "trsv timing"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        total += ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != NPCG_OK) return st;
    int flags = 0;
    NPCG_TRY(read_scalar(h, P->ctl.p + 1, &flags));
    if (flags & kFlagTimeout) return set_error(h, NPCG_ETIMEOUT, "triangular solve wait timed out");
    *ms_per_launch = reps > 0 ? total / reps : 0.0;
    return NPCG_OK;
}

namespace {
__global__ void k_fill_value(int64_t n, double* x, double v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}
}  // namespace

// Times the forward + backward solve in both designs on this pattern (with a
// placeholder factor: timing depends on the structure only) and keeps the
// faster.  Runs once, at analysis.
npcg_status trsv_autotune(Handle* h, Pattern* P) {
    if (!P->cfwd.built || cta_stages(P->cfwd) < 2 || cta_stages(P->cbwd) < 2) {
        P->trsv_mode = kTrsvSyncFree;
        return NPCG_OK;
    }
    NPCG_TRY(ensure_pcg_workspace(h, P));
    DevBuf<double> L, r, y;
    NPCG_CUDA(h, L.alloc(P->nnzL));
    NPCG_CUDA(h, r.alloc(P->n));
    NPCG_CUDA(h, y.alloc(P->n));
    int blocks = std::max(1, std::min(ceil_div(P->n, 256), h->num_sms * 8));
    k_fill_value<<<blocks, 256, 0, h->stream>>>(P->nnzL, L.p, 1.0);
    k_fill_value<<<blocks, 256, 0, h->stream>>>(P->n, r.p, 1.0);
    NPCG_CUDA(h, cudaGetLastError());
    // all entries 1: a well-defined solve of the same structure (values do not
    // change the timing)
    NPCG_TRY(factor_load(h, P, L.p));
    // one large system in row blocks: the number of blocks (one per SM, or
    // half or a quarter as many thicker ones) is chosen by timing the
    // level-synchronous solve, and the layouts are rebuilt for it
    if (P->cfwd.blocked) {
        const int cand[3] = {h->num_sms, h->num_sms / 2, h->num_sms / 4};
        double best_u = 1e30;
        int best = cand[0];
        P->trsv_mode = kTrsvCta;
        P->cta_flag = P->cta_split = P->cta_merge = false;
        for (int U : cand) {
            if (U < 1) continue;
            if (U != P->block_units) {
                P->block_units = U;
                NPCG_TRY(cta_layout_build(h, P, false, &P->cfwd));
                NPCG_TRY(cta_layout_build(h, P, true, &P->cbwd));
                NPCG_TRY(cta_link(h, P));
                NPCG_TRY(factor_load(h, P, L.p));
            }
            if (cta_stages(P->cfwd) < 2 || cta_stages(P->cbwd) < 2) continue;
            double t = 1e30;
            for (int rep = 0; rep < 3; ++rep) {
                double f = 0.0, b = 0.0;
                NPCG_TRY(sptrsv_timed_run(h, P, 0, r.p, y.p, 1, &f, true));
                NPCG_TRY(sptrsv_timed_run(h, P, 1, r.p, y.p, 1, &b, true));
                t = std::min(t, f + b);
            }
            if (t < best_u) { best_u = t; best = U; }
        }
        if (best != P->block_units) {
            P->block_units = best;
            NPCG_TRY(cta_layout_build(h, P, false, &P->cfwd));
            NPCG_TRY(cta_layout_build(h, P, true, &P->cbwd));
            NPCG_TRY(cta_link(h, P));
            NPCG_TRY(factor_load(h, P, L.p));
        }
    }
    // sync-free and level order with a barrier per step; the flag-synchronised
    // and split-role variants measured slower on every workload and are not
    // timed (npcg_pattern_set_trsv still selects them)
    const int modes[2] = {kTrsvSyncFree, kTrsvCta};
    P->tune_ms[2] = 0.f;
    P->tune_ms[3] = 0.f;
    for (int m = 0; m < 2; ++m) {
        P->trsv_mode = modes[m];
        P->cta_flag = false;
        P->cta_split = false;
        double best = 1e30;
        for (int rep = 0; rep < 3; ++rep) {
            double f = 0.0, b = 0.0;
            NPCG_TRY(sptrsv_timed_run(h, P, 0, r.p, y.p, 1, &f, true));
            NPCG_TRY(sptrsv_timed_run(h, P, 1, r.p, y.p, 1, &b, true));
            best = std::min(best, f + b);
        }
        P->tune_ms[m] = (float)best;
    }
    // merged levels: the fastest of 2, 4 and 8 levels per step
    P->tune_ms[4] = 0.f;
    P->merge_G = 0;
    if (kMergeEnabled && P->n <= ((int64_t)1 << 22)) {
        // the host plan grows with G (eight levels per group on 2^21 rows
        // take several gigabytes and tens of seconds to plan, four about 8 s):
        // above 2^20 rows only G = 2 is tried (on the 128^3 grid G = 4 never
        // beat it)
        const int cand[3] = {2, 4, 8};
        double best_all = 1e30;
        for (int G : cand) {
            if (G >= 4 && P->n > ((int64_t)1 << 20)) continue;
            if (merge_build(h, P, G) != NPCG_OK) continue;
            if (cta_stages(P->mfwd.lay) < 2 || cta_stages(P->mbwd.lay) < 2) continue;
            P->trsv_mode = kTrsvCta;
            P->cta_flag = false;
            P->cta_split = false;
            P->cta_merge = true;
            NPCG_TRY(merge_factor_load(h, P, L.p));
            double best = 1e30;
            for (int rep = 0; rep < 3; ++rep) {
                double f = 0.0, b = 0.0;
                NPCG_TRY(sptrsv_timed_run(h, P, 0, r.p, y.p, 1, &f, true));
                NPCG_TRY(sptrsv_timed_run(h, P, 1, r.p, y.p, 1, &b, true));
                best = std::min(best, f + b);
            }
            if (best < best_all) {
                best_all = best;
                P->merge_G = G;
            }
        }
        P->cta_merge = false;
        if (P->merge_G) {
            P->tune_ms[4] = (float)best_all;
            NPCG_TRY(merge_build(h, P, P->merge_G));
        }
    }
    trsv_pick_tuned(P);
    return NPCG_OK;
}

// the fastest measured design (a zero time: the design does not apply)
void trsv_pick_tuned(Pattern* P) {
    int m = 0;
    for (int k = 1; k < 5; ++k)
        if (P->tune_ms[k] > 0.f && P->tune_ms[k] < P->tune_ms[m]) m = k;
    P->trsv_mode = m == 0 ? kTrsvSyncFree : kTrsvCta;
    P->cta_flag = m == 2;
    P->cta_split = m == 3;
    P->cta_merge = m == 4 && P->mfwd.built && P->mbwd.built;
}

npcg_status spmv_run(Handle* h, Pattern* P, const double* A_val, const double* x, double* y) {
    if (P->max_row <= kShortRow) {
        const int blocks = std::max(1, std::min(ceil_div(P->n, 256), h->num_sms * 8));
        k_spmv_rows<<<blocks, 256, 0, h->stream>>>(P->n, P->rp.p, P->ci.p, A_val, x, y);
        NPCG_CUDA(h, cudaGetLastError());
        return NPCG_OK;
    }
    int blocks = std::min(ceil_div(P->n * 8, 256), h->num_sms * 8);
    k_spmv_plain<<<blocks, 256, 0, h->stream>>>(P->n, P->rp.p, P->ci.p, A_val, x, y);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

npcg_status pcg_run(Handle* h, Pattern* P, const double* A_val, const double* b, double* x,
                    int precond, const double* L_val, double rtol, int max_iter,
                    npcg_solve_stats* stats, int stall_k) {
    if (precond < 0 || precond > NPCG_PREC_LLT32) return set_error(h, NPCG_EINVAL, "unknown preconditioner");
    if (precond >= NPCG_PREC_LLT && !L_val) return set_error(h, NPCG_EINVAL, "L_val required for PREC_LLT");
    if (!(rtol >= 0.0)) return set_error(h, NPCG_EINVAL, "rtol must be >= 0");
    if (max_iter < 0) return set_error(h, NPCG_EINVAL, "max_iter must be >= 0");
    NPCG_TRY(ensure_pcg_workspace(h, P));
    const int64_t n = P->n;
    if (A_val != P->Aval_dev.p)
        NPCG_CUDA(h, cudaMemcpyAsync(P->Aval_dev.p, A_val, P->nnz * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    if (b != P->b.p)
        NPCG_CUDA(h, cudaMemcpyAsync(P->b.p, b, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    if (x != P->x.p)
        NPCG_CUDA(h, cudaMemcpyAsync(P->x.p, x, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    if (precond >= NPCG_PREC_LLT) NPCG_TRY(factor_load(h, P, L_val));
    {
        // ctl: n_active, flags, tickets, loop trips, trip bound (2 iterations per trip)
        const int init[6] = {0, 0, 0, 0, 0, max_iter / 2 + 2};
        NPCG_CUDA(h, cudaMemcpyAsync(P->ctl.p, init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
    }
    PcgArgs a = pcg_args(P, precond);
    k_init<<<P->nchunks, kChunkThreads, 0, h->stream>>>(a, rtol, max_iter, P->p0.p, P->p1.p, stall_k);
    if (precond >= NPCG_PREC_LLT) NPCG_TRY(apply_llt(h, h->stream, P, P->nsys > 1, precond == NPCG_PREC_LLT32));
    k_dot_rz<<<P->nchunks, kChunkThreads, 0, h->stream>>>(a, 1);
    NPCG_CUDA(h, cudaGetLastError());
    // the default launches a row-block solve's iterations one by one: with
    // its triangular solves they measured faster than the same kernels in
    // the loop graph, while the graph wins for the other designs and for the
    // elementwise preconditioners
    const bool eager = h->pcg_eager > 0 ||
                       (h->pcg_eager < 0 && precond >= NPCG_PREC_LLT && P->trsv_mode == kTrsvCta &&
                        P->cfwd.built && P->cfwd.blocked);
    if (eager) {
        // the graph body's kernels enqueued one launch at a time, 16
        // iterations between tests of the active count (a system that has
        // stopped makes the kernels of later iterations return at once)
        constexpr int kEagerPairs = 8;
        for (int done = 0; done < max_iter; done += 2 * kEagerPairs) {
            for (int k = 0; k < kEagerPairs; ++k) {
                NPCG_TRY(enqueue_iteration(h, h->stream, P, a, P->p0.p, P->p1.p));
                NPCG_TRY(enqueue_iteration(h, h->stream, P, a, P->p1.p, P->p0.p));
            }
            int ctl2[2] = {0, 0};
            NPCG_CUDA(h, cudaMemcpyAsync(ctl2, P->ctl.p, sizeof(ctl2), cudaMemcpyDeviceToHost, h->stream));
            NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
            if (ctl2[0] <= 0 || (ctl2[1] & kFlagAbort)) break;
        }
    } else {
        NPCG_TRY(build_graph(h, P, precond));
        if (max_iter > 0) NPCG_CUDA(h, cudaGraphLaunch(P->graph[precond], h->stream));
    }
    // stats
    k_stats<<<ceil_div(P->nsys, 128), 128, 0, h->stream>>>(P->nsys, P->st.p, P->stats_dev.p);
    NPCG_CUDA(h, cudaMemcpyAsync(stats, P->stats_dev.p, P->nsys * sizeof(npcg_solve_stats),
                                 cudaMemcpyDeviceToHost, h->stream));
    if (x != P->x.p)
        NPCG_CUDA(h, cudaMemcpyAsync(x, P->x.p, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    int ctl[6] = {0, 0, 0, 0, 0, 0};
    NPCG_CUDA(h, cudaMemcpyAsync(ctl, P->ctl.p, 6 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    if (ctl[1] & (kFlagTimeout | kFlagTripBound)) {
        std::string why = (ctl[1] & kFlagTimeout) ? "triangular solve wait timed out"
                                                  : "iteration loop exceeded its trip bound";
        return set_error(h, NPCG_ETIMEOUT,
                         why + " (trips " + std::to_string(ctl[4]) + ", active systems " +
                             std::to_string(ctl[0]) + ", system 0 iterations " +
                             std::to_string(stats[0].iters) + ", status " + std::to_string(stats[0].status) + ")");
    }
    for (int s = 0; s < P->nsys; ++s)
        if (stats[s].status != NPCG_OK)
            return set_error(h, (npcg_status)stats[s].status,
                             "system " + std::to_string(s) + " did not converge: " +
                                 npcg_status_string((npcg_status)stats[s].status));
    return NPCG_OK;
}

// A factored solve that breaks down, reaches max_iter or stagnates is
// handed to IC(0) (Sec. 5.1's baseline): the factor is recomputed with
// npcg_ic0_factor's kernel and PCG restarts, from the last iterate after
// max_iter or stagnation and from x_0 after a breakdown, with a fresh
// max_iter.  Systems that had converged take no update in the second run.
npcg_status pcg_run_ex(Handle* h, Pattern* P, const double* A_val, const double* b, double* x, int precond,
                       const double* L_val, double rtol, int max_iter, const npcg_solve_opts* opts,
                       npcg_solve_stats* stats) {
    const int stall_k = opts ? std::max(0, (int)opts->stall_iters) : 0;
    const bool fb = opts && opts->fallback_ic0 && precond >= NPCG_PREC_LLT;
    if (fb) {
        NPCG_CUDA(h, P->x0_fb.ensure(P->n));
        NPCG_CUDA(h, cudaMemcpyAsync(P->x0_fb.p, x, P->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    }
    npcg_status st = pcg_run(h, P, A_val, b, x, precond, L_val, rtol, max_iter, stats, stall_k);
    for (int s = 0; s < P->nsys; ++s) {
        stats[s].fallback = 0;
        stats[s].fallback_iters = 0;
    }
    if (!fb || st == NPCG_OK || st == NPCG_ETIMEOUT || st == NPCG_ECUDA || st == NPCG_EINVAL ||
        st == NPCG_ENOMEM)
        return st;
    std::vector<npcg_solve_stats> first(stats, stats + P->nsys);
    bool restart_x0 = false;
    for (int s = 0; s < P->nsys; ++s) restart_x0 |= first[s].status == NPCG_EBREAKDOWN;
    if (restart_x0) {
        // a broken-down system restarts from x_0; the others keep their iterate
        std::vector<double> keep(P->n);
        std::vector<double> x0(P->n);
        NPCG_CUDA(h, cudaMemcpyAsync(keep.data(), x, P->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        NPCG_CUDA(h, cudaMemcpyAsync(x0.data(), P->x0_fb.p, P->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
        for (int s = 0; s < P->nsys; ++s)
            if (first[s].status == NPCG_EBREAKDOWN)
                for (int64_t i = P->sys_ptr_h[s]; i < P->sys_ptr_h[s + 1]; ++i) keep[i] = x0[i];
        NPCG_CUDA(h, cudaMemcpyAsync(x, keep.data(), P->n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    NPCG_CUDA(h, P->Lval_fb.ensure(P->nnzL));
    NPCG_TRY(ic0_run(h, P, A_val, P->Lval_fb.p, nullptr));
    st = pcg_run(h, P, A_val, b, x, precond, P->Lval_fb.p, rtol, max_iter, stats, stall_k);
    for (int s = 0; s < P->nsys; ++s) {
        if (first[s].status == NPCG_OK) {
            stats[s] = first[s];
            stats[s].fallback = 0;
            stats[s].fallback_iters = 0;
        } else {
            stats[s].fallback = 1;
            stats[s].fallback_iters = stats[s].iters;
            stats[s].iters += first[s].iters;
        }
    }
    return st;
}

}  // namespace npcg
