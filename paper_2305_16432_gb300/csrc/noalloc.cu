// Allocation-free solve: plain CG or Jacobi-preconditioned CG on a raw CSR
// matrix, for callers that cannot allocate device memory -- code that runs
// while a custom arena owns all device memory, real-time loops where an
// allocation's latency or failure is not acceptable, and hosts whose
// allocator is reserved by another runtime.  Nothing here calls cudaMalloc,
// cudaFree, or any allocating library routine: the working vectors, the
// per-block partial sums and the solver state live in one file-scope device
// array of fixed size, shared by every call on a device.
#include <mutex>
#include <string>

#include "npcg_internal.cuh"

namespace npcg {
namespace {

constexpr int64_t kNaMaxN = NPCG_NOALLOC_MAX_N;
constexpr int kNaThreads = 256;
constexpr int kNaRows = 512;                                   // rows per block (512 blocks at the largest n)
constexpr int kNaMaxBlocks = (int)((kNaMaxN + kNaRows - 1) / kNaRows);
constexpr int kMaxDevices = 64;

// Layout (doubles): r | z | p | w | 1 / diag(A) (kNaMaxN each) | partials
// (4 per block) | control block (solver state and counters).
constexpr int64_t kOffR = 0, kOffZ = kNaMaxN, kOffP = 2 * kNaMaxN, kOffW = 3 * kNaMaxN, kOffD = 4 * kNaMaxN;
constexpr int64_t kOffPart = 5 * kNaMaxN;
constexpr int64_t kOffCtl = kOffPart + 4 * (int64_t)kNaMaxBlocks;
constexpr int64_t kCtlDoubles = 16;

__device__ __align__(256) double g_noalloc_scratch[kOffCtl + kCtlDoubles];

struct NaState {          // inside the control block
    double tol2, rr, rz, pw, alpha, beta, bnorm2;
    int iters, status, active, max_iter;
    unsigned arrive;
    int bad_diag;         // Jacobi: a row without a nonzero finite diagonal
};
static_assert(sizeof(NaState) <= kCtlDoubles * sizeof(double), "control block too small");

struct NaArgs {
    int n;
    const int32_t* rp;
    const int32_t* ci;
    const double* av;
    const double* b;
    double* x;
    double *r, *z, *p, *w, *dinv, *part;
    NaState* st;
    int jacobi;
    int nblocks;
};

__device__ double na_diag(const NaArgs& a, int row) {
    for (int k = a.rp[row]; k < a.rp[row + 1]; ++k)
        if (a.ci[k] == row) return a.av[k];
    return 0.0;
}

template <int N>
__device__ void na_block_sum(double (&v)[N]) {
    __shared__ double sh[N][kNaThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        double x = v[j];
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[j][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double s = 0.0;
            for (int w = 0; w < kNaThreads / 32; ++w) s += sh[j][w];
            v[j] = s;
        }
}

// thread 0 of the last block to arrive gets true and the block-order sums
template <int N>
__device__ bool na_finish(const NaArgs& a, double (&v)[N]) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        for (int j = 0; j < N; ++j) a.part[4 * blockIdx.x + j] = v[j];
        __threadfence();
        last = atomicAdd(&a.st->arrive, 1u) == (unsigned)(a.nblocks - 1);
    }
    __syncthreads();
    if (threadIdx.x != 0 || !last) return false;
    __threadfence();
    for (int j = 0; j < N; ++j) v[j] = 0.0;
    for (int q = 0; q < a.nblocks; ++q)
        for (int j = 0; j < N; ++j) v[j] += __ldcg(a.part + 4 * q + j);
    a.st->arrive = 0u;
    return true;
}

// r = b - A x, z = M^-1 r, p = z; ||b||^2, ||r||^2, r^T z
__global__ void k_na_init(NaArgs a, double rtol, int max_iter) {
    double acc[3] = {0.0, 0.0, 0.0};
    const int r0 = blockIdx.x * kNaRows, r1 = min(a.n, r0 + kNaRows);
    for (int i = r0 + threadIdx.x; i < r1; i += kNaThreads) {
        double s = 0.0;
        for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) s = fma(a.av[k], a.x[a.ci[k]], s);
        const double bi = a.b[i], ri = bi - s;
        double zi = ri;
        if (a.jacobi) {
            const double d = na_diag(a, i);
            if (!(d != 0.0) || !isfinite(d)) atomicOr(&a.st->bad_diag, 1);
            a.dinv[i] = 1.0 / d;
            zi = ri * a.dinv[i];
        }
        a.r[i] = ri;
        a.z[i] = zi;
        a.p[i] = zi;
        acc[0] = fma(bi, bi, acc[0]);
        acc[1] = fma(ri, ri, acc[1]);
        acc[2] = fma(ri, zi, acc[2]);
    }
    na_block_sum<3>(acc);
    if (na_finish<3>(a, acc)) {
        NaState& s = *a.st;
        s.bnorm2 = acc[0];
        s.tol2 = rtol * rtol * acc[0];
        s.rr = acc[1];
        s.rz = acc[2];
        s.iters = 0;
        s.max_iter = max_iter;
        s.status = NPCG_OK;
        s.active = 0;
        if (s.bad_diag) {
            s.status = NPCG_EINVAL;          // Jacobi needs every diagonal entry
        } else if (!(acc[1] <= s.tol2)) {
            if (max_iter <= 0) s.status = NPCG_EMAXITER;
            else if (!(acc[2] > 0.0) || !isfinite(acc[2])) s.status = NPCG_EBREAKDOWN;
            else s.active = 1;
        }
    }
}

// w = A p; p^T w; alpha
__global__ void k_na_spmv(NaArgs a) {
    if (!a.st->active) return;
    double acc[1] = {0.0};
    const int r0 = blockIdx.x * kNaRows, r1 = min(a.n, r0 + kNaRows);
    for (int i = r0 + threadIdx.x; i < r1; i += kNaThreads) {
        double s = 0.0;
        for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) s = fma(a.av[k], a.p[a.ci[k]], s);
        a.w[i] = s;
        acc[0] = fma(a.p[i], s, acc[0]);
    }
    na_block_sum<1>(acc);
    if (na_finish<1>(a, acc)) {
        NaState& s = *a.st;
        s.pw = acc[0];
        if (!(acc[0] > 0.0) || !isfinite(acc[0])) { s.status = NPCG_EBREAKDOWN; s.active = 0; }
        else s.alpha = s.rz / acc[0];
    }
}

// x += alpha p; r -= alpha w; z = M^-1 r; convergence test; beta
__global__ void k_na_update(NaArgs a) {
    if (!a.st->active) return;
    const double alpha = a.st->alpha;
    double acc[2] = {0.0, 0.0};
    const int r0 = blockIdx.x * kNaRows, r1 = min(a.n, r0 + kNaRows);
    for (int i = r0 + threadIdx.x; i < r1; i += kNaThreads) {
        a.x[i] = fma(alpha, a.p[i], a.x[i]);
        const double ri = fma(-alpha, a.w[i], a.r[i]);
        const double zi = a.jacobi ? ri * a.dinv[i] : ri;
        a.r[i] = ri;
        a.z[i] = zi;
        acc[0] = fma(ri, ri, acc[0]);
        acc[1] = fma(ri, zi, acc[1]);
    }
    na_block_sum<2>(acc);
    if (na_finish<2>(a, acc)) {
        NaState& s = *a.st;
        s.rr = acc[0];
        s.iters += 1;
        if (acc[0] <= s.tol2) { s.active = 0; }
        else if (!isfinite(acc[0])) { s.status = NPCG_EBREAKDOWN; s.active = 0; }
        else if (s.iters >= s.max_iter) { s.status = NPCG_EMAXITER; s.active = 0; }
        else if (!(acc[1] > 0.0) || !isfinite(acc[1])) { s.status = NPCG_EBREAKDOWN; s.active = 0; }
        else { s.beta = acc[1] / s.rz; s.rz = acc[1]; }
    }
}

// p = z + beta p
__global__ void k_na_pupdate(NaArgs a) {
    if (!a.st->active) return;
    const double beta = a.st->beta;
    const int r0 = blockIdx.x * kNaRows, r1 = min(a.n, r0 + kNaRows);
    for (int i = r0 + threadIdx.x; i < r1; i += kNaThreads) a.p[i] = fma(beta, a.p[i], a.z[i]);
}

std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is a stand-in, not a device address).
npcg_status scratch_on_current_device(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NPCG_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return NPCG_ECUDA;
        g_dev_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_dev_ptr[dev];
    return NPCG_OK;
}

}  // namespace
}  // namespace npcg

using namespace npcg;

extern "C" npcg_status npcg_pcg_solve_noalloc(void* stream, int64_t n, int64_t nnz,
                                              const int32_t* row_ptr, const int32_t* col_idx,
                                              const double* A_val, const double* b, double* x,
                                              int32_t precond, double rtol, int32_t max_iter,
                                              npcg_solve_stats* stats) {
    if (n < 1 || n > kNaMaxN || nnz < n || nnz >= (1LL << 31)) return NPCG_EINVAL;
    if (precond != NPCG_PREC_NONE && precond != NPCG_PREC_JACOBI) return NPCG_EINVAL;
    if (!row_ptr || !col_idx || !A_val || !b || !x || !stats || !(rtol >= 0.0) || max_iter < 0)
        return NPCG_EINVAL;
    // an error left by earlier work on this thread is not this call's: report
    // it before launching anything rather than take it for our own later
    if (cudaPeekAtLastError() != cudaSuccess) return NPCG_ECUDA;
    double* base = nullptr;
    npcg_status st = scratch_on_current_device(&base);
    if (st != NPCG_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    NaArgs a;
    a.n = (int)n;
    a.rp = row_ptr;
    a.ci = col_idx;
    a.av = A_val;
    a.b = b;
    a.x = x;
    a.r = base + kOffR;
    a.z = base + kOffZ;
    a.p = base + kOffP;
    a.w = base + kOffW;
    a.dinv = base + kOffD;
    a.part = base + kOffPart;
    a.st = reinterpret_cast<NaState*>(base + kOffCtl);
    a.jacobi = precond == NPCG_PREC_JACOBI;
    a.nblocks = (int)((n + kNaRows - 1) / kNaRows);
    // the array keeps the previous call's contents: the control block (and
    // with it the arrival counter) must start at zero
    if (cudaMemsetAsync(a.st, 0, kCtlDoubles * sizeof(double), s) != cudaSuccess) return NPCG_ECUDA;
    k_na_init<<<a.nblocks, kNaThreads, 0, s>>>(a, rtol, max_iter);
    if (cudaGetLastError() != cudaSuccess) return NPCG_ECUDA;
    NaState hs;
    const int kCheck = 16;           // iterations between host checks
    for (int it = 0; it < max_iter; it += kCheck) {
        for (int k = 0; k < kCheck; ++k) {
            k_na_spmv<<<a.nblocks, kNaThreads, 0, s>>>(a);
            k_na_update<<<a.nblocks, kNaThreads, 0, s>>>(a);
            k_na_pupdate<<<a.nblocks, kNaThreads, 0, s>>>(a);
        }
        if (cudaGetLastError() != cudaSuccess) return NPCG_ECUDA;
        if (cudaMemcpyAsync(&hs, a.st, sizeof(NaState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return NPCG_ECUDA;
        if (!hs.active) break;
    }
    if (cudaGetLastError() != cudaSuccess) return NPCG_ECUDA;
    if (cudaMemcpyAsync(&hs, a.st, sizeof(NaState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return NPCG_ECUDA;
    stats->iters = hs.iters;
    stats->status = hs.status;
    stats->relres = hs.bnorm2 > 0.0 ? sqrt(hs.rr / hs.bnorm2) : sqrt(hs.rr);
    stats->fallback = 0;
    stats->fallback_iters = 0;
    return (npcg_status)hs.status;
}
