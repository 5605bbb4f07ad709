// Internal declarations of the npcg CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/npcg.h"

namespace npcg {

// ---------------------------------------------------------------------------
// limits and launch shapes
// ---------------------------------------------------------------------------
constexpr int kWarp = 32;
constexpr int kSlice = 32;                 // rows per SELL slice = one warp of the solve
constexpr int kChunk = 512;                // fewest rows per reduction chunk (one block)
constexpr int kChunkMax = 4096;            // most rows per reduction chunk
constexpr int kChunkThreads = 256;
constexpr int kShortRow = 16;    // rows up to this length: one thread per row in the SpMV
constexpr long long kSpinLimit = 1LL << 22; // default polls before a device wait gives up (~1-2 s)

// bits of a canonical-free signalling NaN: "value not yet written"
constexpr unsigned long long kSentinelBits = 0x7FF4DEADBEEFCAFEull;
constexpr int kLevelUnset = -1;

// status word flags (device)
enum : int { kFlagTimeout = 1, kFlagBadPattern = 2, kFlagNotSpd = 4, kFlagAbort = 8, kFlagTripBound = 16 };

// ---------------------------------------------------------------------------
// device memory: a typed, owned allocation
// ---------------------------------------------------------------------------
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    cudaError_t alloc(size_t count) {
        release();
        n = count;
        if (count == 0) return cudaSuccess;
        return cudaMalloc(&p, count * sizeof(T));
    }
    // grow-only reuse
    cudaError_t ensure(size_t count) { return count <= n && p ? cudaSuccess : alloc(count); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

struct Handle;

// Per-system PCG state (device).
struct SysState {
    double tol2;      // (rtol ||b||)^2
    double rr;        // ||r||^2
    double rz;        // r^T z (current)
    double pw;        // p^T A p
    double alpha, beta;
    double bnorm2;
    int iters;
    int status;       // npcg_status
    int active;       // 1 while iterating
    int max_iter;
    double best_rr;   // smallest ||r||^2 so far (stagnation test)
    int since_best;   // updates since best_rr last fell
    int stall_k;      // stagnation window (0: off)
};

// Chunk of rows of one system (reductions and vector kernels).
struct Chunk {
    int32_t sys;
    int32_t row0, row1;     // [row0, row1)
    int32_t slot;           // index of this chunk's partial
};

// Level-ordered SELL-32 layout of one triangular factor (off-diagonals only).
struct TriLayout {
    int32_t nslices = 0;
    int32_t nlev = 0;
    DevBuf<int32_t> perm;        // [n] row at each position
    DevBuf<int32_t> level;       // [n] level of each row
    DevBuf<int64_t> slice_off;   // [nslices+1] slot offset of each slice
    DevBuf<int32_t> slice_w;     // [nslices] width
    DevBuf<int32_t> col;         // [slots] column, -1 = padding
    DevBuf<int32_t> src;         // [slots] index into L_val, -1 = padding
    DevBuf<int32_t> diag_src;    // [n by position] index of the diagonal in L_val
    DevBuf<double> val, dinv;    // [slots] factor values, [n by position] 1 / diagonal (FP64)
    DevBuf<float> val32, dinv32; // the same in FP32
    int64_t slots = 0;
};

// Per-system level-synchronous layout of one triangular solve (one CTA per
// system, steps of <= 256 rows of one level, TMA-prefetched).
// consecutive steps of one system moved into one shared-memory stage by
// three bulk copies (structure, values, right-hand side)
struct alignas(16) CtaChunk {
    long long soff;                // structure offset (int32 units)
    long long voff;                // value offset (elements of the value type)
    int q0e;                       // first right-hand-side position copied (16-byte aligned)
    int nsteps;
    unsigned sbytes, vbytes, rbytes;
    int pad;
};

struct CtaLayout {
    bool built = false;
    bool window_ok = false;        // every dependency within the shared window
    bool blocked = false;          // one large system in per-SM row blocks (remote dependencies)
    bool far = false;              // hybrid window: dependencies beyond it read the output (-(pos + 2))
    int nunits = 0;                // CTAs of a solve: systems, or row blocks
    int win_slots = 0;             // window size (power of two) when window_ok
    int nsteps = 0, max_w = 0, max_np = 0;
    int64_t sbuf_len = 0, vbuf_len = 0;
    DevBuf<int32_t> cperm, cpos;   // processing order and its inverse
    DevBuf<int32_t> other;         // backward layout: forward position of the row at each position
    DevBuf<int4> steps;            // {q0, nrows, width, 0}
    DevBuf<int64_t> soff, voff;
    DevBuf<int32_t> sys_step0;
    DevBuf<int32_t> sbuf, vsrc, is_diag, step_of_pos;
    DevBuf<double> vbuf;
    DevBuf<float> vbuf32;
    // per kernel ([0] FP64 and [1] FP32 with a barrier per step, [2] FP32
    // flag-synchronised): chunks, their per-system ranges, stage capacity in
    // bytes and number of ring stages (0: does not fit)
    DevBuf<CtaChunk> chunks[3];
    DevBuf<int32_t> sys_chunk0[3];
    int nchunks[3] = {0, 0, 0};
    int stage_cap[3] = {0, 0, 0};
    int nstages[3] = {0, 0, 0};
    bool flag_ok = false;          // the window also covers the drift of the flag-synchronised kernel
    int split_stages[2] = {0, 0};  // ring stages of the split-role kernel per value type (0: not offered)
};

enum TrsvMode : int { kTrsvAuto = 0, kTrsvSyncFree = 1, kTrsvCta = 2 };

// graph-network feature buffers, grown on demand
struct GnnStore {
    DevBuf<float> v, e, s;         // node / edge features, decoder outputs
    DevBuf<double> sc;             // per-system input scales
    DevBuf<unsigned long long> sckey;  // their running maxima as ordered keys (zero between calls)
    DevBuf<float> aux;             // adjoint scratch
    DevBuf<double> dL;             // adjoint of L (loss)
    DevBuf<double> Lv;             // L values of the current pair
    DevBuf<unsigned short> bf;     // BF16 node / edge features (tensor-core path)
};

// Product structure of L L^T for the Frobenius loss Eq. (loss_A): the
// lower triangle (with diagonal) of pattern(L L^T), per entry the pairs of L
// entries whose product it sums, its A entry, and per L entry the (L entry,
// product entry) pairs of (R L).  Built on first use.
struct FrobLayout {
    bool built = false;
    int64_t nS = 0;
    DevBuf<int32_t> sptr, s2a, srow;      // [nS + 1], [nS], [nS] (srow < 0: off-diagonal entry of row -srow - 1)
    DevBuf<int2> spairs;                  // (a, b): L_a L_b
    DevBuf<int32_t> gptr;                 // [nnzL + 1]
    DevBuf<int2> gpairs;                  // (b, s): R_s L_b
    DevBuf<double> R;                     // [nS]
};

// Merged-level solve of one direction (groups of G levels, see
// level_merge.h): the plan on the device, the level-synchronous layout of
// the pattern of M (unit diagonal), and the numeric M (+ a trailing 1 for the
// diagonal) and C of the loaded factor.
struct MergeDir {
    bool built = false;
    int G = 0;
    int64_t nM = 0, nC = 0;
    CtaLayout lay;
    DevBuf<int64_t> mrp, mtp, mtk, mts, crp, ctp, ctk, cts, diag;
    DevBuf<int32_t> mcol, ccol, ccolpos, prows;
    std::vector<int64_t> pptr;     // host: rows of pass s are prows[pptr[s] .. pptr[s + 1])
    DevBuf<double> M, C;
};

struct Pattern {
    Handle* h = nullptr;
    int64_t n = 0, nnz = 0, nnzL = 0;
    int32_t nsys = 1;
    int32_t max_row = 0;           // longest row of A (entries)
    std::vector<int64_t> sys_ptr_h;
    DevBuf<int64_t> sys_ptr;       // [nsys+1]
    DevBuf<int32_t> row_sys;       // [n] system of each row
    DevBuf<int32_t> rp, ci;        // A pattern copy
    DevBuf<int32_t> edge_row;      // [nnz]
    DevBuf<int32_t> mirror;        // [nnz] position of (j,i)
    DevBuf<int32_t> adiag;         // [n] position of (i,i) in A
    DevBuf<int32_t> a2l;           // [nnz] L position of (i,j), j <= i, else -1
    DevBuf<int32_t> Lrp, Lci, l2a; // tril pattern and L -> A map
    TriLayout fwd, bwd;            // L y = r and L^T z = y
    CtaLayout cfwd, cbwd;          // level-synchronous layouts
    int trsv_mode = kTrsvSyncFree; // chosen by the autotuner
    float tune_ms[5] = {0.f, 0.f, 0.f, 0.f, 0.f}; // measured fwd+bwd time: sync-free, level barrier,
                                                  // level flags, split roles, merged levels
    int merge_G = 0;               // levels per step of the tuned merged-level layouts (0: none)
    int block_units = 0;           // row blocks of a blocked layout (0: one per SM), tuned
    bool cta_flag = false;         // level-ordered solves use the flag-synchronised FP32 kernel
    bool cta_split = false;        // level-ordered solves use the split-role kernel
    DevBuf<double> r_cf, y_cb, yglob;  // rhs in processing order, window backing
    DevBuf<double> yq;             // solution of a level-synchronous solve in processing order
    // reduction chunks
    std::vector<Chunk> chunks_h;
    DevBuf<Chunk> chunks;
    DevBuf<int32_t> sys_chunk0;    // [nsys+1] first chunk of each system
    int32_t nchunks = 0;
    // PCG workspace
    DevBuf<double> x, r, z, y, w, p0, p1, b;
    DevBuf<double> part;           // [nchunks * 4] partial sums
    DevBuf<unsigned int> arrive;   // [nsys] arrival counters
    DevBuf<SysState> st;           // [nsys]
    DevBuf<npcg_solve_stats> stats_dev;  // [nsys]
    DevBuf<int> ctl;               // [0] n_active, [1] flags, [2] fwd ticket, [3] bwd ticket
    DevBuf<double> Aval_dev;       // host-path copy of A values
    DevBuf<double> Lval_dev;       // host-path factor
    DevBuf<double> Lval_fb, x0_fb; // IC(0) fallback: its factor and the first attempt's x_0
    // cached iteration graphs (keyed by precond)
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    int graph_mode[4] = {0, 0, 0, 0};
    long long graph_spin[4] = {0, 0, 0, 0};   // wait limit the graph's launches were captured with
    GnnStore gnn;
    FrobLayout frob;
    MergeDir mfwd, mbwd;           // merged-level solves (built on request)
    bool cta_merge = false;        // level-ordered solves use the merged-level layouts
    ~Pattern();
};

struct Handle {
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;   // private, for graph capture
    int device = 0;
    int num_sms = 0;
    long long spin_limit = kSpinLimit;       // polls before a device wait gives up (npcg_set_wait_limit)
    int pcg_eager = -1;                      // PCG iterations: 1 separate launches, 0 graph, -1 auto (npcg_set_pcg_eager)
    std::string last_error;
    DevBuf<int> scratch_i;      // small device scratch
    void* host_pinned = nullptr; // small pinned host scratch
    size_t host_pinned_bytes = 0;
    std::vector<Pattern*> patterns;   // live patterns analysed with this handle
};

// ---------------------------------------------------------------------------
// error helpers
// ---------------------------------------------------------------------------
npcg_status set_error(Handle* h, npcg_status s, const std::string& msg);
npcg_status cuda_fail(Handle* h, cudaError_t e, const char* where);

#define NPCG_CUDA(h, expr)                                              \
    do {                                                                \
        cudaError_t _e = (expr);                                        \
        if (_e != cudaSuccess) return ::npcg::cuda_fail((h), _e, #expr); \
    } while (0)

#define NPCG_TRY(expr)                         \
    do {                                       \
        npcg_status _s = (expr);               \
        if (_s != NPCG_OK) return _s;          \
    } while (0)

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// device helpers: relaxed / acquire / release accesses at GPU scope
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const void* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const void* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(void* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_u64(void* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_s32(int* p, int v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ double sentinel_f64() { return __longlong_as_double((long long)kSentinelBits); }

// ---------------------------------------------------------------------------
// cross-file host entry points
// ---------------------------------------------------------------------------
npcg_status pattern_build(Handle* h, int64_t n, int64_t nnz, const int32_t* rp,
                          const int32_t* ci, int32_t nsys, const int64_t* sys_ptr, Pattern* P);
npcg_status factor_load(Handle* h, Pattern* P, const double* L_val);
npcg_status sptrsv_run(Handle* h, Pattern* P, int transpose, const double* r, double* y,
                       const int32_t* sys_active);
// the sync-free solve with the first `skip` slices never claimed (failure-path tests)
npcg_status sptrsv_unclaimed_run(Handle* h, Pattern* P, int transpose, int skip, const double* r, double* y);
npcg_status spmv_run(Handle* h, Pattern* P, const double* A_val, const double* x, double* y);
// An arbitrary dependency pattern for cta_layout_build instead of the
// direction's rows of tril(A): host levels and row pointer, device row
// pointer and dependency rows; the value of dependency e is entry e of the
// value array handed to cta_factor_load, the (unit) diagonal entry diag_src.
struct CtaDeps {
    const std::vector<int32_t>* lev;
    const std::vector<int64_t>* drp;
    const int64_t* drp_dev;
    const int32_t* drow_dev;
    int64_t diag_src;
};
npcg_status cta_layout_build(Handle* h, Pattern* P, bool upper, CtaLayout* C, const CtaDeps* dep = nullptr);
npcg_status cta_link(Handle* h, Pattern* P);
int cta_stages(const CtaLayout& C);
void trsv_pick_tuned(Pattern* P);
npcg_status cta_factor_load(Handle* h, CtaLayout* C, const double* L_val);
npcg_status cta_gather(Handle* h, cudaStream_t s, const CtaLayout& C, int64_t n, const double* x, void* xp,
                       bool f32);
npcg_status cta_trsv_launch(Handle* h, cudaStream_t s, Pattern* P, const CtaLayout& C, const void* rhs_perm,
                            void* outq, const SysState* st, bool f32, int* ticket = nullptr,
                            double* pub = nullptr);
npcg_status cta_permute(Handle* h, cudaStream_t s, Pattern* P, const CtaLayout& C, void* outq, bool f32,
                        const int32_t* idx, void* dst, bool dst_f32);
npcg_status trsv_autotune(Handle* h, Pattern* P);
npcg_status sptrsv_timed_run(Handle* h, Pattern* P, int transpose, const double* r, double* y, int reps,
                             double* ms_per_launch, bool f32);
npcg_status pcg_run(Handle* h, Pattern* P, const double* A_val, const double* b, double* x,
                    int precond, const double* L_val, double rtol, int max_iter,
                    npcg_solve_stats* stats, int stall_k = 0);
// PCG with the options of npcg_pcg_solve_ex: stagnation window and the
// IC(0) fallback for a failed factored solve
npcg_status pcg_run_ex(Handle* h, Pattern* P, const double* A_val, const double* b, double* x, int precond,
                       const double* L_val, double rtol, int max_iter, const npcg_solve_opts* opts,
                       npcg_solve_stats* stats);
npcg_status ic0_run(Handle* h, Pattern* P, const double* A_val, double* L_val, double* alpha_out);
npcg_status sgs_run(Handle* h, Pattern* P, const double* A_val, double* L_val);
// merged-level solves (G levels per step): offered to the autotuner and to
// npcg_pattern_set_trsv
constexpr bool kMergeEnabled = true;
constexpr int kMergeLevels = 4;
npcg_status merge_build(Handle* h, Pattern* P, int G);
npcg_status merge_sptrsv(Handle* h, cudaStream_t s, Pattern* P, int transpose, const double* r, double* y, bool f32,
                         cudaEvent_t e0, cudaEvent_t e1);
npcg_status merge_factor_load(Handle* h, Pattern* P, const double* L_val);
npcg_status merge_apply(Handle* h, cudaStream_t s, Pattern* P, bool f32);
npcg_status gnn_forward_run(Handle* h, Pattern* P, const double* A_val, const double* b,
                            const npcg_gnn_config* cfg, const float* w, double* L_val);
npcg_status loss_grad_run(Handle* h, Pattern* P, const double* A_val, int npairs,
                          const double* X, const double* B, const npcg_gnn_config* cfg,
                          const float* w, double* loss_out, float* grad);
npcg_status adam_run(Handle* h, int64_t n, float* w, const float* g, float* m, float* v, int t,
                     float lr, float b1, float b2, float eps);
npcg_status assemble_count_run(Handle* h, const npcg_problem* p, int64_t* n, int64_t* nnz);
npcg_status assemble_run(Handle* h, const npcg_problem* p, int32_t* rp, int32_t* ci, double* v);

// exclusive scan of int32 counts into int32/int64 offsets (device), out[0..n]
npcg_status scan_i32_to_i64(Handle* h, const int32_t* in, int64_t* out, int64_t n);
npcg_status scan_i32_to_i32(Handle* h, const int32_t* in, int32_t* out, int64_t n);
// read a device scalar (synchronises)
template <class T>
npcg_status read_scalar(Handle* h, const T* dev, T* host) {
    NPCG_CUDA(h, cudaMemcpyAsync(host, dev, sizeof(T), cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    return NPCG_OK;
}

}  // namespace npcg

struct npcg_handle_s : npcg::Handle {};
struct npcg_pattern_s : npcg::Pattern {};
