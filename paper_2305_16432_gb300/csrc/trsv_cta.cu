// Level-synchronous sparse triangular solve in one CTA per system, for the
// two solves of "Solve P z = r" (Algorithm 1) with P = L L^T.
//
// The rows of a system are visited level by level (a level's rows depend
// only on earlier levels), split into steps of at most one row per consumer
// thread.  Each step's structure (row ids, dependency positions, header),
// factor values (reciprocal diagonal first) and right-hand side are laid out
// contiguously in processing order.  A producer warp streams them into a
// shared-memory ring with TMA bulk copies (cp.async.bulk), a "full" mbarrier
// per stage completing on the transferred bytes and an "empty" mbarrier per
// stage released by the eight consumer warps.  Solution values of recent
// positions live in a shared-memory window indexed by position, so the only
// synchronisation on the dependency chain is one named barrier among the
// consumer warps per step.  When a dependency reaches further back than the
// window, consumers read the position-ordered global copy (kWindow = false).
// Values (T) are FP64 or FP32; right-hand side and solution stay FP64.
#include <algorithm>
#include <vector>

#include "npcg_internal.cuh"

namespace npcg {

namespace {

constexpr int kCtaRows = 256;            // rows per step = consumer threads per CTA
constexpr int kCtaThreads = kCtaRows + 32;   // + one producer warp
constexpr int kWin = 8192;               // shared window (positions), power of two
constexpr int kMaxStages = 8;
constexpr long long kMbarSpin = 1LL << 22;
constexpr int kHdrInts = 4;              // {q0, nrows, width, pad} heads every structure block

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (long long s = 0; s < kMbarSpin; ++s)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

struct CtaDev {
    const int32_t* sys_step0;   // [nsys+1]
    const int4* steps;          // {q0, nrows, width, 0}
    const int64_t* soff;        // [nsteps] int32 offset of the step's structure block
    const int64_t* voff;        // [nsteps] element offset of the step's value block
    const int32_t* sbuf;        // structure: hdr[4] | row[np] | pos2[np] | dep[w][np]
    const void* vbuf;           // values (T): dinv[np] | val[w][np]
    int max_np, max_w;
    int stages;
};

__host__ __device__ __forceinline__ int pad4(int x) { return (x + 3) & ~3; }
__host__ __device__ __forceinline__ size_t al128(size_t x) { return (x + 127) & ~size_t(127); }

template <class T>
struct StageGeom {
    size_t sb, vb, rb, stage;
    __host__ __device__ StageGeom(int max_np, int max_w) {
        const int np = pad4(max_np);
        sb = al128((size_t)(kHdrInts + (size_t)np * (2 + max_w)) * 4);
        vb = al128((size_t)np * (1 + max_w) * sizeof(T));
        rb = al128((size_t)(np + 4) * 8);
        stage = sb + vb + rb;
    }
};

// right-hand-side copies start on a 16-byte boundary: positions rounded down
// to a multiple of kRhsAl<T> elements
template <class T>
__host__ __device__ constexpr int rhs_align() { return 16 / (int)sizeof(T); }

template <bool kWindow, class T>
__global__ void __launch_bounds__(kCtaThreads) k_trsv_cta(CtaDev D, const T* __restrict__ rhs,
                                                         double* out, T* out2, double* yglob,
                                                         const SysState* st, int* flags) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int sys = blockIdx.x;
    if (st && !st[sys].active) return;
    const int s0 = D.sys_step0[sys], s1 = D.sys_step0[sys + 1];
    if (s0 >= s1) return;
    const int S = D.stages;
    const StageGeom<T> G(D.max_np, D.max_w);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kMaxStages;
    T* win = reinterpret_cast<T*>(smem + 256);
    unsigned char* ring = smem + 256 + (kWindow ? kWin * sizeof(T) : 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCtaRows / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kCtaRows / 32) {
        // ---------------- producer warp: stream the steps through the ring
        // the 32 lanes fetch the descriptors of 32 steps at a time; lane 0 issues
        int issued = 0;
        bool ok = true;
        for (int j0 = s0; j0 < s1 && ok; j0 += 32) {
            int4 dl = make_int4(0, 0, 0, 0);
            long long sol = 0, vol = 0;
            if (j0 + lane < s1) {
                dl = D.steps[j0 + lane];
                sol = D.soff[j0 + lane];
                vol = D.voff[j0 + lane];
            }
            const int cnt = min(32, s1 - j0);
            for (int u = 0; u < cnt; ++u) {
                const int4 d = make_int4(__shfl_sync(0xffffffffu, dl.x, u), __shfl_sync(0xffffffffu, dl.y, u),
                                         __shfl_sync(0xffffffffu, dl.z, u), 0);
                const long long so = __shfl_sync(0xffffffffu, sol, u);
                const long long vo = __shfl_sync(0xffffffffu, vol, u);
                const int j = j0 + u, k = j - s0, s = k % S;
                if (lane == 0) {
                    if (k >= S) {
                        ok = mbar_wait_bounded(&empty[s], (uint32_t)((k / S - 1) & 1));
                        if (ok) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    }
                    if (ok) {
                        const int np = pad4(d.y);
                        const uint32_t sbytes = (uint32_t)(kHdrInts + np * (2 + d.z)) * 4;
                        const uint32_t vbytes = (uint32_t)np * (1 + d.z) * sizeof(T);
                        constexpr int al = rhs_align<T>();
                        const int q0e = d.x & ~(al - 1);
                        const uint32_t rbytes = (uint32_t)(((d.x + d.y - q0e) + al - 1) & ~(al - 1)) * sizeof(T);
                        unsigned char* base = ring + (size_t)s * G.stage;
                        mbar_expect_tx(&full[s], sbytes + vbytes + rbytes);
                        bulk_g2s(base, D.sbuf + so, sbytes, &full[s]);
                        bulk_g2s(base + G.sb, static_cast<const T*>(D.vbuf) + vo, vbytes, &full[s]);
                        bulk_g2s(base + G.sb + G.vb, rhs + q0e, rbytes, &full[s]);
                        ++issued;
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;
            }
        }
        if (lane != 0) return;
        if (!ok) atomicOr(flags, kFlagTimeout | kFlagAbort);
        // copies still in flight complete before this warp (and the CTA) leaves
        for (int j = max(s0, s0 + issued - S); j < s0 + issued; ++j) {
            const int k = j - s0;
            mbar_wait_bounded(&full[k % S], (uint32_t)((k / S) & 1));
        }
        return;
    }

    // ---------------- consumer warps
    for (int i = s0; i < s1; ++i) {
        const int k = i - s0, s = k % S;
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((k / S) & 1));
        const unsigned char* base = ring + (size_t)s * G.stage;
        const int32_t* hdr = reinterpret_cast<const int32_t*>(base);
        const int q0 = hdr[0], nrows = hdr[1], width = hdr[2];
        const int np = pad4(nrows);
        const int32_t* srow = hdr + kHdrInts;
        const int32_t* spos2 = srow + np;
        const int32_t* sdep = spos2 + np;
        const T* sdinv = reinterpret_cast<const T*>(base + G.sb);
        const T* sval = sdinv + np;
        const T* srhs = reinterpret_cast<const T*>(base + G.sb + G.vb) + (q0 & (rhs_align<T>() - 1));
        const int t = threadIdx.x;
        if (ok && t < nrows) {
            T acc = srhs[t];
            if (width <= 4) {
                // common case: issue every dependency load first, then fold in slot order
                int p[4];
                T lv[4], yv[4];
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    p[kk] = kk < width ? sdep[kk * np + t] : -1;
                    lv[kk] = kk < width ? sval[kk * np + t] : (T)0;
                }
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    yv[kk] = p[kk] >= 0 ? (kWindow ? win[p[kk] & (kWin - 1)] : (T)__ldcg(yglob + p[kk])) : (T)0;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    if (p[kk] >= 0) acc = fma(-lv[kk], yv[kk], acc);
            } else {
                for (int kk = 0; kk < width; ++kk) {
                    const int pk = sdep[kk * np + t];
                    if (pk >= 0) {
                        const T yv = kWindow ? win[pk & (kWin - 1)] : (T)__ldcg(yglob + pk);
                        acc = fma(-sval[kk * np + t], yv, acc);
                    }
                }
            }
            const T y = acc * sdinv[t];
            const int q = q0 + t;
            if (kWindow) win[q & (kWin - 1)] = y;
            else yglob[q] = (double)y;
            if (out) out[srow[t]] = (double)y;
            if (out2) out2[spos2[t]] = y;
        }
        // every consumer is done with this step (window writes visible, stage
        // free) and all take the same decision: a thread whose wait gave up
        // must not leave the others at this barrier
        uint32_t all_ok;
        asm volatile(
            "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(all_ok)
            : "r"((uint32_t)ok), "r"(kCtaRows)
            : "memory");
        if (!all_ok) {
            if (threadIdx.x == 0) atomicOr(flags, kFlagTimeout | kFlagAbort);
            return;
        }
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ------------------------------------------------------------ layout build
__global__ void k_cta_fill(int64_t n, const int32_t* cperm, const int32_t* step_of_pos,
                           const int4* steps, const int64_t* soff, const int64_t* voff,
                           const int32_t* cpos, const int32_t* Lrp, const int32_t* Lci,
                           const int32_t* rp, const int32_t* ci, const int32_t* mirror,
                           const int32_t* a2l, int upper, int32_t* sbuf, int32_t* vsrc) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int row = cperm[q];
        const int stp = step_of_pos[q];
        const int4 d = steps[stp];
        const int np = pad4(d.y);
        const int t = (int)(q - d.x);
        int32_t* sb = sbuf + soff[stp];
        int32_t* vs = vsrc + voff[stp];
        if (t == 0) { sb[0] = d.x; sb[1] = d.y; sb[2] = d.z; sb[3] = 0; }
        int32_t* body = sb + kHdrInts;
        body[t] = row;
        body[np + t] = 0;                               // pos2: set by k_cta_pos2
        const int nl = Lrp[row + 1] - Lrp[row];
        int cnt, first;
        if (upper) { cnt = (rp[row + 1] - rp[row]) - nl; first = rp[row + 1] - cnt; }
        else { cnt = nl - 1; first = Lrp[row]; }
        vs[t] = Lrp[row + 1] - 1;                       // diagonal (stored as its reciprocal)
        for (int k = 0; k < d.z; ++k) {
            int dep = -1, src = -1;
            if (k < cnt) {
                if (upper) { dep = cpos[ci[first + k]]; src = a2l[mirror[first + k]]; }
                else { dep = cpos[Lci[first + k]]; src = first + k; }
            }
            body[(2 + k) * np + t] = dep;
            vs[(1 + k) * np + t] = src;
        }
    }
}

__global__ void k_cta_reach(int64_t n, const int32_t* step_of_pos, const int4* steps,
                            const int32_t* level_end, const int32_t* sbuf, const int64_t* soff,
                            unsigned long long* reach) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int stp = step_of_pos[q];
        const int4 d = steps[stp];
        const int np = pad4(d.y);
        const int t = (int)(q - d.x);
        const int32_t* body = sbuf + soff[stp] + kHdrInts;
        for (int k = 0; k < d.z; ++k) {
            int p = body[(2 + k) * np + t];
            if (p >= 0) atomicMax(reach, (unsigned long long)(level_end[stp] - p));
        }
    }
}

__global__ void k_cta_pos2(int64_t n, const int32_t* step_of_pos, const int4* steps, const int64_t* soff,
                           const int32_t* cpos_other, int32_t* sbuf) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int stp = step_of_pos[q];
        const int4 d = steps[stp];
        const int np = pad4(d.y);
        const int t = (int)(q - d.x);
        int32_t* body = sbuf + soff[stp] + kHdrInts;
        body[np + t] = cpos_other[body[t]];
    }
}

// values: reciprocal of the diagonal in the first np slots of every block,
// off-diagonals after; padding gets finite placeholders
__global__ void k_cta_load(int64_t nv, const int32_t* vsrc, const int32_t* is_diag, const double* L,
                           double* v64, float* v32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int s = vsrc[i];
        double v = 0.0;
        if (s >= 0) v = is_diag[i] ? 1.0 / L[s] : L[s];
        v64[i] = v;
        v32[i] = (float)v;
    }
}

__global__ void k_mark_diag(int nsteps, const int4* steps, const int64_t* voff, int32_t* is_diag, int64_t nv) {
    for (int stp = blockIdx.x; stp < nsteps; stp += gridDim.x) {
        const int4 d = steps[stp];
        const int np = pad4(d.y);
        for (int k = threadIdx.x; k < np * (1 + d.z); k += blockDim.x)
            if (voff[stp] + k < nv) is_diag[voff[stp] + k] = k < np ? 1 : 0;
    }
}

template <class T>
__global__ void k_gather_perm(int64_t n, const int32_t* cperm, const double* x, T* xp) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        xp[q] = (T)x[cperm[q]];
}

size_t smem_bytes(const CtaLayout& C, int stages, bool f32) {
    const size_t stage = f32 ? StageGeom<float>(C.max_np, C.max_w).stage : StageGeom<double>(C.max_np, C.max_w).stage;
    const size_t win = C.window_ok ? (size_t)kWin * (f32 ? 4 : 8) : 0;
    return 256 + win + stage * stages;
}

int stages_for(const CtaLayout& C, bool f32) {
    for (int s = kMaxStages; s >= 2; --s)
        if (smem_bytes(C, s, f32) <= 220 * 1024) return s;
    return 0;
}

}  // namespace

// Host: builds the per-system level-synchronous layout of one direction.
// Order: positions sorted by (system, level, row), i.e. the level order of
// each system, systems one after another.
npcg_status cta_layout_build(Handle* h, Pattern* P, bool upper, CtaLayout* C) {
    const int64_t n = P->n;
    const TriLayout& T = upper ? P->bwd : P->fwd;
    std::vector<int32_t> lev(n), rp_h(n + 1), Lrp_h(n + 1);
    NPCG_CUDA(h, cudaMemcpyAsync(lev.data(), T.level.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(rp_h.data(), P->rp.p, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(Lrp_h.data(), P->Lrp.p, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    std::vector<int32_t> cperm(n), cpos(n), step_of_pos(n), sys_step0(P->nsys + 1, 0), level_end;
    std::vector<int4> steps;
    auto offdiag = [&](int row) {
        int nl = Lrp_h[row + 1] - Lrp_h[row];
        return upper ? (rp_h[row + 1] - rp_h[row]) - nl : nl - 1;
    };
    int64_t q = 0;
    int maxw = 0, maxnp = 0;
    for (int s = 0; s < P->nsys; ++s) {
        sys_step0[s] = (int32_t)steps.size();
        const int64_t r0 = P->sys_ptr_h[s], r1 = P->sys_ptr_h[s + 1];
        int nl = 0;
        for (int64_t r = r0; r < r1; ++r) nl = std::max(nl, lev[r] + 1);
        std::vector<int64_t> cnt(nl + 1, 0);
        for (int64_t r = r0; r < r1; ++r) cnt[lev[r] + 1]++;
        for (int l = 0; l < nl; ++l) cnt[l + 1] += cnt[l];
        std::vector<int64_t> fill(cnt.begin(), cnt.end());
        for (int64_t r = r0; r < r1; ++r) cperm[q + fill[lev[r]]++] = (int32_t)r;
        for (int l = 0; l < nl; ++l) {
            const int64_t a = q + cnt[l], b = q + cnt[l + 1];
            for (int64_t c0 = a; c0 < b; c0 += kCtaRows) {
                const int64_t c1 = std::min<int64_t>(b, c0 + kCtaRows);
                int w = 0;
                for (int64_t p = c0; p < c1; ++p) w = std::max(w, offdiag(cperm[p]));
                const int sid = (int)steps.size();
                steps.push_back(make_int4((int)c0, (int)(c1 - c0), w, 0));
                level_end.push_back((int32_t)b);
                for (int64_t p = c0; p < c1; ++p) step_of_pos[p] = sid;
                maxw = std::max(maxw, w);
                maxnp = std::max(maxnp, (int)(c1 - c0));
            }
        }
        q += r1 - r0;
    }
    sys_step0[P->nsys] = (int32_t)steps.size();
    for (int64_t p = 0; p < n; ++p) cpos[cperm[p]] = (int32_t)p;
    const int nsteps = (int)steps.size();
    std::vector<int64_t> soff(nsteps), voff(nsteps);
    int64_t so = 0, vo = 0;
    for (int i = 0; i < nsteps; ++i) {
        const int np = pad4(steps[i].y);
        soff[i] = so;
        voff[i] = vo;
        so += kHdrInts + (int64_t)np * (2 + steps[i].z);
        vo += (int64_t)np * (1 + steps[i].z);
    }
    C->nsteps = nsteps;
    C->max_w = maxw;
    C->max_np = maxnp;
    C->sbuf_len = so;
    C->vbuf_len = vo;
    NPCG_CUDA(h, C->cperm.alloc(n));
    NPCG_CUDA(h, C->cpos.alloc(n));
    NPCG_CUDA(h, C->steps.alloc(nsteps));
    NPCG_CUDA(h, C->soff.alloc(nsteps));
    NPCG_CUDA(h, C->voff.alloc(nsteps));
    NPCG_CUDA(h, C->sys_step0.alloc(P->nsys + 1));
    NPCG_CUDA(h, C->sbuf.alloc(std::max<int64_t>(so, 4)));
    NPCG_CUDA(h, C->vbuf.alloc(std::max<int64_t>(vo, 4)));
    NPCG_CUDA(h, C->vbuf32.alloc(std::max<int64_t>(vo, 4)));
    NPCG_CUDA(h, C->vsrc.alloc(std::max<int64_t>(vo, 4)));
    NPCG_CUDA(h, C->is_diag.alloc(std::max<int64_t>(vo, 4)));
    NPCG_CUDA(h, C->step_of_pos.alloc(n));
    DevBuf<int32_t> lend;
    NPCG_CUDA(h, lend.alloc(nsteps));
    NPCG_CUDA(h, cudaMemcpyAsync(C->cperm.p, cperm.data(), n * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(C->cpos.p, cpos.data(), n * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(C->steps.p, steps.data(), nsteps * sizeof(int4), cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(C->soff.p, soff.data(), nsteps * 8, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(C->voff.p, voff.data(), nsteps * 8, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(C->sys_step0.p, sys_step0.data(), (P->nsys + 1) * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(C->step_of_pos.p, step_of_pos.data(), n * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(lend.p, level_end.data(), nsteps * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemsetAsync(C->sbuf.p, 0, C->sbuf.n * 4, h->stream));
    NPCG_CUDA(h, cudaMemsetAsync(C->vsrc.p, 0xff, C->vsrc.n * 4, h->stream));
    const int blocks = std::max(1, std::min(ceil_div(n, 256), h->num_sms * 8));
    k_cta_fill<<<blocks, 256, 0, h->stream>>>(n, C->cperm.p, C->step_of_pos.p, C->steps.p, C->soff.p,
                                              C->voff.p, C->cpos.p, P->Lrp.p, P->Lci.p, P->rp.p, P->ci.p,
                                              P->mirror.p, P->a2l.p, upper ? 1 : 0, C->sbuf.p, C->vsrc.p);
    k_mark_diag<<<std::max(1, std::min(nsteps, h->num_sms * 8)), 256, 0, h->stream>>>(
        nsteps, C->steps.p, C->voff.p, C->is_diag.p, vo);
    NPCG_CUDA(h, cudaGetLastError());
    DevBuf<unsigned long long> reach;
    NPCG_CUDA(h, reach.alloc(1));
    NPCG_CUDA(h, cudaMemsetAsync(reach.p, 0, 8, h->stream));
    k_cta_reach<<<blocks, 256, 0, h->stream>>>(n, C->step_of_pos.p, C->steps.p, lend.p, C->sbuf.p,
                                               C->soff.p, reach.p);
    NPCG_CUDA(h, cudaGetLastError());
    unsigned long long rh = 0;
    NPCG_TRY(read_scalar(h, reach.p, &rh));
    C->window_ok = rh <= (unsigned long long)kWin;
    // the launch size never exceeds 220 KB; set once here, outside any capture
    const int mx = 220 * 1024;
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    C->built = true;
    return NPCG_OK;
}

// forward records carry the backward position of their row (the forward
// solve writes y straight into the backward solve's processing order)
npcg_status cta_link(Handle* h, Pattern* P) {
    const int blocks = std::max(1, std::min(ceil_div(P->n, 256), h->num_sms * 8));
    k_cta_pos2<<<blocks, 256, 0, h->stream>>>(P->n, P->cfwd.step_of_pos.p, P->cfwd.steps.p, P->cfwd.soff.p,
                                              P->cbwd.cpos.p, P->cfwd.sbuf.p);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

int cta_stages(const CtaLayout& C) { return std::min(stages_for(C, false), stages_for(C, true)); }

npcg_status cta_factor_load(Handle* h, CtaLayout* C, const double* L_val) {
    const int blocks = std::max(1, std::min(ceil_div(C->vbuf_len, 256), h->num_sms * 8));
    k_cta_load<<<blocks, 256, 0, h->stream>>>(C->vbuf_len, C->vsrc.p, C->is_diag.p, L_val, C->vbuf.p, C->vbuf32.p);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

npcg_status cta_gather(Handle* h, cudaStream_t s, const CtaLayout& C, int64_t n, const double* x, void* xp,
                       bool f32) {
    const int blocks = std::max(1, std::min(ceil_div(n, 256), h->num_sms * 8));
    if (f32) k_gather_perm<float><<<blocks, 256, 0, s>>>(n, C.cperm.p, x, static_cast<float*>(xp));
    else k_gather_perm<double><<<blocks, 256, 0, s>>>(n, C.cperm.p, x, static_cast<double*>(xp));
    return NPCG_OK;
}

// rhs_perm: right-hand side in this direction's processing order (n + 4
// entries of the value type, the last ones padding); out (natural order,
// FP64) and/or out2 (positions of the other direction, value type) receive
// the solution.  f32: FP32 factor, arithmetic, right-hand side and out2.
npcg_status cta_trsv_launch(Handle* h, cudaStream_t s, Pattern* P, const CtaLayout& C, const void* rhs_v,
                            double* out, void* out2_v, const SysState* st, bool f32) {
    const int stages = stages_for(C, f32);
    if (stages < 2) return set_error(h, NPCG_EINVAL, "level-synchronous layout does not fit shared memory");
    CtaDev d;
    d.sys_step0 = C.sys_step0.p;
    d.steps = C.steps.p;
    d.soff = C.soff.p;
    d.voff = C.voff.p;
    d.sbuf = C.sbuf.p;
    d.vbuf = f32 ? (const void*)C.vbuf32.p : (const void*)C.vbuf.p;
    d.max_np = C.max_np;
    d.max_w = C.max_w;
    d.stages = stages;
    const size_t smem = smem_bytes(C, stages, f32);
    int* flags = P->ctl.p + 1;
    if (f32) {
        const float* rp = static_cast<const float*>(rhs_v);
        float* o2 = static_cast<float*>(out2_v);
        if (C.window_ok) k_trsv_cta<true, float><<<P->nsys, kCtaThreads, smem, s>>>(d, rp, out, o2, nullptr, st, flags);
        else k_trsv_cta<false, float><<<P->nsys, kCtaThreads, smem, s>>>(d, rp, out, o2, P->yglob.p, st, flags);
    } else {
        const double* rp = static_cast<const double*>(rhs_v);
        double* o2 = static_cast<double*>(out2_v);
        if (C.window_ok) k_trsv_cta<true, double><<<P->nsys, kCtaThreads, smem, s>>>(d, rp, out, o2, nullptr, st, flags);
        else k_trsv_cta<false, double><<<P->nsys, kCtaThreads, smem, s>>>(d, rp, out, o2, P->yglob.p, st, flags);
    }
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

}  // namespace npcg
