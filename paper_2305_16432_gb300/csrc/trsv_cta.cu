// Level-synchronous sparse triangular solve in one CTA per system, for the
// two solves of "Solve P z = r" (Algorithm 1) with P = L L^T.
//
// The rows of a system are visited level by level (a level's rows depend
// only on earlier levels), split into steps of at most one row per consumer
// thread.  Each step's structure (row ids, dependency positions, header),
// factor values (reciprocal diagonal first) and right-hand side are laid out
// contiguously in processing order.  Consecutive steps are grouped into
// chunks that fill one shared-memory stage; a producer warp streams the
// chunks into a ring of stages with three TMA bulk copies each
// (cp.async.bulk), a "full" mbarrier per stage completing on the transferred
// bytes and an "empty" mbarrier per stage released by the eight consumer
// warps.  Chunking keeps many small steps in flight, so the copy latency is
// hidden behind the dependency chain rather than paid every few steps.
// Solution values of recent positions live in a shared-memory window indexed
// by position, so the only synchronisation on the dependency chain is one
// named barrier among the consumer warps per step.  When a dependency reaches
// further back than the window, consumers read the position-ordered global
// copy (kWindow = false).  Values (T) are FP64 or FP32.
#include <algorithm>
#include <vector>

#include "npcg_internal.cuh"

namespace npcg {

namespace {

constexpr int kCtaRows = 256;            // rows per step = consumer threads per CTA
constexpr int kCtaThreads = kCtaRows + 32;   // + one producer warp
constexpr int kWinMax = 8192;            // largest shared window (positions), power of two
constexpr int kWinMin = 1024;            // smallest window
constexpr int kMaxStages = 8;
constexpr int kHdrInts = 4;              // {q0, nrows, width, pad} heads every structure block
constexpr int kRec = 4;                  // dependencies held in a row's packed record
constexpr int kWinPad = 32;              // window slots past the window; the first stays zero
constexpr int64_t kBlockedRows = 1 << 18;  // one system this large is split into per-SM row blocks

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
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    for (long long s = 0; s < limit; ++s)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

struct CtaDev {
    const int32_t* sys_chunk0;  // [nsys+1]
    const CtaChunk* chunks;
    const int32_t* sbuf;        // structure: hdr[4] | row[np] | pos2[np] | dep[w][np] per step
    const void* vbuf;           // values (T): dinv[np] | val[w][np] per step
    int stages;
    int stage_cap;              // bytes per stage (multiple of 128)
    int win;                    // window slots (power of two)
    long long spin;             // polls before a wait gives up (the handle's wait limit)
};

__host__ __device__ __forceinline__ int pad4(int x) { return (x + 3) & ~3; }
__host__ __device__ __forceinline__ int n_extra(int w) { return w > kRec ? w - kRec : 0; }
// Step blocks, np = nrows rounded up to 4.  Structure (int32):
//   hdr[4] | dep[np][4] | {row, pos2}[np] | extra dep[n_extra][np]
// dep holds processing positions (window slots once the window is known to
// suffice: position mod W, a missing dependency -> the zero slot W, where W
// is the window size, the smallest power of two >= max(kWinMin, reach);
// otherwise absolute positions, -1 when missing).  Values (T):
//   l[np][4] | 1/diag[np] | extra l[n_extra][np]
__host__ __device__ __forceinline__ int s_ints(int np, int w) { return kHdrInts + np * (6 + n_extra(w)); }
__host__ __device__ __forceinline__ int v_elems(int np, int w) { return np * (5 + n_extra(w)); }

// right-hand-side copies start on a 16-byte boundary: positions rounded down
// to a multiple of rhs_align<T>() elements
template <class T>
__host__ __device__ constexpr int rhs_align() { return 16 / (int)sizeof(T); }

// barrier + mbarrier area at the start of shared memory: full[8], empty[8],
// and per stage the chunk's {nsteps, value offset, rhs offset, q0e}
constexpr int kBarBytes = 512;           // + the claimed unit (blocked layouts) at byte 256

// operands of one row of one step, held in registers by its consumer thread
template <class T>
struct StepOps {
    int q0, nrows, width, np;
    int4 dep;
    int row;
    T l[4];
    T rhs, dinv;
};

__device__ __forceinline__ void ld_vec4(float (&l)[4], const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    l[0] = v.x; l[1] = v.y; l[2] = v.z; l[3] = v.w;
}
__device__ __forceinline__ void ld_vec4(double (&l)[4], const double* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    l[0] = a.x; l[1] = a.y; l[2] = b.x; l[3] = b.y;
}

template <bool kRow, class T>
__device__ __forceinline__ void load_step(StepOps<T>& o, const int32_t* hdr, const T* vals, const T* rh, int q0e,
                                          int t) {
    const int4 h = *reinterpret_cast<const int4*>(hdr);
    o.q0 = h.x;
    o.nrows = h.y;
    o.width = h.z;
    o.np = pad4(h.y);
    if (t < o.nrows) {
        o.dep = reinterpret_cast<const int4*>(hdr + kHdrInts)[t];
        if (kRow) o.row = reinterpret_cast<const int2*>(hdr + kHdrInts + 4 * o.np)[t].x;
        ld_vec4(o.l, vals + 4 * t);
        o.dinv = vals[4 * o.np + t];
        o.rhs = rh[o.q0 - q0e + t];
    }
}

// named barrier 1 among the consumer threads, returning whether every
// consumer passed ok (all take the same decision)
__device__ __forceinline__ bool consumers_agree(bool ok) {
    uint32_t all_ok;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(all_ok)
        : "r"((uint32_t)ok), "r"(kCtaRows)
        : "memory");
    return all_ok != 0;
}

// value of a dependency on a row of an earlier unit (blocked layouts): the
// unit that owns it publishes it to pub (FP64, sentinel until written)
__device__ __forceinline__ double remote_dep(const double* pub, int row, int* flags, long long limit) {
    long long spins = 0;
    unsigned long long bits;
    while ((bits = ld_relaxed_u64(pub + row)) == kSentinelBits) {
        // a solve that already gave up does not wait again
        if ((++spins & 255) == 0 && (ld_relaxed_s32(flags) & kFlagAbort)) return 0.0;
        if (spins > limit) {
            atomicOr(flags, kFlagTimeout | kFlagAbort);
            return 0.0;
        }
    }
    return __longlong_as_double((long long)bits);
}

// Producer warp: streams the system's chunks through the ring of stages.
// The 32 lanes fetch 32 chunk descriptors at a time; lane 0 issues the three
// bulk copies of a chunk once every consumer warp has released the stage.
// Copies still in flight complete before the warp leaves.
template <class T>
__device__ __forceinline__ void ring_producer(const CtaDev& D, const T* rhs, unsigned char* ring, uint64_t* full,
                                              uint64_t* empty, int4* info, int c0, int c1, int* flags) {
    const int S = D.stages, lane = threadIdx.x & 31;
    int issued = 0;
    bool ok = true;
    for (int j0 = c0; j0 < c1 && ok; j0 += 32) {
        CtaChunk cl{};
        if (j0 + lane < c1) cl = D.chunks[j0 + lane];
        const int cnt = min(32, c1 - j0);
        for (int u = 0; u < cnt; ++u) {
            const long long so = __shfl_sync(0xffffffffu, cl.soff, u);
            const long long vo = __shfl_sync(0xffffffffu, cl.voff, u);
            const int q0e = __shfl_sync(0xffffffffu, cl.q0e, u);
            const int nst = __shfl_sync(0xffffffffu, cl.nsteps, u);
            const unsigned sb = __shfl_sync(0xffffffffu, cl.sbytes, u);
            const unsigned vb = __shfl_sync(0xffffffffu, cl.vbytes, u);
            const unsigned rb = __shfl_sync(0xffffffffu, cl.rbytes, u);
            const int j = j0 + u, k = j - c0, s = k % S;
            if (lane == 0) {
                if (k >= S) {
                    ok = mbar_wait_bounded(&empty[s], (uint32_t)((k / S - 1) & 1), D.spin);
                    if (ok) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                }
                if (ok) {
                    unsigned char* base = ring + (size_t)s * D.stage_cap;
                    // read by the consumers after the phase completes
                    // (the arrive below releases this store)
                    info[s] = make_int4(nst, (int)sb, (int)(sb + vb), q0e);
                    mbar_expect_tx(&full[s], sb + vb + rb);
                    bulk_g2s(base, D.sbuf + so, sb, &full[s]);
                    bulk_g2s(base + sb, static_cast<const T*>(D.vbuf) + vo, vb, &full[s]);
                    bulk_g2s(base + sb + vb, rhs + q0e, rb, &full[s]);
                    ++issued;
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
        }
    }
    if (lane != 0) return;
    if (!ok) atomicOr(flags, kFlagTimeout | kFlagAbort);
    for (int j = max(c0, c0 + issued - S); j < c0 + issued; ++j) {
        const int k = j - c0;
        mbar_wait_bounded(&full[k % S], (uint32_t)((k / S) & 1), D.spin);
    }
}

// kRemote: blocked layout of one large system.  CTAs claim units (contiguous
// row blocks) in dependency order from a ticket, so every unit a CTA polls
// on is owned by a CTA that is already running; dependencies outside the
// unit are encoded -(row + 2) and read from pub, and every row's value is
// published there.
// kFar: hybrid window; a dependency encoded -(position + 2) lies beyond the
// window and is read from the processing-order output (written in an earlier
// step, before a consumer barrier).
template <bool kWindow, bool kRemote, bool kFar, class T>
__global__ void __launch_bounds__(kCtaThreads, 1) k_trsv_cta(CtaDev D, const T* __restrict__ rhs,
                                                         T* outq, double* yglob,
                                                         const SysState* st, int* flags,
                                                         int* ticket, double* pub) {
    extern __shared__ __align__(128) unsigned char smem[];
    int sys = blockIdx.x;
    if (kRemote) {
        int* s_unit = reinterpret_cast<int*>(smem + 256);
        if (threadIdx.x == 0) *s_unit = atomicAdd(ticket, 1);
        __syncthreads();
        sys = *s_unit;
        if (st && !st[0].active) return;
    } else if (st && !st[sys].active) {
        return;
    }
    const int c0 = D.sys_chunk0[sys], c1 = D.sys_chunk0[sys + 1];
    if (c0 >= c1) return;
    const int S = D.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kMaxStages;
    int4* info = reinterpret_cast<int4*>(empty + kMaxStages);
    T* win = reinterpret_cast<T*>(smem + kBarBytes);
    const int W = D.win;
    unsigned char* ring = smem + kBarBytes + (kWindow ? (size_t)(W + kWinPad) * sizeof(T) : 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCtaRows / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (kWindow && threadIdx.x < kWinPad) win[W + threadIdx.x] = (T)0;
    __syncthreads();

    if (warp == kCtaRows / 32) {
        ring_producer<T>(D, rhs, ring, full, empty, info, c0, c1, flags);
        return;
    }

    // ---------------- consumer warps
    // Software pipeline: the operands of the next step (structure, values,
    // right-hand side: nothing that depends on solution values) are loaded
    // into registers before the current step computes, so only the window
    // loads, the multiply-adds and the barrier sit on the dependency chain.
    const int t = threadIdx.x;
    StepOps<T> cur, nxt;
    int c = c0, s = 0, u = 0, nst;
    const int32_t* hdr;
    const T* vals;
    const T* rh;
    int q0e;
    {
        const bool ok = mbar_wait_bounded(&full[0], 0u, D.spin);
        if (!consumers_agree(ok)) {
            if (threadIdx.x == 0) atomicOr(flags, kFlagTimeout | kFlagAbort);
            return;
        }
        const int4 inf = info[0];
        nst = inf.x;
        hdr = reinterpret_cast<const int32_t*>(ring);
        vals = reinterpret_cast<const T*>(ring + inf.y);
        rh = reinterpret_cast<const T*>(ring + inf.z);
        q0e = inf.w;
        load_step<kRemote>(cur, hdr, vals, rh, q0e, t);
    }
    for (;;) {
        // the current step's window reads are issued first: their latency
        // overlaps the bookkeeping and the next step's operand loads (the
        // warp issues in order)
        T yw0 = (T)0, yw1 = (T)0, yw2 = (T)0, yw3 = (T)0;
        // row blocks: the step's remote values (published by earlier blocks)
        // and local ones (window, or the global solution) are all requested
        // here, so the L2 round trip of the remote ones overlaps the
        // bookkeeping below; a remote value not yet published is polled for
        // when it is used
        unsigned long long rq[4] = {0ull, 0ull, 0ull, 0ull};
        T yl[4] = {(T)0, (T)0, (T)0, (T)0};
        if (kRemote && t < cur.nrows) {
            const int pd[4] = {cur.dep.x, cur.dep.y, cur.dep.z, cur.dep.w};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                if (pd[kk] <= -2) {
                    rq[kk] = ld_relaxed_u64(pub + (-pd[kk] - 2));
                } else if (kWindow) {
                    yl[kk] = win[pd[kk]];
                } else if (pd[kk] >= 0) {
                    yl[kk] = (T)__ldcg(yglob + pd[kk]);
                }
            }
        }
        if (kWindow && !kRemote && t < cur.nrows) {
            if (kFar) {
                yw0 = cur.dep.x >= 0 ? win[cur.dep.x] : __ldcg(outq + (-cur.dep.x - 2));
                yw1 = cur.dep.y >= 0 ? win[cur.dep.y] : __ldcg(outq + (-cur.dep.y - 2));
                yw2 = cur.dep.z >= 0 ? win[cur.dep.z] : __ldcg(outq + (-cur.dep.z - 2));
                yw3 = cur.dep.w >= 0 ? win[cur.dep.w] : __ldcg(outq + (-cur.dep.w - 2));
            } else {
                yw0 = win[cur.dep.x];
                yw1 = win[cur.dep.y];
                yw2 = win[cur.dep.z];
                yw3 = win[cur.dep.w];
            }
        }
        // locate and load the next step
        const int32_t* chdr = hdr;          // the current step, for rows wider than the registers
        const T* cvals = vals;
        bool has_next = true, waited = false, ok = true;
        int nc = c, ns = s, nu = u + 1, nnst = nst;
        if (u + 1 < nst) {
            hdr += s_ints(cur.np, cur.width);
            vals += v_elems(cur.np, cur.width);
        } else if (c + 1 < c1) {
            nc = c + 1;
            ns = (nc - c0) % S;
            nu = 0;
            waited = true;
            ok = mbar_wait_bounded(&full[ns], (uint32_t)(((nc - c0) / S) & 1), D.spin);
            if (ok) {
                const int4 inf = info[ns];
                const unsigned char* base = ring + (size_t)ns * D.stage_cap;
                nnst = inf.x;
                hdr = reinterpret_cast<const int32_t*>(base);
                vals = reinterpret_cast<const T*>(base + inf.y);
                rh = reinterpret_cast<const T*>(base + inf.z);
                q0e = inf.w;
            }
        } else {
            has_next = false;
        }
        if (has_next && ok) load_step<kRemote>(nxt, hdr, vals, rh, q0e, t);
        // the current step
        if (t < cur.nrows) {
            T acc = cur.rhs;
            if (kWindow && !kRemote) {
                // missing dependencies read the zero slot with a zero value
                acc = fma(-cur.l[0], yw0, acc);
                acc = fma(-cur.l[1], yw1, acc);
                acc = fma(-cur.l[2], yw2, acc);
                acc = fma(-cur.l[3], yw3, acc);
            } else {
                const int pd[4] = {cur.dep.x, cur.dep.y, cur.dep.z, cur.dep.w};
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const int p = pd[kk];
                    if (kRemote && p <= -2) {
                        const double yv = rq[kk] != kSentinelBits ? __longlong_as_double((long long)rq[kk])
                                                                  : remote_dep(pub, -p - 2, flags, D.spin);
                        acc = fma(-cur.l[kk], (T)yv, acc);
                    } else if (kRemote) {
                        acc = fma(-cur.l[kk], yl[kk], acc);   // zero for a missing dependency
                    } else if (kWindow) {
                        acc = fma(-cur.l[kk], win[p], acc);
                    } else if (p >= 0) {
                        acc = fma(-cur.l[kk], (T)__ldcg(yglob + p), acc);
                    }
                }
            }
            if (cur.width > kRec) {
                const int32_t* xdep = chdr + kHdrInts + 6 * cur.np;
                const T* xval = cvals + 5 * cur.np;
                for (int k0 = 0; k0 < cur.width - kRec; k0 += 4) {
                    const int kn = min(4, cur.width - kRec - k0);
                    int pk[4];
                    unsigned long long rb[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        pk[j] = j < kn ? xdep[(k0 + j) * cur.np + t] : -1;
                        if (kRemote && pk[j] <= -2) rb[j] = ld_relaxed_u64(pub + (-pk[j] - 2));
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (j >= kn) break;
                        const T lv = xval[(k0 + j) * cur.np + t];
                        const int q = pk[j];
                        if (kRemote && q <= -2) {
                            const double yv = rb[j] != kSentinelBits ? __longlong_as_double((long long)rb[j])
                                                                     : remote_dep(pub, -q - 2, flags, D.spin);
                            acc = fma(-lv, (T)yv, acc);
                        } else if (kFar && q <= -2) {
                            acc = fma(-lv, __ldcg(outq + (-q - 2)), acc);
                        } else if (kWindow) {
                            acc = fma(-lv, win[q], acc);
                        } else if (q >= 0) {
                            acc = fma(-lv, (T)__ldcg(yglob + q), acc);
                        }
                    }
                }
            }
            const T y = acc * cur.dinv;
            const int q = cur.q0 + t;
            // the solution in processing order (coalesced); a gather moves it
            // to the order its reader needs
            if (kWindow) {
                win[q & (W - 1)] = y;
                outq[q] = y;
                if (kFar) __threadfence_block();
            } else {
                yglob[q] = (double)y;
            }
            if (kRemote) st_relaxed_u64(pub + cur.row, (unsigned long long)__double_as_longlong((double)y));
        }
        if (!kWindow) __threadfence_block();
        // this step's solutions are visible to the next step; a next chunk
        // is used only if every consumer's wait for it succeeded
        if (waited) {
            if (!consumers_agree(ok)) {
                if (threadIdx.x == 0) atomicOr(flags, kFlagTimeout | kFlagAbort);
                return;
            }
        } else {
            asm volatile("bar.sync 1, %0;" ::"r"(kCtaRows) : "memory");
        }
        if (u + 1 == nst && lane == 0) mbar_arrive(&empty[s]);   // chunk c fully read
        if (!has_next) break;
        cur = nxt;
        c = nc;
        s = ns;
        u = nu;
        nst = nnst;
    }
}

// ------------------------------------------------------------ split-role variant
// The same layout, ring and window, with the two instruction streams of a
// step on different warps: eight operand warps walk the step headers and
// stage step k+1's operands (dependency slots, factor values, reciprocal
// diagonal, right-hand side) into a double-buffered shared-memory slot while
// eight compute warps solve step k from the slot staged during step k-1.
// One named barrier per step (with the AND of the operand warps' waits)
// separates the steps; a compute warp's step is then five independent slot
// loads, the window loads, four FMAs and the stores.  Chunks are released
// by the compute warps once the last step of a chunk is solved (its extra
// dependencies are read from the ring during that step).
constexpr int kSplitThreads = 2 * kCtaRows + 32;
constexpr int kMetaInts = 8;   // {nrows, q0, np, width, header offset, values offset, release stage, last}

template <class T>
__host__ __device__ constexpr size_t split_staging_bytes() {
    return 2 * (size_t)kCtaRows * (16 + 6 * sizeof(T)) + 128;
}

// named barrier 1 among the compute and operand warps, returning the AND of ok
__device__ __forceinline__ bool split_agree(bool ok) {
    uint32_t all_ok;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(all_ok)
        : "r"((uint32_t)ok), "r"(2 * kCtaRows)
        : "memory");
    return all_ok != 0;
}

__device__ __forceinline__ void st_vec4(float* p, const float (&l)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(l[0], l[1], l[2], l[3]);
}
__device__ __forceinline__ void st_vec4(double* p, const double (&l)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(l[0], l[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(l[2], l[3]);
}

template <bool kFar, class T>
__global__ void __launch_bounds__(kSplitThreads, 1) k_trsv_split(CtaDev D, const T* __restrict__ rhs, T* outq,
                                                                 const SysState* st, int* flags) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int sys = blockIdx.x;
    if (st && !st[sys].active) return;
    const int c0 = D.sys_chunk0[sys], c1 = D.sys_chunk0[sys + 1];
    if (c0 >= c1) return;
    const int S = D.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kMaxStages;
    int4* info = reinterpret_cast<int4*>(empty + kMaxStages);
    T* win = reinterpret_cast<T*>(smem + kBarBytes);
    const int W = D.win;
    unsigned char* stg = smem + kBarBytes + (size_t)(W + kWinPad) * sizeof(T);
    int4* s_dep = reinterpret_cast<int4*>(stg);                          // [2][kCtaRows]
    T* s_l = reinterpret_cast<T*>(stg + 2 * kCtaRows * 16);               // [2][kCtaRows][4]
    T* s_dinv = s_l + 2 * kCtaRows * 4;                                   // [2][kCtaRows]
    T* s_rhs = s_dinv + 2 * kCtaRows;                                     // [2][kCtaRows]
    int* s_meta = reinterpret_cast<int*>(s_rhs + 2 * kCtaRows);           // [2][kMetaInts]
    unsigned char* ring = stg + split_staging_bytes<T>();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCtaRows / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < kWinPad) win[W + threadIdx.x] = (T)0;
    __syncthreads();

    if (warp == 2 * kCtaRows / 32) {
        ring_producer<T>(D, rhs, ring, full, empty, info, c0, c1, flags);
        return;
    }

    if (threadIdx.x >= kCtaRows) {
        // ---------------- operand warps: stage step j during step j - 1
        const int t2 = threadIdx.x - kCtaRows;
        bool ok = mbar_wait_bounded(&full[0], 0u, D.spin);
        int c = c0, s = 0, u = 0, nst = 0, q0e = 0;
        const int32_t* hdr = nullptr;
        const T* vals = nullptr;
        const T* rh = nullptr;
        if (ok) {
            const int4 inf = info[0];
            nst = inf.x;
            hdr = reinterpret_cast<const int32_t*>(ring);
            vals = reinterpret_cast<const T*>(ring + inf.y);
            rh = reinterpret_cast<const T*>(ring + inf.z);
            q0e = inf.w;
        }
        bool have = true;
        for (int j = 0;; ++j) {
            const bool prep = have;
            if (prep && ok) {
                const int sl = j & 1;
                const int4 h = *reinterpret_cast<const int4*>(hdr);
                const int nrows = h.y, np = pad4(h.y), width = h.z;
                if (t2 < nrows) {
                    s_dep[sl * kCtaRows + t2] = reinterpret_cast<const int4*>(hdr + kHdrInts)[t2];
                    T l[4];
                    ld_vec4(l, vals + 4 * t2);
                    st_vec4(s_l + 4 * (sl * kCtaRows + t2), l);
                    s_dinv[sl * kCtaRows + t2] = vals[4 * np + t2];
                    s_rhs[sl * kCtaRows + t2] = rh[h.x - q0e + t2];
                }
                const bool chunk_end = u + 1 == nst;
                if (t2 == 0) {
                    int* m = s_meta + sl * kMetaInts;
                    m[0] = nrows;
                    m[1] = h.x;
                    m[2] = np;
                    m[3] = width;
                    m[4] = (int)(reinterpret_cast<const unsigned char*>(hdr) - ring);
                    m[5] = (int)(reinterpret_cast<const unsigned char*>(vals) - ring);
                    m[6] = chunk_end ? s : -1;
                    m[7] = chunk_end && c + 1 == c1;
                }
                // advance to the next step
                if (!chunk_end) {
                    hdr += s_ints(np, width);
                    vals += v_elems(np, width);
                    ++u;
                } else if (c + 1 < c1) {
                    ++c;
                    s = (c - c0) % S;
                    u = 0;
                    ok = mbar_wait_bounded(&full[s], (uint32_t)(((c - c0) / S) & 1), D.spin);
                    if (ok) {
                        const int4 inf = info[s];
                        const unsigned char* base = ring + (size_t)s * D.stage_cap;
                        nst = inf.x;
                        hdr = reinterpret_cast<const int32_t*>(base);
                        vals = reinterpret_cast<const T*>(base + inf.y);
                        rh = reinterpret_cast<const T*>(base + inf.z);
                        q0e = inf.w;
                    }
                } else {
                    have = false;
                }
            }
            if (!split_agree(ok)) {
                if (t2 == 0) atomicOr(flags, kFlagTimeout | kFlagAbort);
                return;
            }
            if (!prep) break;
        }
        return;
    }

    // ---------------- compute warps: solve step k from slot k & 1
    const int t = threadIdx.x;
    if (!split_agree(true)) return;
    for (int k = 0;; ++k) {
        const int sl = k & 1;
        const int* m = s_meta + sl * kMetaInts;
        const int nrows = m[0], q0 = m[1], np = m[2], width = m[3], hoff = m[4], voff = m[5], rel = m[6], last = m[7];
        if (t < nrows) {
            const int4 dep = s_dep[sl * kCtaRows + t];
            T l[4];
            ld_vec4(l, s_l + 4 * (sl * kCtaRows + t));
            const T dinv = s_dinv[sl * kCtaRows + t];
            T acc = s_rhs[sl * kCtaRows + t];
            T y0, y1, y2, y3;
            if (kFar) {
                y0 = dep.x >= 0 ? win[dep.x] : __ldcg(outq + (-dep.x - 2));
                y1 = dep.y >= 0 ? win[dep.y] : __ldcg(outq + (-dep.y - 2));
                y2 = dep.z >= 0 ? win[dep.z] : __ldcg(outq + (-dep.z - 2));
                y3 = dep.w >= 0 ? win[dep.w] : __ldcg(outq + (-dep.w - 2));
            } else {
                y0 = win[dep.x];
                y1 = win[dep.y];
                y2 = win[dep.z];
                y3 = win[dep.w];
            }
            acc = fma(-l[0], y0, acc);
            acc = fma(-l[1], y1, acc);
            acc = fma(-l[2], y2, acc);
            acc = fma(-l[3], y3, acc);
            if (width > kRec) {
                const int32_t* xdep = reinterpret_cast<const int32_t*>(ring + hoff) + kHdrInts + 6 * np;
                const T* xval = reinterpret_cast<const T*>(ring + voff) + 5 * np;
                for (int kk = 0; kk < width - kRec; ++kk) {
                    const int pk = xdep[kk * np + t];
                    if (kFar && pk <= -2) acc = fma(-xval[kk * np + t], __ldcg(outq + (-pk - 2)), acc);
                    else acc = fma(-xval[kk * np + t], win[pk], acc);
                }
            }
            const T y = acc * dinv;
            const int q = q0 + t;
            win[q & (W - 1)] = y;
            outq[q] = y;
            if (kFar) __threadfence_block();
        }
        if (!split_agree(true)) return;
        if (rel >= 0 && lane == 0) mbar_arrive(&empty[rel]);   // chunk solved
        if (last) break;
    }
}

// ------------------------------------------------------------ flag-synchronised variant
// FP32 only.  The same layout and ring, without the barrier per step: every
// window slot is one 64-bit word {position, value} written with a single
// store, and a consumer polls its dependencies' slots until each holds the
// position it expects (slot and position agree modulo the window).  The
// ring, released per warp, lets a warp run at most (stages - 1) chunks
// ahead of the slowest; the window is sized to that drift plus the
// dependency reach, so a slot is never rewritten while a reader still needs
// it.  The dependency chain is then one shared-memory store and load per
// level instead of a CTA barrier.
__device__ __forceinline__ unsigned long long ld_slot(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.cta.shared.b64 %0, [%1];" : "=l"(v) : "r"(smem_u32(p)));
    return v;
}
__device__ __forceinline__ void st_slot(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.cta.shared.b64 [%0], %1;" ::"r"(smem_u32(p)), "l"(v));
}
__device__ __forceinline__ unsigned long long slot_word(int pos, float y) {
    return ((unsigned long long)(unsigned)pos << 32) | (unsigned long long)__float_as_uint(y);
}
__device__ __forceinline__ int slot_pos(unsigned long long w) { return (int)(w >> 32); }
__device__ __forceinline__ float slot_val(unsigned long long w) { return __uint_as_float((unsigned)w); }

// position held by dependency slot sl of the row at position q (the zero
// slot W stands for a missing dependency and carries position -1)
__device__ __forceinline__ int dep_pos(int q, int sl, int W) { return sl == W ? -1 : q - ((q - sl) & (W - 1)); }

__global__ void __launch_bounds__(kCtaThreads, 1) k_trsv_flag(CtaDev D, const float* __restrict__ rhs,
                                                             float* outq, const SysState* st, int* flags) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int sys = blockIdx.x;
    if (st && !st[sys].active) return;
    const int c0 = D.sys_chunk0[sys], c1 = D.sys_chunk0[sys + 1];
    if (c0 >= c1) return;
    const int S = D.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kMaxStages;
    int4* info = reinterpret_cast<int4*>(empty + kMaxStages);
    unsigned long long* win = reinterpret_cast<unsigned long long*>(smem + kBarBytes);
    const int W = D.win;
    unsigned char* ring = smem + kBarBytes + (size_t)(W + kWinPad) * sizeof(unsigned long long);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCtaRows / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // no slot holds a position yet; the zero slot (and the padding) holds
    // position -1 with value 0
    for (int i = threadIdx.x; i < W + kWinPad; i += blockDim.x) win[i] = slot_word(i >= W ? -1 : -2, 0.0f);
    __syncthreads();

    if (warp == kCtaRows / 32) {
        ring_producer<float>(D, rhs, ring, full, empty, info, c0, c1, flags);
        return;
    }

    // ---------------- consumer warps
    // Steps rotate over the warps: a step of nrows rows takes ceil(nrows/32)
    // consecutive warps (mod 8), starting where the previous step's ended,
    // so consecutive levels run on different warps and a warp's bookkeeping
    // for its next step overlaps the other warps' work on the levels before.
    // Each warp walks every step header (a "walker"), takes part in the
    // steps that reach it, and loads the operands of its next step before it
    // computes the current one.  It releases a chunk once it holds no step
    // of it any more; the walker enters a new chunk only when the ring can
    // hold it without this warp's own release (else it resumes after the
    // current step is done).
    const unsigned kAll = 0xffffffffu;
    int wc = c0, wu = 0, wnst, wq0e, wrb = 0;
    const int32_t* whdr;
    const float* wvals;
    const float* wrh;
    int4 wh;
    {
        const bool ok = mbar_wait_bounded(&full[0], 0u, D.spin);
        if (!__all_sync(kAll, ok)) {
            if (lane == 0) atomicOr(flags, kFlagTimeout | kFlagAbort);
            return;
        }
        const int4 inf = info[0];
        wnst = inf.x;
        whdr = reinterpret_cast<const int32_t*>(ring);
        wvals = reinterpret_cast<const float*>(ring + inf.y);
        wrh = reinterpret_cast<const float*>(ring + inf.z);
        wq0e = inf.w;
        wh = *reinterpret_cast<const int4*>(whdr);
    }
    bool wdone = false, wexam = false, dead = false;
    int rel = c0;                         // chunks below rel are released by this warp
    StepOps<float> cur, nxt;
    bool have_cur = false;
    int cur_e = 0, nxt_c = c0, nxt_e = 0;
    const int32_t* cur_hdr = whdr;
    const float* cur_vals = wvals;
    const int32_t* nxt_hdr = whdr;
    const float* nxt_vals = wvals;
    for (;;) {
        const bool live = have_cur && cur_e < cur.nrows;
        const int q = cur.q0 + cur_e;
        int e0 = 0, e1 = 0, e2 = 0, e3 = 0;
        unsigned long long w0 = 0, w1 = 0, w2 = 0, w3 = 0;
        if (live) {
            // first poll of the current row's dependencies, before the walk
            e0 = dep_pos(q, cur.dep.x, W);
            e1 = dep_pos(q, cur.dep.y, W);
            e2 = dep_pos(q, cur.dep.z, W);
            e3 = dep_pos(q, cur.dep.w, W);
            w0 = ld_slot(win + cur.dep.x);
            w1 = ld_slot(win + cur.dep.y);
            w2 = ld_slot(win + cur.dep.z);
            w3 = ld_slot(win + cur.dep.w);
        }
        // ---- walk to the next step this warp takes part in
        bool have_nxt = false;
        while (!wdone) {
            const int nw = (wh.y + 31) >> 5;
            if (!wexam) {
                wexam = true;
                const int slot = (warp - wrb) & 7;
                if (slot < nw) {
                    nxt_e = slot * 32 + lane;
                    load_step<false>(nxt, whdr, wvals, wrh, wq0e, nxt_e);
                    nxt_c = wc;
                    nxt_hdr = whdr;
                    nxt_vals = wvals;
                    have_nxt = true;
                }
            }
            // advance past the examined step
            if (wu + 1 < wnst) {
                const int np = pad4(wh.y);
                whdr += s_ints(np, wh.z);
                wvals += v_elems(np, wh.z);
                ++wu;
            } else if (wc + 1 >= c1) {
                wdone = true;
                break;
            } else {
                // the stage of chunk wc + 1 is refilled only after every warp
                // released chunk wc + 1 - S
                if (wc + 1 - S >= rel) break;
                ++wc;
                const int ws = (wc - c0) % S;
                const bool ok = mbar_wait_bounded(&full[ws], (uint32_t)(((wc - c0) / S) & 1), D.spin);
                if (!__all_sync(kAll, ok)) {
                    if (lane == 0) atomicOr(flags, kFlagTimeout | kFlagAbort);
                    return;
                }
                const int4 inf = info[ws];
                const unsigned char* base = ring + (size_t)ws * D.stage_cap;
                wnst = inf.x;
                whdr = reinterpret_cast<const int32_t*>(base);
                wvals = reinterpret_cast<const float*>(base + inf.y);
                wrh = reinterpret_cast<const float*>(base + inf.z);
                wq0e = inf.w;
                wu = 0;
            }
            wrb = (wrb + nw) & 7;
            wh = *reinterpret_cast<const int4*>(whdr);
            wexam = false;
            if (have_nxt) break;
        }
        // ---- the current row
        if (live) {
            long long spins = 0;
            while (!dead && (slot_pos(w0) != e0 || slot_pos(w1) != e1 || slot_pos(w2) != e2 || slot_pos(w3) != e3)) {
                if (slot_pos(w0) != e0) w0 = ld_slot(win + cur.dep.x);
                if (slot_pos(w1) != e1) w1 = ld_slot(win + cur.dep.y);
                if (slot_pos(w2) != e2) w2 = ld_slot(win + cur.dep.z);
                if (slot_pos(w3) != e3) w3 = ld_slot(win + cur.dep.w);
                if ((++spins & 255) == 0) {
                    if (ld_relaxed_s32(flags) & kFlagAbort) dead = true;
                    else if (spins > D.spin) { atomicOr(flags, kFlagTimeout | kFlagAbort); dead = true; }
                }
            }
            float acc = cur.rhs;
            acc = fmaf(-cur.l[0], slot_val(w0), acc);
            acc = fmaf(-cur.l[1], slot_val(w1), acc);
            acc = fmaf(-cur.l[2], slot_val(w2), acc);
            acc = fmaf(-cur.l[3], slot_val(w3), acc);
            if (cur.width > kRec) {
                const int32_t* xdep = cur_hdr + kHdrInts + 6 * cur.np;
                const float* xval = cur_vals + 5 * cur.np;
                for (int kk = 0; kk < cur.width - kRec; ++kk) {
                    const int sl = xdep[kk * cur.np + cur_e];
                    const int e = dep_pos(q, sl, W);
                    unsigned long long wx = ld_slot(win + sl);
                    while (!dead && slot_pos(wx) != e) {
                        wx = ld_slot(win + sl);
                        if ((++spins & 255) == 0) {
                            if (ld_relaxed_s32(flags) & kFlagAbort) dead = true;
                            else if (spins > D.spin) { atomicOr(flags, kFlagTimeout | kFlagAbort); dead = true; }
                        }
                    }
                    acc = fmaf(-xval[kk * cur.np + cur_e], slot_val(wx), acc);
                }
            }
            const float y = acc * cur.dinv;
            st_slot(win + (q & (W - 1)), slot_word(q, y));
            outq[q] = y;
        }
        __syncwarp();
        // release the chunks this warp no longer reads: below the walker's
        // chunk and below its next step's chunk
        int lim = wdone ? c1 : wc;
        if (have_nxt) lim = min(lim, nxt_c);
        for (; rel < lim; ++rel)
            if (lane == 0) mbar_arrive(&empty[(rel - c0) % S]);
        if (__any_sync(kAll, dead)) return;
        if (!have_nxt && wdone) break;
        have_cur = have_nxt;
        cur = nxt;
        cur_e = nxt_e;
        cur_hdr = nxt_hdr;
        cur_vals = nxt_vals;
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
        body[4 * np + 2 * t] = row;
        body[4 * np + 2 * t + 1] = 0;                   // pos2: set by k_cta_pos2
        const int nl = Lrp[row + 1] - Lrp[row];
        int cnt, first;
        if (upper) { cnt = (rp[row + 1] - rp[row]) - nl; first = rp[row + 1] - cnt; }
        else { cnt = nl - 1; first = Lrp[row]; }
        vs[4 * np + t] = Lrp[row + 1] - 1;              // diagonal (stored as its reciprocal)
        const int kmax = d.z > kRec ? d.z : kRec;
        for (int k = 0; k < kmax; ++k) {
            int dep = -1, src = -1;
            if (k < cnt) {
                if (upper) { dep = cpos[ci[first + k]]; src = a2l[mirror[first + k]]; }
                else { dep = cpos[Lci[first + k]]; src = first + k; }
            }
            if (k < kRec) {
                body[4 * t + k] = dep;
                vs[4 * t + k] = src;
            } else {
                body[6 * np + (k - kRec) * np + t] = dep;
                vs[5 * np + (k - kRec) * np + t] = src;
            }
        }
    }
}

// k_cta_fill for an arbitrary dependency pattern (drp / drow, value index =
// dependency entry) with the diagonal's value at diag_src
__global__ void k_cta_fill_dep(int64_t n, const int32_t* cperm, const int32_t* step_of_pos, const int4* steps,
                               const int64_t* soff, const int64_t* voff, const int32_t* cpos, const int64_t* drp,
                               const int32_t* drow, int64_t diag_src, int32_t* sbuf, int32_t* vsrc) {
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
        body[4 * np + 2 * t] = row;
        body[4 * np + 2 * t + 1] = 0;
        vs[4 * np + t] = (int32_t)diag_src;
        const int64_t e0 = drp[row];
        const int cnt = (int)(drp[row + 1] - e0);
        const int kmax = d.z > kRec ? d.z : kRec;
        for (int k = 0; k < kmax; ++k) {
            int dep = -1, src = -1;
            if (k < cnt) {
                dep = cpos[drow[e0 + k]];
                src = (int32_t)(e0 + k);
            }
            if (k < kRec) {
                body[4 * t + k] = dep;
                vs[4 * t + k] = src;
            } else {
                body[6 * np + (k - kRec) * np + t] = dep;
                vs[5 * np + (k - kRec) * np + t] = src;
            }
        }
    }
}

__device__ __forceinline__ int32_t* dep_slot(int32_t* body, int np, int t, int k) {
    return k < kRec ? body + 4 * t + k : body + 6 * np + (k - kRec) * np + t;
}

__global__ void k_cta_reach(int64_t n, const int32_t* step_of_pos, const int4* steps,
                            const int32_t* level_end, int32_t* sbuf, const int64_t* soff,
                            unsigned long long* reach) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int stp = step_of_pos[q];
        const int4 d = steps[stp];
        const int np = pad4(d.y);
        const int t = (int)(q - d.x);
        int32_t* body = sbuf + soff[stp] + kHdrInts;
        for (int k = 0; k < d.z; ++k) {
            const int p = *dep_slot(body, np, t, k);
            if (p >= 0) atomicMax(reach, (unsigned long long)(level_end[stp] - p));
        }
    }
}

// blocked layouts: a dependency outside the row's unit becomes -(row + 2)
__global__ void k_cta_remote(int64_t n, const int32_t* step_of_pos, const int4* steps, const int2* step_unit,
                             const int64_t* soff, const int32_t* cperm, int32_t* sbuf) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int stp = step_of_pos[q];
        const int4 d = steps[stp];
        const int2 u = step_unit[stp];
        const int np = pad4(d.y);
        const int t = (int)(q - d.x);
        int32_t* body = sbuf + soff[stp] + kHdrInts;
        const int kmax = d.z > kRec ? d.z : kRec;
        for (int k = 0; k < kmax; ++k) {
            int32_t* p = dep_slot(body, np, t, k);
            if (*p >= 0 && (*p < u.x || *p >= u.y)) *p = -(cperm[*p] + 2);
        }
    }
}

// dependency positions become window slots; with lend (hybrid window) a
// dependency further back than the window (level end - position > W) is
// read from the processing-order output instead and encoded -(position + 2)
__global__ void k_cta_window(int64_t n, const int32_t* step_of_pos, const int4* steps, const int64_t* soff,
                             int W, const int32_t* lend, int32_t* sbuf) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int stp = step_of_pos[q];
        const int4 d = steps[stp];
        const int np = pad4(d.y);
        const int t = (int)(q - d.x);
        int32_t* body = sbuf + soff[stp] + kHdrInts;
        const int kmax = d.z > kRec ? d.z : kRec;
        for (int k = 0; k < kmax; ++k) {
            int32_t* p = dep_slot(body, np, t, k);
            if (*p >= 0) *p = lend && lend[stp] - *p > W ? -(*p + 2) : (*p & (W - 1));
            else if (*p == -1) *p = W;              // missing: the zero slot; <= -2 (remote) stays
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
        body[4 * np + 2 * t + 1] = cpos_other[body[4 * np + 2 * t]];
    }
}

// values: reciprocal of the diagonal in the 1/diag slots of every block,
// off-diagonals elsewhere; padding and missing slots get zero
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
        for (int k = threadIdx.x; k < v_elems(np, d.z); k += blockDim.x)
            if (voff[stp] + k < nv) is_diag[voff[stp] + k] = (k >= 4 * np && k < 5 * np) ? 1 : 0;
    }
}

__global__ void k_compose(int64_t n, const int32_t* perm, const int32_t* pos, int32_t* out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        out[q] = pos[perm[q]];
}

template <class S, class D>
__global__ void k_permute(int64_t n, const int32_t* idx, const S* __restrict__ src, D* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (D)src[idx[i]];
}

template <class T>
__global__ void k_gather_perm(int64_t n, const int32_t* cperm, const double* x, T* xp) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        xp[q] = (T)x[cperm[q]];
}

size_t win_bytes(const CtaLayout& C, bool f32) {
    return C.window_ok ? (size_t)(C.win_slots + kWinPad) * (f32 ? 4 : 8) : 0;
}

size_t smem_bytes(const CtaLayout& C, bool f32) {
    return kBarBytes + win_bytes(C, f32) + (size_t)C.stage_cap[f32] * C.nstages[f32];
}

size_t smem_bytes_flag(const CtaLayout& C) {
    return kBarBytes + (size_t)(C.win_slots + kWinPad) * sizeof(unsigned long long) +
           (size_t)C.stage_cap[2] * C.nstages[2];
}

// shared memory per CTA: everything when each system has an SM of its own,
// half when more systems than SMs share the GPU (two CTAs per SM)
constexpr size_t kSmemMax = 220 * 1024;
constexpr size_t kSmemHalf = 110 * 1024;

// Groups the steps of every system into chunks of at most cap bytes
// (structure + values + right-hand side) for value size vsz; returns false
// when a single step does not fit.
bool build_chunks(const std::vector<int4>& steps, const std::vector<int64_t>& soff,
                  const std::vector<int64_t>& voff, const std::vector<int32_t>& sys_step0, int nsys,
                  size_t vsz, size_t cap, std::vector<CtaChunk>& out, std::vector<int32_t>& sys_chunk0) {
    const int al = (int)(16 / vsz);
    out.clear();
    sys_chunk0.assign(nsys + 1, 0);
    auto sbytes_of = [&](int i) { return (size_t)s_ints(pad4(steps[i].y), steps[i].z) * 4; };
    auto vbytes_of = [&](int i) { return (size_t)v_elems(pad4(steps[i].y), steps[i].z) * vsz; };
    for (int sy = 0; sy < nsys; ++sy) {
        sys_chunk0[sy] = (int32_t)out.size();
        int i = sys_step0[sy];
        const int e = sys_step0[sy + 1];
        while (i < e) {
            CtaChunk c{};
            c.soff = soff[i];
            c.voff = voff[i];
            c.q0e = steps[i].x & ~(al - 1);
            size_t sb = 0, vb = 0, rb = 0;
            int j = i;
            while (j < e) {
                const size_t sb2 = sb + sbytes_of(j), vb2 = vb + vbytes_of(j);
                const int qend = steps[j].x + steps[j].y;
                const size_t rb2 = (size_t)(((qend - c.q0e) + al - 1) & ~(al - 1)) * vsz;
                if (sb2 + vb2 + rb2 > cap) break;
                sb = sb2; vb = vb2; rb = rb2;
                ++j;
            }
            if (j == i) return false;
            c.nsteps = j - i;
            c.sbytes = (unsigned)sb;
            c.vbytes = (unsigned)vb;
            c.rbytes = (unsigned)rb;
            out.push_back(c);
            i = j;
        }
    }
    sys_chunk0[nsys] = (int32_t)out.size();
    return true;
}

}  // namespace

// Host: builds the per-system level-synchronous layout of one direction.
// Order: positions sorted by (system, level, row), i.e. the level order of
// each system, systems one after another.
npcg_status cta_layout_build(Handle* h, Pattern* P, bool upper, CtaLayout* C, const CtaDeps* dep) {
    const int64_t n = P->n;
    const TriLayout& T = upper ? P->bwd : P->fwd;
    std::vector<int32_t> lev(n), rp_h(n + 1), Lrp_h(n + 1);
    if (dep) lev = *dep->lev;
    else NPCG_CUDA(h, cudaMemcpyAsync(lev.data(), T.level.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(rp_h.data(), P->rp.p, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(Lrp_h.data(), P->Lrp.p, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    // units: one per system, or (one large system) contiguous row blocks,
    // one per SM, listed in dependency order (the backward solve runs from
    // the last row, so its blocks come last-first)
    std::vector<std::pair<int64_t, int64_t>> units;
    C->blocked = P->nsys == 1 && n >= kBlockedRows;
    if (C->blocked) {
        // fewer, thicker blocks put fewer cross-SM hand-offs on the critical
        // path of a long level chain; their number is tuned at analysis
        // (merged-level layouts keep one block per SM: fewer blocks measured slower there)
        const int U = !dep && P->block_units > 0 ? P->block_units : h->num_sms;
        const int64_t B = (n + U - 1) / U;
        for (int64_t r0 = 0; r0 < n; r0 += B) units.push_back({r0, std::min<int64_t>(n, r0 + B)});
        if (upper) std::reverse(units.begin(), units.end());
    } else {
        for (int s = 0; s < P->nsys; ++s) units.push_back({P->sys_ptr_h[s], P->sys_ptr_h[s + 1]});
    }
    const int nunits = (int)units.size();
    C->nunits = nunits;
    std::vector<int32_t> cperm(n), cpos(n), step_of_pos(n), sys_step0(nunits + 1, 0), level_end;
    std::vector<int4> steps;
    std::vector<int2> step_unit;                   // processing-position range of each step's unit
    auto offdiag = [&](int row) {
        if (dep) return (int)((*dep->drp)[row + 1] - (*dep->drp)[row]);
        int nl = Lrp_h[row + 1] - Lrp_h[row];
        return upper ? (rp_h[row + 1] - rp_h[row]) - nl : nl - 1;
    };
    int64_t q = 0;
    int maxw = 0, maxnp = 0;
    for (int s = 0; s < nunits; ++s) {
        sys_step0[s] = (int32_t)steps.size();
        const int64_t r0 = units[s].first, r1 = units[s].second;
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
                step_unit.push_back(make_int2((int)q, (int)(q + (r1 - r0))));
                level_end.push_back((int32_t)b);
                for (int64_t p = c0; p < c1; ++p) step_of_pos[p] = sid;
                maxw = std::max(maxw, w);
                maxnp = std::max(maxnp, (int)(c1 - c0));
            }
        }
        q += r1 - r0;
    }
    sys_step0[nunits] = (int32_t)steps.size();
    for (int64_t p = 0; p < n; ++p) cpos[cperm[p]] = (int32_t)p;
    const int nsteps = (int)steps.size();
    std::vector<int64_t> soff(nsteps), voff(nsteps);
    int64_t so = 0, vo = 0;
    for (int i = 0; i < nsteps; ++i) {
        const int np = pad4(steps[i].y);
        soff[i] = so;
        voff[i] = vo;
        so += s_ints(np, steps[i].z);
        vo += v_elems(np, steps[i].z);
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
    NPCG_CUDA(h, C->sys_step0.alloc(nunits + 1));
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
    NPCG_CUDA(h, cudaMemcpyAsync(C->sys_step0.p, sys_step0.data(), (nunits + 1) * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(C->step_of_pos.p, step_of_pos.data(), n * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(lend.p, level_end.data(), nsteps * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemsetAsync(C->sbuf.p, 0, C->sbuf.n * 4, h->stream));
    NPCG_CUDA(h, cudaMemsetAsync(C->vsrc.p, 0xff, C->vsrc.n * 4, h->stream));
    const int blocks = std::max(1, std::min(ceil_div(n, 256), h->num_sms * 8));
    if (dep)
        k_cta_fill_dep<<<blocks, 256, 0, h->stream>>>(n, C->cperm.p, C->step_of_pos.p, C->steps.p, C->soff.p,
                                                      C->voff.p, C->cpos.p, dep->drp_dev, dep->drow_dev,
                                                      dep->diag_src, C->sbuf.p, C->vsrc.p);
    else
        k_cta_fill<<<blocks, 256, 0, h->stream>>>(n, C->cperm.p, C->step_of_pos.p, C->steps.p, C->soff.p,
                                                  C->voff.p, C->cpos.p, P->Lrp.p, P->Lci.p, P->rp.p, P->ci.p,
                                                  P->mirror.p, P->a2l.p, upper ? 1 : 0, C->sbuf.p, C->vsrc.p);
    k_mark_diag<<<std::max(1, std::min(nsteps, h->num_sms * 8)), 256, 0, h->stream>>>(
        nsteps, C->steps.p, C->voff.p, C->is_diag.p, vo);
    NPCG_CUDA(h, cudaGetLastError());
    if (C->blocked) {
        DevBuf<int2> su;
        NPCG_CUDA(h, su.alloc(nsteps));
        NPCG_CUDA(h, cudaMemcpyAsync(su.p, step_unit.data(), nsteps * sizeof(int2), cudaMemcpyHostToDevice, h->stream));
        k_cta_remote<<<blocks, 256, 0, h->stream>>>(n, C->step_of_pos.p, C->steps.p, su.p, C->soff.p, C->cperm.p,
                                                    C->sbuf.p);
        NPCG_CUDA(h, cudaGetLastError());
        NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    DevBuf<unsigned long long> reach;
    NPCG_CUDA(h, reach.alloc(1));
    NPCG_CUDA(h, cudaMemsetAsync(reach.p, 0, 8, h->stream));
    k_cta_reach<<<blocks, 256, 0, h->stream>>>(n, C->step_of_pos.p, C->steps.p, lend.p, C->sbuf.p,
                                               C->soff.p, reach.p);
    NPCG_CUDA(h, cudaGetLastError());
    unsigned long long rh = 0;
    NPCG_TRY(read_scalar(h, reach.p, &rh));
    C->window_ok = rh <= (unsigned long long)kWinMax;
    C->win_slots = kWinMin;
    if (C->window_ok)
        while ((unsigned long long)C->win_slots < rh) C->win_slots *= 2;
    // Hybrid window: a dependency-free row sits at level 0 wherever it is in
    // the mesh, so one late reader can stretch the reach of a whole system.
    // One system per CTA then keeps the largest window and reads only the
    // dependencies beyond it from the processing-order output.
    C->far = !C->window_ok && !C->blocked;
    if (C->far) {
        C->window_ok = true;
        C->win_slots = kWinMax;
    }
    const size_t budget = nunits > h->num_sms ? kSmemHalf : kSmemMax;
    // largest single step (structure + values + right-hand side) for value size vsz
    auto single_bytes = [&](size_t vsz) {
        const int al = (int)(16 / vsz);
        size_t single = 0;
        for (int i = 0; i < nsteps; ++i) {
            const int np = pad4(steps[i].y);
            const int q0e = steps[i].x & ~(al - 1);
            const size_t rb = (size_t)(((steps[i].x + steps[i].y - q0e) + al - 1) & ~(al - 1)) * vsz;
            single = std::max(single, (size_t)s_ints(np, steps[i].z) * 4 + (size_t)v_elems(np, steps[i].z) * vsz + rb);
        }
        return single;
    };
    // Flag-synchronised kernel: the smallest window, up to kWinMax, that
    // holds the dependency reach plus the positions of the ring's stages
    // (how far one consumer warp can run ahead of another); its chunks are
    // kernel [2].  The barrier kernels share that window size.
    std::vector<CtaChunk> fch;
    std::vector<int32_t> fsc0;
    size_t fcap = 0;
    int fstages = 0;
    C->flag_ok = false;
    if (C->window_ok && !C->blocked && !C->far && !dep) {
        const size_t single = single_bytes(4);
        for (int W = C->win_slots; W <= kWinMax; W *= 2) {
            const size_t wb = (size_t)(W + kWinPad) * sizeof(unsigned long long);
            if (budget <= kBarBytes + wb) break;
            const size_t avail = budget - kBarBytes - wb;
            size_t cap = std::max(single, avail / kMaxStages);
            cap = (cap + 127) & ~size_t(127);
            const int stages = (int)std::min<size_t>(kMaxStages, avail / cap);
            if (stages < 2 || !build_chunks(steps, soff, voff, sys_step0, nunits, 4, cap, fch, fsc0)) break;
            // positions spanned by any `stages` consecutive chunks of a unit
            int64_t drift = 0;
            for (int un = 0; un < nunits; ++un) {
                std::vector<int64_t> cs, ce;
                int i = sys_step0[un];
                for (int j = fsc0[un]; j < fsc0[un + 1]; ++j) {
                    const int last = i + fch[j].nsteps - 1;
                    cs.push_back(steps[i].x);
                    ce.push_back((int64_t)steps[last].x + steps[last].y);
                    i = last + 1;
                }
                for (size_t k = 0; k < cs.size(); ++k)
                    drift = std::max(drift, ce[std::min(cs.size() - 1, k + stages - 1)] - cs[k]);
            }
            if ((int64_t)rh + drift + kCtaRows <= (int64_t)W) {
                C->win_slots = W;
                C->flag_ok = true;
                fcap = cap;
                fstages = stages;
                break;
            }
        }
    }
    if (C->window_ok) {
        k_cta_window<<<blocks, 256, 0, h->stream>>>(n, C->step_of_pos.p, C->steps.p, C->soff.p, C->win_slots,
                                                    C->far ? lend.p : nullptr, C->sbuf.p);
        NPCG_CUDA(h, cudaGetLastError());
    }
    // chunks per value type: the stage capacity is the larger of the biggest
    // single step and an even split of the free shared memory into kMaxStages
    for (int f32 = 0; f32 < 2; ++f32) {
        const size_t vsz = f32 ? 4 : 8;
        const size_t single = single_bytes(vsz);
        const size_t avail = budget - kBarBytes - win_bytes(*C, f32 != 0);
        size_t cap = std::max(single, avail / kMaxStages);
        cap = (cap + 127) & ~size_t(127);
        const int stages = (int)std::min<size_t>(kMaxStages, avail / cap);
        C->stage_cap[f32] = (int)cap;
        C->nstages[f32] = 0;
        C->nchunks[f32] = 0;
        std::vector<CtaChunk> ch;
        std::vector<int32_t> sc0;
        if (stages < 2 || !build_chunks(steps, soff, voff, sys_step0, nunits, vsz, cap, ch, sc0)) continue;
        C->nstages[f32] = stages;
        C->nchunks[f32] = (int)ch.size();
        NPCG_CUDA(h, C->chunks[f32].alloc(std::max<size_t>(ch.size(), 1)));
        NPCG_CUDA(h, C->sys_chunk0[f32].alloc(nunits + 1));
        NPCG_CUDA(h, cudaMemcpyAsync(C->chunks[f32].p, ch.data(), ch.size() * sizeof(CtaChunk),
                                     cudaMemcpyHostToDevice, h->stream));
        NPCG_CUDA(h, cudaMemcpyAsync(C->sys_chunk0[f32].p, sc0.data(), (nunits + 1) * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, h->stream));
        NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    // split-role kernel: the same chunks in a shallower ring beside the
    // staging slots (one CTA per SM)
    for (int f32 = 0; f32 < 2; ++f32) {
        C->split_stages[f32] = 0;
        if (!C->window_ok || C->blocked || dep || nunits > h->num_sms || C->nstages[f32] < 2) continue;
        const size_t used = kBarBytes + win_bytes(*C, f32 != 0) +
                            (f32 ? split_staging_bytes<float>() : split_staging_bytes<double>());
        if (used >= kSmemMax) continue;
        const int st = (int)std::min<size_t>((size_t)C->nstages[f32], (kSmemMax - used) / (size_t)C->stage_cap[f32]);
        C->split_stages[f32] = st >= 2 ? st : 0;
    }
    C->nstages[2] = 0;
    C->nchunks[2] = 0;
    if (C->flag_ok) {
        C->stage_cap[2] = (int)fcap;
        C->nstages[2] = fstages;
        C->nchunks[2] = (int)fch.size();
        NPCG_CUDA(h, C->chunks[2].alloc(std::max<size_t>(fch.size(), 1)));
        NPCG_CUDA(h, C->sys_chunk0[2].alloc(nunits + 1));
        NPCG_CUDA(h, cudaMemcpyAsync(C->chunks[2].p, fch.data(), fch.size() * sizeof(CtaChunk),
                                     cudaMemcpyHostToDevice, h->stream));
        NPCG_CUDA(h, cudaMemcpyAsync(C->sys_chunk0[2].p, fsc0.data(), (nunits + 1) * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, h->stream));
        NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    // the launch size never exceeds 220 KB; set once here, outside any capture
    const int mx = 220 * 1024;
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_flag, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_split<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_split<true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_split<false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_split<true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<true, false, false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<false, false, false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<true, false, false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<false, false, false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<true, true, false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<false, true, false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<true, true, false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<false, true, false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<true, false, true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    NPCG_CUDA(h, cudaFuncSetAttribute(k_trsv_cta<true, false, true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
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
    NPCG_CUDA(h, P->cbwd.other.alloc(P->n));
    k_compose<<<blocks, 256, 0, h->stream>>>(P->n, P->cbwd.cperm.p, P->cfwd.cpos.p, P->cbwd.other.p);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

// where the direction's solution is in processing order: the output buffer
// (value type) with the window, else the FP64 global copy
static void out_source(Pattern* P, const CtaLayout& C, void* outq, bool f32, const void** src, int* src_kind) {
    if (C.window_ok) { *src = outq; *src_kind = f32 ? 1 : 0; }
    else { *src = P->yglob.p; *src_kind = 0; }
}

// dst[i] = src[idx[i]]: the solution of a solve (processing order) into the
// order its reader needs (idx = positions); dst FP64 or the value type
npcg_status cta_permute(Handle* h, cudaStream_t s, Pattern* P, const CtaLayout& C, void* outq, bool f32,
                        const int32_t* idx, void* dst, bool dst_f32) {
    const void* src;
    int kind;
    out_source(P, C, outq, f32, &src, &kind);
    const int blocks = std::max(1, std::min(ceil_div(P->n, 256), h->num_sms * 8));
    const int64_t n = P->n;
    if (kind == 1 && dst_f32)
        k_permute<float, float><<<blocks, 256, 0, s>>>(n, idx, static_cast<const float*>(src), static_cast<float*>(dst));
    else if (kind == 1)
        k_permute<float, double><<<blocks, 256, 0, s>>>(n, idx, static_cast<const float*>(src), static_cast<double*>(dst));
    else if (dst_f32)
        k_permute<double, float><<<blocks, 256, 0, s>>>(n, idx, static_cast<const double*>(src), static_cast<float*>(dst));
    else
        k_permute<double, double><<<blocks, 256, 0, s>>>(n, idx, static_cast<const double*>(src), static_cast<double*>(dst));
    return NPCG_OK;
}

int cta_stages(const CtaLayout& C) { return std::min(C.nstages[0], C.nstages[1]); }

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
// rhs_perm: right-hand side in this direction's processing order (n + 4
// entries of the value type, the last ones padding); outq (n entries of the
// value type) receives the solution in processing order when the shared
// window suffices, otherwise the solution is in P->yglob (FP64); cta_permute
// moves it on.  f32: FP32 factor, arithmetic, right-hand side and outq.
npcg_status cta_trsv_launch(Handle* h, cudaStream_t s, Pattern* P, const CtaLayout& C, const void* rhs_v,
                            void* outq, const SysState* st, bool f32, int* ticket, double* pub) {
    if (P->cta_split && C.split_stages[f32] >= 2) {
        CtaDev d;
        d.sys_chunk0 = C.sys_chunk0[f32].p;
        d.chunks = C.chunks[f32].p;
        d.sbuf = C.sbuf.p;
        d.vbuf = f32 ? (const void*)C.vbuf32.p : (const void*)C.vbuf.p;
        d.stages = C.split_stages[f32];
        d.stage_cap = C.stage_cap[f32];
        d.win = C.win_slots;
        d.spin = h->spin_limit;
        const size_t smem = kBarBytes + win_bytes(C, f32) +
                            (f32 ? split_staging_bytes<float>() : split_staging_bytes<double>()) +
                            (size_t)C.stage_cap[f32] * C.split_stages[f32];
        int* flags = P->ctl.p + 1;
#define NPCG_SPLIT_LAUNCH(F, TT)                                                                              \
    k_trsv_split<F, TT><<<C.nunits, kSplitThreads, smem, s>>>(d, static_cast<const TT*>(rhs_v),                \
                                                              static_cast<TT*>(outq), st, flags)
        if (f32) { if (C.far) NPCG_SPLIT_LAUNCH(true, float); else NPCG_SPLIT_LAUNCH(false, float); }
        else { if (C.far) NPCG_SPLIT_LAUNCH(true, double); else NPCG_SPLIT_LAUNCH(false, double); }
#undef NPCG_SPLIT_LAUNCH
        NPCG_CUDA(h, cudaGetLastError());
        return NPCG_OK;
    }
    if (f32 && P->cta_flag && C.flag_ok && C.nstages[2] >= 2) {
        CtaDev d;
        d.sys_chunk0 = C.sys_chunk0[2].p;
        d.chunks = C.chunks[2].p;
        d.sbuf = C.sbuf.p;
        d.vbuf = C.vbuf32.p;
        d.stages = C.nstages[2];
        d.stage_cap = C.stage_cap[2];
        d.win = C.win_slots;
        d.spin = h->spin_limit;
        k_trsv_flag<<<C.nunits, kCtaThreads, smem_bytes_flag(C), s>>>(d, static_cast<const float*>(rhs_v),
                                                                      static_cast<float*>(outq), st, P->ctl.p + 1);
        NPCG_CUDA(h, cudaGetLastError());
        return NPCG_OK;
    }
    const int stages = C.nstages[f32];
    if (stages < 2) return set_error(h, NPCG_EINVAL, "level-synchronous layout does not fit shared memory");
    if (C.blocked && (!ticket || !pub)) return set_error(h, NPCG_EINVAL, "blocked solve needs a ticket and pub");
    CtaDev d;
    d.sys_chunk0 = C.sys_chunk0[f32].p;
    d.chunks = C.chunks[f32].p;
    d.sbuf = C.sbuf.p;
    d.vbuf = f32 ? (const void*)C.vbuf32.p : (const void*)C.vbuf.p;
    d.stages = stages;
    d.stage_cap = C.stage_cap[f32];
    d.win = C.win_slots;
    d.spin = h->spin_limit;
    const size_t smem = smem_bytes(C, f32);
    int* flags = P->ctl.p + 1;
    const int g = C.nunits;
    double* yg = P->yglob.p;
#define NPCG_CTA_LAUNCH(W, R, F, TT)                                                                        \
    k_trsv_cta<W, R, F, TT><<<g, kCtaThreads, smem, s>>>(d, static_cast<const TT*>(rhs_v),                   \
                                                         W ? static_cast<TT*>(outq) : nullptr, W ? nullptr : yg, \
                                                         st, flags, ticket, pub)
    if (f32) {
        if (C.blocked) { if (C.window_ok) NPCG_CTA_LAUNCH(true, true, false, float); else NPCG_CTA_LAUNCH(false, true, false, float); }
        else if (C.far) NPCG_CTA_LAUNCH(true, false, true, float);
        else { if (C.window_ok) NPCG_CTA_LAUNCH(true, false, false, float); else NPCG_CTA_LAUNCH(false, false, false, float); }
    } else {
        if (C.blocked) { if (C.window_ok) NPCG_CTA_LAUNCH(true, true, false, double); else NPCG_CTA_LAUNCH(false, true, false, double); }
        else if (C.far) NPCG_CTA_LAUNCH(true, false, true, double);
        else { if (C.window_ok) NPCG_CTA_LAUNCH(true, false, false, double); else NPCG_CTA_LAUNCH(false, false, false, double); }
    }
#undef NPCG_CTA_LAUNCH
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

}  // namespace npcg
