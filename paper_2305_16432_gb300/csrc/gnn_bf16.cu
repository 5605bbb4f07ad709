// Graph-network factor, BF16 tensor-core path (Sec. 4.2 "Architecture",
// App. A.3), hidden width h = 64.
//
// Every node / edge MLP runs as a chain of dense [128 x K] x [K x 64] products
// on the 5th-generation tensor cores: one elected thread issues tcgen05.mma
// (kind::f16, BF16 operands from shared memory, FP32 accumulator in tensor
// memory), tcgen05.commit signals an mbarrier, and the four warps read their
// 32-lane quarter of the accumulator with tcgen05.ld, add the bias, apply
// ReLU and write the next layer's operand back to shared memory as BF16.
// Operands use the 128-byte-swizzled K-major layout (8-row x 128-byte atoms,
// 16-byte chunk c of row r at chunk c ^ (r & 7)); weights are converted from
// the FP32 master copy and staged once per CTA.  Features between layers are
// BF16 in global memory; the message-passing gather accumulates in FP32.
// The scalar input layer of the encoders and the scalar output layer of the
// decoder run on the CUDA cores inside the same kernel.
#include <cuda_bf16.h>

#include <algorithm>

#include "gnn_common.cuh"
#include "tc_common.cuh"

namespace npcg {

namespace {

struct Bf16Args {
    int64_t nrows;
    const float* w;           // FP32 master weights of this MLP
    int depth;
    const int32_t* rp;
    const int32_t* ci;
    const int32_t* erow;
    const int32_t* row_sys;
    const double* sc;
    const double* av;
    const double* b;
    const __nv_bfloat16* vin;
    const __nv_bfloat16* ein;
    __nv_bfloat16* out;       // H-wide BF16 output rows
    float* sout;              // decoder: FP32 scalar output
    float* out32;             // optional FP32 copy of the output rows (training tape)
    float* agg32;             // optional FP32 aggregation sum_j e_ij (.) v_j (NODE, training tape)
    int* flags;
    const int32_t* adiag_scaled;  // diag_mode 2: positions of the diagonal (scaled edge input)
};

// tensor-core layers of each mode: NODE/EDGE all, ENC from layer 1, DEC to depth-1
__host__ __device__ constexpr int tc_first(int mode) { return mode == MODE_ENC_NODE || mode == MODE_ENC_EDGE ? 1 : 0; }

// modes whose first operand is a pure copy of feature rows: gathered with
// cp.async into a second buffer while the previous tile computes
__host__ __device__ constexpr bool async_gather(int mode) { return mode == MODE_EDGE || mode == MODE_DEC; }

struct SmemPlan {
    uint32_t a0, a0b, a1, w, bias, idx, misc, total;
};

__host__ __device__ inline SmemPlan plan(int mode, int depth) {
    const int in = mode_in(mode, kH);
    const int kin0 = (mode == MODE_ENC_NODE || mode == MODE_ENC_EDGE) ? kH : in;   // first TC layer input
    const int first = tc_first(mode);
    const int last = mode == MODE_DEC ? depth - 1 : depth;
    uint32_t wbytes = 0;
    for (int l = first; l <= last; ++l) wbytes += (uint32_t)((l == first ? kin0 : kH) / 64) * (kH * 128);
    const uint32_t a0bytes = (uint32_t)(kin0 / 64) * (kM * 128);
    SmemPlan p;
    p.a0 = 0;                                         // [128 x kin0] operand (kin0 / 64 K-blocks)
    p.a0b = p.a0;                                     // (single operand buffer)
    // [128 x 64] hidden operand.  Every layer's product has completed before
    // its epilogue writes the next operand, so without the async gather (which
    // refills A0 for the next tile after the first layer) the hidden operand
    // reuses A0's first K-block: less shared memory, more CTAs per SM
    p.a1 = async_gather(mode) ? p.a0 + a0bytes : p.a0;
    p.w = p.a0 + a0bytes + (async_gather(mode) ? kM * 128 : 0);
    p.bias = p.w + wbytes;                            // FP32 biases of every layer + scalar layer weights
    p.idx = p.bias + (uint32_t)(depth + 1) * kH * 4 + 2 * kH * 4 + 64;
    p.idx = (p.idx + 15) & ~15u;                      // async gather: [2 tiles][row, col][128] indices
    p.misc = p.idx + (async_gather(mode) ? 2u * 2u * kM * 4u : 0u);
    p.misc = (p.misc + 15) & ~15u;
    p.total = p.misc + 64;
    return p;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// EDGE: [e | v_row | v_col], DEC: [e]; rows past the end are zero-filled.
// The row / column indices of the tile come from shared memory (staged one
// tile ahead), so issuing the copies never waits on a global load.
template <int MODE>
__device__ __forceinline__ void gather_async(const Bf16Args& a, unsigned char* A, int64_t row0, int tid,
                                             const int* sidx) {
    constexpr int IN = mode_in(MODE, kH);
    constexpr int CH = IN / 8;
    for (int idx = tid; idx < kM * CH; idx += kThreads) {
        const int r = idx / CH, c = idx % CH;
        const int64_t k = row0 + r;
        const bool in = k < a.nrows;
        const int seg = c >> 3, cc = c & 7;
        const __nv_bfloat16* src = seg == 0 ? a.ein + (in ? k : 0) * kH
                                 : seg == 1 ? a.vin + (int64_t)sidx[r] * kH
                                            : a.vin + (int64_t)sidx[kM + r] * kH;
        cp_async16(s_addr(A + (uint32_t)(c >> 3) * (kM * 128) + swz(r, (c & 7) * 8)), src + cc * 8, in ? 16u : 0u);
    }
    cp_async_commit();
}

// this thread's row of a tile: its edge's row and column (0 past the end)
__device__ __forceinline__ int2 tile_index(const Bf16Args& a, int64_t tile, int64_t ntiles, int tid) {
    const int64_t k = tile * kM + tid;
    if (tile >= ntiles || k >= a.nrows) return make_int2(0, 0);
    return make_int2(a.erow[k], a.ci[k]);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_mlp_bf16(Bf16Args a) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    // swizzled operands need 1024-byte aligned shared addresses
    unsigned char* sm = sm_raw + ((1024u - (s_addr(sm_raw) & 1023u)) & 1023u);
    constexpr int IN = mode_in(MODE, kH);
    constexpr bool kEnc = MODE == MODE_ENC_NODE || MODE == MODE_ENC_EDGE;
    constexpr int KIN0 = kEnc ? kH : IN;
    const int depth = a.depth;
    const int first = tc_first(MODE);
    const int last = MODE == MODE_DEC ? depth - 1 : depth;
    const SmemPlan P = plan(MODE, depth);
    unsigned char* A0 = sm + P.a0;
    unsigned char* A1 = sm + P.a1;
    unsigned char* W = sm + P.w;
    float* bias = reinterpret_cast<float*>(sm + P.bias);          // [depth+1][64]
    float* s_w0 = bias + (depth + 1) * kH;                         // encoder layer 0: W[64] then b[64]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P.misc);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + P.misc + 8);
    const int tid = threadIdx.x, warp = tid >> 5;

    // ---- stage weights: BF16 swizzled K-blocks of every tensor-core layer, FP32 biases
    {
        const float* src = a.w;
        uint32_t woff = 0;
        for (int l = 0; l <= depth; ++l) {
            const int fi = l == 0 ? IN : kH, fo = (MODE == MODE_DEC && l == depth) ? 1 : kH;
            const bool tc = l >= first && l <= last;
            if (tc) {
                const int nkb = fi / 64;
                for (int t = tid; t < fo * fi; t += kThreads) {
                    const int n = t / fi, k = t % fi;
                    unsigned char* blk = W + woff + (uint32_t)(k / 64) * (kH * 128);
                    *reinterpret_cast<__nv_bfloat16*>(blk + swz(n, k % 64)) = __float2bfloat16_rn(src[t]);
                }
                woff += (uint32_t)nkb * (kH * 128);
            } else if (l == 0) {                 // encoder scalar input layer
                for (int t = tid; t < kH; t += kThreads) { s_w0[t] = src[t]; s_w0[kH + t] = src[kH + t]; }
            } else {                             // decoder scalar output layer: W[64], b
                for (int t = tid; t < kH; t += kThreads) s_w0[t] = src[t];
                if (tid == 0) s_w0[kH] = src[kH];
            }
            for (int t = tid; t < fo; t += kThreads) bias[l * kH + t] = src[fi * fo + t];
            src += fi * fo + fo;
        }
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(s_addr(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t my_lanes = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    bool ok = true;

    const int64_t ntiles = (a.nrows + kM - 1) / kM;
    constexpr bool kAsync = async_gather(MODE);
    int* sidx = reinterpret_cast<int*>(sm + P.idx);      // [2][2][kM]
    int2 nidx = make_int2(0, 0);
    if (kAsync) {
        const int2 i0 = tile_index(a, blockIdx.x, ntiles, tid);
        const int2 i1 = tile_index(a, (int64_t)blockIdx.x + gridDim.x, ntiles, tid);
        sidx[tid] = i0.x;
        sidx[kM + tid] = i0.y;
        sidx[2 * kM + tid] = i1.x;
        sidx[3 * kM + tid] = i1.y;
        __syncthreads();
        if constexpr (kAsync)
            if ((int64_t)blockIdx.x < ntiles) gather_async<MODE>(a, A0, (int64_t)blockIdx.x * kM, tid, sidx);
    }
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
        const int64_t row0 = tile * kM;
        if (kAsync) {
            // this tile's operand was requested while the previous tile was
            // still computing (right after its first layer had read the
            // buffer); the indices of the tile after next are loaded now and
            // staged at the end
            cp_async_wait<0>();
            nidx = tile_index(a, tile + 2 * (int64_t)gridDim.x, ntiles, tid);
        }
        // ---- stage 0: operand of the first tensor-core layer into A0
        if (kAsync) {
            // gathered above
        } else if (kEnc) {
            const int64_t row = row0 + tid;
            float x = 0.0f;
            if (row < a.nrows) {
                if (MODE == MODE_ENC_NODE) x = (float)(a.b[row] / a.sc[2 * a.row_sys[row] + 1]);
                else x = (float)edge_input(a.av, a.sc, a.row_sys, a.erow, a.ci, a.adiag_scaled, row);
            }
            for (int c = 0; c < 8; ++c) {
                __nv_bfloat16 h8[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int o = c * 8 + j;
                    h8[j] = __float2bfloat16_rn(fmaxf(fmaf(s_w0[o], x, bias[o]), 0.0f));
                }
                *reinterpret_cast<uint4*>(A0 + swz(tid, c * 8)) = *reinterpret_cast<uint4*>(h8);
            }
        } else if (MODE == MODE_NODE) {
            // v_i: eight threads per row, one 16-byte chunk each
            for (int idx = tid; idx < kM * 8; idx += kThreads) {
                const int r = idx >> 3, c = idx & 7;
                const int64_t i = row0 + r;
                uint4 val = make_uint4(0, 0, 0, 0);
                if (i < a.nrows) val = *reinterpret_cast<const uint4*>(a.vin + i * kH + c * 8);
                *reinterpret_cast<uint4*>(A0 + swz(r, c * 8)) = val;
            }
            // sum_j e_ij (.) v_j over the row's edges in ascending order,
            // eight threads per row (one chunk each, so that the edge and node
            // rows are read as whole lines).  A thread's eight (row, chunk)
            // items are software-pipelined: every item's edge range is read
            // first, and the column indices of item k + 1's first eight edges
            // are requested while item k's edge and node chunks are in
            // flight, so an item costs about one round trip instead of three
            // (rows with more than eight edges finish in batches of eight)
            constexpr int kItems = kM * 8 / kThreads;
            int rs[kItems], re[kItems];
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const int64_t i = row0 + ((tid + k * kThreads) >> 3);
                rs[k] = i < a.nrows ? a.rp[i] : 0;
                re[k] = i < a.nrows ? a.rp[i + 1] : 0;
            }
            int cj[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) cj[q] = rs[0] + q < re[0] ? a.ci[rs[0] + q] : -1;
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const int idx = tid + k * kThreads, r = idx >> 3, c = idx & 7;
                const int64_t i = row0 + r;
                float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                uint4 e4[8], v4[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (cj[q] >= 0) {
                        e4[q] = *reinterpret_cast<const uint4*>(a.ein + (int64_t)(rs[k] + q) * kH + c * 8);
                        v4[q] = *reinterpret_cast<const uint4*>(a.vin + (int64_t)cj[q] * kH + c * 8);
                    }
                }
                int cn[8];
                if (k + 1 < kItems) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) cn[q] = rs[k + 1] + q < re[k + 1] ? a.ci[rs[k + 1] + q] : -1;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (cj[q] < 0) break;
                    const __nv_bfloat16* e8 = reinterpret_cast<const __nv_bfloat16*>(&e4[q]);
                    const __nv_bfloat16* v8 = reinterpret_cast<const __nv_bfloat16*>(&v4[q]);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        acc[j] = fmaf(__bfloat162float(e8[j]), __bfloat162float(v8[j]), acc[j]);
                }
                for (int kb = rs[k] + 8; kb < re[k]; kb += 8) {
                    int cx[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) cx[q] = kb + q < re[k] ? a.ci[kb + q] : -1;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (cx[q] >= 0) {
                            e4[q] = *reinterpret_cast<const uint4*>(a.ein + (int64_t)(kb + q) * kH + c * 8);
                            v4[q] = *reinterpret_cast<const uint4*>(a.vin + (int64_t)cx[q] * kH + c * 8);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (cx[q] < 0) break;
                        const __nv_bfloat16* e8 = reinterpret_cast<const __nv_bfloat16*>(&e4[q]);
                        const __nv_bfloat16* v8 = reinterpret_cast<const __nv_bfloat16*>(&v4[q]);
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            acc[j] = fmaf(__bfloat162float(e8[j]), __bfloat162float(v8[j]), acc[j]);
                    }
                }
                uint4 val = make_uint4(0, 0, 0, 0);
                if (i < a.nrows) {
                    __nv_bfloat16 h8[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) h8[j] = __float2bfloat16_rn(acc[j]);
                    val = *reinterpret_cast<uint4*>(h8);
                    if (a.agg32) {
                        float4* g = reinterpret_cast<float4*>(a.agg32 + i * kH + c * 8);
                        g[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
                        g[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
                    }
                }
                *reinterpret_cast<uint4*>(A0 + kM * 128 + swz(r, c * 8)) = val;
                if (k + 1 < kItems) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) cj[q] = cn[q];
                }
            }
        } else {      // EDGE: [e | v_row | v_col], DEC: [e]
            constexpr int CH = IN >= 8 ? IN / 8 : 1;     // (encoders never reach here)
            for (int idx = tid; idx < kM * CH; idx += kThreads) {
                const int r = idx / CH, c = idx % CH;
                const int64_t k = row0 + r;
                uint4 val = make_uint4(0, 0, 0, 0);
                if (k < a.nrows) {
                    const int seg = c >> 3, cc = c & 7;
                    const __nv_bfloat16* src = seg == 0 ? a.ein + k * kH
                                             : seg == 1 ? a.vin + (int64_t)a.erow[k] * kH
                                                        : a.vin + (int64_t)a.ci[k] * kH;
                    val = *reinterpret_cast<const uint4*>(src + cc * 8);
                }
                *reinterpret_cast<uint4*>(A0 + (uint32_t)(c >> 3) * (kM * 128) + swz(r, (c & 7) * 8)) = val;
            }
        }
        // ---- tensor-core layers
        uint32_t woff = 0;
        for (int l = first; l <= last; ++l) {
            const int kin = l == first ? KIN0 : kH;
            const unsigned char* Aop = l == first ? A0 : A1;
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                const uint32_t abase = s_addr(Aop), wbase = s_addr(W + woff);
                for (int s = 0; s < kin / 16; ++s) {
                    const uint32_t kb = (uint32_t)(s >> 2), ko = (uint32_t)(s & 3) * 32;
                    mma_bf16(tmem, smem_desc(abase + kb * (kM * 128) + ko), smem_desc(wbase + kb * (kH * 128) + ko),
                             s > 0 ? 1u : 0u);
                }
                mma_commit(bar);
            }
            woff += (uint32_t)(kin / 64) * (kH * 128);
            ok = bar_wait(bar, phase);
            phase ^= 1u;
            if (!__syncthreads_and(ok)) {
                ok = false;          // every thread leaves the tile loop together
                break;
            }
            tc_fence_after();
            if constexpr (kAsync) {
                if (l == first && tile + gridDim.x < ntiles) {
                    // the first layer has read the operand buffer: the next
                    // tile's rows stream in while this tile finishes
                    gather_async<MODE>(a, A0, (tile + gridDim.x) * kM, tid, sidx + ((it + 1) & 1) * 2 * kM);
                }
            }
            float v[64];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float t16[16];
                tmem_ld16(my_lanes + q * 16, t16);
#pragma unroll
                for (int i = 0; i < 16; ++i) v[q * 16 + i] = t16[i];
            }
            tmem_wait_ld();
            const float* bl = bias + l * kH;
            const bool relu = l < depth;
            const int64_t row = row0 + tid;
            if (l < last || (MODE != MODE_DEC && l < depth)) {
                // next layer's operand (A1) -- the layer that read A1 has completed
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    __nv_bfloat16 h8[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float z = v[c * 8 + j] + bl[c * 8 + j];
                        h8[j] = __float2bfloat16_rn(relu ? fmaxf(z, 0.0f) : z);
                    }
                    *reinterpret_cast<uint4*>(A1 + swz(tid, c * 8)) = *reinterpret_cast<uint4*>(h8);
                }
            } else if (MODE == MODE_DEC) {
                // hidden layer depth-1 done: scalar output layer on the CUDA cores
                float s = s_w0[kH];
#pragma unroll
                for (int o = 0; o < kH; ++o) s = fmaf(s_w0[o], fmaxf(v[o] + bl[o], 0.0f), s);
                if (row < a.nrows) a.sout[row] = s;
            } else {
                // last layer: BF16 feature rows to global memory through A1
                // (its last reader, this layer's product, has completed), so
                // that the global stores are whole lines
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    __nv_bfloat16 h8[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) h8[j] = __float2bfloat16_rn(v[c * 8 + j] + bl[c * 8 + j]);
                    *reinterpret_cast<uint4*>(A1 + swz(tid, c * 8)) = *reinterpret_cast<uint4*>(h8);
                }
                __syncthreads();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = i * 16 + (tid >> 3), cc = tid & 7;
                    if (row0 + rr < a.nrows)
                        *reinterpret_cast<uint4*>(a.out + (row0 + rr) * kH + cc * 8) =
                            *reinterpret_cast<const uint4*>(A1 + swz(rr, cc * 8));
                }
                if (row < a.nrows) {
                    if (a.out32) {
                        float4* o = reinterpret_cast<float4*>(a.out32 + row * kH);
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            o[c] = make_float4(v[4 * c] + bl[4 * c], v[4 * c + 1] + bl[4 * c + 1],
                                               v[4 * c + 2] + bl[4 * c + 2], v[4 * c + 3] + bl[4 * c + 3]);
                    }
                }
            }
        }
        if (kAsync) {
            // the slot of this tile's indices was last read by the gather
            // issued one tile ago; it now receives the tile after next
            sidx[(it & 1) * 2 * kM + tid] = nidx.x;
            sidx[(it & 1) * 2 * kM + kM + tid] = nidx.y;
            __syncthreads();
        } else {
            // the output tile staged in A0 is read out before the next tile's
            // operand is written there
            __syncthreads();
        }
    }
    if (kAsync) cp_async_wait<0>();      // no copy may land after the CTA leaves
    if (!ok) {
        // give the outstanding products one more bounded wait before the
        // tensor memory is released
        bar_wait(bar, phase ^ 1u);
        if (tid == 0) atomicOr(a.flags, kFlagTimeout);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------ warp-specialised
// Edge update and decoder (modes whose first operand is a pure copy of
// feature rows), with tiles pipelined through the CTA: a producer warp
// gathers the rows of upcoming tiles with cp.async into a ring of operand
// stages (completion tracked by an mbarrier per stage), and two epilogue
// warpgroups take alternate tiles: one elected thread of a warpgroup issues
// the tile's tcgen05.mma chain into the warpgroup's own TMEM accumulator
// (64 columns each) while the other warpgroup drains its accumulator with
// tcgen05.ld, adds the bias, applies ReLU and stages the next layer's
// operand.  The first layer's commit releases the operand stage to the
// producer.  One CTA per SM; every wait is bounded.
// NG epilogue warpgroups (NG tiles in flight per SM), S operand stages
__host__ __device__ constexpr int ws_threads(int ng) { return ng * kM + 32; }
// TMEM columns: 64 per warpgroup, allocated as a power of two
__host__ __device__ constexpr uint32_t ws_tmem_cols(int ng) { return ng <= 2 ? 128u : 256u; }

struct WsPlan {
    uint32_t w, a0, a1, bias, bars, tslot, gen, total;
};

__host__ __device__ inline WsPlan ws_plan(int mode, int depth, int ng, int stages) {
    const int in = mode_in(mode, kH);
    const int last = mode == MODE_DEC ? depth - 1 : depth;
    uint32_t wbytes = 0;
    for (int l = 0; l <= last; ++l) wbytes += (uint32_t)((l == 0 ? in : kH) / 64) * (kH * 128);
    WsPlan p;
    p.w = 0;
    p.a0 = p.w + wbytes;                                        // [stage][in / 64 K-blocks][128 x 64]
    p.a1 = p.a0 + (uint32_t)stages * (uint32_t)(in / 64) * (kM * 128);   // [warpgroup][128 x 64]
    p.bias = p.a1 + (uint32_t)ng * (kM * 128);                  // FP32 biases + decoder scalar layer
    p.bars = p.bias + (uint32_t)(depth + 1) * kH * 4 + (kH + 1) * 4;
    p.bars = (p.bars + 15) & ~15u;                              // full[S], empty[S], mma[NG]
    p.tslot = p.bars + (uint32_t)(2 * stages + ng) * 8;
    p.gen = p.tslot + 16;                                       // tile last started in each stage
    p.total = p.gen + (uint32_t)stages * 4 + 16;
    return p;
}

__device__ __forceinline__ void ws_bar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(b)), "r"(count) : "memory");
}

// one arrive on the barrier once every cp.async this thread issued before has landed
__device__ __forceinline__ void cp_async_arrive(uint64_t* b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(s_addr(b)) : "memory");
}

// named barrier of one epilogue warpgroup that also ANDs a flag over it
__device__ __forceinline__ bool group_agree(int g, bool ok) {
    uint32_t all_ok;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(all_ok)
        : "r"((uint32_t)ok), "r"(1 + g), "r"(kM)
        : "memory");
    return all_ok != 0;
}

template <int MODE, int NG, int S>
__global__ void __launch_bounds__(ws_threads(NG), 1) k_mlp_bf16_ws(Bf16Args a) {
    constexpr int kWsStages = S;
    constexpr int kWsThreads = ws_threads(NG);
    static_assert(MODE == MODE_EDGE || MODE == MODE_DEC, "pure-copy operand modes only");
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((1024u - (s_addr(sm_raw) & 1023u)) & 1023u);
    constexpr int IN = mode_in(MODE, kH);
    constexpr int NKB = IN / 64;               // K-blocks of the first operand
    constexpr int CH = IN / 8;                 // 16-byte chunks per operand row
    const int depth = a.depth;
    const int last = MODE == MODE_DEC ? depth - 1 : depth;
    const WsPlan P = ws_plan(MODE, depth, NG, S);
    unsigned char* W = sm + P.w;
    unsigned char* A0 = sm + P.a0;
    unsigned char* A1 = sm + P.a1;
    float* bias = reinterpret_cast<float*>(sm + P.bias);
    float* s_out = bias + (depth + 1) * kH;    // decoder scalar layer: W[64], b
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + P.bars);
    uint64_t* empty = full + kWsStages;
    uint64_t* mbar = empty + kWsStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + P.tslot);
    int* sgen = reinterpret_cast<int*>(sm + P.gen);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- weights (BF16, swizzled K-blocks) and biases, once per CTA
    {
        const float* src = a.w;
        uint32_t woff = 0;
        for (int l = 0; l <= depth; ++l) {
            const int fi = l == 0 ? IN : kH, fo = (MODE == MODE_DEC && l == depth) ? 1 : kH;
            if (l <= last) {
                for (int t = tid; t < fo * fi; t += kWsThreads) {
                    const int n = t / fi, k = t % fi;
                    unsigned char* blk = W + woff + (uint32_t)(k / 64) * (kH * 128);
                    *reinterpret_cast<__nv_bfloat16*>(blk + swz(n, k % 64)) = __float2bfloat16_rn(src[t]);
                }
                woff += (uint32_t)(fi / 64) * (kH * 128);
                for (int t = tid; t < fo; t += kWsThreads) bias[l * kH + t] = src[fi * fo + t];
            } else {                            // decoder scalar output layer
                for (int t = tid; t < kH; t += kWsThreads) s_out[t] = src[t];
                if (tid == 0) s_out[kH] = src[kH];
            }
            src += fi * fo + fo;
        }
    }
    if (tid == 0) {
        for (int s = 0; s < kWsStages; ++s) {
            ws_bar_init(&full[s], 32);
            ws_bar_init(&empty[s], 1);
        }
        for (int g = 0; g < NG; ++g) ws_bar_init(&mbar[g], 1);
        for (int q = 0; q < S; ++q) sgen[q] = -1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(tmem_slot)),
                     "n"(ws_tmem_cols(NG))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t ntiles = (a.nrows + kM - 1) / kM;
    bool ok = true;

    if (warp == NG * kM / 32) {
        // ---------------- producer warp: operand rows of tile j into stage j % S
        int nrow[4], ncol[4];
        auto load_idx = [&](int64_t tile) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t k = tile * kM + lane + 32 * q;
                const bool in = tile < ntiles && k < a.nrows;
                nrow[q] = in && MODE == MODE_EDGE ? a.erow[k] : 0;
                ncol[q] = in && MODE == MODE_EDGE ? a.ci[k] : 0;
            }
        };
        load_idx(blockIdx.x);
        for (int64_t j = 0;; ++j) {
            const int64_t tile = blockIdx.x + j * gridDim.x;
            if (tile >= ntiles) break;
            const int s = (int)(j % kWsStages);
            if (j >= kWsStages) {
                if (!bar_wait(&empty[s], (uint32_t)(((j / kWsStages) - 1) & 1))) {
                    ok = false;
                    break;
                }
            }
            // the stage is free for tile j (its previous tile j - S was read)
            if (lane == 0) *reinterpret_cast<volatile int*>(sgen + s) = (int)j;
            unsigned char* dst = A0 + (uint32_t)s * NKB * (kM * 128);
            int crow[4], ccol[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { crow[q] = nrow[q]; ccol[q] = ncol[q]; }
            // eight lanes per 128-byte row segment, four rows per instruction:
            // every copy instruction reads whole lines (lane l of the warp
            // holds the indices of rows l, l + 32, l + 64, l + 96)
            const int rsub = lane >> 3, cc = lane & 7;
#pragma unroll
            for (int i = 0; i < kM / 4; ++i) {
                const int r = 4 * i + rsub;
                const int64_t k = tile * kM + r;
                const bool in = k < a.nrows;
                const int jr = __shfl_sync(0xffffffffu, crow[i >> 3], r & 31);
                const int jc = __shfl_sync(0xffffffffu, ccol[i >> 3], r & 31);
#pragma unroll
                for (int seg = 0; seg < NKB; ++seg) {
                    const __nv_bfloat16* src = seg == 0 ? a.ein + (in ? k : 0) * kH
                                             : seg == 1 ? a.vin + (int64_t)jr * kH
                                                        : a.vin + (int64_t)jc * kH;
                    cp_async16(s_addr(dst + (uint32_t)seg * (kM * 128) + swz(r, cc * 8)), src + cc * 8, in ? 16u : 0u);
                }
            }
            cp_async_arrive(&full[s]);
            load_idx(tile + gridDim.x);          // the next tile's indices, under this tile's copies
        }
        cp_async_wait<0>();                      // no copy may land after the CTA leaves
        if (!ok) atomicOr(a.flags, kFlagTimeout);
    } else {
        // ---------------- epilogue warpgroup g: tiles j = g, g + 2, ...
        const int g = warp >> 2, r = tid & (kM - 1);
        const uint32_t acc_col = tmem + (uint32_t)(g * kH);
        const uint32_t my_lanes = acc_col + ((uint32_t)((warp & 3) * 32) << 16);
        unsigned char* A1g = A1 + (uint32_t)g * (kM * 128);
        uint32_t mphase = 0;
        const bool elected = r == 0;
        for (int64_t j = g;; j += NG) {
            const int64_t tile = blockIdx.x + j * gridDim.x;
            if (tile >= ntiles) break;
            const int s = (int)(j % kWsStages);
            // A parity wait tells only the last two phases of a stage apart.
            // With more warpgroups than stages this warpgroup can ask for tile
            // j while the stage still waits for tile j - S, whose phase has
            // the other parity but is not the one wanted; it first waits
            // (bounded) until the producer has started tile j in the stage.
            bool got = true;
            if constexpr (NG > S) {
                long long spins = 0;
                while (*reinterpret_cast<volatile int*>(sgen + s) < (int)j)
                    if (++spins >= kWaitSpin) { got = false; break; }
            }
            got = got && bar_wait(&full[s], (uint32_t)((j / kWsStages) & 1));
            if (!group_agree(g, got)) { ok = false; break; }
            tc_fence_after();
            uint32_t woff = 0;
            const int64_t row = tile * kM + r;
            for (int l = 0; l <= last; ++l) {
                const int kin = l == 0 ? IN : kH;
                if (elected) {
                    // the operand rows landed through cp.async (observed on the
                    // stage's barrier) or generic stores: order them before the
                    // tensor core's reads
                    fence_async_smem();
                    const uint32_t abase = l == 0 ? s_addr(A0 + (uint32_t)s * NKB * (kM * 128)) : s_addr(A1g);
                    const uint32_t wbase = s_addr(W + woff);
                    for (int q = 0; q < kin / 16; ++q) {
                        const uint32_t kb = (uint32_t)(q >> 2), ko = (uint32_t)(q & 3) * 32;
                        mma_bf16(acc_col, smem_desc(abase + kb * (kM * 128) + ko),
                                 smem_desc(wbase + kb * (kH * 128) + ko), q > 0 ? 1u : 0u);
                    }
                    if (l == 0) mma_commit(&empty[s]);      // the operand stage is free once read
                    mma_commit(&mbar[g]);
                }
                woff += (uint32_t)(kin / 64) * (kH * 128);
                const bool done = bar_wait(&mbar[g], mphase);
                mphase ^= 1u;
                if (!group_agree(g, done)) { ok = false; break; }
                tc_fence_after();
                float v[64];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float t16[16];
                    tmem_ld16(my_lanes + q * 16, t16);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[q * 16 + i] = t16[i];
                }
                tmem_wait_ld();
                const float* bl = bias + l * kH;
                if (l < last || (MODE != MODE_DEC && l < depth)) {
                    // the next layer's operand (its previous reader has completed)
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        __nv_bfloat16 h8[8];
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) h8[jj] = __float2bfloat16_rn(fmaxf(v[c * 8 + jj] + bl[c * 8 + jj], 0.0f));
                        *reinterpret_cast<uint4*>(A1g + swz(r, c * 8)) = *reinterpret_cast<uint4*>(h8);
                    }
                    fence_async_smem();
                    tc_fence_before();
                    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kM) : "memory");
                    tc_fence_after();
                } else if (MODE == MODE_DEC) {
                    float sacc = s_out[kH];
#pragma unroll
                    for (int o = 0; o < kH; ++o) sacc = fmaf(s_out[o], fmaxf(v[o] + bl[o], 0.0f), sacc);
                    if (row < a.nrows) a.sout[row] = sacc;
                } else {
                    // the output row goes through the warpgroup's operand
                    // buffer (its last reader, this layer's product, has
                    // completed), so that the global stores are whole lines
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        __nv_bfloat16 h8[8];
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) h8[jj] = __float2bfloat16_rn(v[c * 8 + jj] + bl[c * 8 + jj]);
                        *reinterpret_cast<uint4*>(A1g + swz(r, c * 8)) = *reinterpret_cast<uint4*>(h8);
                    }
                    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kM) : "memory");
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int rr = i * 16 + (r >> 3), cc = r & 7;
                        const int64_t orow = tile * kM + rr;
                        if (orow < a.nrows)
                            *reinterpret_cast<uint4*>(a.out + orow * kH + cc * 8) =
                                *reinterpret_cast<const uint4*>(A1g + swz(rr, cc * 8));
                    }
                    if (row < a.nrows) {
                        if (a.out32) {
                            float4* o = reinterpret_cast<float4*>(a.out32 + row * kH);
#pragma unroll
                            for (int c = 0; c < 16; ++c)
                                o[c] = make_float4(v[4 * c] + bl[4 * c], v[4 * c + 1] + bl[4 * c + 1],
                                                   v[4 * c + 2] + bl[4 * c + 2], v[4 * c + 3] + bl[4 * c + 3]);
                        }
                    }
                }
            }
            if (!ok) break;
            // this tile's accumulator reads are done before the next tile's
            // first product is issued into it
            tc_fence_before();
            asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kM) : "memory");
            tc_fence_after();
        }
        if (!ok) {
            // a product still in flight gets one more bounded wait before the
            // tensor memory is released
            bar_wait(&mbar[g], mphase);
            if (r == 0) atomicOr(a.flags, kFlagTimeout);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(ws_tmem_cols(NG))
                     : "memory");
}

template <int MODE, int NG, int S>
bool launch_ws(Handle* h, const Bf16Args& a, npcg_status* st) {
    const WsPlan p = ws_plan(MODE, a.depth, NG, S);
    const size_t smem = p.total + 1024;   // alignment slack
    if (smem > 227 * 1024) return false;
    *st = NPCG_OK;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_bf16_ws<MODE, NG, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) { *st = cuda_fail(h, e, "cudaFuncSetAttribute(k_mlp_bf16_ws)"); return true; }
    const int64_t ntiles = (a.nrows + kM - 1) / kM;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)h->num_sms));
    k_mlp_bf16_ws<MODE, NG, S><<<grid, ws_threads(NG), smem, h->stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) *st = cuda_fail(h, e, "k_mlp_bf16_ws");
    return true;
}

template <int MODE>
npcg_status launch_bf16(Handle* h, const Bf16Args& a) {
    if (a.nrows == 0) return NPCG_OK;
    if constexpr (MODE == MODE_EDGE || MODE == MODE_DEC) {
        // three tiles in flight per SM where three operand stages fit beside
        // them, else three tiles over two stages, else two tiles over three
        npcg_status st = NPCG_OK;
        if (launch_ws<MODE, 3, 3>(h, a, &st)) return st;
        if (launch_ws<MODE, 3, 2>(h, a, &st)) return st;
        if (launch_ws<MODE, 2, 3>(h, a, &st)) return st;
    }
    const SmemPlan p = plan(MODE, a.depth);
    const size_t smem = p.total + 1024;       // alignment slack
    if (smem > 227 * 1024) return set_error(h, NPCG_EINVAL, "MLP too deep for the BF16 kernel");
    NPCG_CUDA(h, cudaFuncSetAttribute(k_mlp_bf16<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int per_sm = std::max(1, std::min(3, (int)((227 * 1024) / (smem + 1024))));
    const int64_t ntiles = (a.nrows + kM - 1) / kM;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)h->num_sms * per_sm));
    k_mlp_bf16<MODE><<<grid, kThreads, smem, h->stream>>>(a);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

}  // namespace

npcg_status gnn_scales_run(Handle* h, Pattern* P, const double* A_val, const double* b, double* sc);

// Forward on the tensor cores: decoder outputs into sout; with tV/tE/tAGG
// (n_mp + 1, n_mp + 1 and n_mp FP32 buffers) also the training tape of
// node / edge states and aggregations.
npcg_status gnn_bf16_forward_core(Handle* h, Pattern* P, const double* A_val, const double* b,
                                  const npcg_gnn_config* cfg, const float* w, double* sc, float* sout,
                                  float* const* tV, float* const* tE, float* const* tAGG) {
    if (cfg->h != kH) return set_error(h, NPCG_EINVAL, "the BF16 tensor-core path needs hidden width h = 64");
    GnnStore& S = P->gnn;
    const size_t fe = (size_t)P->nnz * kH, fv = (size_t)P->n * kH;
    NPCG_CUDA(h, S.bf.ensure(2 * (fe + fv)));
    __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(S.bf.p);
    __nv_bfloat16* V[2] = {base, base + fv};
    __nv_bfloat16* E[2] = {base + 2 * fv, base + 2 * fv + fe};
    NPCG_TRY(gnn_scales_run(h, P, A_val, b, sc));
    NPCG_CUDA(h, cudaMemsetAsync(P->ctl.p + 1, 0, sizeof(int), h->stream));
    const GnnOffsets off = gnn_offsets(kH, cfg->l, cfg->l_mp, cfg->n_mp);
    Bf16Args a{};
    a.rp = P->rp.p;
    a.ci = P->ci.p;
    a.erow = P->edge_row.p;
    a.row_sys = P->row_sys.p;
    a.sc = sc;
    a.av = A_val;
    a.b = b;
    a.flags = P->ctl.p + 1;
    a.adiag_scaled = cfg->diag_mode == NPCG_DIAG_LDLT_ROWS ? P->adiag.p : nullptr;
    a.nrows = P->n; a.w = w + off.enc_v; a.depth = cfg->l; a.out = V[0]; a.out32 = tV ? tV[0] : nullptr;
    NPCG_TRY(launch_bf16<MODE_ENC_NODE>(h, a));
    a.nrows = P->nnz; a.w = w + off.enc_e; a.depth = cfg->l; a.out = E[0]; a.out32 = tE ? tE[0] : nullptr;
    NPCG_TRY(launch_bf16<MODE_ENC_EDGE>(h, a));
    for (int t = 0; t < cfg->n_mp; ++t) {
        const int c = t & 1;
        a.nrows = P->n; a.w = w + off.node[t]; a.depth = cfg->l_mp; a.vin = V[c]; a.ein = E[c]; a.out = V[c ^ 1];
        a.out32 = tV ? tV[t + 1] : nullptr;
        a.agg32 = tAGG ? tAGG[t] : nullptr;
        NPCG_TRY(launch_bf16<MODE_NODE>(h, a));
        a.agg32 = nullptr;
        a.nrows = P->nnz; a.w = w + off.edge[t]; a.depth = cfg->l_mp; a.vin = V[c ^ 1]; a.ein = E[c]; a.out = E[c ^ 1];
        a.out32 = tE ? tE[t + 1] : nullptr;
        NPCG_TRY(launch_bf16<MODE_EDGE>(h, a));
    }
    a.nrows = P->nnz; a.w = w + off.dec; a.depth = cfg->l; a.ein = E[cfg->n_mp & 1]; a.out = nullptr;
    a.out32 = nullptr; a.sout = sout;
    NPCG_TRY(launch_bf16<MODE_DEC>(h, a));
    return NPCG_OK;
}

npcg_status gnn_bf16_check_flags(Handle* h, Pattern* P) {
    int flags = 0;
    NPCG_TRY(read_scalar(h, P->ctl.p + 1, &flags));
    if (flags & kFlagTimeout) return set_error(h, NPCG_ETIMEOUT, "tensor-core MLP wait timed out");
    return NPCG_OK;
}

// initial-guess head on the final BF16 node features of the last forward
// (the decoder's tensor-core MLP over node rows)
npcg_status gnn_bf16_head_run(Handle* h, Pattern* P, const npcg_gnn_config* cfg, const float* w_head, float* out) {
    GnnStore& S = P->gnn;
    const size_t fv = (size_t)P->n * kH;
    const __nv_bfloat16* V = reinterpret_cast<const __nv_bfloat16*>(S.bf.p) + (cfg->n_mp & 1) * fv;
    NPCG_CUDA(h, cudaMemsetAsync(P->ctl.p + 1, 0, sizeof(int), h->stream));
    Bf16Args a{};
    a.rp = P->rp.p;
    a.ci = P->ci.p;
    a.erow = P->edge_row.p;
    a.row_sys = P->row_sys.p;
    a.sc = S.sc.p;
    a.flags = P->ctl.p + 1;
    a.nrows = P->n;
    a.w = w_head;
    a.depth = cfg->l;
    a.ein = V;
    a.sout = out;
    NPCG_TRY(launch_bf16<MODE_DEC>(h, a));
    return gnn_bf16_check_flags(h, P);
}

npcg_status gnn_forward_bf16_run(Handle* h, Pattern* P, const double* A_val, const double* b,
                                 const npcg_gnn_config* cfg, const float* w, double* L_val) {
    GnnStore& S = P->gnn;
    NPCG_CUDA(h, S.s.ensure(P->nnz));
    NPCG_CUDA(h, S.sc.ensure((size_t)2 * P->nsys));
    NPCG_TRY(gnn_bf16_forward_core(h, P, A_val, b, cfg, w, S.sc.p, S.s.p, nullptr, nullptr, nullptr));
    GnnBuffers gb{};
    gb.s = S.s.p;
    gb.sc = S.sc.p;
    gb.av = A_val;
    gb.diag_mode = cfg->diag_mode;
    NPCG_TRY(gnn_assemble_L(h, P, gb, L_val));
    return gnn_bf16_check_flags(h, P);
}

}  // namespace npcg
