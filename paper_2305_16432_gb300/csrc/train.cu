// Training: the loss Eq. (loss_Ab),
//   loss = mean over pairs p and systems s of || L L^T x_p - b_p ||^2,
// with each pair's L from its own network forward (the node input is b_p,
// Sec. 4.1), and its hand-written adjoint back to the network weights; Adam
// (App. A.4) updates the FP32 master weights.
//
// Adjoint of the loss in L (y = L^T x, u = L y, r = u - b, w = L^T r):
//   d loss / d L_ij = c (r_i y_j + x_i w_j),  c = 2 / (npairs nsys),
// then through L_ij = sqrt(s) (s_ij + s_ji)/2, L_ii = sqrt(s) softplus(s_ii),
// the decoder, the message-passing layers in reverse, and the encoders.
// Every MLP backward recomputes its activations per tile from the layer
// input (kept in a feature tape), writes the per-layer output gradients and
// activations, and the weight gradients are reduced from those by a split
// reduction kernel.  FP32 throughout the network; the loss part is FP64.
#include <algorithm>
#include <array>
#include <vector>

#include <cuda_bf16.h>

#include "gnn_common.cuh"
#include "tc_common.cuh"

namespace npcg {

namespace {

// ------------------------------------------------------------ loss in L (FP64)
// y_j = sum_i L_ij x_i over column j of L = entries (j, c), c >= j, of row j of A
__global__ void k_lt_mv(int64_t n, const int32_t* rp, const int32_t* ci, const int32_t* mirror,
                        const int32_t* a2l, const double* Lv, const double* x, double* y) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = rp[j]; k < rp[j + 1]; ++k) {
            const int c = ci[k];
            if (c >= j) s = fma(Lv[a2l[mirror[k]]], x[c], s);
        }
        y[j] = s;
    }
}

// u = L y, r = u - b, per-system sum of r^2
__global__ void k_l_mv_res(int64_t n, const int32_t* Lrp, const int32_t* Lci, const double* Lv,
                           const double* y, const double* b, const int32_t* row_sys, double* r,
                           double* loss_sys) {
    // warp-uniform loop so the whole warp takes part in the reduction
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = w0; base < n; base += stride) {
        const int64_t i = base + lane;
        const bool valid = i < n;
        double v = 0.0;
        int sys = row_sys[base];
        if (valid) {
            double u = 0.0;
            for (int q = Lrp[i]; q < Lrp[i + 1]; ++q) u = fma(Lv[q], y[Lci[q]], u);
            const double ri = u - b[i];
            r[i] = ri;
            v = ri * ri;
            sys = row_sys[i];
        }
        // one atomic per warp when its rows share a system, else one per row
        if (__all_sync(0xffffffffu, sys == __shfl_sync(0xffffffffu, sys, 0))) {
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) atomicAdd(&loss_sys[sys], v);
        } else if (valid) {
            atomicAdd(&loss_sys[sys], v);
        }
    }
}

// dL_q = c (r_i y_j + x_i w_j) for q = (i, j)
__global__ void k_dL(int64_t nnzL, const int32_t* l2a, const int32_t* erow, const int32_t* ci, double c,
                     const double* r, const double* y, const double* x, const double* w, double* dL) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnzL;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int ka = l2a[q];
        const int i = erow[ka], j = ci[ka];
        dL[q] = c * (r[i] * y[j] + x[i] * w[j]);
    }
}

// d loss / d s_k for every A entry k = (i, j): one L entry feeds each.
// diag_mode 1: L_ii = sqrt(A_ii) is fixed, L_ij = sqrt(A_jj) (s_ij + s_ji)/2;
// diag_mode 2: L_ii = sqrt(A_ii) is fixed, L_ij = sqrt(A_ii) (s_ij + s_ji)/2.
__global__ void k_dS(int64_t nnz, const int32_t* erow, const int32_t* ci, const int32_t* mirror,
                     const int32_t* a2l, const int32_t* row_sys, const double* sc, const float* S,
                     const double* dL, const double* av, const int32_t* adiag, int diag_mode, float* dS) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int i = erow[k], j = ci[k];
        double g;
        if (diag_mode == 1 || diag_mode == 2) {
            // the L entry holding s_k is (max(i,j), min(i,j)); its scale is
            // sqrt(A_cc) with c the column min(i,j) (mode 1) or the row max(i,j) (mode 2)
            const int cc = diag_mode == 1 ? min(i, j) : max(i, j);
            if (i == j) g = 0.0;
            else if (i > j) g = sqrt(av[adiag[cc]]) * 0.5 * dL[a2l[k]];
            else g = sqrt(av[adiag[cc]]) * 0.5 * dL[a2l[mirror[k]]];
        } else {
            const double rs = sqrt(sc[2 * row_sys[i]]);
            if (i == j) g = rs * (1.0 / (1.0 + exp(-(double)S[k]))) * dL[a2l[k]];
            else if (i > j) g = rs * 0.5 * dL[a2l[k]];
            else g = rs * 0.5 * dL[a2l[mirror[k]]];
        }
        dS[k] = (float)g;
    }
}

// ------------------------------------------------------------ MLP backward
struct MlpBwdArgs {
    MlpArgs f;                        // forward gather (rows, weights, depth, inputs)
    const float* gout;                // upstream gradient [rows x OUT]
    float* tapeA[kMaxDepth + 1];      // [l] activations A_l (input of Linear l), l = 1..depth
    float* tapeG[kMaxDepth + 1];      // [l] gradient of Linear l's output, l = 0..depth-1
    float* dx[3];                     // input-gradient segments (H wide each)
};

// acc[i][j] = sum_k A[(r0+i)*lda + k] * B[k*ldb_k + (c0 + o0 + j)*ldb_n]
template <int H>
__device__ __forceinline__ void mm_rows(const float* A, int lda, const float* B, int ldb_k, int ldb_n, int K,
                                        int c0, float (&acc)[4][4]) {
    const int to = threadIdx.x % Tile<H>::TO, tr = threadIdx.x / Tile<H>::TO;
    const int r0 = tr * 4, o0 = c0 + to * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k = 0; k < K; ++k) {
        float a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = A[(r0 + i) * lda + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = B[k * ldb_k + (o0 + j) * ldb_n];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
}

__host__ __device__ constexpr int bwd_ldw(int in) { return in + 1; }

inline size_t bwd_smem_floats(int mode, int H, int depth) {
    const int in = mode_in(mode, H), out = mode_out(mode, H), R = 4096 / H;
    size_t w = (size_t)H * bwd_ldw(in) + H + (size_t)(depth - 1) * (H * bwd_ldw(H) + H) +
               (size_t)out * bwd_ldw(H) + out;
    w = (w + 3) & ~size_t(3);
    return w + (size_t)R * (in + 1) + (size_t)depth * R * (H + 1) + 2 * (size_t)R * (H + 1) + 4;
}

template <int H, int MODE>
__global__ void __launch_bounds__(256) k_mlp_bwd(MlpBwdArgs a) {
    extern __shared__ __align__(16) float sm[];
    constexpr int R = Tile<H>::R;
    constexpr int IN = mode_in(MODE, H);
    constexpr int OUT = mode_out(MODE, H);
    const int depth = a.f.depth;
    // weights row-major with padded rows (ld = in + 1), biases after each
    float* Wl[kMaxDepth + 1];
    float* bl[kMaxDepth + 1];
    {
        float* dst = sm;
        const float* src = a.f.w;
        for (int l = 0; l <= depth; ++l) {
            const int fi = l == 0 ? IN : H, fo = l == depth ? OUT : H, ld = bwd_ldw(fi);
            for (int t = threadIdx.x; t < fi * fo; t += blockDim.x) dst[(t / fi) * ld + t % fi] = src[t];
            for (int t = threadIdx.x; t < fo; t += blockDim.x) dst[fo * ld + t] = src[fi * fo + t];
            Wl[l] = dst;
            bl[l] = dst + fo * ld;
            dst += fo * ld + fo;
            src += fi * fo + fo;
        }
    }
    size_t wfl = (size_t)H * bwd_ldw(IN) + H + (size_t)(depth - 1) * (H * bwd_ldw(H) + H) +
                 (size_t)OUT * bwd_ldw(H) + OUT;
    wfl = (wfl + 3) & ~size_t(3);
    float* X = sm + wfl;
    float* Ab = X + R * (IN + 1);                 // depth buffers [R][H+1]
    float* G0 = Ab + (size_t)depth * R * (H + 1);
    float* G1 = G0 + R * (H + 1);
    __syncthreads();
    const int to = threadIdx.x % Tile<H>::TO, tr = threadIdx.x / Tile<H>::TO;
    const int64_t ntiles = (a.f.nrows + R - 1) / R;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row0 = tile * R;
        gather_tile<H, MODE>(a.f, row0, X);
        __syncthreads();
        // forward recompute of the hidden activations A_1..A_depth
        const float* in = X;
        int ldin = IN + 1, kin = IN;
        for (int l = 0; l < depth; ++l) {
            float acc[4][4];
            mm_rows<H>(in, ldin, Wl[l], 1, bwd_ldw(kin), kin, 0, acc);
            float* A = Ab + (size_t)l * R * (H + 1);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = tr * 4 + i, o = to * 4 + j;
                    const float v = fmaxf(acc[i][j] + bl[l][o], 0.0f);
                    A[r * (H + 1) + o] = v;
                    if (row0 + r < a.f.nrows) a.tapeA[l + 1][(row0 + r) * H + o] = v;
                }
            __syncthreads();
            in = A;
            ldin = H + 1;
            kin = H;
        }
        // upstream gradient of the last Linear
        for (int t = threadIdx.x; t < R * OUT; t += blockDim.x) {
            const int r = t / OUT, o = t % OUT;
            G0[r * (H + 1) + o] = row0 + r < a.f.nrows ? a.gout[(row0 + r) * OUT + o] : 0.0f;
        }
        __syncthreads();
        float* G = G0;
        float* Gn = G1;
        for (int l = depth; l >= 1; --l) {
            // gradient at A_l: G (R x out_l) . W_l (out_l x H), masked by A_l > 0
            const int ol = l == depth ? OUT : H;
            float acc[4][4];
            mm_rows<H>(G, H + 1, Wl[l], bwd_ldw(H), 1, ol, 0, acc);
            const float* A = Ab + (size_t)(l - 1) * R * (H + 1);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = tr * 4 + i, o = to * 4 + j;
                    const float v = A[r * (H + 1) + o] > 0.0f ? acc[i][j] : 0.0f;
                    Gn[r * (H + 1) + o] = v;
                    if (row0 + r < a.f.nrows) a.tapeG[l - 1][(row0 + r) * H + o] = v;
                }
            __syncthreads();
            float* t = G; G = Gn; Gn = t;
        }
        // gradient of the MLP input: G_0 (R x H) . W_0 (H x IN), by H-wide segments
        if (MODE != MODE_ENC_NODE && MODE != MODE_ENC_EDGE) {
            for (int seg = 0; seg < IN / H; ++seg) {
                float acc[4][4];
                mm_rows<H>(G, H + 1, Wl[0], bwd_ldw(IN), 1, H, seg * H, acc);
                float* dst = a.dx[seg];
                if (!dst) continue;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int64_t row = row0 + tr * 4 + i;
                    if (row < a.f.nrows)
                        *reinterpret_cast<float4*>(dst + row * H + to * 4) =
                            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                }
            }
        }
        __syncthreads();
    }
}

template <int H, int MODE>
npcg_status launch_bwd_mode(Handle* h, const MlpBwdArgs& a) {
    if (a.f.nrows == 0) return NPCG_OK;
    const size_t smem = bwd_smem_floats(MODE, H, a.f.depth) * sizeof(float);
    if (smem > 227 * 1024) return set_error(h, NPCG_EINVAL, "MLP too deep for the backward kernel");
    NPCG_CUDA(h, cudaFuncSetAttribute(k_mlp_bwd<H, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (227 * 1024) / (smem + 1024)));
    const int64_t ntiles = (a.f.nrows + Tile<H>::R - 1) / Tile<H>::R;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)h->num_sms * per_sm));
    k_mlp_bwd<H, MODE><<<grid, 256, smem, h->stream>>>(a);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

template <int H>
npcg_status launch_bwd(Handle* h, int mode, const MlpBwdArgs& a) {
    switch (mode) {
        case MODE_ENC_NODE: return launch_bwd_mode<H, MODE_ENC_NODE>(h, a);
        case MODE_ENC_EDGE: return launch_bwd_mode<H, MODE_ENC_EDGE>(h, a);
        case MODE_NODE: return launch_bwd_mode<H, MODE_NODE>(h, a);
        case MODE_EDGE: return launch_bwd_mode<H, MODE_EDGE>(h, a);
        default: return launch_bwd_mode<H, MODE_DEC>(h, a);
    }
}

// ---- MLP backward on the tensor cores (BF16 operands, FP32 accumulate)
// Per 128-row tile: the layer input is gathered from the FP32 tapes into the
// swizzled K-major BF16 operand (the forward's BF16 operands are the BF16
// roundings of these tapes, so the recompute reproduces them); the hidden
// activations A_1..A_depth are recomputed (tapeA, ReLU masks kept as bits);
// then G_{l-1} = (G_l W_l) (.) [A_l > 0] down the layers (tapeG) and the
// input gradient G_0 W_0 by 64-wide segments.  Backward products use W_l^T,
// staged once per CTA: B[i][o] = W_l[o][i] (K = o).  The node update reads
// its aggregation from the forward's tape.
struct BtPlan {
    uint32_t a0, ah, g, wf, wb, bias, misc, st, total;
};
__host__ __device__ inline BtPlan bt_plan(int in, int depth, bool dec) {
    BtPlan p;
    const uint32_t blk = kM * 128;                                  // [128 x 64] BF16
    const uint32_t wblk = kH * 128;                                 // [64 x 64] BF16
    p.a0 = 0;
    p.ah = p.a0 + (uint32_t)(in / 64) * blk;                        // A_1..A_depth
    p.g = p.ah + (uint32_t)depth * blk;                             // gradient operand
    p.wf = p.g + blk;                                               // forward W_0..W_{depth-1}
    p.wb = p.wf + (uint32_t)(in / 64) * wblk + (uint32_t)(depth - 1) * wblk;
    // backward W_l^T: l = 0 (in/64 blocks), 1..depth-1, depth (unless scalar)
    p.bias = p.wb + (uint32_t)(in / 64) * wblk + (uint32_t)(depth - 1 + (dec ? 0 : 1)) * wblk;
    p.misc = p.bias + (uint32_t)(depth + 1) * kH * 4;
    // FP32 staging of half a tile (128 rows x 32 columns): rows move between
    // registers and global memory through it as whole lines
    p.st = (p.misc + 64 + 127) & ~127u;
    p.total = p.st + kM * 32 * 4;
    return p;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_mlp_bwd_tc(MlpBwdArgs a, const float* agg_in, int* flags) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((1024u - (s_addr(sm_raw) & 1023u)) & 1023u);
    constexpr int IN = mode_in(MODE, kH);
    constexpr bool kDec = MODE == MODE_DEC;
    constexpr int NKB = IN / 64;
    const int depth = a.f.depth;
    const BtPlan P = bt_plan(IN, depth, kDec);
    unsigned char* A0 = sm + P.a0;
    unsigned char* Ah = sm + P.ah;
    unsigned char* Gop = sm + P.g;
    unsigned char* Wf = sm + P.wf;
    unsigned char* Wb = sm + P.wb;
    float* bias = reinterpret_cast<float*>(sm + P.bias);       // [depth][64]; [depth] = scalar layer W (DEC)
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P.misc);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + P.misc + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t blk = kM * 128, wblk = kH * 128;

    // ---- stage weights (BF16, K-major) and biases
    {
        const float* src = a.f.w;
        for (int l = 0; l <= depth; ++l) {
            const int fi = l == 0 ? IN : kH, fo = (kDec && l == depth) ? 1 : kH;
            if (l < depth) {
                // forward: B rows = output o, K = input i
                unsigned char* base = Wf + (l == 0 ? 0u : (uint32_t)NKB * wblk + (uint32_t)(l - 1) * wblk);
                for (int t = tid; t < fo * fi; t += kThreads) {
                    const int o = t / fi, i = t % fi;
                    *reinterpret_cast<__nv_bfloat16*>(base + (uint32_t)(i / 64) * wblk + swz(o, i % 64)) =
                        __float2bfloat16_rn(src[t]);
                }
                for (int t = tid; t < kH; t += kThreads) bias[l * kH + t] = src[fi * fo + t];
            }
            if (!(kDec && l == depth)) {
                // backward: B rows = input i, K = output o
                unsigned char* base = Wb + (l == 0 ? 0u : (uint32_t)NKB * wblk + (uint32_t)(l - 1) * wblk);
                for (int t = tid; t < fo * fi; t += kThreads) {
                    const int o = t / fi, i = t % fi;
                    *reinterpret_cast<__nv_bfloat16*>(base + (uint32_t)(i / 64) * wblk + swz(i % 64, o)) =
                        __float2bfloat16_rn(src[t]);
                }
            } else {
                for (int t = tid; t < kH; t += kThreads) bias[depth * kH + t] = src[t];   // W_depth[0][i]
            }
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

    // one MMA chain D = A (128 x 64*nkb) . B^T, then wait; false on timeout
    auto mma_wait = [&](const unsigned char* Aop, const unsigned char* Bop, int nkb) -> bool {
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            const uint32_t abase = s_addr(Aop), bbase = s_addr(Bop);
            for (int s = 0; s < nkb * 4; ++s) {
                const uint32_t kb = (uint32_t)(s >> 2), ko = (uint32_t)(s & 3) * 32;
                mma_bf16(tmem, smem_desc(abase + kb * blk + ko), smem_desc(bbase + kb * wblk + ko), s > 0 ? 1u : 0u);
            }
            mma_commit(bar);
        }
        bool w = bar_wait(bar, phase);
        phase ^= 1u;
        if (!__syncthreads_and(w)) return false;
        tc_fence_after();
        return true;
    };
    auto ld64 = [&](float (&v)[64]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float t16[16];
            tmem_ld16(my_lanes + q * 16, t16);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[q * 16 + i] = t16[i];
        }
        tmem_wait_ld();
    };
    // row tid of a [128 x 64] operand from 64 FP32 values
    auto put_row = [&](unsigned char* Op, const float (&v)[64]) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            __nv_bfloat162 h2[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) h2[j] = __floats2bfloat162_rn(v[c * 8 + 2 * j], v[c * 8 + 2 * j + 1]);
            *reinterpret_cast<uint4*>(Op + swz(tid, c * 8)) = *reinterpret_cast<uint4*>(h2);
        }
    };
    // Rows of the tile (row0 + tid) to / from global memory through the
    // staging buffer, 32 columns at a time: thread tid owns row tid in
    // registers; in the staging buffer 16-byte chunk c of row r sits at
    // c ^ (r & 7) (no bank conflicts either way), and the global side moves
    // four rows' 128-byte halves per warp instruction.  Every thread of the
    // CTA calls these.
    float4* stg = reinterpret_cast<float4*>(sm + P.st);
    auto store_rows = [&](float* dst, int64_t row0, const float (&v)[64]) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int o = h * 32 + c * 4;
                stg[tid * 8 + (c ^ (tid & 7))] = make_float4(v[o], v[o + 1], v[o + 2], v[o + 3]);
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int idx = i * kThreads + tid, rr = idx >> 3, cc = idx & 7;
                if (row0 + rr < a.f.nrows)
                    reinterpret_cast<float4*>(dst + (row0 + rr) * kH + h * 32)[cc] = stg[rr * 8 + (cc ^ (rr & 7))];
            }
            __syncthreads();
        }
    };
    auto load_rows = [&](const float* src, int64_t row0, float (&v)[64]) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int idx = i * kThreads + tid, rr = idx >> 3, cc = idx & 7;
                stg[rr * 8 + (cc ^ (rr & 7))] =
                    row0 + rr < a.f.nrows ? reinterpret_cast<const float4*>(src + (row0 + rr) * kH + h * 32)[cc]
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 q = stg[tid * 8 + (c ^ (tid & 7))];
                const int o = h * 32 + c * 4;
                v[o] = q.x; v[o + 1] = q.y; v[o + 2] = q.z; v[o + 3] = q.w;
            }
            __syncthreads();
        }
    };

    const int64_t ntiles = (a.f.nrows + kM - 1) / kM;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t row0 = tile * kM, row = row0 + tid;
        const bool live = row < a.f.nrows;
        // ---- layer input: 8-feature chunks of the FP32 tapes -> BF16 operand
        for (int idx = tid; idx < kM * (IN / 8); idx += kThreads) {
            const int r = idx / (IN / 8), c = idx % (IN / 8);
            const int64_t k = row0 + r;
            float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
            if (k < a.f.nrows) {
                const int seg = c >> 3, cc = c & 7;
                const float* src;
                if (MODE == MODE_EDGE)
                    src = seg == 0 ? a.f.ein + k * kH : seg == 1 ? a.f.vin + (int64_t)a.f.erow[k] * kH
                                                                 : a.f.vin + (int64_t)a.f.ci[k] * kH;
                else if (MODE == MODE_NODE)
                    src = seg == 0 ? a.f.vin + k * kH : agg_in + k * kH;
                else
                    src = a.f.ein + k * kH;
                x0 = *reinterpret_cast<const float4*>(src + cc * 8);
                x1 = *reinterpret_cast<const float4*>(src + cc * 8 + 4);
            }
            __nv_bfloat162 h2[4] = {__floats2bfloat162_rn(x0.x, x0.y), __floats2bfloat162_rn(x0.z, x0.w),
                                    __floats2bfloat162_rn(x1.x, x1.y), __floats2bfloat162_rn(x1.z, x1.w)};
            *reinterpret_cast<uint4*>(A0 + (uint32_t)(c >> 3) * blk + swz(r, (c & 7) * 8)) =
                *reinterpret_cast<uint4*>(h2);
        }
        // ---- forward recompute of A_1..A_depth
        uint64_t mask[kMaxDepth + 1];
        for (int l = 0; l < depth && ok; ++l) {
            const unsigned char* Aop = l == 0 ? A0 : Ah + (uint32_t)(l - 1) * blk;
            const unsigned char* Bop = Wf + (l == 0 ? 0u : (uint32_t)NKB * wblk + (uint32_t)(l - 1) * wblk);
            if (!mma_wait(Aop, Bop, l == 0 ? NKB : 1)) { ok = false; break; }
            float v[64];
            ld64(v);
            uint64_t m = 0;
#pragma unroll
            for (int o = 0; o < 64; ++o) {
                v[o] = fmaxf(v[o] + bias[l * kH + o], 0.0f);
                m |= (uint64_t)(v[o] > 0.0f) << o;
            }
            mask[l + 1] = m;
            put_row(Ah + (uint32_t)l * blk, v);
            store_rows(a.tapeA[l + 1], row0, v);
        }
        if (!ok) break;
        // ---- G_{depth-1}
        {
            float v[64];
            if (kDec) {
                const float g = live ? a.gout[row] : 0.0f;
#pragma unroll
                for (int i = 0; i < 64; ++i) v[i] = g * bias[depth * kH + i];
            } else {
                load_rows(a.gout, row0, v);
                put_row(Gop, v);
                const unsigned char* Bop = Wb + (uint32_t)NKB * wblk + (uint32_t)(depth - 1) * wblk;
                if (!mma_wait(Gop, Bop, 1)) { ok = false; break; }
                ld64(v);
            }
            const uint64_t m = mask[depth];
#pragma unroll
            for (int i = 0; i < 64; ++i) v[i] = (m >> i) & 1 ? v[i] : 0.0f;
            put_row(Gop, v);
            store_rows(a.tapeG[depth - 1], row0, v);
        }
        // ---- G_{l-1} = (G_l W_l) (.) [A_l > 0], l = depth-1 .. 1
        for (int l = depth - 1; l >= 1 && ok; --l) {
            const unsigned char* Bop = Wb + (uint32_t)NKB * wblk + (uint32_t)(l - 1) * wblk;
            if (!mma_wait(Gop, Bop, 1)) { ok = false; break; }
            float v[64];
            ld64(v);
            const uint64_t m = mask[l];
#pragma unroll
            for (int i = 0; i < 64; ++i) v[i] = (m >> i) & 1 ? v[i] : 0.0f;
            put_row(Gop, v);
            store_rows(a.tapeG[l - 1], row0, v);
        }
        if (!ok) break;
        // ---- input gradient G_0 W_0, one 64-wide segment per product
        for (int s = 0; s < NKB && ok; ++s) {
            if (!mma_wait(Gop, Wb + (uint32_t)s * wblk, 1)) { ok = false; break; }
            float v[64];
            ld64(v);
            if (a.dx[s]) store_rows(a.dx[s], row0, v);
        }
    }
    if (!ok) {
        bar_wait(bar, phase ^ 1u);
        if (tid == 0) atomicOr(flags, kFlagTimeout);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

template <int MODE>
npcg_status launch_bwd_tc(Handle* h, const MlpBwdArgs& a, const float* agg_in, int* flags) {
    if (a.f.nrows == 0) return NPCG_OK;
    const BtPlan p = bt_plan(mode_in(MODE, kH), a.f.depth, MODE == MODE_DEC);
    const size_t smem = p.total + 1024;
    if (smem > 227 * 1024) return set_error(h, NPCG_EINVAL, "MLP too deep for the tensor-core backward");
    NPCG_CUDA(h, cudaFuncSetAttribute(k_mlp_bwd_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int per_sm = std::max(1, std::min(2, (int)((227 * 1024) / (smem + 1024))));
    const int64_t ntiles = (a.f.nrows + kM - 1) / kM;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)h->num_sms * per_sm));
    k_mlp_bwd_tc<MODE><<<grid, kThreads, smem, h->stream>>>(a, agg_in, flags);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

// ------------------------------------------------------------ weight gradients
// dW[o][q] += sum_k G[k][o] X[k][q], db[o] += sum_k G[k][o]; X's columns come
// in segments, each a row-gather of a [rows x width] array (idx may be null).
struct WSeg {
    const float* ptr;
    const int32_t* idx;
    int width;
};
struct WgradArgs {
    int64_t M;
    const float* G;
    int O;
    WSeg seg[3];
    int nseg;
    int I;
    float* dW;      // [O][I] then db[O]
    int bf16;       // BF16 tensor-core path allowed
    int* flags;     // device status word (tensor-core path)
};

constexpr int kWgRows = 32;
constexpr int kWgMaxEntries = 64 * 192;
constexpr int kWgPer = kWgMaxEntries / 256;

__global__ void __launch_bounds__(256) k_wgrad(WgradArgs a) {
    __shared__ float Gs[kWgRows][64 + 1];
    __shared__ float Xs[kWgRows][192 + 1];
    float acc[kWgPer];
    float bacc = 0.0f;
#pragma unroll
    for (int m = 0; m < kWgPer; ++m) acc[m] = 0.0f;
    const int64_t per = (a.M + gridDim.x - 1) / gridDim.x;
    const int64_t m0 = blockIdx.x * per, m1 = (a.M < m0 + per ? a.M : m0 + per);
    const int E = a.O * a.I;
    for (int64_t t0 = m0; t0 < m1; t0 += kWgRows) {
        const int rows = (int)(m1 - t0 < kWgRows ? m1 - t0 : kWgRows);
        for (int t = threadIdx.x; t < kWgRows * a.O; t += blockDim.x) {
            const int r = t / a.O, o = t % a.O;
            Gs[r][o] = r < rows ? a.G[(t0 + r) * a.O + o] : 0.0f;
        }
        int c0 = 0;
        for (int s = 0; s < a.nseg; ++s) {
            const WSeg sg = a.seg[s];
            for (int t = threadIdx.x; t < kWgRows * sg.width; t += blockDim.x) {
                const int r = t / sg.width, q = t % sg.width;
                float v = 0.0f;
                if (r < rows) {
                    const int64_t src = sg.idx ? sg.idx[t0 + r] : t0 + r;
                    v = sg.ptr[src * sg.width + q];
                }
                Xs[r][c0 + q] = v;
            }
            c0 += sg.width;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < kWgPer; ++m) {
            const int e = threadIdx.x + 256 * m;
            if (e < E) {
                const int o = e / a.I, q = e % a.I;
                float s = acc[m];
                for (int r = 0; r < rows; ++r) s = fmaf(Gs[r][o], Xs[r][q], s);
                acc[m] = s;
            }
        }
        if (threadIdx.x < a.O)
            for (int r = 0; r < rows; ++r) bacc += Gs[r][threadIdx.x];
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < kWgPer; ++m) {
        const int e = threadIdx.x + 256 * m;
        if (e < E && acc[m] != 0.0f) atomicAdd(&a.dW[e], acc[m]);
    }
    if (threadIdx.x < a.O && bacc != 0.0f) atomicAdd(&a.dW[E + threadIdx.x], bacc);
}

// ---- weight gradients on the tensor cores (BF16 operands, FP32 accumulate)
// dW^T = X^T G over the rows: one CTA per slice of the rows; per 128-row
// tile the FP32 tapes are read with coalesced float4 loads into a row-major
// BF16 staging area, transposed into the K-major swizzled operands
// (A = X^T: 128 q-rows per M-tile, B = G^T: 64 o-rows; K = the tile's rows)
// and multiplied into tensor memory.  Row q = I of A holds ones, so the
// bias gradient sum_r G[r][o] comes out of the same product.  The CTA's
// partial dW is added to the FP32 gradient at the end.
constexpr int kWtRows = 128;                 // rows (K) per tile
constexpr int kWtIMax = 192;                 // input width
constexpr int kWtLd = kWtIMax + 8;           // staging row stride (BF16)
struct WtPlan {
    uint32_t a, b, xs, gs, misc, total;
};
__host__ __device__ inline WtPlan wt_plan() {
    WtPlan p;
    p.a = 0;                                         // 2 M-tiles x 2 K-blocks x [128 x 64] BF16
    p.b = p.a + 2 * 2 * kM * 128;                    // 2 K-blocks x [64 x 64] BF16
    p.xs = p.b + 2 * kH * 128;                       // staging X [128][kWtLd] BF16
    p.gs = p.xs + kWtRows * kWtLd * 2;               // staging G [128][72] BF16
    p.misc = p.gs + kWtRows * 72 * 2;
    p.total = p.misc + 64;
    return p;
}

// eight BF16 values a column apart (stride ld) packed into one 16-byte chunk
__device__ __forceinline__ uint4 gather8(const unsigned short* p, int ld) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = (uint32_t)p[(2 * i) * ld] | ((uint32_t)p[(2 * i + 1) * ld] << 16);
    return make_uint4(w[0], w[1], w[2], w[3]);
}

constexpr int kWtThreads = 256;

// 128 rows x 64 FP32 (row r of ptr, or of ptr[idx[r]]) -> row-major BF16
// staging with row stride ld; eight float4 loads per thread are issued
// before any is converted
__device__ __forceinline__ void stage64(const float* ptr, const int32_t* idx, int64_t t0, int rows, int tid,
                                        __nv_bfloat16* dst, int ld) {
    float4 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int t = tid + k * kWtThreads, r = t >> 4, q4 = t & 15;
        v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < rows) {
            const int64_t src = idx ? idx[t0 + r] : t0 + r;
            v[k] = *reinterpret_cast<const float4*>(ptr + src * 64 + q4 * 4);
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int t = tid + k * kWtThreads, r = t >> 4, q4 = t & 15;
        __nv_bfloat162 lo = __floats2bfloat162_rn(v[k].x, v[k].y), hi = __floats2bfloat162_rn(v[k].z, v[k].w);
        uint2 pk;
        pk.x = *reinterpret_cast<uint32_t*>(&lo);
        pk.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(dst + r * ld + q4 * 4) = pk;
    }
}

__global__ void __launch_bounds__(kWtThreads) k_wgrad_tc(WgradArgs a) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((1024u - (s_addr(sm_raw) & 1023u)) & 1023u);
    const WtPlan P = wt_plan();
    unsigned char* Aop = sm + P.a;
    unsigned char* Bop = sm + P.b;
    __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(sm + P.xs);
    __nv_bfloat16* gs = reinterpret_cast<__nv_bfloat16*>(sm + P.gs);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P.misc);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + P.misc + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int I = a.I;
    const int nmt = (I + 1 + kM - 1) / kM;           // M-tiles of q (with the ones row)
    // A rows past the ones row stay zero
    for (int t = tid; t < 2 * 2 * kM * 128 / 16; t += kWtThreads)
        reinterpret_cast<uint4*>(Aop)[t] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(s_addr(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t per = ((a.M + gridDim.x - 1) / gridDim.x + kWtRows - 1) / kWtRows * kWtRows;
    const int64_t m0 = blockIdx.x * per, m1 = a.M < m0 + per ? a.M : m0 + per;
    uint32_t phase = 0;
    bool ok = true, issued = false;
    for (int64_t t0 = m0; t0 < m1 && ok; t0 += kWtRows) {
        const int rows = (int)(m1 - t0 < kWtRows ? m1 - t0 : kWtRows);
        // ---- stage the tile row-major in BF16 (coalesced float4 loads)
        {
            int c0 = 0;
#pragma unroll
            for (int sidx = 0; sidx < 3; ++sidx) {
                if (sidx >= a.nseg) break;
                const WSeg sg = a.seg[sidx];
                stage64(sg.ptr, sg.idx, t0, rows, tid, xs + c0, kWtLd);
                c0 += 64;
            }
            stage64(a.G, nullptr, t0, rows, tid, gs, 72);
        }
        // ---- the previous tile's products must be done before the operands change
        if (issued) {
            ok = bar_wait(bar, phase);
            phase ^= 1u;
            if (!__syncthreads_and(ok)) {
                ok = false;
                break;
            }
        } else {
            __syncthreads();
        }
        // ---- transpose into K-major operands: chunk = 8 consecutive rows of one column
        for (int t = tid; t < (I + 1) * (kWtRows / 8); t += kWtThreads) {
            const int q = t % (I + 1), r8 = t / (I + 1);
            uint4 val;
            if (q == I) {
                const uint32_t one2 = 0x3F803F80u;              // two BF16 ones
                val = make_uint4(one2, one2, one2, one2);
            } else {
                val = gather8(reinterpret_cast<const unsigned short*>(xs) + (r8 * 8) * kWtLd + q, kWtLd);
            }
            const int mt = q / kM, qq = q % kM, kb = r8 / 8;
            *reinterpret_cast<uint4*>(Aop + (uint32_t)(mt * 2 + kb) * (kM * 128) + swz(qq, (r8 % 8) * 8)) = val;
        }
        for (int t = tid; t < 64 * (kWtRows / 8); t += kWtThreads) {
            const int o = t % 64, r8 = t / 64;
            const int kb = r8 / 8;
            *reinterpret_cast<uint4*>(Bop + (uint32_t)kb * (kH * 128) + swz(o, (r8 % 8) * 8)) =
                gather8(reinterpret_cast<const unsigned short*>(gs) + (r8 * 8) * 72 + o, 72);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            for (int mt = 0; mt < nmt; ++mt)
                for (int s = 0; s < kWtRows / 16; ++s) {
                    const uint32_t kb = (uint32_t)(s >> 2), ko = (uint32_t)(s & 3) * 32;
                    mma_bf16(tmem + (uint32_t)mt * 64,
                             smem_desc(s_addr(Aop) + (uint32_t)(mt * 2 + kb) * (kM * 128) + ko),
                             smem_desc(s_addr(Bop) + kb * (kH * 128) + ko), (t0 > m0 || s > 0) ? 1u : 0u);
                }
            mma_commit(bar);
        }
        issued = true;
    }
    if (issued && ok) {
        ok = bar_wait(bar, phase);
        ok = __syncthreads_and(ok);
        tc_fence_after();
        if (ok) {
            // lane quarter of each M-tile: q = mt * 128 + 32 * warp + lane, 64 o columns
            // warps 0-3 read M-tile 0, warps 4-7 M-tile 1 (lane quarter = warp % 4)
            const int mt = warp >> 2, wq = warp & 3;
            if (mt < nmt) {
                const int q = mt * kM + wq * 32 + (tid & 31);
                for (int c4 = 0; c4 < 4; ++c4) {
                    float v[16];
                    tmem_ld16(tmem + (uint32_t)mt * 64 + ((uint32_t)(wq * 32) << 16) + c4 * 16, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int o = c4 * 16 + i;
                        if (v[i] == 0.0f) continue;
                        if (q < I) atomicAdd(&a.dW[o * I + q], v[i]);
                        else if (q == I) atomicAdd(&a.dW[64 * I + o], v[i]);
                    }
                }
            }
        }
    } else if (issued) {
        bar_wait(bar, phase);        // one more bounded wait for products in flight
    }
    if (!ok && tid == 0) atomicOr(a.flags, kFlagTimeout);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

npcg_status wgrad_tc(Handle* h, const WgradArgs& a) {
    const size_t smem = wt_plan().total + 1024;
    NPCG_CUDA(h, cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t tiles = (a.M + kWtRows - 1) / kWtRows;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)h->num_sms));
    k_wgrad_tc<<<grid, kWtThreads, smem, h->stream>>>(a);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

npcg_status wgrad(Handle* h, const WgradArgs& a) {
    if (a.M == 0) return NPCG_OK;
    // tensor cores for the BF16 path when the shape fits the MMA tiles
    if (a.bf16 && a.O == 64 && (a.I == 64 || a.I == 128 || a.I == 192)) {
        bool w64 = true;
        for (int s = 0; s < a.nseg; ++s) w64 = w64 && a.seg[s].width == 64;
        if (w64) return wgrad_tc(h, a);
    }
    if (a.O > 64 || a.I > 192 || a.O * a.I > kWgMaxEntries)
        return set_error(h, NPCG_EINVAL, "weight-gradient shape out of range");
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>((a.M + kWgRows - 1) / kWgRows, (int64_t)h->num_sms * 4));
    k_wgrad<<<grid, 256, 0, h->stream>>>(a);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

// ------------------------------------------------------------ node / edge adjoint glue
// dV[i] += sum_{k in row i} Gr[k] + Gc[mirror[k]]   (edge MLP's v_i and v_j inputs)
__global__ void k_node_from_edges(int64_t n, int H, const int32_t* rp, const int32_t* mirror,
                                  const float* Gr, const float* Gc, float* dV) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * H;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / H;
        const int q = (int)(t % H);
        float s = dV[t];
        for (int k = rp[i]; k < rp[i + 1]; ++k) s += Gr[(int64_t)k * H + q] + Gc[(int64_t)mirror[k] * H + q];
        dV[t] = s;
    }
}

// aggregation agg_i = sum_j e_ij (.) v_j:
//   dE[k] += dAgg[row_k] (.) V[col_k];  dV[j] += sum_{k in row j} dAgg[col_k] (.) E[mirror k]
__global__ void k_agg_bwd_edges(int64_t nnz, int H, const int32_t* erow, const int32_t* ci,
                                const float* dAgg, const float* V, float* dE) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz * H;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / H;
        const int q = (int)(t % H);
        dE[t] += dAgg[(int64_t)erow[k] * H + q] * V[(int64_t)ci[k] * H + q];
    }
}

__global__ void k_agg_bwd_nodes(int64_t n, int H, const int32_t* rp, const int32_t* ci,
                                const int32_t* mirror, const float* dAgg, const float* E, float* dV) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * H;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / H;
        const int q = (int)(t % H);
        float s = dV[t];
        for (int k = rp[j]; k < rp[j + 1]; ++k)
            s = fmaf(dAgg[(int64_t)ci[k] * H + q], E[(int64_t)mirror[k] * H + q], s);
        dV[t] = s;
    }
}

// regression of the initial-guess head: d_i = out_i - x_i s / ||b||_inf,
// loss_sys += d_i^2, dout_i = c d_i (c = 2 / (pairs * systems))
__global__ void k_x0_loss(int64_t n, const int32_t* row_sys, const double* sc, const double* x, const float* out,
                          double c, float* dout, double* loss_sys) {
    const unsigned full = 0xffffffffu;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        double d2 = 0.0;
        int sys = -1;
        if (i < n) {
            sys = row_sys[i];
            const double d = (double)out[i] - x[i] * sc[2 * sys] / sc[2 * sys + 1];
            dout[i] = (float)(c * d);
            d2 = d * d;
        }
        const int s0 = __shfl_sync(full, sys, 0);
        if (__all_sync(full, sys == s0 || sys < 0)) {
            for (int o = 16; o; o >>= 1) d2 += __shfl_xor_sync(full, d2, o);
            if ((threadIdx.x & 31) == 0 && s0 >= 0) atomicAdd(&loss_sys[s0], d2);
        } else if (sys >= 0) {
            atomicAdd(&loss_sys[sys], d2);
        }
    }
}

__global__ void k_enc_inputs(int64_t n, int64_t nnz, const double* b, const double* av, const int32_t* erow,
                             const int32_t* ci, const int32_t* adiag_scaled, const int32_t* row_sys,
                             const double* sc, float* xv, float* xe) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n) xv[i] = (float)(b[i] / sc[2 * row_sys[i] + 1]);
        xe[i] = (float)edge_input(av, sc, row_sys, erow, ci, adiag_scaled, i);
    }
}

// ------------------------------------------------------------ driver
// Frobenius loss Eq. (loss_A): R = L L^T - A on the lower triangle of
// pattern(L L^T), R_e = sum of its L products (k ascending) - A_e, and the
// system's loss += w_e R_e^2 (w = 1 on the diagonal, 2 off it: R is
// symmetric and both triangles count)
__global__ void k_frob_R(int64_t nS, const int32_t* sptr, const int2* spairs, const int32_t* s2a,
                         const int32_t* srow, const int32_t* row_sys, const double* Lv, const double* A_val,
                         double* R, double* loss_sys) {
    const unsigned full = 0xffffffffu;
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x; e0 < nS; e0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = e0 + threadIdx.x;
        double v = 0.0;
        int sys = -1;
        if (e < nS) {
            double sum = 0.0;
            for (int q = sptr[e]; q < sptr[e + 1]; ++q) {
                const int2 ab = spairs[q];
                sum = fma(Lv[ab.x], Lv[ab.y], sum);
            }
            const int a = s2a[e];
            const double r = sum - (a >= 0 ? A_val[a] : 0.0);
            R[e] = r;
            const int sr = srow[e];
            sys = row_sys[sr >= 0 ? sr : -sr - 1];
            v = (sr >= 0 ? 1.0 : 2.0) * r * r;
        }
        const int s0 = __shfl_sync(full, sys, 0);
        if (__all_sync(full, sys == s0 || sys < 0)) {
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(full, v, o);
            if ((threadIdx.x & 31) == 0 && s0 >= 0) atomicAdd(&loss_sys[s0], v);
        } else if (sys >= 0) {
            atomicAdd(&loss_sys[sys], v);
        }
    }
}

// dL_a = c2 (R L)_a: for L entry a = (i, k), the sum over the entries b of
// column k (rows j ascending) of R_(i,j) L_b
__global__ void k_frob_dL(int64_t nnzL, const int32_t* gptr, const int2* gpairs, const double* Lv,
                          const double* R, double c2, double* dL) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < nnzL;
         a += (int64_t)gridDim.x * blockDim.x) {
        double sum = 0.0;
        for (int q = gptr[a]; q < gptr[a + 1]; ++q) {
            const int2 bs = gpairs[q];
            sum = fma(R[bs.y], Lv[bs.x], sum);
        }
        dL[a] = c2 * sum;
    }
}

struct TrainBufs {
    std::vector<float*> V, E, AGG;
    float *S, *dS, *dEc, *dEp, *dVc, *dVp, *Gr, *Gc, *dAgg, *xv, *xe;
    float* tapeA[kMaxDepth + 1];
    float* tapeG[kMaxDepth + 1];
    double *Lv, *dL, *y, *r, *w, *loss_sys;
    int bf16;          // weight gradients on the tensor cores
    int* flags;        // device status word
    float *xh, *dxh;   // initial-guess head: outputs and their adjoint [n]
};

inline int grid1(Handle* h, int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)h->num_sms * 8)); }

// weight gradient of one MLP (depth Linears + output layer) from its tapes
npcg_status mlp_wgrad(Handle* h, int64_t M, int H, int in_w, int out_w, int depth, const float* gout,
                      const TrainBufs& T, const WSeg* inseg, int nin, float* gw) {
    // layers depth..1: input A_l, gradient G_l (G_depth = gout)
    float* cur = gw;
    std::vector<float*> lay(depth + 1);
    for (int l = 0; l <= depth; ++l) {
        lay[l] = cur;
        const int fi = l == 0 ? in_w : H, fo = l == depth ? out_w : H;
        cur += (int64_t)fi * fo + fo;
    }
    for (int l = depth; l >= 0; --l) {
        WgradArgs a{};
        a.bf16 = T.bf16;
        a.flags = T.flags;
        a.M = M;
        a.G = l == depth ? gout : T.tapeG[l];
        a.O = l == depth ? out_w : H;
        a.dW = lay[l];
        if (l == 0) {
            for (int s = 0; s < nin; ++s) a.seg[s] = inseg[s];
            a.nseg = nin;
            a.I = in_w;
        } else {
            a.seg[0] = WSeg{T.tapeA[l], nullptr, H};
            a.nseg = 1;
            a.I = H;
        }
        NPCG_TRY(wgrad(h, a));
    }
    return NPCG_OK;
}

// MLP backward: tensor cores on the BF16 path (h = 64, node / edge / decoder),
// FP32 CUDA cores otherwise
template <int H>
npcg_status run_bwd(Handle* h, int mode, const MlpBwdArgs& bw, const float* agg_in, const TrainBufs& T) {
    if constexpr (H == 64) {
        if (T.bf16) {
            if (mode == MODE_EDGE) return launch_bwd_tc<MODE_EDGE>(h, bw, agg_in, T.flags);
            if (mode == MODE_NODE) return launch_bwd_tc<MODE_NODE>(h, bw, agg_in, T.flags);
            if (mode == MODE_DEC) return launch_bwd_tc<MODE_DEC>(h, bw, agg_in, T.flags);
        }
    }
    return launch_bwd<H>(h, mode, bw);
}

template <int H>
npcg_status train_pair(Handle* h, Pattern* P, const double* A_val, const double* x, const double* b,
                       const npcg_gnn_config* cfg, const float* w, float* gw, TrainBufs& T, double c) {
    const int l = cfg->l, lm = cfg->l_mp, nmp = cfg->n_mp;
    const int64_t n = P->n, nnz = P->nnz, nnzL = P->nnzL;
    const GnnOffsets off = gnn_offsets(H, l, lm, nmp, cfg->x0_head);
    double* sc = P->gnn.sc.p;
    // ---- forward with tape
    MlpArgs a = {};
    a.rp = P->rp.p;
    a.ci = P->ci.p;
    a.erow = P->edge_row.p;
    a.row_sys = P->row_sys.p;
    a.sc = sc;
    a.av = A_val;
    a.b = b;
    a.adiag_scaled = cfg->diag_mode == NPCG_DIAG_LDLT_ROWS ? P->adiag.p : nullptr;
    if (cfg->precision == NPCG_BF16) {
        // tensor-core forward; the tape holds its node / edge states in FP32
        NPCG_TRY(gnn_bf16_forward_core(h, P, A_val, b, cfg, w, sc, T.S, T.V.data(), T.E.data(), T.AGG.data()));
        NPCG_TRY(gnn_bf16_check_flags(h, P));
    } else {
        a.nrows = n; a.w = w + off.enc_v; a.depth = l; a.out = T.V[0];
        NPCG_TRY(launch_mlp<H>(h, MODE_ENC_NODE, a));
        a.nrows = nnz; a.w = w + off.enc_e; a.depth = l; a.out = T.E[0];
        NPCG_TRY(launch_mlp<H>(h, MODE_ENC_EDGE, a));
        for (int t = 0; t < nmp; ++t) {
            a.nrows = n; a.w = w + off.node[t]; a.depth = lm; a.vin = T.V[t]; a.ein = T.E[t]; a.out = T.V[t + 1];
            a.agg_out = T.AGG[t];
            NPCG_TRY(launch_mlp<H>(h, MODE_NODE, a));
            a.agg_out = nullptr;
            a.nrows = nnz; a.w = w + off.edge[t]; a.depth = lm; a.vin = T.V[t + 1]; a.ein = T.E[t]; a.out = T.E[t + 1];
            NPCG_TRY(launch_mlp<H>(h, MODE_EDGE, a));
        }
        a.nrows = nnz; a.w = w + off.dec; a.depth = l; a.ein = T.E[nmp]; a.out = T.S;
        NPCG_TRY(launch_mlp<H>(h, MODE_DEC, a));
    }
    GnnBuffers gb{};
    gb.s = T.S;
    gb.sc = sc;
    gb.av = A_val;
    gb.diag_mode = cfg->diag_mode;
    NPCG_TRY(gnn_assemble_L(h, P, gb, T.Lv));
    // ---- loss and its adjoint in L
    if (cfg->loss == NPCG_LOSS_FROB) {
        const FrobLayout& F = P->frob;
        k_frob_R<<<grid1(h, F.nS), 256, 0, h->stream>>>(F.nS, F.sptr.p, F.spairs.p, F.s2a.p, F.srow.p,
                                                        P->row_sys.p, T.Lv, A_val, F.R.p, T.loss_sys);
        k_frob_dL<<<grid1(h, nnzL), 256, 0, h->stream>>>(nnzL, F.gptr.p, F.gpairs.p, T.Lv, F.R.p, 2.0 * c, T.dL);
    } else {
        k_lt_mv<<<grid1(h, n), 256, 0, h->stream>>>(n, P->rp.p, P->ci.p, P->mirror.p, P->a2l.p, T.Lv, x, T.y);
        k_l_mv_res<<<grid1(h, n), 256, 0, h->stream>>>(n, P->Lrp.p, P->Lci.p, T.Lv, T.y, b, P->row_sys.p, T.r,
                                                      T.loss_sys);
        k_lt_mv<<<grid1(h, n), 256, 0, h->stream>>>(n, P->rp.p, P->ci.p, P->mirror.p, P->a2l.p, T.Lv, T.r, T.w);
        k_dL<<<grid1(h, nnzL), 256, 0, h->stream>>>(nnzL, P->l2a.p, P->edge_row.p, P->ci.p, c, T.r, T.y, x, T.w,
                                                    T.dL);
    }
    k_dS<<<grid1(h, nnz), 256, 0, h->stream>>>(nnz, P->edge_row.p, P->ci.p, P->mirror.p, P->a2l.p, P->row_sys.p,
                                              sc, T.S, T.dL, A_val, P->adiag.p, cfg->diag_mode, T.dS);
    NPCG_CUDA(h, cudaGetLastError());
    // ---- decoder
    MlpBwdArgs bw{};
    for (int k = 0; k <= kMaxDepth; ++k) { bw.tapeA[k] = T.tapeA[k]; bw.tapeG[k] = T.tapeG[k]; }
    bw.f = a;
    bw.f.nrows = nnz; bw.f.w = w + off.dec; bw.f.depth = l; bw.f.ein = T.E[nmp];
    bw.gout = T.dS;
    bw.dx[0] = T.dEc; bw.dx[1] = bw.dx[2] = nullptr;
    NPCG_TRY(run_bwd<H>(h, MODE_DEC, bw, nullptr, T));
    {
        WSeg s0{T.E[nmp], nullptr, H};
        NPCG_TRY(mlp_wgrad(h, nnz, H, H, 1, l, T.dS, T, &s0, 1, gw + off.dec));
    }
    NPCG_CUDA(h, cudaMemsetAsync(T.dVc, 0, (size_t)n * H * sizeof(float), h->stream));
    for (int t = nmp - 1; t >= 0; --t) {
        // edge update t: input [E_t | V_{t+1}(row) | V_{t+1}(col)], upstream dE_{t+1}
        bw.f = a;
        bw.f.nrows = nnz; bw.f.w = w + off.edge[t]; bw.f.depth = lm; bw.f.vin = T.V[t + 1]; bw.f.ein = T.E[t];
        bw.gout = T.dEc;
        bw.dx[0] = T.dEp; bw.dx[1] = T.Gr; bw.dx[2] = T.Gc;
        NPCG_TRY(run_bwd<H>(h, MODE_EDGE, bw, nullptr, T));
        {
            WSeg s[3] = {{T.E[t], nullptr, H}, {T.V[t + 1], P->edge_row.p, H}, {T.V[t + 1], P->ci.p, H}};
            NPCG_TRY(mlp_wgrad(h, nnz, H, 3 * H, H, lm, T.dEc, T, s, 3, gw + off.edge[t]));
        }
        k_node_from_edges<<<grid1(h, n * H), 256, 0, h->stream>>>(n, H, P->rp.p, P->mirror.p, T.Gr, T.Gc, T.dVc);
        // node update t: input [V_t | agg_t], upstream dV_{t+1}
        bw.f = a;
        bw.f.nrows = n; bw.f.w = w + off.node[t]; bw.f.depth = lm; bw.f.vin = T.V[t]; bw.f.ein = T.E[t];
        bw.gout = T.dVc;
        bw.dx[0] = T.dVp; bw.dx[1] = T.dAgg; bw.dx[2] = nullptr;
        NPCG_TRY(run_bwd<H>(h, MODE_NODE, bw, T.AGG[t], T));
        {
            WSeg s[2] = {{T.V[t], nullptr, H}, {T.AGG[t], nullptr, H}};
            NPCG_TRY(mlp_wgrad(h, n, H, 2 * H, H, lm, T.dVc, T, s, 2, gw + off.node[t]));
        }
        k_agg_bwd_edges<<<grid1(h, nnz * H), 256, 0, h->stream>>>(nnz, H, P->edge_row.p, P->ci.p, T.dAgg, T.V[t], T.dEp);
        k_agg_bwd_nodes<<<grid1(h, n * H), 256, 0, h->stream>>>(n, H, P->rp.p, P->ci.p, P->mirror.p, T.dAgg, T.E[t], T.dVp);
        NPCG_CUDA(h, cudaGetLastError());
        std::swap(T.dEc, T.dEp);
        std::swap(T.dVc, T.dVp);
    }
    // encoders: weight gradients only
    k_enc_inputs<<<grid1(h, nnz), 256, 0, h->stream>>>(n, nnz, b, A_val, P->edge_row.p, P->ci.p,
                                                       cfg->diag_mode == NPCG_DIAG_LDLT_ROWS ? P->adiag.p : nullptr,
                                                       P->row_sys.p, sc, T.xv, T.xe);
    bw.f = a;
    bw.f.nrows = n; bw.f.w = w + off.enc_v; bw.f.depth = l;
    bw.gout = T.dVc;
    bw.dx[0] = bw.dx[1] = bw.dx[2] = nullptr;
    NPCG_TRY(launch_bwd<H>(h, MODE_ENC_NODE, bw));
    {
        WSeg s0{T.xv, nullptr, 1};
        NPCG_TRY(mlp_wgrad(h, n, H, 1, H, l, T.dVc, T, &s0, 1, gw + off.enc_v));
    }
    bw.f.nrows = nnz; bw.f.w = w + off.enc_e;
    bw.gout = T.dEc;
    NPCG_TRY(launch_bwd<H>(h, MODE_ENC_EDGE, bw));
    {
        WSeg s0{T.xe, nullptr, 1};
        NPCG_TRY(mlp_wgrad(h, nnz, H, 1, H, l, T.dEc, T, &s0, 1, gw + off.enc_e));
    }
    if (cfg->x0_head) {
        // initial-guess head: regression to x on the final node features; the
        // trunk is not differentiated through it (no input gradient)
        MlpArgs ax = a;
        ax.nrows = n; ax.w = w + off.x0; ax.depth = l; ax.ein = T.V[nmp]; ax.out = T.xh;
        NPCG_TRY(launch_mlp<H>(h, MODE_DEC, ax));
        k_x0_loss<<<grid1(h, n), 256, 0, h->stream>>>(n, P->row_sys.p, sc, x, T.xh, c, T.dxh, T.loss_sys);
        NPCG_CUDA(h, cudaGetLastError());
        MlpBwdArgs bx{};
        for (int k = 0; k <= kMaxDepth; ++k) { bx.tapeA[k] = T.tapeA[k]; bx.tapeG[k] = T.tapeG[k]; }
        bx.f = ax;
        bx.gout = T.dxh;
        bx.dx[0] = bx.dx[1] = bx.dx[2] = nullptr;
        NPCG_TRY(run_bwd<H>(h, MODE_DEC, bx, nullptr, T));
        WSeg s0{T.V[nmp], nullptr, H};
        NPCG_TRY(mlp_wgrad(h, n, H, H, 1, l, T.dxh, T, &s0, 1, gw + off.x0));
    }
    // tensor-core waits of this pair (the next pair's forward clears the word)
    if (T.bf16) NPCG_TRY(gnn_bf16_check_flags(h, P));
    return NPCG_OK;
}

__global__ void k_adam(int64_t n, float* w, const float* g, float* m, float* v, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace

npcg_status gnn_scales_run(Handle* h, Pattern* P, const double* A_val, const double* b, double* sc);

// Builds the product structure of L L^T (host, once per pattern): the
// entries (i, j), j <= i, of pattern(L L^T) row by row with their product
// pairs (L_ik, L_jk) in ascending k, the A entry of each, and for every L
// entry (i, k) the pairs (L_jk, entry (max(i,j), min(i,j))) over the rows j
// of column k in ascending order.
static npcg_status frob_build(Handle* h, Pattern* P) {
    FrobLayout& F = P->frob;
    if (F.built) return NPCG_OK;
    const int64_t n = P->n, nnzL = P->nnzL, nnz = P->nnz;
    std::vector<int32_t> Lrp(n + 1), Lci(nnzL), rp(n + 1), ci(nnz);
    NPCG_CUDA(h, cudaMemcpyAsync(Lrp.data(), P->Lrp.p, (n + 1) * 4, cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(Lci.data(), P->Lci.p, nnzL * 4, cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(rp.data(), P->rp.p, (n + 1) * 4, cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(ci.data(), P->ci.p, nnz * 4, cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    // columns of L: entries in ascending row order
    std::vector<int32_t> cptr(n + 1, 0), cent(nnzL), Lrow(nnzL);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t a = Lrp[i]; a < Lrp[i + 1]; ++a) { cptr[Lci[a] + 1]++; Lrow[a] = (int32_t)i; }
    for (int64_t k = 0; k < n; ++k) cptr[k + 1] += cptr[k];
    {
        std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int32_t a = Lrp[i]; a < Lrp[i + 1]; ++a) cent[fill[Lci[a]]++] = a;
    }
    // entries of the lower triangle of L L^T, row by row
    std::vector<int32_t> srp(n + 1, 0), scol, sptr(1, 0), s2a, srow;
    std::vector<int2> spairs;
    std::vector<std::array<int32_t, 3>> cand;     // (j, a, b)
    for (int64_t i = 0; i < n; ++i) {
        cand.clear();
        for (int32_t a = Lrp[i]; a < Lrp[i + 1]; ++a) {
            const int32_t k = Lci[a];
            for (int32_t q = cptr[k]; q < cptr[k + 1]; ++q) {
                const int32_t b = cent[q];
                if (Lrow[b] <= i) cand.push_back({Lrow[b], a, b});
            }
        }
        std::sort(cand.begin(), cand.end());
        for (size_t t = 0; t < cand.size();) {
            const int32_t j = cand[t][0];
            for (; t < cand.size() && cand[t][0] == j; ++t) spairs.push_back(make_int2(cand[t][1], cand[t][2]));
            scol.push_back(j);
            sptr.push_back((int32_t)spairs.size());
            const int32_t* lo = ci.data() + rp[i];
            const int32_t* hi = ci.data() + rp[i + 1];
            const int32_t* f = std::lower_bound(lo, hi, j);
            s2a.push_back(f != hi && *f == j ? (int32_t)(f - ci.data()) : -1);
            srow.push_back(j == i ? (int32_t)i : (int32_t)(-i - 1));
        }
        srp[i + 1] = (int32_t)scol.size();
    }
    auto sidx = [&](int32_t p, int32_t q) {       // entry (p, q), q <= p
        const int32_t* lo = scol.data() + srp[p];
        const int32_t* hi = scol.data() + srp[p + 1];
        return (int32_t)(std::lower_bound(lo, hi, q) - scol.data());
    };
    // (R L) pairs per L entry
    std::vector<int32_t> gptr(nnzL + 1, 0);
    std::vector<int2> gpairs;
    for (int64_t a = 0; a < nnzL; ++a) {
        const int32_t i = Lrow[a], k = Lci[a];
        for (int32_t q = cptr[k]; q < cptr[k + 1]; ++q) {
            const int32_t b = cent[q], j = Lrow[b];
            gpairs.push_back(make_int2(b, i >= j ? sidx(i, j) : sidx(j, i)));
        }
        gptr[a + 1] = (int32_t)gpairs.size();
    }
    if (spairs.size() >= (size_t)INT32_MAX || gpairs.size() >= (size_t)INT32_MAX)
        return set_error(h, NPCG_EINVAL, "pattern too large for the Frobenius loss structure");
    F.nS = (int64_t)scol.size();
    NPCG_CUDA(h, F.sptr.alloc(sptr.size()));
    NPCG_CUDA(h, F.s2a.alloc(std::max<size_t>(s2a.size(), 1)));
    NPCG_CUDA(h, F.srow.alloc(std::max<size_t>(srow.size(), 1)));
    NPCG_CUDA(h, F.spairs.alloc(std::max<size_t>(spairs.size(), 1)));
    NPCG_CUDA(h, F.gptr.alloc(gptr.size()));
    NPCG_CUDA(h, F.gpairs.alloc(std::max<size_t>(gpairs.size(), 1)));
    NPCG_CUDA(h, F.R.alloc(std::max<int64_t>(F.nS, 1)));
    NPCG_CUDA(h, cudaMemcpyAsync(F.sptr.p, sptr.data(), sptr.size() * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(F.s2a.p, s2a.data(), s2a.size() * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(F.srow.p, srow.data(), srow.size() * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(F.spairs.p, spairs.data(), spairs.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                 h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(F.gptr.p, gptr.data(), gptr.size() * 4, cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(F.gpairs.p, gpairs.data(), gpairs.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                 h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    F.built = true;
    return NPCG_OK;
}

npcg_status loss_grad_run(Handle* h, Pattern* P, const double* A_val, int npairs, const double* X,
                          const double* B, const npcg_gnn_config* cfg, const float* w, double* loss_out,
                          float* grad) {
    NPCG_TRY(gnn_check_config(h, cfg));
    if (cfg->loss != NPCG_LOSS_AB && cfg->loss != NPCG_LOSS_FROB)
        return set_error(h, NPCG_EINVAL, "loss must be NPCG_LOSS_AB or NPCG_LOSS_FROB");
    if (cfg->loss == NPCG_LOSS_FROB) NPCG_TRY(frob_build(h, P));
    if (cfg->precision == NPCG_BF16 && cfg->h != 64)
        return set_error(h, NPCG_EINVAL, "the BF16 tensor-core forward needs hidden width h = 64");
    const int H = cfg->h, nmp = cfg->n_mp;
    const int64_t n = P->n, nnz = P->nnz, nnzL = P->nnzL;
    const int dmax = std::max(cfg->l, cfg->l_mp);
    const GnnOffsets off = gnn_offsets(H, cfg->l, cfg->l_mp, nmp, cfg->x0_head);
    GnnStore& S = P->gnn;
    const size_t fe = (size_t)nnz * H, fv = (size_t)n * H;
    // tape: V_0..V_nmp, E_0..E_nmp, AGG_0..AGG_{nmp-1}; adjoint buffers
    // every buffer starts on a 256-byte boundary (vector loads of the tapes)
    auto al64 = [](size_t k) { return (k + 63) & ~size_t(63); };
    const size_t need = (size_t)(nmp + 1) * (al64(fe) + al64(fv)) + (size_t)std::max(nmp, 1) * al64(fv) +
                        4 * al64(fe) + 5 * al64(fv) + 4 * al64(nnz) + (size_t)(2 * dmax + 2) * al64(std::max(fe, fv)) +
                        2 * al64((size_t)n);
    NPCG_CUDA(h, S.aux.ensure(need));
    NPCG_CUDA(h, S.sc.ensure((size_t)2 * P->nsys));
    NPCG_CUDA(h, S.Lv.ensure((size_t)nnzL));
    NPCG_CUDA(h, S.dL.ensure((size_t)nnzL + 3 * (size_t)n + P->nsys));
    TrainBufs T;
    float* p = S.aux.p;
    auto take = [&](size_t k) { float* r = p; p += al64(k); return r; };
    for (int t = 0; t <= nmp; ++t) T.V.push_back(take(fv));
    for (int t = 0; t <= nmp; ++t) T.E.push_back(take(fe));
    for (int t = 0; t < std::max(nmp, 1); ++t) T.AGG.push_back(take(fv));
    T.dEc = take(fe); T.dEp = take(fe); T.Gr = take(fe); T.Gc = take(fe);
    T.dVc = take(fv); T.dVp = take(fv); T.dAgg = take(fv); T.xv = take(fv); T.xe = take(nnz);
    T.S = take(nnz); T.dS = take(nnz);
    for (int k = 0; k <= kMaxDepth; ++k) { T.tapeA[k] = nullptr; T.tapeG[k] = nullptr; }
    for (int k = 0; k <= dmax; ++k) { T.tapeA[k] = take(std::max(fe, fv)); T.tapeG[k] = take(std::max(fe, fv)); }
    T.xh = take((size_t)n);
    T.dxh = take((size_t)n);
    T.bf16 = cfg->precision == NPCG_BF16;
    T.flags = P->ctl.p + 1;
    T.Lv = S.Lv.p;
    T.dL = S.dL.p;
    T.y = T.dL + nnzL;
    T.r = T.y + n;
    T.w = T.r + n;
    T.loss_sys = T.w + n;
    NPCG_CUDA(h, cudaMemsetAsync(grad, 0, off.total * sizeof(float), h->stream));
    NPCG_CUDA(h, cudaMemsetAsync(T.loss_sys, 0, P->nsys * sizeof(double), h->stream));
    const double c = 2.0 / ((double)npairs * (double)P->nsys);
    for (int pp = 0; pp < npairs; ++pp) {
        const double* x = X + (size_t)pp * n;
        const double* b = B + (size_t)pp * n;
        NPCG_TRY(gnn_scales_run(h, P, A_val, b, S.sc.p));
        npcg_status st;
        switch (H) {
            case 16: st = train_pair<16>(h, P, A_val, x, b, cfg, w, grad, T, c); break;
            case 32: st = train_pair<32>(h, P, A_val, x, b, cfg, w, grad, T, c); break;
            default: st = train_pair<64>(h, P, A_val, x, b, cfg, w, grad, T, c); break;
        }
        if (st != NPCG_OK) return st;
    }
    std::vector<double> ls(P->nsys);
    NPCG_CUDA(h, cudaMemcpyAsync(ls.data(), T.loss_sys, P->nsys * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));

    double tot = 0.0;
    for (double v : ls) tot += v;
    *loss_out = tot / ((double)npairs * (double)P->nsys);
    return NPCG_OK;
}

npcg_status adam_run(Handle* h, int64_t n, float* w, const float* g, float* m, float* v, int t,
                     float lr, float b1, float b2, float eps) {
    if (n == 0) return NPCG_OK;
    const float c1 = (float)(1.0 - pow((double)b1, t)), c2 = (float)(1.0 - pow((double)b2, t));
    k_adam<<<grid1(h, n), 256, 0, h->stream>>>(n, w, g, m, v, lr, b1, b2, eps, c1, c2);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

}  // namespace npcg
