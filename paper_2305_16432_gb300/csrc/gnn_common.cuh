// Shared machinery of the graph-network kernels (forward and adjoint):
// weight layout, buffers, and the fused gather + MLP kernel (FP32 path).
#pragma once

#include <algorithm>

#include "npcg_internal.cuh"

namespace npcg {

constexpr int kMaxDepth = 4;
constexpr int kMaxMp = 64;

enum MlpMode { MODE_ENC_NODE = 0, MODE_ENC_EDGE = 1, MODE_NODE = 2, MODE_EDGE = 3, MODE_DEC = 4 };

// Offsets (in floats) of each MLP inside the flat weight vector: node
// encoder, edge encoder, n_mp x (node MLP, edge MLP), decoder; every Linear
// W[out][in] then bias[out].
struct GnnOffsets {
    int64_t enc_v, enc_e, node[kMaxMp], edge[kMaxMp], dec, x0, total;
};

inline int64_t mlp_size(int in, int h, int out, int depth) {
    return (int64_t)in * h + h + (int64_t)(depth - 1) * (h * h + h) + (int64_t)h * out + out;
}

// x0_head: the initial-guess head (an MLP of depth l, h -> 1) after the decoder
inline GnnOffsets gnn_offsets(int h, int l, int lm, int n_mp, int x0_head = 0) {
    GnnOffsets o{};
    int64_t p = 0;
    o.enc_v = p; p += mlp_size(1, h, h, l);
    o.enc_e = p; p += mlp_size(1, h, h, l);
    for (int t = 0; t < n_mp; ++t) {
        o.node[t] = p; p += mlp_size(2 * h, h, h, lm);
        o.edge[t] = p; p += mlp_size(3 * h, h, h, lm);
    }
    o.dec = p; p += mlp_size(h, h, 1, l);
    o.x0 = p;
    if (x0_head) p += mlp_size(h, h, 1, l);
    o.total = p;
    return o;
}

struct GnnBuffers {
    float* v[2];
    float* e[2];
    float* s;
    double* sc;     // per system: [2s] max diagonal, [2s+1] ||b||_inf
    const double* av = nullptr;   // A values (diag_mode 1 reads diag(A))
    int diag_mode = 0;
};

struct MlpArgs {
    int64_t nrows;
    const float* w;
    int depth;
    const int32_t* rp;
    const int32_t* ci;
    const int32_t* erow;
    const int32_t* row_sys;
    const double* sc;
    const double* av;
    const double* b;
    const float* vin;
    const float* ein;
    float* out;
    float* agg_out;      // node update: optional copy of sum_j e_ij (.) v_j (training tape)
    const int32_t* adiag_scaled;  // diag_mode 2: positions of the diagonal (edge input scaled by it)
};

// Encoder input of edge k = (i, j): A_ij / s with s the system's largest
// diagonal (diag_mode 0 and 1), or, given the diagonal positions
// (diag_mode 2), the entry of the Jacobi-scaled matrix A_ij / sqrt(A_ii A_jj).
__device__ __forceinline__ double edge_input(const double* av, const double* sc, const int32_t* row_sys,
                                             const int32_t* erow, const int32_t* ci, const int32_t* adiag,
                                             int64_t k) {
    const int i = erow[k];
    if (adiag) return av[k] / sqrt(av[adiag[i]] * av[adiag[ci[k]]]);
    return av[k] / sc[2 * row_sys[i]];
}

npcg_status gnn_check_config(Handle* h, const npcg_gnn_config* cfg);
npcg_status gnn_buffers(Handle* h, Pattern* P, int H, int nsets, GnnStore& S);
npcg_status gnn_forward_into(Handle* h, Pattern* P, const double* A_val, const double* b,
                             const npcg_gnn_config* cfg, const float* w, GnnBuffers& B);
npcg_status gnn_assemble_L(Handle* h, Pattern* P, const GnnBuffers& B, double* L_val);
npcg_status gnn_forward_bf16_run(Handle* h, Pattern* P, const double* A_val, const double* b,
                                 const npcg_gnn_config* cfg, const float* w, double* L_val);
npcg_status gnn_bf16_forward_core(Handle* h, Pattern* P, const double* A_val, const double* b,
                                  const npcg_gnn_config* cfg, const float* w, double* sc, float* sout,
                                  float* const* tV, float* const* tE, float* const* tAGG);
npcg_status gnn_bf16_check_flags(Handle* h, Pattern* P);
npcg_status gnn_bf16_head_run(Handle* h, Pattern* P, const npcg_gnn_config* cfg, const float* w_head, float* out);
npcg_status gnn_factor_x0_run(Handle* h, Pattern* P, const double* A_val, const double* b,
                              const npcg_gnn_config* cfg, const float* w, double* L_val, double* x0);

namespace {

__host__ __device__ constexpr int mode_in(int mode, int H) {
    return mode == MODE_ENC_NODE || mode == MODE_ENC_EDGE ? 1
         : mode == MODE_NODE ? 2 * H
         : mode == MODE_EDGE ? 3 * H : H;
}
__host__ __device__ constexpr int mode_out(int mode, int H) { return mode == MODE_DEC ? 1 : H; }

template <int H>
struct Tile {
    static constexpr int R = 4096 / H;     // rows per tile: (R/4) x (H/4) = 256 threads
    static constexpr int TO = H / 4;
};

// shared-memory footprint in floats
inline size_t mlp_smem_floats(int mode, int H, int depth) {
    const int in = mode_in(mode, H), out = mode_out(mode, H), R = 4096 / H;
    size_t w = (size_t)in * H + H + (size_t)(depth - 1) * (H * H + H) + (size_t)H * out + out;
    w = (w + 3) & ~size_t(3);
    return w + (size_t)R * (in + 1) + 2 * (size_t)R * (H + 1) + 4;
}

// Y[R x H] = act(X[R x K] W^T + b); Wt is [K][H]; thread (tr, to) owns a 4x4 block.
template <int H>
__device__ __forceinline__ void dense_tile(const float* X, int ldx, int K, const float* Wt,
                                           const float* bias, float (&acc)[4][4]) {
    const int to = threadIdx.x % Tile<H>::TO, tr = threadIdx.x / Tile<H>::TO;
    const int r0 = tr * 4, o0 = to * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = bias[o0 + j];
    for (int q = 0; q < K; ++q) {
        const float4 wv = *reinterpret_cast<const float4*>(Wt + (size_t)q * H + o0);
        float x[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = X[(r0 + i) * ldx + q];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            acc[i][0] = fmaf(x[i], wv.x, acc[i][0]);
            acc[i][1] = fmaf(x[i], wv.y, acc[i][1]);
            acc[i][2] = fmaf(x[i], wv.z, acc[i][2]);
            acc[i][3] = fmaf(x[i], wv.w, acc[i][3]);
        }
    }
}

template <int H>
__device__ __forceinline__ void store_tile_smem(float (&acc)[4][4], float* Y, int ldy, bool relu) {
    const int to = threadIdx.x % Tile<H>::TO, tr = threadIdx.x / Tile<H>::TO;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float v = acc[i][j];
            Y[(tr * 4 + i) * ldy + to * 4 + j] = relu ? fmaxf(v, 0.0f) : v;
        }
}

// load one MLP's weights transposed: Wt_k[q][o] = W_k[o][q]
__device__ void load_mlp_weights(const float* w, int in, int H, int out, int depth, float* sm) {
    float* dst = sm;
    const float* src = w;
    for (int layer = 0; layer <= depth; ++layer) {
        const int fi = layer == 0 ? in : H;
        const int fo = layer == depth ? out : H;
        for (int t = threadIdx.x; t < fi * fo; t += blockDim.x) {
            int o = t / fi, q = t % fi;
            dst[q * fo + o] = src[t];
        }
        for (int t = threadIdx.x; t < fo; t += blockDim.x) dst[fi * fo + t] = src[fi * fo + t];
        dst += fi * fo + fo;
        src += fi * fo + fo;
    }
}

template <int H, int MODE>
__device__ __forceinline__ void gather_tile(const MlpArgs& a, int64_t row0, float* X) {
    constexpr int R = Tile<H>::R;
    constexpr int IN = mode_in(MODE, H);
    constexpr int LD = IN + 1;
    if (MODE == MODE_ENC_NODE) {
        for (int r = threadIdx.x; r < R; r += blockDim.x) {
            int64_t i = row0 + r;
            X[r * LD] = i < a.nrows ? (float)(a.b[i] / a.sc[2 * a.row_sys[i] + 1]) : 0.0f;
        }
    } else if (MODE == MODE_ENC_EDGE) {
        for (int r = threadIdx.x; r < R; r += blockDim.x) {
            int64_t k = row0 + r;
            X[r * LD] = k < a.nrows ? (float)edge_input(a.av, a.sc, a.row_sys, a.erow, a.ci, a.adiag_scaled, k)
                                    : 0.0f;
        }
    } else if (MODE == MODE_NODE) {
        for (int idx = threadIdx.x; idx < R * H; idx += blockDim.x) {
            int r = idx / H, q = idx % H;
            int64_t i = row0 + r;
            float v = 0.0f, agg = 0.0f;
            if (i < a.nrows) {
                v = a.vin[i * H + q];
                for (int k = a.rp[i]; k < a.rp[i + 1]; ++k)
                    agg = fmaf(a.ein[(int64_t)k * H + q], a.vin[(int64_t)a.ci[k] * H + q], agg);
            }
            X[r * LD + q] = v;
            X[r * LD + H + q] = agg;
            if (a.agg_out && i < a.nrows) a.agg_out[i * H + q] = agg;
        }
    } else if (MODE == MODE_EDGE) {
        for (int idx = threadIdx.x; idx < R * 3 * H; idx += blockDim.x) {
            int r = idx / (3 * H), qq = idx % (3 * H);
            int part = qq / H, q = qq % H;
            int64_t k = row0 + r;
            float v = 0.0f;
            if (k < a.nrows) {
                if (part == 0) v = a.ein[k * H + q];
                else if (part == 1) v = a.vin[(int64_t)a.erow[k] * H + q];
                else v = a.vin[(int64_t)a.ci[k] * H + q];
            }
            X[r * LD + qq] = v;
        }
    } else {
        for (int idx = threadIdx.x; idx < R * H; idx += blockDim.x) {
            int r = idx / H, q = idx % H;
            int64_t k = row0 + r;
            X[r * LD + q] = k < a.nrows ? a.ein[k * H + q] : 0.0f;
        }
    }
}

// Fused gather + MLP over tiles of rows (grid-stride).  MLP layers:
// Linear(in,H) ReLU [Linear(H,H) ReLU] x (depth-1) Linear(H,out).
template <int H, int MODE>
__global__ void __launch_bounds__(256) k_mlp(MlpArgs a) {
    extern __shared__ __align__(16) float sm[];
    constexpr int R = Tile<H>::R;
    constexpr int IN = mode_in(MODE, H);
    constexpr int OUT = mode_out(MODE, H);
    const int depth = a.depth;
    load_mlp_weights(a.w, IN, H, OUT, depth, sm);
    size_t wfl = (size_t)IN * H + H + (size_t)(depth - 1) * (H * H + H) + (size_t)H * OUT + OUT;
    wfl = (wfl + 3) & ~size_t(3);
    const float* Wt0 = sm;
    const float* b0 = Wt0 + IN * H;
    const float* Wh = b0 + H;
    const float* WtL = Wh + (size_t)(depth - 1) * (H * H + H);
    const float* bL = WtL + H * OUT;
    float* X = sm + wfl;
    float* Hb0 = X + R * (IN + 1);
    float* Hb1 = Hb0 + R * (H + 1);
    __syncthreads();
    const int64_t ntiles = (a.nrows + R - 1) / R;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row0 = tile * R;
        gather_tile<H, MODE>(a, row0, X);
        __syncthreads();
        float acc[4][4];
        dense_tile<H>(X, IN + 1, IN, Wt0, b0, acc);
        store_tile_smem<H>(acc, Hb0, H + 1, true);
        __syncthreads();
        float* cur = Hb0;
        float* nxt = Hb1;
        for (int k = 1; k < depth; ++k) {
            const float* Wk = Wh + (size_t)(k - 1) * (H * H + H);
            dense_tile<H>(cur, H + 1, H, Wk, Wk + H * H, acc);
            store_tile_smem<H>(acc, nxt, H + 1, true);
            __syncthreads();
            float* t = cur; cur = nxt; nxt = t;
        }
        if (OUT == H) {
            dense_tile<H>(cur, H + 1, H, WtL, bL, acc);
            const int to = threadIdx.x % Tile<H>::TO, tr = threadIdx.x / Tile<H>::TO;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int64_t row = row0 + tr * 4 + i;
                if (row < a.nrows)
                    *reinterpret_cast<float4*>(a.out + row * H + to * 4) =
                        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            }
        } else {
            for (int r = threadIdx.x; r < R; r += blockDim.x) {
                int64_t row = row0 + r;
                float s = bL[0];
                for (int q = 0; q < H; ++q) s = fmaf(WtL[q], cur[r * (H + 1) + q], s);
                if (row < a.nrows) a.out[row] = s;
            }
        }
        __syncthreads();
    }
}

template <int H, int MODE>
npcg_status launch_mode(Handle* h, const MlpArgs& a) {
    if (a.nrows == 0) return NPCG_OK;
    const size_t smem = mlp_smem_floats(MODE, H, a.depth) * sizeof(float);
    NPCG_CUDA(h, cudaFuncSetAttribute(k_mlp<H, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (227 * 1024) / (smem + 1024)));
    const int64_t ntiles = (a.nrows + Tile<H>::R - 1) / Tile<H>::R;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)h->num_sms * per_sm));
    k_mlp<H, MODE><<<grid, 256, smem, h->stream>>>(a);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

template <int H>
npcg_status launch_mlp(Handle* h, int mode, const MlpArgs& a) {
    switch (mode) {
        case MODE_ENC_NODE: return launch_mode<H, MODE_ENC_NODE>(h, a);
        case MODE_ENC_EDGE: return launch_mode<H, MODE_ENC_EDGE>(h, a);
        case MODE_NODE: return launch_mode<H, MODE_NODE>(h, a);
        case MODE_EDGE: return launch_mode<H, MODE_EDGE>(h, a);
        default: return launch_mode<H, MODE_DEC>(h, a);
    }
}

}  // namespace

}  // namespace npcg
