// Graph-network factor (Sec. 4.2 "Architecture", App. A.3), FP32 path.
//
// Nodes are the rows of A, edges its nonzeros (self-loops included), edge id
// = CSR position.  Each stage is one fused kernel that gathers its input
// rows into shared memory (the message-passing gather included) and runs the
// whole MLP on them with the weights staged in shared memory:
//   encode nodes   v_i  = MLP_v(b_i / ||b||_inf)
//   encode edges   e_ij = MLP_e(A_ij / s),  s = max_i A_ii (per system)
//   node update    v_i  = MLP([v_i || sum_j e_ij (.) v_j])
//   edge update    e_ij = MLP([e_ij || v_i || v_j])
//   decode         s_ij = MLP_dec(e_ij)
//   L_ij = sqrt(s) (s_ij + s_ji) / 2 (i > j),  L_ii = sqrt(s) softplus(s_ii)
#include <algorithm>

#include "gnn_common.cuh"

namespace npcg {

namespace {

// Per-system input scales: sc[2s] = s (max diagonal), sc[2s+1] = ||b||_inf.
// Every reduction chunk (rows of one system) reduces in a block and folds
// its maxima into the system's running maxima, kept as unsigned keys whose
// order is the order of the doubles (so atomicMax is exact and the result
// does not depend on the order of the chunks); a second kernel decodes them
// and leaves the keys at zero for the next call.
__device__ __forceinline__ unsigned long long order_key(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double order_key_inv(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
}

__global__ void k_scales_part(const Chunk* chunks, const int32_t* adiag, const double* av, const double* b,
                              unsigned long long* keys) {
    __shared__ double m0[256], m1[256];
    const Chunk c = chunks[blockIdx.x];
    double a = 0.0, bb = 0.0;
    for (int i = c.row0 + threadIdx.x; i < c.row1; i += blockDim.x) {
        a = fmax(a, av[adiag[i]]);
        if (b) bb = fmax(bb, fabs(b[i]));
    }
    m0[threadIdx.x] = a;
    m1[threadIdx.x] = bb;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) {
            m0[threadIdx.x] = fmax(m0[threadIdx.x], m0[threadIdx.x + o]);
            m1[threadIdx.x] = fmax(m1[threadIdx.x], m1[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicMax(&keys[2 * c.sys], order_key(m0[0]));
        atomicMax(&keys[2 * c.sys + 1], order_key(m1[0]));
    }
}

__global__ void k_scales_fin(int nsys, unsigned long long* keys, double* sc) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsys) {
        const double a = order_key_inv(keys[2 * s]), bb = order_key_inv(keys[2 * s + 1]);
        sc[2 * s] = a;
        sc[2 * s + 1] = bb > 0.0 ? bb : 1.0;
        keys[2 * s] = 0ull;
        keys[2 * s + 1] = 0ull;
    }
}

}  // namespace

npcg_status gnn_scales_run(Handle* h, Pattern* P, const double* A_val, const double* b, double* sc);

namespace {

__device__ __forceinline__ double softplus_d(double z) { return fmax(z, 0.0) + log1p(exp(-fabs(z))); }

// diag_mode 0: L_ij = sqrt(s) (s_ij + s_ji)/2, L_ii = sqrt(s) softplus(s_ii);
// diag_mode 1 (App. A.3, P = L' D L'^T, D = diag(A), unit-diagonal L'):
//   L = L' D^{1/2}: L_ii = sqrt(A_ii), L_ij = sqrt(A_jj) (s_ij + s_ji)/2;
// diag_mode 2 (the same form, rows scaled): L = D^{1/2} L~:
//   L_ii = sqrt(A_ii), L_ij = sqrt(A_ii) (s_ij + s_ji)/2
__global__ void k_assemble_L(int64_t nnzL, const int32_t* l2a, const int32_t* erow, const int32_t* ci,
                             const int32_t* mirror, const int32_t* row_sys, const double* sc,
                             const float* S, const double* av, const int32_t* adiag, int diag_mode,
                             double* L) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnzL;
         q += (int64_t)gridDim.x * blockDim.x) {
        int ka = l2a[q];
        int i = erow[ka], j = ci[ka];
        double v;
        if (diag_mode == 1 || diag_mode == 2) {
            const double dc = sqrt(av[adiag[diag_mode == 1 ? j : i]]);
            v = i == j ? dc : dc * 0.5 * ((double)S[ka] + (double)S[mirror[ka]]);
        } else {
            const double rs = sqrt(sc[2 * row_sys[i]]);
            v = i == j ? rs * softplus_d((double)S[ka]) : rs * 0.5 * ((double)S[ka] + (double)S[mirror[ka]]);
        }
        L[q] = v;
    }
}

template <int H>
npcg_status run_forward(Handle* h, Pattern* P, const double* A_val, const double* b,
                        const npcg_gnn_config* cfg, const float* w, GnnBuffers& B) {
    const int l = cfg->l, lm = cfg->l_mp;
    const int64_t n = P->n, nnz = P->nnz;
    NPCG_TRY(gnn_scales_run(h, P, A_val, b, B.sc));
    GnnOffsets off = gnn_offsets(H, l, lm, cfg->n_mp);
    MlpArgs a = {};
    a.rp = P->rp.p;
    a.ci = P->ci.p;
    a.erow = P->edge_row.p;
    a.row_sys = P->row_sys.p;
    a.sc = B.sc;
    a.av = A_val;
    a.b = b;
    a.adiag_scaled = cfg->diag_mode == NPCG_DIAG_LDLT_ROWS ? P->adiag.p : nullptr;
    // encoders
    a.nrows = n; a.w = w + off.enc_v; a.depth = l; a.out = B.v[0];
    NPCG_TRY(launch_mlp<H>(h, MODE_ENC_NODE, a));
    a.nrows = nnz; a.w = w + off.enc_e; a.depth = l; a.out = B.e[0];
    NPCG_TRY(launch_mlp<H>(h, MODE_ENC_EDGE, a));
    for (int t = 0; t < cfg->n_mp; ++t) {
        const float* vin = B.v[t % 2 == 0 ? 0 : 1];
        float* vout = B.v[t % 2 == 0 ? 1 : 0];
        const float* ein = B.e[t % 2 == 0 ? 0 : 1];
        float* eout = B.e[t % 2 == 0 ? 1 : 0];
        a.nrows = n; a.w = w + off.node[t]; a.depth = lm; a.vin = vin; a.ein = ein; a.out = vout;
        NPCG_TRY(launch_mlp<H>(h, MODE_NODE, a));
        a.nrows = nnz; a.w = w + off.edge[t]; a.depth = lm; a.vin = vout; a.ein = ein; a.out = eout;
        NPCG_TRY(launch_mlp<H>(h, MODE_EDGE, a));
    }
    a.nrows = nnz; a.w = w + off.dec; a.depth = l; a.ein = B.e[cfg->n_mp % 2 == 0 ? 0 : 1]; a.out = B.s;
    NPCG_TRY(launch_mlp<H>(h, MODE_DEC, a));
    return NPCG_OK;
}

// x0_i = (||b||_inf / s) * head output, with the row's system scales
__global__ void k_x0_scale(int64_t n, const int32_t* row_sys, const double* sc, const float* out, double* x0) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int s = row_sys[i];
        x0[i] = sc[2 * s + 1] / sc[2 * s] * (double)out[i];
    }
}

}  // namespace

npcg_status gnn_check_config(Handle* h, const npcg_gnn_config* cfg) {
    if (!cfg) return set_error(h, NPCG_EINVAL, "config is NULL");
    if (cfg->h != 16 && cfg->h != 32 && cfg->h != 64)
        return set_error(h, NPCG_EINVAL, "hidden width h must be 16, 32 or 64");
    if (cfg->n_mp < 0 || cfg->n_mp > 64) return set_error(h, NPCG_EINVAL, "n_mp must be in [0, 64]");
    if (cfg->l < 1 || cfg->l > kMaxDepth || cfg->l_mp < 1 || cfg->l_mp > kMaxDepth)
        return set_error(h, NPCG_EINVAL, "l and l_mp must be in [1, 4]");
    if (cfg->diag_mode != NPCG_DIAG_SOFTPLUS && cfg->diag_mode != NPCG_DIAG_LDLT_DIAGA &&
        cfg->diag_mode != NPCG_DIAG_LDLT_ROWS)
        return set_error(h, NPCG_EINVAL, "unsupported diag_mode");
    if (cfg->precision != NPCG_FP32 && cfg->precision != NPCG_BF16)
        return set_error(h, NPCG_EINVAL, "precision must be NPCG_FP32 or NPCG_BF16");
    if (cfg->x0_head != 0 && cfg->x0_head != 1) return set_error(h, NPCG_EINVAL, "x0_head must be 0 or 1");
    return NPCG_OK;
}

npcg_status gnn_buffers(Handle* h, Pattern* P, int H, int nsets, GnnStore& S) {
    NPCG_CUDA(h, S.v.ensure((size_t)nsets * P->n * H));
    NPCG_CUDA(h, S.e.ensure((size_t)nsets * P->nnz * H));
    NPCG_CUDA(h, S.s.ensure(P->nnz));
    NPCG_CUDA(h, S.sc.ensure((size_t)2 * P->nsys));
    return NPCG_OK;
}

npcg_status gnn_forward_into(Handle* h, Pattern* P, const double* A_val, const double* b,
                             const npcg_gnn_config* cfg, const float* w, GnnBuffers& B) {
    switch (cfg->h) {
        case 16: return run_forward<16>(h, P, A_val, b, cfg, w, B);
        case 32: return run_forward<32>(h, P, A_val, b, cfg, w, B);
        default: return run_forward<64>(h, P, A_val, b, cfg, w, B);
    }
}

npcg_status gnn_scales_run(Handle* h, Pattern* P, const double* A_val, const double* b, double* sc) {
    GnnStore& S = P->gnn;
    if (S.sckey.n < (size_t)2 * P->nsys) {
        NPCG_CUDA(h, S.sckey.alloc((size_t)2 * P->nsys));
        NPCG_CUDA(h, cudaMemsetAsync(S.sckey.p, 0, S.sckey.n * sizeof(unsigned long long), h->stream));
    }
    k_scales_part<<<P->nchunks, 256, 0, h->stream>>>(P->chunks.p, P->adiag.p, A_val, b, S.sckey.p);
    k_scales_fin<<<ceil_div(P->nsys, 128), 128, 0, h->stream>>>(P->nsys, S.sckey.p, sc);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

npcg_status gnn_assemble_L(Handle* h, Pattern* P, const GnnBuffers& B, double* L_val) {
    int blocks = std::max(1, std::min(ceil_div(P->nnzL, 256), h->num_sms * 16));
    k_assemble_L<<<blocks, 256, 0, h->stream>>>(P->nnzL, P->l2a.p, P->edge_row.p, P->ci.p, P->mirror.p,
                                               P->row_sys.p, B.sc, B.s, B.av, P->adiag.p, B.diag_mode, L_val);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

npcg_status gnn_forward_run(Handle* h, Pattern* P, const double* A_val, const double* b,
                            const npcg_gnn_config* cfg, const float* w, double* L_val) {
    NPCG_TRY(gnn_check_config(h, cfg));
    if (cfg->precision == NPCG_BF16) return gnn_forward_bf16_run(h, P, A_val, b, cfg, w, L_val);
    GnnStore& S = P->gnn;
    NPCG_TRY(gnn_buffers(h, P, cfg->h, 2, S));
    GnnBuffers B;
    B.v[0] = S.v.p;
    B.v[1] = S.v.p + (size_t)P->n * cfg->h;
    B.e[0] = S.e.p;
    B.e[1] = S.e.p + (size_t)P->nnz * cfg->h;
    B.s = S.s.p;
    B.sc = S.sc.p;
    B.av = A_val;
    B.diag_mode = cfg->diag_mode;
    NPCG_TRY(gnn_forward_into(h, P, A_val, b, cfg, w, B));
    return gnn_assemble_L(h, P, B, L_val);
}

}  // namespace npcg

namespace npcg {

// Factor and initial guess: the trunk runs once; the head (the decoder's MLP
// shape, h -> 1) runs over the node rows of the final node features.
npcg_status gnn_factor_x0_run(Handle* h, Pattern* P, const double* A_val, const double* b,
                              const npcg_gnn_config* cfg, const float* w, double* L_val, double* x0) {
    NPCG_TRY(gnn_check_config(h, cfg));
    const GnnOffsets off = gnn_offsets(cfg->h, cfg->l, cfg->l_mp, cfg->n_mp, 1);
    GnnStore& S = P->gnn;
    NPCG_TRY(gnn_forward_run(h, P, A_val, b, cfg, w, L_val));     // decoder outputs in S.s are consumed
    if (cfg->precision == NPCG_BF16) {
        NPCG_TRY(gnn_bf16_head_run(h, P, cfg, w + off.x0, S.s.p));
    } else {
        const size_t fv = (size_t)P->n * cfg->h;
        MlpArgs a = {};
        a.rp = P->rp.p;
        a.ci = P->ci.p;
        a.erow = P->edge_row.p;
        a.row_sys = P->row_sys.p;
        a.sc = S.sc.p;
        a.av = A_val;
        a.b = b;
        a.nrows = P->n;
        a.w = w + off.x0;
        a.depth = cfg->l;
        a.ein = S.v.p + (cfg->n_mp % 2) * fv;                       // final node features
        a.out = S.s.p;
        switch (cfg->h) {
            case 16: NPCG_TRY(launch_mlp<16>(h, MODE_DEC, a)); break;
            case 32: NPCG_TRY(launch_mlp<32>(h, MODE_DEC, a)); break;
            default: NPCG_TRY(launch_mlp<64>(h, MODE_DEC, a)); break;
        }
    }
    const int blocks = std::max(1, std::min(ceil_div(P->n, 256), h->num_sms * 8));
    k_x0_scale<<<blocks, 256, 0, h->stream>>>(P->n, P->row_sys.p, S.sc.p, S.s.p, x0);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

}  // namespace npcg
