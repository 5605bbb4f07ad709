// Merged-level triangular solves for "Solve P z = r" (Algorithm 1,
// P = L L^T): G consecutive levels form one step of the level-synchronous
// kernel.  With the plan of level_merge.h,
//   y_i = sum_a C_ia r_a - sum_b M_ib y_b   (b in earlier groups, a in the row's own),
// so a direction's solve is one pass r' = C r followed by the
// level-synchronous solve of the unit-diagonal system y = r' - M y over the
// groups.  M and C are evaluated from the loaded factor in G passes.
#include <algorithm>
#include <vector>

#include "level_merge.h"
#include "npcg_internal.cuh"

namespace npcg {

namespace {

// pass s of the plan: the rows of level s modulo G; every term reads L and
// entries of rows of earlier passes of the same group
__global__ void k_merge_pass(int64_t cnt, const int32_t* rows, const int64_t* diag, const double* Lv,
                             const int64_t* mrp, const int64_t* mtp, const int64_t* mtk, const int64_t* mts,
                             double* M, const int64_t* crp, const int64_t* ctp, const int64_t* ctk,
                             const int64_t* cts, double* Cv) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < cnt;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int i = rows[x];
        const double d = Lv[diag[i]];
        for (int64_t e = mrp[i]; e < mrp[i + 1]; ++e) {
            double v = 0.0;
            for (int64_t t = mtp[e]; t < mtp[e + 1]; ++t)
                v += mts[t] < 0 ? Lv[mtk[t]] / d : -(Lv[mtk[t]] / d) * M[mts[t]];
            M[e] = v;
        }
        for (int64_t e = crp[i]; e < crp[i + 1]; ++e) {
            double v = 0.0;
            for (int64_t t = ctp[e]; t < ctp[e + 1]; ++t)
                v += ctk[t] < 0 ? 1.0 / d : -(Lv[ctk[t]] / d) * Cv[cts[t]];
            Cv[e] = v;
        }
    }
}

// out[q] = sum over the C entries e of row cperm[q] of C[e] x[idx[e]]: the
// right-hand side of the merged solve in its processing order
template <class S, class T>
__global__ void k_merge_rhs(int64_t n, const int32_t* cperm, const int64_t* crp, const int32_t* idx,
                            const double* Cv, const S* __restrict__ x, T* __restrict__ out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = cperm[q];
        double v = 0.0;
        for (int64_t e = crp[i]; e < crp[i + 1]; ++e) v = fma(Cv[e], (double)x[idx[e]], v);
        out[q] = (T)v;
    }
}

__global__ void k_merge_fill(int64_t n, double* y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = sentinel_f64();
}

template <class T>
static npcg_status upload(Handle* h, DevBuf<T>& d, const std::vector<T>& v) {
    NPCG_CUDA(h, d.alloc(std::max<size_t>(v.size(), 1)));
    if (!v.empty())
        NPCG_CUDA(h, cudaMemcpyAsync(d.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    return NPCG_OK;
}

// the plan and the layout of one direction
npcg_status merge_build_dir(Handle* h, Pattern* P, bool upper, int G, MergeDir* D) {
    const int64_t n = P->n, nnzL = P->nnzL;
    const TriLayout& T = upper ? P->bwd : P->fwd;
    std::vector<int32_t> Lrp(n + 1), Lci(nnzL), lev(n);
    NPCG_CUDA(h, cudaMemcpyAsync(Lrp.data(), P->Lrp.p, (n + 1) * 4, cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(Lci.data(), P->Lci.p, nnzL * 4, cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(lev.data(), T.level.p, n * 4, cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    // dependencies of every row in this direction, rows ascending: L y = r
    // reads row i's entries left of the diagonal; L^T z = y reads column i
    // below it (through L_ji)
    std::vector<int64_t> drp(n + 1, 0), dval, diag(n);
    std::vector<int32_t> drow;
    for (int64_t i = 0; i < n; ++i) diag[i] = Lrp[i + 1] - 1;
    if (!upper) {
        for (int64_t i = 0; i < n; ++i) {
            for (int32_t k = Lrp[i]; k < Lrp[i + 1] - 1; ++k) {
                drow.push_back(Lci[k]);
                dval.push_back(k);
            }
            drp[i + 1] = (int64_t)drow.size();
        }
    } else {
        for (int64_t i = 0; i < n; ++i)
            for (int32_t k = Lrp[i]; k < Lrp[i + 1] - 1; ++k) drp[Lci[k] + 1]++;
        for (int64_t i = 0; i < n; ++i) drp[i + 1] += drp[i];
        drow.resize(drp[n]);
        dval.resize(drp[n]);
        std::vector<int64_t> fill(drp.begin(), drp.end() - 1);
        for (int64_t i = 0; i < n; ++i)                  // rows ascending within each column
            for (int32_t k = Lrp[i]; k < Lrp[i + 1] - 1; ++k) {
                const int64_t e = fill[Lci[k]]++;
                drow[e] = (int32_t)i;
                dval[e] = k;
            }
    }
    const MergePlan plan = build_merge_plan(n, drp, drow, dval, diag, lev, G);
    if ((int64_t)plan.mcol.size() >= INT32_MAX || (int64_t)plan.ccol.size() >= INT32_MAX)
        return set_error(h, NPCG_EINVAL, "merged-level plan too large");
    D->G = G;
    D->nM = (int64_t)plan.mcol.size();
    D->nC = (int64_t)plan.ccol.size();
    NPCG_TRY(upload(h, D->mrp, plan.mrp));
    NPCG_TRY(upload(h, D->mcol, plan.mcol));
    NPCG_TRY(upload(h, D->mtp, plan.mtp));
    NPCG_TRY(upload(h, D->mtk, plan.mtk));
    NPCG_TRY(upload(h, D->mts, plan.mts));
    NPCG_TRY(upload(h, D->crp, plan.crp));
    NPCG_TRY(upload(h, D->ccol, plan.ccol));
    NPCG_TRY(upload(h, D->ctp, plan.ctp));
    NPCG_TRY(upload(h, D->ctk, plan.ctk));
    NPCG_TRY(upload(h, D->cts, plan.cts));
    NPCG_TRY(upload(h, D->diag, plan.diag));
    // rows by pass
    D->pptr.assign(G + 1, 0);
    for (int64_t i = 0; i < n; ++i) D->pptr[plan.pass[i] + 1]++;
    for (int s = 0; s < G; ++s) D->pptr[s + 1] += D->pptr[s];
    std::vector<int32_t> prows(n);
    {
        std::vector<int64_t> fill(D->pptr.begin(), D->pptr.end() - 1);
        for (int64_t i = 0; i < n; ++i) prows[fill[plan.pass[i]]++] = (int32_t)i;
    }
    NPCG_TRY(upload(h, D->prows, prows));
    // values: M with a trailing 1 (the unit diagonal of the merged system), C
    NPCG_CUDA(h, D->M.alloc(D->nM + 1));
    NPCG_CUDA(h, D->C.alloc(std::max<int64_t>(D->nC, 1)));
    const double one = 1.0;
    NPCG_CUDA(h, cudaMemcpyAsync(D->M.p + D->nM, &one, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    // the level-synchronous layout of the unit-diagonal system over the groups
    CtaDeps deps;
    deps.lev = &plan.grp;
    deps.drp = &plan.mrp;
    deps.drp_dev = D->mrp.p;
    deps.drow_dev = D->mcol.p;
    deps.diag_src = D->nM;
    NPCG_TRY(cta_layout_build(h, P, upper, &D->lay, &deps));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    D->built = true;
    return NPCG_OK;
}

}  // namespace

// Both directions, groups of G levels (one system per CTA, or one large
// system in per-SM row blocks whose dependencies on earlier blocks are
// published, as in the level-synchronous design).
npcg_status merge_build(Handle* h, Pattern* P, int G) {
    if (G < 1 || G > 64) return set_error(h, NPCG_EINVAL, "levels per group must be in [1, 64]");
    // the plan is built on the host (about a kilobyte per row in flight)
    if (P->n > (int64_t)1 << 22) return set_error(h, NPCG_EINVAL, "merged levels are built for up to 2^22 rows");
    if (P->mfwd.built && P->mfwd.G == G && P->mbwd.built && P->mbwd.G == G) return NPCG_OK;
    P->mfwd.built = P->mbwd.built = false;
    NPCG_TRY(merge_build_dir(h, P, false, G, &P->mfwd));
    NPCG_TRY(merge_build_dir(h, P, true, G, &P->mbwd));
    // the backward right-hand side reads y in the forward processing order
    std::vector<int32_t> ccol(std::max<int64_t>(P->mbwd.nC, 1)), cposf(P->n);
    NPCG_CUDA(h, cudaMemcpyAsync(ccol.data(), P->mbwd.ccol.p, P->mbwd.nC * 4, cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(cposf.data(), P->mfwd.lay.cpos.p, P->n * 4, cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int64_t e = 0; e < P->mbwd.nC; ++e) ccol[e] = cposf[ccol[e]];
    ccol.resize(std::max<int64_t>(P->mbwd.nC, 1));
    NPCG_TRY(upload(h, P->mbwd.ccolpos, ccol));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    return NPCG_OK;
}

// M and C of both directions from the factor, and the merged layouts' values
npcg_status merge_factor_load(Handle* h, Pattern* P, const double* L_val) {
    for (MergeDir* D : {&P->mfwd, &P->mbwd}) {
        if (!D->built) return set_error(h, NPCG_EINVAL, "merged-level layouts are not built");
        for (int s = 0; s < D->G; ++s) {
            const int64_t cnt = D->pptr[s + 1] - D->pptr[s];
            if (cnt == 0) continue;
            const int blocks = std::max(1, std::min(ceil_div(cnt, 128), h->num_sms * 8));
            k_merge_pass<<<blocks, 128, 0, h->stream>>>(cnt, D->prows.p + D->pptr[s], D->diag.p, L_val, D->mrp.p,
                                                        D->mtp.p, D->mtk.p, D->mts.p, D->M.p, D->crp.p, D->ctp.p,
                                                        D->ctk.p, D->cts.p, D->C.p);
            NPCG_CUDA(h, cudaGetLastError());
        }
        NPCG_TRY(cta_factor_load(h, &D->lay, D->M.p));
    }
    return NPCG_OK;
}

// z = L^-T L^-1 r through the merged layouts (r natural order, z natural)
npcg_status merge_apply(Handle* h, cudaStream_t s, Pattern* P, bool f32) {
    const int64_t n = P->n;
    const int blocks = std::max(1, std::min(ceil_div(n, 256), h->num_sms * 8));
    const MergeDir& F = P->mfwd;
    const MergeDir& B = P->mbwd;
    if (F.lay.blocked) {
        // row blocks publish y and z in natural order (FP64; the update
        // kernel resets both to the sentinel and the tickets to zero every
        // iteration), so the backward right-hand side reads y there and z
        // needs no permutation
        if (f32) {
            k_merge_rhs<double, float><<<blocks, 256, 0, s>>>(n, F.lay.cperm.p, F.crp.p, F.ccol.p, F.C.p, P->r.p,
                                                              reinterpret_cast<float*>(P->r_cf.p));
            NPCG_TRY(cta_trsv_launch(h, s, P, F.lay, P->r_cf.p, P->yq.p, P->st.p, true, P->ctl.p + 2, P->y.p));
            k_merge_rhs<double, float><<<blocks, 256, 0, s>>>(n, B.lay.cperm.p, B.crp.p, B.ccol.p, B.C.p, P->y.p,
                                                              reinterpret_cast<float*>(P->y_cb.p));
            NPCG_TRY(cta_trsv_launch(h, s, P, B.lay, P->y_cb.p, P->yq.p, P->st.p, true, P->ctl.p + 3, P->z.p));
        } else {
            k_merge_rhs<double, double><<<blocks, 256, 0, s>>>(n, F.lay.cperm.p, F.crp.p, F.ccol.p, F.C.p, P->r.p,
                                                               reinterpret_cast<double*>(P->r_cf.p));
            NPCG_TRY(cta_trsv_launch(h, s, P, F.lay, P->r_cf.p, P->yq.p, P->st.p, false, P->ctl.p + 2, P->y.p));
            k_merge_rhs<double, double><<<blocks, 256, 0, s>>>(n, B.lay.cperm.p, B.crp.p, B.ccol.p, B.C.p, P->y.p,
                                                               reinterpret_cast<double*>(P->y_cb.p));
            NPCG_TRY(cta_trsv_launch(h, s, P, B.lay, P->y_cb.p, P->yq.p, P->st.p, false, P->ctl.p + 3, P->z.p));
        }
        return NPCG_OK;
    }
    if (f32) {
        k_merge_rhs<double, float><<<blocks, 256, 0, s>>>(n, F.lay.cperm.p, F.crp.p, F.ccol.p, F.C.p, P->r.p,
                                                          reinterpret_cast<float*>(P->r_cf.p));
        NPCG_TRY(cta_trsv_launch(h, s, P, F.lay, P->r_cf.p, P->yq.p, P->st.p, true));
        k_merge_rhs<float, float><<<blocks, 256, 0, s>>>(n, B.lay.cperm.p, B.crp.p, B.ccolpos.p, B.C.p,
                                                         reinterpret_cast<const float*>(P->yq.p),
                                                         reinterpret_cast<float*>(P->y_cb.p));
        NPCG_TRY(cta_trsv_launch(h, s, P, B.lay, P->y_cb.p, P->yq.p, P->st.p, true));
    } else {
        k_merge_rhs<double, double><<<blocks, 256, 0, s>>>(n, F.lay.cperm.p, F.crp.p, F.ccol.p, F.C.p, P->r.p,
                                                           reinterpret_cast<double*>(P->r_cf.p));
        NPCG_TRY(cta_trsv_launch(h, s, P, F.lay, P->r_cf.p, P->yq.p, P->st.p, false));
        k_merge_rhs<double, double><<<blocks, 256, 0, s>>>(n, B.lay.cperm.p, B.crp.p, B.ccolpos.p, B.C.p,
                                                           reinterpret_cast<const double*>(P->yq.p),
                                                           reinterpret_cast<double*>(P->y_cb.p));
        NPCG_TRY(cta_trsv_launch(h, s, P, B.lay, P->y_cb.p, P->yq.p, P->st.p, false));
    }
    return cta_permute(h, s, P, B.lay, P->yq.p, f32, B.lay.cpos.p, P->z.p, false);
}

// One direction alone (L y = r, or L^T y = r with transpose): natural-order
// r and y (FP64); the events, when given, bracket the triangular-solve kernel.
npcg_status merge_sptrsv(Handle* h, cudaStream_t s, Pattern* P, int transpose, const double* r, double* y, bool f32,
                         cudaEvent_t e0, cudaEvent_t e1) {
    const MergeDir& D = transpose ? P->mbwd : P->mfwd;
    if (!D.built) return set_error(h, NPCG_EINVAL, "merged-level layouts are not built");
    const int64_t n = P->n;
    const int blocks = std::max(1, std::min(ceil_div(n, 256), h->num_sms * 8));
    if (f32)
        k_merge_rhs<double, float><<<blocks, 256, 0, s>>>(n, D.lay.cperm.p, D.crp.p, D.ccol.p, D.C.p, r,
                                                          reinterpret_cast<float*>(P->r_cf.p));
    else
        k_merge_rhs<double, double><<<blocks, 256, 0, s>>>(n, D.lay.cperm.p, D.crp.p, D.ccol.p, D.C.p, r,
                                                           reinterpret_cast<double*>(P->r_cf.p));
    NPCG_CUDA(h, cudaGetLastError());
    if (D.lay.blocked) {
        // row blocks: published values (sentinel until written) and a ticket
        k_merge_fill<<<blocks, 256, 0, s>>>(n, P->y.p);
        NPCG_CUDA(h, cudaMemsetAsync(P->ctl.p + 2 + (transpose ? 1 : 0), 0, sizeof(int), s));
    }
    if (e0) NPCG_CUDA(h, cudaEventRecord(e0, s));
    NPCG_TRY(cta_trsv_launch(h, s, P, D.lay, P->r_cf.p, P->yq.p, nullptr, f32, P->ctl.p + 2 + (transpose ? 1 : 0),
                             P->y.p));
    if (e1) NPCG_CUDA(h, cudaEventRecord(e1, s));
    return cta_permute(h, s, P, D.lay, P->yq.p, f32, D.lay.cpos.p, y, false);
}

}  // namespace npcg
