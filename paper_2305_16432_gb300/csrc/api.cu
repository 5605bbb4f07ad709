// C-ABI entry points of libnpcg (declared in include/npcg.h): argument
// validation, handle / pattern lifetime, and dispatch to the kernels.
#include <cstring>
#include <new>

#include "gnn_common.cuh"
#include "npcg_internal.cuh"

namespace npcg {

npcg_status set_error(Handle* h, npcg_status s, const std::string& msg) {
    if (h) h->last_error = msg;
    return s;
}

npcg_status cuda_fail(Handle* h, cudaError_t e, const char* where) {
    std::string m = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
                    ") at " + where;
    if (e == cudaErrorMemoryAllocation) return set_error(h, NPCG_ENOMEM, m);
    return set_error(h, NPCG_ECUDA, m);
}

}  // namespace npcg

using namespace npcg;

namespace {

Handle* H(npcg_handle h) { return static_cast<Handle*>(h); }
Pattern* PT(npcg_pattern p) { return static_cast<Pattern*>(p); }

npcg_status check_hp(npcg_handle h, npcg_pattern p) {
    if (!h) return NPCG_EINVAL;
    if (!p) return set_error(H(h), NPCG_EINVAL, "pattern is NULL");
    if (!PT(p)->h) return set_error(H(h), NPCG_EINVAL, "the pattern's handle was destroyed");
    if (PT(p)->h != H(h)) return set_error(H(h), NPCG_EINVAL, "pattern was analysed with another handle");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != H(h)->device) return set_error(H(h), NPCG_EINVAL, "current device differs from the handle's device");
    return NPCG_OK;
}

}  // namespace

extern "C" {

const char* npcg_status_string(npcg_status s) {
    switch (s) {
        case NPCG_OK: return "NPCG_OK";
        case NPCG_EINVAL: return "NPCG_EINVAL";
        case NPCG_ENOMEM: return "NPCG_ENOMEM";
        case NPCG_ECUDA: return "NPCG_ECUDA";
        case NPCG_ENOTSPD: return "NPCG_ENOTSPD";
        case NPCG_EBREAKDOWN: return "NPCG_EBREAKDOWN";
        case NPCG_EMAXITER: return "NPCG_EMAXITER";
        case NPCG_ETIMEOUT: return "NPCG_ETIMEOUT";
        case NPCG_ESTALL: return "NPCG_ESTALL";
    }
    return "NPCG_UNKNOWN";
}

npcg_status npcg_create(npcg_handle* out, void* stream) {
    if (!out) return NPCG_EINVAL;
    *out = nullptr;
    npcg_handle_s* h = new (std::nothrow) npcg_handle_s();
    if (!h) return NPCG_ENOMEM;
    h->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete h;
        return e == cudaErrorMemoryAllocation ? NPCG_ENOMEM : NPCG_ECUDA;
    }
    *out = h;
    return NPCG_OK;
}

npcg_status npcg_destroy(npcg_handle h) {
    if (!h) return NPCG_EINVAL;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    // patterns that outlive their handle are detached: every later call with
    // them fails the handle check, and npcg_pattern_free only frees memory
    for (Pattern* p : h->patterns) p->h = nullptr;
    delete h;
    return NPCG_OK;
}

const char* npcg_last_error(npcg_handle h) { return h ? h->last_error.c_str() : "handle is NULL"; }

npcg_status npcg_set_wait_limit(npcg_handle h, int64_t polls) {
    if (!h) return NPCG_EINVAL;
    h->spin_limit = polls > 0 ? (long long)polls : kSpinLimit;
    return NPCG_OK;
}

npcg_status npcg_set_pcg_eager(npcg_handle h, int32_t eager) {
    if (!h) return NPCG_EINVAL;
    h->pcg_eager = eager > 0 ? 1 : eager == 0 ? 0 : -1;
    return NPCG_OK;
}

npcg_status npcg_assemble_count(npcg_handle h, const npcg_problem* p, int64_t* n_out, int64_t* nnz_out) {
    if (!h) return NPCG_EINVAL;
    if (!n_out || !nnz_out) return set_error(H(h), NPCG_EINVAL, "n_out / nnz_out are NULL");
    return assemble_count_run(H(h), p, n_out, nnz_out);
}

npcg_status npcg_assemble_system(npcg_handle h, const npcg_problem* p, int32_t* row_ptr,
                                 int32_t* col_idx, double* val) {
    if (!h) return NPCG_EINVAL;
    if (!row_ptr || !col_idx || !val) return set_error(H(h), NPCG_EINVAL, "output arrays are NULL");
    return assemble_run(H(h), p, row_ptr, col_idx, val);
}

npcg_status npcg_analyse(npcg_handle h, int64_t n, int64_t nnz, const int32_t* row_ptr,
                         const int32_t* col_idx, int32_t nsys, const int64_t* sys_ptr,
                         npcg_pattern* out) {
    if (!h) return NPCG_EINVAL;
    if (!out || !row_ptr || !col_idx) return set_error(H(h), NPCG_EINVAL, "NULL argument");
    *out = nullptr;
    npcg_pattern_s* P = new (std::nothrow) npcg_pattern_s();
    if (!P) return set_error(H(h), NPCG_ENOMEM, "host allocation failed");
    npcg_status s = pattern_build(H(h), n, nnz, row_ptr, col_idx, nsys, sys_ptr, P);
    if (s != NPCG_OK) {
        delete P;
        return s;
    }
    H(h)->patterns.push_back(P);
    *out = P;
    return NPCG_OK;
}

npcg_status npcg_pattern_free(npcg_pattern p) {
    if (!p) return NPCG_EINVAL;
    if (p->h) {
        if (p->h->stream) cudaStreamSynchronize(p->h->stream);
        auto& v = p->h->patterns;
        for (size_t k = 0; k < v.size(); ++k)
            if (v[k] == p) { v.erase(v.begin() + (long)k); break; }
    }
    delete p;
    return NPCG_OK;
}

npcg_status npcg_pattern_get_info(npcg_pattern p, npcg_pattern_info* out) {
    if (!p || !out) return NPCG_EINVAL;
    out->n = p->n;
    out->nnz = p->nnz;
    out->nnz_L = p->nnzL;
    out->nsys = p->nsys;
    out->nlev_fwd = p->fwd.nlev;
    out->nlev_bwd = p->bwd.nlev;
    out->trsv_mode = p->trsv_mode != kTrsvCta ? NPCG_TRSV_SYNCFREE
                   : p->cta_flag ? NPCG_TRSV_LEVELFLAG
                   : p->cta_split ? NPCG_TRSV_LEVELSPLIT
                   : p->cta_merge ? NPCG_TRSV_LEVELMERGE : NPCG_TRSV_LEVELSYNC;
    out->tuned_ms_syncfree = p->tune_ms[0];
    out->tuned_ms_levelsync = p->tune_ms[1];
    out->tuned_ms_levelflag = p->tune_ms[2];
    out->tuned_ms_levelsplit = p->tune_ms[3];
    out->tuned_ms_levelmerge = p->tune_ms[4];
    out->merge_levels = p->mfwd.built ? p->mfwd.G : 0;
    out->block_units = p->cfwd.blocked ? p->cfwd.nunits : 0;
    out->max_row = p->max_row;
    return NPCG_OK;
}

npcg_status npcg_pattern_set_trsv(npcg_pattern p, int32_t mode) {
    if (!p || !p->h) return NPCG_EINVAL;
    if (mode == NPCG_TRSV_AUTO) {
        trsv_pick_tuned(p);
    } else if (mode == NPCG_TRSV_LEVELMERGE) {
        if (!kMergeEnabled) return set_error(p->h, NPCG_EINVAL, "merged-level solves are not enabled yet");
        if (!p->cfwd.built || cta_stages(p->cfwd) < 2 || cta_stages(p->cbwd) < 2)
            return set_error(p->h, NPCG_EINVAL, "level-synchronous layout does not fit shared memory");
        NPCG_TRY(merge_build(p->h, p, p->merge_G ? p->merge_G : kMergeLevels));
        if (cta_stages(p->mfwd.lay) < 2 || cta_stages(p->mbwd.lay) < 2)
            return set_error(p->h, NPCG_EINVAL, "merged-level layout does not fit shared memory");
        p->trsv_mode = kTrsvCta;
        p->cta_flag = false;
        p->cta_split = false;
        p->cta_merge = true;
    } else if (mode == NPCG_TRSV_SYNCFREE) {
        p->trsv_mode = kTrsvSyncFree;
        p->cta_flag = false;
        p->cta_split = false;
        p->cta_merge = false;
    } else if (mode == NPCG_TRSV_LEVELSYNC || mode == NPCG_TRSV_LEVELFLAG || mode == NPCG_TRSV_LEVELSPLIT) {
        if (!p->cfwd.built || cta_stages(p->cfwd) < 2 || cta_stages(p->cbwd) < 2)
            return set_error(p->h, NPCG_EINVAL, "level-synchronous layout does not fit shared memory");
        if (mode == NPCG_TRSV_LEVELFLAG && !(p->cfwd.flag_ok && p->cbwd.flag_ok))
            return set_error(p->h, NPCG_EINVAL, "flag-synchronised solve: the window does not cover its drift");
        if (mode == NPCG_TRSV_LEVELSPLIT &&
            !(p->cfwd.split_stages[0] >= 2 && p->cfwd.split_stages[1] >= 2 && p->cbwd.split_stages[0] >= 2 &&
              p->cbwd.split_stages[1] >= 2))
            return set_error(p->h, NPCG_EINVAL, "split-role solve: the layout does not fit beside the staging slots");
        p->trsv_mode = kTrsvCta;
        p->cta_flag = mode == NPCG_TRSV_LEVELFLAG;
        p->cta_split = mode == NPCG_TRSV_LEVELSPLIT;
        p->cta_merge = false;
    } else {
        return set_error(p->h, NPCG_EINVAL, "unknown triangular-solve mode");
    }
    return NPCG_OK;
}

npcg_status npcg_pattern_export(npcg_handle h, npcg_pattern p, int32_t* L_row_ptr, int32_t* L_col_idx,
                                int32_t* lev_fwd, int32_t* lev_bwd, int32_t* perm_fwd, int32_t* perm_bwd) {
    NPCG_TRY(check_hp(h, p));
    Handle* hh = H(h);
    Pattern* P = PT(p);
    auto cp = [&](int32_t* dst, const int32_t* src, int64_t cnt) -> npcg_status {
        if (dst) NPCG_CUDA(hh, cudaMemcpyAsync(dst, src, cnt * sizeof(int32_t), cudaMemcpyDeviceToDevice, hh->stream));
        return NPCG_OK;
    };
    NPCG_TRY(cp(L_row_ptr, P->Lrp.p, P->n + 1));
    NPCG_TRY(cp(L_col_idx, P->Lci.p, P->nnzL));
    NPCG_TRY(cp(lev_fwd, P->fwd.level.p, P->n));
    NPCG_TRY(cp(lev_bwd, P->bwd.level.p, P->n));
    NPCG_TRY(cp(perm_fwd, P->fwd.perm.p, P->n));
    NPCG_TRY(cp(perm_bwd, P->bwd.perm.p, P->n));
    return NPCG_OK;
}

npcg_status npcg_gnn_nparams(const npcg_gnn_config* cfg, int64_t* out) {
    if (!cfg || !out) return NPCG_EINVAL;
    if (cfg->n_mp < 0 || cfg->n_mp > kMaxMp || cfg->h <= 0 || cfg->l < 1 || cfg->l_mp < 1) return NPCG_EINVAL;
    *out = gnn_offsets(cfg->h, cfg->l, cfg->l_mp, cfg->n_mp, cfg->x0_head).total;
    return NPCG_OK;
}

npcg_status npcg_gnn_factor(npcg_handle h, npcg_pattern p, const double* A_val, const double* b,
                            const npcg_gnn_config* cfg, const float* weights, double* L_val) {
    NPCG_TRY(check_hp(h, p));
    if (!A_val || !b || !weights || !L_val) return set_error(H(h), NPCG_EINVAL, "NULL array argument");
    return gnn_forward_run(H(h), PT(p), A_val, b, cfg, weights, L_val);
}

npcg_status npcg_gnn_factor_x0(npcg_handle h, npcg_pattern p, const double* A_val, const double* b,
                               const npcg_gnn_config* cfg, const float* weights, double* L_val, double* x0) {
    NPCG_TRY(check_hp(h, p));
    if (!A_val || !b || !cfg || !weights || !L_val || !x0) return set_error(H(h), NPCG_EINVAL, "NULL argument");
    if (cfg->x0_head != 1) return set_error(H(h), NPCG_EINVAL, "npcg_gnn_factor_x0 needs cfg->x0_head = 1");
    return gnn_factor_x0_run(H(h), PT(p), A_val, b, cfg, weights, L_val, x0);
}

npcg_status npcg_sgs_factor(npcg_handle h, npcg_pattern p, const double* A_val, double* L_val) {
    NPCG_TRY(check_hp(h, p));
    if (!A_val || !L_val) return set_error(H(h), NPCG_EINVAL, "NULL argument");
    return sgs_run(H(h), PT(p), A_val, L_val);
}

npcg_status npcg_ic0_factor(npcg_handle h, npcg_pattern p, const double* A_val, double* L_val,
                            double* alpha_out) {
    NPCG_TRY(check_hp(h, p));
    if (!A_val || !L_val) return set_error(H(h), NPCG_EINVAL, "NULL array argument");
    return ic0_run(H(h), PT(p), A_val, L_val, alpha_out);
}

npcg_status npcg_pcg_solve(npcg_handle h, npcg_pattern p, const double* A_val, const double* b,
                           double* x, int32_t precond, const double* L_val, double rtol,
                           int32_t max_iter, npcg_solve_stats* stats) {
    NPCG_TRY(check_hp(h, p));
    if (PT(p)->nsys != 1) return set_error(H(h), NPCG_EINVAL, "npcg_pcg_solve needs a single-system pattern; use npcg_pcg_solve_batched");
    if (!A_val || !b || !x || !stats) return set_error(H(h), NPCG_EINVAL, "NULL array argument");
    return pcg_run(H(h), PT(p), A_val, b, x, precond, L_val, rtol, max_iter, stats);
}

npcg_status npcg_pcg_solve_batched(npcg_handle h, npcg_pattern p, const double* A_val, const double* b,
                                   double* x, int32_t precond, const double* L_val, double rtol,
                                   int32_t max_iter, npcg_solve_stats* stats) {
    NPCG_TRY(check_hp(h, p));
    if (!A_val || !b || !x || !stats) return set_error(H(h), NPCG_EINVAL, "NULL array argument");
    return pcg_run(H(h), PT(p), A_val, b, x, precond, L_val, rtol, max_iter, stats);
}

npcg_status npcg_pcg_solve_ex(npcg_handle h, npcg_pattern p, const double* A_val, const double* b, double* x,
                              int32_t precond, const double* L_val, double rtol, int32_t max_iter,
                              const npcg_solve_opts* opts, npcg_solve_stats* stats) {
    NPCG_TRY(check_hp(h, p));
    if (!A_val || !b || !x || !stats) return set_error(H(h), NPCG_EINVAL, "NULL array argument");
    return pcg_run_ex(H(h), PT(p), A_val, b, x, precond, L_val, rtol, max_iter, opts, stats);
}

npcg_status npcg_spmv(npcg_handle h, npcg_pattern p, const double* A_val, const double* x, double* y) {
    NPCG_TRY(check_hp(h, p));
    if (!A_val || !x || !y) return set_error(H(h), NPCG_EINVAL, "NULL array argument");
    return spmv_run(H(h), PT(p), A_val, x, y);
}

npcg_status npcg_factor_load(npcg_handle h, npcg_pattern p, const double* L_val) {
    NPCG_TRY(check_hp(h, p));
    if (!L_val) return set_error(H(h), NPCG_EINVAL, "NULL array argument");
    return factor_load(H(h), PT(p), L_val);
}

npcg_status npcg_sptrsv(npcg_handle h, npcg_pattern p, int32_t transpose, const double* r, double* y) {
    NPCG_TRY(check_hp(h, p));
    if (!r || !y || r == y) return set_error(H(h), NPCG_EINVAL, "r and y must be distinct non-NULL arrays");
    npcg_status s = sptrsv_run(H(h), PT(p), transpose ? 1 : 0, r, y, nullptr);
    if (s != NPCG_OK) return s;
    int flags = 0;
    NPCG_TRY(read_scalar(H(h), PT(p)->ctl.p + 1, &flags));
    if (flags & kFlagTimeout) return set_error(H(h), NPCG_ETIMEOUT, "triangular solve wait timed out");
    return NPCG_OK;
}

npcg_status npcg_sptrsv_unclaimed(npcg_handle h, npcg_pattern p, int32_t transpose, int32_t skip, const double* r,
                                  double* y) {
    NPCG_TRY(check_hp(h, p));
    if (!r || !y || r == y) return set_error(H(h), NPCG_EINVAL, "r and y must be distinct non-NULL arrays");
    NPCG_TRY(sptrsv_unclaimed_run(H(h), PT(p), transpose ? 1 : 0, skip, r, y));
    int flags = 0;
    NPCG_TRY(read_scalar(H(h), PT(p)->ctl.p + 1, &flags));
    if (flags & kFlagTimeout) return set_error(H(h), NPCG_ETIMEOUT, "triangular solve wait timed out");
    return NPCG_OK;
}

npcg_status npcg_sptrsv_timed(npcg_handle h, npcg_pattern p, int32_t transpose, int32_t f32, const double* r,
                              double* y, int32_t reps, double* ms_per_launch) {
    NPCG_TRY(check_hp(h, p));
    if (!r || !y || r == y || !ms_per_launch || reps < 1)
        return set_error(H(h), NPCG_EINVAL, "bad argument");
    return sptrsv_timed_run(H(h), PT(p), transpose ? 1 : 0, r, y, reps, ms_per_launch, f32 != 0);
}

npcg_status npcg_loss_and_grad(npcg_handle h, npcg_pattern p, const double* A_val, int32_t npairs,
                               const double* X, const double* B, const npcg_gnn_config* cfg,
                               const float* weights, double* loss_out, float* grad) {
    NPCG_TRY(check_hp(h, p));
    if (!A_val || !X || !B || !cfg || !weights || !loss_out || !grad)
        return set_error(H(h), NPCG_EINVAL, "NULL argument");
    if (npairs < 1) return set_error(H(h), NPCG_EINVAL, "npairs must be >= 1");
    return loss_grad_run(H(h), PT(p), A_val, npairs, X, B, cfg, weights, loss_out, grad);
}

npcg_status npcg_adam_step(npcg_handle h, int64_t n, float* w, const float* g, float* m, float* v,
                           int32_t t, float lr, float beta1, float beta2, float eps) {
    if (!h) return NPCG_EINVAL;
    if (!w || !g || !m || !v || n < 0 || t < 1) return set_error(H(h), NPCG_EINVAL, "bad Adam argument");
    return adam_run(H(h), n, w, g, m, v, t, lr, beta1, beta2, eps);
}

npcg_status npcg_solve_host(npcg_handle h, npcg_pattern p, int32_t method, const npcg_gnn_config* cfg,
                            const float* weights, const double* A_val_host, const double* b_host,
                            double* x_host, double rtol, int32_t max_iter, int32_t f32_apply,
                            npcg_solve_stats* stats) {
    NPCG_TRY(check_hp(h, p));
    Handle* hh = H(h);
    Pattern* P = PT(p);
    if (!A_val_host || !b_host || !x_host || !stats) return set_error(hh, NPCG_EINVAL, "NULL argument");
    if (method < NPCG_METHOD_GNN || method > NPCG_METHOD_SGS) return set_error(hh, NPCG_EINVAL, "unknown method");
    if (method == NPCG_METHOD_GNN && (!cfg || !weights)) return set_error(hh, NPCG_EINVAL, "GNN method needs cfg and weights");
    NPCG_CUDA(hh, P->Aval_dev.ensure(P->nnz));
    NPCG_CUDA(hh, P->b.ensure(P->n));
    NPCG_CUDA(hh, P->x.ensure(P->n));
    NPCG_CUDA(hh, P->Lval_dev.ensure(P->nnzL));
    NPCG_CUDA(hh, cudaMemcpyAsync(P->Aval_dev.p, A_val_host, P->nnz * sizeof(double), cudaMemcpyHostToDevice, hh->stream));
    NPCG_CUDA(hh, cudaMemcpyAsync(P->b.p, b_host, P->n * sizeof(double), cudaMemcpyHostToDevice, hh->stream));
    NPCG_CUDA(hh, cudaMemsetAsync(P->x.p, 0, P->n * sizeof(double), hh->stream));
    int precond = f32_apply ? NPCG_PREC_LLT32 : NPCG_PREC_LLT;
    if (method == NPCG_METHOD_GNN) NPCG_TRY(gnn_forward_run(hh, P, P->Aval_dev.p, P->b.p, cfg, weights, P->Lval_dev.p));
    else if (method == NPCG_METHOD_IC0) NPCG_TRY(ic0_run(hh, P, P->Aval_dev.p, P->Lval_dev.p, nullptr));
    else if (method == NPCG_METHOD_SGS) NPCG_TRY(sgs_run(hh, P, P->Aval_dev.p, P->Lval_dev.p));
    else precond = method == NPCG_METHOD_JACOBI ? NPCG_PREC_JACOBI : NPCG_PREC_NONE;
    // the learned factor falls back to IC(0) on breakdown, max_iter or stagnation
    npcg_solve_opts fb = {200, 1};
    npcg_status s = pcg_run_ex(hh, P, P->Aval_dev.p, P->b.p, P->x.p, precond, P->Lval_dev.p, rtol, max_iter,
                               method == NPCG_METHOD_GNN ? &fb : nullptr, stats);
    cudaError_t e = cudaMemcpyAsync(x_host, P->x.p, P->n * sizeof(double), cudaMemcpyDeviceToHost, hh->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hh->stream);
    if (e != cudaSuccess) return cuda_fail(hh, e, "copy of x to the host");
    return s;
}

}  // extern "C"
