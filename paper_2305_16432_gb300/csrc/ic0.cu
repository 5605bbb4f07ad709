// IC(0) (Sec. 5.1 baseline "IC"): textbook row-oriented incomplete Cholesky
// on the pattern of tril(A),
//   L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj,   L_ii = sqrt(A_ii - sum_k L_ik^2),
// computed sync-free on the device.  Rows are claimed in forward-level order
// (the dependency DAG of IC(0) is the one of L y = r), one lane per row.  A
// row publishes its diagonal last with release semantics; a row that needs
// row j waits (acquire) for L_jj to leave the sentinel.  A non-positive pivot
// marks the system; the host retries it on A + alpha diag(A),
// alpha = 1e-3 * 2^t.
#include <vector>

#include "npcg_internal.cuh"

namespace npcg {

namespace {

__global__ void k_ic0_reset(int64_t n, const int32_t* Lrp, const int32_t* row_sys, const int* todo,
                            double* Lv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (todo[row_sys[i]]) Lv[Lrp[i + 1] - 1] = sentinel_f64();
}

__global__ void __launch_bounds__(256) k_ic0(int64_t n, int nslices, const int32_t* perm,
                                             const int32_t* Lrp, const int32_t* Lci,
                                             const int32_t* l2a, const double* Av,
                                             const int32_t* row_sys, const int* todo,
                                             const double* alpha, double* Lv, int* ticket,
                                             int* flags, int* fail, long long spin_limit) {
    const int lane = threadIdx.x & 31;
    const unsigned long long kS = kSentinelBits;
    for (;;) {
        int slice = 0;
        if (lane == 0) slice = atomicAdd(ticket, 1);
        slice = __shfl_sync(0xffffffffu, slice, 0);
        if (slice >= nslices) return;
        const int64_t q = (int64_t)slice * kSlice + lane;
        int row = q < n ? perm[q] : -1;
        int sys = row >= 0 ? row_sys[row] : 0;
        bool done = row < 0 || !todo[sys];
        int cur = 0;
        double al = 0.0;
        if (!done) { cur = Lrp[row]; al = alpha[sys]; }
        long long spins = 0;
        while (__any_sync(0xffffffffu, !done)) {
            // advance this row as far as its dependencies allow
            while (!done) {
                const int j = Lci[cur];
                const double aij = Av[l2a[cur]];
                if (j < row) {
                    const int dj = Lrp[j + 1] - 1;
                    unsigned long long bits = ld_acquire_u64(Lv + dj);
                    if (bits == kS) break;                    // row j not finished
                    const double ljj = __longlong_as_double((long long)bits);
                    // sum over k < j present in row i and row j
                    double s = aij;
                    int a = Lrp[row], b = Lrp[j];
                    while (a < cur && b < dj) {
                        int ca = Lci[a], cb = Lci[b];
                        if (ca == cb) { s = fma(-Lv[a], __ldcg(Lv + b), s); ++a; ++b; }
                        else if (ca < cb) ++a;
                        else ++b;
                    }
                    Lv[cur] = s / ljj;
                    ++cur;
                } else {
                    double s = aij + al * aij;
                    for (int a = Lrp[row]; a < cur; ++a) s = fma(-Lv[a], Lv[a], s);
                    double lii;
                    if (!(s > 0.0) || !isfinite(s)) {
                        atomicOr(&fail[sys], 1);
                        lii = 1.0;                              // release dependants
                    } else {
                        lii = sqrt(s);
                    }
                    st_release_u64(Lv + cur, (unsigned long long)__double_as_longlong(lii));
                    done = true;
                }
            }
            if (++spins > spin_limit) {
                if (!done) atomicOr(flags, kFlagTimeout | kFlagAbort);
                return;
            }
            if ((spins & 255) == 0) {
                int f = lane == 0 ? ld_relaxed_s32(flags) : 0;
                if (__shfl_sync(0xffffffffu, f, 0) & kFlagAbort) return;
            }
        }
    }
}

}  // namespace

npcg_status ic0_run(Handle* h, Pattern* P, const double* A_val, double* L_val, double* alpha_out) {
    const int nsys = P->nsys;
    DevBuf<int> todo, fail;
    DevBuf<double> alpha;
    NPCG_CUDA(h, todo.alloc(nsys));
    NPCG_CUDA(h, fail.alloc(nsys));
    NPCG_CUDA(h, alpha.alloc(nsys));
    std::vector<int> todo_h(nsys, 1), fail_h(nsys, 0);
    std::vector<double> alpha_h(nsys, 0.0);
    const int blocks = std::max(1, std::min(ceil_div(P->fwd.nslices, 8), h->num_sms * 4));
    for (int t = -1; t <= 30; ++t) {
        NPCG_CUDA(h, cudaMemcpyAsync(todo.p, todo_h.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, h->stream));
        NPCG_CUDA(h, cudaMemcpyAsync(alpha.p, alpha_h.data(), nsys * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        NPCG_CUDA(h, cudaMemsetAsync(fail.p, 0, nsys * sizeof(int), h->stream));
        NPCG_CUDA(h, cudaMemsetAsync(P->ctl.p + 1, 0, 2 * sizeof(int), h->stream));
        k_ic0_reset<<<h->num_sms * 4, 256, 0, h->stream>>>(P->n, P->Lrp.p, P->row_sys.p, todo.p, L_val);
        k_ic0<<<blocks, 256, 0, h->stream>>>(P->n, P->fwd.nslices, P->fwd.perm.p, P->Lrp.p, P->Lci.p,
                                            P->l2a.p, A_val, P->row_sys.p, todo.p, alpha.p, L_val,
                                            P->ctl.p + 2, P->ctl.p + 1, fail.p, h->spin_limit);
        NPCG_CUDA(h, cudaGetLastError());
        int flags = 0;
        NPCG_TRY(read_scalar(h, P->ctl.p + 1, &flags));
        if (flags & kFlagTimeout) return set_error(h, NPCG_ETIMEOUT, "IC(0) wait timed out");
        NPCG_CUDA(h, cudaMemcpyAsync(fail_h.data(), fail.p, nsys * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
        bool any = false;
        for (int s = 0; s < nsys; ++s) {
            todo_h[s] = fail_h[s] ? 1 : 0;
            if (fail_h[s]) {
                any = true;
                alpha_h[s] = 1e-3 * (double)(1LL << (t + 1));
            }
        }
        if (!any) {
            if (alpha_out)
                for (int s = 0; s < nsys; ++s) alpha_out[s] = alpha_h[s];
            return NPCG_OK;
        }
    }
    return set_error(h, NPCG_ENOTSPD, "IC(0) broke down for every shift up to 1e-3 * 2^30");
}

// Symmetric Gauss-Seidel (Sec. 5.1 baseline "Gauss-Seidel", read as the
// symmetric sweep P = (D + L_A) D^-1 (D + L_A)^T): as P = L L^T with
// L = (D + L_A) D^{-1/2} on tril(A), i.e. L_ii = sqrt(A_ii) and
// L_ij = A_ij / sqrt(A_jj).  One thread per entry of L.
__global__ void k_sgs_factor(int64_t nnzL, const int32_t* Lci, const int32_t* l2a, const int32_t* adiag,
                             const double* A_val, double* L_val) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnzL;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int j = Lci[k];
        const int a = l2a[k], dj = adiag[j];
        const double ajj = A_val[dj];
        L_val[k] = a == dj ? sqrt(ajj) : A_val[a] / sqrt(ajj);
    }
}

npcg_status sgs_run(Handle* h, Pattern* P, const double* A_val, double* L_val) {
    const int blocks = std::max(1, std::min(ceil_div(P->nnzL, 256), h->num_sms * 8));
    k_sgs_factor<<<blocks, 256, 0, h->stream>>>(P->nnzL, P->Lci.p, P->l2a.p, P->adiag.p, A_val, L_val);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

}  // namespace npcg
