// Pattern analysis: the sparsity graph of A (Sec. 4.2: one node per row, one
// edge per nonzero, self-loops included), the pattern of L = tril(A) that the
// network writes (Sec. 4.2, App. A.3), and the level sets of the two
// triangular solves of "Solve P z = r" in Algorithm 1, computed on the device.
#include <algorithm>

#include "npcg_internal.cuh"

namespace npcg {

npcg_status radix_sort_pairs(Handle* h, uint32_t* keys, int32_t* vals, int64_t n, int key_bits);

namespace {

__device__ __forceinline__ int find_sys(const int64_t* sys_ptr, int nsys, int64_t row) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sys_ptr[mid] <= row) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Row checks: ascending in-range columns inside the row's system, diagonal
// present.  Counts tril entries and records the row of every entry.
__global__ void k_rows(int64_t n, const int32_t* rp, const int32_t* ci, const int64_t* sys_ptr,
                       int nsys, int32_t* row_sys, int32_t* adiag, int32_t* lcount,
                       int32_t* edge_row, int* flags, int* max_row) {
    int longest = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int s = find_sys(sys_ptr, nsys, i);
        row_sys[i] = s;
        int64_t lo = sys_ptr[s], hi = sys_ptr[s + 1];
        int32_t a = rp[i], b = rp[i + 1];
        int bad = (b < a);
        int d = -1, cnt = 0, prev = -1;
        for (int32_t k = a; k < b && !bad; ++k) {
            int c = ci[k];
            if (c < lo || c >= hi || c <= prev) bad = 1;
            prev = c;
            if (c == i) d = k;
            if (c <= i) ++cnt;
            edge_row[k] = (int32_t)i;
        }
        if (d < 0) bad = 1;
        adiag[i] = d;
        lcount[i] = cnt;
        if (bad) atomicOr(flags, kFlagBadPattern);
        longest = max(longest, b - a);
    }
    // longest row (selects the SpMV mapping): one atomic per warp
    longest = __reduce_max_sync(0xffffffffu, longest);
    if ((threadIdx.x & 31) == 0) atomicMax(max_row, longest);
}

// mirror[k] = position of (j, i) for k = (i, j); the pattern must be symmetric.
__global__ void k_mirror(int64_t nnz, const int32_t* rp, const int32_t* ci, const int32_t* erow,
                         int32_t* mirror, int* flags) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        int i = erow[k], j = ci[k];
        int lo = rp[j], hi = rp[j + 1] - 1, pos = -1;
        while (lo <= hi) {
            int mid = (lo + hi) >> 1;
            int c = ci[mid];
            if (c == i) { pos = mid; break; }
            if (c < i) lo = mid + 1; else hi = mid - 1;
        }
        mirror[k] = pos;
        if (pos < 0) atomicOr(flags, kFlagBadPattern);
    }
}

__global__ void k_fill_tril(int64_t n, const int32_t* rp, const int32_t* ci, const int32_t* Lrp,
                            int32_t* Lci, int32_t* l2a, int32_t* a2l) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t q = Lrp[i];
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            int c = ci[k];
            if (c <= i) {
                Lci[q] = c;
                l2a[q] = k;
                a2l[k] = q;
                ++q;
            } else {
                a2l[k] = -1;
            }
        }
    }
}

// Longest-path levels, sync-free.  Rows are claimed in dependency order
// (ascending for L, descending for L^T) in warp-sized tickets, so every row a
// lane waits on was claimed earlier by a running warp.  A level of -1 means
// "not yet computed".  Each lane polls all of its pending dependencies every
// round; no lane blocks another lane of its warp.
template <bool kUpper>
__global__ void k_levels(int64_t n, const int32_t* rp, const int32_t* ci, int* lev, int* ticket,
                         int* flags, long long spin_limit) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(ticket, 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) return;
        int64_t t = base + lane;
        bool done = t >= n;
        int64_t row = kUpper ? (n - 1 - t) : t;
        int32_t a = 0, b = 0;
        if (!done) { a = rp[row]; b = rp[row + 1]; }
        int best = 0;
        long long spins = 0;
        while (__any_sync(0xffffffffu, !done)) {
            if (!done) {
                bool all = true;
                int m = 0;
                for (int32_t k = a; k < b; ++k) {
                    int c = ci[k];
                    bool dep = kUpper ? (c > row) : (c < row);
                    if (!dep) continue;
                    int lv = ld_relaxed_s32(&lev[c]);
                    if (lv < 0) { all = false; break; }
                    m = max(m, lv + 1);
                }
                if (all) {
                    best = m;
                    st_relaxed_s32(&lev[row], best);
                    done = true;
                }
            }
            if (++spins > spin_limit) {
                if (!done) atomicOr(flags, kFlagTimeout);
                return;
            }
            if ((spins & 1023) == 0 && (ld_relaxed_s32(flags) & kFlagTimeout)) return;
        }
    }
}

__global__ void k_iota_keys(int64_t n, const int* lev, uint32_t* keys, int32_t* vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = (uint32_t)lev[i];
        vals[i] = (int32_t)i;
    }
}

// off-diagonal count of the row at each slot position, reduced to slice width
template <bool kUpper>
__global__ void k_slice_width(int64_t n, int nslices, const int32_t* perm, const int32_t* rp,
                              const int32_t* Lrp, int32_t* width) {
    int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t s = gt >> 5;
    int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    int64_t q = s * kSlice + lane;
    int c = 0;
    if (q < n) {
        int row = perm[q];
        int nl = Lrp[row + 1] - Lrp[row];
        c = kUpper ? (rp[row + 1] - rp[row]) - nl : nl - 1;
    }
    for (int o = 16; o; o >>= 1) c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
    if (lane == 0) width[s] = c;
}

template <bool kUpper>
__global__ void k_slice_fill(int64_t n, int nslices, const int32_t* perm, const int32_t* rp,
                             const int32_t* ci, const int32_t* Lrp, const int32_t* Lci,
                             const int32_t* mirror, const int32_t* a2l, const int64_t* soff,
                             const int32_t* width, int32_t* col, int32_t* src, int32_t* diag_src) {
    int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t s = gt >> 5;
    int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    int64_t q = s * kSlice + lane;
    int w = width[s];
    int64_t off = soff[s];
    int row = q < n ? perm[q] : -1;
    int cnt = 0, first = 0;
    if (row >= 0) {
        int nl = Lrp[row + 1] - Lrp[row];
        if (kUpper) {
            cnt = (rp[row + 1] - rp[row]) - nl;
            first = rp[row + 1] - cnt;         // A entries right of the diagonal
        } else {
            cnt = nl - 1;
            first = Lrp[row];
        }
        diag_src[q] = Lrp[row + 1] - 1;
    }
    for (int k = 0; k < w; ++k) {
        int64_t slot = off + (int64_t)k * kSlice + lane;
        if (k < cnt) {
            if (kUpper) {
                int ka = first + k;                  // (row, c) with c > row
                col[slot] = ci[ka];
                src[slot] = a2l[mirror[ka]];         // L_{c,row}
            } else {
                col[slot] = Lci[first + k];
                src[slot] = first + k;
            }
        } else {
            col[slot] = -1;
            src[slot] = -1;
        }
    }
}

inline int grid_for(long long n, int threads, int cap) {
    long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    return (int)std::min<long long>(g, cap);
}

npcg_status build_tri(Handle* h, Pattern* P, bool upper, TriLayout* T) {
    const int64_t n = P->n;
    NPCG_CUDA(h, T->level.alloc(n));
    NPCG_CUDA(h, T->perm.alloc(n));
    NPCG_CUDA(h, cudaMemsetAsync(T->level.p, 0xff, n * sizeof(int32_t), h->stream));
    NPCG_CUDA(h, cudaMemsetAsync(P->ctl.p, 0, 4 * sizeof(int), h->stream));
    // ctl[2] ticket, ctl[1] flags
    int blocks = h->num_sms * 8;
    if (upper)
        k_levels<true><<<blocks, 256, 0, h->stream>>>(n, P->rp.p, P->ci.p, T->level.p, P->ctl.p + 2, P->ctl.p + 1,
                                                      h->spin_limit);
    else
        k_levels<false><<<blocks, 256, 0, h->stream>>>(n, P->rp.p, P->ci.p, T->level.p, P->ctl.p + 2, P->ctl.p + 1,
                                                      h->spin_limit);
    NPCG_CUDA(h, cudaGetLastError());
    int flags = 0;
    NPCG_TRY(read_scalar(h, P->ctl.p + 1, &flags));
    if (flags & kFlagTimeout) return set_error(h, NPCG_ETIMEOUT, "level-set computation timed out");
    // max level
    DevBuf<uint32_t> keys;
    NPCG_CUDA(h, keys.alloc(n));
    k_iota_keys<<<grid_for(n, 256, 65535), 256, 0, h->stream>>>(n, T->level.p, keys.p, T->perm.p);
    NPCG_CUDA(h, cudaGetLastError());
    NPCG_TRY(radix_sort_pairs(h, keys.p, T->perm.p, n, 32));
    uint32_t maxlev = 0;
    NPCG_TRY(read_scalar(h, keys.p + (n - 1), &maxlev));
    T->nlev = (int32_t)maxlev + 1;
    // SELL-32 slices in level order
    T->nslices = ceil_div(n, kSlice);
    DevBuf<int32_t> width;
    NPCG_CUDA(h, width.alloc(T->nslices));
    NPCG_CUDA(h, T->slice_w.alloc(T->nslices));
    NPCG_CUDA(h, T->slice_off.alloc(T->nslices + 1));
    int thr = 256;
    int g = ceil_div((long long)T->nslices * 32, thr);
    if (upper)
        k_slice_width<true><<<g, thr, 0, h->stream>>>(n, T->nslices, T->perm.p, P->rp.p, P->Lrp.p, T->slice_w.p);
    else
        k_slice_width<false><<<g, thr, 0, h->stream>>>(n, T->nslices, T->perm.p, P->rp.p, P->Lrp.p, T->slice_w.p);
    NPCG_CUDA(h, cudaGetLastError());
    // slot counts = 32 * width
    std::vector<int32_t> wh(T->nslices);
    NPCG_CUDA(h, cudaMemcpyAsync(wh.data(), T->slice_w.p, T->nslices * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    std::vector<int64_t> off(T->nslices + 1, 0);
    for (int s = 0; s < T->nslices; ++s) off[s + 1] = off[s] + (int64_t)wh[s] * kSlice;
    T->slots = off[T->nslices];
    NPCG_CUDA(h, cudaMemcpyAsync(T->slice_off.p, off.data(), off.size() * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, T->col.alloc(std::max<int64_t>(T->slots, 1)));
    NPCG_CUDA(h, T->src.alloc(std::max<int64_t>(T->slots, 1)));
    NPCG_CUDA(h, T->val.alloc(std::max<int64_t>(T->slots, 1)));
    NPCG_CUDA(h, T->val32.alloc(std::max<int64_t>(T->slots, 1)));
    NPCG_CUDA(h, T->diag_src.alloc(n));
    NPCG_CUDA(h, T->dinv.alloc(n));
    NPCG_CUDA(h, T->dinv32.alloc(n));
    if (upper)
        k_slice_fill<true><<<g, thr, 0, h->stream>>>(n, T->nslices, T->perm.p, P->rp.p, P->ci.p, P->Lrp.p,
                                                     P->Lci.p, P->mirror.p, P->a2l.p, T->slice_off.p,
                                                     T->slice_w.p, T->col.p, T->src.p, T->diag_src.p);
    else
        k_slice_fill<false><<<g, thr, 0, h->stream>>>(n, T->nslices, T->perm.p, P->rp.p, P->ci.p, P->Lrp.p,
                                                      P->Lci.p, P->mirror.p, P->a2l.p, T->slice_off.p,
                                                      T->slice_w.p, T->col.p, T->src.p, T->diag_src.p);
    NPCG_CUDA(h, cudaGetLastError());
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    return NPCG_OK;
}

}  // namespace

npcg_status pattern_build(Handle* h, int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                          int32_t nsys, const int64_t* sys_ptr, Pattern* P) {
    if (n <= 0 || nnz < n || n >= (1LL << 31) - 64 || nnz >= (1LL << 31) - 64)
        return set_error(h, NPCG_EINVAL, "n must be > 0, nnz >= n, both < 2^31");
    if (nsys < 1) return set_error(h, NPCG_EINVAL, "nsys must be >= 1");
    P->h = h;
    P->n = n;
    P->nnz = nnz;
    P->nsys = nsys;
    P->sys_ptr_h.assign(nsys + 1, 0);
    if (nsys == 1 || !sys_ptr) {
        if (nsys != 1) return set_error(h, NPCG_EINVAL, "sys_ptr required when nsys > 1");
        P->sys_ptr_h[1] = n;
    } else {
        for (int s = 0; s <= nsys; ++s) P->sys_ptr_h[s] = sys_ptr[s];
        if (P->sys_ptr_h[0] != 0 || P->sys_ptr_h[nsys] != n)
            return set_error(h, NPCG_EINVAL, "sys_ptr must start at 0 and end at n");
        for (int s = 0; s < nsys; ++s)
            if (P->sys_ptr_h[s + 1] <= P->sys_ptr_h[s])
                return set_error(h, NPCG_EINVAL, "every system needs at least one row");
    }
    // host-side check of the row pointer ends (cheap, catches size mismatches)
    int32_t ends[2];
    NPCG_CUDA(h, cudaMemcpyAsync(&ends[0], rp, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(&ends[1], rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    if (ends[0] != 0 || ends[1] != nnz) return set_error(h, NPCG_EINVAL, "row_ptr[0] != 0 or row_ptr[n] != nnz");

    NPCG_CUDA(h, P->sys_ptr.alloc(nsys + 1));
    NPCG_CUDA(h, cudaMemcpyAsync(P->sys_ptr.p, P->sys_ptr_h.data(), (nsys + 1) * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, P->rp.alloc(n + 1));
    NPCG_CUDA(h, P->ci.alloc(nnz));
    NPCG_CUDA(h, cudaMemcpyAsync(P->rp.p, rp, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(P->ci.p, ci, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, h->stream));
    NPCG_CUDA(h, P->row_sys.alloc(n));
    NPCG_CUDA(h, P->adiag.alloc(n));
    NPCG_CUDA(h, P->edge_row.alloc(nnz));
    NPCG_CUDA(h, P->mirror.alloc(nnz));
    NPCG_CUDA(h, P->a2l.alloc(nnz));
    NPCG_CUDA(h, P->ctl.alloc(8));
    NPCG_CUDA(h, cudaMemsetAsync(P->ctl.p, 0, 8 * sizeof(int), h->stream));
    DevBuf<int32_t> lcount, longest;
    NPCG_CUDA(h, lcount.alloc(n));
    NPCG_CUDA(h, longest.alloc(1));
    NPCG_CUDA(h, cudaMemsetAsync(longest.p, 0, sizeof(int32_t), h->stream));
    k_rows<<<grid_for(n, 256, 65535), 256, 0, h->stream>>>(n, P->rp.p, P->ci.p, P->sys_ptr.p, nsys,
                                                           P->row_sys.p, P->adiag.p, lcount.p,
                                                           P->edge_row.p, P->ctl.p + 1, longest.p);
    NPCG_CUDA(h, cudaGetLastError());
    NPCG_TRY(read_scalar(h, longest.p, &P->max_row));
    int flags = 0;
    NPCG_TRY(read_scalar(h, P->ctl.p + 1, &flags));
    if (flags) return set_error(h, NPCG_EINVAL, "malformed CSR: columns must ascend, stay inside the row's system, and include the diagonal");
    k_mirror<<<grid_for(nnz, 256, 65535), 256, 0, h->stream>>>(nnz, P->rp.p, P->ci.p, P->edge_row.p,
                                                               P->mirror.p, P->ctl.p + 1);
    NPCG_CUDA(h, cudaGetLastError());
    NPCG_TRY(read_scalar(h, P->ctl.p + 1, &flags));
    if (flags) return set_error(h, NPCG_EINVAL, "pattern of A is not structurally symmetric");
    NPCG_CUDA(h, P->Lrp.alloc(n + 1));
    NPCG_TRY(scan_i32_to_i32(h, lcount.p, P->Lrp.p, n));
    int32_t nnzL = 0;
    NPCG_TRY(read_scalar(h, P->Lrp.p + n, &nnzL));
    P->nnzL = nnzL;
    NPCG_CUDA(h, P->Lci.alloc(nnzL));
    NPCG_CUDA(h, P->l2a.alloc(nnzL));
    k_fill_tril<<<grid_for(n, 256, 65535), 256, 0, h->stream>>>(n, P->rp.p, P->ci.p, P->Lrp.p, P->Lci.p,
                                                                P->l2a.p, P->a2l.p);
    NPCG_CUDA(h, cudaGetLastError());
    NPCG_TRY(build_tri(h, P, false, &P->fwd));
    NPCG_TRY(build_tri(h, P, true, &P->bwd));
    // reduction chunks: each covers rows of exactly one system.  The
    // elementwise PCG kernels run one block per chunk: the chunk doubles from
    // kChunk rows while the matrix would still give more than about four
    // chunks per SM (up to kChunkMax), so a large system is streamed by fewer,
    // longer-lived blocks (on the 128^3 grid 4096 rows measured best: 0.22 ->
    // 0.17 ms per Jacobi-PCG iteration) and a small one still spreads over
    // the GPU
    int64_t crows = kChunk;
    while (crows < kChunkMax && crows * 4 * h->num_sms < n) crows *= 2;
    P->chunks_h.clear();
    std::vector<int32_t> first(nsys + 1, 0);
    for (int s = 0; s < nsys; ++s) {
        first[s] = (int32_t)P->chunks_h.size();
        for (int64_t r0 = P->sys_ptr_h[s]; r0 < P->sys_ptr_h[s + 1]; r0 += crows) {
            Chunk c;
            c.sys = s;
            c.row0 = (int32_t)r0;
            c.row1 = (int32_t)std::min<int64_t>(r0 + crows, P->sys_ptr_h[s + 1]);
            c.slot = (int32_t)P->chunks_h.size();
            P->chunks_h.push_back(c);
        }
    }
    first[nsys] = (int32_t)P->chunks_h.size();
    P->nchunks = (int32_t)P->chunks_h.size();
    NPCG_CUDA(h, P->chunks.alloc(P->nchunks));
    NPCG_CUDA(h, P->sys_chunk0.alloc(nsys + 1));
    NPCG_CUDA(h, cudaMemcpyAsync(P->chunks.p, P->chunks_h.data(), P->nchunks * sizeof(Chunk),
                                 cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaMemcpyAsync(P->sys_chunk0.p, first.data(), (nsys + 1) * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, h->stream));
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    // level-synchronous layouts (one CTA per system) and the choice of design
    NPCG_TRY(cta_layout_build(h, P, false, &P->cfwd));
    NPCG_TRY(cta_layout_build(h, P, true, &P->cbwd));
    NPCG_TRY(cta_link(h, P));
    NPCG_TRY(trsv_autotune(h, P));
    return NPCG_OK;
}

Pattern::~Pattern() {
    for (auto& g : graph)
        if (g) cudaGraphExecDestroy(g);
}

}  // namespace npcg
