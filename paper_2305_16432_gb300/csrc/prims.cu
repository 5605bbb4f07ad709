// Device primitives used by pattern analysis: exclusive scan and a stable LSD
// radix sort of (key, value) pairs.  Pattern analysis runs once per sparsity
// pattern, so these favour simplicity over peak throughput.
#include "npcg_internal.cuh"

namespace npcg {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* total) {
    __shared__ long long warp_sums[kScanThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    long long before = warp ? warp_sums[warp - 1] : 0;
    *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void scan_tile_sums(const int32_t* in, int64_t n, long long* bsum) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    long long s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    long long tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void scan_block_offsets(long long* bsum, int64_t nb) {
    long long carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        int64_t i = b0 + threadIdx.x;
        long long v = i < nb ? bsum[i] : 0;
        long long tot;
        long long ex = block_exclusive_scan(v, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
}

template <class OutT>
__global__ void scan_tile_apply(const int32_t* in, int64_t n, const long long* boff, OutT* out) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    long long tot;
    long long ex = block_exclusive_scan(s, &tot) + boff[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = (OutT)ex;
        ex += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = (OutT)ex;
}

template <class OutT>
npcg_status scan_impl(Handle* h, const int32_t* in, OutT* out, int64_t n) {
    int64_t nb = n > 0 ? ceil_div(n, kScanTile) : 1;
    DevBuf<long long> bsum;
    NPCG_CUDA(h, bsum.alloc(nb));
    if (n == 0) {
        NPCG_CUDA(h, cudaMemsetAsync(out, 0, sizeof(OutT), h->stream));
        return NPCG_OK;
    }
    scan_tile_sums<<<(unsigned)nb, kScanThreads, 0, h->stream>>>(in, n, bsum.p);
    scan_block_offsets<<<1, kScanThreads, 0, h->stream>>>(bsum.p, nb);
    scan_tile_apply<OutT><<<(unsigned)nb, kScanThreads, 0, h->stream>>>(in, n, bsum.p, out);
    NPCG_CUDA(h, cudaGetLastError());
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));   // bsum is freed on return
    return NPCG_OK;
}

// ---------------------------------------------------------------- radix sort
constexpr int kRadixThreads = 256;
constexpr int kRadixChunks = 16;
constexpr int kRadixTile = kRadixThreads * kRadixChunks;

__global__ void radix_hist(const uint32_t* keys, int64_t n, int shift, int32_t* hist, int nblocks) {
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int c = 0; c < kRadixChunks; ++c) {
        int64_t i = base + (int64_t)c * kRadixThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: within a block items keep their input order per digit.
__global__ void radix_scatter(const uint32_t* kin, const int32_t* vin, uint32_t* kout,
                              int32_t* vout, int64_t n, int shift, const int32_t* offs,
                              int nblocks) {
    __shared__ int run[256];
    __shared__ int wcnt[kRadixThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int c = 0; c < kRadixChunks; ++c) {
        for (int w = 0; w < kRadixThreads / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)c * kRadixThreads + tid;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        int digit = (int)((key >> shift) & 255u);
        unsigned peers = __match_any_sync(0xffffffffu, valid ? digit : 0x1000);
        int intra = __popc(peers & lt_mask);
        if (valid && intra == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            int acc = run[tid];
            for (int w = 0; w < kRadixThreads / 32; ++w) {
                int t = wcnt[w][tid];
                wcnt[w][tid] = acc;
                acc += t;
            }
            run[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            int pos = wcnt[warp][digit] + intra;
            kout[pos] = key;
            vout[pos] = vin[i];
        }
        __syncthreads();
    }
}

}  // namespace

npcg_status scan_i32_to_i64(Handle* h, const int32_t* in, int64_t* out, int64_t n) {
    return scan_impl<int64_t>(h, in, out, n);
}
npcg_status scan_i32_to_i32(Handle* h, const int32_t* in, int32_t* out, int64_t n) {
    return scan_impl<int32_t>(h, in, out, n);
}

// Sorts (keys, vals) stably by the low key_bits of keys.  Results end in the
// original buffers.  n < 2^31.
npcg_status radix_sort_pairs(Handle* h, uint32_t* keys, int32_t* vals, int64_t n, int key_bits) {
    if (n <= 1) return NPCG_OK;
    int nblocks = ceil_div(n, kRadixTile);
    DevBuf<uint32_t> k2;
    DevBuf<int32_t> v2, hist, offs;
    NPCG_CUDA(h, k2.alloc(n));
    NPCG_CUDA(h, v2.alloc(n));
    NPCG_CUDA(h, hist.alloc((size_t)256 * nblocks));
    NPCG_CUDA(h, offs.alloc((size_t)256 * nblocks + 1));
    uint32_t *ka = keys, *kb = k2.p;
    int32_t *va = vals, *vb = v2.p;
    int passes = 0;
    for (int shift = 0; shift < key_bits; shift += 8, ++passes) {
        radix_hist<<<nblocks, kRadixThreads, 0, h->stream>>>(ka, n, shift, hist.p, nblocks);
        NPCG_TRY(scan_i32_to_i32(h, hist.p, offs.p, (int64_t)256 * nblocks));
        radix_scatter<<<nblocks, kRadixThreads, 0, h->stream>>>(ka, va, kb, vb, n, shift, offs.p,
                                                                 nblocks);
        NPCG_CUDA(h, cudaGetLastError());
        uint32_t* tk = ka; ka = kb; kb = tk;
        int32_t* tv = va; va = vb; vb = tv;
    }
    if (passes & 1) {
        NPCG_CUDA(h, cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, h->stream));
        NPCG_CUDA(h, cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, h->stream));
    }
    NPCG_CUDA(h, cudaStreamSynchronize(h->stream));
    return NPCG_OK;
}

}  // namespace npcg
