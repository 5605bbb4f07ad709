// Training: the loss Eq. (loss_Ab) with its hand-written adjoint through the
// graph network, and Adam (App. A.4).
#include "gnn_common.cuh"

namespace npcg {

namespace {

__global__ void k_adam(int64_t n, float* w, const float* g, float* m, float* v, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace

npcg_status adam_run(Handle* h, int64_t n, float* w, const float* g, float* m, float* v, int t,
                     float lr, float b1, float b2, float eps) {
    if (n == 0) return NPCG_OK;
    float c1 = (float)(1.0 - pow((double)b1, t)), c2 = (float)(1.0 - pow((double)b2, t));
    int blocks = std::max(1, std::min(ceil_div(n, 256), h->num_sms * 8));
    k_adam<<<blocks, 256, 0, h->stream>>>(n, w, g, m, v, lr, b1, b2, eps, c1, c2);
    NPCG_CUDA(h, cudaGetLastError());
    return NPCG_OK;
}

npcg_status loss_grad_run(Handle* h, Pattern*, const double*, int, const double*, const double*,
                          const npcg_gnn_config*, const float*, double*, float*) {
    return set_error(h, NPCG_EINVAL, "loss_and_grad is not available in this build");
}

npcg_status gnn_forward_bf16_run(Handle* h, Pattern*, const double*, const double*,
                                 const npcg_gnn_config*, const float*, double*) {
    return set_error(h, NPCG_EINVAL, "BF16 path is not available in this build");
}

}  // namespace npcg
