// Reverse-mode step (FP32) and the loss reduction of the differentiable run.
#include "adjoint_binned.cuh"

namespace rsol {

cudaError_t adjoint_step_f32(const AdjDesc &d, cudaStream_t s) { return adjoint_dispatch<float>(d, s); }

cudaError_t loss_norm(const void *fb, int64_t n_nodes, int precision, double *partials, int blocks,
                      double *loss, cudaStream_t s)
{
    if (precision == 32)
        loss_partials_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float *>(fb), n_nodes, partials);
    else
        loss_partials_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double *>(fb), n_nodes, partials);
    loss_final_kernel<<<1, 256, 0, s>>>(partials, blocks, loss);
    return cudaGetLastError();
}

namespace {

// out_q[perm[t]] = in_q[t] for the six adjoint arrays (E: 4- or 8-byte words)
template <typename E>
__global__ void __launch_bounds__(256) unpermute_kernel(int64_t n, const uint32_t *__restrict__ perm,
                                                        const E *i0, const E *i1, const E *i2,
                                                        const E *i3, const E *i4, const E *i5, E *o0,
                                                        E *o1, E *o2, E *o3, E *o4, E *o5)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += stride) {
        const uint32_t d = perm[t];
        o0[d] = i0[t];
        o1[d] = i1[t];
        o2[d] = i2[t];
        o3[d] = i3[t];
        o4[d] = i4[t];
        o5[d] = i5[t];
    }
}

} // namespace

cudaError_t unpermute6(int64_t n, int es, const uint32_t *perm, void *const xb_in[3],
                       void *const ub_in[3], void *const xb_out[3], void *const ub_out[3],
                       int sm_count, cudaStream_t s)
{
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = int64_t(sm_count) * 8 * 4;
    blocks = blocks > cap ? cap : (blocks < 1 ? 1 : blocks);
    if (es == 4) {
        using E = uint32_t;
        unpermute_kernel<E><<<unsigned(blocks), 256, 0, s>>>(
            n, perm, static_cast<const E *>(xb_in[0]), static_cast<const E *>(xb_in[1]),
            static_cast<const E *>(xb_in[2]), static_cast<const E *>(ub_in[0]),
            static_cast<const E *>(ub_in[1]), static_cast<const E *>(ub_in[2]), static_cast<E *>(xb_out[0]),
            static_cast<E *>(xb_out[1]), static_cast<E *>(xb_out[2]), static_cast<E *>(ub_out[0]),
            static_cast<E *>(ub_out[1]), static_cast<E *>(ub_out[2]));
    } else {
        using E = unsigned long long;
        unpermute_kernel<E><<<unsigned(blocks), 256, 0, s>>>(
            n, perm, static_cast<const E *>(xb_in[0]), static_cast<const E *>(xb_in[1]),
            static_cast<const E *>(xb_in[2]), static_cast<const E *>(ub_in[0]),
            static_cast<const E *>(ub_in[1]), static_cast<const E *>(ub_in[2]), static_cast<E *>(xb_out[0]),
            static_cast<E *>(xb_out[1]), static_cast<E *>(xb_out[2]), static_cast<E *>(ub_out[0]),
            static_cast<E *>(ub_out[1]), static_cast<E *>(ub_out[2]));
    }
    return cudaGetLastError();
}

} // namespace rsol
