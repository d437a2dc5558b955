// Reverse-mode step (FP32) and the loss reduction of the differentiable run.
#include "adjoint.cuh"

namespace rsol {

cudaError_t adjoint_step_f32(const AdjDesc &d, cudaStream_t s) { return launch_adjoint<float>(d, s); }

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

} // namespace rsol
