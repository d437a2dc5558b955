// FP32 instantiation of the push, state-moment and totals kernels.
#include "push.cuh"
#include "push_binned.cuh"

namespace rsol {
cudaError_t push_f32(const PushDesc &d, cudaStream_t s) { return push_dispatch<float>(d, s); }
cudaError_t moments_grid_f32(const MomentsDesc &d, cudaStream_t s) { return moments_dispatch<float>(d, s); }
cudaError_t totals_f32(const TotalsDesc &d, cudaStream_t s) { return totals_dispatch<float>(d, s); }
cudaError_t losses_f32(const LossDesc &d, cudaStream_t s) { return losses_dispatch<float>(d, s); }
cudaError_t fixed_to_grid_f32(long long *fx, void *grid, int64_t count, double inv_scale,
                              int sm_count, cudaStream_t s)
{
    return fixed_dispatch<float>(fx, grid, count, inv_scale, sm_count, s);
}
} // namespace rsol
