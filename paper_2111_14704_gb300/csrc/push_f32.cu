// FP32 instantiation of the push, state-moment and totals kernels.
#include "push.cuh"
#include "push_binned.cuh"
#include "moments_binned.cuh"

namespace rsol {
cudaError_t push_f32(const PushDesc &d, cudaStream_t s) { return push_dispatch<float>(d, s); }
cudaError_t moments_grid_f32(const MomentsDesc &d, cudaStream_t s)
{
    if (d.bin_start && !d.det && (d.bin == 4 || d.bin == 8))
        return moments_binned_dispatch<float>(d, s);
    return moments_dispatch<float>(d, s);
}
cudaError_t totals_f32(const TotalsDesc &d, cudaStream_t s) { return totals_dispatch<float>(d, s); }
cudaError_t losses_f32(const LossDesc &d, cudaStream_t s)
{
    if (d.nn && d.bin_start && (d.bin == 4 || d.bin == 8))
        return losses_binned_dispatch<float>(d, s);
    return losses_dispatch<float>(d, s);
}
cudaError_t fixed_to_grid_f32(long long *fx, void *grid, int64_t count, double inv_scale,
                              int sm_count, cudaStream_t s)
{
    return fixed_dispatch<float>(fx, grid, count, inv_scale, sm_count, s);
}
size_t batch_box_size(int precision) { return batch_box_bytes(precision); }
cudaError_t push_batch_f32(const PushDesc &d, const void *boxes, int n_boxes, uint32_t total_bins,
                           int warps, uint32_t *work, cudaStream_t s)
{
    return push_batch_dispatch<float>(d, boxes, n_boxes, total_bins, warps, work, s);
}
void fill_batch_box_f32(void *dst, int nx, int ny, int nz, int nbx, int nby, int nbz,
                        int64_t node_off, uint32_t bin_base, double h, double adv, double qv, double c)
{
    fill_batch_box<float>(dst, nx, ny, nz, nbx, nby, nbz, node_off, bin_base, h, adv, qv, c);
}
} // namespace rsol
