// FP64 instantiation of the push, state-moment and totals kernels.  Compiled
// with -fmad=false so every product is rounded as written (like the oracle).
#include "push.cuh"
#include "push_binned.cuh"
#include "moments_binned.cuh"

namespace rsol {
cudaError_t push_f64(const PushDesc &d, cudaStream_t s) { return push_dispatch<double>(d, s); }
cudaError_t moments_grid_f64(const MomentsDesc &d, cudaStream_t s)
{
    if (d.bin_start && !d.det && (d.bin == 4 || d.bin == 8))
        return moments_binned_dispatch<double>(d, s);
    return moments_dispatch<double>(d, s);
}
cudaError_t totals_f64(const TotalsDesc &d, cudaStream_t s) { return totals_dispatch<double>(d, s); }
cudaError_t losses_f64(const LossDesc &d, cudaStream_t s)
{
    if (d.nn && d.bin_start && (d.bin == 4 || d.bin == 8))
        return losses_binned_dispatch<double>(d, s);
    return losses_dispatch<double>(d, s);
}
cudaError_t fixed_to_grid_f64(long long *fx, void *grid, int64_t count, double inv_scale,
                              int sm_count, cudaStream_t s)
{
    return fixed_dispatch<double>(fx, grid, count, inv_scale, sm_count, s);
}
cudaError_t push_batch_f64(const PushDesc &d, const void *boxes, int n_boxes, uint32_t total_bins,
                           int warps, uint32_t *work, cudaStream_t s)
{
    return push_batch_dispatch<double>(d, boxes, n_boxes, total_bins, warps, work, s);
}
void fill_batch_box_f64(void *dst, int nx, int ny, int nz, int nbx, int nby, int nbz,
                        int64_t node_off, uint32_t bin_base, double h, double adv, double qv, double c)
{
    fill_batch_box<double>(dst, nx, ny, nz, nbx, nby, nbz, node_off, bin_base, h, adv, qv, c);
}
} // namespace rsol
