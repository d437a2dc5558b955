// FP64 instantiation of the sub-cycled push (-fmad=false, as push_f64.cu).
#include "subcycle.cuh"

namespace rsol {
cudaError_t push_subcycled_f64(const PushDesc &d, const SubDesc &sd, cudaStream_t s)
{
    return subcycle_dispatch<double>(d, sd, s);
}
cudaError_t level_keys_f64(const PushDesc &d, const SubDesc &sd, int lb, int nbx, int nby,
                          uint32_t nbins, uint32_t *keys, cudaStream_t s)
{
    return level_keys_dispatch<double>(d, sd, lb, nbx, nby, nbins, keys, s);
}
} // namespace rsol
