// FP32 instantiation of the sub-cycled push (same flags as push_f32.cu).
#include "subcycle.cuh"

namespace rsol {
cudaError_t push_subcycled_f32(const PushDesc &d, const SubDesc &sd, cudaStream_t s)
{
    return subcycle_dispatch<float>(d, sd, s);
}
cudaError_t level_keys_f32(const PushDesc &d, const SubDesc &sd, int lb, int nbx, int nby,
                          uint32_t nbins, uint32_t *keys, cudaStream_t s)
{
    return level_keys_dispatch<float>(d, sd, lb, nbx, nby, nbins, keys, s);
}
} // namespace rsol
