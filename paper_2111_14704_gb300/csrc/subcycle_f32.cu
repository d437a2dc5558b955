// FP32 instantiation of the sub-cycled push (same flags as push_f32.cu).
#include "subcycle.cuh"

namespace rsol {
cudaError_t push_subcycled_f32(const PushDesc &d, const SubDesc &sd, cudaStream_t s)
{
    return subcycle_dispatch<float>(d, sd, s);
}
} // namespace rsol
