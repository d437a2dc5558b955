// FP64 instantiation of the sub-cycled push (-fmad=false, as push_f64.cu).
#include "subcycle.cuh"

namespace rsol {
cudaError_t push_subcycled_f64(const PushDesc &d, const SubDesc &sd, cudaStream_t s)
{
    return subcycle_dispatch<double>(d, sd, s);
}
} // namespace rsol
