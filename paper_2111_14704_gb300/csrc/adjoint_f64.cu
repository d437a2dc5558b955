// Reverse-mode step (FP64), compiled with -fmad=false like the FP64 forward
// step so that the recomputed forward quantities round as written.
#include "adjoint_binned.cuh"

namespace rsol {

cudaError_t adjoint_step_f64(const AdjDesc &d, cudaStream_t s) { return adjoint_dispatch<double>(d, s); }

} // namespace rsol
