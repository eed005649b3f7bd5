// Mixed-precision CUDA-core kernels and dispatch, float low-precision storage.
#include "ihdg_mixed_kern.cuh"

namespace ihdg {
template cudaError_t mixed_launch<float>(MixedArgs& m, int which, int has_e, int count);
}  // namespace ihdg
