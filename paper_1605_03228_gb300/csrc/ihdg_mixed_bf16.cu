// Mixed-precision CUDA-core kernels and dispatch, __nv_bfloat16 low-precision storage.
#include "ihdg_mixed_kern.cuh"

namespace ihdg {
template cudaError_t mixed_launch<__nv_bfloat16>(MixedArgs& m, int which, int has_e, int count);
}  // namespace ihdg
