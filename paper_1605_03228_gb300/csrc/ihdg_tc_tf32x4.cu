// Tensor-core inner sweeps, TC_TF32X4 instantiations.
#include "ihdg_tc.cuh"

IHDG_TC_INSTANTIATE(ihdg::TC_TF32X4)
