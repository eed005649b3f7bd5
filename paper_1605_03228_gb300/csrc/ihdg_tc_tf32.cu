// Tensor-core inner sweeps, TC_TF32 instantiations.
#include "ihdg_tc.cuh"

IHDG_TC_INSTANTIATE(ihdg::TC_TF32)
