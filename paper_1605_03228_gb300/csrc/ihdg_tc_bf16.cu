// Tensor-core inner sweeps, TC_BF16 instantiations.
#include "ihdg_tc.cuh"

IHDG_TC_INSTANTIATE(ihdg::TC_BF16)
