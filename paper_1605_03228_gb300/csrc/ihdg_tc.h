// Tensor-core inner sweeps (tcgen05): operand modes and the launcher, defined in ihdg_tc.cuh
// and instantiated per mode in ihdg_tc_bf16.cu, ihdg_tc_tf32.cu and ihdg_tc_tf32x4.cu.
#pragma once

#include <cuda_runtime.h>

#include "ihdg_mixed.h"

namespace ihdg {

// Operand modes.  TC_BF16: bf16 storage and operands (kind::f16).  TC_TF32: float32 storage,
// operands read as tf32 (kind::tf32, one pass).  TC_TF32X4: float32 storage, each operand
// split x = hi + lo with hi = x rounded to the nearest tf32 value and lo = x - hi (exact in
// float32, |lo| <= 2^-11 |x|) also rounded to tf32, so hi + lo is within 2^-23 of x;
// D = A_lo B_lo + A_lo B_hi + A_hi B_lo + A_hi B_hi in four MMA passes, accumulated in
// float32.  The products then carry about float32's accuracy at tensor-core speed.
enum TcMode { TC_BF16 = 0, TC_TF32 = 1, TC_TF32X4 = 2 };

// One persistent cooperative launch of the tensor-core inner loop on (rl, e0, e1), whose
// element type is bf16 for TC_BF16 and float otherwise.  Returns cudaErrorNotSupported, with
// nothing launched, when the shape does not fit the kernel (n_in > 64, n_exp > 32) or its
// grid would not be co-resident.
template <int NF, int NLF, bool PER_AXIS, int MODE>
cudaError_t launch_tc(MixedArgs& m, void* rl, void* e0, void* e1);

}  // namespace ihdg
