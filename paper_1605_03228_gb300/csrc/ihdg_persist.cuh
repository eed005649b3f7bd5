// Device helpers shared by the persistent inner-sweep kernels (CUDA-core and tensor-core):
// low-precision conversions, loads through L2, the release/acquire primitives of the grid
// barrier, and the lagged grid reduction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ihdg_dev.h"

namespace ihdg {
namespace {

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Load through L2 (ld.global.cg): values other blocks wrote earlier in the same persistent
// launch must not come from this SM's L1, which is not coherent with their writes.
template <typename T> __device__ __forceinline__ float ldcg_f(const T* p);
template <> __device__ __forceinline__ float ldcg_f<float>(const float* p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ldcg_f<__nv_bfloat16>(const __nv_bfloat16* p) {
  const unsigned short b = __ldcg(reinterpret_cast<const unsigned short*>(p));
  return __uint_as_float((unsigned)b << 16);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Lagged grid reduction for the register and tile kernels.  After sweep s every block
// publishes its float partial in partf[(s & 1) * grid + block] and arrives at the barrier
// (thread 0: release add, bounded acquire poll).  At the top of sweep s+1 every thread loads
// its share of sweep s's partials together with its trace gathers; sum_partials then folds
// them with a fixed tree (the same in every block) and thread 0 takes the loop decision.
// Everything per thread is float32 (GB300's float64 latency would dominate a sweep).
__device__ __forceinline__ void arrive_wait(float* partf, unsigned* count, unsigned nb, float mine, Ctrl* ctrl,
                                            int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    partf[blockIdx.x] = mine;
    if ((int)blockIdx.x != ctrl->stall_block) red_release_add(count, 1u);
    const unsigned target = nb * gridDim.x;
    const long long lim = ctrl->wait_cycles;
    const long long t0 = clock64();
    while (ld_acquire_u32(count) < target) {
      if (clock64() - t0 > lim) { atomicExch(&ctrl->timeout, 1); break; }
    }
    *s_flag = *(volatile int*)&ctrl->timeout;
  }
  __syncthreads();
}

template <int NT>
__device__ __forceinline__ float sum_partials(float pv, float* wred) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pv += __shfl_down_sync(0xffffffffu, pv, o);
  if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = pv;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) t += wred[w];
  return t;   // valid in thread 0
}

}  // namespace
}  // namespace ihdg
