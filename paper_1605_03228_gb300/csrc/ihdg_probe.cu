// Peak-rate probes of the device: the denominators of the rooflines the sweep kernels are
// measured against where neither HBM bandwidth nor the bf16 tensor rate binds.
//   * float64 FMA rate: bounds the float64 sweep (GB300 runs float64 at a small fraction of
//     its float32 rate, so the float64 sweep is arithmetic-bound, not bandwidth-bound);
//   * float32 FMA rate: bounds the CUDA-core low-precision sweeps' arithmetic;
//   * L2 read bandwidth: the ceiling of a sweep whose state stays resident in L2.
// Each probe is one kernel timed with CUDA events after a warm-up launch.
#include <cuda_runtime.h>

#include "../../include/ihdg.h"

namespace {

constexpr int PROBE_NT = 256;
constexpr int CHAINS = 8;

// CHAINS independent FMA chains per thread (x <- x*a + b); the result is stored so that the
// chains cannot be removed.  a < 1 keeps every value bounded.
template <typename T>
__global__ void __launch_bounds__(PROBE_NT) k_probe_fma(T* out, int iters, T a, T b) {
  T x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = T(threadIdx.x) * T(1e-3) + T(c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[(size_t)blockIdx.x * PROBE_NT + threadIdx.x] = s;
}

// Every thread reads float4 values of an L2-resident buffer with ld.global.cg (L1 bypassed)
// `reps` times in a grid-stride loop and stores one sum.
__global__ void __launch_bounds__(PROBE_NT) k_probe_l2(const float4* __restrict__ buf, long long n4, int reps,
                                                        float* out) {
  float s = 0.f;
  const long long stride = (long long)gridDim.x * PROBE_NT;
  for (int r = 0; r < reps; ++r)
    for (long long i = (long long)blockIdx.x * PROBE_NT + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      s += v.x + v.y + v.z + v.w;
    }
  out[(size_t)blockIdx.x * PROBE_NT + threadIdx.x] = s;
}

struct ProbeMem {
  void* p[2] = {nullptr, nullptr};
  cudaEvent_t e[2] = {nullptr, nullptr};
  ~ProbeMem() {
    for (void* q : p)
      if (q) cudaFree(q);
    for (cudaEvent_t x : e)
      if (x) cudaEventDestroy(x);
  }
};

// Best of `tries` timed launches of `launch` (after one warm-up), in milliseconds.
template <typename F>
cudaError_t best_ms(F launch, cudaEvent_t a, cudaEvent_t b, int tries, float* ms) {
  launch();
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  float best = 1e30f;
  for (int t = 0; t < tries; ++t) {
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    if (e != cudaSuccess) return e;
    float x = 0.f;
    cudaEventElapsedTime(&x, a, b);
    if (x < best) best = x;
  }
  *ms = best;
  return cudaGetLastError();
}

}  // namespace

extern "C" ihdg_status ihdg_measure_peaks(int device, ihdg_peaks* out) {
  if (!out) return IHDG_ERR_INVALID;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return IHDG_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return IHDG_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return IHDG_ERR_CUDA;
  ProbeMem m;
  const int blocks = sms * 8;   // 8 blocks of 256 threads per SM: 64 warps, full occupancy
  const size_t nthreads = (size_t)blocks * PROBE_NT;
  const size_t l2_bytes = 48ull << 20;   // resident in GB300's L2 (126 MB)
  if (cudaMalloc(&m.p[0], nthreads * sizeof(double)) != cudaSuccess) return IHDG_ERR_NOMEM;
  if (cudaMalloc(&m.p[1], l2_bytes) != cudaSuccess) return IHDG_ERR_NOMEM;
  if (cudaEventCreate(&m.e[0]) != cudaSuccess || cudaEventCreate(&m.e[1]) != cudaSuccess) return IHDG_ERR_CUDA;
  if (cudaMemset(m.p[1], 0, l2_bytes) != cudaSuccess) return IHDG_ERR_CUDA;
  float ms = 0.f;
  // float64: 2 flops per FMA
  const int it64 = 4096;
  cudaError_t e = best_ms([&] { k_probe_fma<double><<<blocks, PROBE_NT>>>((double*)m.p[0], it64, 0.999999, 1e-7); },
                          m.e[0], m.e[1], 5, &ms);
  if (e != cudaSuccess) return IHDG_ERR_CUDA;
  out->fp64_fma_tflops = 2.0 * CHAINS * (double)it64 * nthreads / (ms * 1e-3) / 1e12;
  const int it32 = 65536;
  e = best_ms([&] { k_probe_fma<float><<<blocks, PROBE_NT>>>((float*)m.p[0], it32, 0.999999f, 1e-7f); }, m.e[0],
              m.e[1], 5, &ms);
  if (e != cudaSuccess) return IHDG_ERR_CUDA;
  out->fp32_fma_tflops = 2.0 * CHAINS * (double)it32 * nthreads / (ms * 1e-3) / 1e12;
  const long long n4 = (long long)(l2_bytes / sizeof(float4));
  const int reps = 20;
  e = best_ms([&] { k_probe_l2<<<blocks, PROBE_NT>>>((const float4*)m.p[1], n4, reps, (float*)m.p[0]); }, m.e[0],
              m.e[1], 5, &ms);
  if (e != cudaSuccess) return IHDG_ERR_CUDA;
  out->l2_read_gbs = (double)l2_bytes * reps / (ms * 1e-3) / 1e9;
  out->sms = sms;
  return IHDG_OK;
}
