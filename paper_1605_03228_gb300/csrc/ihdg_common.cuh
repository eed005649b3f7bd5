// Device helpers shared by the sweep kernels (internal header, included by .cu files).
//
// Element coordinates and neighbours on the box mesh, the trace gather (step a1 of the
// sweep), fixed-order block and grid reductions, and the float64 loop decision.
#pragma once
#include <cuda_runtime.h>

#include "ihdg_dev.h"

namespace ihdg {
namespace {

// Allow kernel `kern` the device's largest dynamic shared memory (the opt-in maximum less its
// static shared memory).  Launches still request their own size; the attribute is only the
// ceiling.  Setting it to a fixed value, rather than to each launch's size, keeps launches
// from concurrent host threads (serving slots) from lowering it under one another.
template <typename K>
inline cudaError_t allow_dynamic_smem(K kern) {
  int dev = 0, mx = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)kern);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
  return e;
}

constexpr int BS = 128;   // threads per block of the element kernels
constexpr int PBS = 256;  // threads per block of the persistent kernels

__device__ __forceinline__ void coords(const DevGeo& g, long long K, int* c) {
  if (g.nel <= 0xffffffffLL && K <= 0xffffffffLL) {
    // every mesh of up to 2^32 elements: 32-bit unsigned division (a 64-bit division is a
    // long instruction sequence, and the sweeps take coordinates per element)
    const unsigned k = (unsigned)K, n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
    const unsigned t = k / n0, t2 = t / n1;
    c[0] = (int)(k - t * n0);
    c[1] = (int)(t - t2 * n1);
    c[2] = (int)t2;
    return;
  }
  c[0] = (int)(K % g.n[0]);
  long long t = K / g.n[0];
  c[1] = (int)(t % g.n[1]);
  c[2] = (int)(t / g.n[1]);
}
__device__ __forceinline__ bool on_bnd(const DevGeo& g, const int* c, int f) {
  const int a = f >> 1;
  return (f & 1) ? (c[a] == g.n[a] - 1) : (c[a] == 0);
}
__device__ __forceinline__ long long nbr_of(const DevGeo& g, long long K, int f) {
  const int a = f >> 1;
  return (f & 1) ? K + g.stride[a] : K - g.stride[a];
}
// boundary-face number of local face f of the element at coordinates c (global face order)
__device__ __forceinline__ long long bface_of(const DevGeo& g, const int* c, int f) {
  const int a = f >> 1, s = f & 1;
  if (a == 0) return 2LL * (c[1] + (long long)g.n[1] * c[2]) + s;
  if (a == 1) return g.nbf_off[1] + (long long)c[2] * 2 * g.n[0] + (long long)s * g.n[0] + c[0];
  return g.nbf_off[2] + (long long)s * g.n[0] * g.n[1] + (long long)c[1] * g.n[0] + c[0];
}

// a1: the trace values t (n_in = nlf * NF) element K needs, from export array E.  Every load
// is unconditional: a face that needs no own (or no neighbour) value reads an in-bounds
// stand-in, and selects combine them (the same arithmetic as reading only what is needed),
// so all of an element's loads are in flight at once.
template <int NF, int NLF, typename TE, typename TA, typename Out>
__device__ __forceinline__ void gather(const DevGeo& g, const TE* __restrict__ E, long long K,
                                       const int* c, Out&& put) {
#pragma unroll
  for (int f = 0; f < NLF; ++f) {
    const int kind = g.kind[f];
    const bool bnd = on_bnd(g, c, f);
    const bool need_own = kind == FK_OWN_D || kind == FK_SUM_D;
    const bool need_nb = (kind == FK_NBR_D || kind == FK_SUM_D) && !bnd;
    const TE* own = E + (long long)(need_own ? g.own_off[f] : 0) * g.ld + K;
    const TE* nb = need_nb ? E + (long long)g.nbr_off[f] * g.ld + nbr_of(g, K, f) : own;
    TA o[NF], n[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) {
      o[j] = (TA)own[(long long)j * g.ld];
      n[j] = (TA)nb[(long long)j * g.ld];
    }
#pragma unroll
    for (int j = 0; j < NF; ++j) {
      TA v = TA(0);
      if (kind == FK_OWN_D) v = o[j];
      else if (kind == FK_NBR_D) v = need_nb ? n[j] : TA(0);
      else if (kind == FK_SUM_D) v = need_nb ? o[j] + n[j] : (g.bc_mirror ? o[j] + o[j] : TA(0));
      put(f * NF + j, v);
    }
  }
}

// Export slot e carries a value (transport: the axis has an outflow face).
__device__ __forceinline__ bool row_live(const DevGeo& g, int e, int /*nf*/) { return (g.live >> e) & 1ull; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum; the result is valid in thread 0.  Reuses `ws` (BS/32 doubles).
__device__ __forceinline__ double block_sum(double v, double* ws) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += ws[i];
  return t;
}

// Publish this block's partial sum; returns true in every thread of the last block to
// arrive, which then holds the fixed-order total of all partials in thread 0.
__device__ bool arrive(Ctrl* ctrl, double* partials, double v, double* ws, double* total) {
  __shared__ int s_last;
  double s = block_sum(v, ws);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    const unsigned t = atomicAdd(&ctrl->ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double acc = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) acc += __ldcg(partials + i);
  *total = block_sum(acc, ws);
  if (threadIdx.x == 0) ctrl->ticket = 0u;
  return true;
}

// Loop decision of a float64 stopping residual (thread 0 of the last block).
__device__ void decide(Ctrl* ctrl, double res2, double* res_hist, bool count_fp64) {
  const double res = sqrt(res2);
  const int k = ctrl->iter + 1;
  ctrl->iter = k;
  if (count_fp64) ctrl->fp64_sweeps += 1; else ctrl->lowp_sweeps += 1;
  ctrl->res = res;
  if (res_hist) res_hist[k] = res;
  if (res < ctrl->tol) { ctrl->done = 1; ctrl->status = 0; return; }
  if (!(res == res) || isinf(res) ||
      (ctrl->diverge_factor > 0.0 && res > ctrl->diverge_factor * ctrl->res_min)) {
    ctrl->done = 1; ctrl->status = 5; return;
  }
  if (res < ctrl->res_min) ctrl->res_min = res;
  if (k >= ctrl->max_iters) { ctrl->done = 1; ctrl->status = 4; }
}

// the loop has stopped: finished, or a bounded wait ran out (later launches return at once)
__device__ __forceinline__ int ctrl_done(const Ctrl* c) {
  return *(volatile const int*)&c->done | *(volatile const int*)&c->timeout;
}
__device__ __forceinline__ int ctrl_iter(const Ctrl* c) { return *(volatile const int*)&c->iter; }

}  // namespace
}  // namespace ihdg
