// Tensor-core inner-sweep kernel (tcgen05) and its launcher, included by one translation unit
// per operand mode (ihdg_tc_bf16.cu, ihdg_tc_tf32.cu, ihdg_tc_tf32x4.cu) so that they compile
// in parallel.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>

#include "ihdg_common.cuh"
#include "ihdg_dev.h"
#include "ihdg_kernels.h"
#include "ihdg_mixed.h"
#include "ihdg_persist.cuh"
#include "ihdg_tc.h"

namespace ihdg {
namespace {

// ---------------------------------------------------------------------------------------
// Tensor-core local apply (tcgen05): persistent inner loop with bf16 or tf32 operands and a
// float32 accumulator in tensor memory.  Per tile of 128 elements the GEMM
//     D[128 x NP] = A[128 x KP] . B[NP x KP]^T,   A = gathered traces t, B = L_E (rows = exports)
// runs as KP/KSTEP tcgen05.mma (kind::f16, K16, or kind::tf32, K8; M128, N NP) issued by one
// thread; operands sit in shared memory in the K-major, no-swizzle core-matrix layout (8 rows
// x 16 bytes per core matrix; cores adjacent along K are 128 B apart, 8-row groups are
// KP/(16/element size) x 128 B apart).  The
// accumulator of each of the block's G tiles occupies 32 columns of tensor memory allocated
// for the whole launch; each warp reads its 32 lanes back (tcgen05.ld 32x32b) for the epilogue
// e_{j+1} = r + D.  Every wait (mbarrier, grid barrier) is bounded; on expiry the kernel sets
// ctrl->timeout, waits (bounded) for its MMAs, frees its tensor memory and returns.
namespace tc {
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);   // version 1, no swizzle
}
// kind::f16 instruction descriptor: D f32, A and B bf16, both K-major, N and M encoded
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
// kind::tf32 instruction descriptor: D f32, A and B tf32 (format 2), both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {   // bounded (~1 s)
  const long long t0 = clock64();
  while (!mbar_try(mbar, parity))
    if (clock64() - t0 > 2000000000LL) return false;
  return true;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void ld32(uint32_t taddr, float* d) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) d[i] = __uint_as_float(r[i]);
}
// round to the nearest tf32 value (ties away from zero), returned as a float32 bit pattern
__device__ __forceinline__ float rna_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void group_bar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
// OR of v over the 128 threads of named barrier `id` (also a barrier)
__device__ __forceinline__ int group_or(int id, int v) {
  int r;
  asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, %2, 128, p;\n\t"
               "selp.s32 %0, 1, 0, q;\n\t}\n" : "=r"(r) : "r"(v), "r"(id) : "memory");
  return r;
}
}  // namespace tc

// Tile shapes and shared memory of k_inner_tc: B (and B_lo), then per group its A (and A_lo),
// all in the K-major no-swizzle core-matrix layout.
template <int NF, int NLF, bool PER_AXIS, int MODE>
struct TcShape {
  static constexpr int NIN = NF * NLF;
  static constexpr int NEXP = PER_AXIS ? NF * (NLF / 2) : NF * NLF;
  static constexpr int ESZ = MODE == TC_BF16 ? 2 : 4;      // bytes per operand element
  static constexpr int EPC = 16 / ESZ;                      // elements per 16-byte core row
  static constexpr int KSTEP = 32 / ESZ;                    // K of one MMA (two core matrices)
  static constexpr int KP = (NIN + KSTEP - 1) / KSTEP * KSTEP;
  static constexpr int NP = (NEXP + 15) / 16 * 16;          // N padded to a multiple of 16
  static constexpr int ROWB = KP / EPC * 128;               // bytes per 8-row group
  static constexpr int NSPLIT = MODE == TC_TF32X4 ? 2 : 1;  // hi (and lo) buffers
  static constexpr int BBYTES = NP / 8 * ROWB;
  static constexpr int ABYTES = 128 / 8 * ROWB;
  static constexpr int FIT = (227 * 1024 - 2048 - NSPLIT * BBYTES) / (NSPLIT * ABYTES);
  static constexpr int G = FIT >= 4 ? 4 : (FIT < 1 ? 1 : FIT);   // tiles in flight per block
  static constexpr int SMEM = NSPLIT * BBYTES + G * NSPLIT * ABYTES;
  static constexpr uint32_t TCOLS = G * 32 <= 32 ? 32 : G * 32 <= 64 ? 64 : G * 32 <= 128 ? 128 : 256;
  static constexpr bool OK = NP <= 32 && KP <= 64 && FIT >= 1;
};

// Group gr of the block handles tiles blockIdx.x * G + gr, + gridDim.x * G, ...; the
// assignment is the same in every sweep, so each thread always owns the same elements.  A
// group loads the residual its epilogue needs together with its tile's traces, packs the
// traces into its A buffer(s), and one thread issues the MMAs into the group's 32
// tensor-memory columns.  Groups synchronise among themselves with named barriers only, so
// the block's tiles overlap their latencies.
template <int NF, int NLF, bool PER_AXIS, int MODE>
__global__ void __launch_bounds__(128 * TcShape<NF, NLF, PER_AXIS, MODE>::G, 1)
    k_inner_tc(const DevGeo g, const typename std::conditional<MODE == TC_BF16, __nv_bfloat16, float>::type* __restrict__ rlp,
               typename std::conditional<MODE == TC_BF16, __nv_bfloat16, float>::type* e0,
               typename std::conditional<MODE == TC_BF16, __nv_bfloat16, float>::type* e1, Ctrl* ctrl,
               double* partials, const unsigned char* __restrict__ Bg) {
  using TL = typename std::conditional<MODE == TC_BF16, __nv_bfloat16, float>::type;
  using RAW = typename std::conditional<MODE == TC_BF16, unsigned short, unsigned>::type;
  using S = TcShape<NF, NLF, PER_AXIS, MODE>;
  constexpr int G = S::G, NT = 128 * G, NIN = S::NIN, NEXP = S::NEXP, KP = S::KP, NP = S::NP, ROWB = S::ROWB;
  constexpr int EPC = S::EPC, KSTEP = S::KSTEP, NSPLIT = S::NSPLIT;
  static_assert(S::OK, "tile shape");
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long s_mbar[G];
  __shared__ uint32_t s_tmem;
  __shared__ float wsum[NT / 32];
  __shared__ int s_to, s_stop;
  if (ctrl_done(ctrl) || *(volatile const int*)&ctrl->inner_done) return;
  const int jj0 = *(volatile const int*)&ctrl->inner_iter;
  const int iter0 = *(volatile const int*)&ctrl->iter;
  const int lowp0 = *(volatile const int*)&ctrl->lowp_sweeps;
  const int max_iters = ctrl->max_iters, inner_max = ctrl->inner_max;
  const float limf = (float)(ctrl->inner_rtol * ctrl->rnorm);
  const int tid = threadIdx.x, gr = tid >> 7, gt = tid & 127, wq = (tid >> 5) & 3;
  unsigned char* sB = tc_smem;                                               // B_hi [, B_lo]
  unsigned char* sA = tc_smem + NSPLIT * S::BBYTES + gr * NSPLIT * S::ABYTES;  // A_hi [, A_lo]
  // set-up: tensor memory, one mbarrier per group, operator B
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&s_tmem)),
                 "r"(S::TCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid < G) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&s_mbar[tid])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    const uint4* src = reinterpret_cast<const uint4*>(Bg);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    for (int i = tid; i < NSPLIT * S::BBYTES / 16; i += NT) dst[i] = src[i];
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem0 = s_tmem;
  const uint32_t tcol = tmem0 + (uint32_t)(gr * 32);                 // this group's accumulator
  const uint32_t tld = tcol + ((uint32_t)(wq * 32) << 16);            // this warp's 32 lanes of it
  const uint32_t mbar = tc::smem_u32(&s_mbar[gr]);
  const uint32_t aaddr = tc::smem_u32(sA), baddr = tc::smem_u32(sB);
  constexpr uint32_t IDESC = MODE == TC_BF16 ? tc::idesc_bf16(128, NP) : tc::idesc_tf32(128, NP);
  const int bar_id = 1 + gr;
  uint32_t phase = 0;
  const int ld = (int)g.ld, nel = (int)g.nel;
  const int ntiles = (nel + 127) / 128;
  const int tile0 = blockIdx.x * G + gr, tstride = gridDim.x * G;
  unsigned* count = &ctrl->bar_count;
  float* partf = reinterpret_cast<float*>(partials);
  int failed = 0;
  auto widen = [](RAW r) -> float {
    if constexpr (MODE == TC_BF16) return __uint_as_float((unsigned)r << 16);
    else return __uint_as_float(r);
  };
  // a1: gather element (tile*128 + gt)'s traces into row gt of this group's A.  Every load is
  // unconditional (rows past the mesh and faces on the boundary read a safe address and are
  // masked afterwards), so all of them are in flight at once.  own[] keeps the element's
  // current exports for the epilogue's step norm.
  float own[NEXP];
  auto gather_pack = [&](int tile, const TL* __restrict__ ec) {
    const int K = tile * 128 + gt;
    const bool valid = K < nel;
    const int Kc = valid ? K : 0;
    int c[3] = {0, 0, 0};
    if (valid) coords(g, K, c);
    const RAW* eb = reinterpret_cast<const RAW*>(ec);
    int o1[NLF], o2[NLF];
    bool u1[NLF], u2[NLF], z[NLF];
#pragma unroll
    for (int f = 0; f < NLF; ++f) {
      const int kind = g.kind[f], a = f >> 1;
      const bool bnd = valid && on_bnd(g, c, f);
      const int os = PER_AXIS ? a * NF : f * NF;
      const int ns = PER_AXIS ? a * NF : (f ^ 1) * NF;
      const int Kn = Kc + ((f & 1) ? (int)g.stride[a] : -(int)g.stride[a]);
      const bool nbr = valid && !bnd && (kind == FK_NBR_D || kind == FK_SUM_D);
      if (PER_AXIS) {   // one source per face: own (outflow) or the neighbour's (inflow)
        u1[f] = valid && (kind == FK_OWN_D || (kind == FK_NBR_D && !bnd));
        o1[f] = (kind == FK_NBR_D && nbr) ? ns * ld + Kn : os * ld + Kc;
        u2[f] = false;
        o2[f] = 0;
        z[f] = kind != FK_OWN_D;    // not an own row
      } else {          // own + neighbour; on the boundary mirror (2 own) or zero
        u1[f] = valid && (kind == FK_OWN_D || (kind == FK_SUM_D && (!bnd || g.bc_mirror)));
        o1[f] = os * ld + Kc;
        u2[f] = nbr || (valid && kind == FK_SUM_D && bnd && g.bc_mirror);
        o2[f] = nbr ? ns * ld + Kn : os * ld + Kc;
        z[f] = !(kind == FK_OWN_D || kind == FK_SUM_D);
      }
    }
    RAW r1[NIN], r2[PER_AXIS ? 1 : NIN];
#pragma unroll
    for (int f = 0; f < NLF; ++f)
#pragma unroll
      for (int q = 0; q < NF; ++q) r1[f * NF + q] = __ldcg(eb + o1[f] + q * ld);
    if constexpr (!PER_AXIS) {
#pragma unroll
      for (int f = 0; f < NLF; ++f)
#pragma unroll
        for (int q = 0; q < NF; ++q) r2[f * NF + q] = __ldcg(eb + o2[f] + q * ld);
    }
    float t[KP];
#pragma unroll
    for (int k = NIN; k < KP; ++k) t[k] = 0.f;
#pragma unroll
    for (int f = 0; f < NLF; ++f) {
      const int os = PER_AXIS ? (f >> 1) * NF : f * NF;
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        const float xo = widen(r1[f * NF + q]);
        float v = u1[f] ? xo : 0.f;
        if constexpr (!PER_AXIS) v += u2[f] ? widen(r2[f * NF + q]) : 0.f;
        t[f * NF + q] = v;
        // the own export row: read in full (also on the boundary) for the step norm
        if (PER_AXIS) { if (!z[f]) own[os + q] = valid ? xo : 0.f; }
        else own[os + q] = (valid && !z[f]) ? xo : 0.f;
      }
    }
    unsigned char* row = sA + (gt >> 3) * ROWB + (gt & 7) * 16;
#pragma unroll
    for (int kc = 0; kc < KP / EPC; ++kc) {
      if constexpr (MODE == TC_BF16) {
        __align__(16) __nv_bfloat16 h[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) h[u] = __float2bfloat16_rn(t[kc * 8 + u]);
        *reinterpret_cast<uint4*>(row + kc * 128) = *reinterpret_cast<uint4*>(h);
      } else if constexpr (MODE == TC_TF32) {
        *reinterpret_cast<float4*>(row + kc * 128) = make_float4(t[kc * 4], t[kc * 4 + 1], t[kc * 4 + 2], t[kc * 4 + 3]);
      } else {
        float hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          hi[u] = tc::rna_tf32(t[kc * 4 + u]);
          lo[u] = tc::rna_tf32(t[kc * 4 + u] - hi[u]);   // the difference is exact in float32
        }
        *reinterpret_cast<float4*>(row + kc * 128) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4*>(row + S::ABYTES + kc * 128) = make_float4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
  };
  for (int s = 0;; ++s) {
    const TL* __restrict__ ec = ((jj0 + s) & 1) ? e1 : e0;
    TL* __restrict__ en = ((jj0 + s) & 1) ? e0 : e1;
    // previous sweep's partials, in flight together with the first tile's gathers
    float pv = 0.f;
    if (s > 0)
      for (int i = tid; i < (int)gridDim.x; i += NT) pv += __ldcg(partf + ((s - 1) & 1) * gridDim.x + i);
    if (tile0 < ntiles) gather_pack(tile0, ec);
    // lagged loop decision (as in k_inner_reg)
    {
      const float tot = sum_partials<NT>(pv, wsum);
      if (tid == 0) {
        const float step = sqrtf(tot);
        const bool budget = jj0 + s >= inner_max || iter0 + s >= max_iters;
        const bool stop = budget || (s > 0 && (step <= limf || !(step == step) || isinf(step)));
        s_stop = stop ? 1 : 0;
        if (blockIdx.x == 0) {
          ctrl->inner_iter = jj0 + s;
          ctrl->iter = iter0 + s;
          ctrl->lowp_sweeps = lowp0 + s;
          if (s > 0) ctrl->inner_step = (double)step;
          if (stop) ctrl->inner_done = 1;
        }
      }
      __syncthreads();
      if (s_stop) break;
    }
    float acc = 0.f;
    for (int tile = tile0; tile < ntiles; tile += tstride) {
      // the epilogue's residual loads, issued with this tile's gathers (one round trip)
      const int K = tile * 128 + gt;
      const bool valid = K < nel;
      RAW rr[NEXP];
      const RAW* rb = reinterpret_cast<const RAW*>(rlp);
#pragma unroll
      for (int e = 0; e < NEXP; ++e) rr[e] = rb[e * ld + (valid ? K : 0)];
      if (tile != tile0) gather_pack(tile, ec);
      tc::fence_proxy_async();
      tc::fence_before();
      tc::group_bar(bar_id);
      tc::fence_after();
      // a3: D = A . B^T on the tensor cores (four passes for the split operands)
      if (gt == 0) {
#pragma unroll
        for (int kk = 0; kk < KP / KSTEP; ++kk) {
          const uint64_t ah = tc::sdesc(aaddr + kk * 256, 128, ROWB), bh = tc::sdesc(baddr + kk * 256, 128, ROWB);
          if constexpr (MODE == TC_BF16) {
            tc::mma_bf16(tcol, ah, bh, IDESC, kk > 0 ? 1u : 0u);
          } else if constexpr (MODE == TC_TF32) {
            tc::mma_tf32(tcol, ah, bh, IDESC, kk > 0 ? 1u : 0u);
          } else {
            const uint64_t al = tc::sdesc(aaddr + S::ABYTES + kk * 256, 128, ROWB);
            const uint64_t bl = tc::sdesc(baddr + S::BBYTES + kk * 256, 128, ROWB);
            tc::mma_tf32(tcol, al, bl, IDESC, kk > 0 ? 1u : 0u);   // smallest terms first
            tc::mma_tf32(tcol, al, bh, IDESC, 1u);
            tc::mma_tf32(tcol, ah, bl, IDESC, 1u);
            tc::mma_tf32(tcol, ah, bh, IDESC, 1u);
          }
        }
        tc::commit(mbar);
      }
      __syncwarp();
      // the group agrees on the outcome of the (bounded) wait, so all its threads take one path
      const int ok = tc::mbar_wait(mbar, phase) ? 1 : 0;
      const int bad = tc::group_or(bar_id, !ok);
      phase ^= 1u;
      if (bad) { failed = 1; break; }
      tc::fence_after();
      // a4: e_{j+1} = r + D from this warp's 32 accumulator lanes
      float d[32];
      tc::ld32(tld, d);
      if (valid) {
#pragma unroll
        for (int e = 0; e < NEXP; ++e) {
          if ((g.live >> e) & 1ull) {
            const TL nv = from_f<TL>(widen(rr[e]) + d[e]);
            const float dl = to_f(nv) - own[e];
            acc = fmaf(dl, dl, acc);
            en[e * ld + K] = nv;
          }
        }
      }
    }
    if (__syncthreads_or(failed)) {
      if (tid == 0) atomicExch(&ctrl->timeout, 1);
      break;
    }
    const float blk = sum_partials<NT>(acc, wsum);
    arrive_wait(partf + (s & 1) * gridDim.x, count, (unsigned)(s + 1), blk, ctrl, &s_to);
    if (s_to) break;
  }
  // release tensor memory on every path (a group whose MMA wait expired waits once more)
  if (failed) tc::mbar_wait(mbar, phase ^ 1u);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem0), "r"(S::TCOLS) : "memory");
}

// ---------------------------------------------------------------------------------------
// Staged variant for the per-axis export layout (transport) with bf16 storage: the traces of
// a tile of 128 consecutive elements are runs of consecutive element numbers in each export
// slot -- the element's own exports at K on outflow faces, the upstream neighbour's at
// K -+ (element-number step of the axis) on inflow faces -- so one thread of the group copies
// them global -> shared memory with tiled TMA tensor copies (cp.async.bulk.tensor.2d over the
// correction array seen as a [slots x ld] bf16 tensor, completion counted in bytes on a
// per-stage mbarrier): one box of all slots' own runs (128 values each), and per inflow axis
// one box of its slots' windows of 136 values from the 8-aligned number at or below the run's
// start (a tensor copy's inner coordinate must be a multiple of 8 bf16 values; the run begins
// delta = start mod 8 values into the window; coordinates outside the tensor read zeros).
// Two stages per group: while a tile is packed, multiplied and written back, the next tile's
// copies are in flight, and no register holds a gathered value before it is packed.  The rest
// (A in the core-matrix layout, MMA, epilogue, lagged decision, bounded waits) is
// k_inner_tc's.
template <int NF, int NLF>
struct TcsShape {
  using S = TcShape<NF, NLF, true, TC_BF16>;
  static constexpr int D = NLF / 2;
  static constexpr int NEXP = S::NEXP;                // D * NF slots
  static constexpr int NBW = 136;                     // values per inflow window
  static constexpr int OWNB = NEXP * 256;             // own runs: 128 bf16 per slot
  static constexpr int WB = (NF * NBW * 2 + 127) / 128 * 128;   // one axis's inflow windows
  static constexpr int STAGE = OWNB + D * WB;         // a multiple of 128 (tensor-copy alignment)
  static constexpr int GROUPB = S::ABYTES + 2 * STAGE;
  static constexpr int FIT = (227 * 1024 - 4096 - S::BBYTES) / GROUPB;
  static constexpr int G = FIT >= 4 ? 4 : (FIT < 1 ? 1 : FIT);
  static constexpr int SMEM = S::BBYTES + G * GROUPB;
  static constexpr uint32_t TCOLS = G * 32 <= 32 ? 32 : G * 32 <= 64 ? 64 : G * 32 <= 128 ? 128 : 256;
  static constexpr bool OK = S::OK && FIT >= 1 && NLF % 2 == 0;
};

namespace tc {
__device__ __forceinline__ void expect_bytes(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
// tiled tensor copy of a 2D box (x: element number, y: slot) global -> shared memory;
// coordinates outside the tensor read zeros
__device__ __forceinline__ void tensor_g2s(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
  asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
               ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar) : "memory");
}
// values other SMs stored with ordinary stores (made visible by the grid barrier) become
// visible to this thread's bulk copies
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
}  // namespace tc

template <int NF, int NLF>
__global__ void __launch_bounds__(128 * TcsShape<NF, NLF>::G, 1)
    k_inner_tcs(const DevGeo g, const __nv_bfloat16* __restrict__ rlp, __nv_bfloat16* e0, __nv_bfloat16* e1,
                Ctrl* ctrl, double* partials, const unsigned char* __restrict__ Bg,
                const __grid_constant__ CUtensorMap own0, const __grid_constant__ CUtensorMap own1,
                const __grid_constant__ CUtensorMap win0m, const __grid_constant__ CUtensorMap win1m) {
  using TL = __nv_bfloat16;
  using RAW = unsigned short;
  using S = TcShape<NF, NLF, true, TC_BF16>;
  using Z = TcsShape<NF, NLF>;
  constexpr int G = Z::G, NT = 128 * G, NIN = S::NIN, NEXP = S::NEXP, KP = S::KP, NP = S::NP, ROWB = S::ROWB;
  constexpr int D = Z::D, KSTEP = S::KSTEP;
  static_assert(Z::OK, "tile shape");
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long s_mbar[G];        // MMA completion, per group
  __shared__ __align__(8) unsigned long long s_stage[2 * G];   // copy completion, per group and stage
  __shared__ uint32_t s_tmem;
  __shared__ float wsum[NT / 32];
  __shared__ int s_to, s_stop;
  if (ctrl_done(ctrl) || *(volatile const int*)&ctrl->inner_done) return;
  const int jj0 = *(volatile const int*)&ctrl->inner_iter;
  const int iter0 = *(volatile const int*)&ctrl->iter;
  const int lowp0 = *(volatile const int*)&ctrl->lowp_sweeps;
  const int max_iters = ctrl->max_iters, inner_max = ctrl->inner_max;
  const float limf = (float)(ctrl->inner_rtol * ctrl->rnorm);
  const int tid = threadIdx.x, gr = tid >> 7, gt = tid & 127, wq = (tid >> 5) & 3;
  unsigned char* sB = tc_smem;
  unsigned char* sA = tc_smem + S::BBYTES + gr * Z::GROUPB;
  unsigned char* sStage = sA + S::ABYTES;                       // two stages of Z::STAGE bytes
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&s_tmem)),
                 "r"(Z::TCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid < 3 * G) {
    const uint32_t mb = tid < G ? tc::smem_u32(&s_mbar[tid]) : tc::smem_u32(&s_stage[tid - G]);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    const uint4* src = reinterpret_cast<const uint4*>(Bg);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    for (int i = tid; i < S::BBYTES / 16; i += NT) dst[i] = src[i];
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem0 = s_tmem;
  const uint32_t tcol = tmem0 + (uint32_t)(gr * 32);
  const uint32_t tld = tcol + ((uint32_t)(wq * 32) << 16);
  const uint32_t mbar = tc::smem_u32(&s_mbar[gr]);
  const uint32_t smb[2] = {tc::smem_u32(&s_stage[2 * gr]), tc::smem_u32(&s_stage[2 * gr + 1])};
  const uint32_t aaddr = tc::smem_u32(sA), baddr = tc::smem_u32(sB);
  const uint32_t stage_addr = tc::smem_u32(sStage);
  constexpr uint32_t IDESC = tc::idesc_bf16(128, NP);
  const int bar_id = 1 + gr;
  uint32_t phase = 0, sphase[2] = {0u, 0u};
  int pending[2] = {0, 0};
  const int ld = (int)g.ld, nel = (int)g.nel;
  const int ntiles = (nel + 127) / 128;
  const int tile0 = blockIdx.x * G + gr, tstride = gridDim.x * G;
  unsigned* count = &ctrl->bar_count;
  float* partf = reinterpret_cast<float*>(partials);
  int failed = 0;
  // per axis: which face takes the element's own exports (outflow) and where the upstream
  // neighbour of an inflow face sits (-1: below, +1: above, 0: no inflow face)
  bool own_ax[D];
  int up[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int k0 = g.kind[2 * a], k1 = g.kind[2 * a + 1];
    own_ax[a] = k0 == FK_OWN_D || k1 == FK_OWN_D;
    up[a] = k0 == FK_NBR_D ? -1 : (k1 == FK_NBR_D ? 1 : 0);
  }
  // start of the inflow window of axis a for the tile at K0 (8-aligned, at or below the run)
  auto win0 = [&](int a, int K0) -> int {
    const int x = K0 + up[a] * (int)g.stride[a];
    return x - (((x % 8) + 8) % 8);
  };
  // one thread of the group: the copies of tile T into stage st -- one box of all slots'
  // own runs [NEXP x 128] at (K0, 0), and per inflow axis one box of its slots' windows
  // [NF x 136] at (window start, a NF)
  auto issue = [&](int T, int st, int parity) {
    const int K0 = T * 128;
    const CUtensorMap* mo = parity ? &own1 : &own0;
    const CUtensorMap* mw = parity ? &win1m : &win0m;
    uint32_t bytes = (uint32_t)Z::OWNB;
#pragma unroll
    for (int a = 0; a < D; ++a) bytes += up[a] != 0 ? (uint32_t)(NF * Z::NBW * 2) : 0u;
    tc::expect_bytes(smb[st], bytes);
    const uint32_t base = stage_addr + (uint32_t)(st * Z::STAGE);
    tc::tensor_g2s(base, mo, K0, 0, smb[st]);
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (up[a] != 0) tc::tensor_g2s(base + Z::OWNB + a * Z::WB, mw, win0(a, K0), a * NF, smb[st]);
  };
  auto widen = [](RAW r) -> float { return __uint_as_float((unsigned)r << 16); };
  for (int s = 0;; ++s) {
    const TL* __restrict__ ec = ((jj0 + s) & 1) ? e1 : e0;
    TL* __restrict__ en = ((jj0 + s) & 1) ? e0 : e1;
    float pv = 0.f;
    if (s > 0)
      for (int i = tid; i < (int)gridDim.x; i += NT) pv += __ldcg(partf + ((s - 1) & 1) * gridDim.x + i);
    // lagged loop decision (as in k_inner_tc)
    {
      const float tot = sum_partials<NT>(pv, wsum);
      if (tid == 0) {
        const float step = sqrtf(tot);
        const bool budget = jj0 + s >= inner_max || iter0 + s >= max_iters;
        const bool stop = budget || (s > 0 && (step <= limf || !(step == step) || isinf(step)));
        s_stop = stop ? 1 : 0;
        if (blockIdx.x == 0) {
          ctrl->inner_iter = jj0 + s;
          ctrl->iter = iter0 + s;
          ctrl->lowp_sweeps = lowp0 + s;
          if (s > 0) ctrl->inner_step = (double)step;
          if (stop) ctrl->inner_done = 1;
        }
      }
      __syncthreads();
      if (s_stop) break;
    }
    const int par = (jj0 + s) & 1;   // which correction array is current
    if (gt == 0 && tile0 < ntiles) {
      tc::fence_proxy_async_global();
      issue(tile0, 0, par);
    }
    pending[0] = tile0 < ntiles;
    float acc = 0.f;
    int i = 0;
    for (int tile = tile0; tile < ntiles; tile += tstride, ++i) {
      const int st = i & 1;
      const int K0 = tile * 128, K = K0 + gt;
      const bool valid = K < nel;
      // the epilogue's residual
      RAW rr[NEXP];
      const RAW* rb = reinterpret_cast<const RAW*>(rlp);
#pragma unroll
      for (int e = 0; e < NEXP; ++e) rr[e] = rb[e * ld + (valid ? K : 0)];
      // this tile's copies (bounded wait; the group agrees on the outcome at the barrier)
      const int okc = tc::mbar_wait(smb[st], sphase[st]) ? 1 : 0;
      if (okc) {
        sphase[st] ^= 1u;
        pending[st] = 0;
      }
      // a1: pack row gt of A from the stage (own runs at gt, inflow windows at gt + delta)
      const RAW* own_s = reinterpret_cast<const RAW*>(sStage + st * Z::STAGE);
      const RAW* nb_s = reinterpret_cast<const RAW*>(sStage + st * Z::STAGE + Z::OWNB);
      {
        int c[3] = {0, 0, 0};
        if (valid) coords(g, K, c);
        // the stage holds bf16 already: A takes the bit patterns as they are (zeros where masked)
        unsigned t[KP];
#pragma unroll
        for (int k = NIN; k < KP; ++k) t[k] = 0u;
#pragma unroll
        for (int f = 0; f < NLF; ++f) {
          const int a = f >> 1, kind = g.kind[f];
          const bool bnd = valid && on_bnd(g, c, f);
          const int dl = up[a] != 0 ? (K0 + up[a] * (int)g.stride[a]) - win0(a, K0) : 0;
          const bool use_own = valid && kind == FK_OWN_D;
          const bool use_nb = valid && !bnd && kind == FK_NBR_D;
          // the face's kind is the same in every thread: one shared load per value
          if (kind == FK_OWN_D) {
#pragma unroll
            for (int q = 0; q < NF; ++q) t[f * NF + q] = use_own ? (unsigned)own_s[(a * NF + q) * 128 + gt] : 0u;
          } else if (kind == FK_NBR_D) {
#pragma unroll
            for (int q = 0; q < NF; ++q) t[f * NF + q] = use_nb ? (unsigned)nb_s[a * (Z::WB / 2) + q * Z::NBW + gt + dl] : 0u;
          } else {
#pragma unroll
            for (int q = 0; q < NF; ++q) t[f * NF + q] = 0u;
          }
        }
        unsigned char* row = sA + (gt >> 3) * ROWB + (gt & 7) * 16;
#pragma unroll
        for (int kc = 0; kc < KP / 8; ++kc) {
          const unsigned* v = t + kc * 8;
          *reinterpret_cast<uint4*>(row + kc * 128) =
              make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16), v[6] | (v[7] << 16));
        }
      }
      // one group barrier: A is complete, the copy wait's outcome is agreed, and every
      // thread is past the previous tile (its stage reads, its accumulator reads)
      tc::fence_proxy_async();
      tc::fence_before();
      const int badc = tc::group_or(bar_id, !okc);
      tc::fence_after();
      if (badc) { failed = 1; break; }
      // a3: D = A . B^T on the tensor cores; then the next tile's copies into the other stage,
      // read last by the previous tile (after the MMAs: they are on the tile's critical path)
      if (gt == 0) {
#pragma unroll
        for (int kk = 0; kk < KP / KSTEP; ++kk) {
          const uint64_t ah = tc::sdesc(aaddr + kk * 256, 128, ROWB), bh = tc::sdesc(baddr + kk * 256, 128, ROWB);
          tc::mma_bf16(tcol, ah, bh, IDESC, kk > 0 ? 1u : 0u);
        }
        tc::commit(mbar);
      }
      if (tile + tstride < ntiles) {
        if (gt == 0) issue(tile + tstride, st ^ 1, par);
        pending[st ^ 1] = 1;
      }
      __syncwarp();
      const int ok = tc::mbar_wait(mbar, phase) ? 1 : 0;
      const int bad = tc::group_or(bar_id, !ok);
      phase ^= 1u;
      if (bad) { failed = 1; break; }
      tc::fence_after();
      // a4: e_{j+1} = r + D; the step norm against the current exports in the stage
      float d[32];
      tc::ld32(tld, d);
      if (valid) {
#pragma unroll
        for (int e = 0; e < NEXP; ++e) {
          if ((g.live >> e) & 1ull) {
            const TL nv = from_f<TL>(widen(rr[e]) + d[e]);
            const float dl = to_f(nv) - widen(own_s[e * 128 + gt]);
            acc = fmaf(dl, dl, acc);
            en[e * ld + K] = nv;
          }
        }
      }
    }
    if (__syncthreads_or(failed)) {
      if (tid == 0) atomicExch(&ctrl->timeout, 1);
      break;
    }
    const float blk = sum_partials<NT>(acc, wsum);
    arrive_wait(partf + (s & 1) * gridDim.x, count, (unsigned)(s + 1), blk, ctrl, &s_to);
    if (s_to) break;
  }
  // copies still in flight (only after an expired wait) land before the block exits; an
  // expired MMA wait is waited for once more; then tensor memory is released
  for (int st = 0; st < 2; ++st)
    if (pending[st]) tc::mbar_wait(smb[st], sphase[st]);
  if (failed) tc::mbar_wait(mbar, phase ^ 1u);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem0), "r"(Z::TCOLS) : "memory");
}

// Launch the tensor-core inner kernel.  B = L_E (and its low part) in the core-matrix layout
// is built on the host and copied to the workspace once per solve.
}  // namespace

// Tensor maps of the staged tensor-core kernel over the correction arrays e0 and e1, each seen
// as a bf16 tensor [nexp slots][ld values] (row stride ld * 2 bytes): boxes [nexp x 128] of
// the own runs and [nf x nbw] of one axis's inflow windows, no swizzle, zeros outside.  The
// encoder is the driver's cuTensorMapEncodeTiled, reached through the runtime's entry-point
// query (no link to the driver library).  False when it is unavailable or refuses a map.
inline bool encode_tcs_maps(CUtensorMap* maps, void* e0, void* e1, long long ld, int nexp, int nf, int nbw) {
  using Enc = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                           const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                           CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Enc enc = nullptr;
  static bool tried = false;
  if (!tried) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      enc = reinterpret_cast<Enc>(fn);
    tried = true;
  }
  if (!enc || nexp > 256 || nf > 256) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)nexp};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box_own[2] = {128u, (cuuint32_t)nexp}, box_win[2] = {(cuuint32_t)nbw, (cuuint32_t)nf};
  const cuuint32_t es[2] = {1u, 1u};
  void* bases[2] = {e0, e1};
  for (int i = 0; i < 2; ++i) {
    if (enc(&maps[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, bases[i], dims, strides, box_own, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    if (enc(&maps[2 + i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, bases[i], dims, strides, box_win, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

// host twin of tc::rna_tf32: round a finite float32 to 10 mantissa bits, ties away from zero
inline float rna_tf32_host(float x) {
  unsigned u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

template <int NF, int NLF, bool PER_AXIS, int MODE>
cudaError_t launch_tc(MixedArgs& m, void* rlv, void* e0v, void* e1v) {
  using TL = typename std::conditional<MODE == TC_BF16, __nv_bfloat16, float>::type;
  TL* rl = static_cast<TL*>(rlv);
  TL* e0 = static_cast<TL*>(e0v);
  TL* e1 = static_cast<TL*>(e1v);
  using S = TcShape<NF, NLF, PER_AXIS, MODE>;
  if constexpr (!S::OK) {
    return cudaErrorNotSupported;
  } else {
    constexpr int NIN = S::NIN, NEXP = S::NEXP, EPC = S::EPC, G = S::G;
    const LaunchArgs& a = m.base;
    if (!m.LE32h || !m.dLT || a.g.n_exp != NEXP || (long long)a.g.ld * NEXP >= (1LL << 31)) return cudaErrorNotSupported;
    static_assert((size_t)S::NSPLIT * S::BBYTES <= MIXED_LT_BYTES, "operator scratch");
    auto k = k_inner_tc<NF, NLF, PER_AXIS, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 128 * G, S::SMEM);
    if (e != cudaSuccess) return e;
    if (per > (int)(512 / S::TCOLS)) per = (int)(512 / S::TCOLS);   // 512 tensor-memory columns per SM
    if (per < 1) return cudaErrorNotSupported;
    long long grid = (long long)per * sms;
    const long long ntiles = (a.g.nel + 127) / 128;
    const long long need = (ntiles + G - 1) / G;
    if (grid > need) grid = need;
    if (grid > m.max_grid) grid = m.max_grid;
    if (grid > m.slots / 2) return cudaErrorNotSupported;
    if (m.lt_kind != 2 + MODE) {
      // B[n][k] = L_E[n][k] at byte (n/8)*ROWB + (k/EPC)*128 + (n%8)*16 + (k%EPC)*ESZ; the
      // split mode stores B_hi, then B_lo
      std::vector<unsigned char> hb((size_t)S::NSPLIT * S::BBYTES, 0);
      for (int n = 0; n < NEXP; ++n)
        for (int kk = 0; kk < NIN; ++kk) {
          const size_t off = (size_t)(n / 8) * S::ROWB + (kk / EPC) * 128 + (n % 8) * 16 + (kk % EPC) * S::ESZ;
          const float v = m.LE32h[n * NIN + kk];
          if constexpr (MODE == TC_BF16) {
            const __nv_bfloat16 b = __float2bfloat16_rn(v);
            std::memcpy(&hb[off], &b, 2);
          } else if constexpr (MODE == TC_TF32) {
            std::memcpy(&hb[off], &v, 4);
          } else {
            const float hi = rna_tf32_host(v);
            const float lo = rna_tf32_host(v - hi);
            std::memcpy(&hb[off], &hi, 4);
            std::memcpy(&hb[S::BBYTES + off], &lo, 4);
          }
        }
      e = cudaMemcpyAsync(m.dLT, hb.data(), hb.size(), cudaMemcpyHostToDevice, a.stream);
      if (e != cudaSuccess) return e;
      m.lt_kind = 2 + MODE;
    }
    e = cudaMemsetAsync(&a.ctrl->bar_count, 0, sizeof(unsigned), a.stream);
    if (e != cudaSuccess) return e;
    DevGeo gg = a.g;
    const TL* rlc = rl;
    Ctrl* ct = a.ctrl;
    double* pp = a.partials;
    const unsigned char* bp = reinterpret_cast<const unsigned char*>(m.dLT);
    void* args[] = {&gg, &rlc, &e0, &e1, &ct, &pp, &bp};
    m.tc_staged = 0;
    if constexpr (MODE == TC_BF16 && PER_AXIS) {
      // the staged variant when the correction arrays carry guard bands wide enough for its
      // windows (IHDG_TC_STAGED=0 keeps the register-gather kernel)
      using Z = TcsShape<NF, NLF>;
      long long step = 1;
      for (int ax = 0; ax < a.g.dim; ++ax) step = a.g.stride[ax] > step ? a.g.stride[ax] : step;
      const char* env = std::getenv("IHDG_TC_STAGED");
      const bool want = !(env && std::strcmp(env, "0") == 0);
      if constexpr (Z::OK) {
        CUtensorMap maps[4];
        const bool have_maps = want && encode_tcs_maps(maps, e0, e1, a.g.ld, Z::NEXP, NF, Z::NBW);
        if (have_maps && m.e_pad >= step + 8 + Z::NBW) {
          auto ks = k_inner_tcs<NF, NLF>;
          e = cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, Z::SMEM);
          if (e != cudaSuccess) return e;
          int pers = 0;
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pers, ks, 128 * Z::G, Z::SMEM);
          if (e != cudaSuccess) return e;
          if (pers > (int)(512 / Z::TCOLS)) pers = (int)(512 / Z::TCOLS);
          if (pers >= 1) {
            long long gs = (long long)pers * sms;
            const long long needs = (ntiles + Z::G - 1) / Z::G;
            if (gs > needs) gs = needs;
            if (gs > m.max_grid) gs = m.max_grid;
            if (gs <= m.slots / 2) {
              void* args_s[] = {&gg, &rlc, &e0, &e1, &ct, &pp, &bp, &maps[0], &maps[1], &maps[2], &maps[3]};
              e = cudaLaunchCooperativeKernel((const void*)ks, dim3((unsigned)gs), dim3(128 * Z::G), args_s, Z::SMEM,
                                              a.stream);
              if (e != cudaSuccess) return e;
              m.tc_staged = 1;
              return cudaGetLastError();
            }
          }
        }
      }
    }
    e = cudaLaunchCooperativeKernel((const void*)k, dim3((unsigned)grid), dim3(128 * G), args, S::SMEM, a.stream);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
}

}  // namespace ihdg

// explicit instantiation over the element shapes the mixed path dispatches
#define IHDG_TC_INSTANTIATE(MODE)                                                             \
  namespace ihdg {                                                                            \
  template cudaError_t launch_tc<2, 4, true, MODE>(MixedArgs&, void*, void*, void*);          \
  template cudaError_t launch_tc<2, 4, false, MODE>(MixedArgs&, void*, void*, void*);         \
  template cudaError_t launch_tc<3, 4, true, MODE>(MixedArgs&, void*, void*, void*);          \
  template cudaError_t launch_tc<3, 4, false, MODE>(MixedArgs&, void*, void*, void*);         \
  template cudaError_t launch_tc<4, 4, true, MODE>(MixedArgs&, void*, void*, void*);          \
  template cudaError_t launch_tc<4, 4, false, MODE>(MixedArgs&, void*, void*, void*);         \
  template cudaError_t launch_tc<5, 4, true, MODE>(MixedArgs&, void*, void*, void*);          \
  template cudaError_t launch_tc<5, 4, false, MODE>(MixedArgs&, void*, void*, void*);         \
  template cudaError_t launch_tc<4, 6, true, MODE>(MixedArgs&, void*, void*, void*);          \
  template cudaError_t launch_tc<4, 6, false, MODE>(MixedArgs&, void*, void*, void*);         \
  template cudaError_t launch_tc<9, 6, true, MODE>(MixedArgs&, void*, void*, void*);          \
  template cudaError_t launch_tc<9, 6, false, MODE>(MixedArgs&, void*, void*, void*);         \
  }
