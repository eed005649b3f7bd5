// Transport with a velocity field that varies in space: the per-element local solves on the
// device (see ihdg_var.h).  The state is the volume solution u, element-major ([K][node]).
//
// A group of GS lanes (the power of two >= the element's node count) owns one element at a
// time.  a1: the lanes gather the element's trace values t (own face nodes on outflow faces,
// the neighbour's on inflow faces, 0 on the inflow boundary), a few per lane; a3: lane i
// accumulates node i of A_K^{-1} b_K + L_K t, streaming the element's operator one trace column
// at a time (a column is the group's consecutive nodes, so every load is coalesced) and taking
// each trace value from its lane by a shuffle; a4: the change of the iterate and its mass
// norm (tensor-product mass matrix, one 1D application per axis by shuffles), reduced per
// block in a fixed order and over the grid by the last block to arrive, which takes the loop
// decision.  This is the batched GEMV of heterogeneous elements: each element streams its own
// operator, so the sweep is bound by HBM bandwidth in float32 / bf16 and by the float64 FMA
// rate in float64.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <sstream>
#include <string>
#include <vector>

#include "ihdg_common.cuh"
#include "ihdg_kernels.h"
#include "ihdg_persist.cuh"
#include "ihdg_var.h"

namespace ihdg {
namespace {

constexpr int VNT = 256;   // threads per block

template <int D, int P>
struct VShape {
  static constexpr int NB1 = P + 1;
  static constexpr int NB = D == 2 ? NB1 * NB1 : NB1 * NB1 * NB1;
  static constexpr int NF = D == 2 ? NB1 : NB1 * NB1;
  static constexpr int NLF = 2 * D;
  static constexpr int NIN = NLF * NF;
  static constexpr int Q = P + 2;
  static constexpr int NQV = D == 2 ? Q * Q : Q * Q * Q;
  static constexpr int NQF = D == 2 ? Q : Q * Q;
  static constexpr int GS = NB <= 4 ? 4 : NB <= 8 ? 8 : NB <= 16 ? 16 : 32;   // lanes per element
  static constexpr int EPW = 32 / GS;                                          // elements per warp
  static constexpr int EPB = (VNT / 32) * EPW;                                 // elements per block pass
  static constexpr int TPL = (NIN + GS - 1) / GS;                              // trace values per lane
};

// Scalars of one problem, passed by value.
struct VGeo {
  int n[3];
  long long nel;
  int kind[6];
  int sign[3];
  double jac;
  long long nbf_off[3];
};

VGeo vgeo(const VarDev& d) {
  VGeo g{};
  for (int a = 0; a < 3; ++a) {
    g.n[a] = d.n[a];
    g.sign[a] = d.sign[a];
  }
  for (int f = 0; f < 6; ++f) g.kind[f] = d.kind[f];
  g.nel = d.nel;
  g.jac = d.jac;
  g.nbf_off[0] = 0;
  g.nbf_off[1] = 2LL * d.n[1] * d.n[2];
  g.nbf_off[2] = g.nbf_off[1] + 2LL * d.n[0] * d.n[2];
  return g;
}

__device__ __forceinline__ void vcoords(const VGeo& g, long long K, int* c) {
  c[0] = (int)(K % g.n[0]);
  const long long t = K / g.n[0];
  c[1] = (int)(t % g.n[1]);
  c[2] = (int)(t / g.n[1]);
}
__device__ __forceinline__ long long vstride(const VGeo& g, int a) {
  return a == 0 ? 1LL : (a == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
}
// boundary-face number of local face f of the element at coordinates c (global face order)
__device__ __forceinline__ long long vbface(const VGeo& g, const int* c, int f) {
  const int a = f >> 1, s = f & 1;
  if (a == 0) return 2LL * (c[1] + (long long)g.n[1] * c[2]) + s;
  if (a == 1) return g.nbf_off[1] + (long long)c[2] * 2 * g.n[0] + (long long)s * g.n[0] + c[0];
  return g.nbf_off[2] + (long long)s * g.n[0] * g.n[1] + (long long)c[1] * g.n[0] + c[0];
}

template <typename T> __device__ __forceinline__ float vld(const T* p);
template <> __device__ __forceinline__ float vld<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float vld<__nv_bfloat16>(const __nv_bfloat16* p) {
  const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p));
  return __uint_as_float((unsigned)b << 16);
}

// plain loads of state arrays written by earlier launches
__device__ __forceinline__ double vld_or(const double* p, long long i) { return p[i]; }
__device__ __forceinline__ float vld_or(const float* p, long long i) { return p[i]; }
__device__ __forceinline__ float vld_or(const __nv_bfloat16* p, long long i) { return __bfloat162float(p[i]); }

// Per lane: the trace slots it gathers (k = lane + GS c): its face, own node and the
// neighbour's node at the same point.
template <class S>
struct Slots {
  int f[S::TPL], own[S::TPL], nbr[S::TPL];
  __device__ void load(const int* facevol, int gl) {
#pragma unroll
    for (int c = 0; c < S::TPL; ++c) {
      const int k = gl + S::GS * c;
      const int kk = k < S::NIN ? k : 0;
      f[c] = k < S::NIN ? kk / S::NF : -1;
      const int fr = kk / S::NF, r = kk % S::NF;
      own[c] = facevol[fr * S::NF + r];
      nbr[c] = facevol[(fr ^ 1) * S::NF + r];
    }
  }
};

// a1 for one element: trace value of each of this lane's slots, from state x (plus y when
// given: the mixed outer sweep gathers u + e).
template <class S, typename TX, typename TY, typename TA>
__device__ __forceinline__ void vgather(const VGeo& g, const Slots<S>& sl, const TX* x, const TY* y, long long K,
                                        const int* c, bool valid, TA* t) {
#pragma unroll
  for (int s = 0; s < S::TPL; ++s) {
    TA v = TA(0);
    const int f = sl.f[s];
    if (valid && f >= 0) {
      const int kind = g.kind[f];
      const int a = f >> 1;
      if (kind == 1) {
        const long long at = K * S::NB + sl.own[s];
        v = (TA)vld_or(x, at);
        if (y) v += (TA)vld_or(y, at);
      } else if (kind == 2) {
        const bool bnd = (f & 1) ? (c[a] == g.n[a] - 1) : (c[a] == 0);
        if (!bnd) {
          const long long Kn = (f & 1) ? K + vstride(g, a) : K - vstride(g, a);
          const long long at = Kn * S::NB + sl.nbr[s];
          v = (TA)vld_or(x, at);
          if (y) v += (TA)vld_or(y, at);
        }
      }
    }
    t[s] = v;
  }
}

// sum over the GS lanes of a group (result in every lane of the group)
template <int GS, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = GS / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, GS);
  return v;
}

// x^T M x for the element held one node per lane (x = 0 on lanes >= NB), M = jac (M1 x M1
// (x M1)): one 1D application per axis by shuffles within the group
template <class S>
__device__ __forceinline__ double mass_norm(double x, int gl, const double* sM1, double jac) {
  double z = x;
  int stride = 1;
#pragma unroll
  for (int a = 0; a < (S::NB == S::NB1 * S::NB1 ? 2 : 3); ++a) {
    const int ia = (gl / stride) % S::NB1;
    double w = 0.0;
#pragma unroll
    for (int b = 0; b < S::NB1; ++b) {
      const int src = (gl - ia * stride + b * stride) & (S::GS - 1);
      w += sM1[ia * S::NB1 + b] * __shfl_sync(0xffffffffu, z, src, S::GS);
    }
    z = w;
    stride *= S::NB1;
  }
  return group_sum<S::GS>(gl < S::NB ? jac * x * z : 0.0);
}

// Fixed-order block and grid reduction of two doubles over the nblk blocks of one problem
// (bid: this block's number among them); true in thread 0 of the last block to arrive, which
// then holds the totals.
__device__ bool var_arrive2(Ctrl* ctrl, double* partials, double a, double b, double* ta, double* tb, int bid,
                            int nblk) {
  __shared__ double sa[VNT / 32], sb[VNT / 32];
  __shared__ int s_last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0.0, B = 0.0;
    for (int i = 0; i < VNT / 32; ++i) {
      A += sa[i];
      B += sb[i];
    }
    partials[2 * bid] = A;
    partials[2 * bid + 1] = B;
    __threadfence();
    const unsigned t = atomicAdd(&ctrl->ticket, 1u);
    s_last = (t == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double A = 0.0, B = 0.0;
  for (int i = threadIdx.x; i < nblk; i += VNT) {
    A += __ldcg(partials + 2 * i);
    B += __ldcg(partials + 2 * i + 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    A += __shfl_down_sync(0xffffffffu, A, o);
    B += __shfl_down_sync(0xffffffffu, B, o);
  }
  __syncthreads();
  if (lane == 0) {
    sa[w] = A;
    sb[w] = B;
  }
  __syncthreads();
  if (threadIdx.x != 0) return false;
  A = B = 0.0;
  for (int i = 0; i < VNT / 32; ++i) {
    A += sa[i];
    B += sb[i];
  }
  *ta = A;
  *tb = B;
  ctrl->ticket = 0u;
  return true;
}

// a2: b_K = (f, phi_i)_K + the inflow boundary data, V_K = A_K^{-1} b_K (once per solve); the
// initial state u^0 = u0 (or 0).
template <int D, int P>
__global__ void __launch_bounds__(VNT) k_var_forcing(const VGeo g, const double* __restrict__ Ainv,
                                                     const double* __restrict__ Wq, const double* __restrict__ FBv,
                                                     const double* __restrict__ bw, const double* __restrict__ f,
                                                     const double* __restrict__ gb, const double* __restrict__ u0,
                                                     double* __restrict__ V, double* __restrict__ u) {
  using S = VShape<D, P>;
  const int lane = threadIdx.x & 31, gl = lane % S::GS;
  const long long first = (long long)blockIdx.x * S::EPB + (threadIdx.x >> 5) * S::EPW;
  for (long long base = first; base < g.nel; base += (long long)gridDim.x * S::EPB) {
    const long long K = base + lane / S::GS;
    const bool valid = K < g.nel;
    double b = 0.0;
    int c[3] = {0, 0, 0};
    if (valid) {
      vcoords(g, K, c);
      if (gl < S::NB) {
#pragma unroll 4
        for (int q = 0; q < S::NQV; ++q) b += Wq[gl * S::NQV + q] * f[K * S::NQV + q];
#pragma unroll
        for (int lf = 0; lf < S::NLF; ++lf) {
          const int a = lf >> 1;
          const bool bnd = (lf & 1) ? (c[a] == g.n[a] - 1) : (c[a] == 0);
          if (!bnd || g.kind[lf] != 2) continue;
          const long long bf = vbface(g, c, lf);
          for (int q = 0; q < S::NQF; ++q) b += bw[bf * S::NQF + q] * gb[bf * S::NQF + q] * FBv[(lf * S::NB + gl) * S::NQF + q];
        }
      }
    }
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < S::NB; ++j) {
      const double bj = __shfl_sync(0xffffffffu, b, j, S::GS);
      if (valid && gl < S::NB) v += Ainv[(K * S::NB + j) * S::NB + gl] * bj;
    }
    if (valid && gl < S::NB) {
      V[K * S::NB + gl] = v;
      u[K * S::NB + gl] = u0 ? u0[K * S::NB + gl] : 0.0;
    }
  }
}

// Float64 sweep.  MODE 0 (the plain iteration): u^{k+1} = V + L t(u^k), stopping residual
// ||u^{k+1} - u^k||_M.  MODE 1 (mixed outer sweep): u' = u + e, r = V + L t(u') - u', written
// in float64 and as the low-precision residual and first correction; its norm ||r||_M is the
// stopping residual of the exact sweep from u'.
template <typename TL>
struct VSweepArgs {
  VGeo g;
  const double* L;
  const double* M1;
  const int* facevol;
  const double* V;
  double* u0p;
  double* u1p;
  const TL* e0;
  const TL* e1;
  double* r64;
  TL* rlp;
  Ctrl* ctrl;
  double* partials;
  double* res_hist;
  int nblk;   // blocks of this problem's launch
};

template <int D, int P, int MODE, typename TL>
__device__ __forceinline__ void var_sweep_body(const VSweepArgs<TL>& A, int bid) {
  using S = VShape<D, P>;
  __shared__ double sM1[S::NB1 * S::NB1];
  const VGeo& g = A.g;
  Ctrl* ctrl = A.ctrl;
  if (ctrl_done(ctrl)) return;
  // the mixed outer sweep runs once per inner loop: first, or after the inner loop has stopped
  const int outer0 = *(volatile const int*)&ctrl->outer;
  if (MODE == 1 && outer0 > 0 && !*(volatile const int*)&ctrl->inner_done) return;
  for (int i = threadIdx.x; i < S::NB1 * S::NB1; i += VNT) sM1[i] = A.M1[i];
  const int lane = threadIdx.x & 31, gl = lane % S::GS, grp = lane / S::GS;
  Slots<S> sl;
  sl.load(A.facevol, gl);
  __syncthreads();
  const int k0 = MODE == 0 ? ctrl_iter(ctrl) : outer0;
  const double* ucur = (k0 & 1) ? A.u1p : A.u0p;
  double* unext = (k0 & 1) ? A.u0p : A.u1p;
  // the correction of the last inner loop (none before the first outer step): after j >= 1
  // inner sweeps it is in e[j & 1]
  const TL* ec = nullptr;
  if (MODE == 1 && outer0 > 0) ec = (*(volatile const int*)&ctrl->inner_iter & 1) ? A.e1 : A.e0;
  double accM = 0.0, acc2 = 0.0;
  const long long first = (long long)bid * S::EPB + (threadIdx.x >> 5) * S::EPW;
  for (long long base = first; base < g.nel; base += (long long)A.nblk * S::EPB) {
    const long long K = base + grp;
    const bool valid = K < g.nel;
    int c[3] = {0, 0, 0};
    if (valid) vcoords(g, K, c);
    double t[S::TPL];
    vgather<S, double, TL, double>(g, sl, ucur, ec, K, c, valid, t);
    const bool row = valid && gl < S::NB;
    double uo = 0.0, s = 0.0;
    if (row) {
      uo = ucur[K * S::NB + gl];
      if (ec) uo += (double)vld_or(ec, K * S::NB + gl);
      s = A.V[K * S::NB + gl];
    }
    const double* Lk = A.L + (size_t)(valid ? K : 0) * S::NIN * S::NB + (gl < S::NB ? gl : 0);
#pragma unroll
    for (int k = 0; k < S::NIN; ++k) {
      const double tk = __shfl_sync(0xffffffffu, t[k / S::GS], k % S::GS, S::GS);
      s = fma(Lk[(size_t)k * S::NB], tk, s);
    }
    const double dlt = row ? s - uo : 0.0;
    const double m = mass_norm<S>(dlt, gl, sM1, g.jac);
    if (gl == 0 && valid) accM += m;
    if (row) {
      if (MODE == 0) {
        unext[K * S::NB + gl] = s;
      } else {
        unext[K * S::NB + gl] = uo;
        A.r64[K * S::NB + gl] = dlt;
        A.rlp[K * S::NB + gl] = from_f<TL>((float)dlt);
        acc2 += dlt * dlt;
      }
    }
  }
  double tM, t2;
  if (var_arrive2(ctrl, A.partials, accM, acc2, &tM, &t2, bid, A.nblk)) {
    decide(ctrl, tM, A.res_hist, true);
    if (MODE == 1) {
      ctrl->rnorm = sqrt(t2);
      ctrl->outer = k0 + 1;
      ctrl->inner_iter = 0;
      ctrl->inner_done = 0;
    }
  }
}

// Float64 sweep of one problem.  MODE 0 (the plain iteration): u^{k+1} = V + L t(u^k), stopping
// residual ||u^{k+1} - u^k||_M.  MODE 1 (mixed outer sweep): u' = u + e, r = V + L t(u') - u',
// written in float64 and as the low-precision residual; its norm ||r||_M is the stopping
// residual of the exact sweep from u'.
template <int D, int P, int MODE, typename TL>
__global__ void __launch_bounds__(VNT) k_var_sweep(const VSweepArgs<TL> A) {
  var_sweep_body<D, P, MODE, TL>(A, (int)blockIdx.x);
}

// Index of the problem that block b belongs to in a grouped launch (off: prefix sums of the
// problems' block counts, n + 1 entries).
__device__ __forceinline__ int group_item(const int* off, int n, int b) {
  int i = 0;
  while (i + 1 < n && __ldg(off + i + 1) <= b) ++i;
  return i;
}

// The same sweep for several problems of one shape in one launch: each problem keeps its own
// grid (block b - off[i] of nblk), reduction and loop state, so its result is bitwise the one
// of its own launch.
template <int D, int P, int MODE, typename TL>
__global__ void __launch_bounds__(VNT) k_var_sweep_group(const VSweepArgs<TL>* __restrict__ items,
                                                         const int* __restrict__ off, int n) {
  const int i = group_item(off, n, (int)blockIdx.x);
  const VSweepArgs<TL> A = items[i];
  var_sweep_body<D, P, MODE, TL>(A, (int)blockIdx.x - __ldg(off + i));
}

// The TMA engine's untiled bulk copy, global -> this CTA's shared memory, its completion
// counted in bytes on an mbarrier; bounded waits (the caller decides what to do on expiry).
__device__ __forceinline__ uint32_t vsmem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void vbulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
__device__ __forceinline__ bool vmbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool vmbar_wait(uint32_t mbar, uint32_t parity, long long lim) {
  const long long t0 = clock64();
  while (!vmbar_try(mbar, parity))
    if (clock64() - t0 > lim) return false;
  return true;
}

// Low-precision inner sweep of the mixed path: e_{j+1} = r + L t(e_j) with float32 arithmetic
// and TL storage of e, r and the operator; the inner loop stops when the step norm falls to
// inner_rtol * ||r|| (Euclidean norms over all nodes), after inner_max sweeps, or at the sweep
// budget.  Each warp streams the operators of its elements through a private ring of R stages
// in shared memory: one stage holds the EPW consecutive elements the warp computes together
// (their operator blocks are contiguous, each padded to lsb bytes, a multiple of 16), filled by
// one bulk copy that lane 0 issues R batches ahead, so R - 1 copies stay in flight while the
// warp gathers its traces and computes from shared memory.  Every wait is bounded: on expiry
// the kernel sets ctrl->timeout, waits (bounded) for its own copies still in flight and stops
// the loop.
template <typename TL>
struct VInnerArgs {
  VGeo g;
  const TL* L;
  int lsb, R;
  const int* facevol;
  const TL* rlp;
  TL* e0;
  TL* e1;
  Ctrl* ctrl;
  double* partials;
  int nblk;   // blocks of this problem's launch
};

template <int D, int P, typename TL>
__device__ __forceinline__ void var_inner_body(const VInnerArgs<TL>& A, int bid) {
  using S = VShape<D, P>;
  constexpr int NW = VNT / 32;
  extern __shared__ __align__(128) unsigned char vsm[];
  __shared__ __align__(8) unsigned long long s_mb[NW * 8];
  const VGeo& g = A.g;
  const TL* __restrict__ L = A.L;
  const TL* __restrict__ rlp = A.rlp;
  const int lsb = A.lsb, R = A.R;
  Ctrl* ctrl = A.ctrl;
  // nothing to do before the first outer step, after the inner loop stopped, or when done
  if (ctrl_done(ctrl) || *(volatile const int*)&ctrl->inner_done || *(volatile const int*)&ctrl->outer == 0) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, gl = lane % S::GS, grp = lane / S::GS;
  Slots<S> sl;
  sl.load(A.facevol, gl);
  // e_0 = r (the first correction from zero); e_j in e[j & 1] for j >= 1
  const int j = *(volatile const int*)&ctrl->inner_iter;
  const TL* ec = j == 0 ? rlp : ((j & 1) ? A.e1 : A.e0);
  TL* en = (j & 1) ? A.e0 : A.e1;
  const int SB = S::EPW * lsb;
  unsigned char* ring = vsm + (size_t)w * R * SB;
  const uint32_t mb0 = vsmem(&s_mb[w * 8]);
  if (lane == 0) {
    for (int q = 0; q < R; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0 + 8 * q) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const long long gw = (long long)bid * NW + w, GW = (long long)A.nblk * NW;
  const long long nbatch = (g.nel + S::EPW - 1) / S::EPW;
  // failure-detection test hook: warp 0 of block ctrl->stall_block issues no copy, so its
  // first wait runs out
  const bool stall = bid == ctrl->stall_block && w == 0;
  auto issue = [&](long long i) {   // lane 0: batch i of this warp into stage i % R
    const long long b = gw + i * GW;
    if (b >= nbatch || stall) return;
    const long long k0 = b * S::EPW;
    const long long cnt = g.nel - k0 < S::EPW ? g.nel - k0 : S::EPW;
    vbulk_load(vsmem(ring + (size_t)(i % R) * SB), reinterpret_cast<const char*>(L) + k0 * lsb, (uint32_t)(cnt * lsb),
               mb0 + 8 * (uint32_t)(i % R));
  };
  if (lane == 0)
    for (int q = 0; q < R; ++q) issue(q);
  const long long lim = ctrl->wait_cycles;
  float st = 0.f;
  long long fail = -1;
  // the gather of batch i + 1 (its traces, r and e values, plain loads) is issued before batch
  // i is computed, so its round trip overlaps the computation from shared memory
  struct Pre {
    long long K;
    bool valid;
    float t[S::TPL], s, old;
  };
  auto fetch = [&](long long i, Pre& q) {
    const long long b = gw + i * GW;
    q.K = b * S::EPW + grp;
    q.valid = b < nbatch && q.K < g.nel;
    int c[3] = {0, 0, 0};
    if (q.valid) vcoords(g, q.K, c);
    vgather<S, TL, TL, float>(g, sl, ec, (const TL*)nullptr, q.K, c, q.valid, q.t);
    q.s = q.old = 0.f;
    if (q.valid && gl < S::NB) {
      q.s = vld_or(rlp, q.K * S::NB + gl);
      q.old = vld_or(ec, q.K * S::NB + gl);
    }
  };
  Pre cur, nxt;
  fetch(0, cur);
  for (long long i = 0;; ++i) {
    const long long b = gw + i * GW;
    if (b >= nbatch) break;
    fetch(i + 1, nxt);
    const int stg = (int)(i % R);
    const bool ok = __all_sync(0xffffffffu, vmbar_wait(mb0 + 8 * stg, (uint32_t)((i / R) & 1), lim));
    if (!ok) {
      fail = i;
      break;
    }
    const TL* Ls = reinterpret_cast<const TL*>(ring + (size_t)stg * SB + (size_t)grp * lsb) + (gl < S::NB ? gl : 0);
    float acc = cur.s;
#pragma unroll
    for (int k = 0; k < S::NIN; ++k) {
      const float tk = __shfl_sync(0xffffffffu, cur.t[k / S::GS], k % S::GS, S::GS);
      acc = fmaf(to_f(Ls[k * S::NB]), tk, acc);
    }
    if (cur.valid && gl < S::NB) {
      const TL nv = from_f<TL>(acc);
      const float d = to_f(nv) - cur.old;
      st = fmaf(d, d, st);
      en[cur.K * S::NB + gl] = nv;
    }
    __syncwarp();
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(i + R);
    }
    cur = nxt;
  }
  if (fail >= 0) {   // a copy did not arrive in time: flag it, then wait for this warp's copies in flight
    if (lane == 0) {
      atomicExch(&ctrl->timeout, 1);
      for (long long i = fail; !stall && i < fail + R && gw + i * GW < nbatch; ++i)   // ~1 s each at most
        vmbar_wait(mb0 + 8 * (uint32_t)(i % R), (uint32_t)((i / R) & 1), 2000000000LL);
    }
    __syncwarp();
  }
  double tA, tB;
  if (var_arrive2(ctrl, A.partials, (double)st, 0.0, &tA, &tB, bid, A.nblk)) {
    const int jn = j + 1, it = ctrl->iter + 1;
    ctrl->inner_iter = jn;
    ctrl->iter = it;
    ctrl->lowp_sweeps += 1;
    const double step = sqrt(tA);
    ctrl->inner_step = step;
    if (*(volatile int*)&ctrl->timeout) {
      ctrl->inner_done = 1;
      ctrl->done = 1;
      ctrl->status = IHDG_ERR_TIMEOUT;
    } else if (step <= ctrl->inner_rtol * ctrl->rnorm || jn >= ctrl->inner_max || it >= ctrl->max_iters ||
               !(step == step) || isinf(step)) {
      ctrl->inner_done = 1;
    }
  }
}

template <int D, int P, typename TL>
__global__ void __launch_bounds__(VNT) k_var_inner(const VInnerArgs<TL> A) {
  var_inner_body<D, P, TL>(A, (int)blockIdx.x);
}

// The inner sweep of several problems of one shape in one launch (as k_var_sweep_group).
template <int D, int P, typename TL>
__global__ void __launch_bounds__(VNT) k_var_inner_group(const VInnerArgs<TL>* __restrict__ items,
                                                         const int* __restrict__ off, int n) {
  const int i = group_item(off, n, (int)blockIdx.x);
  const VInnerArgs<TL> A = items[i];
  var_inner_body<D, P, TL>(A, (int)blockIdx.x - __ldg(off + i));
}

// u_out = the final state (plain) or the last outer state plus its exact-sweep residual
// (mixed: one float64 sweep from u').
__global__ void k_var_output(long long n, const double* __restrict__ u, const double* __restrict__ r,
                             double* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = u[i] + (r ? r[i] : 0.0);
}

// The trace on every global face at its GLL nodes: the upwind element's nodal values on
// interior faces (the average where beta_a = 0), the L2 projection of g on inflow boundary
// faces, the element's own values on the rest of the boundary.
template <int D, int P>
__global__ void k_var_trace(const VGeo g, const double* __restrict__ u, const int* __restrict__ facevol,
                            const double* __restrict__ Pg, const double* __restrict__ gb, long long nface,
                            double* __restrict__ tr) {
  using S = VShape<D, P>;
  const long long n2 = D == 3 ? g.n[2] : 1;
  const long long off1 = (long long)(g.n[0] + 1) * g.n[1] * n2;
  const long long off2 = off1 + (long long)g.n[0] * (g.n[1] + 1) * n2;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nface * S::NF;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long fid = idx / S::NF;
    const int r = (int)(idx % S::NF);
    const int a = fid < off1 ? 0 : (fid < off2 ? 1 : 2);
    long long loc = fid - (a == 0 ? 0 : (a == 1 ? off1 : off2));
    const int e0 = g.n[0] + (a == 0), e1 = g.n[1] + (a == 1);
    int c[3];
    c[0] = (int)(loc % e0);
    loc /= e0;
    c[1] = (int)(loc % e1);
    c[2] = (int)(loc / e1);
    const bool hasL = c[a] >= 1, hasR = c[a] < g.n[a];
    int cl[3] = {c[0], c[1], c[2]};
    cl[a] -= 1;
    const long long KL = hasL ? cl[0] + (long long)g.n[0] * (cl[1] + (long long)g.n[1] * cl[2]) : -1;
    const long long KR = hasR ? c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]) : -1;
    const double vL = hasL ? u[KL * S::NB + facevol[(2 * a + 1) * S::NF + r]] : 0.0;
    const double vR = hasR ? u[KR * S::NB + facevol[(2 * a) * S::NF + r]] : 0.0;
    double v;
    if (hasL && hasR) {
      v = g.sign[a] > 0 ? vL : (g.sign[a] < 0 ? vR : 0.5 * (vL + vR));
    } else {
      const int lf = hasL ? 2 * a + 1 : 2 * a;
      if (g.kind[lf] == 2) {
        const long long bf = vbface(g, hasL ? cl : c, lf);
        double s = 0.0;
        for (int q = 0; q < S::NQF; ++q) s += Pg[r * S::NQF + q] * gb[bf * S::NQF + q];
        v = s;
      } else {
        v = hasL ? vL : vR;
      }
    }
    tr[idx] = v;
  }
}

// float32 and bf16 copies of the operators, each element's block padded to ls32 / ls16 values
__global__ void k_var_convert(long long nel, int per, const double* __restrict__ x, float* __restrict__ y32, int ls32,
                              __nv_bfloat16* __restrict__ y16, int ls16) {
  const long long n = nel * per;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long K = i / per, jx = i % per;
    const double v = x[i];
    y32[K * ls32 + jx] = (float)v;
    y16[K * ls16 + jx] = __float2bfloat16_rn((float)v);
  }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Launches of one shape.
template <int D, int P>
struct VarRun {
  static cudaError_t forcing(VarDev& d, const double* f, const double* gb, const double* u0, cudaStream_t s) {
    k_var_forcing<D, P><<<d.grid, VNT, 0, s>>>(vgeo(d), d.Ainv, d.Wq, d.FBv, d.bw, f, gb, u0, d.V, d.u[0]);
    return cudaGetLastError();
  }
  template <typename TL>
  static VSweepArgs<TL> sweep_args(VarDev& d) {
    VSweepArgs<TL> A{};
    A.g = vgeo(d);
    A.L = d.L64;
    A.M1 = d.M1;
    A.facevol = d.facevol;
    A.V = d.V;
    A.u0p = d.u[0];
    A.u1p = d.u[1];
    A.e0 = static_cast<const TL*>(d.e[0]);
    A.e1 = static_cast<const TL*>(d.e[1]);
    A.r64 = d.r64;
    A.rlp = static_cast<TL*>(d.rlp);
    A.ctrl = d.ctrl;
    A.partials = d.partials;
    A.res_hist = d.res_hist;
    A.nblk = d.grid;
    return A;
  }
  template <typename TL>
  static cudaError_t sweep(VarDev& d, int mode, cudaStream_t s) {
    const VSweepArgs<TL> A = sweep_args<TL>(d);
    if (mode == 0) k_var_sweep<D, P, 0, TL><<<d.grid, VNT, 0, s>>>(A);
    else k_var_sweep<D, P, 1, TL><<<d.grid, VNT, 0, s>>>(A);
    return cudaGetLastError();
  }
  // the inner kernel's launch shape: stages per warp for ~100 KB of shared memory per block (two
  // blocks per SM), 2..8; grid capped by residency and by the partials array (d.grid blocks)
  template <typename TL>
  static cudaError_t inner_args(VarDev& d, VInnerArgs<TL>* A, size_t* smem) {
    using S = VShape<D, P>;
    const bool f32 = std::is_same<TL, float>::value;
    const int lsb = f32 ? d.lsb32 : d.lsb16;
    const int nw = VNT / 32, sb = S::EPW * lsb;
    int R = (100 * 1024) / (nw * sb);
    R = R < 2 ? 2 : (R > 8 ? 8 : R);
    *smem = (size_t)nw * R * sb;
    auto k = k_var_inner<D, P, TL>;
    auto kg = k_var_inner_group<D, P, TL>;
    cudaError_t e = allow_dynamic_smem(k);
    if (e == cudaSuccess) e = allow_dynamic_smem(kg);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, VNT, *smem);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    const long long nbatch = (d.nel + S::EPW - 1) / S::EPW;
    long long grid = (nbatch + nw - 1) / nw;
    if (grid > (long long)per * sms) grid = (long long)per * sms;
    if (grid > d.grid) grid = d.grid;
    *A = VInnerArgs<TL>{};
    A->g = vgeo(d);
    A->L = f32 ? (const TL*)d.L32 : (const TL*)d.L16;
    A->lsb = lsb;
    A->R = R;
    A->facevol = d.facevol;
    A->rlp = static_cast<const TL*>(d.rlp);
    A->e0 = static_cast<TL*>(d.e[0]);
    A->e1 = static_cast<TL*>(d.e[1]);
    A->ctrl = d.ctrl;
    A->partials = d.partials;
    A->nblk = (int)grid;
    return cudaSuccess;
  }
  template <typename TL>
  static cudaError_t inner(VarDev& d, cudaStream_t s) {
    VInnerArgs<TL> A;
    size_t smem = 0;
    cudaError_t e = inner_args<TL>(d, &A, &smem);
    if (e != cudaSuccess) return e;
    k_var_inner<D, P, TL><<<(unsigned)A.nblk, VNT, smem, s>>>(A);
    return cudaGetLastError();
  }
  // grouped launches over device descriptor arrays (items, off: n + 1 prefix sums of blocks)
  template <typename TL>
  static cudaError_t sweep_group(const void* items, const int* off, int n, int blocks, int mode, cudaStream_t s) {
    const auto* it = static_cast<const VSweepArgs<TL>*>(items);
    if (mode == 0) k_var_sweep_group<D, P, 0, TL><<<blocks, VNT, 0, s>>>(it, off, n);
    else k_var_sweep_group<D, P, 1, TL><<<blocks, VNT, 0, s>>>(it, off, n);
    return cudaGetLastError();
  }
  template <typename TL>
  static cudaError_t inner_group(const void* items, const int* off, int n, int blocks, size_t smem, cudaStream_t s) {
    k_var_inner_group<D, P, TL><<<blocks, VNT, smem, s>>>(static_cast<const VInnerArgs<TL>*>(items), off, n);
    return cudaGetLastError();
  }
  static cudaError_t trace(VarDev& d, const double* u, const double* gb, double* tr, cudaStream_t s) {
    const long long n = d.nface * d.nf;
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, 4096);
    k_var_trace<D, P><<<grid, 256, 0, s>>>(vgeo(d), u, d.facevol, d.Pg, gb, d.nface, tr);
    return cudaGetLastError();
  }
};

// Dispatch on (dim, p); F is a generic callable taking a VarRun type tag.
template <typename F>
cudaError_t var_dispatch(const VarDev& d, F&& fn) {
  if (d.dim == 2) {
    switch (d.p) {
      case 1: return fn(VarRun<2, 1>{});
      case 2: return fn(VarRun<2, 2>{});
      case 3: return fn(VarRun<2, 3>{});
      case 4: return fn(VarRun<2, 4>{});
    }
  } else {
    switch (d.p) {
      case 1: return fn(VarRun<3, 1>{});
      case 2: return fn(VarRun<3, 2>{});
    }
  }
  return cudaErrorNotSupported;
}

int elements_per_pass(int dim, int p) {
  const int nb = dim == 2 ? (p + 1) * (p + 1) : (p + 1) * (p + 1) * (p + 1);
  const int gs = nb <= 4 ? 4 : nb <= 8 ? 8 : nb <= 16 ? 16 : 32;
  return (VNT / 32) * (32 / gs);
}

}  // namespace

cudaError_t var_upload(const VarHost& h, VarDev& d, int max_hist) {
  d.dim = h.dim;
  d.p = h.p;
  d.nb = h.nb;
  d.nb1 = h.nb1;
  d.nf = h.nf;
  d.nlf = h.nlf;
  d.nin = h.nin;
  d.nqv = h.nqv;
  d.nqf = h.nqf;
  for (int a = 0; a < 3; ++a) {
    d.n[a] = h.n[a];
    d.sign[a] = h.sign[a];
  }
  for (int f = 0; f < 6; ++f) d.kind[f] = h.kind[f];
  d.nel = h.nel;
  d.nface = h.nface;
  d.nbface = h.nbface;
  d.jac = h.jac;
  d.max_hist = max_hist;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long epb = elements_per_pass(h.dim, h.p);
  long long grid = (h.nel + epb - 1) / epb;
  if (grid > (long long)sms * 8) grid = (long long)sms * 8;   // 8 blocks of 256 threads per SM
  d.grid = (int)grid;
  const size_t nL = (size_t)h.nel * h.nin * h.nb, nA = (size_t)h.nel * h.nb * h.nb, nS = (size_t)h.nel * h.nb;
  // layout of the single allocation
  size_t at = 0;
  auto take = [&](size_t bytes) { size_t r = at; at += a256(bytes); return r; };
  const int per = h.nin * h.nb;
  d.lsb32 = (per * 4 + 15) / 16 * 16;   // bytes per element block, multiples of 16 (bulk copies)
  d.lsb16 = (per * 2 + 15) / 16 * 16;
  const size_t oL64 = take(nL * 8), oL32 = take((size_t)h.nel * d.lsb32), oL16 = take((size_t)h.nel * d.lsb16);
  const size_t oA = take(nA * 8);
  const size_t oWq = take(h.Wq.size() * 8), oFB = take(h.FBv.size() * 8), obw = take(std::max<size_t>(1, h.bw.size()) * 8);
  const size_t ofv = take(h.facevol.size() * 4), oM1 = take(h.M1.size() * 8), oPg = take(h.Pg.size() * 8);
  const size_t ou0 = take(nS * 8), ou1 = take(nS * 8), oV = take(nS * 8), or64 = take(nS * 8), orl = take(nS * 4);
  const size_t oe0 = take(nS * 4), oe1 = take(nS * 4), oc = take(sizeof(Ctrl)), op = take((size_t)grid * 2 * 8);
  const size_t oh = take((size_t)(max_hist + 2) * 8);
  d.bytes = at;
  cudaError_t e = cudaMalloc(&d.mem, d.bytes);
  if (e != cudaSuccess) {
    d.mem = nullptr;
    return e;
  }
  char* b = static_cast<char*>(d.mem);
  d.L64 = reinterpret_cast<const double*>(b + oL64);
  d.L32 = reinterpret_cast<const float*>(b + oL32);
  d.L16 = b + oL16;
  d.Ainv = reinterpret_cast<const double*>(b + oA);
  d.Wq = reinterpret_cast<const double*>(b + oWq);
  d.FBv = reinterpret_cast<const double*>(b + oFB);
  d.bw = reinterpret_cast<const double*>(b + obw);
  d.facevol = reinterpret_cast<const int*>(b + ofv);
  d.M1 = reinterpret_cast<const double*>(b + oM1);
  d.Pg = reinterpret_cast<const double*>(b + oPg);
  d.u[0] = reinterpret_cast<double*>(b + ou0);
  d.u[1] = reinterpret_cast<double*>(b + ou1);
  d.V = reinterpret_cast<double*>(b + oV);
  d.r64 = reinterpret_cast<double*>(b + or64);
  d.rlp = b + orl;
  d.e[0] = b + oe0;
  d.e[1] = b + oe1;
  d.ctrl = reinterpret_cast<Ctrl*>(b + oc);
  d.partials = reinterpret_cast<double*>(b + op);
  d.res_hist = reinterpret_cast<double*>(b + oh);
  auto up = [&](size_t off, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(b + off, src, bytes, cudaMemcpyHostToDevice);
  };
  up(oL64, h.L.data(), nL * 8);
  up(oA, h.Ainv.data(), nA * 8);
  up(oWq, h.Wq.data(), h.Wq.size() * 8);
  up(oFB, h.FBv.data(), h.FBv.size() * 8);
  up(obw, h.bw.data(), h.bw.size() * 8);
  up(ofv, h.facevol.data(), h.facevol.size() * 4);
  up(oM1, h.M1.data(), h.M1.size() * 8);
  up(oPg, h.Pg.data(), h.Pg.size() * 8);
  if (e == cudaSuccess) e = cudaMemset(b + oL32, 0, (size_t)h.nel * d.lsb32);
  if (e == cudaSuccess) e = cudaMemset(b + oL16, 0, (size_t)h.nel * d.lsb16);
  if (e == cudaSuccess) {
    k_var_convert<<<(unsigned)std::min<size_t>((nL + 255) / 256, (size_t)sms * 16), 256>>>(
        (long long)h.nel, per, d.L64, reinterpret_cast<float*>(b + oL32), d.lsb32 / 4,
        reinterpret_cast<__nv_bfloat16*>(b + oL16), d.lsb16 / 2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) var_free(d);
  return e;
}

void var_free(VarDev& d) {
  if (d.mem) cudaFree(d.mem);
  d.mem = nullptr;
}

ihdg_status var_solve(VarDev& d, const double* f, const double* gb, const ihdg_options& o, double* u_out,
                      double* tr_out, cudaStream_t s, Ctrl* hc, std::string& err, ihdg_result* res) {
  NvtxRange nv(o.prec == IHDG_FP64 ? "ihdg variable-coefficient solve (float64)" : "ihdg variable-coefficient solve (mixed)");
  auto ck = [&](cudaError_t e, const char* where) {
    if (e != cudaSuccess) {
      err = std::string(where) + ": " + cudaGetErrorString(e);
      return false;
    }
    return true;
  };
  if (o.prec == IHDG_MIXED_TF32) {
    err = "variable-coefficient transport takes FP64, MIXED_FP32 or MIXED_BF16";
    return IHDG_ERR_UNSUPPORTED;
  }
  if (o.krylov_restart != 0) {
    err = "variable-coefficient solves run Algorithm 1 (opts.krylov_restart = 0)";
    return IHDG_ERR_UNSUPPORTED;
  }
  const int max_iters = std::min(o.max_iters, d.max_hist);
  double inner_rtol = o.inner_rtol > 0.0 ? o.inner_rtol : (o.prec == IHDG_MIXED_BF16 ? 0.2 : 2e-3);
  struct Ev {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Ev() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  if (!ck(cudaEventCreate(&ev.a), "cudaEventCreate") || !ck(cudaEventCreate(&ev.b), "cudaEventCreate")) return IHDG_ERR_CUDA;
  LaunchArgs la{};
  la.ctrl = d.ctrl;
  la.stream = s;
  // bound of the inner kernel's waits for its operator copies (~1 s of SM clock); the
  // failure-detection tests shorten it with IHDG_TEST_WAIT_CYCLES
  long long wait_cycles = 2000000000LL;
  int stall_block = -1;
  if (const char* wv = std::getenv("IHDG_TEST_WAIT_CYCLES")) {
    const long long v = std::atoll(wv);
    if (v > 0) wait_cycles = v;
  }
  if (const char* sb = std::getenv("IHDG_TEST_STALL_BLOCK")) stall_block = std::atoi(sb);
  int launches = 0;
  if (!ck(cudaEventRecord(ev.a, s), "cudaEventRecord") ||
      !ck(launch_ctrl_init(la, o.tol, o.diverge_factor, max_iters, o.inner_max, inner_rtol, wait_cycles, stall_block), "ctrl init") ||
      !ck(var_dispatch(d, [&](auto R) { return decltype(R)::forcing(d, f, gb, o.u0, s); }), "forcing kernel"))
    return IHDG_ERR_CUDA;
  launches += 2;
  auto readback = [&](const char* where) {
    return ck(cudaMemcpyAsync(hc, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s), where) &&
           ck(cudaStreamSynchronize(s), where);
  };
  const bool mixed = o.prec != IHDG_FP64;
  const bool bf16 = o.prec == IHDG_MIXED_BF16;
  // profile: events around every sweep launch (synchronised), averaged per kind
  struct Prof {
    cudaEvent_t a = nullptr, b = nullptr;
    double ms64 = 0.0, mslp = 0.0;
    int n64 = 0, nlp = 0;
    ~Prof() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } pf;
  const bool prof = o.profile != 0;
  if (prof && (!ck(cudaEventCreate(&pf.a), "cudaEventCreate") || !ck(cudaEventCreate(&pf.b), "cudaEventCreate")))
    return IHDG_ERR_CUDA;
  auto timed = [&](auto&& launch, bool fp64) {
    if (!prof) return launch();
    cudaEventRecord(pf.a, s);
    cudaError_t e = launch();
    if (e != cudaSuccess) return e;
    cudaEventRecord(pf.b, s);
    e = cudaEventSynchronize(pf.b);
    float t = 0.f;
    cudaEventElapsedTime(&t, pf.a, pf.b);
    if (fp64) { pf.ms64 += t; pf.n64 += 1; } else { pf.mslp += t; pf.nlp += 1; }
    return e;
  };
  const double* ufinal = nullptr;
  const double* rfinal = nullptr;
  if (!mixed) {
    int batch = 2;
    for (;;) {
      if (!readback("sweep loop")) return IHDG_ERR_CUDA;
      if (hc->done) break;
      const int left = hc->max_iters - hc->iter;
      const int n = std::min(batch, left);
      if (n <= 0) break;
      for (int i = 0; i < n; ++i)
        if (!ck(timed([&] { return var_dispatch(d, [&](auto R) { return decltype(R)::template sweep<float>(d, 0, s); }); },
                      true),
                "sweep kernel"))
          return IHDG_ERR_CUDA;
      launches += n;
      if (batch < 32) batch *= 2;
    }
    ufinal = d.u[hc->iter & 1];
  } else {
    for (;;) {
      cudaError_t e = timed([&] {
        return var_dispatch(d, [&](auto R) {
          return bf16 ? decltype(R)::template sweep<__nv_bfloat16>(d, 1, s)
                      : decltype(R)::template sweep<float>(d, 1, s);
        });
      }, true);
      if (!ck(e, "outer sweep kernel")) return IHDG_ERR_CUDA;
      launches += 1;
      if (!readback("outer sweep")) return IHDG_ERR_CUDA;
      if (hc->done) break;
      int batch = 4;
      for (;;) {
        for (int i = 0; i < batch; ++i) {
          e = timed([&] {
            return var_dispatch(d, [&](auto R) {
              return bf16 ? decltype(R)::template inner<__nv_bfloat16>(d, s) : decltype(R)::template inner<float>(d, s);
            });
          }, false);
          if (!ck(e, "inner sweep kernel")) return IHDG_ERR_CUDA;
        }
        launches += batch;
        if (!readback("inner loop")) return IHDG_ERR_CUDA;
        if (hc->timeout) {
          err = "inner sweep: an operator copy into shared memory did not complete in time";
          return IHDG_ERR_TIMEOUT;
        }
        if (hc->inner_done || hc->done) break;
        if (batch < 64) batch *= 2;
      }
    }
    ufinal = d.u[hc->outer & 1];
    rfinal = d.r64;
  }
  const long long nS = d.nel * d.nb;
  k_var_output<<<(unsigned)std::min<long long>((nS + 255) / 256, 4096), 256, 0, s>>>(nS, ufinal, rfinal, u_out);
  if (!ck(cudaGetLastError(), "output kernel")) return IHDG_ERR_CUDA;
  launches += 1;
  if (tr_out) {
    if (!ck(var_dispatch(d, [&](auto R) { return decltype(R)::trace(d, u_out, gb, tr_out, s); }), "trace kernel"))
      return IHDG_ERR_CUDA;
    launches += 1;
  }
  if (!ck(cudaEventRecord(ev.b, s), "cudaEventRecord") || !readback("solve")) return IHDG_ERR_CUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev.a, ev.b);
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->iterations = hc->iter;
    res->fp64_sweeps = hc->fp64_sweeps;
    res->lowp_sweeps = hc->lowp_sweeps;
    res->residual = hc->res;
    res->status = (ihdg_status)hc->status;
    res->solve_ms = ms;
    res->kernel_launches = launches;
    // inner launches that found the loop stopped return at once; the average is over the
    // sweeps the inner loop ran
    res->fp64_sweep_ms = pf.n64 ? pf.ms64 / pf.n64 : 0.0;
    res->lowp_sweep_ms = hc->lowp_sweeps ? pf.mslp / hc->lowp_sweeps : 0.0;
    res->fp64_launches = pf.n64;
    res->lowp_launches = pf.nlp;
  }
  return IHDG_OK;
}

}  // namespace ihdg

namespace ihdg {

// Several plans solved together: every sweep step is one grouped launch per (dim, p) class
// over all the class's plans (each block works for one plan, as that block of the plan's own
// launch), so problems of any size and order share launches while each keeps its own grid,
// reductions and loop state.  Forcing, output and trace stay per plan (once per solve).
ihdg_status var_solve_group(std::vector<VarDev*>& ds, const std::vector<const double*>& f,
                            const std::vector<const double*>& gb, const ihdg_options& o,
                            const std::vector<double*>& u_out, const std::vector<double*>& tr_out, cudaStream_t s,
                            std::string& err, ihdg_result* res) {
  NvtxRange nv("ihdg variable-coefficient grouped solve");
  const int n = (int)ds.size();
  auto ck = [&](cudaError_t e, const char* where) {
    if (e != cudaSuccess) {
      err = std::string(where) + ": " + cudaGetErrorString(e);
      return false;
    }
    return true;
  };
  if (o.prec == IHDG_MIXED_TF32) {
    err = "variable-coefficient transport takes FP64, MIXED_FP32 or MIXED_BF16";
    return IHDG_ERR_UNSUPPORTED;
  }
  if (o.krylov_restart != 0) {
    err = "variable-coefficient solves run Algorithm 1 (opts.krylov_restart = 0)";
    return IHDG_ERR_UNSUPPORTED;
  }
  const bool mixed = o.prec != IHDG_FP64, bf16 = o.prec == IHDG_MIXED_BF16;
  const double inner_rtol = o.inner_rtol > 0.0 ? o.inner_rtol : (bf16 ? 0.2 : 2e-3);
  long long wait_cycles = 2000000000LL;
  if (const char* wv = std::getenv("IHDG_TEST_WAIT_CYCLES")) {
    const long long v = std::atoll(wv);
    if (v > 0) wait_cycles = v;
  }
  // resources released on every return path
  struct Res {
    void* dbuf = nullptr;
    Ctrl* hc = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    ~Res() {
      if (dbuf) cudaFree(dbuf);
      if (hc) cudaFreeHost(hc);
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } rs;
  if (!ck(cudaMallocHost(&rs.hc, sizeof(Ctrl) * n), "pinned loop state") || !ck(cudaEventCreate(&rs.a), "event") ||
      !ck(cudaEventCreate(&rs.b), "event"))
    return IHDG_ERR_CUDA;
  // classes of equal shape and their descriptor tables (host images, one device buffer)
  struct Cls {
    int dim, p;
    std::vector<int> plans;
    std::vector<unsigned char> sw, in;   // VSweepArgs / VInnerArgs images
    std::vector<int> soff, ioff;
    size_t smem = 0;
    size_t o_sw = 0, o_in = 0, o_soff = 0, o_ioff = 0;
  };
  std::vector<Cls> cls;
  for (int i = 0; i < n; ++i) {
    int c = -1;
    for (int k = 0; k < (int)cls.size(); ++k)
      if (cls[k].dim == ds[i]->dim && cls[k].p == ds[i]->p) c = k;
    if (c < 0) {
      cls.push_back(Cls{ds[i]->dim, ds[i]->p, {}, {}, {}, {0}, {0}});
      c = (int)cls.size() - 1;
    }
    cls[c].plans.push_back(i);
  }
  for (auto& C : cls) {
    for (int i : C.plans) {
      VarDev& d = *ds[i];
      cudaError_t e = var_dispatch(d, [&](auto R) -> cudaError_t {
        using Run = decltype(R);
        auto put = [](std::vector<unsigned char>& v, const void* p, size_t b) {
          v.insert(v.end(), static_cast<const unsigned char*>(p), static_cast<const unsigned char*>(p) + b);
        };
        if (bf16) {
          const auto A = Run::template sweep_args<__nv_bfloat16>(d);
          put(C.sw, &A, sizeof(A));
          VInnerArgs<__nv_bfloat16> I;
          cudaError_t r = mixed ? Run::template inner_args<__nv_bfloat16>(d, &I, &C.smem) : cudaSuccess;
          if (r != cudaSuccess) return r;
          put(C.in, &I, sizeof(I));
          C.ioff.push_back(C.ioff.back() + (mixed ? I.nblk : 0));
        } else {
          const auto A = Run::template sweep_args<float>(d);
          put(C.sw, &A, sizeof(A));
          VInnerArgs<float> I;
          cudaError_t r = mixed ? Run::template inner_args<float>(d, &I, &C.smem) : cudaSuccess;
          if (r != cudaSuccess) return r;
          put(C.in, &I, sizeof(I));
          C.ioff.push_back(C.ioff.back() + (mixed ? I.nblk : 0));
        }
        C.soff.push_back(C.soff.back() + d.grid);
        return cudaSuccess;
      });
      if (!ck(e, "grouped launch set-up")) return IHDG_ERR_CUDA;
    }
  }
  size_t at = 0;
  auto take = [&](size_t b) { size_t r = at; at += (b + 255) & ~size_t(255); return r; };
  for (auto& C : cls) {
    C.o_sw = take(C.sw.size());
    C.o_in = take(C.in.size());
    C.o_soff = take(C.soff.size() * sizeof(int));
    C.o_ioff = take(C.ioff.size() * sizeof(int));
  }
  if (!ck(cudaMalloc(&rs.dbuf, at), "grouped launch descriptors")) return IHDG_ERR_CUDA;
  char* db = static_cast<char*>(rs.dbuf);
  for (auto& C : cls) {
    if (!ck(cudaMemcpy(db + C.o_sw, C.sw.data(), C.sw.size(), cudaMemcpyHostToDevice), "descriptors") ||
        !ck(cudaMemcpy(db + C.o_in, C.in.data(), C.in.size(), cudaMemcpyHostToDevice), "descriptors") ||
        !ck(cudaMemcpy(db + C.o_soff, C.soff.data(), C.soff.size() * sizeof(int), cudaMemcpyHostToDevice), "descriptors") ||
        !ck(cudaMemcpy(db + C.o_ioff, C.ioff.data(), C.ioff.size() * sizeof(int), cudaMemcpyHostToDevice), "descriptors"))
      return IHDG_ERR_CUDA;
  }
  // loop state and forcing of every plan
  int launches = 0;
  if (!ck(cudaEventRecord(rs.a, s), "event")) return IHDG_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    VarDev& d = *ds[i];
    LaunchArgs la{};
    la.ctrl = d.ctrl;
    la.stream = s;
    const int max_iters = std::min(o.max_iters, d.max_hist);
    if (!ck(launch_ctrl_init(la, o.tol, o.diverge_factor, max_iters, o.inner_max, inner_rtol, wait_cycles, -1), "ctrl init") ||
        !ck(var_dispatch(d, [&](auto R) { return decltype(R)::forcing(d, f[i], gb[i], nullptr, s); }), "forcing kernel"))
      return IHDG_ERR_CUDA;
    launches += 2;
  }
  auto readback = [&](const char* where) {
    for (int i = 0; i < n; ++i)
      if (!ck(cudaMemcpyAsync(rs.hc + i, ds[i]->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s), where)) return false;
    return ck(cudaStreamSynchronize(s), where);
  };
  auto all_done = [&]() {
    for (int i = 0; i < n; ++i)
      if (!rs.hc[i].done) return false;
    return true;
  };
  auto launch_all = [&](int which) -> bool {   // 0 float64 sweep, 1 outer sweep, 2 inner sweep
    for (auto& C : cls) {
      VarDev& d0 = *ds[C.plans[0]];
      const int np = (int)C.plans.size();
      cudaError_t e = var_dispatch(d0, [&](auto R) -> cudaError_t {
        using Run = decltype(R);
        if (which < 2)
          return bf16 ? Run::template sweep_group<__nv_bfloat16>(db + C.o_sw, (const int*)(db + C.o_soff), np, C.soff.back(), which, s)
                      : Run::template sweep_group<float>(db + C.o_sw, (const int*)(db + C.o_soff), np, C.soff.back(), which, s);
        return bf16 ? Run::template inner_group<__nv_bfloat16>(db + C.o_in, (const int*)(db + C.o_ioff), np, C.ioff.back(), C.smem, s)
                    : Run::template inner_group<float>(db + C.o_in, (const int*)(db + C.o_ioff), np, C.ioff.back(), C.smem, s);
      });
      if (!ck(e, which == 2 ? "grouped inner sweep" : "grouped sweep")) return false;
      ++launches;
    }
    return true;
  };
  if (!mixed) {
    int batch = 2;
    for (;;) {
      if (!readback("grouped sweep loop")) return IHDG_ERR_CUDA;
      if (all_done()) break;
      for (int i = 0; i < batch; ++i)
        if (!launch_all(0)) return IHDG_ERR_CUDA;
      if (batch < 32) batch *= 2;
    }
  } else {
    int batch = 4;
    for (;;) {
      if (!launch_all(1)) return IHDG_ERR_CUDA;   // plans whose inner loop has stopped (or first)
      for (int i = 0; i < batch; ++i)
        if (!launch_all(2)) return IHDG_ERR_CUDA;
      if (!readback("grouped mixed loop")) return IHDG_ERR_CUDA;
      for (int i = 0; i < n; ++i)
        if (rs.hc[i].timeout) {
          err = "inner sweep: an operator copy into shared memory did not complete in time";
          return IHDG_ERR_TIMEOUT;
        }
      if (all_done()) break;
      if (batch < 64) batch *= 2;
    }
  }
  for (int i = 0; i < n; ++i) {
    VarDev& d = *ds[i];
    const Ctrl& hc = rs.hc[i];
    const double* uf = mixed ? d.u[hc.outer & 1] : d.u[hc.iter & 1];
    const long long nS = d.nel * d.nb;
    k_var_output<<<(unsigned)std::min<long long>((nS + 255) / 256, 4096), 256, 0, s>>>(nS, uf, mixed ? d.r64 : nullptr,
                                                                                         u_out[i]);
    if (!ck(cudaGetLastError(), "output kernel")) return IHDG_ERR_CUDA;
    ++launches;
    if (tr_out[i]) {
      if (!ck(var_dispatch(d, [&](auto R) { return decltype(R)::trace(d, u_out[i], gb[i], tr_out[i], s); }), "trace kernel"))
        return IHDG_ERR_CUDA;
      ++launches;
    }
  }
  if (!ck(cudaEventRecord(rs.b, s), "event") || !readback("grouped solve")) return IHDG_ERR_CUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, rs.a, rs.b);
  for (int i = 0; i < n; ++i) {
    ihdg_result& r = res[i];
    std::memset(&r, 0, sizeof(r));
    r.iterations = rs.hc[i].iter;
    r.fp64_sweeps = rs.hc[i].fp64_sweeps;
    r.lowp_sweeps = rs.hc[i].lowp_sweeps;
    r.residual = rs.hc[i].res;
    r.status = (ihdg_status)rs.hc[i].status;
    r.solve_ms = ms;
    r.kernel_launches = launches;
  }
  return IHDG_OK;
}

}  // namespace ihdg
