// CUDA-core kernels of the mixed-precision loop (outer float64 sweep, residual check, the
// persistent inner kernels) and their per-shape dispatch, included by one translation unit
// per low-precision element type (ihdg_mixed_f32.cu, ihdg_mixed_bf16.cu) so that they
// compile in parallel; the loop itself is in ihdg_mixed.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
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

// gather from a low-precision array, widening to TA (through L2, see ldcg_f)
template <int NF, int NLF, typename TL, typename TA, typename Out>
__device__ __forceinline__ void gather_lp(const DevGeo& g, const TL* __restrict__ E, long long K, const int* c, Out&& put) {
#pragma unroll
  for (int f = 0; f < NLF; ++f) {
    const int kind = g.kind[f];
    const bool bnd = on_bnd(g, c, f);
    const bool need_own = kind == FK_OWN_D || kind == FK_SUM_D;
    const bool need_nb = (kind == FK_NBR_D || kind == FK_SUM_D) && !bnd;
    // unconditional loads from in-bounds stand-ins, combined by selects (as gather())
    const TL* own = E + (long long)(need_own ? g.own_off[f] : 0) * g.ld + K;
    const TL* nb = need_nb ? E + (long long)g.nbr_off[f] * g.ld + nbr_of(g, K, f) : own;
    TA o[NF], n[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) {
      o[j] = (TA)ldcg_f(own + (long long)j * g.ld);
      n[j] = (TA)ldcg_f(nb + (long long)j * g.ld);
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

constexpr int CH = 8;   // outputs per chunk: their loads are issued together, then stored

// Outer float64 sweep: E' = E + e (own and gathered), r = F + L_E t(E') - E'.
template <int NF, int NLF, typename TL>
__global__ void __launch_bounds__(BS) k_outer64(DevGeo g, OpsDev op, const double* __restrict__ F, double* E64,
                                                long long es, double* __restrict__ r64, TL* __restrict__ rlp,
                                                const TL* e0, const TL* e1, int has_e, Ctrl* ctrl, double* partials) {
  constexpr int NIN = NF * NLF;
  __shared__ double ws[BS / 32];
  extern __shared__ double sdyn[];
  if (ctrl_done(ctrl)) return;
  const int o = *(volatile const int*)&ctrl->outer;
  const int j = *(volatile const int*)&ctrl->inner_iter;
  double* sLE = sdyn;
  double* st = sLE + g.n_exp * NIN + threadIdx.x;
  for (int i = threadIdx.x; i < g.n_exp * NIN; i += BS) sLE[i] = op.LE[i];
  __syncthreads();
  const double* Ecur = E64 + (long long)(o & 1) * es;
  double* Enx = E64 + (long long)((o + 1) & 1) * es;
  const TL* ecur = (j & 1) ? e1 : e0;
  const long long K = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (K < g.nel) {
    int c[3];
    coords(g, K, c);
    gather<NF, NLF, double, double>(g, Ecur, K, c, [&](int s, double v) { st[s * BS] = v; });
    if (has_e) gather_lp<NF, NLF, TL, double>(g, ecur, K, c, [&](int s, double v) { st[s * BS] += v; });
#pragma unroll
    for (int c0 = 0; c0 < NIN; c0 += CH) {
      double own[CH], fv[CH];
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int e = c0 + i;
        own[i] = 0.0;
        fv[i] = 0.0;
        if (e < g.n_exp && row_live(g, e, NF)) {
          const long long at = (long long)e * g.ld + K;
          own[i] = Ecur[at] + (has_e ? (double)to_f(ecur[at]) : 0.0);
          fv[i] = F[at];
        }
      }
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int e = c0 + i;
        if (e < g.n_exp && row_live(g, e, NF)) {
          const long long at = (long long)e * g.ld + K;
          double v = fv[i];
          const double* row = sLE + e * NIN;
#pragma unroll
          for (int s = 0; s < NIN; ++s) v += row[s] * st[s * BS];
          const double r = v - own[i];
          Enx[at] = own[i];
          r64[at] = r;
          rlp[at] = from_f<TL>((float)r);
          acc += r * r;
        }
      }
    }
  }
  double tot;
  if (arrive(ctrl, partials, acc, ws, &tot) && threadIdx.x == 0) {
    ctrl->rnorm = sqrt(tot);
    ctrl->outer = o + 1;
    ctrl->iter += 1;
    ctrl->fp64_sweeps += 1;
  }
}

// Float64 stopping residual of the next exact sweep, sqrt(t(r)^T Q t(r)), fused with the
// first useful inner sweep e = r + L_E t(r) (low precision).
template <int NF, int NLF, typename TL>
__global__ void __launch_bounds__(BS) k_inner_first(DevGeo g, OpsDev op, const double* __restrict__ r64,
                                                    TL* __restrict__ e0, Ctrl* ctrl, double* partials,
                                                    double* res_hist) {
  constexpr int NIN = NF * NLF;
  constexpr int NQ = NIN * (NIN + 1) / 2;
  __shared__ double ws[BS / 32];
  extern __shared__ double sdyn[];
  if (ctrl_done(ctrl)) return;
  double* sQ = sdyn;
  float* sL = reinterpret_cast<float*>(sQ + NQ);
  for (int i = threadIdx.x; i < NQ; i += BS) sQ[i] = op.Qp[i];
  for (int i = threadIdx.x; i < g.n_exp * NIN; i += BS) sL[i] = op.LE32[i];
  __syncthreads();
  const long long K = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (K < g.nel) {
    int c[3];
    coords(g, K, c);
    double d[NIN];
    gather<NF, NLF, double, double>(g, r64, K, c, [&](int s, double v) { d[s] = v; });
    int q = 0;
#pragma unroll
    for (int s = 0; s < NIN; ++s) {
      double r = 0.0;
#pragma unroll
      for (int u = s; u < NIN; ++u) r += sQ[q + u - s] * d[u];
      q += NIN - s;
      acc += d[s] * r;
    }
    float df[NIN];
#pragma unroll
    for (int s = 0; s < NIN; ++s) df[s] = (float)d[s];
#pragma unroll
    for (int c0 = 0; c0 < NIN; c0 += CH) {
      float rv[CH];
#pragma unroll
      for (int i = 0; i < CH; ++i) rv[i] = (c0 + i < g.n_exp && row_live(g, c0 + i, NF)) ? (float)r64[(long long)(c0 + i) * g.ld + K] : 0.f;
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int e = c0 + i;
        if (e < g.n_exp && row_live(g, e, NF)) {
          float v = rv[i];
          const float* row = sL + e * NIN;
#pragma unroll
          for (int s = 0; s < NIN; ++s) v = fmaf(row[s], df[s], v);
          e0[(long long)e * g.ld + K] = from_f<TL>(v);
        }
      }
    }
  }
  double tot;
  if (arrive(ctrl, partials, acc, ws, &tot) && threadIdx.x == 0) {
    decide(ctrl, tot, res_hist, false);
    ctrl->inner_iter = 0;
    ctrl->inner_done = 0;
  }
}

// Grid barrier plus sum of one double per block, for cooperative launches.  The arrival
// counter only grows (cleared before the launch): barrier number b completes when it
// reaches (b+1) * gridDim.x.  Thread 0 publishes the block's partial, arrives with a
// release add and polls with acquire loads (bounded by ~1 s of SM clock, then
// ctrl->timeout); warp 0 then sums the partials in block order with a fixed shuffle tree,
// so every block obtains the same total.
template <int NT>
__device__ double barrier_sum(double* part, unsigned* count, unsigned nb, double mine, Ctrl* ctrl, double* s_out,
                              int* s_flag) {
  // GB300's float64 rate is a small fraction of float32: every per-thread step here is
  // float32, and only thread 0 touches float64 (the published partial and the final sum)
  __shared__ float wred[NT / 32];
  __syncthreads();
  if (threadIdx.x == 0) {
    part[blockIdx.x] = mine;
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
  // every thread loads its share of the partials at once (one round trip), then a fixed tree
  float v = 0.f;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) v += (float)__ldcg(part + i);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += (double)wred[w];
    *s_out = t;
  }
  __syncthreads();
  return *s_out;
}


// Low-precision operator passed by value: the kernel reads it from the parameter (constant)
// bank, so every multiply-add takes its matrix entry straight from there.
template <int NF, int NLF, bool PER_AXIS>
struct LTile {
  static constexpr int NIN = NF * NLF;
  static constexpr int NEXP = PER_AXIS ? NF * (NLF / 2) : NF * NLF;
  float L[NEXP][NIN];
};

// Persistent inner loop on the correction equation with the state in global memory (meshes
// whose state fits neither registers nor shared memory): e_{j+1} = r + L_E t(e_j), until the
// step norm falls below inner_rtol * ||r||, inner_max sweeps, or the sweep budget.  One
// element per thread and grid-stride pass, software-pipelined: all loads of the next element
// (its own exports, also the reference of the step norm; the neighbours' facing exports, an
// in-bounds stand-in where none is read; r) are issued before the current element's operator
// apply, so every warp keeps its next element's bytes in flight while it computes (operators
// of up to 20 trace values; larger ones load and compute one element at a time).  Element
// coordinates advance by the grid stride written as mixed-radix digits (no division per
// element); ALL: every export slot carries a value (no per-slot tests).  The operator comes
// from the parameter bank, one accumulation chain per row.  Each sweep ends with a grid
// barrier after which every block sums the per-block partials in the same fixed order, so all
// blocks take the same decision; block 0 records the loop state.
template <int NF, int NLF, bool PER_AXIS, bool ALL, typename TL>
__global__ void __launch_bounds__(PBS, NF * NLF <= 20 ? 2 : 1)
    k_inner_persist(const DevGeo g, const TL* __restrict__ rlp, TL* e0, TL* e1, Ctrl* ctrl, double* partials,
                    const LTile<NF, NLF, PER_AXIS> Lp) {
  constexpr int NIN = NF * NLF;
  constexpr int NEXP = LTile<NF, NLF, PER_AXIS>::NEXP;
  constexpr bool PIPE = NIN <= 20;   // the next element's loads fit beside the current element's values
  __shared__ double s_tot;
  __shared__ int s_to, s_stop;
  __shared__ float wsum_p[PBS / 32];
  if (ctrl_done(ctrl) || *(volatile const int*)&ctrl->inner_done) return;
  int j = *(volatile const int*)&ctrl->inner_iter;
  const int iter0 = *(volatile const int*)&ctrl->iter;
  const int lowp0 = *(volatile const int*)&ctrl->lowp_sweeps;
  const int max_iters = ctrl->max_iters, inner_max = ctrl->inner_max;
  const double lim = ctrl->inner_rtol * ctrl->rnorm;
  const long long stride = (long long)gridDim.x * PBS, ld = g.ld, nel = g.nel;
  const long long Kfirst = (long long)blockIdx.x * PBS + threadIdx.x;
  int cfirst[3], ds[3];
  coords(g, Kfirst, cfirst);
  coords(g, stride, ds);   // the stride as digits (ds[0] < n0, ds[1] < n1)
  auto live = [&](int e) { return ALL || ((g.live >> e) & 1ull); };
  for (int s = 0;; ++s) {
    const TL* __restrict__ ec = (j & 1) ? e1 : e0;
    TL* __restrict__ en = (j & 1) ? e0 : e1;
    float acc = 0.f;
    float ov[NEXP], rv[NEXP], nv[NLF][NF];
    // all loads of element K at coordinates c (a thread past the end loads nothing)
    auto fetch = [&](long long K, const int* c) {
      const bool in = K < nel;
      const long long Ks = in ? K : 0;
#pragma unroll
      for (int e = 0; e < NEXP; ++e) {
        ov[e] = (in && live(e)) ? ldcg_f(ec + e * ld + Ks) : 0.f;
        rv[e] = (in && live(e)) ? to_f(rlp[e * ld + Ks]) : 0.f;
      }
#pragma unroll
      for (int f = 0; f < NLF; ++f) {
        const int kind = g.kind[f];
        const bool nbm = in && !on_bnd(g, c, f) && (kind == FK_NBR_D || kind == FK_SUM_D);
        const int ns = PER_AXIS ? (f >> 1) * NF : (f ^ 1) * NF;
        const TL* nb = ec + (long long)ns * ld + (nbm ? nbr_of(g, Ks, f) : Ks);
#pragma unroll
        for (int q = 0; q < NF; ++q) nv[f][q] = ldcg_f(nb + q * ld);
      }
    };
    long long K = Kfirst;
    int c[3] = {cfirst[0], cfirst[1], cfirst[2]};
    if (PIPE) fetch(K, c);
    while (K < nel) {
      if (!PIPE) fetch(K, c);
      // a1: this element's traces; its exports and r stay for the rows
      float t[NIN], oc[NEXP], rc[NEXP];
#pragma unroll
      for (int f = 0; f < NLF; ++f) {
        const int kind = g.kind[f];
        const bool bnd = on_bnd(g, c, f);
        const bool nbm = !bnd && (kind == FK_NBR_D || kind == FK_SUM_D);
        const float wo = kind == FK_OWN_D ? 1.f : kind == FK_SUM_D ? (!bnd ? 1.f : (g.bc_mirror ? 2.f : 0.f)) : 0.f;
        const int os = PER_AXIS ? (f >> 1) * NF : f * NF;
#pragma unroll
        for (int q = 0; q < NF; ++q) t[f * NF + q] = wo * ov[os + q] + (nbm ? nv[f][q] : 0.f);
      }
#pragma unroll
      for (int e = 0; e < NEXP; ++e) {
        oc[e] = ov[e];
        rc[e] = rv[e];
      }
      const long long Kc = K;
      // the next element: coordinates by digit addition with carries, then its loads
      K += stride;
      c[0] += ds[0];
      int cy = c[0] >= g.n[0];
      if (cy) c[0] -= g.n[0];
      c[1] += ds[1] + cy;
      cy = c[1] >= g.n[1];
      if (cy) c[1] -= g.n[1];
      c[2] += ds[2] + cy;
      if (PIPE) fetch(K, c);
      // a3 + a4: e_new = r + L_E t, rounded to the storage type; the step norm
#pragma unroll
      for (int e = 0; e < NEXP; ++e) {
        if (!live(e)) continue;
        float v = rc[e];
#pragma unroll
        for (int k = 0; k < NIN; ++k) v = fmaf(Lp.L[e][k], t[k], v);
        const TL nt = from_f<TL>(v);
        const float dl = to_f(nt) - oc[e];
        acc = fmaf(dl, dl, acc);
        en[e * ld + Kc] = nt;
      }
    }
    const int it = iter0 + s + 1;
    float bsf = acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bsf += __shfl_down_sync(0xffffffffu, bsf, o);
    if ((threadIdx.x & 31) == 0) wsum_p[threadIdx.x >> 5] = bsf;
    __syncthreads();
    double bs = 0.0;
    if (threadIdx.x == 0)
      for (int w = 0; w < PBS / 32; ++w) bs += (double)wsum_p[w];
    const double tot = barrier_sum<PBS>(partials + (size_t)(s & 1) * gridDim.x, &ctrl->bar_count, (unsigned)(s + 1), bs,
                                        ctrl, &s_tot, &s_to);
    if (s_to) break;
    j += 1;
    if (threadIdx.x == 0) {
      const double step = sqrt(tot);
      const bool stop = step <= lim || j >= inner_max || it >= max_iters || !(step == step) || isinf(step);
      s_stop = stop ? 1 : 0;
      if (blockIdx.x == 0) {
        ctrl->inner_iter = j;
        ctrl->iter = it;
        ctrl->lowp_sweeps = lowp0 + s + 1;
        ctrl->inner_step = step;
        if (stop) ctrl->inner_done = 1;
      }
    }
    __syncthreads();
    if (s_stop) break;
  }
}

// Persistent inner loop with block-resident state.  Block b owns elements
// [b*epb, b*epb + epb); their own exports e_j and the residual r stay in shared memory
// (TL precision: the values the neighbours see), with each element's boundary-face mask.
// LPE lanes of a warp share one element: lane l gathers the traces of the faces
// f = l, l + LPE, ... (own exports from shared memory, the neighbour's from global memory),
// the lanes exchange them by shuffles, and lane l computes the export rows of its faces
// (per-face layout) or axes (per-axis layout), reading the operator from the parameter
// bank.  Per sweep only neighbours' exports cross global memory; the loop decision is the
// same as k_inner_persist's.
template <int NF, int NLF, bool PER_AXIS, typename TL, int NT, int LPE>
__global__ void __launch_bounds__(NT) k_inner_tile(const DevGeo g, const TL* __restrict__ rlp, TL* e0, TL* e1,
                                                   Ctrl* ctrl, double* partials, const int epb,
                                                   const LTile<NF, NLF, PER_AXIS> Lp) {
  constexpr int NIN = NF * NLF;
  constexpr int NEXP = LTile<NF, NLF, PER_AXIS>::NEXP;
  constexpr int FPL = NLF / LPE;                    // faces per lane
  constexpr int NBLK = PER_AXIS ? NLF / 2 : NLF;    // export row blocks (axes or faces)
  constexpr int EPP = NT / LPE;                     // elements per pass
  static_assert(NLF % LPE == 0 && 32 % LPE == 0, "lanes per element must divide faces and warps");
  __shared__ double s_tot;
  __shared__ int s_to, s_stop;
  extern __shared__ __align__(16) unsigned char smraw[];
  if (ctrl_done(ctrl) || *(volatile const int*)&ctrl->inner_done) return;
  int j = *(volatile const int*)&ctrl->inner_iter;
  const int iter0 = *(volatile const int*)&ctrl->iter;
  const int lowp0 = *(volatile const int*)&ctrl->lowp_sweeps;
  const int max_iters = ctrl->max_iters, inner_max = ctrl->inner_max;
  const double lim = ctrl->inner_rtol * ctrl->rnorm;
  TL* ev = reinterpret_cast<TL*>(smraw);        // [NEXP][epb]
  TL* rv = ev + (size_t)NEXP * epb;             // [NEXP][epb]
  unsigned char* bm = reinterpret_cast<unsigned char*>(rv + (size_t)NEXP * epb);
  const int ld = (int)g.ld;
  const int K0 = blockIdx.x * epb;
  const int cnt = min(epb, (int)g.nel - K0);
  unsigned* count = &ctrl->bar_count;
  {
    const TL* ec = (j & 1) ? e1 : e0;
    for (int le = threadIdx.x; le < cnt; le += NT) {
      const int K = K0 + le;
      int c[3];
      coords(g, K, c);
      unsigned m = 0;
#pragma unroll
      for (int f = 0; f < NLF; ++f) m |= (on_bnd(g, c, f) ? 1u : 0u) << f;
      bm[le] = (unsigned char)m;
#pragma unroll
      for (int e = 0; e < NEXP; ++e) {
        ev[e * epb + le] = ((g.live >> e) & 1ull) ? ec[e * ld + K] : from_f<TL>(0.f);
        rv[e * epb + le] = ((g.live >> e) & 1ull) ? rlp[e * ld + K] : from_f<TL>(0.f);
      }
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & (LPE - 1);
  const int wl = threadIdx.x & 31;
  const int gbase = wl & ~(LPE - 1);
  const int npass = (cnt + EPP - 1) / EPP;
  for (int s = 0;; ++s) {
    const TL* __restrict__ ec = (j & 1) ? e1 : e0;
    TL* __restrict__ en = (j & 1) ? e0 : e1;
    float acc = 0.f;
    for (int pass = 0; pass < npass; ++pass) {
      const int le = pass * EPP + threadIdx.x / LPE;
      const bool valid = le < cnt;
      const int K = K0 + le;
      const unsigned m = valid ? bm[le] : 0u;
      // a1: this lane's faces.  The neighbours' exports are read with unconditional loads
      // (an in-bounds index where nothing is needed), so all of them are in flight at once.
      float lt[FPL][NF];
      int nbi[FPL];
      bool nbm[FPL];
      float wo[FPL];
#pragma unroll
      for (int i = 0; i < FPL; ++i) {
        const int f = i * LPE + lane;                 // runtime face of this lane
        const int kind = g.kind[f];
        const bool bnd = (m >> f) & 1u;
        const int a = f >> 1;
        const int ns = PER_AXIS ? a * NF : (f ^ 1) * NF;
        const int Kn = K + ((f & 1) ? (int)g.stride[a] : -(int)g.stride[a]);
        nbm[i] = valid && !bnd && (kind == FK_NBR_D || kind == FK_SUM_D);
        nbi[i] = nbm[i] ? ns * ld + Kn : ns * ld + K0;
        wo[i] = !valid ? 0.f
                : kind == FK_OWN_D ? 1.f
                : kind == FK_SUM_D ? (!bnd ? 1.f : (g.bc_mirror ? 2.f : 0.f)) : 0.f;
      }
#pragma unroll
      for (int i = 0; i < FPL; ++i)
#pragma unroll
        for (int q = 0; q < NF; ++q) lt[i][q] = to_f(ec[nbi[i] + q * ld]);
      const int lc = valid ? le : 0;
#pragma unroll
      for (int i = 0; i < FPL; ++i) {
        const int f = i * LPE + lane;
        const int os = PER_AXIS ? (f >> 1) * NF : f * NF;
#pragma unroll
        for (int q = 0; q < NF; ++q)
          lt[i][q] = wo[i] * to_f(ev[(os + q) * epb + lc]) + (nbm[i] ? lt[i][q] : 0.f);
      }
      // exchange: every lane of the element obtains all NIN traces
      float t[NIN];
#pragma unroll
      for (int f = 0; f < NLF; ++f)
#pragma unroll
        for (int q = 0; q < NF; ++q) {
          if constexpr (LPE == 1) t[f * NF + q] = lt[f][q];
          else t[f * NF + q] = __shfl_sync(0xffffffffu, lt[f / LPE][q], gbase + (f % LPE));
        }
      if constexpr (LPE > 1) __syncwarp();
      // a3/a4: this lane's export rows
      if (valid) {
#pragma unroll
        for (int rb = 0; rb < NBLK; ++rb) {
          if (LPE > 1 && rb % LPE != lane) continue;
#pragma unroll
          for (int q = 0; q < NF; ++q) {
            const int e = rb * NF + q;
            float v = to_f(rv[e * epb + le]);
#pragma unroll
            for (int k = 0; k < NIN; ++k) v = fmaf(Lp.L[e][k], t[k], v);
            const TL nv = from_f<TL>(v);
            const float d = to_f(nv) - to_f(ev[e * epb + le]);
            acc = fmaf(d, d, acc);
            ev[e * epb + le] = nv;
            if ((g.live >> e) & 1ull) en[e * ld + K] = nv;
          }
        }
      }
      if constexpr (LPE > 1) __syncwarp();
    }
    const int it = iter0 + s + 1;
    float bs = acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bs += __shfl_down_sync(0xffffffffu, bs, o);
    __shared__ float wsum[NT / 32];
    if (wl == 0) wsum[threadIdx.x >> 5] = bs;
    __syncthreads();
    double blk = 0.0;
    if (threadIdx.x == 0)
      for (int w = 0; w < NT / 32; ++w) blk += (double)wsum[w];
    const double tot = barrier_sum<NT>(partials + (size_t)(s & 1) * gridDim.x, count, (unsigned)(s + 1), blk, ctrl, &s_tot, &s_to);
    if (s_to) break;
    j += 1;
    if (threadIdx.x == 0) {
      const double step = sqrt(tot);
      const bool stop = step <= lim || j >= inner_max || it >= max_iters || !(step == step) || isinf(step);
      s_stop = stop ? 1 : 0;
      if (blockIdx.x == 0) {
        ctrl->inner_iter = j;
        ctrl->iter = it;
        ctrl->lowp_sweeps = lowp0 + s + 1;
        ctrl->inner_step = step;
        if (stop) ctrl->inner_done = 1;
      }
    }
    __syncthreads();
    if (s_stop) break;
  }
}

// Launch the tile kernel when its block state fits in shared memory; returns
// cudaErrorNotSupported (nothing launched) otherwise.
template <int NF, int NLF, bool PER_AXIS, typename TL, int NT, int LPE>
cudaError_t launch_tile_v(MixedArgs& m, TL* rl, TL* e0, TL* e1) {
  using LT = LTile<NF, NLF, PER_AXIS>;
  const LaunchArgs& a = m.base;
  if (!m.LE32h || a.g.n_exp != LT::NEXP || (long long)a.g.ld * LT::NEXP >= (1LL << 31)) return cudaErrorNotSupported;
  auto k = k_inner_tile<NF, NLF, PER_AXIS, TL, NT, LPE>;
  int dev = 0, sms = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  smem_max -= 1024;   // static shared memory of the kernel
  const long long nel = a.g.nel;
  for (int bps = 2; bps >= 1; --bps) {
    long long grid = (long long)bps * sms;
    const long long cap = (nel + 63) / 64;          // at least 64 elements per block
    if (grid > cap) grid = cap;
    if (grid > m.max_grid) grid = m.max_grid;
    if (grid < 1) grid = 1;
    const long long epb = (nel + grid - 1) / grid;
    grid = (nel + epb - 1) / epb;
    if (grid > m.slots / 2) continue;
    const size_t smem = (size_t)epb * (2 * LT::NEXP * sizeof(TL) + 1) + 16;
    if (smem > (size_t)smem_max) continue;
    cudaError_t e = allow_dynamic_smem(k);
    if (e != cudaSuccess) return e;
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, NT, smem);
    if (e != cudaSuccess) return e;
    if ((long long)per * sms < grid) continue;
    LT L;
    for (int r = 0; r < LT::NEXP; ++r)
      for (int q = 0; q < LT::NIN; ++q) L.L[r][q] = m.LE32h[r * LT::NIN + q];
    DevGeo gg = a.g;
    const TL* rlc = rl;
    Ctrl* ct = a.ctrl;
    double* pp = a.partials;
    int ep = (int)epb;
    e = cudaMemsetAsync(&a.ctrl->bar_count, 0, sizeof(unsigned), a.stream);
    if (e != cudaSuccess) return e;
    void* args[] = {&gg, &rlc, &e0, &e1, &ct, &pp, &ep, &L};
    e = cudaLaunchCooperativeKernel((const void*)k, dim3((unsigned)grid), dim3(NT), args, smem, a.stream);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  return cudaErrorNotSupported;
}

// Persistent inner loop for 2D meshes with register-resident state: LPE lanes per element
// (2 or 4); lane l owns the faces f = l, l + LPE.  For each of its faces a lane keeps in
// registers the exports of that face (per-face layout) or of the face's axis when the face is
// the axis' outflow face (per-axis layout), and the matching residual values; it gathers its
// faces' traces (own registers + the neighbour's exports from global memory), broadcasts them
// to the element's other lanes by shuffles, and accumulates its rows as the traces arrive.
// The operator sits in shared memory transposed and padded, LT[k][rowblock * RW + r], so one
// 128-bit load gives a lane the coefficients of trace k for 4 rows of one block.  Every thread
// owns one (element, lane) pair for the whole launch.
template <int NF, bool PER_AXIS, typename TL, int LPE, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_inner_reg(const DevGeo g, const TL* __restrict__ rlp, TL* e0,
                                                             TL* e1, Ctrl* ctrl, double* partials,
                                                             const float* __restrict__ LTg, const int epb) {
  constexpr int NIN = 4 * NF, FPL = 4 / LPE;
  constexpr int RW = (NF + 3) & ~3;          // padded row-block width
  constexpr int NRB = 4;                     // row blocks stored (faces; axes use the first 2)
  __shared__ __align__(16) float LT[NIN * NRB * RW];
  __shared__ float wsum[NT / 32], wdec[NT / 32];
  __shared__ int s_to;
  if (ctrl_done(ctrl) || *(volatile const int*)&ctrl->inner_done) return;
  int j = *(volatile const int*)&ctrl->inner_iter;
  const int iter0 = *(volatile const int*)&ctrl->iter;
  const int lowp0 = *(volatile const int*)&ctrl->lowp_sweeps;
  const int max_iters = ctrl->max_iters, inner_max = ctrl->inner_max;
  const double lim = ctrl->inner_rtol * ctrl->rnorm;
  for (int i = threadIdx.x; i < NIN * NRB * RW; i += NT) LT[i] = LTg[i];
  const int lane = threadIdx.x % LPE;
  const int gbase = (threadIdx.x & 31) - lane;
  const int K = blockIdx.x * epb + threadIdx.x / LPE;   // epb <= NT / LPE elements per block
  const bool valid = (int)(threadIdx.x / LPE) < epb && K < (int)g.nel;
  const int ld = (int)g.ld;
  int c[3] = {0, 0, 0};
  if (valid) coords(g, K, c);
  // per face of this lane: where the neighbour's exports sit (nbi, an in-bounds index also
  // where nothing is read, so that every sweep's gathers are unconditional loads) and how
  // the trace combines own (wo) and neighbour (wn) values
  int kind[FPL], nbi[FPL], row0[FPL];
  bool rows[FPL], nbm[FPL];
  float wo[FPL];
#pragma unroll
  for (int i = 0; i < FPL; ++i) {
    const int f = lane + LPE * i, a = f >> 1;
    kind[i] = g.kind[f];
    const bool bnd = valid && on_bnd(g, c, f);
    const int Kn = K + ((f & 1) ? (int)g.stride[a] : -(int)g.stride[a]);
    const int ns = PER_AXIS ? a * NF : (f ^ 1) * NF;
    row0[i] = PER_AXIS ? a * NF : f * NF;
    const bool owns = PER_AXIS ? kind[i] == FK_OWN_D : (kind[i] == FK_SUM_D || kind[i] == FK_OWN_D);
    rows[i] = valid && owns && ((g.live >> row0[i]) & 1ull);
    const bool nb = valid && !bnd && (kind[i] == FK_NBR_D || kind[i] == FK_SUM_D);
    nbi[i] = nb ? ns * ld + Kn : ns * ld + (valid ? K : 0);
    nbm[i] = nb;
    wo[i] = !valid ? 0.f
            : kind[i] == FK_OWN_D ? 1.f
            : kind[i] == FK_SUM_D ? (!bnd ? 1.f : (g.bc_mirror ? 2.f : 0.f)) : 0.f;
  }
  float ev[FPL][NF], rv[FPL][NF];
  {
    const TL* ec = (j & 1) ? e1 : e0;
#pragma unroll
    for (int i = 0; i < FPL; ++i)
#pragma unroll
      for (int r = 0; r < NF; ++r) {
        ev[i][r] = rows[i] ? to_f(ec[(row0[i] + r) * ld + K]) : 0.f;
        rv[i][r] = rows[i] ? to_f(rlp[(row0[i] + r) * ld + K]) : 0.f;
      }
  }
  __syncthreads();
  unsigned* count = &ctrl->bar_count;
  float* partf = reinterpret_cast<float*>(partials);
  const float limf = (float)lim;
  for (int s = 0;; ++s) {
    const TL* __restrict__ ec = ((j + s) & 1) ? e1 : e0;
    TL* __restrict__ en = ((j + s) & 1) ? e0 : e1;
    // previous sweep's partials (one round trip, together with the trace gathers below)
    float pv = 0.f;
    if (s > 0)
      for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) pv += __ldcg(partf + ((s - 1) & 1) * gridDim.x + i);
    float lt[FPL][NF];
#pragma unroll
    for (int i = 0; i < FPL; ++i)
#pragma unroll
      for (int q = 0; q < NF; ++q) lt[i][q] = ldcg_f(ec + nbi[i] + q * ld);
#pragma unroll
    for (int i = 0; i < FPL; ++i)
#pragma unroll
      for (int q = 0; q < NF; ++q) lt[i][q] = wo[i] * ev[i][q] + (nbm[i] ? lt[i][q] : 0.f);   // never 0 * (unread)
    float acc[FPL][RW];
#pragma unroll
    for (int i = 0; i < FPL; ++i)
#pragma unroll
      for (int r = 0; r < RW; ++r) acc[i][r] = r < NF ? rv[i][r] : 0.f;
#pragma unroll
    for (int src = 0; src < LPE; ++src)
#pragma unroll
      for (int is = 0; is < FPL; ++is)
#pragma unroll
        for (int q = 0; q < NF; ++q) {
          const float x = __shfl_sync(0xffffffffu, lt[is][q], gbase + src);
          const int k = (src + LPE * is) * NF + q;        // trace index: face src + LPE*is, node q
#pragma unroll
          for (int i = 0; i < FPL; ++i) {
            const int rbi = row0[i] / NF;
            const float* col = LT + (k * NRB + rbi) * RW;
#pragma unroll
            for (int r4 = 0; r4 < RW; r4 += 4) {
              const float4 cf = *reinterpret_cast<const float4*>(col + r4);
              acc[i][r4 + 0] = fmaf(cf.x, x, acc[i][r4 + 0]);
              acc[i][r4 + 1] = fmaf(cf.y, x, acc[i][r4 + 1]);
              acc[i][r4 + 2] = fmaf(cf.z, x, acc[i][r4 + 2]);
              acc[i][r4 + 3] = fmaf(cf.w, x, acc[i][r4 + 3]);
            }
          }
        }
    // decision on the s sweeps done so far (the last one's step norm when s > 0), taken
    // after the local apply so that the partial sums have arrived.  Every thread folds the
    // warp sums in the same order: all threads of all blocks take the same decision.
    {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
      if ((threadIdx.x & 31) == 0) wdec[threadIdx.x >> 5] = pv;
      __syncthreads();
      float tot = 0.f;
#pragma unroll
      for (int w = 0; w < NT / 32; ++w) tot += wdec[w];
      const float step = sqrtf(tot);
      const bool budget = j + s >= inner_max || iter0 + s >= max_iters;
      const bool stop = budget || (s > 0 && (step <= limf || !(step == step) || isinf(step)));
      if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctrl->inner_iter = j + s;
        ctrl->iter = iter0 + s;
        ctrl->lowp_sweeps = lowp0 + s;
        if (s > 0) ctrl->inner_step = (double)step;
        if (stop) ctrl->inner_done = 1;
      }
      if (stop) break;
    }
    float st = 0.f;
#pragma unroll
    for (int i = 0; i < FPL; ++i) {
      if (!rows[i]) continue;
#pragma unroll
      for (int r = 0; r < NF; ++r) {
        const TL nv = from_f<TL>(acc[i][r]);
        const float nvf = to_f(nv);
        const float d = nvf - ev[i][r];
        st = fmaf(d, d, st);
        ev[i][r] = nvf;
        en[(row0[i] + r) * ld + K] = nv;
      }
    }
    const float blk = sum_partials<NT>(st, wsum);
    arrive_wait(partf + (s & 1) * gridDim.x, count, (unsigned)(s + 1), blk, ctrl, &s_to);
    if (s_to) break;
  }
}

// Launch k_inner_reg with the most lanes per element whose grid is co-resident (NT threads
// per block: 512, two blocks per SM, or 1024, one block per SM and half the barrier arrivals).
template <int NF, bool PER_AXIS, typename TL, int LPE, int NT>
cudaError_t launch_reg_v(MixedArgs& m, TL* rl, TL* e0, TL* e1) {
  constexpr int NIN = 4 * NF, RW = (NF + 3) & ~3, NRB = 4;
  const LaunchArgs& a = m.base;
  if (a.g.dim != 2 || !m.LE32h || !m.dLT || (long long)a.g.ld * a.g.n_exp >= (1LL << 31)) return cudaErrorNotSupported;
  auto k = k_inner_reg<NF, PER_AXIS, TL, LPE, NT>;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, NT, 0);
  if (e != cudaSuccess) return e;
  // the grid is a multiple of the SM count with the elements spread evenly over it
  long long grid = (long long)per * sms;
  const long long small = (a.g.nel + 127) / 128;   // small problems keep >= 128 elements per block
  if (grid > small) grid = small;
  if (grid > m.max_grid) grid = m.max_grid;
  const long long epb = (a.g.nel + grid - 1) / grid;
  if (epb > NT / LPE) return cudaErrorNotSupported;
  grid = (a.g.nel + epb - 1) / epb;
  if (grid > m.slots / 2) return cudaErrorNotSupported;
  // transposed, padded operator: LT[k][rb * RW + r] = L_E[rb * NF + r][k]
  std::vector<float> lt((size_t)NIN * NRB * RW, 0.f);
  const int nrb = a.g.n_exp / NF;
  for (int kk = 0; kk < NIN; ++kk)
    for (int b = 0; b < nrb; ++b)
      for (int r = 0; r < NF; ++r) lt[((size_t)kk * NRB + b) * RW + r] = m.LE32h[(b * NF + r) * NIN + kk];
  if (m.lt_kind != 1) {
    e = cudaMemcpyAsync(m.dLT, lt.data(), lt.size() * sizeof(float), cudaMemcpyHostToDevice, a.stream);
    if (e != cudaSuccess) return e;
    m.lt_kind = 1;
  }
  e = cudaMemsetAsync(&a.ctrl->bar_count, 0, sizeof(unsigned), a.stream);
  if (e != cudaSuccess) return e;
  DevGeo gg = a.g;
  const TL* rlc = rl;
  Ctrl* ct = a.ctrl;
  double* pp = a.partials;
  const float* ltp = m.dLT;
  int ep = (int)epb;
  void* args[] = {&gg, &rlc, &e0, &e1, &ct, &pp, &ltp, &ep};
  e = cudaLaunchCooperativeKernel((const void*)k, dim3((unsigned)grid), dim3(NT), args, 0, a.stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int NF, bool PER_AXIS, typename TL>
cudaError_t launch_reg(MixedArgs& m, TL* rl, TL* e0, TL* e1) {
  cudaError_t e;
  if (m.reg_nt == 1024) {
    e = launch_reg_v<NF, PER_AXIS, TL, 2, 1024>(m, rl, e0, e1);
    if (e != cudaErrorNotSupported) return e;
  }
  e = launch_reg_v<NF, PER_AXIS, TL, 4, 512>(m, rl, e0, e1);
  if (e != cudaErrorNotSupported) return e;
  return launch_reg_v<NF, PER_AXIS, TL, 2, 512>(m, rl, e0, e1);
}

// Temporally blocked inner loop for 2D meshes.  The mesh is cut into tiles (one per block,
// tiles_x across); every block keeps its tile plus a halo of H elements on each side (clipped
// at the mesh boundary) in shared memory: the current and next correction e (TL values held
// as float, so every value is exactly what the element-per-sweep kernels store) and the
// residual r.  One super-step runs h <= H sweeps of e <- r + L_E t(e) without leaving the SM:
// sweep t updates the tile grown by H - t elements, whose inputs all lie in the area that
// sweep t-1 updated, so after h sweeps the tile holds exactly the iterate the plain sweep
// reaches after h sweeps.  The block then stores the elements within H of its tile's edges
// (its neighbours' halo) into the global buffer of the next super-step and arrives at the
// grid barrier; at the top of the next super-step it reloads its halo from that buffer.
// One grid barrier and one L2 round trip thus serve h sweeps, at the price of recomputing
// the halo (the redundant work grows with H).  The stopping test is the one of the other
// inner kernels, taken on the step norm of the last sweep of each super-step (tile elements
// only, so every element counts once), lagged by one super-step; on stopping, each block
// stores its whole tile into the buffer the outer sweep reads for that sweep count.
struct BlkShape {
  int tiles_x, tx, ty, halo, ra_max;   // ra_max: largest (pitch x rows) of a region, shared-memory sizing
};

// Row pitch (elements) of a region row in shared memory: the smallest value >= width that is
// 8 or 24 modulo 32, so that the 8 x 4 element patch of a warp (and the patch moved by one
// element or one row) falls on 32 distinct banks.
__host__ __device__ __forceinline__ int blk_pitch(int width) {
  const int r = width & 31;
  return width + (r <= 8 ? 8 - r : (r <= 24 ? 24 - r : 40 - r));
}

template <int NF, bool PER_AXIS, typename TL, int NT>
__global__ void __launch_bounds__(NT, 1) k_inner_blk(const DevGeo g, const TL* __restrict__ rlp, TL* e0, TL* e1,
                                                     Ctrl* ctrl, double* partials, const BlkShape sh,
                                                     const LTile<NF, 4, PER_AXIS> Lp) {
  constexpr int NLF = 4;
  constexpr int NIN = NF * NLF;
  constexpr int NEXP = LTile<NF, NLF, PER_AXIS>::NEXP;
  constexpr int SP = NEXP | 1;   // odd word stride per element: conflict-free shared loads
  extern __shared__ float smf[];
  __shared__ float wred[NT / 32];
  __shared__ int s_to;
  if (ctrl_done(ctrl) || *(volatile const int*)&ctrl->inner_done) return;
  const int j0 = *(volatile const int*)&ctrl->inner_iter;
  const int iter0 = *(volatile const int*)&ctrl->iter;
  const int lowp0 = *(volatile const int*)&ctrl->lowp_sweeps;
  const int max_iters = ctrl->max_iters, inner_max = ctrl->inner_max;
  const float limf = (float)(ctrl->inner_rtol * ctrl->rnorm);
  const int n0 = g.n[0], n1 = g.n[1], H = sh.halo, ld = (int)g.ld;
  const int tx0 = (int)(blockIdx.x % sh.tiles_x) * sh.tx, ty0 = (int)(blockIdx.x / sh.tiles_x) * sh.ty;
  const int tx1 = min(n0, tx0 + sh.tx), ty1 = min(n1, ty0 + sh.ty);
  const int tw = tx1 - tx0, th = ty1 - ty0;
  const int rx0 = max(0, tx0 - H), ry0 = max(0, ty0 - H);
  const int RX = min(n0, tx1 + H) - rx0, RY = min(n1, ty1 + H) - ry0;
  const int RA = RX * RY, P = blk_pitch(RX);
  float* const es0 = smf;
  float* const es1 = smf + (size_t)sh.ra_max * SP;
  float* rs = smf + 2 * (size_t)sh.ra_max * SP;
  // the whole region of e_j0 (written by the previous launch) and of r
  {
    const TL* eb = (j0 & 1) ? e1 : e0;
    for (int i = threadIdx.x; i < RA; i += NT) {
      const int K = (rx0 + i % RX) + n0 * (ry0 + i / RX);
      const int li = (i / RX) * P + i % RX;
#pragma unroll
      for (int e = 0; e < NEXP; ++e) {
        const bool live = (g.live >> e) & 1ull;
        es0[li * SP + e] = live ? ldcg_f(eb + (long long)e * ld + K) : 0.f;
        rs[li * SP + e] = live ? to_f(rlp[(long long)e * ld + K]) : 0.f;
      }
    }
  }
  unsigned* count = &ctrl->bar_count;
  float* partf = reinterpret_cast<float*>(partials);
  int cur = 0, done = 0;
  for (int m = 0;; ++m) {
    float* ec = cur ? es1 : es0;
    // halo of the current level (stored by the neighbours before the barrier) and the last
    // super-step's partial step norms, in one round trip
    float pv = 0.f;
    if (m > 0) {
      for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) pv += __ldcg(partf + ((m - 1) & 1) * gridDim.x + i);
      // the halo (region minus tile): the region's rows above and below the tile, then the
      // columns left and right of the tile in its rows; every thread issues all loads of
      // its halo element before storing any, so one round trip serves the whole halo
      const TL* gb = ((j0 + m) & 1) ? e1 : e0;
      const int nab = (ty0 - ry0) * RX, nbe = (ry0 + RY - ty1) * RX;
      const int lw = tx0 - rx0, sw = lw + (rx0 + RX - tx1);
      const int nh = nab + nbe + th * sw;
      for (int i = threadIdx.x; i < nh; i += NT) {
        int gx, gy;
        if (i < nab) {
          gx = rx0 + i % RX;
          gy = ry0 + i / RX;
        } else if (i < nab + nbe) {
          gx = rx0 + (i - nab) % RX;
          gy = ty1 + (i - nab) / RX;
        } else {
          const int k = i - nab - nbe, c = k % sw;
          gy = ty0 + k / sw;
          gx = c < lw ? rx0 + c : tx1 + (c - lw);
        }
        const int K = gx + n0 * gy;
        const int li = (gy - ry0) * P + (gx - rx0);
        float v[NEXP];
#pragma unroll
        for (int e = 0; e < NEXP; ++e) v[e] = ((g.live >> e) & 1ull) ? ldcg_f(gb + (long long)e * ld + K) : 0.f;
#pragma unroll
        for (int e = 0; e < NEXP; ++e) ec[li * SP + e] = v[e];
      }
    }
    // fixed-order fold (the same in every thread of every block): warp sums, then the warp
    // sums by one shuffle tree in each warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
    if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = pv;
    __syncthreads();
    float tot = (threadIdx.x & 31) < NT / 32 ? wred[threadIdx.x & 31] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    const float step = sqrtf(tot);
    const int j = j0 + done, it = iter0 + done;
    const bool budget = j >= inner_max || it >= max_iters;
    const bool stop = budget || (m > 0 && (step <= limf || !(step == step) || isinf(step)));
    if (threadIdx.x == 0 && blockIdx.x == 0) {
      ctrl->inner_iter = j;
      ctrl->iter = it;
      ctrl->lowp_sweeps = lowp0 + done;
      if (m > 0) ctrl->inner_step = (double)step;
      if (stop) ctrl->inner_done = 1;
    }
    if (stop) {
      // the whole tile into the buffer the outer sweep reads after j inner sweeps
      TL* fb = (j & 1) ? e1 : e0;
      for (int i = threadIdx.x; i < tw * th; i += NT) {
        const int gx = tx0 + i % tw, gy = ty0 + i / tw;
        const int li = (gy - ry0) * P + (gx - rx0);
        const int K = gx + n0 * gy;
#pragma unroll
        for (int e = 0; e < NEXP; ++e)
          if ((g.live >> e) & 1ull) fb[(long long)e * ld + K] = from_f<TL>(ec[li * SP + e]);
      }
      break;
    }
    const int h = min(H, min(inner_max - j, max_iters - it));
    float snorm = 0.f;
    TL* nbuf = ((j0 + m + 1) & 1) ? e1 : e0;   // the next super-step's buffer
    for (int t = 1; t <= h; ++t) {
      const float* src = cur ? es1 : es0;
      float* dst = cur ? es0 : es1;
      const int grow = H - t;
      const int ax0 = max(0, tx0 - grow), ay0 = max(0, ty0 - grow);
      const int aw = min(n0, tx1 + grow) - ax0, ah = min(n1, ty1 + grow) - ay0;
      // one element per thread; a warp takes an 8 x 4 patch of the area
      const int npx = (aw + 7) >> 3, npatch = npx * ((ah + 3) >> 2);
      const int dx = threadIdx.x & 7, dy = (threadIdx.x >> 3) & 3;
      auto sweep = [&](auto last_c) {
        constexpr bool LAST = decltype(last_c)::value;
        for (int pch = threadIdx.x >> 5; pch < npatch; pch += NT / 32) {
          const int ix = (pch % npx) * 8 + dx, iy = (pch / npx) * 4 + dy;
          if (ix >= aw || iy >= ah) continue;
          const int gx = ax0 + ix, gy = ay0 + iy;
          const int li = (gy - ry0) * P + (gx - rx0);
          // a1: the traces of the four faces (own and neighbour exports from shared memory)
          float tr[NIN];
#pragma unroll
          for (int f = 0; f < NLF; ++f) {
            const int a = f >> 1;
            const int c = a ? gy : gx, nn = a ? n1 : n0;
            const bool bnd = (f & 1) ? (c == nn - 1) : (c == 0);
            const int kind = g.kind[f];
            const int lin = li + ((f & 1) ? 1 : -1) * (a ? P : 1);
            const int os = PER_AXIS ? a * NF : f * NF;
            const int ns = PER_AXIS ? a * NF : (f ^ 1) * NF;
            const float wo = kind == FK_OWN_D ? 1.f : kind == FK_SUM_D ? (!bnd ? 1.f : (g.bc_mirror ? 2.f : 0.f)) : 0.f;
            const bool nbm = !bnd && (kind == FK_NBR_D || kind == FK_SUM_D);
#pragma unroll
            for (int q = 0; q < NF; ++q) {
              const float nb = nbm ? src[lin * SP + ns + q] : 0.f;
              tr[f * NF + q] = wo * src[li * SP + os + q] + nb;
            }
          }
          bool in_tile = false, strip = false;
          if constexpr (LAST) {
            in_tile = gx >= tx0 && gx < tx1 && gy >= ty0 && gy < ty1;
            strip = in_tile && (gx - tx0 < H || tx1 - 1 - gx < H || gy - ty0 < H || ty1 - 1 - gy < H);
          }
          const int K = gx + n0 * gy;
          // a4: rounded to the storage type.  In the last sweep: the step norm over the tile,
          // and the tile elements within H of its edges (the neighbours' halo) go straight to
          // the next super-step's global buffer
          auto finish = [&](int e, float v) {
            const TL nt = from_f<TL>(v);
            const float nv = to_f(nt);
            if constexpr (LAST) {
              const float d = nv - src[li * SP + e];
              if (in_tile) snorm = fmaf(d, d, snorm);
              if (strip && ((g.live >> e) & 1ull)) nbuf[(long long)e * ld + K] = nt;
            }
            return nv;
          };
          // a3: e_new = r + L_E t, one accumulation chain per row in trace order (a chain
          // reuses its accumulator register: twice the FMA issue rate of interleaving all rows
          // per trace value).  Rows of slots that carry no value have zero operator rows and
          // zero r, so they stay zero.
#pragma unroll
          for (int e = 0; e < NEXP; ++e) {
            float v = rs[li * SP + e];
#pragma unroll
            for (int k = 0; k < NIN; ++k) v = fmaf(Lp.L[e][k], tr[k], v);
            dst[li * SP + e] = finish(e, v);
          }
        }
      };
      if (t == h) sweep(std::true_type{});
      else sweep(std::false_type{});
      __syncthreads();
      cur ^= 1;
    }
    done += h;
    const float blk = sum_partials<NT>(snorm, wred);
    arrive_wait(partf + (m & 1) * gridDim.x, count, (unsigned)(m + 1), blk, ctrl, &s_to);
    if (s_to) break;
  }
}

// Launch k_inner_blk with halo m.blk_h (>= 2): the tile shape minimises the tile + halo area
// over at most one tile per SM; returns cudaErrorNotSupported (nothing launched) when the
// state does not fit in shared memory or the grid would not be co-resident.
template <int NF, bool PER_AXIS, typename TL, int NT>
cudaError_t launch_blk_v(MixedArgs& m, TL* rl, TL* e0, TL* e1) {
  using LT = LTile<NF, 4, PER_AXIS>;
  constexpr int SP = LT::NEXP | 1;   // as in k_inner_blk
  const LaunchArgs& a = m.base;
  const int H = m.blk_h;
  if (a.g.dim != 2 || H < 2 || !m.LE32h || a.g.n_exp != LT::NEXP || (long long)a.g.ld * LT::NEXP >= (1LL << 31))
    return cudaErrorNotSupported;
  auto k = k_inner_blk<NF, PER_AXIS, TL, NT>;
  int dev = 0, sms = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  smem_max -= 1024;   // static shared memory of the kernel
  const int n0 = a.g.n[0], n1 = a.g.n[1];
  int cap = sms;
  if (cap > m.max_grid) cap = m.max_grid;
  if (cap > m.slots / 2) cap = m.slots / 2;
  // the distinct tile shapes over at most one tile per SM whose state fits in shared memory,
  // in order of increasing tile + halo area; m.blk_rank picks one (the autotuner times several)
  struct Cand {
    long long area;
    int txn, tiles_x, tx, ty, grid;
  };
  std::vector<Cand> cands;
  for (int txn = 1; txn <= n0 && txn <= cap; ++txn) {
    const int tx = (n0 + txn - 1) / txn, tiles_x = (n0 + tx - 1) / tx;
    const int tyn = cap / tiles_x;
    if (tyn < 1) continue;
    const int ty = (n1 + tyn - 1) / tyn, tiles_y = (n1 + ty - 1) / ty;
    const long long area = (long long)blk_pitch(std::min(n0, tx + 2 * H)) * std::min(n1, ty + 2 * H);
    if ((size_t)3 * area * SP * sizeof(float) > (size_t)smem_max) continue;
    bool dup = false;
    for (const Cand& c : cands) dup = dup || (c.tx == tx && c.ty == ty);
    if (!dup) cands.push_back({area, txn, tiles_x, tx, ty, tiles_x * tiles_y});
  }
  if (cands.empty()) return cudaErrorNotSupported;
  std::stable_sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) { return x.area < y.area; });
  const Cand& pick = cands[std::min((size_t)std::max(m.blk_rank, 0), cands.size() - 1)];
  BlkShape sh{pick.tiles_x, pick.tx, pick.ty, H, (int)pick.area};
  const int grid = pick.grid;
  if (grid < 1) return cudaErrorNotSupported;
  const size_t smem = (size_t)3 * sh.ra_max * SP * sizeof(float);
  cudaError_t e = allow_dynamic_smem(k);
  if (e != cudaSuccess) return e;
  int per = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, NT, smem);
  if (e != cudaSuccess) return e;
  if ((long long)per * sms < grid) return cudaErrorNotSupported;
  LT L;
  for (int r = 0; r < LT::NEXP; ++r)   // rows of slots that carry no value: zero
    for (int q = 0; q < LT::NIN; ++q) L.L[r][q] = ((a.g.live >> r) & 1ull) ? m.LE32h[r * LT::NIN + q] : 0.f;
  DevGeo gg = a.g;
  const TL* rlc = rl;
  Ctrl* ct = a.ctrl;
  double* pp = a.partials;
  e = cudaMemsetAsync(&a.ctrl->bar_count, 0, sizeof(unsigned), a.stream);
  if (e != cudaSuccess) return e;
  void* args[] = {&gg, &rlc, &e0, &e1, &ct, &pp, &sh, &L};
  e = cudaLaunchCooperativeKernel((const void*)k, dim3((unsigned)grid), dim3(NT), args, smem, a.stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Tile kernel shape: one element per thread (default) or, with IHDG_TILE_LPE=4 on 2D
// meshes, four lanes per element (one face each) with shuffled traces.
template <int NF, int NLF, bool PER_AXIS, typename TL>
cudaError_t launch_tile(MixedArgs& m, TL* rl, TL* e0, TL* e1) {
  return launch_tile_v<NF, NLF, PER_AXIS, TL, 512, 1>(m, rl, e0, e1);
}

// Cooperative launch of k_inner_persist: as many co-resident blocks as the elements need.
template <int NF, int NLF, bool PER_AXIS, typename TL>
cudaError_t launch_persist(MixedArgs& m, TL* rl, TL* e0, TL* e1) {
  using LT = LTile<NF, NLF, PER_AXIS>;
  const LaunchArgs& a = m.base;
  if (!m.LE32h || a.g.n_exp != LT::NEXP) return cudaErrorNotSupported;
  const size_t smem = 0;
  const unsigned long long all = LT::NEXP >= 64 ? ~0ull : (1ull << LT::NEXP) - 1;
  auto k = (a.g.live & all) == all ? k_inner_persist<NF, NLF, PER_AXIS, true, TL>
                                   : k_inner_persist<NF, NLF, PER_AXIS, false, TL>;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, PBS, smem);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  long long need = (a.g.nel + PBS - 1) / PBS;
  long long cap = (long long)per * sms;
  int grid = (int)(need < cap ? need : cap);
  if (grid > m.max_grid) grid = m.max_grid;
  LT L;
  for (int r = 0; r < LT::NEXP; ++r)
    for (int q = 0; q < LT::NIN; ++q) L.L[r][q] = m.LE32h[r * LT::NIN + q];
  DevGeo gg = a.g;
  const TL* rlc = rl;
  Ctrl* ct = a.ctrl;
  double* pp = a.partials;
  void* args[] = {&gg, &rlc, &e0, &e1, &ct, &pp, &L};
  e = cudaMemsetAsync(&a.ctrl->bar_count, 0, sizeof(unsigned), a.stream);
  if (e != cudaSuccess) return e;
  e = cudaLaunchCooperativeKernel((const void*)k, dim3(grid), dim3(PBS), args, smem, a.stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

inline unsigned grid_for(long long n) { return (unsigned)((n + BS - 1) / BS); }

template <typename TL>
struct MixedRunner {
  template <int NF, int NLF>
  struct Fn {
    static cudaError_t run(MixedArgs& m, int which, int has_e, int count) {
      constexpr int NIN = NF * NLF;
      const LaunchArgs& a = m.base;
      TL* e0 = static_cast<TL*>(m.e[0]);
      TL* e1 = static_cast<TL*>(m.e[1]);
      TL* rl = static_cast<TL*>(m.rlp);
      if (which == 0) {
        size_t smem = ((size_t)a.g.n_exp * NIN + (size_t)NIN * BS) * sizeof(double);
        auto k = k_outer64<NF, NLF, TL>;
        if (smem > 32 * 1024) {
          cudaError_t e = allow_dynamic_smem(k);
          if (e != cudaSuccess) return e;
        }
        k<<<grid_for(a.g.nel), BS, smem, a.stream>>>(a.g, a.op, a.F, m.E64, a.ring_stride, m.r64, rl, e0, e1, has_e,
                                                      a.ctrl, a.partials);
      } else if (which == 1) {
        size_t smem = (size_t)NIN * (NIN + 1) / 2 * sizeof(double) + (size_t)a.g.n_exp * NIN * sizeof(float);
        auto k = k_inner_first<NF, NLF, TL>;
        if (smem > 32 * 1024) {
          cudaError_t e = allow_dynamic_smem(k);
          if (e != cudaSuccess) return e;
        }
        k<<<grid_for(a.g.nel), BS, smem, a.stream>>>(a.g, a.op, m.r64, e0, a.ctrl, a.partials, a.res_hist);
      } else {
        if (m.use_tc) {
          cudaError_t ce;
          if constexpr (std::is_same<TL, __nv_bfloat16>::value) {
            ce = a.g.per_axis ? launch_tc<NF, NLF, true, TC_BF16>(m, rl, e0, e1)
                              : launch_tc<NF, NLF, false, TC_BF16>(m, rl, e0, e1);
          } else if (m.prec == IHDG_MIXED_TF32) {
            ce = a.g.per_axis ? launch_tc<NF, NLF, true, TC_TF32>(m, rl, e0, e1)
                              : launch_tc<NF, NLF, false, TC_TF32>(m, rl, e0, e1);
          } else {
            ce = a.g.per_axis ? launch_tc<NF, NLF, true, TC_TF32X4>(m, rl, e0, e1)
                              : launch_tc<NF, NLF, false, TC_TF32X4>(m, rl, e0, e1);
          }
          if (ce != cudaErrorNotSupported) return m.ran = m.tc_staged ? 6 : 1, ce;
          // shapes the tensor-core kernel does not take (n_in > 64 or n_exp > 32) fall through
          // to the CUDA-core kernels in full float32
        }
        if (!m.no_tile) {
          if constexpr (NLF == 4) {
            if (m.blk_h >= 2) {
              cudaError_t be = a.g.per_axis ? launch_blk_v<NF, true, TL, 1024>(m, rl, e0, e1)
                                            : launch_blk_v<NF, false, TL, 1024>(m, rl, e0, e1);
              if (be != cudaErrorNotSupported) return m.ran = 2, be;
            }
            if (m.tile_lpe != 1) {
              cudaError_t re = a.g.per_axis ? launch_reg<NF, true, TL>(m, rl, e0, e1)
                                            : launch_reg<NF, false, TL>(m, rl, e0, e1);
              if (re != cudaErrorNotSupported) return m.ran = 3, re;
            }
          }
          cudaError_t te = a.g.per_axis ? launch_tile<NF, NLF, true, TL>(m, rl, e0, e1)
                                        : launch_tile<NF, NLF, false, TL>(m, rl, e0, e1);
          if (te != cudaErrorNotSupported) return m.ran = 4, te;
        }
        m.ran = 5;
        return a.g.per_axis ? launch_persist<NF, NLF, true, TL>(m, rl, e0, e1)
                            : launch_persist<NF, NLF, false, TL>(m, rl, e0, e1);
      }
      return cudaGetLastError();
    }
  };
};

}  // namespace

template <typename TL>
cudaError_t mixed_launch(MixedArgs& m, int which, int has_e, int count) {
  const DevGeo& g = m.base.g;
  using R = MixedRunner<TL>;
  if (g.dim == 2) {
    switch (g.nf) {
      case 2: return R::template Fn<2, 4>::run(m, which, has_e, count);
      case 3: return R::template Fn<3, 4>::run(m, which, has_e, count);
      case 4: return R::template Fn<4, 4>::run(m, which, has_e, count);
      case 5: return R::template Fn<5, 4>::run(m, which, has_e, count);
    }
  } else {
    switch (g.nf) {
      case 4: return R::template Fn<4, 6>::run(m, which, has_e, count);
      case 9: return R::template Fn<9, 6>::run(m, which, has_e, count);
    }
  }
  return cudaErrorNotSupported;
}

}  // namespace ihdg
