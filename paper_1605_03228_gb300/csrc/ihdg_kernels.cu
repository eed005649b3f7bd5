// CUDA kernels of the element-parallel iHDG sweep (sm_103a).
//
// One sweep of Algorithm 1 (Section 2) on the export state E (see ihdg_ops.h):
//   a1  gather the traces every element needs from its own and its neighbours' exports of
//       iterate k, combined by the upwind flux (transport: upwind value, Eq. transportLocale;
//       convection-diffusion: (h^- + h^+)/alpha, Section 4.1; shallow water: h^- + h^+, or
//       2h^- at a wall, the trace formula under Eq. localSolverDD);
//   a2  the per-sweep right-hand side is only the trace-dependent part: forcing, boundary
//       data and time-step data are folded once per solve into F (k_forcing);
//   a3  apply the precomputed local solve, E^{k+1} = F + L_E t^k;
//   a4  write E^{k+1} (three-slot ring) and accumulate the stopping residual
//       ||u^{k+1} - u^k||^2 = dt^T Q dt with dt = t(E^k) - t(E^{k-1});
//   a5  the last block to finish sums the per-block partial sums in a fixed order
//       (deterministic, no floating-point atomics) and takes the loop decision on the device.
//
// Layout: every per-element array is slot-major, x[slot * ld + element], so a warp of
// consecutive elements reads consecutive addresses for every slot (neighbours along x are
// one element away, along y n0, along z n0*n1).  Elements are numbered x fastest.
#include <cuda_runtime.h>

#include <cstdio>
#include <vector>

#include "ihdg_dev.h"
#include "ihdg_kernels.h"
#include "ihdg_common.cuh"
#include "ihdg_persist.cuh"

namespace ihdg {

namespace {

// ---------------------------------------------------------------------------------------
// a2 (once per solve / per time step): the volume source V = A^{-1} b and the export forcing
// F = R A^{-1} b of every element in float64, from the forcing f at the quadrature points and
// the boundary data g (steady problems) or from the time-step data q^m (shallow water).  The
// block's input rows ([element][nin] in global memory) are first copied, coalesced, into
// shared memory as columns [nin][element] (pitch BS + 1 doubles), so each thread reads its
// element's inputs from there for every output row instead of re-fetching its row through
// L1; the operator rows are the same for every thread.
__global__ void __launch_bounds__(BS) k_forcing(DevGeo g, OpsDev op, SrcDev src, double* __restrict__ F,
                                                double* __restrict__ V) {
  extern __shared__ double s_in[];
  constexpr int SPI = BS + 1;
  const long long K0 = (long long)blockIdx.x * BS;
  const int cnt = (int)(g.nel - K0 < BS ? g.nel - K0 : BS);
  const int nin = g.steady ? g.nqv : g.nvol;
  const double* in = (g.steady ? src.f : src.q) + K0 * nin;
  for (int idx = threadIdx.x; idx < cnt * nin; idx += BS) {
    const int e = idx / nin, q = idx - e * nin;
    s_in[q * SPI + e] = in[idx];
  }
  __syncthreads();
  if (threadIdx.x >= cnt) return;
  const long long K = K0 + threadIdx.x;
  const double* x = s_in + threadIdx.x;   // x[q * SPI]: this element's input q
  int c[3];
  coords(g, K, c);
  // row r of operator M (nin inputs) and boundary operators Mb, applied to this element
  auto apply = [&](const double* M, const double* const* Mb, int r) {
    double v = 0.0;
    const double* row = M + (long long)r * nin;
    for (int q = 0; q < nin; ++q) v += row[q] * x[q * SPI];
    if (g.steady)
      for (int f = 0; f < g.nlf; ++f) {
        if (!on_bnd(g, c, f)) continue;
        const double* gb = src.g + bface_of(g, c, f) * g.nqf;
        const double* rb = Mb[f] + (long long)r * g.nqf;
        for (int q = 0; q < g.nqf; ++q) v += rb[q] * gb[q];
      }
    return v;
  };
  // the volume source, kept for the first sweep's residual and the reconstruction
  for (int i = 0; i < g.nvol; ++i) V[(long long)i * g.ld + K] = apply(g.steady ? op.PV : op.PqV, op.PVb, i);
  for (int e = 0; e < g.n_exp; ++e)
    if (row_live(g, e, g.nf)) F[(long long)e * g.ld + K] = apply(g.steady ? op.PF : op.PqF, op.PFb, e);
}

// Operator of the GMRES solve around the sweep (Section 4.2, closing remark): on the live
// export rows, w = s (v - L_E t(v)) + F, i.e. s (I - T) v + F with T v = L_E t(v) the linear
// part of one float64 sweep (its forcing F left out).  s = 1 with no forcing gives the Arnoldi
// product (I - T) v; s = -1 with the forcing gives the residual F - (I - T) v.  Dead rows and
// the padding columns of w are not written.  Returns at once when *done is set.
template <int NF, int NLF>
__global__ void __launch_bounds__(BS) k_kry_apply(DevGeo g, OpsDev op, const double* __restrict__ v,
                                                  const double* __restrict__ F, double s, double* __restrict__ w,
                                                  const int* __restrict__ done) {
  constexpr int NIN = NF * NLF;
  extern __shared__ double sdyn[];
  if (done && *(const volatile int*)done) return;
  for (int i = threadIdx.x; i < g.n_exp * NIN; i += BS) sdyn[i] = op.LE[i];
  __syncthreads();
  const long long K = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= g.nel) return;
  int c[3];
  coords(g, K, c);
  double t[NIN];
  gather<NF, NLF, double, double>(g, v, K, c, [&](int q, double x) { t[q] = x; });
  for (int e = 0; e < g.n_exp; ++e) {
    if (!row_live(g, e, NF)) continue;
    const double* row = sdyn + e * NIN;
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < NIN; ++q) acc += row[q] * t[q];
    double r = s * (v[(long long)e * g.ld + K] - acc);
    if (F) r += F[(long long)e * g.ld + K];
    w[(long long)e * g.ld + K] = r;
  }
}

// Initial export E^0 = R u^0 (u^0 in the volume layout [nel][nvol]).
__global__ void __launch_bounds__(BS) k_export0(DevGeo g, OpsDev op, const double* __restrict__ u0,
                                                double* __restrict__ E0) {
  const long long K = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= g.nel) return;
  for (int e = 0; e < g.n_exp; ++e) {
    if (!row_live(g, e, g.nf)) continue;
    double v = 0.0;
    if (u0) {
      const double* row = op.R + (long long)e * g.nvol;
      for (int i = 0; i < g.nvol; ++i) v += row[i] * u0[K * g.nvol + i];
    }
    E0[(long long)e * g.ld + K] = v;
  }
}

// First sweep (k = 0 -> 1): E^1 = F + L_E t(E^0), and the residual ||u^1 - u^0|| on the
// full volume state (u^0 is the initial guess, not a previous local solve).
template <int NF, int NLF>
__global__ void __launch_bounds__(BS) k_first(DevGeo g, OpsDev op, const double* __restrict__ V,
                                              const double* __restrict__ u0, const double* __restrict__ F,
                                              double* ring, long long ring_stride, Ctrl* ctrl, double* partials,
                                              double* res_hist) {
  constexpr int NIN = NF * NLF;
  __shared__ double ws[BS / 32];
  extern __shared__ double sdyn[];
  double* du = sdyn + threadIdx.x;    // per-thread column of nvol doubles, stride BS
  const long long K = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (K < g.nel) {
    double* E1 = ring + ring_stride;
    if (u0) {
      int c[3];
      coords(g, K, c);
      double t[NIN];
      gather<NF, NLF, double, double>(g, ring, K, c, [&](int s, double v) { t[s] = v; });
      for (int e = 0; e < g.n_exp; ++e) {
        if (!row_live(g, e, NF)) continue;
        double v = F[(long long)e * g.ld + K];
        const double* row = op.LE + (long long)e * NIN;
#pragma unroll
        for (int s = 0; s < NIN; ++s) v += row[s] * t[s];
        E1[(long long)e * g.ld + K] = v;
      }
      for (int i = 0; i < g.nvol; ++i) {
        double v = V[(long long)i * g.ld + K];
        const double* row = op.Lvol + (long long)i * NIN;
#pragma unroll
        for (int s = 0; s < NIN; ++s) v += row[s] * t[s];
        du[i * BS] = v - u0[K * g.nvol + i];
      }
    } else {
      // u^0 = 0: E^0 = 0, so t(E^0) = 0, E^1 = F and u^1 - u^0 = A^{-1} b
      for (int e = 0; e < g.n_exp; ++e)
        if (row_live(g, e, NF)) E1[(long long)e * g.ld + K] = F[(long long)e * g.ld + K];
      for (int i = 0; i < g.nvol; ++i) du[i * BS] = V[(long long)i * g.ld + K];
    }
    // ||du||^2 in the stopping norm: sum over components c of w_c du_c^T M du_c
    for (int comp = 0; comp < g.nvol / g.nb; ++comp) {
      const double w = op.wcomp[comp];
      if (w == 0.0) continue;
      const double* dc = du + comp * g.nb * BS;
      double sc = 0.0;
      for (int i = 0; i < g.nb; ++i) {
        double s = 0.0;
        const double* row = op.Mb + (long long)i * g.nb;
        for (int j = 0; j < g.nb; ++j) s += row[j] * dc[j * BS];
        sc += dc[i * BS] * s;
      }
      acc += w * sc;
    }
  }
  double tot;
  if (arrive(ctrl, partials, acc, ws, &tot) && threadIdx.x == 0) decide(ctrl, tot, res_hist, true);
}

// Plain sweep in float64 (k -> k+1, k >= 1): a1..a5.  E^k in ring slot k%3, E^{k-1} in
// (k+2)%3, E^{k+1} written to (k+1)%3.  The operators L_E (n_exp x NIN) and the packed upper
// triangle of Q (off-diagonals doubled) are staged in shared memory; the gathered traces
// live in a per-thread shared-memory column, their increments in registers.
template <int NF, int NLF>
__global__ void __launch_bounds__(BS) k_sweep64(DevGeo g, OpsDev op, const double* __restrict__ F,
                                                double* ring, long long ring_stride, Ctrl* ctrl,
                                                double* partials, double* res_hist) {
  constexpr int NIN = NF * NLF;
  constexpr int NQ = NIN * (NIN + 1) / 2;
  __shared__ double ws[BS / 32];
  extern __shared__ double sdyn[];
  if (ctrl_done(ctrl)) return;
  const int it = ctrl_iter(ctrl);
  double* sLE = sdyn;                       // n_exp * NIN
  double* sQ = sLE + g.n_exp * NIN;         // NQ
  double* st = sQ + NQ + threadIdx.x;       // per-thread trace column, stride BS
  for (int i = threadIdx.x; i < g.n_exp * NIN; i += BS) sLE[i] = op.LE[i];
  for (int i = threadIdx.x; i < NQ; i += BS) sQ[i] = op.Qp[i];
  __syncthreads();
  const double* Ecur = ring + (long long)(it % 3) * ring_stride;
  const double* Eprv = ring + (long long)((it + 2) % 3) * ring_stride;
  double* Enxt = ring + (long long)((it + 1) % 3) * ring_stride;
  const long long K = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (K < g.nel) {
    int c[3];
    coords(g, K, c);
    double d[NIN];
    gather<NF, NLF, double, double>(g, Ecur, K, c, [&](int s, double v) { st[s * BS] = v; d[s] = v; });
    gather<NF, NLF, double, double>(g, Eprv, K, c, [&](int s, double v) { d[s] -= v; });
    // a4 residual: dt^T Q dt with Q packed upper-triangular, off-diagonals doubled
    int q = 0;
#pragma unroll
    for (int s = 0; s < NIN; ++s) {
      double r = 0.0;
#pragma unroll
      for (int u = s; u < NIN; ++u) r += sQ[q + u - s] * d[u];
      q += NIN - s;
      acc += d[s] * r;
    }
    // a3: E^{k+1} = F + L_E t^k, in chunks whose forcing loads are issued together
    constexpr int CH = 8;
#pragma unroll
    for (int c0 = 0; c0 < NIN; c0 += CH) {
      double fv[CH];
#pragma unroll
      for (int i = 0; i < CH; ++i) fv[i] = (c0 + i < g.n_exp && row_live(g, c0 + i, NF)) ? F[(long long)(c0 + i) * g.ld + K] : 0.0;
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int e = c0 + i;
        if (e < g.n_exp && row_live(g, e, NF)) {
          double v = fv[i];
          const double* row = sLE + e * NIN;
#pragma unroll
          for (int s = 0; s < NIN; ++s) v += row[s] * st[s * BS];
          Enxt[(long long)e * g.ld + K] = v;
        }
      }
    }
  }
  double tot;
  if (arrive(ctrl, partials, acc, ws, &tot) && threadIdx.x == 0) decide(ctrl, tot, res_hist, true);
}

// Grid barrier plus the float64 sum of one value per block, for cooperative launches: the
// same fixed-order sum as arrive() (thread-strided partial loads, then block_sum), so the
// residual is bitwise the one of the launch-per-sweep path.  Thread 0 publishes the block's
// value, arrives with a release add and polls with acquire loads bounded by
// ctrl->wait_cycles (then ctrl->timeout).  The total is valid in every thread.
__device__ double barrier_sum64(double* part, unsigned* count, unsigned nb, double mine, Ctrl* ctrl, double* ws,
                                double* s_out, int* s_flag, int bid, int nblk) {
  __syncthreads();
  if (threadIdx.x == 0) {
    part[bid] = mine;
    if (bid != ctrl->stall_block) red_release_add(count, 1u);
    const unsigned target = nb * (unsigned)nblk;
    const long long lim = ctrl->wait_cycles;
    const long long t0 = clock64();
    while (ld_acquire_u32(count) < target) {
      if (clock64() - t0 > lim) { atomicExch(&ctrl->timeout, 1); break; }
    }
    *s_flag = *(volatile int*)&ctrl->timeout;
  }
  __syncthreads();
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += __ldcg(part + i);
  const double t = block_sum(acc, ws);
  if (threadIdx.x == 0) *s_out = t;
  __syncthreads();
  return *s_out;
}

// The float64 sweep loop in one cooperative launch (meshes whose one-element-per-thread grid
// is co-resident): every sweep is k_sweep64's a1..a4, then a grid barrier with the residual
// sum, then the loop decision, which every block takes identically from the same total
// (decide()'s rules); block 0 records it in ctrl.  Per sweep this saves a launch and a host
// check, which dominate on small meshes.
// One problem's arguments of the persistent float64 loop (also one item of a grouped launch).
struct P64Args {
  DevGeo g;
  OpsDev op;
  const double* F;
  double* ring;
  long long ring_stride;
  Ctrl* ctrl;
  double* partials;
  double* res_hist;
};

// The loop body of block bid of the nblk blocks that work for one problem.
template <int NF, int NLF>
__device__ __forceinline__ void sweep64_persist_body(const DevGeo& g, const OpsDev& op, const double* __restrict__ F,
                                                     double* ring, long long ring_stride, Ctrl* ctrl,
                                                     double* partials, double* res_hist, int bid, int nblk) {
  constexpr int NIN = NF * NLF;
  constexpr int NQ = NIN * (NIN + 1) / 2;
  __shared__ double ws[BS / 32];
  __shared__ double s_tot;
  __shared__ int s_to;
  extern __shared__ double sdyn[];
  if (ctrl_done(ctrl)) return;
  int it = ctrl_iter(ctrl);
  double res_min = ctrl->res_min;
  const double tol = ctrl->tol, divf = ctrl->diverge_factor;
  const int max_iters = ctrl->max_iters;
  double* sLE = sdyn;                       // n_exp * NIN
  double* sQ = sLE + g.n_exp * NIN;         // NQ
  double* st = sQ + NQ + threadIdx.x;       // per-thread trace column, stride BS
  for (int i = threadIdx.x; i < g.n_exp * NIN; i += BS) sLE[i] = op.LE[i];
  for (int i = threadIdx.x; i < NQ; i += BS) sQ[i] = op.Qp[i];
  __syncthreads();
  const long long K = (long long)bid * blockDim.x + threadIdx.x;
  int c[3] = {0, 0, 0};
  if (K < g.nel) coords(g, K, c);
  for (int s = 0;; ++s) {
    const double* Ecur = ring + (long long)(it % 3) * ring_stride;
    const double* Eprv = ring + (long long)((it + 2) % 3) * ring_stride;
    double* Enxt = ring + (long long)((it + 1) % 3) * ring_stride;
    double acc = 0.0;
    if (K < g.nel) {
      double d[NIN];
      gather<NF, NLF, double, double>(g, Ecur, K, c, [&](int q, double v) { st[q * BS] = v; d[q] = v; });
      gather<NF, NLF, double, double>(g, Eprv, K, c, [&](int q, double v) { d[q] -= v; });
      int qq = 0;
#pragma unroll
      for (int a = 0; a < NIN; ++a) {
        double r = 0.0;
#pragma unroll
        for (int u = a; u < NIN; ++u) r += sQ[qq + u - a] * d[u];
        qq += NIN - a;
        acc += d[a] * r;
      }
      constexpr int CH = 8;
#pragma unroll
      for (int c0 = 0; c0 < NIN; c0 += CH) {
        double fv[CH];
#pragma unroll
        for (int i = 0; i < CH; ++i) fv[i] = (c0 + i < g.n_exp && row_live(g, c0 + i, NF)) ? F[(long long)(c0 + i) * g.ld + K] : 0.0;
#pragma unroll
        for (int i = 0; i < CH; ++i) {
          const int e = c0 + i;
          if (e < g.n_exp && row_live(g, e, NF)) {
            double v = fv[i];
            const double* row = sLE + e * NIN;
#pragma unroll
            for (int q = 0; q < NIN; ++q) v += row[q] * st[q * BS];
            Enxt[(long long)e * g.ld + K] = v;
          }
        }
      }
    }
    const double blk = block_sum(acc, ws);
    const double tot = barrier_sum64(partials + (size_t)(s & 1) * nblk, &ctrl->bar_count, (unsigned)(s + 1),
                                     blk, ctrl, ws, &s_tot, &s_to, bid, nblk);
    if (s_to) break;
    // decide()'s rules, taken identically in every block
    const double res = sqrt(tot);
    const int k = it + 1;
    bool done = false;
    int status = 4;
    if (res < tol) {
      done = true;
      status = 0;
    } else if (!(res == res) || isinf(res) || (divf > 0.0 && res > divf * res_min)) {
      done = true;
      status = 5;
    } else {
      if (res < res_min) res_min = res;
      if (k >= max_iters) done = true;
    }
    if (bid == 0 && threadIdx.x == 0) {
      ctrl->iter = k;
      ctrl->fp64_sweeps += 1;
      ctrl->res = res;
      if (res_hist) res_hist[k] = res;
      ctrl->res_min = res_min;
      if (done) {
        ctrl->status = status;
        ctrl->done = 1;
      }
    }
    it = k;
    if (done) break;
  }
}

template <int NF, int NLF>
__global__ void __launch_bounds__(BS) k_sweep64_persist(DevGeo g, OpsDev op, const double* __restrict__ F,
                                                        double* ring, long long ring_stride, Ctrl* ctrl,
                                                        double* partials, double* res_hist) {
  sweep64_persist_body<NF, NLF>(g, op, F, ring, ring_stride, ctrl, partials, res_hist, (int)blockIdx.x,
                                (int)gridDim.x);
}

// Several problems' float64 loops in one cooperative launch: blocks off[i] .. off[i+1]-1 work
// for item i exactly as the blocks of its own launch would (the same block ids, count and
// reduction order, so the results are bitwise those of solving it alone); each problem stops
// on its own, and its blocks leave the launch when it does.
template <int NF, int NLF>
__global__ void __launch_bounds__(BS) k_sweep64_persist_group(const P64Args* __restrict__ items,
                                                              const int* __restrict__ off, int n) {
  int lo = 0, hi = n - 1;   // the item whose block range holds this block
  const int b = (int)blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  const P64Args& A = items[lo];   // read from global memory where used (no register copy)
  const int base = __ldg(off + lo), nblk = __ldg(off + lo + 1) - base;
  sweep64_persist_body<NF, NLF>(A.g, A.op, A.F, A.ring, A.ring_stride, A.ctrl, A.partials, A.res_hist, b - base, nblk);
}

// Volume reconstruction u = A^{-1} b + L_vol t(E) (+ L_vol t(E2) when E2 is given).
template <int NF, int NLF>
__global__ void __launch_bounds__(BS) k_reconstruct(DevGeo g, OpsDev op, const double* __restrict__ V,
                                                    const double* __restrict__ E, const double* __restrict__ E2,
                                                    double* __restrict__ u) {
  constexpr int NIN = NF * NLF;
  const long long K = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= g.nel) return;
  int c[3];
  coords(g, K, c);
  double t[NIN];
  gather<NF, NLF, double, double>(g, E, K, c, [&](int s, double v) { t[s] = v; });
  if (E2) gather<NF, NLF, double, double>(g, E2, K, c, [&](int s, double v) { t[s] += v; });
  for (int i = 0; i < g.nvol; ++i) {
    double v = V[(long long)i * g.ld + K];
    const double* row = op.Lvol + (long long)i * NIN;
#pragma unroll
    for (int s = 0; s < NIN; ++s) v += row[s] * t[s];
    u[K * g.nvol + i] = v;
  }
}

// Trace output on every face node (Algorithm 1 step 3 applied to the final iterate):
// transport: the upwind export (inflow boundary: projected g; beta.n = 0: {{u}});
// convection-diffusion: (h^- + h^+)/alpha inside, projected g on the boundary;
// shallow water: h^- + h^+ inside, 2 h^- at walls.
__global__ void __launch_bounds__(BS) k_trace_out(DevGeo g, OpsDev op, SrcDev src, const double* __restrict__ E,
                                                  const double* __restrict__ E2, const double* __restrict__ u,
                                                  int pde, double beta0, double beta1, double beta2,
                                                  double al0, double al1, double al2, long long nface,
                                                  double* __restrict__ tr) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nface * g.nf) return;
  const long long fc = idx / g.nf;
  const int j = (int)(idx % g.nf);
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long cnt0 = (long long)(n0 + 1) * n1 * n2;
  const long long cnt1 = (long long)n0 * (n1 + 1) * n2;
  int a;
  long long loc;
  if (fc < cnt0) { a = 0; loc = fc; } else if (fc < cnt0 + cnt1) { a = 1; loc = fc - cnt0; } else { a = 2; loc = fc - cnt0 - cnt1; }
  int ci, cj, ck;
  long long L = -1, R = -1, bf = -1;
  auto eid = [&](long long i, long long jj, long long k) { return i + (long long)n0 * (jj + (long long)n1 * k); };
  if (a == 0) {
    ci = (int)(loc % (n0 + 1)); cj = (int)((loc / (n0 + 1)) % n1); ck = (int)(loc / ((long long)(n0 + 1) * n1));
    if (ci > 0) L = eid(ci - 1, cj, ck);
    if (ci < n0) R = eid(ci, cj, ck);
    if (ci == 0 || ci == n0) bf = 2LL * (cj + (long long)n1 * ck) + (ci == n0);
  } else if (a == 1) {
    ci = (int)(loc % n0); cj = (int)((loc / n0) % (n1 + 1)); ck = (int)(loc / ((long long)n0 * (n1 + 1)));
    if (cj > 0) L = eid(ci, cj - 1, ck);
    if (cj < n1) R = eid(ci, cj, ck);
    if (cj == 0 || cj == n1) bf = g.nbf_off[1] + (long long)ck * 2 * n0 + (long long)(cj == n1) * n0 + ci;
  } else {
    ci = (int)(loc % n0); cj = (int)((loc / n0) % n1); ck = (int)(loc / ((long long)n0 * n1));
    if (ck > 0) L = eid(ci, cj, ck - 1);
    if (ck < n2) R = eid(ci, cj, ck);
    if (ck == 0 || ck == n2) bf = g.nbf_off[2] + (long long)(ck == n2) * n0 * n1 + (long long)cj * n0 + ci;
  }
  const int fL = 2 * a + 1, fR = 2 * a;   // the face as seen from its left / right element
  auto ex = [&](long long el, int f) {
    double v = E[(long long)(g.own_off[f] + j) * g.ld + el];
    if (E2) v += E2[(long long)(g.own_off[f] + j) * g.ld + el];
    return v;
  };
  auto proj_g = [&]() {
    double v = 0.0;
    for (int q = 0; q < g.nqf; ++q) v += op.Pg[j * g.nqf + q] * src.g[bf * g.nqf + q];
    return v;
  };
  double v = 0.0;
  if (pde == 0) {
    const double b = a == 0 ? beta0 : (a == 1 ? beta1 : beta2);
    if (b > 0) v = (L >= 0) ? ex(L, fL) : proj_g();
    else if (b < 0) v = (R >= 0) ? ex(R, fR) : proj_g();
    else {
      const double* fvL = op.facevol + fL * g.nf;
      const double* fvR = op.facevol + fR * g.nf;
      if (L >= 0 && R >= 0) v = 0.5 * (u[L * g.nvol + (int)fvL[j]] + u[R * g.nvol + (int)fvR[j]]);
      else if (L >= 0) v = u[L * g.nvol + (int)fvL[j]];
      else v = u[R * g.nvol + (int)fvR[j]];
    }
  } else if (pde == 1) {
    const double al = a == 0 ? al0 : (a == 1 ? al1 : al2);
    if (L >= 0 && R >= 0) v = (ex(L, fL) + ex(R, fR)) / al;
    else v = proj_g();
  } else {
    if (L >= 0 && R >= 0) v = ex(L, fL) + ex(R, fR);
    else if (L >= 0) v = 2.0 * ex(L, fL);
    else v = 2.0 * ex(R, fR);
  }
  tr[idx] = v;
}

__global__ void k_ctrl_init(Ctrl* c, double tol, double div, int max_iters, int inner_max, double inner_rtol,
                            long long wait_cycles, int stall_block) {
  c->ticket = 0u;
  c->done = 0;
  c->status = 4;
  c->iter = 0;
  c->fp64_sweeps = 0;
  c->lowp_sweeps = 0;
  c->inner_done = 0;
  c->inner_iter = 0;
  c->outer = 0;
  c->max_iters = max_iters;
  c->inner_max = inner_max;
  c->timeout = 0;
  c->bar_count = 0u;
  c->bar_gen = 0u;
  c->wait_cycles = wait_cycles;
  c->stall_block = stall_block;
  c->tol = tol;
  c->diverge_factor = div;
  c->inner_rtol = inner_rtol;
  c->res = 0.0;
  c->res_min = 1e300;
  c->rnorm = 0.0;
  c->inner_step = 0.0;
}

inline unsigned grid_for(long long n) { return (unsigned)((n + BS - 1) / BS); }

template <int NF, int NLF>
cudaError_t run_first_t(const LaunchArgs& a) {
  size_t smem = (size_t)a.g.nvol * BS * sizeof(double);
  auto kern = k_first<NF, NLF>;
  if (smem > 32 * 1024) {
    cudaError_t e = allow_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid_for(a.g.nel), BS, smem, a.stream>>>(a.g, a.op, a.V, a.u0, a.F, a.ring, a.ring_stride, a.ctrl, a.partials, a.res_hist);
  return cudaGetLastError();
}

template <int NF, int NLF>
cudaError_t run_sweep64_t(const LaunchArgs& a, int count) {
  constexpr int NIN = NF * NLF;
  size_t smem = ((size_t)a.g.n_exp * NIN + NIN * (NIN + 1) / 2 + (size_t)NIN * BS) * sizeof(double);
  auto kern = k_sweep64<NF, NLF>;
  if (smem > 32 * 1024) {
    cudaError_t e = allow_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
  }
  for (int i = 0; i < count; ++i)
    kern<<<grid_for(a.g.nel), BS, smem, a.stream>>>(a.g, a.op, a.F, a.ring, a.ring_stride, a.ctrl, a.partials, a.res_hist);
  return cudaGetLastError();
}

// One cooperative launch of the whole float64 loop when the grid is co-resident; returns
// cudaErrorNotSupported (nothing launched) otherwise.
template <int NF, int NLF>
cudaError_t run_sweep64_persist_t(const LaunchArgs& a) {
  constexpr int NIN = NF * NLF;
  size_t smem = ((size_t)a.g.n_exp * NIN + NIN * (NIN + 1) / 2 + (size_t)NIN * BS) * sizeof(double);
  auto kern = k_sweep64_persist<NF, NLF>;
  if (smem > 32 * 1024) {
    cudaError_t e = allow_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BS, smem);
  if (e != cudaSuccess) return e;
  const long long grid = grid_for(a.g.nel);
  if (per < 1 || grid > (long long)per * sms || grid > partials_needed(a.g.nel) / 2 - 1) return cudaErrorNotSupported;
  e = cudaMemsetAsync(&a.ctrl->bar_count, 0, sizeof(unsigned), a.stream);
  if (e != cudaSuccess) return e;
  DevGeo gg = a.g;
  OpsDev oo = a.op;
  const double* ff = a.F;
  double* rr = a.ring;
  long long rs = a.ring_stride;
  Ctrl* ct = a.ctrl;
  double* pp = a.partials;
  double* rh = a.res_hist;
  void* args[] = {&gg, &oo, &ff, &rr, &rs, &ct, &pp, &rh};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid), dim3(BS), args, smem, a.stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int NF, int NLF>
cudaError_t run_reconstruct_t(const LaunchArgs& a, const double* E, const double* E2, double* u) {
  k_reconstruct<NF, NLF><<<grid_for(a.g.nel), BS, 0, a.stream>>>(a.g, a.op, a.V, E, E2, u);
  return cudaGetLastError();
}

// dispatch over the built (dim, p) shapes
template <template <int, int> class Fn, typename... Args>
cudaError_t dispatch(const DevGeo& g, Args&&... args) {
  if (g.dim == 2) {
    switch (g.nf) {
      case 2: return Fn<2, 4>::run(args...);
      case 3: return Fn<3, 4>::run(args...);
      case 4: return Fn<4, 4>::run(args...);
      case 5: return Fn<5, 4>::run(args...);
    }
  } else {
    switch (g.nf) {
      case 4: return Fn<4, 6>::run(args...);
      case 9: return Fn<9, 6>::run(args...);
    }
  }
  return cudaErrorNotSupported;
}

// Several problems of one element shape in one cooperative launch of the persistent float64
// loop.  NotSupported when their blocks together are not co-resident.
template <int NF, int NLF>
cudaError_t run_sweep64_persist_group_t(const LaunchArgs* a, int n, void* d_desc, cudaStream_t st) {
  constexpr int NIN = NF * NLF;
  size_t smem = 0;
  std::vector<P64Args> items((size_t)n);
  std::vector<int> off((size_t)n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const size_t sm = ((size_t)a[i].g.n_exp * NIN + NIN * (NIN + 1) / 2 + (size_t)NIN * BS) * sizeof(double);
    smem = sm > smem ? sm : smem;
    const long long grid = grid_for(a[i].g.nel);
    if (grid > partials_needed(a[i].g.nel) / 2 - 1) return cudaErrorNotSupported;
    off[(size_t)i + 1] = off[(size_t)i] + (int)grid;
    items[(size_t)i] = {a[i].g, a[i].op, a[i].F, a[i].ring, a[i].ring_stride, a[i].ctrl, a[i].partials, a[i].res_hist};
  }
  auto kern = k_sweep64_persist_group<NF, NLF>;
  if (smem > 32 * 1024) {
    cudaError_t e = allow_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BS, smem);
  if (e != cudaSuccess) return e;
  if (per < 1 || off[(size_t)n] > per * sms) return cudaErrorNotSupported;
  for (int i = 0; i < n; ++i) {
    e = cudaMemsetAsync(&a[i].ctrl->bar_count, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
  }
  P64Args* d_items = static_cast<P64Args*>(d_desc);
  int* d_off = reinterpret_cast<int*>(static_cast<char*>(d_desc) + sweep64_group_desc_items_bytes(n));
  e = cudaMemcpyAsync(d_items, items.data(), sizeof(P64Args) * (size_t)n, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(d_off, off.data(), sizeof(int) * ((size_t)n + 1), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const P64Args* ci = d_items;
  const int* co = d_off;
  int nn = n;
  void* args[] = {&ci, &co, &nn};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)off[(size_t)n]), dim3(BS), args, smem, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
template <int NF, int NLF> struct Sweep64GroupFn {
  static cudaError_t run(const LaunchArgs* a, int n, void* d_desc, cudaStream_t st) {
    return run_sweep64_persist_group_t<NF, NLF>(a, n, d_desc, st);
  }
};

template <int NF, int NLF>
cudaError_t run_kry_apply_t(const LaunchArgs& a, const double* v, const double* F, double s, double* w, const int* done) {
  const size_t smem = (size_t)a.g.n_exp * NF * NLF * sizeof(double);
  k_kry_apply<NF, NLF><<<grid_for(a.g.nel), BS, smem, a.stream>>>(a.g, a.op, v, F, s, w, done);
  return cudaGetLastError();
}
template <int NF, int NLF> struct KryApplyFn {
  static cudaError_t run(const LaunchArgs& a, const double* v, const double* F, double s, double* w, const int* done) {
    return run_kry_apply_t<NF, NLF>(a, v, F, s, w, done);
  }
};
template <int NF, int NLF> struct FirstFn { static cudaError_t run(const LaunchArgs& a) { return run_first_t<NF, NLF>(a); } };
template <int NF, int NLF> struct Sweep64Fn { static cudaError_t run(const LaunchArgs& a, int n) { return run_sweep64_t<NF, NLF>(a, n); } };
template <int NF, int NLF> struct Sweep64PersistFn { static cudaError_t run(const LaunchArgs& a) { return run_sweep64_persist_t<NF, NLF>(a); } };
template <int NF, int NLF> struct ReconFn {
  static cudaError_t run(const LaunchArgs& a, const double* E, const double* E2, double* u) { return run_reconstruct_t<NF, NLF>(a, E, E2, u); }
};

}  // namespace

bool shape_supported(int dim, int nf) {
  return (dim == 2 && nf >= 2 && nf <= 5) || (dim == 3 && (nf == 4 || nf == 9));
}

cudaError_t launch_ctrl_init(const LaunchArgs& a, double tol, double div, int max_iters, int inner_max, double inner_rtol,
                             long long wait_cycles, int stall_block) {
  k_ctrl_init<<<1, 1, 0, a.stream>>>(a.ctrl, tol, div, max_iters, inner_max, inner_rtol, wait_cycles, stall_block);
  return cudaGetLastError();
}
cudaError_t launch_forcing(const LaunchArgs& a) {
  const int nin = a.g.steady ? a.g.nqv : a.g.nvol;
  const size_t smem = (size_t)nin * (BS + 1) * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = allow_dynamic_smem(k_forcing);
    if (e != cudaSuccess) return e;
  }
  k_forcing<<<grid_for(a.g.nel), BS, smem, a.stream>>>(a.g, a.op, a.src, a.F, a.V);
  return cudaGetLastError();
}
cudaError_t launch_export0(const LaunchArgs& a, const double* u0, double* E0) {
  k_export0<<<grid_for(a.g.nel), BS, 0, a.stream>>>(a.g, a.op, u0, E0);
  return cudaGetLastError();
}
cudaError_t launch_first(const LaunchArgs& a) { return dispatch<FirstFn>(a.g, a); }
cudaError_t launch_sweep64(const LaunchArgs& a, int count) { return dispatch<Sweep64Fn>(a.g, a, count); }
cudaError_t launch_sweep64_persist(const LaunchArgs& a) { return dispatch<Sweep64PersistFn>(a.g, a); }
size_t sweep64_group_desc_items_bytes(int n) { return ((sizeof(P64Args) * (size_t)n) + 255) / 256 * 256; }
size_t sweep64_group_desc_bytes(int n) { return sweep64_group_desc_items_bytes(n) + ((sizeof(int) * ((size_t)n + 1)) + 255) / 256 * 256; }
cudaError_t launch_sweep64_persist_group(const LaunchArgs* a, int n, void* d_desc, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  for (int i = 1; i < n; ++i)
    if (a[i].g.dim != a[0].g.dim || a[i].g.nf != a[0].g.nf) return cudaErrorInvalidValue;
  return dispatch<Sweep64GroupFn>(a[0].g, a, n, d_desc, st);
}
cudaError_t launch_kry_apply(const LaunchArgs& a, const double* v, const double* F, double s, double* w, const int* done) {
  return dispatch<KryApplyFn>(a.g, a, v, F, s, w, done);
}
cudaError_t launch_reconstruct(const LaunchArgs& a, const double* E, const double* E2, double* u) {
  return dispatch<ReconFn>(a.g, a, E, E2, u);
}
cudaError_t launch_trace_out(const LaunchArgs& a, const double* E, const double* E2, const double* u, int pde,
                             const double* beta, const double* alpha, long long nface, double* tr) {
  long long n = nface * a.g.nf;
  k_trace_out<<<grid_for(n), BS, 0, a.stream>>>(a.g, a.op, a.src, E, E2, u, pde, beta[0], beta[1], beta[2],
                                                alpha[0], alpha[1], alpha[2], nface, tr);
  return cudaGetLastError();
}
// Crank-Nicolson step of a linear autonomous system from its backward-Euler half step:
// q^{m+1} = 2 q^{m+1/2} - q^m, elementwise (grid-stride, coalesced float64).
__global__ void __launch_bounds__(256) k_cn_extrapolate(double* __restrict__ q, const double* __restrict__ qh, long long n) {
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
    q[i] = 2.0 * qh[i] - q[i];
}

cudaError_t launch_cn_extrapolate(double* q, const double* qh, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_cn_extrapolate<<<(unsigned)blocks, 256, 0, s>>>(q, qh, n);
  return cudaGetLastError();
}

// two halves (ping-pong) of one slot per block; at least 512 blocks, so that the persistent
// kernels may size their grids by SM count on small meshes too
int partials_needed(long long nel) {
  const long long g = grid_for(nel);
  return 2 * (int)(g > 512 ? g : 512) + 2;
}

}  // namespace ihdg
