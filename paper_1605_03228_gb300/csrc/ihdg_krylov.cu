// GMRES(m) around the float64 iHDG sweep (see ihdg_krylov.h).  Vector kernels: block dot
// products against a set of basis vectors, their fixed-order sums, the Gram-Schmidt update
// with the norm of the result, scaling and the final combination x += V y; one-thread
// kernels for the Hessenberg column (Givens rotations), the cycle start and the triangular
// solve.  Every step kernel returns immediately after the solve has stopped
// (KryState::done), so the host launches steps in batches and reads the state back once per
// batch.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/ihdg.h"
#include "ihdg_common.cuh"
#include "ihdg_krylov.h"

namespace ihdg {

namespace {

constexpr int DBS = 256;  // threads per block of the vector kernels
constexpr int EPT = 4;    // values per thread (consecutive blocks of DBS, coalesced)

long long nblk_for(long long n) { return (n + (long long)DBS * EPT - 1) / ((long long)DBS * EPT); }
size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct KryLayout {
  size_t st, V, H, cs, sn, gv, y, h1, h2, part, total;
};

KryLayout kry_layout(long long n, int m) {
  KryLayout L{};
  size_t at = 0;
  auto take = [&](size_t bytes) { size_t r = at; at += a256(bytes); return r; };
  const size_t d = sizeof(double);
  L.st = take(sizeof(KryState));
  L.V = take(d * (size_t)(m + 1) * (size_t)n);
  L.H = take(d * (size_t)(m + 1) * (size_t)m);
  L.cs = take(d * (size_t)m);
  L.sn = take(d * (size_t)m);
  L.gv = take(d * (size_t)(m + 1));
  L.y = take(d * (size_t)m);
  L.h1 = take(d * (size_t)(m + 1));
  L.h2 = take(d * (size_t)(m + 1));
  L.part = take(d * (size_t)(m + 1) * (size_t)nblk_for(n));
  L.total = at;
  return L;
}

__device__ __forceinline__ bool kdone(const KryState* st) { return *(const volatile int*)&st->done != 0; }

__global__ void k_kry_init(KryState* st, int m, int max_iters, double tol) {
  KryState s{};
  s.m = m;
  s.max_iters = max_iters;
  s.first = 1;
  s.tol = tol;
  *st = s;
}

// part[i * nblk + block] = this block's share of V_i . w over its DBS * EPT values, i < nv.
// w's values are staged in shared memory; each warp takes one basis vector at a time (32
// independent coalesced loads per lane) and reduces with shuffles, so the loop over vectors
// has no block barrier.
__global__ void __launch_bounds__(DBS) k_kry_dots(const double* __restrict__ V, long long ldv, int nv,
                                                  const double* __restrict__ w, long long n, double* __restrict__ part,
                                                  int nblk, const KryState* st, int force) {
  constexpr int R = DBS * EPT;   // values per block
  constexpr int PL = R / 32;     // values per lane for one vector
  __shared__ double sw[R];
  if (!force && kdone(st)) return;
  const long long base = (long long)blockIdx.x * R;
  for (int t = threadIdx.x; t < R; t += DBS) sw[t] = base + t < n ? w[base + t] : 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool full = base + R <= n;
  for (int i = warp; i < nv; i += DBS / 32) {
    const double* vi = V + (long long)i * ldv + base;
    double acc = 0.0;
    if (full) {
#pragma unroll
      for (int k = 0; k < PL; ++k) acc += vi[lane + 32 * k] * sw[lane + 32 * k];
    } else {
      for (int k = 0; k < PL; ++k)
        if (base + lane + 32 * k < n) acc += vi[lane + 32 * k] * sw[lane + 32 * k];
    }
    acc = warp_sum(acc);
    if (lane == 0) part[(long long)i * nblk + blockIdx.x] = acc;
  }
}

// out[i] = sum over blocks of part[i * nblk + b], fixed order; one block per i
__global__ void __launch_bounds__(DBS) k_kry_sum(const double* __restrict__ part, int nblk, double* __restrict__ out,
                                                 const KryState* st) {
  __shared__ double ws[DBS / 32];
  if (kdone(st)) return;
  const double* p = part + (long long)blockIdx.x * nblk;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += DBS) acc += p[b];
  const double t = block_sum(acc, ws);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// w -= sum_{i < nv} h_i V_i (h staged in shared memory, nv doubles of dynamic shared memory;
// four basis vectors per unrolled step, so 16 loads per thread are in flight); with `part`,
// part[block] = this block's share of ||w||^2
__global__ void __launch_bounds__(DBS) k_kry_update(double* __restrict__ w, const double* __restrict__ V, long long ldv,
                                                    int nv, const double* __restrict__ h, long long n,
                                                    double* __restrict__ part, const KryState* st) {
  extern __shared__ double sh[];
  __shared__ double ws[DBS / 32];
  if (kdone(st)) return;
  for (int i = threadIdx.x; i < nv; i += DBS) sh[i] = h[i];
  __syncthreads();
  const long long base = (long long)blockIdx.x * (DBS * EPT) + threadIdx.x;
  double v[EPT];
  bool in[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    in[k] = base + (long long)k * DBS < n;
    v[k] = in[k] ? w[base + (long long)k * DBS] : 0.0;
  }
  int i = 0;
  for (; i + 4 <= nv; i += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double* vi = V + (long long)(i + u) * ldv + base;
      const double c = sh[i + u];
#pragma unroll
      for (int k = 0; k < EPT; ++k)
        if (in[k]) v[k] -= c * vi[k * DBS];
    }
  }
  for (; i < nv; ++i) {
    const double* vi = V + (long long)i * ldv + base;
    const double c = sh[i];
#pragma unroll
    for (int k = 0; k < EPT; ++k)
      if (in[k]) v[k] -= c * vi[k * DBS];
  }
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < EPT; ++k)
    if (in[k]) {
      w[base + (long long)k * DBS] = v[k];
      acc += v[k] * v[k];
    }
  if (part) {
    const double t = block_sum(acc, ws);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// Column j of the Hessenberg matrix (h1 + h2 from the two Gram-Schmidt passes, and the norm
// of the orthogonalised vector from `part`), reduced by the earlier rotations and a new one;
// the rotated right-hand side gives the residual estimate and the stopping decision.
__global__ void __launch_bounds__(DBS) k_kry_finish(KryState* st, const double* __restrict__ part, int nblk, int j,
                                                    double* H, double* cs, double* sn, double* gv,
                                                    const double* __restrict__ h1, const double* __restrict__ h2) {
  __shared__ double ws[DBS / 32];
  if (kdone(st)) return;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += DBS) acc += part[b];
  const double t = block_sum(acc, ws);
  if (threadIdx.x != 0) return;
  const int m = st->m;
  double* Hc = H + (long long)j * (m + 1);
  const double hn = sqrt(t);
  for (int i = 0; i <= j; ++i) Hc[i] = h1[i] + h2[i];
  Hc[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double p = Hc[i], q = Hc[i + 1];
    Hc[i] = cs[i] * p + sn[i] * q;
    Hc[i + 1] = -sn[i] * p + cs[i] * q;
  }
  const double den = hypot(Hc[j], Hc[j + 1]);
  cs[j] = den > 0.0 ? Hc[j] / den : 1.0;
  sn[j] = den > 0.0 ? Hc[j + 1] / den : 0.0;
  Hc[j] = den;
  Hc[j + 1] = 0.0;
  gv[j + 1] = -sn[j] * gv[j];
  gv[j] = cs[j] * gv[j];
  st->j = j + 1;
  st->iters += 1;
  const double res = fabs(gv[j + 1]);
  st->res = res;
  st->inv = hn > 0.0 ? 1.0 / hn : 0.0;
  if (!isfinite(res) || !isfinite(hn)) {
    st->status = IHDG_DIVERGED;
    st->done = 1;
  } else if (res <= st->tol * st->bnorm) {
    st->status = IHDG_OK;
    st->done = 1;
  } else if (st->iters >= st->max_iters) {
    st->status = IHDG_NOT_CONVERGED;
    st->done = 1;
  }
}

// v *= st->inv (the next basis vector's normalisation)
__global__ void __launch_bounds__(DBS) k_kry_scale(double* __restrict__ v, long long n, const KryState* st) {
  if (kdone(st)) return;
  const double s = st->inv;
  const long long base = (long long)blockIdx.x * (DBS * EPT) + threadIdx.x;
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const long long x = base + (long long)k * DBS;
    if (x < n) v[x] *= s;
  }
}

// Start of a cycle from part (the block shares of ||r||^2 of the residual in V_0): beta,
// the right-hand side beta e_1, the scale of V_0 and the check of the restarted residual.
__global__ void __launch_bounds__(DBS) k_kry_cycle(KryState* st, const double* __restrict__ part, int nblk, double* gv) {
  __shared__ double ws[DBS / 32];
  if (kdone(st)) return;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += DBS) acc += part[b];
  const double t = block_sum(acc, ws);
  if (threadIdx.x != 0) return;
  const double beta = sqrt(t);
  if (st->first) {
    st->bnorm = beta;
    st->first = 0;
  }
  gv[0] = beta;
  for (int i = 1; i <= st->m; ++i) gv[i] = 0.0;
  st->beta = beta;
  st->res = beta;
  st->j = 0;
  st->inv = beta > 0.0 ? 1.0 / beta : 0.0;
  if (!isfinite(beta)) {
    st->status = IHDG_DIVERGED;
    st->done = 1;
  } else if (beta <= st->tol * st->bnorm) {
    st->status = IHDG_OK;
    st->done = 1;
  }
}

// y = R^{-1} g over the st->j steps of the cycle (R: the rotated Hessenberg matrix)
__global__ void k_kry_solve_y(const KryState* st, const double* __restrict__ H, const double* __restrict__ gv,
                              double* __restrict__ y) {
  const int j = st->j, m = st->m;
  for (int i = j - 1; i >= 0; --i) {
    double v = gv[i];
    for (int k = i + 1; k < j; ++k) v -= H[(long long)k * (m + 1) + i] * y[k];
    const double d = H[(long long)i * (m + 1) + i];
    y[i] = d != 0.0 ? v / d : 0.0;   // d = 0 only after an exact breakdown of that column
  }
}

// x += sum_{i < st->j} y_i V_i (y staged in shared memory: m doubles of dynamic shared memory)
__global__ void __launch_bounds__(DBS) k_kry_combine(double* __restrict__ x, const double* __restrict__ V, long long ldv,
                                                     const double* __restrict__ y, long long n, const KryState* st) {
  extern __shared__ double sy[];
  const int j = st->j;
  for (int i = threadIdx.x; i < j; i += DBS) sy[i] = y[i];
  __syncthreads();
  const long long base = (long long)blockIdx.x * (DBS * EPT) + threadIdx.x;
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const long long p = base + (long long)k * DBS;
    if (p < n) {
      double v = x[p];
      for (int i = 0; i < j; ++i) v += sy[i] * V[(long long)i * ldv + p];
      x[p] = v;
    }
  }
}

// st->res_true = ||r|| / bnorm from the block shares of ||r||^2
__global__ void __launch_bounds__(DBS) k_kry_true(KryState* st, const double* __restrict__ part, int nblk) {
  __shared__ double ws[DBS / 32];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += DBS) acc += part[b];
  const double t = block_sum(acc, ws);
  if (threadIdx.x == 0) st->res_true = st->bnorm > 0.0 ? sqrt(t) / st->bnorm : sqrt(t);
}

}  // namespace

size_t krylov_bytes(long long n_vec, int m) { return kry_layout(n_vec, m).total; }

cudaError_t run_krylov(const LaunchArgs& a, int m, double tol, int max_iters, double* E, double* tmp, void* scratch,
                       KryOut* out, std::string& err) {
  const long long n = a.ring_stride;
  const long long nb64 = nblk_for(n);
  if (m < 1 || nb64 > 0x7fffffffLL) { err = "krylov: bad restart length or vector size"; return cudaErrorInvalidValue; }
  const int nblk = (int)nb64;
  const KryLayout L = kry_layout(n, m);
  char* base = static_cast<char*>(scratch);
  KryState* st = reinterpret_cast<KryState*>(base + L.st);
  double* V = reinterpret_cast<double*>(base + L.V);
  double* H = reinterpret_cast<double*>(base + L.H);
  double* cs = reinterpret_cast<double*>(base + L.cs);
  double* sn = reinterpret_cast<double*>(base + L.sn);
  double* gv = reinterpret_cast<double*>(base + L.gv);
  double* y = reinterpret_cast<double*>(base + L.y);
  double* h1 = reinterpret_cast<double*>(base + L.h1);
  double* h2 = reinterpret_cast<double*>(base + L.h2);
  double* part = reinterpret_cast<double*>(base + L.part);
  const cudaStream_t s = a.stream;
  const int* dn = &st->done;
  int launches = 0;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r, const char* where) {
    if (r == cudaSuccess) r = cudaGetLastError();
    if (r != cudaSuccess) { e = r; err = std::string("krylov ") + where + ": " + cudaGetErrorString(r); return false; }
    return true;
  };
  KryState hs{};
  auto readback = [&]() {
    return ok(cudaMemcpyAsync(&hs, st, sizeof(KryState), cudaMemcpyDeviceToHost, s), "state readback") &&
           ok(cudaStreamSynchronize(s), "steps");
  };
  // rows the operator never writes (dead export rows, padding columns) stay zero in every
  // basis vector and in the residual scratch
  if (!ok(cudaMemsetAsync(V, 0, sizeof(double) * (size_t)(m + 1) * (size_t)n, s), "memset") ||
      !ok(cudaMemsetAsync(tmp, 0, sizeof(double) * (size_t)n, s), "memset"))
    return e;
  k_kry_init<<<1, 1, 0, s>>>(st, m, max_iters, tol);
  if (!ok(cudaSuccess, "init")) return e;
  // r = F - (I - T) E in V_0, its norm, the cycle start, V_0 /= ||r||
  auto start_cycle = [&]() {
    if (!ok(launch_kry_apply(a, E, a.F, -1.0, V, dn), "residual")) return false;
    k_kry_dots<<<nblk, DBS, 0, s>>>(V, n, 1, V, n, part, nblk, st, 0);
    k_kry_cycle<<<1, DBS, 0, s>>>(st, part, nblk, gv);
    k_kry_scale<<<nblk, DBS, 0, s>>>(V, n, st);
    launches += 4;
    return ok(cudaSuccess, "cycle start");
  };
  // Arnoldi step j: V_{j+1} = (I - T) V_j, orthogonalised against V_0..V_j twice, normalised
  auto step = [&](int j) {
    double* w = V + (long long)(j + 1) * n;
    if (!ok(launch_kry_apply(a, V + (long long)j * n, nullptr, 1.0, w, dn), "apply")) return false;
    k_kry_dots<<<nblk, DBS, 0, s>>>(V, n, j + 1, w, n, part, nblk, st, 0);
    k_kry_sum<<<j + 1, DBS, 0, s>>>(part, nblk, h1, st);
    k_kry_update<<<nblk, DBS, sizeof(double) * (j + 1), s>>>(w, V, n, j + 1, h1, n, nullptr, st);
    k_kry_dots<<<nblk, DBS, 0, s>>>(V, n, j + 1, w, n, part, nblk, st, 0);
    k_kry_sum<<<j + 1, DBS, 0, s>>>(part, nblk, h2, st);
    k_kry_update<<<nblk, DBS, sizeof(double) * (j + 1), s>>>(w, V, n, j + 1, h2, n, part, st);
    k_kry_finish<<<1, DBS, 0, s>>>(st, part, nblk, j, H, cs, sn, gv, h1, h2);
    k_kry_scale<<<nblk, DBS, 0, s>>>(w, n, st);
    launches += 9;
    return ok(cudaSuccess, "step");
  };
  if (!start_cycle() || !readback()) return e;
  long long host_steps = 0;
  while (!hs.done) {
    int j = 0, batch = 4;
    while (j < m) {
      const int nb = batch < m - j ? batch : m - j;
      for (int b = 0; b < nb; ++b)
        if (!step(j + b)) return e;
      j += nb;
      host_steps += nb;
      if (!readback()) return e;
      if (hs.done) break;
      if (batch < 32) batch *= 2;
    }
    k_kry_solve_y<<<1, 1, 0, s>>>(st, H, gv, y);
    k_kry_combine<<<nblk, DBS, sizeof(double) * m, s>>>(E, V, n, y, n, st);
    launches += 2;
    if (!ok(cudaSuccess, "combine")) return e;
    if (hs.done) break;
    // the device stops at max_iters; this bound only guards the host loop
    if (host_steps > (long long)max_iters + m) { err = "krylov: the step loop did not stop"; return cudaErrorUnknown; }
    if (!start_cycle() || !readback()) return e;
  }
  // the true residual of the returned solution
  if (!ok(launch_kry_apply(a, E, a.F, -1.0, tmp, nullptr), "true residual")) return e;
  k_kry_dots<<<nblk, DBS, 0, s>>>(tmp, n, 1, tmp, n, part, nblk, st, 1);
  k_kry_true<<<1, DBS, 0, s>>>(st, part, nblk);
  launches += 3;
  if (!ok(cudaSuccess, "true residual") || !readback()) return e;
  out->iters = hs.iters;
  out->status = hs.status;
  out->res_true = hs.res_true;
  out->launches = launches;
  return cudaSuccess;
}

}  // namespace ihdg
