// Kernel launch interface of the iHDG sweep (internal header).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "ihdg_dev.h"

namespace ihdg {

// Device copies of the float64 operators (see Ops in ihdg_ops.h), row-major.
struct OpsDev {
  const double* LE;      // n_exp x n_in
  const double* Qp;      // packed upper triangle of Q, off-diagonals doubled
  const double* Lvol;    // nvol x n_in
  const double* R;       // n_exp x nvol
  const double* Mn;      // nvol x nvol
  const double* PF;      // n_exp x nqv
  const double* PV;      // nvol x nqv
  const double* PFb[6];  // n_exp x nqf
  const double* PVb[6];  // nvol x nqf
  const double* Pg;      // nf x nqf
  const double* PqF;     // n_exp x nvol
  const double* PqV;     // nvol x nvol
  const double* facevol; // nlf x nf
  const float* LE32;     // n_exp x n_in, float32 copy for the low-precision sweeps
  const double* Mb;      // nb x nb element mass matrix
  double wcomp[4];       // per-component weight of the stopping norm
};

// Problem data: steady forcing/boundary data, or shallow-water step data q^m.
struct SrcDev {
  const double* f;   // [nel][nqv]
  const double* g;   // [n_bface][nqf]
  const double* q;   // [nel][nvol]
};

struct LaunchArgs {
  DevGeo g;
  OpsDev op;
  SrcDev src;
  const double* u0;       // initial guess (volume layout) or nullptr
  double* F;              // export forcing, n_exp x ld
  double* V;              // volume source A^{-1} b, nvol x ld (computed once with F)
  double* ring;           // three export slots of n_exp x ld
  long long ring_stride;  // = n_exp * ld
  Ctrl* ctrl;
  double* partials;       // one per block of the element kernels
  double* res_hist;       // residual after each sweep (index = sweep number), or nullptr
  cudaStream_t stream;
};

// Optional per-launch device timing of the sweep kernels (events around each launch).
struct SweepTimer {
  bool on = false;
  double fp64_ms = 0.0, lowp_ms = 0.0;
  int fp64_n = 0, lowp_n = 0;
  cudaEvent_t a = nullptr, b = nullptr;
  int launches = 0;   // every kernel launch of the solve (counted by the host drivers)
};

bool shape_supported(int dim, int nf);
// NVTX range for profilers (header-only NVTX 3: nothing happens unless a tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

int partials_needed(long long nel);

cudaError_t launch_ctrl_init(const LaunchArgs& a, double tol, double div, int max_iters, int inner_max, double inner_rtol,
                             long long wait_cycles, int stall_block);
cudaError_t launch_forcing(const LaunchArgs& a);
cudaError_t launch_export0(const LaunchArgs& a, const double* u0, double* E0);
cudaError_t launch_first(const LaunchArgs& a);
cudaError_t launch_sweep64(const LaunchArgs& a, int count);
// the whole float64 loop in one cooperative launch; cudaErrorNotSupported when the grid is
// not co-resident (then launch_sweep64 in batches)
cudaError_t launch_sweep64_persist(const LaunchArgs& a);
// the persistent float64 loops of n problems of one element shape (dim, nf) in one cooperative
// launch (bitwise each problem's own launch); d_desc: device scratch of
// sweep64_group_desc_bytes(n) for the launch's descriptors.  NotSupported when the problems'
// blocks together are not co-resident.
size_t sweep64_group_desc_items_bytes(int n);
size_t sweep64_group_desc_bytes(int n);
cudaError_t launch_sweep64_persist_group(const LaunchArgs* a, int n, void* d_desc, cudaStream_t st);
// w = s (I - T) v + F on the live export rows, T the linear part of one float64 sweep (F may
// be null); nothing happens when *done (device) is set
cudaError_t launch_kry_apply(const LaunchArgs& a, const double* v, const double* F, double s, double* w, const int* done);
cudaError_t launch_reconstruct(const LaunchArgs& a, const double* E, const double* E2, double* u);
// q <- 2 qh - q over n values (the Crank-Nicolson step from the backward-Euler half step qh)
cudaError_t launch_cn_extrapolate(double* q, const double* qh, long long n, cudaStream_t s);
cudaError_t launch_trace_out(const LaunchArgs& a, const double* E, const double* E2, const double* u, int pde,
                             const double* beta, const double* alpha, long long nface, double* tr);

}  // namespace ihdg
