// Mixed-precision iHDG sweep loop (internal header).
//
// Defect correction around the float64 iteration E <- S(E) = F + L_E t(E):
//   outer (float64):  E' = E + e,  r = S(E') - E'                      (k_outer64)
//   check (float64):  res = ||u(S(E')) - u(E')|| = sqrt(t(r)^T Q t(r))  (k_inner_first)
//   inner (low):      e <- r + L_E t(e), from e = r, until the step is small  (k_inner)
// The float64 residual is the paper's stopping quantity (Section 5.1) evaluated for the
// next exact sweep from the current state; the output is u(E') with the trace of S(E').
#pragma once
#include <string>

#include "../../include/ihdg.h"
#include "ihdg_kernels.h"

namespace ihdg {

constexpr size_t MIXED_LT_BYTES = 16384;   // operator scratch in the mixed workspace

struct MixedLayout {
  size_t rlp, e0, e1, lt, total;   // byte offsets inside the mixed region
  int lp_bytes;                // bytes per low-precision value
  long long pad = 0;           // guard values before and after each correction array
};

struct MixedArgs {
  LaunchArgs base;
  double* E64;          // two float64 export slots (ring slots 1 and 2), stride base.ring_stride
  double* r64;          // float64 residual (ring slot 0)
  void* rlp;            // low-precision residual
  void* e[2];           // low-precision correction, ping-pong
  int prec;
  int max_grid = 1 << 30;   // cap on the persistent kernel's grid (tests shrink it)
  int no_tile = 0;          // 1: skip the shared-memory-resident tile kernel
  int slots = 0;            // length of the partials array (64-bit slots)
  int tile_lpe = 4;         // 4: 2D meshes use the register-resident kernel when it fits
  float* dLT = nullptr;     // device scratch for the transposed operator (register kernel)
  int reg_nt = 1024;        // register kernel block size (1024: one block per SM; or 512)
  int use_tc = 0;           // bf16: local apply on the tensor cores (tcgen05)
  int lt_kind = 0;          // operator layout now in dLT: 0 none, 1 register kernel, 2 tensor-core B
  int blk_h = 0;            // >= 2: 2D CUDA-core inner sweeps temporally blocked, this many per barrier
  int blk_rank = 0;         // which tile shape of the blocked kernel (0: smallest tile + halo area)
  const float* LE32h = nullptr;  // host copy of the float32 operator (n_exp x n_in)
  int ran = 0;              // inner kernel of the last inner launch (ihdg_result.inner_kernel_used codes)
  long long e_pad = 0;      // guard values below e[0], e[1] and above their last slot
  int tc_staged = 0;        // the last tensor-core launch ran the staged-gather variant
};

// One launch of the mixed loop's kernel `which` (0 outer float64 sweep, 1 residual check + first
// inner sweep, 2 persistent inner loop) with TL low-precision storage; defined in
// ihdg_mixed_kern.cuh and instantiated in ihdg_mixed_f32.cu and ihdg_mixed_bf16.cu.
template <typename TL>
cudaError_t mixed_launch(MixedArgs& m, int which, int has_e, int count);

MixedLayout mixed_layout(const DevGeo& g, int prec);
void mixed_bind(MixedArgs& m, char* region, const MixedLayout& L, int prec);
// Runs the outer/inner loop after the first float64 sweep.  On return, (Eu, Eu2) are the
// exports whose traces feed the final local solve, and (Et, Et2) the exports of u^K.
ihdg_status run_mixed(Ctrl* h_ctrl, MixedArgs& m, const ihdg_options& o, const double** Eu, const double** Eu2,
                      const double** Et, const double** Et2, std::string& err, SweepTimer* tm);

}  // namespace ihdg
