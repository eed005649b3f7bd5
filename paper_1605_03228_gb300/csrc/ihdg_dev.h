// Device-side data structures of the iHDG sweep (internal header, host and device).
#pragma once
#include <cstdint>

namespace ihdg {

// Geometry and gather description of one problem, passed to kernels by value.
struct DevGeo {
  int dim, nf, nlf, n_in, n_exp, nvol, nqv, nqf, nb;
  int n[3];
  long long nel;
  long long ld;           // slot stride of every per-element array (>= nel, multiple of 32)
  long long stride[3];    // element-number step along each axis
  long long nbf_off[3];   // first boundary-face number of each axis group
  int kind[6], own_off[6], nbr_off[6];
  int bc_mirror;
  int steady;             // 1: forcing from (f, g); 0: shallow-water step data q^m
  int per_axis;           // export slot = axis * nf + node (transport) / face * nf + node
  unsigned long long live;  // bit e: export slot e carries a value (n_exp <= 64)
};

// Loop state of one solve, in device memory.  Written only by the last block of each
// reducing kernel (see finish_reduction), read by every kernel at its start.
struct Ctrl {
  unsigned int ticket;    // arrival counter of the current reducing kernel
  int done;               // 1: the loop has stopped (every sweep kernel returns at once)
  int status;             // ihdg_status of the loop
  int iter;               // sweeps completed (k); E^k lives in ring slot iter % 3
  int fp64_sweeps, lowp_sweeps;
  int inner_done;         // mixed: current inner solve has stopped
  int inner_iter;         // mixed: inner sweeps in the current outer step
  int outer;              // mixed: outer steps completed
  int max_iters;
  int inner_max;
  int timeout;            // a bounded device wait ran out (the loop stops, status ERR_TIMEOUT)
  unsigned int bar_gen;   // (unused)
  long long wait_cycles;  // bound of every grid-barrier wait, in SM clock cycles
  int stall_block;        // test hook: this block never arrives at the grid barrier (-1: none)
  double tol, diverge_factor, inner_rtol;
  double res;             // last float64 stopping residual
  double res_min;
  double rnorm;           // mixed: export-space norm of the current r (low precision check)
  double inner_step;      // mixed: last inner step norm
  // arrival counter of the persistent kernels' grid barrier, alone on its cache line: every
  // block polls it, so no other field may share the line
  alignas(128) unsigned int bar_count;
  unsigned int pad_[31];
};

enum { FK_NONE_D = 0, FK_OWN_D = 1, FK_NBR_D = 2, FK_SUM_D = 3 };

}  // namespace ihdg
