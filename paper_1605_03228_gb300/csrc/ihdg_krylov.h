// GMRES around the float64 iHDG sweep (internal header).
//
// The paper (Section 4.2, closing remark) proposes the iHDG iteration as a fine-scale
// preconditioner inside a Krylov method such as GMRES for problems on which the plain
// iteration does not converge.  In the export-state form one float64 sweep is the affine map
// E -> T E + F (T E = L_E t(E)); its fixed point solves (I - T) E = F, and GMRES is applied to
// that system: restarted GMRES(m) of Saad and Schultz, with classical Gram-Schmidt run twice
// (two passes of block dot products and updates, the GPU-friendly equivalent of the modified
// process up to rounding) and Givens rotations of the Hessenberg column by one thread.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "ihdg_kernels.h"

namespace ihdg {

// Loop state of the Krylov solve, in device memory (read back between batches of steps).
struct KryState {
  int done;        // 1: the solve has stopped; every step kernel returns at once
  int status;      // ihdg_status
  int j;           // Arnoldi steps completed in the current cycle
  int iters;       // Arnoldi steps in all (one homogeneous sweep each)
  int m, max_iters, first, pad_;
  double tol;      // stop when the residual estimate <= tol * bnorm
  double bnorm;    // residual norm at the start of the solve
  double beta;     // residual norm at the start of the cycle
  double res;      // current residual estimate |g_{j}|
  double inv;      // scale of the next basis vector (1 / its norm; 0 after a breakdown)
  double res_true; // ||F - (I - T) E||_2 / bnorm of the returned E
};

// Bytes of the Krylov scratch of one solve with n_vec = n_exp * ld unknowns, restart m.
size_t krylov_bytes(long long n_vec, int m);

struct KryOut {
  int iters = 0, status = 0, launches = 0;
  double res_true = 0.0;
};

// GMRES(m) on (I - T) E = F.  E (n_exp x ld, device) is the initial guess on entry (the
// exports of u0, or zeros) and the solution on return; scratch: krylov_bytes(n_exp * ld, m)
// bytes; tmp: one export vector of scratch for the final true residual.
cudaError_t run_krylov(const LaunchArgs& a, int m, double tol, int max_iters, double* E, double* tmp, void* scratch,
                       KryOut* out, std::string& err);

}  // namespace ihdg
