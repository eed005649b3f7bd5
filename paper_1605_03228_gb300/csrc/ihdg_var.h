// Transport with a velocity field beta(x) that varies in space (internal header).
//
// Section 3 states transport for a beta that is continuous across the skeleton, and the
// experiments of Section 5.1 (Table 1) use such fields.  Every element then has its own local
// matrix, so the local solve is precomputed per element (float64, on the host, threads over
// elements) and the device state is the volume solution itself, Algorithm 1 as written:
//     u_K^{k+1} = V_K + L_K t_K(u^k),   V_K = A_K^{-1} b_K,   L_K = A_K^{-1} G_K,
// where t_K are the trace values on K's faces at the face GLL nodes (the upwind element's
// nodal values: the element's own on outflow faces, the neighbour's on inflow faces, zero on
// the inflow boundary whose data enter b_K).  The local equation is (transportLocalk1) in its
// integrated-by-parts form
//     (beta.grad u, v)_K + <|beta.n| (u - u_hat^k), v>_dK = (f, v)_K,
// equal to the printed form under exact integration, with beta sampled at the Gauss points.
// The device path needs one flow direction per axis (beta_a >= 0 everywhere or <= 0
// everywhere), so that every element face is an inflow or an outflow face as a whole.
#pragma once
#include <string>
#include <vector>

#include "../../include/ihdg.h"

namespace ihdg {

struct VarHost {
  int dim = 0, p = 0, nb1 = 0, nb = 0, nf = 0, nlf = 0, nin = 0, q = 0, nqv = 0, nqf = 0;
  int n[3] = {1, 1, 1};
  long long nel = 0, nface = 0, nbface = 0;
  int sign[3] = {0, 0, 0};    // flow direction along each axis (+1, -1, or 0: beta_a = 0)
  int kind[6] = {0, 0, 0, 0, 0, 0};  // per local face: 1 outflow (own values), 2 inflow, 0 none
  double jac = 0.0;           // volume Jacobian (h/2)^d
  std::vector<double> L;      // per element [k][i]: L_K = A_K^{-1} G_K, nin x nb
  std::vector<double> Ainv;   // per element [j][i]: A_K^{-1}, nb x nb
  std::vector<double> Wq;     // [i][g]: (f, phi_i)_K weights, nb x nqv
  std::vector<double> FBv;    // [f][i][g]: phi_i at local face f's Gauss points, nlf x nb x nqf
  std::vector<double> bw;     // [bface][g]: |beta.n| times the face weight on inflow boundary
                              // faces, 0 on outflow boundary faces
  std::vector<int> facevol;   // [f][r]: volume node of face node r of local face f
  std::vector<double> M1;     // 1D GLL mass matrix on [-1, 1], nb1 x nb1
  std::vector<double> Pg;     // [r][g]: face Gauss values -> L2-projected face nodal values
  std::vector<long long> bel; // boundary face -> element
  std::vector<int> blf;       //               -> local face
};

// Validate and build every element's operators from beta sampled at the volume Gauss points
// (beta_vol [n_el][q^dim][dim]) and at the Gauss points of every global face (beta_face
// [n_face][q^(dim-1)][dim]).
ihdg_status build_var(const ihdg_mesh& mesh, const double* beta_vol, const double* beta_face, VarHost& v,
                      std::string& err);

}  // namespace ihdg

// ---------------------------------------------------------------------------------------
// Device side (ihdg_var.cu).
#include <cuda_runtime.h>

#include "ihdg_dev.h"

namespace ihdg {

// A plan on the device: the per-element operators (float64, float32 and bf16 copies of L_K,
// float64 A_K^{-1}), the shared tables, and the solve workspace.  Owned by the C-ABI plan.
struct VarDev {
  int dim = 0, p = 0, nb = 0, nf = 0, nlf = 0, nin = 0, nqv = 0, nqf = 0, nb1 = 0;
  int n[3] = {1, 1, 1};
  long long nel = 0, nface = 0, nbface = 0;
  int sign[3] = {0, 0, 0};
  int kind[6] = {0, 0, 0, 0, 0, 0};
  double jac = 0.0;
  void* mem = nullptr;          // one device allocation holding everything below
  size_t bytes = 0;
  const double* L64 = nullptr;  // [K][k][i]
  const float* L32 = nullptr;   // [K][k][i], each element's block padded to lsb32 bytes
  const void* L16 = nullptr;    // bf16, padded to lsb16 bytes
  int lsb32 = 0, lsb16 = 0;
  const double* Ainv = nullptr; // [K][j][i]
  const double* Wq = nullptr;   // [i][g]
  const double* FBv = nullptr;  // [f][i][g]
  const double* bw = nullptr;   // [bface][g]
  const int* facevol = nullptr; // [f][r]
  const double* M1 = nullptr;   // nb1 x nb1
  const double* Pg = nullptr;   // [r][g]
  // workspace
  double* u[2] = {nullptr, nullptr};   // volume state ping-pong, [K][i]
  double* V = nullptr;                 // A_K^{-1} b_K
  double* r64 = nullptr;               // mixed: float64 residual S(u') - u'
  void* rlp = nullptr;                 // mixed: low-precision residual (float32 or bf16)
  void* e[2] = {nullptr, nullptr};     // mixed: low-precision correction ping-pong
  Ctrl* ctrl = nullptr;
  double* partials = nullptr;          // 2 doubles per block
  double* res_hist = nullptr;          // max_hist + 2 doubles
  int grid = 0, max_hist = 0;
};

// Allocate and upload a plan (operators built by build_var); on failure nothing stays allocated.
cudaError_t var_upload(const VarHost& h, VarDev& d, int max_hist);
void var_free(VarDev& d);
// One solve on `stream`: forcing, the float64 sweep loop or the mixed loop, u_out and the
// trace (may be null).  h_ctrl: pinned host copy of the loop state.
ihdg_status var_solve(VarDev& d, const double* f_qp, const double* g_qp, const ihdg_options& o, double* u_out,
                      double* trace_out, cudaStream_t stream, Ctrl* h_ctrl, std::string& err, ihdg_result* res);

// Several plans solved together with one grouped launch per (dim, p) class per sweep step;
// each plan's result is the one of its own solve (same grids, reductions and decisions).
// solve_ms of every result is the group's device time.
ihdg_status var_solve_group(std::vector<VarDev*>& plans, const std::vector<const double*>& f_qp,
                            const std::vector<const double*>& g_qp, const ihdg_options& o,
                            const std::vector<double*>& u_out, const std::vector<double*>& trace_out,
                            cudaStream_t stream, std::string& err, ihdg_result* res);

}  // namespace ihdg
