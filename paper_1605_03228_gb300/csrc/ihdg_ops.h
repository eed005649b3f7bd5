// Host-side float64 construction of the per-element iHDG operators (internal header).
//
// For a uniform mesh of congruent elements with constant coefficients, every element has
// the same local matrix A (Section 2, Eq. iHDGlocal), so the local solve is precomputed
// once: u^{k+1} = A^{-1}(b + G t^k), where t^k are the trace values an element gathers on
// its faces and b collects the forcing and boundary data.  The device state is not the
// volume solution but the "export" E: the values of u^{k+1} that the element's own and its
// neighbours' next local solves need on its faces:
//   transport:      u on outflow faces (Eq. transportLocale picks the upwind value),
//   conv.-diff.:    h = sigma.n + (alpha + beta.n)/2 u per face node, so that the trace of
//                   Section 4.1 is u_hat = (h^- + h^+) / alpha,
//   shallow water:  h = (phi + sqrt(Phi) vel.n)/2 per face node, so that
//                   phi_hat = {{phi}} + sqrt(Phi){{vel.n}} = h^- + h^+ (walls: 2 h^-).
// One sweep is then E^{k+1} = F + L_E t(E^k), with L_E = R A^{-1} G, and the paper's stopping
// quantity ||u^{k+1} - u^k||^2 = dt^T Q dt, Q = (A^{-1}G)^T M (A^{-1}G), dt = t(E^k) - t(E^{k-1}).
#pragma once
#include <string>
#include <vector>

#include "../../include/ihdg.h"

namespace ihdg {

enum FaceKind { FK_NONE = 0, FK_OWN = 1, FK_NBR = 2, FK_SUM = 3 };

struct Ops {
  int pde = 0, dim = 0, p = 0;
  int nb1 = 0, nb = 0, ncomp = 0, nvol = 0;
  int nf = 0;              // nodes per face, (p+1)^(dim-1)
  int q = 0, nqv = 0, nqf = 0;
  int nlf = 0;             // local faces, 2*dim
  int n_exp = 0, n_in = 0;
  // gather description per local face f = 2a + s (s = 0: -e_a, s = 1: +e_a)
  int face_kind[6] = {0, 0, 0, 0, 0, 0};
  int own_off[6] = {-1, -1, -1, -1, -1, -1};  // export offset of this element's block
  int nbr_off[6] = {-1, -1, -1, -1, -1, -1};  // export offset of the neighbour's opposite block
  int bc_mirror = 0;                          // boundary SUM faces: input = 2 * own
  int layout_per_axis = 0;                    // export slot = axis*nf + node (transport),
                                              // else face*nf + node
  double in_scale[6] = {1, 1, 1, 1, 1, 1};    // input scale folded into G (1/alpha for CD)
  // dense operators, row-major
  std::vector<double> LE;     // n_exp x n_in
  std::vector<double> Lvol;   // nvol x n_in
  std::vector<double> Q;      // n_in x n_in
  std::vector<double> R;      // n_exp x nvol   volume -> export
  std::vector<double> Mn;     // nvol x nvol    norm of the stopping test
  std::vector<double> Mb;     // nb x nb element mass matrix
  double wcomp[4] = {0, 0, 0, 0}; // Mn = blockdiag(wcomp[c] * Mb)
  std::vector<double> PF, PV; // n_exp x nqv, nvol x nqv    forcing -> export / volume
  std::vector<double> PFb[6], PVb[6];  // n_exp x nqf, nvol x nqf per local face (boundary data)
  std::vector<double> Pg;     // nf x nqf   boundary data -> L2-projected face nodal values
  std::vector<double> PqF, PqV;  // shallow water: q^m -> export / volume (n_exp x nvol, nvol x nvol)
  std::vector<double> facevol;   // nlf x nf: volume node index of each face node (as double)
  double alpha_axis[3] = {1, 1, 1};  // conv.-diff.: alpha per axis (|beta.n| only)
  double beta[3] = {0, 0, 0};
};

// Validate (mesh, coeffs) and fill `ops`.  Returns IHDG_OK or an error with `err` set.
ihdg_status build_ops(const ihdg_mesh& mesh, const ihdg_coeffs& co, Ops& ops, std::string& err);

// Geometry helpers shared by the C-ABI (host).
ihdg_status validate(const ihdg_mesh& mesh, const ihdg_coeffs* co, std::string& err);
void quadrature_points(const ihdg_mesh& mesh, double* vol_xyz, double* bnd_xyz);
void node_points(const ihdg_mesh& mesh, double* xyz);
long long count_faces(const ihdg_mesh& mesh, long long* n_bface);
// Per boundary face: (element, local face) in boundary-face order.
void boundary_faces(const ihdg_mesh& mesh, std::vector<long long>& elem, std::vector<int>& lf);
// Quadrature points of every global face, [n_face][q^(dim-1)][dim], global face order.
void face_points(const ihdg_mesh& mesh, double* xyz);

// 1D reference tables of order p: GLL nodes xn (p+1), Gauss points xg and weights wg
// (q = p+2), the Lagrange basis and its derivative at the Gauss points (Lg, Dg: q x (p+1),
// row-major) and the exact 1D mass matrix M1 ((p+1) x (p+1)) on [-1, 1].
struct RefTables {
  int p = 0, q = 0, nb1 = 0;
  std::vector<double> xn, xg, wg, Lg, Dg, M1;
};
RefTables ref_tables(int p);
// Dense LU with partial pivoting: solves A X = B (A n x n, B n x m, both row-major; B is
// overwritten with X).  Returns false for a singular A.
bool dense_solve(std::vector<double> A, int n, std::vector<double>& B, int m);

}  // namespace ihdg
