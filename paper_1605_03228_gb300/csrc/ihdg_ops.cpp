// Host-side float64 operator construction for the iHDG sweep (see ihdg_ops.h).
//
// Reference element: GLL nodes (roots of P_p' by Newton's method, plus the endpoints),
// Gauss-Legendre points (roots of P_q, q = p+2, by Newton's method), the barycentric form of
// the Lagrange basis, and the nodal differentiation matrix.  Element matrices are Kronecker
// products of exact 1D mass and derivative matrices; faces of a GLL element carry exactly the
// nodes with an end index along the face normal, so trace restriction is node selection.
#include "ihdg_ops.h"

#include <cmath>
#include <cstring>
#include <sstream>

namespace ihdg {
namespace {

// Legendre P_n and P_n' at x by the three-term recurrence.
void legendre(int n, double x, double& P, double& dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  // derivative from the recurrence for (x^2 - 1) P_n' = n (x P_n - P_{n-1})
  if (std::fabs(x * x - 1.0) < 1e-300) {
    dP = (x > 0 ? 1.0 : ((n % 2) ? 1.0 : -1.0)) * 0.5 * n * (n + 1.0);
  } else {
    dP = n * (x * p1 - p0) / (x * x - 1.0);
  }
}

struct Ref1D {
  int p = 0, q = 0, nb1 = 0;
  std::vector<double> xn, xg, wg, lam;
  std::vector<double> Lg;   // q x nb1: l_j(xg_a)
  std::vector<double> Dg;   // q x nb1: l_j'(xg_a)
  std::vector<double> M1;   // nb1 x nb1: int l_i l_j
  std::vector<double> S1;   // nb1 x nb1: int l_i' l_j
};

Ref1D make_ref(int p) {
  Ref1D r;
  r.p = p;
  r.nb1 = p + 1;
  r.q = p + 2;
  // GLL nodes: -1, roots of P_p', +1
  r.xn.assign(r.nb1, 0.0);
  r.xn[0] = -1.0;
  r.xn[p] = 1.0;
  for (int j = 1; j < p; ++j) {
    double x = -std::cos(M_PI * j / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, x, P, dP);
      double d2P = (2.0 * x * dP - p * (p + 1.0) * P) / (1.0 - x * x);
      double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    r.xn[j] = x;
  }
  // Gauss-Legendre points and weights
  r.xg.assign(r.q, 0.0);
  r.wg.assign(r.q, 0.0);
  for (int i = 0; i < r.q; ++i) {
    double x = -std::cos(M_PI * (i + 0.75) / (r.q + 0.5));
    double P = 0, dP = 1;
    for (int it = 0; it < 100; ++it) {
      legendre(r.q, x, P, dP);
      double dx = P / dP;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    legendre(r.q, x, P, dP);
    r.xg[i] = x;
    r.wg[i] = 2.0 / ((1.0 - x * x) * dP * dP);
  }
  // barycentric weights
  r.lam.assign(r.nb1, 1.0);
  for (int j = 0; j < r.nb1; ++j)
    for (int k = 0; k < r.nb1; ++k)
      if (k != j) r.lam[j] /= (r.xn[j] - r.xn[k]);
  // Lagrange values at Gauss points (second barycentric form; Gauss points are interior)
  r.Lg.assign(r.q * r.nb1, 0.0);
  for (int a = 0; a < r.q; ++a) {
    double den = 0.0;
    for (int k = 0; k < r.nb1; ++k) den += r.lam[k] / (r.xg[a] - r.xn[k]);
    for (int j = 0; j < r.nb1; ++j) r.Lg[a * r.nb1 + j] = (r.lam[j] / (r.xg[a] - r.xn[j])) / den;
  }
  // nodal differentiation matrix Dn[i][j] = l_j'(xn_i)
  std::vector<double> Dn(r.nb1 * r.nb1, 0.0);
  for (int i = 0; i < r.nb1; ++i) {
    double s = 0.0;
    for (int j = 0; j < r.nb1; ++j) {
      if (j == i) continue;
      Dn[i * r.nb1 + j] = (r.lam[j] / r.lam[i]) / (r.xn[i] - r.xn[j]);
      s += Dn[i * r.nb1 + j];
    }
    Dn[i * r.nb1 + i] = -s;
  }
  // l_j' is a polynomial of degree p-1, so it equals its nodal interpolant
  r.Dg.assign(r.q * r.nb1, 0.0);
  for (int a = 0; a < r.q; ++a)
    for (int j = 0; j < r.nb1; ++j) {
      double s = 0.0;
      for (int i = 0; i < r.nb1; ++i) s += r.Lg[a * r.nb1 + i] * Dn[i * r.nb1 + j];
      r.Dg[a * r.nb1 + j] = s;
    }
  r.M1.assign(r.nb1 * r.nb1, 0.0);
  r.S1.assign(r.nb1 * r.nb1, 0.0);
  for (int i = 0; i < r.nb1; ++i)
    for (int j = 0; j < r.nb1; ++j) {
      double m = 0.0, s = 0.0;
      for (int a = 0; a < r.q; ++a) {
        m += r.wg[a] * r.Lg[a * r.nb1 + i] * r.Lg[a * r.nb1 + j];
        s += r.wg[a] * r.Dg[a * r.nb1 + i] * r.Lg[a * r.nb1 + j];
      }
      r.M1[i * r.nb1 + j] = m;
      r.S1[i * r.nb1 + j] = s;
    }
  return r;
}

// Dense LU with partial pivoting; solves A X = B in place (B is n x m, row-major).
bool lu_solve(std::vector<double> A, int n, std::vector<double>& B, int m) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int pr = k;
    double best = std::fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > best) { best = std::fabs(A[i * n + k]); pr = i; }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    piv[k] = pr;
    if (pr != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[pr * n + j]);
      for (int j = 0; j < m; ++j) std::swap(B[k * m + j], B[pr * m + j]);
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / A[k * n + k];
      A[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
      for (int j = 0; j < m; ++j) B[i * m + j] -= l * B[k * m + j];
    }
  }
  for (int i = n - 1; i >= 0; --i)
    for (int j = 0; j < m; ++j) {
      double s = B[i * m + j];
      for (int k = i + 1; k < n; ++k) s -= A[i * n + k] * B[k * m + j];
      B[i * m + j] = s / A[i * n + i];
    }
  return true;
}

// C = A (r x k) * B (k x c)
std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int r, int k, int c) {
  std::vector<double> C((size_t)r * c, 0.0);
  for (int i = 0; i < r; ++i)
    for (int l = 0; l < k; ++l) {
      double a = A[(size_t)i * k + l];
      if (a == 0.0) continue;
      for (int j = 0; j < c; ++j) C[(size_t)i * c + j] += a * B[(size_t)l * c + j];
    }
  return C;
}

std::vector<double> transpose(const std::vector<double>& A, int r, int c) {
  std::vector<double> T((size_t)r * c);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) T[(size_t)j * r + i] = A[(size_t)i * c + j];
  return T;
}

struct Geo {
  int d, p, nb1, nb, nf, q, nqv, nqf;
  double h[3];
  double J;        // volume Jacobian
  double Jf[3];    // face Jacobian for faces normal to axis a
};

// multi-index helpers (x fastest)
inline void unflat(int I, int nb1, int d, int* i) {
  for (int a = 0; a < d; ++a) { i[a] = I % nb1; I /= nb1; }
}
// face node index of a volume node lying on a face of axis a (tangential axes ascending)
inline int face_index(const int* i, int a, int d, int nb1) {
  int j = 0, stride = 1;
  for (int b = 0; b < d; ++b) {
    if (b == a) continue;
    j += i[b] * stride;
    stride *= nb1;
  }
  return j;
}

}  // namespace

ihdg_status validate(const ihdg_mesh& m, const ihdg_coeffs* co, std::string& err) {
  std::ostringstream os;
  if (m.dim != 2 && m.dim != 3) { os << "mesh.dim must be 2 or 3 (got " << m.dim << ")"; err = os.str(); return IHDG_ERR_INVALID; }
  if (m.p < 1 || m.p > 4) { os << "mesh.p must be in 1..4 (got " << m.p << ")"; err = os.str(); return IHDG_ERR_UNSUPPORTED; }
  long long nel = 1;
  for (int a = 0; a < m.dim; ++a) {
    if (m.n[a] < 1) { os << "mesh.n[" << a << "] must be >= 1"; err = os.str(); return IHDG_ERR_INVALID; }
    if (!(m.hi[a] > m.lo[a]) || !std::isfinite(m.hi[a] - m.lo[a])) { os << "mesh.hi[" << a << "] must exceed mesh.lo[" << a << "]"; err = os.str(); return IHDG_ERR_INVALID; }
    nel *= m.n[a];
  }
  if (nel > (1LL << 31) - 1) { err = "too many elements (> 2^31-1)"; return IHDG_ERR_INVALID; }
  if (!co) return IHDG_OK;
  if (co->pde != IHDG_TRANSPORT && co->pde != IHDG_CONVDIFF && co->pde != IHDG_SWE) { err = "coeffs.pde is not a known PDE"; return IHDG_ERR_INVALID; }
  for (int a = 0; a < m.dim; ++a)
    if (!std::isfinite(co->beta[a])) { err = "coeffs.beta must be finite"; return IHDG_ERR_INVALID; }
  if (co->flux != IHDG_FLUX_UPWIND && co->flux != IHDG_FLUX_NPC) { err = "coeffs.flux is not a known flux"; return IHDG_ERR_INVALID; }
  if (co->flux == IHDG_FLUX_NPC && co->pde != IHDG_TRANSPORT) { err = "the NPC flux is defined for transport only"; return IHDG_ERR_UNSUPPORTED; }
  if (!(co->tau_gamma >= 0.0) || !std::isfinite(co->tau_gamma)) { err = "coeffs.tau_gamma must be finite and >= 0"; return IHDG_ERR_INVALID; }
  if (co->tau_gamma > 0.0 && co->pde != IHDG_CONVDIFF) { err = "the mesh-dependent stabilisation is for convection-diffusion"; return IHDG_ERR_UNSUPPORTED; }
  if (co->time_scheme != IHDG_BACKWARD_EULER && co->time_scheme != IHDG_CRANK_NICOLSON) {
    err = "coeffs.time_scheme must be IHDG_BACKWARD_EULER or IHDG_CRANK_NICOLSON";
    return IHDG_ERR_INVALID;
  }
  if (co->time_scheme != IHDG_BACKWARD_EULER && co->pde != IHDG_SWE) { err = "a time rule applies to shallow water only"; return IHDG_ERR_UNSUPPORTED; }
  if (co->pde == IHDG_CONVDIFF) {
    if (!(co->kappa > 0) || !std::isfinite(co->kappa)) { err = "coeffs.kappa must be > 0"; return IHDG_ERR_INVALID; }
    if (!(co->nu >= 0) || !std::isfinite(co->nu)) { err = "coeffs.nu must be >= 0"; return IHDG_ERR_INVALID; }
  }
  if (co->pde == IHDG_SWE) {
    if (m.dim != 2) { err = "shallow water is two-dimensional (mesh.dim = 2)"; return IHDG_ERR_UNSUPPORTED; }
    if (!(co->Phi > 0) || !std::isfinite(co->Phi)) { err = "coeffs.Phi must be > 0"; return IHDG_ERR_INVALID; }
    if (!(co->dt > 0) || !std::isfinite(co->dt)) { err = "coeffs.dt must be > 0"; return IHDG_ERR_INVALID; }
    if (!(co->friction >= 0) || !std::isfinite(co->friction) || !std::isfinite(co->coriolis_f)) { err = "coeffs.friction must be >= 0 and coriolis_f finite"; return IHDG_ERR_INVALID; }
  }
  if (co->pde == IHDG_TRANSPORT) {
    double s = 0;
    for (int a = 0; a < m.dim; ++a) s += std::fabs(co->beta[a]);
    if (!(s > 0)) { err = "transport needs a nonzero beta"; return IHDG_ERR_INVALID; }
    if (!(co->nu >= 0) || !std::isfinite(co->nu)) { err = "coeffs.nu must be >= 0"; return IHDG_ERR_INVALID; }
  }
  return IHDG_OK;
}

long long count_faces(const ihdg_mesh& m, long long* n_bface) {
  long long nf = 0, nb = 0;
  for (int a = 0; a < m.dim; ++a) {
    long long c = 1, t = 1;
    for (int b = 0; b < m.dim; ++b) {
      c *= (b == a) ? (m.n[b] + 1) : m.n[b];
      if (b != a) t *= m.n[b];
    }
    nf += c;
    nb += 2 * t;
  }
  if (n_bface) *n_bface = nb;
  return nf;
}

void boundary_faces(const ihdg_mesh& m, std::vector<long long>& elem, std::vector<int>& lf) {
  elem.clear();
  lf.clear();
  int d = m.dim;
  int n0 = m.n[0], n1 = m.n[1], n2 = (d == 3) ? m.n[2] : 1;
  auto eid = [&](long long i, long long j, long long k) { return i + (long long)n0 * (j + (long long)n1 * k); };
  // x-normal faces: i + (nx+1)*(j + ny*k)
  for (int k = 0; k < n2; ++k)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i <= n0; ++i) {
        if (i == 0) { elem.push_back(eid(0, j, k)); lf.push_back(0); }
        else if (i == n0) { elem.push_back(eid(n0 - 1, j, k)); lf.push_back(1); }
      }
  for (int k = 0; k < n2; ++k)
    for (int j = 0; j <= n1; ++j)
      for (int i = 0; i < n0; ++i) {
        if (j == 0) { elem.push_back(eid(i, 0, k)); lf.push_back(2); }
        else if (j == n1) { elem.push_back(eid(i, n1 - 1, k)); lf.push_back(3); }
      }
  if (d == 3)
    for (int k = 0; k <= n2; ++k)
      for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n0; ++i) {
          if (k == 0) { elem.push_back(eid(i, j, 0)); lf.push_back(4); }
          else if (k == n2) { elem.push_back(eid(i, j, n2 - 1)); lf.push_back(5); }
        }
}

void quadrature_points(const ihdg_mesh& m, double* vol_xyz, double* bnd_xyz) {
  Ref1D r = make_ref(m.p);
  int d = m.dim, q = r.q;
  double h[3];
  for (int a = 0; a < d; ++a) h[a] = (m.hi[a] - m.lo[a]) / m.n[a];
  long long nel = 1;
  for (int a = 0; a < d; ++a) nel *= m.n[a];
  int nqv = 1;
  for (int a = 0; a < d; ++a) nqv *= q;
  if (vol_xyz) {
    for (long long K = 0; K < nel; ++K) {
      long long t = K;
      int ec[3];
      for (int a = 0; a < d; ++a) { ec[a] = (int)(t % m.n[a]); t /= m.n[a]; }
      for (int g = 0; g < nqv; ++g) {
        int gi[3];
        unflat(g, q, d, gi);
        for (int a = 0; a < d; ++a)
          vol_xyz[((size_t)K * nqv + g) * d + a] = m.lo[a] + ec[a] * h[a] + 0.5 * (r.xg[gi[a]] + 1.0) * h[a];
      }
    }
  }
  if (bnd_xyz) {
    std::vector<long long> el;
    std::vector<int> lf;
    boundary_faces(m, el, lf);
    int nqf = nqv / q;
    for (size_t b = 0; b < el.size(); ++b) {
      long long t = el[b];
      int ec[3];
      for (int a = 0; a < d; ++a) { ec[a] = (int)(t % m.n[a]); t /= m.n[a]; }
      int ax = lf[b] / 2, s = lf[b] % 2;
      for (int g = 0; g < nqf; ++g) {
        int gi[2] = {0, 0};
        unflat(g, q, d - 1, gi);
        int tcount = 0;
        for (int a = 0; a < d; ++a) {
          double x;
          if (a == ax) x = m.lo[a] + (ec[a] + s) * h[a];
          else x = m.lo[a] + ec[a] * h[a] + 0.5 * (r.xg[gi[tcount++]] + 1.0) * h[a];
          bnd_xyz[((size_t)b * nqf + g) * d + a] = x;
        }
      }
    }
  }
}

void face_points(const ihdg_mesh& m, double* xyz) {
  Ref1D r = make_ref(m.p);
  const int d = m.dim, q = r.q;
  const int n0 = m.n[0], n1 = m.n[1], n2 = d == 3 ? m.n[2] : 1;
  double h[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) h[a] = (m.hi[a] - m.lo[a]) / m.n[a];
  int nqf = 1;
  for (int a = 1; a < d; ++a) nqf *= q;
  long long fid = 0;
  for (int ax = 0; ax < d; ++ax) {
    const int e0 = n0 + (ax == 0), e1 = n1 + (ax == 1), e2 = n2 + (ax == 2 && d == 3);
    for (int k = 0; k < e2; ++k)
      for (int j = 0; j < e1; ++j)
        for (int i = 0; i < e0; ++i, ++fid) {
          const int c[3] = {i, j, k};
          for (int g = 0; g < nqf; ++g) {
            int gi[2] = {0, 0};
            unflat(g, q, d - 1, gi);
            int t = 0;
            for (int a = 0; a < d; ++a) {
              const double x = a == ax ? m.lo[a] + c[a] * h[a] : m.lo[a] + c[a] * h[a] + 0.5 * (r.xg[gi[t++]] + 1.0) * h[a];
              xyz[((size_t)fid * nqf + g) * d + a] = x;
            }
          }
        }
  }
}

RefTables ref_tables(int p) {
  Ref1D r = make_ref(p);
  RefTables t;
  t.p = r.p;
  t.q = r.q;
  t.nb1 = r.nb1;
  t.xn = r.xn;
  t.xg = r.xg;
  t.wg = r.wg;
  t.Lg = r.Lg;
  t.Dg = r.Dg;
  t.M1 = r.M1;
  return t;
}

bool dense_solve(std::vector<double> A, int n, std::vector<double>& B, int m) { return lu_solve(std::move(A), n, B, m); }

void node_points(const ihdg_mesh& m, double* xyz) {
  Ref1D r = make_ref(m.p);
  int d = m.dim, nb1 = r.nb1;
  double h[3];
  for (int a = 0; a < d; ++a) h[a] = (m.hi[a] - m.lo[a]) / m.n[a];
  long long nel = 1;
  for (int a = 0; a < d; ++a) nel *= m.n[a];
  int nb = 1;
  for (int a = 0; a < d; ++a) nb *= nb1;
  for (long long K = 0; K < nel; ++K) {
    long long t = K;
    int ec[3];
    for (int a = 0; a < d; ++a) { ec[a] = (int)(t % m.n[a]); t /= m.n[a]; }
    for (int I = 0; I < nb; ++I) {
      int ii[3];
      unflat(I, nb1, d, ii);
      for (int a = 0; a < d; ++a)
        xyz[((size_t)K * nb + I) * d + a] = m.lo[a] + ec[a] * h[a] + 0.5 * (r.xn[ii[a]] + 1.0) * h[a];
    }
  }
}

ihdg_status build_ops(const ihdg_mesh& m, const ihdg_coeffs& co, Ops& o, std::string& err) {
  ihdg_status st = validate(m, &co, err);
  if (st != IHDG_OK) return st;
  Ref1D r = make_ref(m.p);
  Geo g{};
  g.d = m.dim;
  g.p = m.p;
  g.nb1 = r.nb1;
  g.q = r.q;
  g.nb = 1;
  g.nqv = 1;
  for (int a = 0; a < g.d; ++a) { g.nb *= g.nb1; g.nqv *= g.q; }
  g.nf = g.nb / g.nb1;
  g.nqf = g.nqv / g.q;
  g.J = 1.0;
  for (int a = 0; a < g.d; ++a) { g.h[a] = (m.hi[a] - m.lo[a]) / m.n[a]; g.J *= 0.5 * g.h[a]; }
  for (int a = 0; a < g.d; ++a) {
    g.Jf[a] = 1.0;
    for (int b = 0; b < g.d; ++b) if (b != a) g.Jf[a] *= 0.5 * g.h[b];
  }
  const int d = g.d, nb = g.nb, nb1 = g.nb1, nf = g.nf, nlf = 2 * d;
  o = Ops();
  o.pde = co.pde;
  o.dim = d;
  o.p = m.p;
  o.nb1 = nb1;
  o.nb = nb;
  o.nf = nf;
  o.q = g.q;
  o.nqv = g.nqv;
  o.nqf = g.nqf;
  o.nlf = nlf;
  for (int a = 0; a < d; ++a) o.beta[a] = co.beta[a];

  // element matrices
  std::vector<double> M(nb * nb), K[3];
  for (int a = 0; a < d; ++a) K[a].assign(nb * nb, 0.0);
  for (int I = 0; I < nb; ++I) {
    int ii[3];
    unflat(I, nb1, d, ii);
    for (int Jn = 0; Jn < nb; ++Jn) {
      int jj[3];
      unflat(Jn, nb1, d, jj);
      double mm = g.J;
      for (int a = 0; a < d; ++a) mm *= r.M1[ii[a] * nb1 + jj[a]];
      M[I * nb + Jn] = mm;
      for (int a = 0; a < d; ++a) {
        double k = g.J * (2.0 / g.h[a]) * r.S1[ii[a] * nb1 + jj[a]];
        for (int b = 0; b < d; ++b) if (b != a) k *= r.M1[ii[b] * nb1 + jj[b]];
        K[a][I * nb + Jn] = k;   // (phi_J, d_a phi_I)
      }
    }
  }
  // face tables
  std::vector<int> fvol(nlf * nf);           // volume node of face node
  std::vector<double> Mface[3];              // nf x nf per axis
  std::vector<double> Bf[3];                 // nf x nqf per axis: weight * face basis at face points
  for (int a = 0; a < d; ++a) {
    Mface[a].assign(nf * nf, 0.0);
    Bf[a].assign((size_t)nf * g.nqf, 0.0);
    for (int j = 0; j < nf; ++j) {
      int jt[2] = {0, 0};
      unflat(j, nb1, d - 1, jt);
      for (int k = 0; k < nf; ++k) {
        int kt[2] = {0, 0};
        unflat(k, nb1, d - 1, kt);
        double v = g.Jf[a];
        for (int t = 0; t < d - 1; ++t) v *= r.M1[jt[t] * nb1 + kt[t]];
        Mface[a][j * nf + k] = v;
      }
      for (int gq = 0; gq < g.nqf; ++gq) {
        int gt[2] = {0, 0};
        unflat(gq, g.q, d - 1, gt);
        double v = g.Jf[a];
        for (int t = 0; t < d - 1; ++t) v *= r.wg[gt[t]] * r.Lg[gt[t] * nb1 + jt[t]];
        Bf[a][(size_t)j * g.nqf + gq] = v;
      }
    }
  }
  for (int f = 0; f < nlf; ++f) {
    int a = f / 2, s = f % 2;
    for (int I = 0; I < nb; ++I) {
      int ii[3];
      unflat(I, nb1, d, ii);
      if (ii[a] == (s ? nb1 - 1 : 0)) fvol[f * nf + face_index(ii, a, d, nb1)] = I;
    }
  }
  o.facevol.resize(nlf * nf);
  for (int i = 0; i < nlf * nf; ++i) o.facevol[i] = fvol[i];
  auto nsign = [](int f) { return (f % 2) ? 1.0 : -1.0; };
  // volume forcing weights: Bv[I][g] = W_g phi_I(x_g)
  std::vector<double> Bv((size_t)nb * g.nqv);
  for (int I = 0; I < nb; ++I) {
    int ii[3];
    unflat(I, nb1, d, ii);
    for (int gq = 0; gq < g.nqv; ++gq) {
      int gi[3];
      unflat(gq, g.q, d, gi);
      double v = g.J;
      for (int a = 0; a < d; ++a) v *= r.wg[gi[a]] * r.Lg[gi[a] * nb1 + ii[a]];
      Bv[(size_t)I * g.nqv + gq] = v;
    }
  }

  int nc = 1, fcomp = 0;   // forced component
  if (co.pde == IHDG_CONVDIFF) { nc = d + 1; fcomp = d; }
  if (co.pde == IHDG_SWE) nc = 3;
  const int nvol = nc * nb;
  o.ncomp = nc;
  o.nvol = nvol;
  o.n_in = nlf * nf;
  std::vector<double> A((size_t)nvol * nvol, 0.0);
  auto Aat = [&](int rc, int I, int cc, int Jn) -> double& { return A[(size_t)(rc * nb + I) * nvol + cc * nb + Jn]; };
  // add c * (face mass of face f) into block (rc, cc)
  auto add_face_mass = [&](int f, int rc, int cc, double c) {
    int a = f / 2;
    for (int j = 0; j < nf; ++j)
      for (int k = 0; k < nf; ++k) Aat(rc, fvol[f * nf + j], cc, fvol[f * nf + k]) += c * Mface[a][j * nf + k];
  };
  auto add_vol = [&](const std::vector<double>& B, int rc, int cc, double c) {
    for (int I = 0; I < nb; ++I)
      for (int Jn = 0; Jn < nb; ++Jn) Aat(rc, I, cc, Jn) += c * B[I * nb + Jn];
  };
  std::vector<double> G((size_t)nvol * o.n_in, 0.0);       // input -> rhs (scaled inputs)
  std::vector<double> Gb[6];                                 // unscaled, per face: Pi g -> rhs (nvol x nf)
  for (int f = 0; f < nlf; ++f) Gb[f].assign((size_t)nvol * nf, 0.0);
  // coefficient c * (face node j of face f) into rhs row (rc, node of face node i)
  auto add_G = [&](int f, int rc, double c, bool boundary_copy, double scale) {
    int a = f / 2;
    for (int i = 0; i < nf; ++i)
      for (int j = 0; j < nf; ++j) {
        double v = c * Mface[a][i * nf + j];
        G[(size_t)(rc * nb + fvol[f * nf + i]) * o.n_in + f * nf + j] += v * scale;
        if (boundary_copy) Gb[f][(size_t)(rc * nb + fvol[f * nf + i]) * nf + j] += v;
      }
  };
  std::vector<double> R;
  o.Mn.assign((size_t)nvol * nvol, 0.0);

  if (co.pde == IHDG_TRANSPORT) {
    // per-axis export layout: along each axis with beta_a != 0 exactly one face is outflow;
    // slot a * nf + node holds u on it, and the downstream neighbour reads the same slots
    o.n_exp = d * nf;
    o.layout_per_axis = 1;
    for (int f = 0; f < nlf; ++f) {
      double bn = nsign(f) * co.beta[f / 2];
      if (bn > 0) { o.face_kind[f] = FK_OWN; o.own_off[f] = (f / 2) * nf; }
      else if (bn < 0) { o.face_kind[f] = FK_NBR; o.nbr_off[f] = (f / 2) * nf; }
      else o.face_kind[f] = FK_NONE;
    }
    for (int a = 0; a < d; ++a) add_vol(K[a], 0, 0, -co.beta[a]);       // -(u, beta.grad v)
    // nu (u, v): a reaction term, or the L2 term 1/dt (u, v) of a backward-Euler step of the
    // time-dependent equation (the remark on time-dependent transport after Theorem 1)
    if (co.nu != 0.0) add_vol(M, 0, 0, co.nu);
    for (int f = 0; f < nlf; ++f) {
      double bn = nsign(f) * co.beta[f / 2];
      // stabilisation: upwind |beta.n|; NPC (Eq. Ntaub) |beta.n|(1 + sgn(beta.n))/2 - beta.n,
      // which is 0 on outflow faces (no trace coupling there) and |beta.n| on inflow faces
      const double sg = bn > 0 ? 1.0 : (bn < 0 ? -1.0 : 0.0);
      const double tau = co.flux == IHDG_FLUX_NPC ? std::fabs(bn) * (1.0 + sg) / 2.0 - bn : std::fabs(bn);
      add_face_mass(f, 0, 0, bn + tau);                                  // <(beta.n + tau) u, v>
      if (tau != 0) add_G(f, 0, tau, bn < 0, 1.0);                       // <tau u_hat, v>
    }
    R.assign((size_t)o.n_exp * nvol, 0.0);
    for (int f = 0; f < nlf; ++f)
      if (o.face_kind[f] == FK_OWN)
        for (int j = 0; j < nf; ++j) R[(size_t)(o.own_off[f] + j) * nvol + fvol[f * nf + j]] = 1.0;
    for (int i = 0; i < nb * nb; ++i) o.Mn[(i / nb) * nvol + (i % nb)] = M[i];
  } else if (co.pde == IHDG_CONVDIFF) {
    o.n_exp = nlf * nf;
    for (int f = 0; f < nlf; ++f) { o.face_kind[f] = FK_SUM; o.own_off[f] = f * nf; o.nbr_off[f] = (f ^ 1) * nf; }
    const int iu = d;
    for (int c = 0; c < d; ++c) {
      add_vol(M, c, c, 1.0 / co.kappa);     // kappa^-1 (sigma_c, w)
      add_vol(K[c], c, iu, -1.0);           // -(u, d_c w)
      add_vol(K[c], iu, c, -1.0);           // -(sigma_c, d_c v)
      add_vol(K[c], iu, iu, -co.beta[c]);   // -(u, beta.grad v)
    }
    add_vol(M, iu, iu, co.nu);
    R.assign((size_t)o.n_exp * nvol, 0.0);
    // Stabilisation: upwind tau^+- = (alpha - beta.n^+-)/2, alpha = sqrt((beta.n)^2 + 4), so
    // tau^+ + tau^- = alpha; or the mesh-dependent tau = gamma (p+1)(p+2)/h_a on both sides
    // (Section 4.2), so tau^+ + tau^- = 2 tau.  The conservation condition gives
    // u_hat = (h^- + h^+)/(tau^+ + tau^-) with the export h = sigma.n + (tau + beta.n) u.
    auto tau_of = [&](int f, double bn) {
      if (co.tau_gamma > 0) return co.tau_gamma * (m.p + 1) * (m.p + 2) / ((m.hi[f / 2] - m.lo[f / 2]) / m.n[f / 2]);
      return 0.5 * (std::sqrt(bn * bn + 4.0) - bn);
    };
    for (int a = 0; a < d; ++a) {
      const double ba = co.beta[a];
      o.alpha_axis[a] = tau_of(2 * a, -ba) + tau_of(2 * a + 1, ba);   // tau^- + tau^+ on axis a
    }
    for (int f = 0; f < nlf; ++f) {
      int a = f / 2;
      double n = nsign(f), bn = n * co.beta[a];
      const double tau = tau_of(f, bn), tsum = o.alpha_axis[a];
      o.in_scale[f] = 1.0 / tsum;
      add_face_mass(f, iu, a, n);            // <sigma.n, v>
      add_face_mass(f, iu, iu, bn + tau);    // <(beta.n + tau) u, v>
      add_G(f, a, -n, true, 1.0 / tsum);     // -<u_hat, w.n>   (u_hat = (h^- + h^+)/(tau^+ + tau^-))
      add_G(f, iu, tau, true, 1.0 / tsum);   // <tau u_hat, v>
      for (int j = 0; j < nf; ++j) {
        int node = fvol[f * nf + j];
        R[(size_t)(f * nf + j) * nvol + a * nb + node] = n;           // sigma.n
        R[(size_t)(f * nf + j) * nvol + iu * nb + node] = tau + bn;   // (tau + beta.n) u
      }
    }
    for (int i = 0; i < nb * nb; ++i) o.Mn[(size_t)(iu * nb + i / nb) * nvol + iu * nb + (i % nb)] = M[i];
  } else {  // shallow water
    o.n_exp = nlf * nf;
    o.bc_mirror = 1;
    for (int f = 0; f < nlf; ++f) { o.face_kind[f] = FK_SUM; o.own_off[f] = f * nf; o.nbr_off[f] = (f ^ 1) * nf; }
    const double P = co.Phi, sP = std::sqrt(co.Phi), dt = co.dt;
    add_vol(M, 0, 0, 1.0 / dt);
    add_vol(K[0], 0, 1, -P);
    add_vol(K[1], 0, 2, -P);
    add_vol(M, 1, 1, P / dt + co.friction * P);
    add_vol(K[0], 1, 0, -P);
    add_vol(M, 1, 2, -co.coriolis_f * P);
    add_vol(M, 2, 2, P / dt + co.friction * P);
    add_vol(K[1], 2, 0, -P);
    add_vol(M, 2, 1, co.coriolis_f * P);
    R.assign((size_t)o.n_exp * nvol, 0.0);
    for (int f = 0; f < nlf; ++f) {
      int a = f / 2;
      double n = nsign(f);
      add_face_mass(f, 0, 1 + a, P * n);     // <Phi vel.n, w>
      add_face_mass(f, 0, 0, sP);            // <sqrt(Phi) phi, w>
      add_G(f, 0, sP, false, 1.0);           // sqrt(Phi) <phi_hat, w>
      add_G(f, 1 + a, -P * n, false, 1.0);   // -Phi <phi_hat n_a, w>
      for (int j = 0; j < nf; ++j) {
        int node = fvol[f * nf + j];
        R[(size_t)(f * nf + j) * nvol + node] = 0.5;                        // phi / 2
        R[(size_t)(f * nf + j) * nvol + (1 + a) * nb + node] = 0.5 * sP * n; // sqrt(Phi) vel.n / 2
      }
    }
    for (int c = 0; c < 3; ++c) {
      double w = c == 0 ? 1.0 : P;
      for (int i = 0; i < nb * nb; ++i) o.Mn[(size_t)(c * nb + i / nb) * nvol + c * nb + (i % nb)] = w * M[i];
    }
  }
  o.R = R;
  o.Mb = M;
  if (co.pde == IHDG_TRANSPORT) o.wcomp[0] = 1.0;
  else if (co.pde == IHDG_CONVDIFF) o.wcomp[d] = 1.0;
  else { o.wcomp[0] = 1.0; o.wcomp[1] = co.Phi; o.wcomp[2] = co.Phi; }

  // Lvol = A^{-1} G
  o.Lvol = G;
  if (!lu_solve(A, nvol, o.Lvol, o.n_in)) { err = "local matrix is singular"; return IHDG_ERR_INVALID; }
  o.LE = matmul(R, o.Lvol, o.n_exp, nvol, o.n_in);
  {
    std::vector<double> MnL = matmul(o.Mn, o.Lvol, nvol, nvol, o.n_in);
    o.Q = matmul(transpose(o.Lvol, nvol, o.n_in), MnL, o.n_in, nvol, o.n_in);
    for (int i = 0; i < o.n_in; ++i)
      for (int j = 0; j < i; ++j) {
        double s = 0.5 * (o.Q[i * o.n_in + j] + o.Q[j * o.n_in + i]);
        o.Q[i * o.n_in + j] = o.Q[j * o.n_in + i] = s;
      }
  }
  if (co.pde != IHDG_SWE) {
    // forcing: rhs rows of the forced component = Bv f
    std::vector<double> Bfull((size_t)nvol * g.nqv, 0.0);
    for (int I = 0; I < nb; ++I)
      for (int gq = 0; gq < g.nqv; ++gq) Bfull[(size_t)(fcomp * nb + I) * g.nqv + gq] = Bv[(size_t)I * g.nqv + gq];
    o.PV = Bfull;
    if (!lu_solve(A, nvol, o.PV, g.nqv)) { err = "local matrix is singular"; return IHDG_ERR_INVALID; }
    o.PF = matmul(R, o.PV, o.n_exp, nvol, g.nqv);
    // boundary data on local face f: rhs += Gb_f * Pi g, Pi g = Mface^{-1} Bf g
    for (int f = 0; f < nlf; ++f) {
      int a = f / 2;
      std::vector<double> Pg = Bf[a];
      if (!lu_solve(Mface[a], nf, Pg, g.nqf)) { err = "face mass is singular"; return IHDG_ERR_INVALID; }
      if (o.Pg.empty()) o.Pg = Pg;   // the same for every axis (J_f cancels)
      std::vector<double> rhs = matmul(Gb[f], Pg, nvol, nf, g.nqf);
      o.PVb[f] = rhs;
      if (!lu_solve(A, nvol, o.PVb[f], g.nqf)) { err = "local matrix is singular"; return IHDG_ERR_INVALID; }
      o.PFb[f] = matmul(R, o.PVb[f], o.n_exp, nvol, g.nqf);
    }
  } else {
    std::vector<double> Mt((size_t)nvol * nvol, 0.0);
    for (int c = 0; c < 3; ++c) {
      double w = (c == 0 ? 1.0 : co.Phi) / co.dt;
      for (int i = 0; i < nb * nb; ++i) Mt[(size_t)(c * nb + i / nb) * nvol + c * nb + (i % nb)] = w * M[i];
    }
    o.PqV = Mt;
    if (!lu_solve(A, nvol, o.PqV, nvol)) { err = "local matrix is singular"; return IHDG_ERR_INVALID; }
    o.PqF = matmul(R, o.PqV, o.n_exp, nvol, nvol);
  }
  return IHDG_OK;
}

}  // namespace ihdg
