// Host float64 construction of the per-element local solves for transport with a velocity
// field that varies in space (see ihdg_var.h).  Element integrals are Gauss sums with beta
// sampled at the Gauss points; every element's local matrix is factorised once (threads over
// elements) and its solve applied to the trace coupling and to the identity.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <sstream>
#include <thread>

#include "ihdg_ops.h"
#include "ihdg_var.h"

namespace ihdg {
namespace {

inline void unflat_idx(int I, int b, int d, int* i) {
  for (int a = 0; a < d; ++a) {
    i[a] = I % b;
    I /= b;
  }
}

// global face number of local face f of the element at integer coordinates ec
long long global_face(const ihdg_mesh& m, const int* ec, int f) {
  const long long n0 = m.n[0], n1 = m.n[1], n2 = m.dim == 3 ? m.n[2] : 1;
  const int a = f >> 1, s = f & 1;
  const long long off1 = (n0 + 1) * n1 * n2, off2 = off1 + n0 * (n1 + 1) * n2;
  if (a == 0) return (ec[0] + s) + (n0 + 1) * (ec[1] + n1 * ec[2]);
  if (a == 1) return off1 + ec[0] + n0 * ((ec[1] + s) + (n1 + 1) * ec[2]);
  return off2 + ec[0] + n0 * (ec[1] + n1 * (ec[2] + s));
}

}  // namespace

ihdg_status build_var(const ihdg_mesh& m, const double* beta_vol, const double* beta_face, VarHost& v,
                      std::string& err) {
  ihdg_status st = validate(m, nullptr, err);
  if (st != IHDG_OK) return st;
  if (!beta_vol || !beta_face) {
    err = "null beta samples";
    return IHDG_ERR_INVALID;
  }
  if (m.dim == 3 && m.p > 2) {
    err = "variable-coefficient transport is built for 2D p = 1..4 and 3D p = 1..2";
    return IHDG_ERR_UNSUPPORTED;
  }
  const RefTables r = ref_tables(m.p);
  const int d = m.dim, p = m.p, nb1 = p + 1, q = r.q;
  v.dim = d;
  v.p = p;
  v.nb1 = nb1;
  v.q = q;
  v.nb = v.nf = v.nqv = v.nqf = 1;
  for (int a = 0; a < d; ++a) {
    v.nb *= nb1;
    v.nqv *= q;
  }
  for (int a = 1; a < d; ++a) {
    v.nf *= nb1;
    v.nqf *= q;
  }
  v.nlf = 2 * d;
  v.nin = v.nlf * v.nf;
  v.nel = 1;
  double h[3] = {1, 1, 1};
  v.jac = 1.0;
  for (int a = 0; a < 3; ++a) v.n[a] = a < d ? m.n[a] : 1;
  for (int a = 0; a < d; ++a) {
    v.nel *= m.n[a];
    h[a] = (m.hi[a] - m.lo[a]) / m.n[a];
    v.jac *= 0.5 * h[a];
  }
  v.nface = count_faces(m, &v.nbface);
  const int nb = v.nb, nf = v.nf, nqv = v.nqv, nqf = v.nqf, nlf = v.nlf, nin = v.nin;
  // flow direction per axis from the samples on the faces normal to it
  {
    long long fid = 0;
    for (int ax = 0; ax < d; ++ax) {
      long long cnt = 1;
      for (int b = 0; b < d; ++b) cnt *= (b == ax) ? (m.n[b] + 1) : m.n[b];
      double lo = 0.0, hi = 0.0;
      for (long long e = fid; e < fid + cnt; ++e)
        for (int g = 0; g < nqf; ++g) {
          const double b = beta_face[((size_t)e * nqf + g) * d + ax];
          if (!std::isfinite(b)) {
            err = "beta samples must be finite";
            return IHDG_ERR_INVALID;
          }
          lo = std::min(lo, b);
          hi = std::max(hi, b);
        }
      fid += cnt;
      if (lo < 0.0 && hi > 0.0) {
        std::ostringstream os;
        os << "beta_" << ax << " changes sign on the faces normal to axis " << ax
           << "; the device path needs one flow direction per axis";
        err = os.str();
        return IHDG_ERR_UNSUPPORTED;
      }
      v.sign[ax] = hi > 0.0 ? 1 : (lo < 0.0 ? -1 : 0);
    }
    if (!v.sign[0] && !v.sign[1] && !(d == 3 && v.sign[2])) {
      err = "beta vanishes on every face";
      return IHDG_ERR_INVALID;
    }
  }
  for (int f = 0; f < nlf; ++f) {
    const int dir = v.sign[f >> 1] * ((f & 1) ? 1 : -1);
    v.kind[f] = dir > 0 ? 1 : (dir < 0 ? 2 : 0);
  }
  // volume tables: phi_I and its physical gradient at the Gauss points, weights times Jacobian
  std::vector<double> Bv((size_t)nqv * nb), Dv[3], wJ(nqv);
  for (int a = 0; a < d; ++a) Dv[a].assign((size_t)nqv * nb, 0.0);
  for (int Q = 0; Q < nqv; ++Q) {
    int qi[3];
    unflat_idx(Q, q, d, qi);
    double w = v.jac;
    for (int a = 0; a < d; ++a) w *= r.wg[qi[a]];
    wJ[Q] = w;
    for (int I = 0; I < nb; ++I) {
      int ii[3];
      unflat_idx(I, nb1, d, ii);
      double val = 1.0;
      for (int a = 0; a < d; ++a) val *= r.Lg[qi[a] * nb1 + ii[a]];
      Bv[(size_t)Q * nb + I] = val;
      for (int a = 0; a < d; ++a) {
        double der = 2.0 / h[a] * r.Dg[qi[a] * nb1 + ii[a]];
        for (int b = 0; b < d; ++b)
          if (b != a) der *= r.Lg[qi[b] * nb1 + ii[b]];
        Dv[a][(size_t)Q * nb + I] = der;
      }
    }
  }
  v.Wq.assign((size_t)nb * nqv, 0.0);
  for (int i = 0; i < nb; ++i)
    for (int Q = 0; Q < nqv; ++Q) v.Wq[(size_t)i * nqv + Q] = wJ[Q] * Bv[(size_t)Q * nb + i];
  // face tables: basis at each local face's Gauss points, face weights, face nodes
  v.FBv.assign((size_t)nlf * nb * nqf, 0.0);
  v.facevol.assign((size_t)nlf * nf, 0);
  std::vector<double> wf((size_t)nlf * nqf);
  for (int f = 0; f < nlf; ++f) {
    const int a = f >> 1, end = (f & 1) ? p : 0;
    int tang[2] = {0, 0}, nt = 0;
    for (int b = 0; b < d; ++b)
      if (b != a) tang[nt++] = b;
    for (int g = 0; g < nqf; ++g) {
      int gi[2] = {0, 0};
      unflat_idx(g, q, d - 1, gi);
      double w = 1.0;
      for (int t = 0; t < nt; ++t) w *= r.wg[gi[t]] * 0.5 * h[tang[t]];
      wf[(size_t)f * nqf + g] = w;
      for (int I = 0; I < nb; ++I) {
        int ii[3];
        unflat_idx(I, nb1, d, ii);
        if (ii[a] != end) continue;
        double val = 1.0;
        for (int t = 0; t < nt; ++t) val *= r.Lg[gi[t] * nb1 + ii[tang[t]]];
        v.FBv[((size_t)f * nb + I) * nqf + g] = val;
      }
    }
    for (int rr = 0; rr < nf; ++rr) {
      int ri[2] = {0, 0};
      unflat_idx(rr, nb1, d - 1, ri);
      int ii[3] = {0, 0, 0};
      ii[a] = end;
      for (int t = 0; t < nt; ++t) ii[tang[t]] = ri[t];
      int I = 0, stride = 1;
      for (int b = 0; b < d; ++b) {
        I += ii[b] * stride;
        stride *= nb1;
      }
      v.facevol[(size_t)f * nf + rr] = I;
    }
  }
  v.M1 = r.M1;
  // L2 projection of face Gauss values onto the face nodal basis (reference face weights)
  {
    std::vector<double> B((size_t)nqf * nf), Mf((size_t)nf * nf, 0.0), X((size_t)nf * nqf, 0.0);
    for (int g = 0; g < nqf; ++g) {
      int gi[2] = {0, 0};
      unflat_idx(g, q, d - 1, gi);
      double w = 1.0;
      for (int t = 0; t < d - 1; ++t) w *= r.wg[gi[t]];
      for (int rr = 0; rr < nf; ++rr) {
        int ri[2] = {0, 0};
        unflat_idx(rr, nb1, d - 1, ri);
        double val = 1.0;
        for (int t = 0; t < d - 1; ++t) val *= r.Lg[gi[t] * nb1 + ri[t]];
        B[(size_t)g * nf + rr] = val;
        X[(size_t)rr * nqf + g] = w * val;
      }
    }
    for (int a = 0; a < nf; ++a)
      for (int b = 0; b < nf; ++b) {
        double s = 0.0;
        for (int g = 0; g < nqf; ++g) s += X[(size_t)a * nqf + g] * B[(size_t)g * nf + b];
        Mf[(size_t)a * nf + b] = s;
      }
    if (!dense_solve(Mf, nf, X, nqf)) {
      err = "singular face mass matrix";
      return IHDG_ERR_INVALID;
    }
    v.Pg = X;
  }
  // inflow weights on boundary faces
  boundary_faces(m, v.bel, v.blf);
  v.bw.assign((size_t)v.nbface * nqf, 0.0);
  for (long long b = 0; b < v.nbface; ++b) {
    const int f = v.blf[b];
    if (v.kind[f] != 2) continue;
    long long t = v.bel[b];
    int ec[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      ec[a] = (int)(t % m.n[a]);
      t /= m.n[a];
    }
    const long long gf = global_face(m, ec, f);
    for (int g = 0; g < nqf; ++g) {
      const double bn = beta_face[((size_t)gf * nqf + g) * d + (f >> 1)] * ((f & 1) ? 1.0 : -1.0);
      v.bw[(size_t)b * nqf + g] = std::fabs(bn) * wf[(size_t)f * nqf + g];
    }
  }
  // every element: A_K, G_K, then [L_K | A_K^{-1}] = A_K^{-1} [G_K | I]
  v.L.assign((size_t)v.nel * nin * nb, 0.0);
  v.Ainv.assign((size_t)v.nel * nb * nb, 0.0);
  std::atomic<long long> next(0);
  std::atomic<int> bad(0);
  const long long chunk = 256;
  auto work = [&]() {
    std::vector<double> A((size_t)nb * nb), X((size_t)nb * (nin + nb)), bg(nb);
    for (;;) {
      const long long k0 = next.fetch_add(chunk);
      if (k0 >= v.nel || bad.load()) return;
      const long long k1 = std::min(v.nel, k0 + chunk);
      for (long long K = k0; K < k1; ++K) {
        long long t = K;
        int ec[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
          ec[a] = (int)(t % m.n[a]);
          t /= m.n[a];
        }
        std::fill(A.begin(), A.end(), 0.0);
        std::fill(X.begin(), X.end(), 0.0);
        // (beta.grad phi_j, phi_i)_K
        for (int Q = 0; Q < nqv; ++Q) {
          const double* bq = beta_vol + ((size_t)K * nqv + Q) * d;
          for (int a = 0; a < d; ++a)
            if (!std::isfinite(bq[a])) bad.store(1);
          for (int j = 0; j < nb; ++j) {
            double s = 0.0;
            for (int a = 0; a < d; ++a) s += bq[a] * Dv[a][(size_t)Q * nb + j];
            bg[j] = s * wJ[Q];
          }
          for (int i = 0; i < nb; ++i) {
            const double bi = Bv[(size_t)Q * nb + i];
            if (bi == 0.0) continue;
            for (int j = 0; j < nb; ++j) A[(size_t)i * nb + j] += bg[j] * bi;
          }
        }
        // <|beta.n| phi_j, phi_i>_f and the trace coupling <|beta.n| psi_r, phi_i>_f
        for (int f = 0; f < nlf; ++f) {
          const long long gf = global_face(m, ec, f);
          const int* fv = &v.facevol[(size_t)f * nf];
          for (int g = 0; g < nqf; ++g) {
            const double bn = beta_face[((size_t)gf * nqf + g) * d + (f >> 1)] * ((f & 1) ? 1.0 : -1.0);
            const double w = std::fabs(bn) * wf[(size_t)f * nqf + g];
            if (w == 0.0) continue;
            for (int a2 = 0; a2 < nf; ++a2) {
              const int I = fv[a2];
              const double pi = v.FBv[((size_t)f * nb + I) * nqf + g];
              for (int b2 = 0; b2 < nf; ++b2) {
                const int J = fv[b2];
                const double pj = v.FBv[((size_t)f * nb + J) * nqf + g];
                A[(size_t)I * nb + J] += w * pi * pj;
                if (v.kind[f]) X[(size_t)I * (nin + nb) + f * nf + b2] += w * pi * pj;
              }
            }
          }
        }
        for (int i = 0; i < nb; ++i) X[(size_t)i * (nin + nb) + nin + i] = 1.0;
        if (!dense_solve(A, nb, X, nin + nb)) {
          bad.store(2);
          return;
        }
        double* Lk = &v.L[(size_t)K * nin * nb];
        double* Ak = &v.Ainv[(size_t)K * nb * nb];
        for (int i = 0; i < nb; ++i) {
          for (int k = 0; k < nin; ++k) Lk[(size_t)k * nb + i] = X[(size_t)i * (nin + nb) + k];
          for (int j = 0; j < nb; ++j) Ak[(size_t)j * nb + i] = X[(size_t)i * (nin + nb) + nin + j];
        }
      }
    }
  };
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 4;
  if (nt > 64) nt = 64;
  if ((long long)nt * chunk > v.nel) nt = (unsigned)std::max<long long>(1, (v.nel + chunk - 1) / chunk);
  std::vector<std::thread> pool;
  for (unsigned i = 1; i < nt; ++i) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  if (bad.load() == 1) {
    err = "beta samples must be finite";
    return IHDG_ERR_INVALID;
  }
  if (bad.load() == 2) {
    err = "a local matrix is singular";
    return IHDG_ERR_INVALID;
  }
  return IHDG_OK;
}

}  // namespace ihdg
