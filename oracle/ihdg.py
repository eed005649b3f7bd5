"""Plain float64 CPU oracle of the upwind HDG discretisation and of the iHDG iteration.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

What is computed, following the paper:

* Section 2, Eq. (HDGlocal)/(HDGeqn)/(RiemannFluxBoth): the upwind HDG local equations per
  element and the conservation condition per face.
* Section 2, Eq. (iHDGlocal)/(iHDGtrace) and Algorithm 1: the iteration.  Each sweep first
  forms the (weighted) trace on every face from the previous iterate u^k ("face by face"),
  then solves every element's local equation for u^{k+1} ("element by element"), then
  measures ||u^{k+1} - u^k||_{L2(Omega)} (the stopping test of Section 5.1,
  Eq. (tolerancecriteriarelerror)).
* Section 3, Eqs. (transportLocalk1)/(transportLocale): scalar transport; and the NPC flux
  of Section 3 (Eq. Ntaub and the trace formula after it) as the alternative.  TransportVar:
  the same with a velocity field beta(x) that varies in space (the paper's experiments of
  Section 5.1), every element with its own local matrix.
* Section 3, Eq. (localSolverDD) and the trace formula below it: linearized shallow water,
  backward Euler in time; ShallowWaterCN: the same spatial HDG operator with the
  Crank-Nicolson rule the paper's shallow-water experiments use (Section 5, linearized
  shallow water subsection), written as the trapezoidal average of the implicit and explicit
  spatial residuals.
* Section 4.1, Eqs. (ErrorDDMCD1)/(ErrorDDMCD2) and the flux (general_flux_convdiff):
  convection-diffusion in first-order form with the upwind stabilisation.

The state is the full volume solution; traces are evaluated at face Gauss points from the
volume polynomials; every element solve is a dense solve with its local matrix.  The direct
solver eliminates the volume unknowns element by element (static condensation) and solves
the global trace system built from the conservation condition (HDGeqn).

Readings of points the paper leaves open (each is also listed in the design notes):
  R1 Q^p tensor-product spaces with a GLL nodal basis; Gauss quadrature with p+2 points.
  R2 Boundary data enter as g sampled at boundary-face Gauss points; a Dirichlet trace is
     the L2 projection of g onto the face space (which is what integrating g against the
     face basis with that rule gives).
  R3 Transport: outflow boundary faces take the element's own u^k as trace (same rule as an
     interior outflow face); faces with beta.n = 0 carry zero weight and report {{u}}.
  R4 Initial guess u^0 = 0 unless one is given.
  R5 The iteration count K is the number of sweeps run when ||u^K - u^(K-1)|| < tol first
     holds.  Convection-diffusion measures the u component only; shallow water measures
     ||phi||^2 + Phi ||(u,v)||^2.
  R6 Convection-diffusion: tau^+- = (alpha - beta.n^+-)/2 with alpha = sqrt((beta.n)^2+4)
     (gamma = 1), so tau^+ + tau^- = alpha.
  R7 Shallow water walls: the mirror state, phi_hat = phi^- + sqrt(Phi) vel^-.n^-.
  R8 NPC flux (transport): the local equation is the HDG one with stabilisation
     tau = |beta.n| (1 + sgn(beta.n))/2 - beta.n and no weight on the trace; the trace
     ({{tau u}} + {{beta.n u}})/{{tau}} reduces to the upwind value, and g on the inflow
     boundary.
"""
import numpy as np

from .mesh import BoxMesh
from .refelem import RefElement

STATUS_OK, STATUS_NOT_CONVERGED, STATUS_DIVERGED = 0, 4, 5


class Discretisation:
    """Element and face integrals on a uniform box mesh (every element is congruent)."""

    def __init__(self, mesh: BoxMesh, p: int, q=None):
        self.mesh = mesh
        self.d = mesh.d
        self.p = p
        self.ref = RefElement(mesh.d, p, q)
        ref, h, d = self.ref, mesh.h, mesh.d
        self.nb = ref.nb
        self.jac = float(np.prod(h / 2.0))
        wJ = ref.wq * self.jac
        # M[i,j] = (phi_j, phi_i)_K
        self.M = ref.Bq.T @ (wJ[:, None] * ref.Bq)
        # K[a][i,j] = (phi_j, d_a phi_i)_K
        self.K = [(2.0 / h[a]) * (ref.Dq[a].T @ (wJ[:, None] * ref.Bq)) for a in range(d)]
        # face quantities for local face f = 2a + s (normal = (-1)^(s+1) e_a)
        self.normal = np.zeros((2 * d, d))
        self.face_jac = np.zeros(2 * d)
        self.Mf, self.Ff = [], []
        for f in range(2 * d):
            a, s = f // 2, f % 2
            self.normal[f, a] = 1.0 if s == 1 else -1.0
            self.face_jac[f] = float(np.prod([h[b] / 2.0 for b in range(d) if b != a])) if d > 1 else 1.0
            wf = ref.face_w * self.face_jac[f]
            B = ref.face_B[f]
            self.Mf.append(B.T @ (wf[:, None] * B))   # <phi_j, phi_i>_f
            self.Ff.append(B.T * wf[None, :])          # t -> <t, phi_i>_f for t at face points
        self.nq = ref.q ** d
        self.nqf = ref.q ** (d - 1)

    # ---------------------------------------------------------------- points
    def volume_points(self):
        """(nel, q^d, d) physical coordinates of every element's Gauss points."""
        m = self.mesh
        return m.elem_lo[:, None, :] + (self.ref.xq[None, :, :] + 1.0) * 0.5 * m.h[None, None, :]

    def node_points(self):
        """(nel, (p+1)^d, d) physical coordinates of every element's GLL nodes."""
        m = self.mesh
        xr = self.ref.node_ref_points()
        return m.elem_lo[:, None, :] + (xr[None, :, :] + 1.0) * 0.5 * m.h[None, None, :]

    def face_points(self, face_ids):
        """(len(face_ids), q^(d-1), d) physical coordinates of Gauss points on global faces."""
        m = self.mesh
        out = np.zeros((len(face_ids), self.nqf, self.d))
        for r, e in enumerate(face_ids):
            a = m.face_axis[e]
            pts = self.ref.face_ref_points(2 * a)   # normal coordinate -1 -> face_lo[a]
            out[r] = m.face_lo[e][None, :] + (pts + 1.0) * 0.5 * m.h[None, :]
            out[r][:, a] = m.face_lo[e][a]
        return out

    def boundary_points(self):
        return self.face_points(self.mesh.bface_ids)

    # ---------------------------------------------------------------- helpers
    def at_face(self, Uc, f):
        """Values of per-element nodal fields Uc (nel, nb) at local face f's Gauss points."""
        return Uc @ self.ref.face_B[f].T

    def at_volume(self, Uc):
        return Uc @ self.ref.Bq.T

    def mass_norm2(self, Uc):
        """sum_K (u, u)_K for per-element nodal fields Uc (nel, nb)."""
        return float(np.einsum("ki,ij,kj->", Uc, self.M, Uc))

    def load(self, vals):
        """(f, phi_i)_K for f given at volume Gauss points, (nel, q^d) -> (nel, nb)."""
        wJ = self.ref.wq * self.jac
        return (vals * wJ[None, :]) @ self.ref.Bq


class Problem:
    """A linear PDE discretised by upwind HDG; subclasses give the local pieces.

    State U: (nel, nc, nb).  Trace T: (nface, q^(d-1)), one scalar trace per face point.
    """

    nc = 1

    def __init__(self, disc: Discretisation):
        self.disc = disc
        self.mesh = disc.mesh
        self.nvol = self.nc * disc.nb
        self.A = self.local_matrix()

    # subclass API -------------------------------------------------------
    def local_matrix(self):
        raise NotImplementedError

    def volume_rhs(self, f_qp, U_prev=None):
        raise NotImplementedError

    def traces(self, U, g_qp):
        """Trace on every global face from the volume state (Eq. iHDGtrace)."""
        raise NotImplementedError

    def trace_rhs(self, T):
        """Element right-hand-side contributions of the face traces."""
        raise NotImplementedError

    def norm2(self, dU):
        raise NotImplementedError

    def trace_coupling(self):
        """For the direct solve: per local face f, (nvol x q^(d-1)) matrix W_f with
        rhs contribution = W_f @ T_face (the linear map used by trace_rhs)."""
        raise NotImplementedError

    def face_equation(self, e, side_vals, g_row):
        raise NotImplementedError

    # shared -----------------------------------------------------------------
    def elem_traces(self, T):
        """(nel, 2d, q^(d-1)) traces seen by each element on each of its local faces."""
        return T[self.mesh.elem_face]

    def face_side_values(self, U, comps):
        """For each global face: values of components `comps` from its left/right element at
        the face points: dict comp -> (left (nface,nqf), right (nface,nqf)); missing = nan."""
        m, disc = self.mesh, self.disc
        out = {}
        for c in comps:
            L = np.full((m.nface, disc.nqf), np.nan)
            R = np.full((m.nface, disc.nqf), np.nan)
            for a in range(disc.d):
                sel = m.face_axis == a
                ids = np.nonzero(sel)[0]
                left, right = m.face_left[sel], m.face_right[sel]
                okl, okr = left >= 0, right >= 0
                L[ids[okl]] = disc.at_face(U[left[okl], c, :], 2 * a + 1)
                R[ids[okr]] = disc.at_face(U[right[okr], c, :], 2 * a)
            out[c] = (L, R)
        return out

    def solve_local(self, rhs):
        """u = A^{-1} rhs for every element (nel, nvol) -> (nel, nc, nb)."""
        sol = np.linalg.solve(self.A, rhs.T).T
        return sol.reshape(-1, self.nc, self.disc.nb)

    def sweep(self, U, f_qp, g_qp, U_prev=None):
        """One iHDG iteration of Algorithm 1: traces from u^k, then all local solves."""
        T = self.traces(U, g_qp)
        rhs = self.volume_rhs(f_qp, U_prev) + self.trace_rhs(T)
        return self.solve_local(rhs)

    def iterate(self, f_qp, g_qp, tol, max_iters=2000, U0=None, U_prev=None,
                diverge_factor=1e6, history=False):
        """Algorithm 1 until ||u^k - u^(k-1)|| < tol.  Returns (U^K, trace, K, res, status)."""
        U = np.zeros((self.mesh.nel, self.nc, self.disc.nb)) if U0 is None else np.array(U0, dtype=np.float64)
        res_min = np.inf
        hist = []
        status = STATUS_NOT_CONVERGED
        k = 0
        res = np.inf
        while k < max_iters:
            Un = self.sweep(U, f_qp, g_qp, U_prev)
            res = np.sqrt(self.norm2(Un - U))
            U = Un
            k += 1
            hist.append(res)
            if res < tol:
                status = STATUS_OK
                break
            if not np.isfinite(res) or res > diverge_factor * res_min:
                status = STATUS_DIVERGED
                break
            res_min = min(res_min, res)
        T = self.traces(U, g_qp)
        out = (U, T, k, res, status)
        return out + (np.array(hist),) if history else out

    # ---------------------------------------------------------------- direct solve
    def direct_solve(self, f_qp, g_qp, U_prev=None):
        """Static condensation of the monolithic HDG system (HDGlocal + HDGeqn).

        Unknowns: one trace value per face Gauss point (the trace space is represented by
        its point values; with q = p+2 > p+1 points this over-parameterises Q^p(e), so the
        face equations are imposed pointwise-weighted, which is equivalent for polynomial
        traces).  U_K = A^{-1}(b_K + sum_f W_f T_f), then every face's conservation
        residual is linear in T; the square system is solved densely.
        """
        m, disc = self.mesh, self.disc
        nqf = disc.nqf
        nT = m.nface * nqf
        b = self.volume_rhs(f_qp, U_prev)
        Ainv = np.linalg.inv(self.A)
        W = self.trace_coupling()
        # U_K = U0_K + sum_f Lf[f] T_{face(K,f)},  Lf[f] = A^{-1} W_f
        U0 = (Ainv @ b.T).T
        Lf = [Ainv @ W[f] for f in range(2 * disc.d)]
        # build the map T -> face-equation residual: r(T) = S T - r0
        S = np.zeros((nT, nT))
        r0 = np.zeros(nT)
        # affine evaluation by probing: residual(T) is affine in T
        base = self._face_residuals(U0.reshape(-1, self.nc, disc.nb), np.zeros(nT), g_qp)
        r0[:] = -base
        for col in range(nT):
            e, j = divmod(col, nqf)
            Ucol = np.zeros((m.nel, self.nvol))
            for side, lf in ((m.face_left[e], 2 * m.face_axis[e] + 1), (m.face_right[e], 2 * m.face_axis[e])):
                if side >= 0:
                    Ucol[side] += Lf[lf][:, j]
            Tcol = np.zeros(nT)
            Tcol[col] = 1.0
            S[:, col] = self._face_residuals(Ucol.reshape(-1, self.nc, disc.nb), Tcol, g_qp, homogeneous=True)
        T = np.linalg.solve(S, r0).reshape(m.nface, nqf)
        Te = self.elem_traces(T)
        U = U0.copy()
        for f in range(2 * disc.d):
            U += Te[:, f, :] @ Lf[f].T
        return U.reshape(-1, self.nc, disc.nb), T

    def _face_residuals(self, U, Tflat, g_qp, homogeneous=False):
        """Conservation residual of every face at every face point, flattened."""
        m, disc = self.mesh, self.disc
        T = Tflat.reshape(m.nface, disc.nqf)
        vals = self.face_side_values(U, range(self.nc))
        g = np.zeros_like(g_qp) if homogeneous else g_qp
        return self.face_equations(vals, T, g).ravel()


# =============================================================================
class Transport(Problem):
    """Steady scalar transport beta.grad u = f, constant beta (Section 3).

    Upwind HDG flux (flux="upwind"):
      Local equation (transportLocalk1):
          -(u, div(beta v))_K + <beta.n u + |beta.n|(u - u_hat^k), v>_dK = (f, v)_K
      Weighted trace (transportLocale): |beta.n| u_hat = {{beta.n u}} + |beta.n| {{u}},
      i.e. the upwind value; g on the inflow boundary.
    nu >= 0 adds the L2 term nu (u^{k+1}, v)_K to the local equation: the term a backward-
      Euler step of the time-dependent equation adds with nu = 1/dt (the remark on
      time-dependent transport after Theorem 1), the step's u^m/dt going into the forcing.
    NPC flux (flux="npc", Section 3, Eq. Ntaub):
      Local equation -(u, div(beta v))_K + <beta.n u + tau (u - u_hat^k), v>_dK = (f, v)_K
      with tau = |beta.n| (1 + sgn(beta.n))/2 - beta.n: 0 on outflow faces, |beta.n| on
      inflow faces.  Trace ({{tau u}} + {{beta.n u}})/{{tau}}: on a face where the flow goes
      from K^- to K^+ (beta.n^- = b > 0) tau^- = 0 and tau^+ = b, so the trace is u^-, the
      upwind value again; the outflow faces no longer feed back into their own element.
    """

    nc = 1

    def __init__(self, disc, beta, flux="upwind", nu=0.0):
        self.beta = np.asarray(beta, dtype=np.float64)[: disc.d]
        if flux not in ("upwind", "npc"):
            raise ValueError("flux must be 'upwind' or 'npc'")
        self.flux = flux
        self.nu = float(nu)
        super().__init__(disc)

    def bn(self, f):
        return float(self.disc.normal[f] @ self.beta)

    @staticmethod
    def tau_npc(bn):
        """Eq. Ntaub: tau = |beta.n| (1 + sgn(beta.n))/2 - beta.n."""
        return abs(bn) * (1.0 + np.sign(bn)) / 2.0 - bn

    def tau(self, f):
        """Stabilisation on face f: |beta.n| (upwind) or Eq. Ntaub (NPC)."""
        bn = self.bn(f)
        return abs(bn) if self.flux == "upwind" else self.tau_npc(bn)

    def local_matrix(self):
        disc = self.disc
        # -(u, beta.grad v) (constant beta, so div(beta v) = beta.grad v)
        A = -sum(self.beta[a] * disc.K[a] for a in range(disc.d))
        for f in range(2 * disc.d):
            A = A + (self.bn(f) + self.tau(f)) * disc.Mf[f]
        return A + self.nu * disc.M

    def volume_rhs(self, f_qp, U_prev=None):
        return self.disc.load(f_qp)

    def traces(self, U, g_qp):
        m = self.mesh
        L, R = self.face_side_values(U, [0])[0]
        b = self.beta[m.face_axis][:, None]          # beta . (left element's outward normal)
        hasL = (m.face_left >= 0)[:, None]
        hasR = (m.face_right >= 0)[:, None]
        gfull = np.zeros_like(L)
        gfull[m.bface_ids] = g_qp
        up_left = np.where(hasL, L, gfull)            # flow left -> right
        up_right = np.where(hasR, R, gfull)           # flow right -> left
        avg = np.where(hasL & hasR, 0.5 * (np.nan_to_num(L) + np.nan_to_num(R)), np.where(hasL, L, R))
        return np.where(b > 0, up_left, np.where(b < 0, up_right, avg))

    def trace_coupling(self):
        disc = self.disc
        return [self.tau(f) * disc.Ff[f] for f in range(2 * disc.d)]

    def trace_rhs(self, T):
        Te = self.elem_traces(T)
        W = self.trace_coupling()
        return sum(Te[:, f, :] @ W[f].T for f in range(2 * self.disc.d))

    def norm2(self, dU):
        return self.disc.mass_norm2(dU[:, 0, :])

    def face_equations(self, vals, T, g):
        """Conservation (transportGlobal) on interior faces: [[beta.n u + tau (u - u_hat)]]
        = 0; inflow boundary u_hat = g; outflow boundary u_hat = u^-; beta.n = 0: u_hat = {{u}}."""
        m = self.mesh
        L, R = (np.nan_to_num(v) for v in vals[0])
        b = self.beta[m.face_axis][:, None]
        hasL = (m.face_left >= 0)[:, None]
        hasR = (m.face_right >= 0)[:, None]
        gfull = np.zeros_like(T)
        gfull[m.bface_ids] = g
        if self.flux == "upwind":
            tL = tR = np.abs(b)
        else:   # the left element's normal is +axis (beta.n = b), the right one's -axis
            tL = self.tau_npc(b)
            tR = self.tau_npc(-b)
        interior = np.where(b != 0, b * L - b * R + tL * (L - T) + tR * (R - T), 0.5 * (L + R) - T)
        own = np.where(hasL, L, R)
        inflow = ((b > 0) & ~hasL) | ((b < 0) & ~hasR)
        boundary = np.where(inflow, gfull - T, own - T)
        return np.where(hasL & hasR, interior, boundary)



# =============================================================================
class TransportVar(Problem):
    """Steady transport beta.grad u = f with a velocity field beta(x) that varies in space
    (Section 3, Eq. transport; beta continuous across the skeleton), upwind HDG flux.

    Every element has its own local matrix.  The local equation (transportLocalk1) is used in
    its integrated-by-parts form
        (beta.grad u^{k+1}, v)_K + <|beta.n| (u^{k+1} - u_hat^k), v>_dK = (f, v)_K,
    which equals the printed form -(u, div(beta v))_K + <beta.n u + |beta.n|(u - u_hat), v>_dK
    under exact integration and needs beta, not div(beta), at the quadrature points.  Every
    integral is a Gauss sum with beta sampled at the quadrature points.  The weighted trace
    (transportLocale) is formed point by point on each face: the upwind side's u^k where
    beta.n != 0 (g on the inflow boundary), so a face may be inflow in one part and outflow
    in another.  beta_fn maps physical points (..., d) to velocities (..., d).
    """

    nc = 1

    def __init__(self, disc, beta_fn):
        m = disc.mesh
        self.beta_fn = beta_fn
        self.bq = np.asarray(beta_fn(disc.volume_points()), dtype=np.float64)            # (nel, nq, d)
        self.bf = np.asarray(beta_fn(disc.face_points(np.arange(m.nface))), dtype=np.float64)  # (nface, nqf, d)
        # beta . (outward normal of local face f) at that face's points, per element
        self.bn = np.zeros((m.nel, 2 * disc.d, disc.nqf))
        for f in range(2 * disc.d):
            self.bn[:, f, :] = self.bf[m.elem_face[:, f]] @ disc.normal[f]
        super().__init__(disc)

    def local_matrix(self):
        disc, ref, h = self.disc, self.disc.ref, self.mesh.h
        wJ = ref.wq * disc.jac
        # (beta.grad phi_j)(x_q), physical gradient of the reference basis
        bgrad = sum(self.bq[:, :, a, None] * ((2.0 / h[a]) * ref.Dq[a])[None] for a in range(disc.d))
        A = np.einsum("q,kqj,qi->kij", wJ, bgrad, ref.Bq)
        for f in range(2 * disc.d):
            w = np.abs(self.bn[:, f, :]) * (ref.face_w * disc.face_jac[f])[None, :]
            A += np.einsum("kq,qj,qi->kij", w, ref.face_B[f], ref.face_B[f])
        return A

    def solve_local(self, rhs):
        sol = np.linalg.solve(self.A, rhs[:, :, None])[:, :, 0]
        return sol.reshape(-1, self.nc, self.disc.nb)

    def volume_rhs(self, f_qp, U_prev=None):
        return self.disc.load(f_qp)

    def traces(self, U, g_qp):
        m = self.mesh
        L, R = self.face_side_values(U, [0])[0]
        b = self.bf[np.arange(m.nface), :, m.face_axis]   # beta . (left element's outward normal)
        hasL = (m.face_left >= 0)[:, None]
        hasR = (m.face_right >= 0)[:, None]
        gfull = np.zeros_like(L)
        gfull[m.bface_ids] = g_qp
        up_left = np.where(hasL, L, gfull)
        up_right = np.where(hasR, R, gfull)
        avg = np.where(hasL & hasR, 0.5 * (np.nan_to_num(L) + np.nan_to_num(R)), np.where(hasL, L, R))
        return np.where(b > 0, up_left, np.where(b < 0, up_right, avg))

    def trace_coupling(self):
        """Per element and local face: (nel, nb, q^(d-1)) maps of the face trace to the rhs."""
        disc, ref = self.disc, self.disc.ref
        return [ref.face_B[f].T[None, :, :] * (np.abs(self.bn[:, f, :]) * (ref.face_w * disc.face_jac[f])[None, :])[:, None, :]
                for f in range(2 * disc.d)]

    def trace_rhs(self, T):
        Te = self.elem_traces(T)
        W = self.trace_coupling()
        return sum(np.einsum("kiq,kq->ki", W[f], Te[:, f, :]) for f in range(2 * self.disc.d))

    def norm2(self, dU):
        return self.disc.mass_norm2(dU[:, 0, :])

    def face_equations(self, vals, T, g):
        """Conservation (transportGlobal) point by point: [[beta.n u + |beta.n|(u - u_hat)]] = 0
        on interior faces where beta.n != 0, u_hat = {{u}} where beta.n = 0; on the boundary
        u_hat = g where the flow enters and u_hat = u^- elsewhere."""
        m = self.mesh
        L, R = (np.nan_to_num(v) for v in vals[0])
        b = self.bf[np.arange(m.nface), :, m.face_axis]
        hasL = (m.face_left >= 0)[:, None]
        hasR = (m.face_right >= 0)[:, None]
        gfull = np.zeros_like(T)
        gfull[m.bface_ids] = g
        ab = np.abs(b)
        interior = np.where(b != 0, b * L - b * R + ab * (L - T) + ab * (R - T), 0.5 * (L + R) - T)
        own = np.where(hasL, L, R)
        inflow = ((b > 0) & ~hasL) | ((b < 0) & ~hasR)
        boundary = np.where(inflow, gfull - T, own - T)
        return np.where(hasL & hasR, interior, boundary)

    def direct_solve(self, f_qp, g_qp, U_prev=None):
        """Static condensation of (HDGlocal) + (transportGlobal) with per-element local
        matrices: U_K = A_K^{-1}(b_K + sum_f W_Kf T_f), then the face residuals are affine in
        the face-point traces T; the square system is assembled by probing and solved densely."""
        m, disc = self.mesh, self.disc
        nqf = disc.nqf
        nT = m.nface * nqf
        b = self.volume_rhs(f_qp, U_prev)
        U0 = np.linalg.solve(self.A, b[:, :, None])[:, :, 0]
        W = self.trace_coupling()
        Lf = [np.linalg.solve(self.A, W[f]) for f in range(2 * disc.d)]     # (nel, nb, nqf)
        S = np.zeros((nT, nT))
        r0 = -self._face_residuals(U0.reshape(-1, self.nc, disc.nb), np.zeros(nT), g_qp)
        for col in range(nT):
            e, j = divmod(col, nqf)
            Ucol = np.zeros((m.nel, self.nvol))
            for side, lf in ((m.face_left[e], 2 * m.face_axis[e] + 1), (m.face_right[e], 2 * m.face_axis[e])):
                if side >= 0:
                    Ucol[side] += Lf[lf][side][:, j]
            Tcol = np.zeros(nT)
            Tcol[col] = 1.0
            S[:, col] = self._face_residuals(Ucol.reshape(-1, self.nc, disc.nb), Tcol, g_qp, homogeneous=True)
        T = np.linalg.solve(S, r0).reshape(m.nface, nqf)
        Te = self.elem_traces(T)
        U = U0.copy()
        for f in range(2 * disc.d):
            U += np.einsum("kij,kj->ki", Lf[f], Te[:, f, :])
        return U.reshape(-1, self.nc, disc.nb), T


# =============================================================================
class ConvDiff(Problem):
    """Convection-diffusion in first-order form (Section 4.1):
        kappa^{-1} sigma + grad u = 0,  div sigma + beta.grad u + nu u = f,
    unknowns ordered (sigma_1, ..., sigma_d, u).  Local equations (ErrorDDMCD1/2) with the
    forcing and the trace u_hat^k = ([[sigma.n]] + [[beta.n u]] + [[tau u]]) / (tau^+ + tau^-)
    (from the conservation condition), with the upwind stabilisation
    tau^+- = (alpha - beta.n^+-)/2, alpha = sqrt((beta.n)^2 + 4).  Dirichlet u_hat = g.
    tau_gamma > 0 selects the mesh-dependent stabilisation the paper takes for the elliptic
    limit (Section 4.2): tau = tau_gamma (p+1)(p+2)/h on both sides of every face, h the
    element size along the face normal.
    """

    def __init__(self, disc, beta, kappa, nu=0.0, tau_gamma=None):
        self.nc = disc.d + 1
        self.beta = np.asarray(beta, dtype=np.float64)[: disc.d]
        self.kappa, self.nu = float(kappa), float(nu)
        self.tau_gamma = None if not tau_gamma else float(tau_gamma)
        super().__init__(disc)

    def tau_mesh(self, a):
        """Section 4.2: tau = gamma (p+1)(p+2)/h on faces normal to axis a."""
        p = self.disc.p
        return self.tau_gamma * (p + 1) * (p + 2) / float(self.mesh.h[a])

    def side_taus(self, b, a):
        """(tau on the left element's side, on the right element's side) of faces normal to
        axis a, where b = beta.n of the left element (its outward normal is +e_a)."""
        if self.tau_gamma:
            t = self.tau_mesh(a)
            return t + 0.0 * b, t + 0.0 * b
        al = np.sqrt(b * b + 4.0)
        return 0.5 * (al - b), 0.5 * (al + b)

    def bn(self, f):
        return float(self.disc.normal[f] @ self.beta)

    def alpha(self, f):
        return np.sqrt(self.bn(f) ** 2 + 4.0)

    def tau(self, f):
        if self.tau_gamma:
            return self.tau_mesh(f // 2)
        return 0.5 * (self.alpha(f) - self.bn(f))

    def local_matrix(self):
        disc, d, nb = self.disc, self.disc.d, self.disc.nb
        A = np.zeros((self.nc * nb, self.nc * nb))
        blk = lambda r, c: (slice(r * nb, (r + 1) * nb), slice(c * nb, (c + 1) * nb))
        iu = d
        for c in range(d):
            A[blk(c, c)] += disc.M / self.kappa          # kappa^{-1}(sigma_c, w)
            A[blk(c, iu)] += -disc.K[c]                  # -(u, d_c w)
            A[blk(iu, c)] += -disc.K[c]                  # -(sigma_c, d_c v)
        A[blk(iu, iu)] += -sum(self.beta[c] * disc.K[c] for c in range(d))   # -(u, beta.grad v)
        A[blk(iu, iu)] += self.nu * disc.M                                  # +nu (u, v)
        for f in range(2 * d):
            n = disc.normal[f]
            for c in range(d):
                if n[c] != 0:
                    A[blk(iu, c)] += n[c] * disc.Mf[f]                      # <sigma.n, v>
            A[blk(iu, iu)] += (self.bn(f) + self.tau(f)) * disc.Mf[f]       # <(beta.n + tau)u, v>
        return A

    def volume_rhs(self, f_qp, U_prev=None):
        nb, d = self.disc.nb, self.disc.d
        rhs = np.zeros((self.mesh.nel, self.nc * nb))
        rhs[:, d * nb:] = self.disc.load(f_qp)
        return rhs

    def trace_coupling(self):
        disc, d, nb = self.disc, self.disc.d, self.disc.nb
        W = []
        for f in range(2 * d):
            Wf = np.zeros((self.nc * nb, disc.nqf))
            for c in range(d):
                Wf[c * nb:(c + 1) * nb] = -disc.normal[f, c] * disc.Ff[f]   # -<u_hat, w.n>
            Wf[d * nb:] = self.tau(f) * disc.Ff[f]                          # <tau u_hat, v>
            W.append(Wf)
        return W

    def trace_rhs(self, T):
        Te = self.elem_traces(T)
        W = self.trace_coupling()
        return sum(Te[:, f, :] @ W[f].T for f in range(2 * self.disc.d))

    def traces(self, U, g_qp):
        m, d = self.mesh, self.disc.d
        vals = self.face_side_values(U, range(self.nc))
        b = self.beta[m.face_axis][:, None]          # beta . n^- with n^- = +e_a (left element)
        tL, tR = np.zeros_like(b), np.zeros_like(b)
        sL = np.zeros((m.nface, self.disc.nqf))
        sR = np.zeros_like(sL)
        for a in range(d):
            sel = m.face_axis == a
            sL[sel], sR[sel] = vals[a][0][sel], vals[a][1][sel]
            tL[sel], tR[sel] = self.side_taus(b[sel], a)
        uL, uR = vals[d]
        T = (sL - sR + (tL + b) * uL + (tR - b) * uR) / (tL + tR)
        T[m.bface_ids] = g_qp
        return T

    def norm2(self, dU):
        return self.disc.mass_norm2(dU[:, self.disc.d, :])

    def face_equations(self, vals, T, g):
        """[[sigma.n + beta.n u + tau(u - u_hat)]] = 0 inside; u_hat = g on the boundary."""
        m, d = self.mesh, self.disc.d
        b = self.beta[m.face_axis][:, None]
        tL, tR = np.zeros_like(b), np.zeros_like(b)
        sL = np.zeros_like(T)
        sR = np.zeros_like(T)
        for a in range(d):
            sel = m.face_axis == a
            sL[sel], sR[sel] = vals[a][0][sel], vals[a][1][sel]
            tL[sel], tR[sel] = self.side_taus(b[sel], a)
        uL, uR = vals[d]
        out = (sL - sR) + b * uL - b * uR + tL * (uL - T) + tR * (uR - T)
        gfull = np.zeros_like(T)
        gfull[m.bface_ids] = g
        out[m.bface_ids] = (gfull - T)[m.bface_ids]
        return out


# =============================================================================
class ShallowWater(Problem):
    """Linearized shallow water (Section 3), backward Euler step from q^m, unknowns
    (phi, u, v), local solver (localSolverDD) plus the time-derivative data on the right:
        (phi/dt, w) - (Phi vel, grad w) + <Phi vel.n + sqrt(Phi)(phi - phi_hat^k), w> = (phi^m/dt, w)
        (Phi u/dt, w) - (Phi phi, d_x w) + <Phi phi_hat^k n_1, w> = (Phi u^m/dt + f Phi v - g Phi u, w)
        (Phi v/dt, w) - (Phi phi, d_y w) + <Phi phi_hat^k n_2, w> = (Phi v^m/dt - f Phi u - g Phi v, w)
    with phi_hat^k = {{phi^k}} + sqrt(Phi) {{vel^k . n}}; walls use the mirror state.
    (f = Coriolis parameter, constant; g = bottom friction gamma; no wind stress.)
    """

    nc = 3

    def __init__(self, disc, Phi, dt, coriolis=0.0, friction=0.0):
        assert disc.d == 2
        self.Phi, self.dt = float(Phi), float(dt)
        self.fc, self.gam = float(coriolis), float(friction)
        super().__init__(disc)

    def local_matrix(self):
        disc, nb = self.disc, self.disc.nb
        P, sP, dt = self.Phi, np.sqrt(self.Phi), self.dt
        A = np.zeros((3 * nb, 3 * nb))
        blk = lambda r, c: (slice(r * nb, (r + 1) * nb), slice(c * nb, (c + 1) * nb))
        A[blk(0, 0)] += disc.M / dt
        A[blk(0, 1)] += -P * disc.K[0]
        A[blk(0, 2)] += -P * disc.K[1]
        for f in range(4):
            n = disc.normal[f]
            A[blk(0, 1)] += P * n[0] * disc.Mf[f]
            A[blk(0, 2)] += P * n[1] * disc.Mf[f]
            A[blk(0, 0)] += sP * disc.Mf[f]
        A[blk(1, 1)] += (P / dt + self.gam * P) * disc.M
        A[blk(1, 0)] += -P * disc.K[0]
        A[blk(1, 2)] += -self.fc * P * disc.M
        A[blk(2, 2)] += (P / dt + self.gam * P) * disc.M
        A[blk(2, 0)] += -P * disc.K[1]
        A[blk(2, 1)] += self.fc * P * disc.M
        return A

    def volume_rhs(self, f_qp, U_prev):
        disc, nb = self.disc, self.disc.nb
        rhs = np.zeros((self.mesh.nel, 3 * nb))
        rhs[:, :nb] = U_prev[:, 0, :] @ disc.M.T / self.dt
        rhs[:, nb:2 * nb] = self.Phi * U_prev[:, 1, :] @ disc.M.T / self.dt
        rhs[:, 2 * nb:] = self.Phi * U_prev[:, 2, :] @ disc.M.T / self.dt
        return rhs

    def trace_coupling(self):
        disc, nb = self.disc, self.disc.nb
        W = []
        for f in range(4):
            n = disc.normal[f]
            Wf = np.zeros((3 * nb, disc.nqf))
            Wf[:nb] = np.sqrt(self.Phi) * disc.Ff[f]
            Wf[nb:2 * nb] = -self.Phi * n[0] * disc.Ff[f]
            Wf[2 * nb:] = -self.Phi * n[1] * disc.Ff[f]
            W.append(Wf)
        return W

    def trace_rhs(self, T):
        Te = self.elem_traces(T)
        W = self.trace_coupling()
        return sum(Te[:, f, :] @ W[f].T for f in range(4))

    def traces(self, U, g_qp=None):
        m = self.mesh
        vals = self.face_side_values(U, [0, 1, 2])
        sP = np.sqrt(self.Phi)
        phL, phR, vnL, vnR = self._sides(vals)
        hasL = (m.face_left >= 0)[:, None]
        hasR = (m.face_right >= 0)[:, None]
        inner = 0.5 * (phL + phR) + 0.5 * sP * (vnL - vnR)   # n^- = +e_a, n^+ = -e_a
        wall_right = phL + sP * vnL                           # only a left element, normal +e_a
        wall_left = phR - sP * vnR                            # only a right element, normal -e_a
        return np.where(hasL & hasR, inner, np.where(hasL, wall_right, wall_left))

    def _sides(self, vals):
        """phi and the velocity component along the face axis, left/right, nan -> 0."""
        m = self.mesh
        phL, phR = (np.nan_to_num(v) for v in vals[0])
        vnL = np.zeros_like(phL)
        vnR = np.zeros_like(phL)
        for a in range(2):
            sel = m.face_axis == a
            vnL[sel] = np.nan_to_num(vals[1 + a][0][sel])
            vnR[sel] = np.nan_to_num(vals[1 + a][1][sel])
        return phL, phR, vnL, vnR

    def norm2(self, dU):
        d = self.disc
        return d.mass_norm2(dU[:, 0, :]) + self.Phi * (d.mass_norm2(dU[:, 1, :]) + d.mass_norm2(dU[:, 2, :]))

    def face_equations(self, vals, T, g):
        """[[Phi vel.n + sqrt(Phi)(phi - phi_hat)]] = 0 inside; zero mass flux at walls."""
        m = self.mesh
        P, sP = self.Phi, np.sqrt(self.Phi)
        phL, phR, vnL, vnR = self._sides(vals)
        hasL = (m.face_left >= 0)[:, None]
        hasR = (m.face_right >= 0)[:, None]
        inner = P * (vnL - vnR) + sP * (phL + phR - 2 * T)
        wall_right = P * vnL + sP * (phL - T)
        wall_left = -P * vnR + sP * (phR - T)
        return np.where(hasL & hasR, inner, np.where(hasL, wall_right, wall_left))

    def step(self, U_m, tol, max_iters=2000):
        """One backward-Euler step with the iHDG iteration warm-started from q^m."""
        U, T, k, res, status = self.iterate(None, None, tol, max_iters, U0=U_m, U_prev=U_m)
        return U, T, k, res, status

    def step_direct(self, U_m):
        """One time step by the direct (static condensation) solve."""
        U, T = self.direct_solve(None, None, U_prev=U_m)
        return U


class ShallowWaterCN(ShallowWater):
    """Linearized shallow water, one Crank-Nicolson step of size dt (the time rule of the
    paper's shallow-water experiments): with N(q) = S q - sum_f W_f T_f(q) the element's HDG
    spatial residual (S: the local matrix without its time-derivative part; T(q): the trace
    of Section 3's formula evaluated from q), the step solves
        (M/dt)(q^{m+1} - q^m) = -(N(q^{m+1}) + N(q^m)) / 2.
    Multiplied by 2 this is a local problem with the time-derivative part 2M/dt (the
    backward-Euler local matrix at dt/2) and the right-hand side
        (2M/dt) q^m - N(q^m) = 2 (2M/dt) q^m - A q^m + sum_f W_f T_f(q^m),
    where A = 2M/dt + S is that local matrix.  The iHDG iteration is Algorithm 1 on this
    local problem, warm-started from q^m; the stopping test is on q^{m+1}'s iterates.
    """

    def __init__(self, disc, Phi, dt, coriolis=0.0, friction=0.0):
        super().__init__(disc, Phi, 0.5 * dt, coriolis, friction)
        self.dt_step = float(dt)

    def volume_rhs(self, f_qp, U_prev):
        mass = super().volume_rhs(f_qp, U_prev)            # (2M/dt) q^m, Phi-weighted rows
        Aq = U_prev.reshape(self.mesh.nel, -1) @ self.A.T   # A q^m per element
        return 2.0 * mass - Aq + self.trace_rhs(self.traces(U_prev))
