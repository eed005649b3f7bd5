"""Pins for the oracle's transport iHDG (Section 3, Theorem 1, Section 5.1).

* polynomial exactness (consistency of the upwind HDG discretisation);
* the converged iterate equals the static-condensation direct HDG solve (HDGeqn);
* the fixed point equals the textbook upwind DG solution (the trace (transportLocale) is
  the upwind value, so HDG collapses to upwind DG);
* p = 0 reduces to first-order upwind finite volumes (brute force);
* the contraction of Theorem 1: factor 1/2 on the squared outflow norm (transportLocalg),
  spectral radius exactly 1/2 in 1D and for p = 1 (the remark after Theorem 1);
* optimal h-convergence p+1 for the manufactured solution of the 2D transport workload;
* iteration counts nearly independent of p (Table 1 discussion).
"""
import numpy as np
import pytest

from oracle import BoxMesh, Discretisation, Transport
from oracle.ihdg import STATUS_OK


def poly_case(d, n, p, beta):
    m = BoxMesh(d, (n,) * d)
    disc = Discretisation(m, p)
    pr = Transport(disc, beta)
    coef = np.array([1.0, 2.0, -0.5])[:d]
    X = disc.volume_points()
    f = np.full(X.shape[:2], float(np.dot(beta[:d], coef)))
    G = disc.boundary_points()
    g = G @ coef
    ue = disc.node_points() @ coef
    return pr, f, g, ue


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_polynomial_exactness(d, p):
    beta = np.array([1.0, 0.5, 0.75])
    pr, f, g, ue = poly_case(d, 3, p, beta)
    U, T, k, res, st = pr.iterate(f, g, 1e-13)
    assert st == STATUS_OK
    assert np.abs(U[:, 0] - ue).max() < 1e-11
    Ud, Td = pr.direct_solve(f, g)
    assert np.abs(Ud[:, 0] - ue).max() < 1e-12


@pytest.mark.parametrize("d,p,beta", [(2, 2, (1.0, 0.5)), (2, 3, (-0.3, 1.0)), (3, 2, (0.6, -0.4, 0.7))])
def test_iteration_equals_direct_solve(d, p, beta):
    beta = np.array(beta)
    m = BoxMesh(d, (3,) * d)
    disc = Discretisation(m, p)
    pr = Transport(disc, beta)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((m.nel, disc.nq))
    g = rng.standard_normal((m.nbface, disc.nqf))
    U, T, k, res, st = pr.iterate(f, g, 1e-13)
    Ud, Td = pr.direct_solve(f, g)
    assert st == STATUS_OK
    assert np.abs(U - Ud).max() < 1e-11 * max(1.0, np.abs(Ud).max())
    # the iteration's trace on faces with nonzero flux matches the direct trace
    assert np.abs(T - Td).max() < 1e-10 * max(1.0, np.abs(Td).max())


def upwind_dg_solve(pr, f, g):
    """Textbook upwind DG: -(u, beta.grad v)_K + sum_f <beta.n u_up, v>_f = (f, v)_K, with
    u_up the upwind trace (g on the inflow boundary).  Assembled as one global system
    directly from quadrature tables, without traces or the iHDG weighting."""
    disc, m = pr.disc, pr.mesh
    ref, nb = disc.ref, disc.nb
    beta = pr.beta
    N = m.nel * nb
    A = np.zeros((N, N))
    rhs = disc.load(f).ravel()
    wJ = ref.wq * disc.jac
    vol = np.zeros((nb, nb))
    for a in range(disc.d):
        gradv = ref.Dq[a] * (2.0 / m.h[a])
        vol -= beta[a] * (gradv.T @ (wJ[:, None] * ref.Bq))       # row i = test v_i
    gfull = np.zeros((m.nface, disc.nqf))
    gfull[m.bface_ids] = g
    for K in range(m.nel):
        A[K * nb:(K + 1) * nb, K * nb:(K + 1) * nb] += vol
        for f_ in range(2 * disc.d):
            a, s = divmod(f_, 2)
            bn = beta[a] * (1.0 if s == 1 else -1.0)
            wf = ref.face_w * disc.face_jac[f_]
            Bv = ref.face_B[f_]
            if bn > 0:      # outflow: own trace
                A[K * nb:(K + 1) * nb, K * nb:(K + 1) * nb] += bn * Bv.T @ (wf[:, None] * Bv)
            elif bn < 0:    # inflow: neighbour trace or boundary data
                nbk = m.nbr[K, f_]
                if nbk >= 0:
                    Bn = ref.face_B[f_ ^ 1]
                    A[K * nb:(K + 1) * nb, nbk * nb:(nbk + 1) * nb] += bn * Bv.T @ (wf[:, None] * Bn)
                else:
                    e = m.elem_face[K, f_]
                    rhs[K * nb:(K + 1) * nb] -= bn * Bv.T @ (wf * gfull[e])
    return np.linalg.solve(A, rhs).reshape(m.nel, 1, nb)


@pytest.mark.parametrize("d,p,beta", [(2, 1, (1.0, 0.5)), (2, 3, (0.8, -1.0)), (3, 1, (1.0, 1.0, 1.0))])
def test_fixed_point_is_upwind_dg(d, p, beta):
    beta = np.array(beta) / np.linalg.norm(beta)
    m = BoxMesh(d, (3,) * d)
    disc = Discretisation(m, p)
    pr = Transport(disc, beta)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((m.nel, disc.nq))
    g = rng.standard_normal((m.nbface, disc.nqf))
    U, T, k, res, st = pr.iterate(f, g, 1e-13)
    Udg = upwind_dg_solve(pr, f, g)
    assert np.abs(U - Udg).max() < 1e-11 * max(1.0, np.abs(Udg).max())


def test_p0_is_first_order_upwind_fv():
    """p = 0, beta = (b1, b2) > 0: (b1 + b2) u_ij = b1 u_{i-1,j} + b2 u_{i,j-1} + (1/h) int_K f."""
    n, b = 5, np.array([0.7, 1.3])
    m = BoxMesh(2, (n, n))
    disc = Discretisation(m, 0)
    pr = Transport(disc, b)
    rng = np.random.default_rng(11)
    f = rng.standard_normal((m.nel, disc.nq))
    g = rng.standard_normal((m.nbface, disc.nqf))
    U, T, k, res, st = pr.iterate(f, g, 1e-14)
    h = m.h[0]
    intf = (f * (disc.ref.wq * disc.jac)[None, :]).sum(axis=1)
    # boundary inflow data: face averages (p = 0 trace = L2 projection = mean)
    gfull = np.zeros((m.nface, disc.nqf))
    gfull[m.bface_ids] = g
    wf = disc.ref.face_w / disc.ref.face_w.sum()
    gmean = gfull @ wf
    u = np.zeros((n, n))
    for j in range(n):
        for i in range(n):
            K = i + n * j
            left = u[i - 1, j] if i > 0 else gmean[m.elem_face[K, 0]]
            down = u[i, j - 1] if j > 0 else gmean[m.elem_face[K, 2]]
            u[i, j] = (b[0] * left + b[1] * down + intf[K] / h) / (b[0] + b[1])
    assert np.abs(U[:, 0, 0] - u.T.ravel()).max() < 1e-12


def element_self_map(d, p, beta):
    """Homogeneous iteration on one element with zero inflow data:
    u^{k+1} = A^{-1} sum_{outflow f} |beta.n| <u^k, v>_f  (Eqs. transportLocalk1/transportLocale)."""
    beta = np.array(beta, dtype=float)
    m = BoxMesh(d, (1,) * d)
    disc = Discretisation(m, p)
    pr = Transport(disc, beta)
    S = np.zeros((disc.nb, disc.nb))
    for f_ in range(2 * d):
        bn = pr.bn(f_)
        if bn > 0:
            S += bn * disc.Ff[f_] @ disc.ref.face_B[f_]
    return pr, disc, np.linalg.solve(pr.A, S)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_contraction_exactly_one_half_1d(p):
    """1D: testing with v = 1 gives 2 w(h) = 1 for w = A^{-1} e_R, so the only nonzero
    eigenvalue of the self-map is 1/2 for every p (the remark after Theorem 1)."""
    _, _, T = element_self_map(1, p, (1.0,))
    assert abs(np.abs(np.linalg.eigvals(T)).max() - 0.5) < 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_contraction_one_half_p1(d):
    _, _, T = element_self_map(d, 1, (1.0, 0.5, 0.75)[:d])
    assert abs(np.abs(np.linalg.eigvals(T)).max() - 0.5) < 1e-6


@pytest.mark.parametrize("d,p", [(2, 2), (2, 3), (2, 4), (3, 2)])
def test_energy_contraction_inequality(d, p):
    """Eq. (transportLocalg) with div beta = 0 and zero inflow data:
    ||u^{k+1}||^2_{|beta.n|, out} <= 1/2 ||u^k||^2_{|beta.n|, out}; hence the element
    self-map's spectral radius is at most 1/sqrt(2)."""
    beta = (1.0, 0.5, 0.75)[:d]
    pr, disc, T = element_self_map(d, p, beta)
    rng = np.random.default_rng(5)

    def out_norm2(u):
        s = 0.0
        for f_ in range(2 * d):
            bn = pr.bn(f_)
            if bn > 0:
                tr = disc.ref.face_B[f_] @ u
                s += bn * np.sum(disc.ref.face_w * disc.face_jac[f_] * tr ** 2)
        return s

    for _ in range(20):
        u = rng.standard_normal(disc.nb)
        assert out_norm2(T @ u) <= 0.5 * out_norm2(u) * (1 + 1e-12)
    assert np.abs(np.linalg.eigvals(T)).max() <= 1 / np.sqrt(2) + 1e-12


def test_global_spectral_radius_equals_element_value():
    """Whole-mesh homogeneous iteration matrix: block triangular in the upwind order with
    every diagonal block the element self-map, so both spectral radii agree.  Its Jordan
    blocks make computed eigenvalues sensitive at the eps^(1/m) level (loose tolerance)."""
    m = BoxMesh(2, (2, 2))
    disc = Discretisation(m, 2)
    pr = Transport(disc, np.array([1.0, 0.5]))
    N = m.nel * disc.nb
    G = np.zeros((N, N))
    f = np.zeros((m.nel, disc.nq))
    g = np.zeros((m.nbface, disc.nqf))
    for c in range(N):
        U = np.zeros(N)
        U[c] = 1.0
        G[:, c] = pr.sweep(U.reshape(m.nel, 1, disc.nb), f, g).ravel()
    rho = np.abs(np.linalg.eigvals(G)).max()
    _, _, T = element_self_map(2, 2, (1.0, 0.5))
    assert abs(rho - np.abs(np.linalg.eigvals(T)).max()) < 1e-3


def mms_transport_2d(n, p):
    """The 2D transport workload: beta = (1, 0.5), u = sin(pi x) cos(pi y)."""
    beta = np.array([1.0, 0.5])
    m = BoxMesh(2, (n, n))
    disc = Discretisation(m, p)
    pr = Transport(disc, beta)
    X = disc.volume_points()
    x, y = X[..., 0], X[..., 1]
    f = beta[0] * np.pi * np.cos(np.pi * x) * np.cos(np.pi * y) - beta[1] * np.pi * np.sin(np.pi * x) * np.sin(np.pi * y)
    G = disc.boundary_points()
    g = np.sin(np.pi * G[..., 0]) * np.cos(np.pi * G[..., 1])
    U, T, k, res, st = pr.iterate(f, g, 1e-12)
    err = disc.at_volume(U[:, 0]) - np.sin(np.pi * x) * np.cos(np.pi * y)
    l2 = np.sqrt(np.sum(err ** 2 * (disc.ref.wq * disc.jac)[None, :]))
    return l2, k


@pytest.mark.parametrize("p", [1, 2])
def test_mms_rate(p):
    e = [mms_transport_2d(n, p)[0] for n in (4, 8, 16)]
    rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert rates[-1] > p + 0.8, rates


def test_iterations_nearly_independent_of_p():
    """Table 1: the upwind iteration count barely changes with p at a fixed mesh."""
    ks = [mms_transport_2d(8, p)[1] for p in (1, 2, 3, 4)]
    assert max(ks) <= 1.15 * min(ks), ks


# ------------------------------------------------------------------------------ NPC flux
def npc_case(d, n, p, beta, flux="npc"):
    """Manufactured problem of the 2D/3D transport workloads with the given flux."""
    import workloads as W
    m = BoxMesh(d, (n,) * d)
    disc = Discretisation(m, p)
    pr = Transport(disc, np.asarray(beta, dtype=float), flux=flux)
    X, G = disc.volume_points(), disc.boundary_points()
    if d == 2:
        f, g = W.transport2d_forcing(X, beta), W.transport2d_exact(G)
    else:
        f, g = W.transport3d_forcing(X, beta), W.transport3d_exact(G)
    return pr, f, g


def test_npc_tau_is_zero_on_outflow_and_abs_on_inflow():
    """Eq. Ntaub: tau = |b|(1+sgn b)/2 - b is 0 for b > 0, |b| for b < 0, 0 for b = 0."""
    for b in (0.3, 2.0):
        assert Transport.tau_npc(b) == 0.0
        assert Transport.tau_npc(-b) == b
    assert Transport.tau_npc(0.0) == 0.0


@pytest.mark.parametrize("d,n,p,beta", [(2, 4, 1, (1.0, 0.5)), (2, 5, 2, (0.3, 1.0)), (2, 3, 3, (-1.0, 0.7)),
                                        (3, 3, 1, (0.6, 0.8, 0.5)), (3, 2, 2, (1.0, -0.4, 0.9))])
def test_npc_finite_termination(d, n, p, beta):
    """Theorem (iHDG-NPC): with the NPC flux the iteration terminates.  On an n^d box with no
    zero component of beta an element's value depends only on its upwind neighbours, so the
    element at upwind graph distance m from the inflow corner is exact after m+1 sweeps: the
    iterate equals the direct solution after d(n-1)+1 sweeps and not one sweep earlier, and
    the stopping test first holds one sweep later.  (Table 1 lists 2n+1 for the 2D meshes,
    one more than the 2n here; the paper does not state its count convention.)"""
    pr, f, g = npc_case(d, n, p, beta)
    Ud, _ = pr.direct_solve(f, g)
    layers = d * (n - 1) + 1
    U_last = pr.iterate(f, g, 0.0, max_iters=layers)[0]
    U_prev = pr.iterate(f, g, 0.0, max_iters=layers - 1)[0]
    scale = np.abs(Ud).max()
    assert np.abs(U_last - Ud).max() < 1e-12 * scale
    assert np.abs(U_prev - Ud).max() > 1e-6 * scale
    U, T, K, res, st = pr.iterate(f, g, 1e-12, max_iters=1000)
    assert st == STATUS_OK and K == layers + 1


@pytest.mark.parametrize("d,p,beta", [(2, 2, (1.0, 0.5)), (2, 3, (-0.6, 1.0)), (3, 1, (0.6, -0.8, 0.5))])
def test_npc_and_upwind_share_the_fixed_point(d, p, beta):
    """Both fluxes make the trace the upwind value, so both HDG discretisations are upwind DG:
    the NPC direct solve, the NPC iterate and the upwind direct solve coincide."""
    pr_n, f, g = npc_case(d, 3, p, beta, "npc")
    pr_u, _, _ = npc_case(d, 3, p, beta, "upwind")
    Un, Tn = pr_n.direct_solve(f, g)
    Uu, Tu = pr_u.direct_solve(f, g)
    Ui, Ti, K, res, st = pr_n.iterate(f, g, 1e-13, max_iters=1000)
    assert st == STATUS_OK
    assert np.abs(Un - Uu).max() < 1e-11 and np.abs(Tn - Tu).max() < 1e-11
    assert np.abs(Ui - Un).max() < 1e-11


def test_npc_local_matrix_differs_from_upwind_only_on_outflow_faces():
    """A_npc = A_upwind - sum over outflow faces of |beta.n| M_f, and the trace coupling of
    an outflow face vanishes (a plain check of where Eq. Ntaub enters)."""
    disc = Discretisation(BoxMesh(2, (2, 2)), 2)
    beta = np.array([0.8, -0.5])
    pu, pn = Transport(disc, beta), Transport(disc, beta, flux="npc")
    D = pu.A - pn.A
    E = sum(max(pu.bn(f), 0.0) * disc.Mf[f] for f in range(4))
    assert np.abs(D - E).max() < 1e-14
    Wn = pn.trace_coupling()
    for f in range(4):
        if pu.bn(f) > 0:
            assert np.abs(Wn[f]).max() == 0.0
        else:
            assert np.abs(Wn[f] - pu.trace_coupling()[f]).max() < 1e-15
