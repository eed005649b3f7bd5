"""Pins for the oracle's convection-diffusion iHDG (Section 4, Theorem 4, Section 5.3).

* polynomial exactness of the HDG discretisation (u, sigma = -kappa grad u in Q^p);
* converged iteration equals the static-condensation direct solve (convergent regime);
* optimal h-convergence p+1 of the direct solution for the 2D convection-diffusion
  workload's manufactured solution;
* divergence where the paper predicts it: pure diffusion with the upwind tau for any mesh
  (Section 4.2) and the kappa = 1e-2 mixed regime on fine meshes (Section 5.3);
* the upwind count is insensitive to kappa when convection dominates (Table 3).
"""
import numpy as np
import pytest

from oracle import BoxMesh, ConvDiff, Discretisation
from oracle.ihdg import STATUS_DIVERGED, STATUS_OK


def make(d, n, p, beta, kappa, nu, h=None):
    hi = None if h is None else [n * h] * d
    m = BoxMesh(d, (n,) * d, hi=hi)
    disc = Discretisation(m, p)
    return m, disc, ConvDiff(disc, np.array(beta, dtype=float), kappa, nu)


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (3, 1)])
def test_polynomial_exactness(d, p):
    beta, kap, nu = [1.0, -0.5, 0.7][:d], 0.3, 1.0
    m, disc, pr = make(d, 3, p, beta, kap, nu)
    X = disc.volume_points()
    # u = x*y (+ z): sigma = -kappa grad u in Q^1, f = beta.grad u + nu u
    if d == 2:
        ue_f = lambda P: P[..., 0] * P[..., 1]
        grad = lambda P: np.stack([P[..., 1], P[..., 0]], -1)
    else:
        ue_f = lambda P: P[..., 0] * P[..., 1] + P[..., 2]
        grad = lambda P: np.stack([P[..., 1], P[..., 0], np.ones_like(P[..., 0])], -1)
    f = grad(X) @ np.array(beta) + nu * ue_f(X)
    g = ue_f(disc.boundary_points())
    Ud, Td = pr.direct_solve(f, g)
    N = disc.node_points()
    assert np.abs(Ud[:, d] - ue_f(N)).max() < 1e-12
    for c in range(d):
        assert np.abs(Ud[:, c] + kap * grad(N)[..., c]).max() < 1e-11


def test_iteration_equals_direct_solve_convection_dominated():
    m, disc, pr = make(2, 4, 2, [1.0, 0.6], 1e-3, 1.0)
    rng = np.random.default_rng(2)
    f = rng.standard_normal((m.nel, disc.nq))
    g = rng.standard_normal((m.nbface, disc.nqf))
    U, T, k, res, st = pr.iterate(f, g, 1e-13, max_iters=3000)
    Ud, Td = pr.direct_solve(f, g)
    assert st == STATUS_OK
    assert np.abs(U - Ud).max() < 1e-10 * max(1.0, np.abs(Ud).max())


def cd_workload_error(n, p, kappa=1e-2):
    """The 2D convection-diffusion workload: beta = (1,1), nu = 0,
    u = exp(x+y) sin(pi x) sin(pi y), g = 0; solved directly (the iteration diverges here)."""
    m, disc, pr = make(2, n, p, [1.0, 1.0], kappa, 0.0)
    X = disc.volume_points()
    x, y = X[..., 0], X[..., 1]
    E, sx, cx, sy, cy = np.exp(x + y), np.sin(np.pi * x), np.cos(np.pi * x), np.sin(np.pi * y), np.cos(np.pi * y)
    ux = E * sy * (sx + np.pi * cx)
    uy = E * sx * (sy + np.pi * cy)
    uxx = E * sy * ((1 - np.pi ** 2) * sx + 2 * np.pi * cx)
    uyy = E * sx * ((1 - np.pi ** 2) * sy + 2 * np.pi * cy)
    f = -kappa * (uxx + uyy) + ux + uy
    g = np.zeros((m.nbface, disc.nqf))
    Ud, Td = pr.direct_solve(f, g)
    err = disc.at_volume(Ud[:, 2]) - E * sx * sy
    return np.sqrt(np.sum(err ** 2 * (disc.ref.wq * disc.jac)[None, :]))


@pytest.mark.parametrize("p", [1, 2])
def test_mms_rate_direct(p):
    e = [cd_workload_error(n, p) for n in (4, 8, 16)]
    rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert rates[-1] > p + 0.8, rates


def spectral_radius(pr, m, disc, iters=150):
    rng = np.random.default_rng(0)
    U = rng.standard_normal((m.nel, pr.nc, disc.nb))
    f = np.zeros((m.nel, disc.nq))
    g = np.zeros((m.nbface, disc.nqf))
    r = []
    for _ in range(iters):
        U = pr.sweep(U, f, g)
        nn = np.sqrt(np.sum(U ** 2))
        U /= nn
        r.append(nn)
    return float(np.exp(np.mean(np.log(r[-40:]))))


@pytest.mark.parametrize("n", [2, 4, 8])
def test_pure_diffusion_upwind_tau_diverges(n):
    """Section 4.2: beta = 0, kappa = 1: the upwind tau = 1 violates B > 0 for any mesh."""
    m, disc, pr = make(2, n, 2, [0.0, 0.0], 1.0, 1.0)
    assert spectral_radius(pr, m, disc) > 1.0


def test_mixed_regime_diverges_on_fine_mesh_converges_when_convection_dominated():
    """kappa = 1e-2 with h = 1/256 (element Peclet ~0.55) diverges; kappa = 1e-4 at the
    same h (Peclet ~55) converges (Section 5.3, Theorem 4 conditions)."""
    m, disc, pr = make(2, 6, 3, [1.0, 1.0], 1e-2, 0.0, h=1 / 256)
    assert spectral_radius(pr, m, disc) > 5.0
    m, disc, pr = make(2, 6, 3, [1.0, 1.0], 1e-4, 0.0, h=1 / 256)
    assert spectral_radius(pr, m, disc) < 0.95


def test_upwind_count_insensitive_to_kappa():
    """Table 3 discussion: in the convection-dominated regime the upwind iHDG iteration
    count is insensitive to kappa (its stabilisation does not contain kappa)."""
    n, p = 6, 2
    ks = []
    rng = np.random.default_rng(4)
    for kap in (1e-4, 1e-7):
        m, disc, pr = make(2, n, p, [1.0, 0.5], kap, 0.0)
        f = rng.standard_normal((m.nel, disc.nq))
        g = rng.standard_normal((m.nbface, disc.nqf))
        _, _, k, _, st = pr.iterate(f, g, 1e-10, max_iters=3000)
        assert st == STATUS_OK
        ks.append(k)
    assert abs(ks[0] - ks[1]) <= 0.1 * max(ks), ks


# ------------------------------------------------------------------------------ mesh-dependent tau
def make_mesh_tau(d, n, p, beta, kappa, nu, gamma=1.0):
    m = BoxMesh(d, (n,) * d)
    disc = Discretisation(m, p)
    return m, disc, ConvDiff(disc, np.array(beta, dtype=float), kappa, nu, tau_gamma=gamma)


def elliptic_data(disc, d, kappa, nu):
    """u = prod sin(pi x_a): f = (d pi^2 kappa + nu) u (beta = 0), g = u on the boundary."""
    u = lambda P: np.prod(np.sin(np.pi * P), axis=-1)
    return (d * np.pi ** 2 * kappa + nu) * u(disc.volume_points()), u(disc.boundary_points())


def test_mesh_tau_value():
    """Section 4.2: tau = gamma (p+1)(p+2)/h on every face, both sides."""
    m = BoxMesh(2, (4, 5), hi=[2.0, 1.0])
    pr = ConvDiff(Discretisation(m, 3), np.array([0.3, 0.1]), 1.0, 0.0, tau_gamma=0.7)
    for f in range(4):
        h = [0.5, 0.2][f // 2]
        assert abs(pr.tau(f) - 0.7 * 4 * 5 / h) < 1e-12


@pytest.mark.parametrize("d,p", [(2, 2), (3, 1)])
def test_mesh_tau_polynomial_exactness(d, p):
    """The discretisation stays consistent for any tau > 0: u in Q^p is reproduced."""
    beta, kap, nu = [0.4, -0.3, 0.2][:d], 0.5, 1.0
    m, disc, pr = make_mesh_tau(d, 3, p, beta, kap, nu, gamma=2.0)
    coef = np.array([1.0, -2.0, 0.5])[:d]
    X = disc.volume_points()
    f = np.full(X.shape[:2], float(np.dot(beta, coef))) + nu * (X @ coef)
    g = disc.boundary_points() @ coef
    Ud, Td = pr.direct_solve(f, g)
    assert np.abs(Ud[:, d, :] - disc.node_points() @ coef).max() < 1e-10
    for a in range(d):   # sigma = -kappa grad u
        assert np.abs(Ud[:, a, :] + kap * coef[a]).max() < 1e-10


def test_mesh_tau_iteration_equals_direct_solve():
    m, disc, pr = make_mesh_tau(2, 4, 2, [0.0, 0.0], 1.0, 1.0)
    f, g = elliptic_data(disc, 2, 1.0, 1.0)
    U, T, K, r, st = pr.iterate(f, g, 1e-12, max_iters=5000)
    Ud, Td = pr.direct_solve(f, g)
    assert st == STATUS_OK
    assert np.abs(U - Ud).max() < 1e-9 * np.abs(Ud).max()


@pytest.mark.parametrize("d,n,p", [(2, 4, 1), (2, 4, 2), (3, 2, 1)])
def test_elliptic_limit_needs_mesh_tau(d, n, p):
    """Section 4.2: with beta = 0, kappa = 1 the upwind tau diverges and the mesh-dependent
    tau = (p+1)(p+2)/h converges."""
    m, disc, pr_u = make(d, n, p, [0.0] * d, 1.0, 1.0)
    f, g = elliptic_data(disc, d, 1.0, 1.0)
    assert pr_u.iterate(f, g, 1e-10, max_iters=3000)[4] == STATUS_DIVERGED
    pr_m = ConvDiff(disc, np.zeros(d), 1.0, 1.0, tau_gamma=1.0)
    assert pr_m.iterate(f, g, 1e-10, max_iters=3000)[4] == STATUS_OK


def test_mesh_tau_counts_grow_with_n_and_p():
    """Table 5's trend: the count grows with the number of elements and with p."""
    def count(n, p):
        m, disc, pr = make_mesh_tau(2, n, p, [0.0, 0.0], 1.0, 1.0)
        f, g = elliptic_data(disc, 2, 1.0, 1.0)
        U, T, K, r, st = pr.iterate(f, g, 1e-10, max_iters=5000)
        assert st == STATUS_OK
        return K
    k41, k42, k81 = count(4, 1), count(4, 2), count(8, 1)
    assert k41 < k42 and k41 < k81
