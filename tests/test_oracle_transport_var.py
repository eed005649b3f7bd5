"""Pins for the oracle's transport with a velocity field that varies in space (TransportVar,
Section 3 with the experiments of Section 5.1).

What fixes it, independently of its own code path:
  * with a constant field it is the constant-coefficient oracle (a different assembly: per
    element Gauss sums of beta.grad phi_j phi_i against Kronecker-product matrices);
  * polynomial exactness: when u is in Q^p and beta is linear, every integral is exact for
    q = p+2 Gauss points and upwind HDG reproduces u (consistency);
  * the converged iteration equals the static-condensation direct solve of HDGlocal +
    transportGlobal, also when beta.n changes sign inside a face (point-by-point upwinding);
  * Table 1 of the paper: the upwind iteration counts of the 2D experiment (beta = (1 +
    sin(pi y/2), 2), discontinuous inflow data) and of the 3D experiment (beta = (z, x, y))
    under the paper's own stopping tests, and the 3D experiment's convergence rate p+1.
"""
import numpy as np
import pytest

import workloads as W
from oracle import BoxMesh, Discretisation, Transport, TransportVar


def const_field(b):
    b = np.asarray(b, dtype=np.float64)
    return lambda X: np.broadcast_to(b, X.shape).copy()


@pytest.mark.parametrize("d,n,p,beta", [(2, (5, 4), 2, (1.0, 0.5)), (2, (3, 6), 3, (-0.7, 0.4)),
                                        (3, (2, 3, 2), 2, (0.5, -0.8, 0.3))])
def test_constant_field_is_the_constant_coefficient_oracle(d, n, p, beta):
    disc = Discretisation(BoxMesh(d, n), p)
    c, v = Transport(disc, np.array(beta)), TransportVar(disc, const_field(beta))
    assert np.abs(v.A - c.A[None]).max() < 1e-13
    X, B = disc.volume_points(), disc.boundary_points()
    f = W.transport2d_forcing(X, beta) if d == 2 else W.transport3d_forcing(X, beta)
    g = W.transport2d_exact(B) if d == 2 else W.transport3d_exact(B)
    Uc, Tc, Kc, _, _ = c.iterate(f, g, 1e-12)
    Uv, Tv, Kv, _, _ = v.iterate(f, g, 1e-12)
    assert Kc == Kv
    assert np.abs(Uc - Uv).max() < 1e-12 and np.abs(Tc - Tv).max() < 1e-12


def test_polynomial_exactness_2d():
    """beta = (1 + y, 2 - x) (linear, divergence-free), u = x y in Q^1: the converged
    solution is u's nodal interpolant for p = 1, 2, 3."""
    beta = lambda X: np.stack([1.0 + X[..., 1], 2.0 - X[..., 0]], axis=-1)
    u = lambda X: X[..., 0] * X[..., 1]
    f = lambda X: (1.0 + X[..., 1]) * X[..., 1] + (2.0 - X[..., 0]) * X[..., 0]
    for p in (1, 2, 3):
        disc = Discretisation(BoxMesh(2, (4, 3)), p)
        pr = TransportVar(disc, beta)
        U = pr.iterate(f(disc.volume_points()), u(disc.boundary_points()), 1e-13, max_iters=500)[0]
        assert np.abs(U[:, 0, :] - u(disc.node_points())).max() < 1e-11, p


def test_polynomial_exactness_3d():
    beta = lambda X: np.stack([1.0 + X[..., 2], 1.0 + X[..., 0], 1.0 + X[..., 1]], axis=-1)
    u = lambda X: X[..., 0] + 2.0 * X[..., 1] - X[..., 2] + X[..., 0] * X[..., 2]
    f = lambda X: (1.0 + X[..., 2]) * (1.0 + X[..., 2]) + 2.0 * (1.0 + X[..., 0]) + (1.0 + X[..., 1]) * (X[..., 0] - 1.0)
    disc = Discretisation(BoxMesh(3, (2, 3, 2)), 2)
    pr = TransportVar(disc, beta)
    U = pr.iterate(f(disc.volume_points()), u(disc.boundary_points()), 1e-13, max_iters=500)[0]
    assert np.abs(U[:, 0, :] - u(disc.node_points())).max() < 1e-11


@pytest.mark.parametrize("d,n,p,field", [
    (2, (4, 3), 2, "e1"),
    (2, (4, 4), 2, "sign_change"),      # beta_x = y - 0.45 changes sign inside x-faces
    (2, (3, 3), 3, "swirl"),
    (3, (2, 2, 2), 1, "e2"),
])
def test_iteration_equals_direct_solve(d, n, p, field):
    if field == "e1":
        beta, lo, hi = W.e1_beta, [0, 0], [2, 2]
    elif field == "sign_change":
        beta, lo, hi = (lambda X: np.stack([X[..., 1] - 0.45, np.ones_like(X[..., 0])], axis=-1)), None, None
    elif field == "swirl":
        beta, lo, hi = (lambda X: np.stack([1.2 + np.cos(2 * X[..., 1]), 0.8 + np.sin(3 * X[..., 0])], axis=-1)), None, None
    else:
        beta, lo, hi = W.e2_beta, None, None
    disc = Discretisation(BoxMesh(d, n, lo=lo, hi=hi), p)
    pr = TransportVar(disc, beta)
    X, B = disc.volume_points(), disc.boundary_points()
    if d == 2:
        f, g = W.transport2d_forcing(X), W.transport2d_exact(B)
    else:
        f, g = W.e2_forcing(X), W.e2_exact(B)
    U, T, K, res, st = pr.iterate(f, g, 1e-13, max_iters=3000)
    assert st == 0
    Ud, Td = pr.direct_solve(f, g)
    assert np.abs(U - Ud).max() < 1e-10 * max(1.0, np.abs(Ud).max())


# Table 1, upwind columns (the paper's 2D counts for p = 3 and 4 on 16 .. 1024 elements)
TABLE1_2D = {(4, 3): 65, (8, 3): 91, (16, 3): 133, (32, 3): 209, (4, 4): 65, (8, 4): 87, (16, 4): 129, (32, 4): 196}


@pytest.mark.parametrize("n,p", sorted(TABLE1_2D))
def test_table1_2d_upwind_counts(n, p):
    """The 2D experiment of Section 5.1 (f = 0, beta = (1 + sin(pi y/2), 2) on [0,2]^2, g = 1
    on x = 0, sin^6(pi x) on y = 0 up to x = 1, 0 beyond), stopped when ||u^k - u^(k-1)||_L2
    < 1e-10 as the paper states for it: the upwind iteration counts of Table 1, to within one
    sweep (the count convention is not stated; all but the 16-element p = 3 case agree)."""
    disc = Discretisation(BoxMesh(2, (n, n), lo=[0, 0], hi=[2, 2]), p)
    pr = TransportVar(disc, W.e1_beta)
    X, B = disc.volume_points(), disc.boundary_points()
    K = pr.iterate(np.zeros(X.shape[:2]), W.e1_inflow(B), 1e-10, max_iters=5000)[2]
    assert abs(K - TABLE1_2D[(n, p)]) <= 1, (K, TABLE1_2D[(n, p)])


def _e2_run(n, p):
    """E2 sweeps with the paper's 3D stopping test (Eq. tolerancecriteria):
    | ||u^k - u^e|| - ||u^(k-1) - u^e|| | < 1e-10.  Returns (count, final error)."""
    disc = Discretisation(BoxMesh(3, (n, n, n)), p)
    pr = TransportVar(disc, W.e2_beta)
    X, B = disc.volume_points(), disc.boundary_points()
    f, g, ue = W.e2_forcing(X), W.e2_exact(B), W.e2_exact(X)
    wJ = disc.ref.wq * disc.jac
    U = np.zeros((disc.mesh.nel, 1, disc.nb))
    prev = None
    for k in range(1, 2000):
        U = pr.sweep(U, f, g)
        err = float(np.sqrt(np.sum(wJ[None, :] * (disc.at_volume(U[:, 0, :]) - ue) ** 2)))
        if prev is not None and abs(err - prev) < 1e-10:
            return k, err
        prev = err
    raise AssertionError("no convergence")


def test_table1_3d_upwind_counts_and_rate():
    """The 3D experiment (beta = (z, x, y), u = sin(pi x) cos(pi y) sin(pi z)/pi on [0,1]^3):
    Table 1 lists 39 and 49 upwind iterations for p = 3 on 8 and 64 elements.  Exact counts
    depend on details the paper leaves open (initial guess, the norm's quadrature), so the pin
    is within 3 sweeps; the error falls at rate ~p + 1 between the two meshes."""
    K2, e2 = _e2_run(2, 3)
    K4, e4 = _e2_run(4, 3)
    assert abs(K2 - 39) <= 3 and abs(K4 - 49) <= 3, (K2, K4)
    assert np.log2(e2 / e4) > 3.5
