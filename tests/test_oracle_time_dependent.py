"""Pins for the time-dependent remarks: a backward-Euler step of transport (remark after
Theorem 1) or convection-diffusion (remark in Section 4.1) is the steady local problem with
the extra L2 term (u^{k+1}, v)_K / dt, i.e. the reaction nu = 1/dt, and the forcing
f + u^m/dt; the remarks say the term speeds the iteration up.

* a closed form: from u^m = P (a polynomial of the element space) and constant beta, the
  exact backward-Euler step of u_t + beta.grad u = 0 is Q = P - dt D P + dt^2 D^2 P - ...
  (D = beta.grad, nilpotent on polynomials); the HDG step reproduces Q exactly;
* with nu > 0 the iterate equals the direct solve;
* the iteration count falls as nu = 1/dt grows (transport and convection-diffusion).
"""
import numpy as np
import pytest

from oracle import BoxMesh, ConvDiff, Discretisation, Transport
from oracle.ihdg import STATUS_OK


def be_step_case(d, p, beta, dt):
    """u^m = P = x^2 + 2xy - y (+ xz in 3D); Q = P - dt DP + dt^2 D^2 P (D^3 P = 0)."""
    b = np.asarray(beta, dtype=float)

    def P(X):
        x, y = X[..., 0], X[..., 1]
        v = x * x + 2 * x * y - y
        return v + x * X[..., 2] if d == 3 else v

    def DP(X):
        x, y = X[..., 0], X[..., 1]
        v = b[0] * (2 * x + 2 * y) + b[1] * (2 * x - 1)
        if d == 3:
            v = v + b[0] * X[..., 2] + b[2] * x
        return v

    d2 = 2 * b[0] ** 2 + 4 * b[0] * b[1] + (2 * b[0] * b[2] if d == 3 else 0.0)
    Q = lambda X: P(X) - dt * DP(X) + dt * dt * d2
    m = BoxMesh(d, (3,) * d)
    disc = Discretisation(m, p)
    f = P(disc.volume_points()) / dt              # forcing f + u^m/dt with f = 0
    g = Q(disc.boundary_points())                 # inflow data of the stepped solution
    return disc, f, g, Q(disc.node_points()), P(disc.node_points())


@pytest.mark.parametrize("d,p,beta,flux", [(2, 2, (1.0, 0.5), "upwind"), (2, 3, (-0.3, 1.0), "upwind"),
                                           (3, 2, (0.6, -0.4, 0.7), "upwind"), (2, 2, (1.0, 0.5), "npc")])
def test_backward_euler_transport_step_is_exact_for_polynomials(d, p, beta, flux):
    dt = 0.05
    disc, f, g, Qn, Pn = be_step_case(d, p, beta, dt)
    pr = Transport(disc, np.array(beta), flux=flux, nu=1.0 / dt)
    U, T, k, res, st = pr.iterate(f, g, 1e-13, U0=Pn[:, None, :])
    assert st == STATUS_OK
    assert np.abs(U[:, 0] - Qn).max() < 1e-11 * max(1.0, np.abs(Qn).max())
    Ud, Td = pr.direct_solve(f, g)
    assert np.abs(Ud[:, 0] - Qn).max() < 1e-11 * max(1.0, np.abs(Qn).max())


def test_transport_with_reaction_iterate_equals_direct_solve():
    m = BoxMesh(2, (4, 3))
    disc = Discretisation(m, 2)
    pr = Transport(disc, np.array([0.8, -0.6]), nu=3.0)
    rng = np.random.default_rng(11)
    f = rng.standard_normal((m.nel, disc.nq))
    g = rng.standard_normal((m.nbface, disc.nqf))
    U, T, k, res, st = pr.iterate(f, g, 1e-13)
    Ud, Td = pr.direct_solve(f, g)
    assert st == STATUS_OK
    assert np.abs(U - Ud).max() < 1e-11 * max(1.0, np.abs(Ud).max())


def test_time_step_term_speeds_up_the_iteration():
    """The remarks: the L2 term 1/dt improves the convergence (transport: the norm with
    -div(beta)/2 + 1/dt in place of -div(beta)/2; convection-diffusion: lambda + 1/dt)."""
    n = 8
    m = BoxMesh(2, (n, n))
    disc = Discretisation(m, 2)
    rng = np.random.default_rng(5)
    f = rng.standard_normal((m.nel, disc.nq))
    g = np.zeros((m.nbface, disc.nqf))
    counts_tr, counts_cd = [], []
    for nu in (0.0, 1.0 * n, 4.0 * n):
        U, T, k, res, st = Transport(disc, np.array([1.0, 0.5]), nu=nu).iterate(f, g, 1e-10)
        assert st == STATUS_OK
        counts_tr.append(k)
        U, T, k, res, st = ConvDiff(disc, np.array([1.0, 1.0]), 1e-2, nu).iterate(f, g, 1e-10, max_iters=3000)
        assert st == STATUS_OK
        counts_cd.append(k)
    assert counts_tr[0] > counts_tr[1] > counts_tr[2], counts_tr
    assert counts_cd[0] > counts_cd[1] > counts_cd[2], counts_cd
