"""Pins for the oracle's linearized shallow-water iHDG (Section 3, Theorem 3, Section 5.2).

* each backward-Euler step's converged iterate equals the direct HDG solve of that step;
* mass conservation (walls carry zero mass flux; interior fluxes cancel at convergence);
* the backward-Euler energy ||phi||^2 + Phi ||vel||^2 does not increase;
* optimal h-convergence p+1 against the standing-wave exact solution (shallowexact);
* a tiny step needs only a couple of iterations with warm start (Section 5.2 reports 2);
* Theorem 3's step restriction: converges at dt = h/((p+1)(p+2)), diverges at 6x that.
"""
import numpy as np
import pytest

from oracle import BoxMesh, Discretisation, ShallowWater
from oracle.ihdg import STATUS_DIVERGED, STATUS_OK


def setup(n, p, dt, Phi=1.0, fc=0.0, gam=0.0):
    m = BoxMesh(2, (n, n))
    disc = Discretisation(m, p)
    return m, disc, ShallowWater(disc, Phi, dt, fc, gam)


def standing_wave(disc, t):
    N = disc.node_points()
    x, y = N[..., 0], N[..., 1]
    s2 = np.sqrt(2.0)
    U = np.zeros((disc.mesh.nel, 3, disc.nb))
    U[:, 0] = np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(s2 * np.pi * t)
    U[:, 1] = np.sin(np.pi * x) * np.cos(np.pi * y) * np.sin(s2 * np.pi * t) / s2
    U[:, 2] = np.cos(np.pi * x) * np.sin(np.pi * y) * np.sin(s2 * np.pi * t) / s2
    return U


@pytest.mark.parametrize("p,fc,gam", [(1, 0.0, 0.0), (2, 0.5, 0.1)])
def test_step_equals_direct_solve(p, fc, gam):
    n = 3
    m, disc, pr = setup(n, p, dt=0.25 * (1.0 / n) / ((p + 1) * (p + 2)), fc=fc, gam=gam)
    rng = np.random.default_rng(1)
    Um = rng.standard_normal((m.nel, 3, disc.nb))
    U, T, k, res, st = pr.step(Um, 1e-13)
    Ud, Td = pr.direct_solve(None, None, U_prev=Um)
    assert st == STATUS_OK
    assert np.abs(U - Ud).max() < 1e-10 * max(1.0, np.abs(Ud).max())


def test_mass_conserved_and_energy_decays():
    n, p = 6, 2
    m, disc, pr = setup(n, p, dt=(1.0 / n) / ((p + 1) * (p + 2)))
    N = disc.node_points()
    U = np.zeros((m.nel, 3, disc.nb))
    U[:, 0] = np.exp(-((N[..., 0] - 0.4) ** 2 + (N[..., 1] - 0.6) ** 2) / 0.02)
    mass = lambda U: float(np.sum(disc.load(disc.at_volume(U[:, 0]))))
    energy = lambda U: pr.norm2(U)
    m0, e0 = mass(U), energy(U)
    for _ in range(5):
        U, T, k, res, st = pr.step(U, 1e-12)
        assert st == STATUS_OK
        assert abs(mass(U) - m0) < 1e-9
        e1 = energy(U)
        assert e1 <= e0 * (1 + 1e-12)
        e0 = e1


@pytest.mark.parametrize("p", [1, 2])
def test_standing_wave_rate(p):
    """Small steps so the backward-Euler time error stays below the spatial error."""
    errs = []
    dt, nsteps = 1e-5, 4
    for n in (4, 8):
        m, disc, pr = setup(n, p, dt)
        U = standing_wave(disc, 0.0)
        for _ in range(nsteps):
            U, T, k, res, st = pr.step(U, 1e-13)
            assert st == STATUS_OK
        ex = standing_wave(disc, dt * nsteps)
        X = disc.volume_points()
        wJ = disc.ref.wq * disc.jac
        # phi error against the exact field evaluated at Gauss points
        phie = np.cos(np.pi * X[..., 0]) * np.cos(np.pi * X[..., 1]) * np.cos(np.sqrt(2) * np.pi * dt * nsteps)
        err = disc.at_volume(U[:, 0]) - phie
        errs.append(np.sqrt(np.sum(err ** 2 * wJ[None, :])))
    rate = np.log2(errs[0] / errs[1])
    assert rate > p + 0.7, (errs, rate)


def test_tiny_step_needs_few_iterations():
    n, p = 4, 2
    m, disc, pr = setup(n, p, dt=1e-6)
    U = standing_wave(disc, 0.0)
    for _ in range(3):
        U, T, k, res, st = pr.step(U, 1e-10)
        assert st == STATUS_OK and k <= 3


def test_step_restriction_theorem3():
    n, p = 8, 2
    h = 1.0 / n
    rng = np.random.default_rng(0)
    for ratio, converges in ((1.0, True), (6.144, False)):
        m, disc, pr = setup(n, p, dt=ratio * h / ((p + 1) * (p + 2)))
        U = rng.standard_normal((m.nel, 3, disc.nb))
        Z = np.zeros_like(U)
        r = []
        for _ in range(120):
            U = pr.sweep(U, None, None, U_prev=Z)
            nn = np.sqrt(pr.norm2(U))
            U /= nn
            r.append(nn)
        rho = np.exp(np.mean(np.log(r[-40:])))
        assert (rho < 1.0) == converges, (ratio, rho)
