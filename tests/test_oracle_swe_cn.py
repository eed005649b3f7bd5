"""Pins for the oracle's Crank-Nicolson shallow-water step (the time rule of the paper's
linearized shallow-water experiments, Section 5; spatial operator of Section 3).

* the iHDG iterate of a step equals the direct (static condensation) solve of that step;
* for this linear autonomous system a Crank-Nicolson step equals two times a backward-Euler
  half step minus the start state (a consequence of (I - dt L/2)^-1 (I + dt L/2) = 2 (I -
  dt L/2)^-1 - I), checked against the separately pinned backward-Euler oracle;
* second order in time (error ratio ~4 per halving of dt; backward Euler ~2);
* mass conserved, energy ||phi||^2 + Phi ||vel||^2 non-increasing, and less energy lost than
  with backward Euler over the same steps (the upwind dissipation is the only loss);
* the standing wave of Eq. (shallowexact) is followed to the spatial error.
"""
import numpy as np
import pytest

from oracle import BoxMesh, Discretisation, ShallowWater, ShallowWaterCN
from oracle.ihdg import STATUS_OK


def disc_for(n, p):
    return Discretisation(BoxMesh(2, (n, n)), p)


def standing_wave(disc, t):
    N = disc.node_points()
    x, y = N[..., 0], N[..., 1]
    s2 = np.sqrt(2.0)
    U = np.zeros((disc.mesh.nel, 3, disc.nb))
    U[:, 0] = np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(s2 * np.pi * t)
    U[:, 1] = np.sin(np.pi * x) * np.cos(np.pi * y) * np.sin(s2 * np.pi * t) / s2
    U[:, 2] = np.cos(np.pi * x) * np.sin(np.pi * y) * np.sin(s2 * np.pi * t) / s2
    return U


@pytest.mark.parametrize("p,fc,gam", [(1, 0.0, 0.0), (2, 0.5, 0.1), (3, 0.0, 0.0)])
def test_cn_iteration_equals_direct_solve(p, fc, gam):
    n = 3
    disc = disc_for(n, p)
    pr = ShallowWaterCN(disc, 1.0, (1.0 / n) / ((p + 1) * (p + 2)), fc, gam)
    Um = np.random.default_rng(2).standard_normal((disc.mesh.nel, 3, disc.nb))
    U, T, k, res, st = pr.step(Um, 1e-13)
    Ud = pr.step_direct(Um)
    assert st == STATUS_OK
    assert np.abs(U - Ud).max() < 1e-10 * max(1.0, np.abs(Ud).max())


@pytest.mark.parametrize("p,Phi,fc,gam", [(1, 1.0, 0.0, 0.0), (2, 2.0, 0.7, 0.2), (4, 0.5, 0.0, 0.3)])
def test_cn_is_two_backward_euler_half_steps_minus_start(p, Phi, fc, gam):
    n, dt = 3, 0.02
    disc = disc_for(n, p)
    Um = np.random.default_rng(3).standard_normal((disc.mesh.nel, 3, disc.nb))
    cn = ShallowWaterCN(disc, Phi, dt, fc, gam).step_direct(Um)
    half = ShallowWater(disc, Phi, 0.5 * dt, fc, gam).step_direct(Um)
    assert np.abs(cn - (2.0 * half - Um)).max() < 1e-11 * np.abs(cn).max()
    # and it is not the backward-Euler step of the full size
    be = ShallowWater(disc, Phi, dt, fc, gam).step_direct(Um)
    assert np.abs(cn - be).max() > 1e-4 * np.abs(cn).max()


def _march(pr, U, nsteps):
    for _ in range(nsteps):
        U = pr.step_direct(U)
    return U


def test_cn_second_order_in_time():
    """Same spatial discretisation throughout; the reference is 128 Crank-Nicolson steps."""
    n, p, T = 3, 2, 0.2
    disc = disc_for(n, p)
    U0 = standing_wave(disc, 0.0)
    ref = _march(ShallowWaterCN(disc, 1.0, T / 128), U0, 128)
    e_cn = [np.abs(_march(ShallowWaterCN(disc, 1.0, T / k), U0, k) - ref).max() for k in (4, 8, 16)]
    e_be = [np.abs(_march(ShallowWater(disc, 1.0, T / k), U0, k) - ref).max() for k in (8, 16)]
    assert 3.5 < e_cn[0] / e_cn[1] < 4.5 and 3.5 < e_cn[1] / e_cn[2] < 4.5, e_cn
    assert 1.6 < e_be[0] / e_be[1] < 2.4, e_be
    assert e_cn[1] < 0.1 * e_be[0]


def test_cn_mass_energy():
    n, p = 6, 2
    dt = (1.0 / n) / ((p + 1) * (p + 2))
    disc = disc_for(n, p)
    N = disc.node_points()
    U = np.zeros((disc.mesh.nel, 3, disc.nb))
    U[:, 0] = np.exp(-((N[..., 0] - 0.4) ** 2 + (N[..., 1] - 0.6) ** 2) / 0.02)
    cn, be = ShallowWaterCN(disc, 1.0, dt), ShallowWater(disc, 1.0, dt)
    mass = lambda V: float(np.sum(disc.load(disc.at_volume(V[:, 0]))))
    m0, e0 = mass(U), cn.norm2(U)
    Ub = U.copy()
    e = e0
    for _ in range(6):
        U, T, k, res, st = cn.step(U, 1e-12)
        assert st == STATUS_OK
        assert abs(mass(U) - m0) < 1e-9
        e1 = cn.norm2(U)
        assert e1 <= e * (1 + 1e-12)
        e = e1
        Ub = be.step_direct(Ub)
    assert be.norm2(Ub) < e < e0


def test_cn_follows_standing_wave():
    n, p, nsteps = 4, 3, 20
    dt = (1.0 / n) / ((p + 1) * (p + 2))
    disc = disc_for(n, p)
    U = _march(ShallowWaterCN(disc, 1.0, dt), standing_wave(disc, 0.0), nsteps)
    ex = standing_wave(disc, dt * nsteps)
    rel = np.sqrt(ShallowWaterCN(disc, 1.0, dt).norm2(U - ex) / ShallowWaterCN(disc, 1.0, dt).norm2(ex))
    assert rel < 2e-3, rel


def test_iterations_per_step_match_the_papers_table():
    """The paper's table of iHDG iterations per Crank-Nicolson step at dt = h/((p+1)(p+2))
    (tests/golden/swe_cn_iterations_per_step.json).  The paper states no tolerance for it;
    with 1e-9 on ||q^k - q^(k-1)|| (the reading in the design notes) the second step of the
    standing wave reproduces the 16-element row exactly and the 64- and 256-element rows
    within one iteration, including the order p=3 < p=4 < p=1 <= p=2."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "swe_cn_iterations_per_step.json")))
    for n_el, exact in (("16", True), ("64", False), ("256", False)):
        n = int(round(np.sqrt(int(n_el))))
        counts = []
        for p in (1, 2, 3, 4):
            disc = disc_for(n, p)
            pr = ShallowWaterCN(disc, 1.0, (1.0 / n) / ((p + 1) * (p + 2)))
            U = standing_wave(disc, 0.0)
            for _ in range(2):
                U, T, k, res, st = pr.step(U, 1e-9)
                assert st == STATUS_OK
            counts.append(k)
        paper = gold["rows_n_el"][n_el]
        if exact:
            assert counts == paper, (n_el, counts, paper)
        assert max(abs(a - b) for a, b in zip(counts, paper)) <= 1, (n_el, counts, paper)
        assert counts[2] < counts[3] < counts[0] <= counts[1], counts
