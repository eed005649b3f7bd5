"""Pins for the oracle's GMRES and its use around the iHDG sweep (Section 4.2 closing remark,
reading R23).

GMRES alone, on small explicit matrices, against what its definition fixes:
* after k steps of a cycle the iterate minimises ||b - A x|| over x0 + K_k(A, r0): checked
  against a brute-force least-squares problem over the explicit Krylov basis
  [r0, A r0, ..., A^(k-1) r0] (no Arnoldi, no rotations), for every k;
* the recorded residual estimates equal the true residuals ||b - A x_k||;
* restarted GMRES(3) equals two such minimisations in sequence; GMRES(1) equals the
  closed-form minimal-residual step x += (r.Ar / Ar.Ar) r;
* finite termination: full GMRES solves an n x n system in at most n steps;
* A = I: one step.
Around the sweep: the solution equals the oracle's static-condensation direct solve, both
where the plain iteration converges (transport) and where it diverges (conv.-diff. with
kappa = 1e-2 at h = 1/256, spectral radius > 5, the Section 5.3 regime; a shallow-water
step beyond Theorem 3's time-step bound).
"""
import numpy as np
import pytest

from oracle import BoxMesh, ConvDiff, Discretisation, Transport
from oracle.ihdg import STATUS_DIVERGED, STATUS_NOT_CONVERGED, STATUS_OK
from oracle.krylov import gmres, ihdg_gmres


def random_system(n, seed, shift=1.0, scale=0.4):
    rng = np.random.default_rng(seed)
    A = shift * np.eye(n) + scale * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    return A, b


def brute_min_residual(A, b, x0, k):
    """argmin ||b - A x|| over x0 + span{r0, A r0, ..., A^(k-1) r0} by least squares."""
    r0 = b - A @ x0
    K = np.empty((b.size, k))
    v = r0.copy()
    for i in range(k):
        K[:, i] = v
        v = A @ v
    y, *_ = np.linalg.lstsq(A @ K, r0, rcond=None)
    return x0 + K @ y


@pytest.mark.parametrize("seed", [0, 1])
def test_iterates_minimise_the_residual_over_the_krylov_space(seed):
    A, b = random_system(12, seed)
    for k in range(1, 7):
        x, its, st, hist = gmres(lambda v: A @ v, b, tol=0.0, restart=12, max_iters=k)
        assert its == k and st == STATUS_NOT_CONVERGED
        xb = brute_min_residual(A, b, np.zeros_like(b), k)
        assert np.linalg.norm(x - xb) <= 1e-9 * np.linalg.norm(xb)
        # the Givens estimate is the true residual of the iterate
        assert abs(hist[k] - np.linalg.norm(b - A @ x)) <= 1e-10 * np.linalg.norm(b)
    # residuals never increase within a cycle
    _, _, _, hist = gmres(lambda v: A @ v, b, tol=0.0, restart=12, max_iters=12)
    assert np.all(np.diff(hist) <= 1e-14 * hist[0])


def test_restarted_cycles_are_successive_minimisations():
    A, b = random_system(12, 3, shift=1.5)
    x, its, _, _ = gmres(lambda v: A @ v, b, tol=0.0, restart=3, max_iters=6)
    assert its == 6
    x1 = brute_min_residual(A, b, np.zeros_like(b), 3)
    x2 = brute_min_residual(A, b, x1, 3)
    assert np.linalg.norm(x - x2) <= 1e-9 * np.linalg.norm(x2)


def test_gmres1_is_the_minimal_residual_step():
    A, b = random_system(8, 4, shift=2.0, scale=0.3)
    x, its, _, _ = gmres(lambda v: A @ v, b, tol=0.0, restart=1, max_iters=5)
    xr = np.zeros_like(b)
    for _ in range(5):
        r = b - A @ xr
        Ar = A @ r
        xr = xr + (r @ Ar) / (Ar @ Ar) * r
    assert its == 5
    assert np.linalg.norm(x - xr) <= 1e-12 * np.linalg.norm(xr)


def test_full_gmres_terminates_in_n_steps():
    A, b = random_system(10, 5, shift=0.2, scale=1.0)
    x, its, st, _ = gmres(lambda v: A @ v, b, tol=1e-12, restart=10, max_iters=50)
    assert st == STATUS_OK and its <= 10
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-9 * np.linalg.norm(np.linalg.solve(A, b))


def test_identity_takes_one_step():
    b = np.arange(1.0, 6.0)
    x, its, st, _ = gmres(lambda v: v.copy(), b, tol=1e-14, restart=5, max_iters=5)
    assert st == STATUS_OK and its == 1
    assert np.allclose(x, b, rtol=0, atol=1e-15)


def test_nonfinite_operator_reports_divergence():
    b = np.ones(4)
    _, _, st, _ = gmres(lambda v: v * np.nan, b, tol=1e-10, restart=4, max_iters=4)
    assert st == STATUS_DIVERGED


def cd(n, p, kappa, h=None, seed=0):
    m = BoxMesh(2, (n, n), hi=None if h is None else [n * h] * 2)
    disc = Discretisation(m, p)
    pr = ConvDiff(disc, np.array([1.0, 1.0]), kappa, 0.0)
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((m.nel, disc.nq))
    g = rng.standard_normal((m.nbface, disc.nqf))
    return m, disc, pr, f, g


def test_gmres_solves_the_mixed_regime_where_the_sweep_diverges():
    """kappa = 1e-2 at h = 1/256, p = 3 (the 2D conv.-diff. workload's element): Algorithm 1
    diverges, GMRES around its sweep reaches the direct solution."""
    m, disc, pr, f, g = cd(6, 3, 1e-2, h=1 / 256)
    *_, st = pr.iterate(f, g, 1e-10, max_iters=400)
    assert st == STATUS_DIVERGED
    U, T, its, st, hist = ihdg_gmres(pr, f, g, tol=1e-12, restart=60, max_iters=2000)
    Ud, Td = pr.direct_solve(f, g)
    assert st == STATUS_OK
    assert np.abs(U - Ud).max() <= 1e-7 * np.abs(Ud).max()
    assert np.abs(T - Td).max() <= 1e-7 * np.abs(Td).max()


@pytest.mark.parametrize("restart", [5, 200])
def test_gmres_transport_equals_direct_solve(restart):
    m = BoxMesh(2, (5, 4))
    disc = Discretisation(m, 2)
    pr = Transport(disc, np.array([1.0, 0.5]))
    rng = np.random.default_rng(7)
    f = rng.standard_normal((m.nel, disc.nq))
    g = rng.standard_normal((m.nbface, disc.nqf))
    U, T, its, st, _ = ihdg_gmres(pr, f, g, tol=1e-13, restart=restart, max_iters=500)
    Ud, Td = pr.direct_solve(f, g)
    assert st == STATUS_OK
    assert np.abs(U - Ud).max() <= 1e-10 * np.abs(Ud).max()
    # upwind transport sweeps are nilpotent (finite termination, Section 3): GMRES needs at
    # most as many steps as the plain iteration
    _, _, k, _, st2 = pr.iterate(f, g, 1e-13)
    assert st2 == STATUS_OK and its <= k


def test_gmres_shallow_water_step_equals_the_direct_step():
    """A backward-Euler shallow-water step at dt = 6 h / ((p+1)(p+2)), where Algorithm 1
    diverges: GMRES around the sweep (the previous state enters the affine part only) equals
    the direct step."""
    from oracle import ShallowWater
    n, p = 6, 2
    h = 1.0 / n
    disc = Discretisation(BoxMesh(2, (n, n)), p)
    pr = ShallowWater(disc, 1.0, 6.0 * h / ((p + 1) * (p + 2)), 0.3, 0.05)
    rng = np.random.default_rng(3)
    U_m = rng.standard_normal((disc.mesh.nel, 3, disc.nb))
    f0 = np.zeros((disc.mesh.nel, disc.nq))
    g0 = np.zeros((disc.mesh.nbface, disc.nqf))
    *_, st = pr.iterate(f0, g0, 1e-10, U_prev=U_m, max_iters=300)
    assert st == STATUS_DIVERGED
    U, _, its, st, _ = ihdg_gmres(pr, f0, g0, tol=1e-13, restart=100, max_iters=2000, U_prev=U_m)
    Ud = pr.step_direct(U_m)
    assert st == STATUS_OK
    assert np.abs(U - Ud).max() <= 1e-9 * np.abs(Ud).max()
