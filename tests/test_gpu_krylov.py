"""GPU parity of GMRES around the float64 iHDG sweep (Section 4.2, closing remark; reading R23).

The library runs GMRES(m) on the export-state fixed-point system (I - T) E = F; the oracle
runs it on the volume state (oracle/krylov.py) and also has the static-condensation direct
solve.  Both reach the same discrete HDG solution, so the bars compare solutions:
  * against the oracle's direct solve: relative L2 <= 1e-9 at a relative residual of 1e-13;
  * against the oracle's GMRES solution where the direct solve is too large: <= 1e-8 at
    1e-12 (two algebraic errors, each about cond(I - T) x the residual);
  * the returned residual is the true relative residual of the returned solution;
  * full size (the 256^2 p = 3 kappa = 1e-2 conv.-diff. mesh, on which Algorithm 1 diverges):
    the solution is within 1e-6 of the manufactured solution at every node (discretisation
    error ~1e-10 there) and is a fixed point of one float64 sweep.
"""
import numpy as np
import pytest

import workloads as W
from oracle import BoxMesh, ConvDiff, Discretisation, ShallowWater, Transport
from oracle.ihdg import STATUS_OK
from oracle.krylov import ihdg_gmres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1605_03228_gb300 import ihdg
    c = ihdg.Context(0)
    yield c
    c.close()


def ih():
    from paper_1605_03228_gb300 import ihdg
    return ihdg


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cd_case(ihdg, n, p, kappa, h):
    mesh = ihdg.make_mesh(2, n, p, hi=(n[0] * h, n[1] * h))
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1.0, 1.0), kappa=kappa)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.convdiff_forcing(vol, kappa), W.convdiff_exact(bnd)
    om = BoxMesh(2, n, hi=[n[0] * h, n[1] * h])
    disc = Discretisation(om, p)
    return mesh, co, f, g, om, disc, ConvDiff(disc, np.array([1.0, 1.0]), kappa)


def test_gmres_solves_the_diverging_regime_like_the_direct_solve(ctx):
    """kappa = 1e-2 at h = 1/256, p = 3: Algorithm 1 diverges (spectral radius > 5), GMRES
    around its sweep reaches the direct HDG solution."""
    ihdg = ih()
    mesh, co, f, g, om, disc, pr = cd_case(ihdg, (6, 6), 3, 1e-2, 1.0 / 256)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-13, max_iters=2000, krylov_restart=100))
    Ud, Td = pr.direct_solve(f, g)
    assert res.status == ihdg.OK
    assert res.residual <= 1e-12
    assert res.iterations == res.fp64_sweeps and res.lowp_sweeps == 0
    assert rel(u, Ud.reshape(om.nel, -1)) < 1e-9
    # the plain iteration diverges on the same problem
    _, _, res_plain = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-8))
    assert res_plain.status == ihdg.DIVERGED


@pytest.mark.parametrize("restart", [30, 200])
def test_gmres_matches_the_oracles_gmres_on_a_ragged_mesh(ctx, restart):
    """33 x 31 elements (1023: several blocks of every vector kernel plus a ragged tail),
    h = 1/32, kappa = 1e-2: the plain iteration diverges at this h too."""
    ihdg = ih()
    mesh, co, f, g, om, disc, pr = cd_case(ihdg, (33, 31), 3, 1e-2, 1.0 / 32)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-12, max_iters=5000, krylov_restart=restart))
    U, T, its, st, _ = ihdg_gmres(pr, f, g, tol=1e-12, restart=restart, max_iters=5000)
    assert st == STATUS_OK and res.status == ihdg.OK
    assert res.residual <= 1e-11
    assert rel(u, U.reshape(om.nel, -1)) < 1e-8


def test_gmres_restart_lengths_reach_the_same_solution(ctx):
    ihdg = ih()
    mesh, co, f, g, om, disc, pr = cd_case(ihdg, (12, 10), 2, 1e-2, 1.0 / 64)
    u5, _, r5 = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-12, max_iters=20000, krylov_restart=5))
    u300, _, r300 = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-12, max_iters=20000, krylov_restart=300))
    assert r5.status == ihdg.OK and r300.status == ihdg.OK
    assert r5.iterations >= r300.iterations
    assert rel(u5, u300) < 1e-8
    Ud, _ = pr.direct_solve(f, g)
    assert rel(u300, Ud.reshape(om.nel, -1)) < 1e-9


def test_gmres_transport3d_equals_the_plain_iteration(ctx):
    """Upwind transport: the sweep converges (nilpotent in exact arithmetic), and GMRES
    reaches the same solution in no more steps."""
    ihdg = ih()
    n, p, beta = (4, 3, 5), 2, (0.6, 0.5, -0.7)
    mesh = ihdg.make_mesh(3, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    rng = np.random.default_rng(11)
    f = rng.standard_normal(vol.shape[:2])
    g = rng.standard_normal(bnd.shape[:2])
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-14, krylov_restart=60))
    om = BoxMesh(3, n)
    disc = Discretisation(om, p)
    U, T, K, r, st = Transport(disc, np.array(beta)).iterate(f, g, 1e-14)
    assert res.status == ihdg.OK and st == STATUS_OK
    assert res.iterations <= K
    assert rel(u, U.reshape(om.nel, -1)) < 1e-10


def test_gmres_shallow_water_steps_at_a_diverging_time_step(ctx):
    """Backward-Euler shallow water at dt = 6 h / ((p+1)(p+2)) (spectral radius ~6, the
    listed 512^2 configuration's ratio): GMRES steps equal the oracle's direct steps."""
    ihdg = ih()
    n, p = (8, 8), 2
    h = 1.0 / n[0]
    dt = 6.0 * h / ((p + 1) * (p + 2))
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=dt)
    nodes = ihdg.node_points(mesh, co)
    q0 = W.swe_bump(nodes, seed=0, width=0.15)
    q = q0.reshape(q0.shape[0], -1).copy()
    its, res = ctx.swe_steps(mesh, co, q, 3, ihdg.make_options(1e-13, max_iters=3000, krylov_restart=150))
    pr = ShallowWater(Discretisation(BoxMesh(2, n), p), 1.0, dt)
    U = q0.copy()
    for _ in range(3):
        U = pr.step_direct(U)
    assert rel(q, U.reshape(q.shape[0], -1)) < 1e-9
    # Algorithm 1 alone diverges at this time step
    q2 = q0.reshape(q0.shape[0], -1).copy()
    _, r2 = ctx.swe_steps(mesh, co, q2, 1, ihdg.make_options(1e-10))
    assert r2.status == ihdg.DIVERGED


def test_gmres_edge_cases(ctx):
    ihdg = ih()
    mesh, co, f, g, om, disc, pr = cd_case(ihdg, (5, 4), 2, 1e-2, 1.0 / 64)
    # zero data: the zero solution at once
    u, _, res = ctx.solve(mesh, co, np.zeros_like(f), np.zeros_like(g), ihdg.make_options(1e-10, krylov_restart=10))
    assert res.status == ihdg.OK and res.iterations == 0 and np.abs(u).max() == 0.0
    # max_iters stops the solve
    u, _, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-14, max_iters=7, krylov_restart=4))
    assert res.status == ihdg.NOT_CONVERGED and res.iterations == 7 and res.residual > 1e-14
    # a single element
    mesh1, co1, f1, g1, om1, disc1, pr1 = cd_case(ihdg, (1, 1), 3, 1e-2, 1.0 / 256)
    u, _, res = ctx.solve(mesh1, co1, f1, g1, ihdg.make_options(1e-13, krylov_restart=50))
    Ud, _ = pr1.direct_solve(f1, g1)
    assert res.status == ihdg.OK and rel(u, Ud.reshape(1, -1)) < 1e-10
    # float64 only
    with pytest.raises(ihdg.IHDGError):
        ctx.solve(mesh, co, f, g, ihdg.make_options(1e-8, prec=ihdg.MIXED_FP32, krylov_restart=10))
    with pytest.raises(ihdg.IHDGError):
        ctx.solve(mesh, co, f, g, ihdg.make_options(1e-8, krylov_restart=5000))


def test_full_size_convdiff_as_listed_gmres(ctx):
    """The 2D conv.-diff. configuration as listed: 256^2 elements, p = 3, kappa = 1e-2,
    beta = (1,1) on the unit square, on which Algorithm 1 diverges.  Full GMRES (one cycle of
    up to 2048 steps, the basis of 2049 export vectors, 17 GB, resident in HBM) converges to
    the HDG solution."""
    ihdg = ih()
    n, p, kappa = (256, 256), 3, 1e-2
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1.0, 1.0), kappa=kappa)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.convdiff_forcing(vol, kappa), W.convdiff_exact(bnd)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-10, max_iters=2048, krylov_restart=2048))
    assert res.status == ihdg.OK, (res.status, res.iterations, res.residual)
    assert res.residual <= 2e-10
    nel = n[0] * n[1]
    nodes = ihdg.node_points(mesh, co)
    ue = W.convdiff_exact(nodes).reshape(nel, -1)
    uc = u.reshape(nel, 3, -1)[:, 2, :]
    assert np.abs(uc - ue).max() < 1e-6
    # a fixed point of the sweep: one float64 sweep from it moves u by little
    uu = np.ascontiguousarray(u)
    o = ihdg.make_options(1e-30, max_iters=1)
    o.u0 = uu.ctypes.data
    _, _, r1 = ctx.solve(mesh, co, f, g, o)
    assert r1.iterations == 1 and r1.residual < 1e-6
