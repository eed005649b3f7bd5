"""GPU parity: libihdg's CUDA path against the float64 oracle, through the C ABI.

Bars (written here, derived in the design notes):
  * float64 path: the same iteration count K as the oracle (an integer decided by float64
    residuals on both sides; a residual within 1e-9 relative of tol may land one sweep
    apart), and relative L2 difference of u^K <= 1e-10;
  * mixed path (float32 / bf16 inner sweeps, float64 refinement): relative L2 difference
    <= 1e-6 from the oracle's float64 solution at the same tolerance;
  * divergence is an integer outcome too: the same status at the same sweep.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import BoxMesh, ConvDiff, Discretisation, ShallowWater, ShallowWaterCN, Transport
from oracle.ihdg import STATUS_DIVERGED, STATUS_OK

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


def oracle_trace_at_nodes(disc, T):
    """Oracle traces are at face Gauss points; the library reports face GLL nodes.  The
    Gauss-weighted least-squares fit onto the face polynomials (the oracle's own tables) is
    exact for polynomial traces and is the face L2 projection for boundary data."""
    from oracle.refelem import lagrange_matrix
    ref = disc.ref
    B1 = lagrange_matrix(ref.nodes1, ref.xq1)
    B = B1 if disc.d == 2 else np.kron(B1, B1)
    w = ref.face_w
    coef = np.linalg.solve(B.T @ (w[:, None] * B), B.T @ (w[:, None] * T.T))
    return coef.T


def check_iteration_count(K_gpu, K_or, hist_or, tol):
    if K_gpu == K_or:
        return
    assert abs(K_gpu - K_or) == 1, (K_gpu, K_or)
    k = min(K_gpu, K_or)
    assert abs(hist_or[k - 1] - tol) < 1e-9 * tol, "counts differ away from the tolerance boundary"


# ------------------------------------------------------------------------------ transport
@pytest.mark.parametrize("n,p,beta", [((8, 8), 2, (1.0, 0.5)), ((7, 5), 3, (-0.6, 1.0)),
                                      ((6, 9), 1, (0.8, -0.3)), ((5, 6), 4, (-1.0, -0.4))])
def test_transport2d_fp64(ctx, n, p, beta):
    ihdg = ih()
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f = W.transport2d_forcing(vol, beta)
    g = W.transport2d_exact(bnd)
    tol = 1e-10
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(tol))
    om = BoxMesh(2, n)
    disc = Discretisation(om, p)
    U, T, K, r, st, hist = Transport(disc, np.array(beta)).iterate(f, g, tol, history=True)
    assert res.status == ihdg.OK and st == STATUS_OK
    check_iteration_count(res.iterations, K, hist, tol)
    assert rel(u, U.reshape(om.nel, -1)) < 1e-10
    assert rel(tr, oracle_trace_at_nodes(disc, T)) < 1e-10


@pytest.mark.parametrize("n,p,beta", [((4, 3, 5), 2, (1.0, 1.0, 1.0)), ((3, 4, 3), 1, (0.5, -0.8, 0.3)),
                                      ((3, 3, 3), 2, (-0.3, 0.6, -0.9))])
def test_transport3d_fp64(ctx, n, p, beta):
    ihdg = ih()
    b = np.array(beta) / np.linalg.norm(beta)
    mesh = ihdg.make_mesh(3, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=tuple(b))
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f = W.transport3d_forcing(vol, tuple(b))
    g = W.transport3d_exact(bnd)
    tol = 1e-10
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(tol))
    om = BoxMesh(3, n)
    disc = Discretisation(om, p)
    U, T, K, r, st, hist = Transport(disc, b).iterate(f, g, tol, history=True)
    check_iteration_count(res.iterations, K, hist, tol)
    assert rel(u, U.reshape(om.nel, -1)) < 1e-10
    assert rel(tr, oracle_trace_at_nodes(disc, T)) < 1e-10


@pytest.mark.parametrize("d,n,p,beta", [(2, (8, 8), 2, (1.0, 0.5)), (2, (9, 6), 3, (-0.6, 1.0)),
                                        (2, (5, 7), 4, (0.8, -0.3)), (3, (4, 3, 5), 2, (1.0, 1.0, 1.0)),
                                        (3, (3, 4, 3), 1, (0.5, -0.8, 0.3))])
def test_transport_npc_fp64(ctx, d, n, p, beta):
    """NPC flux (Eq. Ntaub) on the float64 path: the oracle's iteration count, which is the
    number of element layers along the flow plus one (finite termination), and its solution."""
    ihdg = ih()
    b = np.array(beta) / np.linalg.norm(beta)
    mesh = ihdg.make_mesh(d, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=tuple(b), flux=ihdg.FLUX_NPC)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    if d == 2:
        f, g = W.transport2d_forcing(vol, tuple(b)), W.transport2d_exact(bnd)
    else:
        f, g = W.transport3d_forcing(vol, tuple(b)), W.transport3d_exact(bnd)
    tol = 1e-10
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(tol))
    om = BoxMesh(d, n)
    disc = Discretisation(om, p)
    U, T, K, r, st, hist = Transport(disc, b, flux="npc").iterate(f, g, tol, history=True)
    assert res.status == ihdg.OK and st == STATUS_OK
    check_iteration_count(res.iterations, K, hist, tol)
    assert K == sum(x - 1 for x in n) + 2
    assert rel(u, U.reshape(om.nel, -1)) < 1e-10
    assert rel(tr, oracle_trace_at_nodes(disc, T)) < 1e-10


@pytest.mark.parametrize("d,p,beta,prec_name", [(2, 2, (1.0, 0.5), "FP64"), (2, 3, (-0.3, 1.0), "FP64"),
                                                (3, 2, (0.6, -0.4, 0.7), "FP64"), (2, 3, (1.0, 0.5), "MIXED_FP32")])
def test_time_dependent_transport_step(ctx, d, p, beta, prec_name):
    """A backward-Euler step of time-dependent transport through ihdg_solve (the remark after
    Theorem 1): reaction nu = 1/dt, forcing u^m/dt at the quadrature points, warm start u^m.
    From a polynomial u^m the exact step Q = P - dt DP + dt^2 D^2 P (D = beta.grad) is in the
    element space, so the GPU reproduces it to the float64 (or mixed) bar; and on random
    data it matches the oracle's step and iteration count."""
    ihdg = ih()
    dt, n = 0.05, (5, 4, 3)[:d]
    mesh = ihdg.make_mesh(d, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta, nu=1.0 / dt)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    nodes = ihdg.node_points(mesh, co)
    b = np.asarray(beta, dtype=float)

    def P(X):
        v = X[..., 0] ** 2 + 2 * X[..., 0] * X[..., 1] - X[..., 1]
        return v + X[..., 0] * X[..., 2] if d == 3 else v

    def DP(X):
        v = b[0] * (2 * X[..., 0] + 2 * X[..., 1]) + b[1] * (2 * X[..., 0] - 1)
        return v + b[0] * X[..., 2] + b[2] * X[..., 0] if d == 3 else v

    d2 = 2 * b[0] ** 2 + 4 * b[0] * b[1] + (2 * b[0] * b[2] if d == 3 else 0.0)
    Q = lambda X: P(X) - dt * DP(X) + dt * dt * d2
    u0 = np.ascontiguousarray(P(nodes))
    o = ihdg.make_options(1e-12, prec=getattr(ihdg, prec_name), max_iters=4000)
    o.u0 = u0.ctypes.data
    u, tr, res = ctx.solve(mesh, co, P(vol) / dt, Q(bnd), o)
    assert res.status == ihdg.OK, res.as_dict()
    bar = 1e-10 if prec_name == "FP64" else 1e-6
    assert rel(u, Q(nodes)) < bar
    # random data against the oracle's step
    rng = np.random.default_rng(13)
    f = rng.standard_normal(vol.shape[:2])
    g = rng.standard_normal(bnd.shape[:2])
    u0r = np.ascontiguousarray(rng.standard_normal(u.shape))
    o.u0 = u0r.ctypes.data
    o.tol = 1e-10
    u2, _, res2 = ctx.solve(mesh, co, f, g, o)
    om = BoxMesh(d, n)
    disc = Discretisation(om, p)
    U, T, K, r, st = Transport(disc, b, nu=1.0 / dt).iterate(f, g, 1e-10, U0=u0r.reshape(om.nel, 1, -1))
    assert res2.status == ihdg.OK and st == STATUS_OK
    if prec_name == "FP64":
        assert abs(res2.iterations - K) <= 1
    assert rel(u2, U.reshape(om.nel, -1)) < (1e-9 if prec_name == "FP64" else 1e-6)


def test_time_dependent_convdiff_steps_converge_faster(ctx):
    """The remark on time-dependent convection-diffusion (Section 4.1): the L2 term 1/dt
    (reaction nu + 1/dt) makes the iteration converge in fewer sweeps; GPU counts equal the
    oracle's."""
    ihdg = ih()
    n, p = (8, 8), 2
    mesh = ihdg.make_mesh(2, n, p)
    om = BoxMesh(2, n)
    disc = Discretisation(om, p)
    rng = np.random.default_rng(5)
    counts = []
    for nu in (0.0, 8.0, 32.0):
        co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1.0, 1.0), kappa=1e-2, nu=nu)
        vol, bnd = ihdg.quadrature_points(mesh, co)
        f = rng.standard_normal(vol.shape[:2])
        g = np.zeros(bnd.shape[:2])
        u, _, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-10, max_iters=3000))
        U, T, K, r, st = ConvDiff(disc, np.array([1.0, 1.0]), 1e-2, nu).iterate(f, g, 1e-10, max_iters=3000)
        assert res.status == ihdg.OK and st == STATUS_OK
        assert abs(res.iterations - K) <= 1
        assert rel(u, U.reshape(om.nel, -1)) < 1e-8
        counts.append(res.iterations)
    assert counts[0] > counts[1] > counts[2], counts


@pytest.mark.parametrize("prec_name", ["MIXED_FP32", "MIXED_BF16"])
def test_transport_npc_mixed(ctx, prec_name):
    """NPC flux through the mixed-precision path (outer float64, inner low precision)."""
    ihdg = ih()
    n, p, beta = (20, 17), 2, (1.0, 0.5)
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta, flux=ihdg.FLUX_NPC)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.transport2d_forcing(vol, beta), W.transport2d_exact(bnd)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-10, prec=getattr(ihdg, prec_name)))
    om = BoxMesh(2, n)
    U, T, K, r, st = Transport(Discretisation(om, p), np.array(beta), flux="npc").iterate(f, g, 1e-10)
    assert res.status == ihdg.OK, res.as_dict()
    assert rel(u, U.reshape(om.nel, -1)) < 1e-6


def test_transport_beta_axis_aligned(ctx):
    """beta . n = 0 on the y faces: zero-weight faces, trace reported as {{u}}."""
    ihdg = ih()
    n, p, beta = (5, 4), 2, (1.0, 0.0)
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.transport2d_forcing(vol, beta), W.transport2d_exact(bnd)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-11))
    om = BoxMesh(2, n)
    disc = Discretisation(om, p)
    U, T, K, r, st = Transport(disc, np.array(beta)).iterate(f, g, 1e-11)
    assert res.iterations == K
    assert rel(u, U.reshape(om.nel, -1)) < 1e-10
    assert rel(tr, oracle_trace_at_nodes(disc, T)) < 1e-10


# ------------------------------------------------------------------------------ conv.-diff.
@pytest.mark.parametrize("n,p,kappa,beta,nu", [((6, 7), 3, 1e-4, (1.0, 1.0), 0.0),
                                                ((5, 4), 2, 1e-3, (-1.0, 0.5), 1.0),
                                                ((4, 4), 4, 1e-5, (0.3, -1.0), 0.0)])
def test_convdiff2d_fp64(ctx, n, p, kappa, beta, nu):
    ihdg = ih()
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=beta, kappa=kappa, nu=nu)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f = W.convdiff_forcing(vol, kappa, beta, nu)
    g = W.convdiff_exact(bnd)
    tol = 1e-10
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(tol, max_iters=3000))
    om = BoxMesh(2, n)
    disc = Discretisation(om, p)
    U, T, K, r, st, hist = ConvDiff(disc, np.array(beta), kappa, nu).iterate(f, g, tol, max_iters=3000, history=True)
    assert st == STATUS_OK and res.status == ihdg.OK
    check_iteration_count(res.iterations, K, hist, tol)
    assert rel(u, U.reshape(om.nel, -1)) < 1e-10
    assert rel(tr, oracle_trace_at_nodes(disc, T)) < 1e-10


@pytest.mark.parametrize("d,n,p,beta,kappa,nu,gamma", [(3, (3, 4, 3), 2, (0.0, 0.0, 0.0), 1.0, 1.0, 1.0),
                                                        (2, (6, 5), 2, (0.3, -0.2), 0.5, 1.0, 1.0),
                                                        (2, (9, 7), 1, (0.0, 0.0), 1.0, 10.0, 1.0)])
def test_convdiff_mesh_tau_fp64(ctx, d, n, p, beta, kappa, nu, gamma):
    """Mesh-dependent stabilisation tau = gamma (p+1)(p+2)/h (Section 4.2) on the float64
    path: the oracle's iteration count and solution, in the diffusion-dominated regime where
    the upwind tau diverges."""
    ihdg = ih()
    mesh = ihdg.make_mesh(d, n, p)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=beta, kappa=kappa, nu=nu, tau_gamma=gamma)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    if d == 2 and any(beta):
        f, g = W.convdiff_forcing(vol, kappa, beta, nu), W.convdiff_exact(bnd)
    else:
        u = lambda P: np.prod(np.sin(np.pi * P[..., :d]), axis=-1)
        f, g = (d * np.pi ** 2 * kappa + nu) * u(vol), u(bnd)
    tol = 1e-10
    u_g, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(tol, max_iters=5000))
    om = BoxMesh(d, n)
    disc = Discretisation(om, p)
    U, T, K, r, st, hist = ConvDiff(disc, np.array(beta[:d]), kappa, nu, tau_gamma=gamma).iterate(
        f, g, tol, max_iters=5000, history=True)
    assert res.status == ihdg.OK and st == STATUS_OK
    check_iteration_count(res.iterations, K, hist, tol)
    assert rel(u_g, U.reshape(om.nel, -1)) < 1e-10
    assert rel(tr, oracle_trace_at_nodes(disc, T)) < 1e-10


def test_convdiff_diverges_like_oracle(ctx):
    """kappa = 1e-2 at h = 1/256 (the 2D convection-diffusion workload's element size): the
    iteration diverges; both sides stop with DIVERGED at the same sweep, same iterate."""
    ihdg = ih()
    n, p, h = (6, 6), 3, 1.0 / 256
    mesh = ihdg.make_mesh(2, n, p, hi=(n[0] * h, n[1] * h))
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1.0, 1.0), kappa=1e-2)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.convdiff_forcing(vol, 1e-2), W.convdiff_exact(bnd)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-8))
    om = BoxMesh(2, n, hi=[n[0] * h, n[1] * h])
    disc = Discretisation(om, p)
    U, T, K, r, st = ConvDiff(disc, np.array([1.0, 1.0]), 1e-2).iterate(f, g, 1e-8)
    assert st == STATUS_DIVERGED and res.status == ihdg.DIVERGED
    assert res.iterations == K
    assert rel(u, U.reshape(om.nel, -1)) < 1e-9


def test_convdiff3d_fp64(ctx):
    ihdg = ih()
    n, p, kappa, beta = (3, 4, 3), 2, 1e-4, (0.6, 0.5, -0.7)
    mesh = ihdg.make_mesh(3, n, p)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=beta, kappa=kappa, nu=0.5)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    rng = np.random.default_rng(5)
    f = rng.standard_normal(vol.shape[:2])
    g = rng.standard_normal(bnd.shape[:2])
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-10, max_iters=3000))
    om = BoxMesh(3, n)
    disc = Discretisation(om, p)
    U, T, K, r, st, hist = ConvDiff(disc, np.array(beta), kappa, 0.5).iterate(f, g, 1e-10, max_iters=3000, history=True)
    check_iteration_count(res.iterations, K, hist, 1e-10)
    assert rel(u, U.reshape(om.nel, -1)) < 1e-10


# ------------------------------------------------------------------------------ edge cases
def test_single_element_and_zero_data(ctx):
    ihdg = ih()
    mesh = ihdg.make_mesh(2, (1, 1), 2)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1.0, 0.5))
    vol, bnd = ihdg.quadrature_points(mesh, co)
    u, tr, res = ctx.solve(mesh, co, np.zeros(vol.shape[:2]), np.zeros(bnd.shape[:2]), ihdg.make_options(1e-10))
    assert res.status == ihdg.OK and res.iterations == 1 and np.abs(u).max() == 0.0
    f, g = W.transport2d_forcing(vol), W.transport2d_exact(bnd)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-12))
    om = BoxMesh(2, (1, 1))
    disc = Discretisation(om, 2)
    U, T, K, r, st = Transport(disc, np.array([1.0, 0.5])).iterate(f, g, 1e-12)
    assert res.iterations == K and rel(u, U.reshape(1, -1)) < 1e-12


def test_max_iters_and_initial_guess(ctx):
    ihdg = ih()
    n, p = (9, 4), 2
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1.0, 0.5))
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.transport2d_forcing(vol), W.transport2d_exact(bnd)
    om = BoxMesh(2, n)
    disc = Discretisation(om, p)
    pr = Transport(disc, np.array([1.0, 0.5]))
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-14, max_iters=7))
    U, T, K, r, st = pr.iterate(f, g, 1e-14, max_iters=7)
    assert res.status == ihdg.NOT_CONVERGED and res.iterations == 7 == K
    assert rel(u, U.reshape(om.nel, -1)) < 1e-12
    u0 = np.random.default_rng(2).standard_normal((om.nel, disc.nb))
    o = ihdg.make_options(1e-10)
    o.u0 = u0.ctypes.data
    u, tr, res = ctx.solve(mesh, co, f, g, o)
    U, T, K, r, st = pr.iterate(f, g, 1e-10, U0=u0.reshape(om.nel, 1, -1))
    assert res.iterations == K and rel(u, U.reshape(om.nel, -1)) < 1e-10


# ------------------------------------------------------------------------------ shallow water
@pytest.mark.parametrize("n,p,ratio,fc,gam", [((8, 8), 2, 0.5, 0.0, 0.0), ((6, 7), 3, 1.0, 0.4, 0.05)])
def test_swe_steps_fp64(ctx, n, p, ratio, fc, gam):
    ihdg = ih()
    h = 1.0 / n[0]
    dt = ratio * h / ((p + 1) * (p + 2))
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=dt, coriolis_f=fc, friction=gam)
    nodes = ihdg.node_points(mesh, co)
    q0 = W.swe_bump(nodes, seed=0, width=0.15)
    q = q0.reshape(q0.shape[0], -1).copy()
    its, res = ctx.swe_steps(mesh, co, q, 3, ihdg.make_options(1e-10))
    om = BoxMesh(2, n)
    disc = Discretisation(om, p)
    pr = ShallowWater(disc, 1.0, dt, fc, gam)
    U = q0.copy()
    for s in range(3):
        U, T, K, r, st = pr.step(U, 1e-10)
        assert its[s] == K
    assert rel(q, U.reshape(om.nel, -1)) < 1e-10


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED_FP32"])
def test_swe_restart_from_state_is_exact(ctx, prec_name):
    """Checkpoint/resume: the volume state q^m is the whole restart state of the time
    stepping (each step warm-starts from R q^m), so 10 steps equal 5 steps followed by 5 more
    from the returned state, bit for bit, with the same per-step iteration counts."""
    ihdg = ih()
    n, p = (20, 16), 2
    dt = 0.5 * (1.0 / n[0]) / ((p + 1) * (p + 2))
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=dt, coriolis_f=0.2, friction=0.05)
    nodes = ihdg.node_points(mesh, co)
    q0 = W.swe_bump(nodes, seed=3, width=0.15)
    opts = ihdg.make_options(1e-10, prec=getattr(ihdg, prec_name))
    q_all = q0.reshape(q0.shape[0], -1).copy()
    its_all, r_all = ctx.swe_steps(mesh, co, q_all, 10, opts)
    q_half = q0.reshape(q0.shape[0], -1).copy()
    its_a, _ = ctx.swe_steps(mesh, co, q_half, 5, opts)
    checkpoint = q_half.copy()                         # what a caller would save
    q_res = checkpoint.copy()
    its_b, r_b = ctx.swe_steps(mesh, co, q_res, 5, opts)
    assert r_all.status == r_b.status == ihdg.OK
    assert its_a + its_b == its_all
    assert np.array_equal(q_res, q_all)


@pytest.mark.parametrize("prec_name,n", [("MIXED_FP32", (20, 16)), ("MIXED_BF16", (20, 16)),
                                         ("MIXED_FP32", (64, 48))])
def test_swe_steps_mixed(ctx, prec_name, n):
    """Mixed precision on the shallow-water path (float32 or bf16 inner sweeps, float64 outer
    sweeps and stopping norm) against the float64 oracle, step by step: each backward-Euler
    step of Eq. localSolverDD (Section 3) at dt = h/((p+1)(p+2)), the step the paper runs in
    Section 5.2, warm-started from the previous step's state on both sides.  Bar: relative
    L2 difference of the volume state <= 1e-6 after every step."""
    ihdg = ih()
    p = 2
    h = 1.0 / n[0]
    dt = h / ((p + 1) * (p + 2))
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=dt, coriolis_f=0.3, friction=0.02)
    nodes = ihdg.node_points(mesh, co)
    q0 = W.swe_bump(nodes, seed=1, width=0.15)
    q = q0.reshape(q0.shape[0], -1).copy()
    om = BoxMesh(2, n)
    disc = Discretisation(om, p)
    pr = ShallowWater(disc, 1.0, dt, 0.3, 0.02)
    U = q0.copy()
    opts = ihdg.make_options(1e-10, prec=getattr(ihdg, prec_name), max_iters=20000)
    for step in range(4):
        its, res = ctx.swe_steps(mesh, co, q, 1, opts)
        U, T, K, r, st = pr.step(U, 1e-10)
        assert res.status == ihdg.OK and st == STATUS_OK, (step, res.as_dict())
        assert res.lowp_sweeps > 0 or res.iterations <= 2
        e = rel(q, U.reshape(om.nel, -1))
        assert e < 1e-6, (step, e)


@pytest.mark.parametrize("prec_name,n,p,fc,gam", [("FP64", (6, 5), 2, 0.0, 0.0), ("FP64", (9, 7), 3, 0.4, 0.1),
                                                  ("MIXED_FP32", (20, 16), 2, 0.3, 0.02)])
def test_swe_crank_nicolson_steps(ctx, prec_name, n, p, fc, gam):
    """Crank-Nicolson steps (the time rule of the paper's shallow-water experiments) against
    the oracle's Crank-Nicolson step written from its definition (trapezoidal average of the
    HDG spatial residuals), step by step from the same state: the library's half-step form
    runs the same iterates, so the float64 iteration counts agree (to one sweep where a
    residual lands on the tolerance) and the states to 1e-9; mixed precision to 1e-6."""
    ihdg = ih()
    dt = (1.0 / n[0]) / ((p + 1) * (p + 2))
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=dt, coriolis_f=fc, friction=gam, time_scheme=ihdg.CRANK_NICOLSON)
    nodes = ihdg.node_points(mesh, co)
    q0 = W.swe_bump(nodes, seed=4, width=0.15)
    q = q0.reshape(q0.shape[0], -1).copy()
    om = BoxMesh(2, n)
    pr = ShallowWaterCN(Discretisation(om, p), 1.0, dt, fc, gam)
    U = q0.copy()
    opts = ihdg.make_options(1e-10, prec=getattr(ihdg, prec_name), max_iters=20000)
    miss = 0
    for step in range(3):
        its, res = ctx.swe_steps(mesh, co, q, 1, opts)
        U, T, K, r, st = pr.step(U, 1e-10)
        assert res.status == ihdg.OK and st == STATUS_OK, (step, res.as_dict())
        e = rel(q, U.reshape(om.nel, -1))
        if prec_name == "FP64":
            assert abs(int(its[0]) - K) <= 1, (step, its, K)
            miss += int(its[0]) != K
            assert e < 1e-9, (step, e)
        else:
            assert e < 1e-6, (step, e)
    assert miss <= 1


def test_swe_crank_nicolson_iterations_match_the_papers_table(ctx):
    """The paper's table of iHDG iterations per Crank-Nicolson step at dt = h/((p+1)(p+2))
    for the standing wave (tests/golden/swe_cn_iterations_per_step.json), on the GPU for all
    four mesh rows, at the tolerance reading 1e-9: the second step's count equal to the
    paper's on 16 elements, within one iteration on 64 and 256, within two on 1024 (measured:
    9, 10, 7, 8 against 7, 10, 7, 7), and equal to the oracle's (to one sweep where a residual
    lands on the tolerance) where the oracle is cheap."""
    import json
    import os
    ihdg = ih()
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "swe_cn_iterations_per_step.json")))
    got = {}
    for n_el, paper in gold["rows_n_el"].items():
        n = int(round(np.sqrt(int(n_el))))
        row = []
        for p in (1, 2, 3, 4):
            dt = (1.0 / n) / ((p + 1) * (p + 2))
            mesh = ihdg.make_mesh(2, (n, n), p)
            co = ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=dt, time_scheme=ihdg.CRANK_NICOLSON)
            q = W.swe_standing_wave(ihdg.node_points(mesh, co), 0.0)
            q = q.reshape(q.shape[0], -1).copy()
            its, res = ctx.swe_steps(mesh, co, q, 2, ihdg.make_options(1e-9))
            assert res.status == ihdg.OK
            row.append(int(its[1]))
            if n <= 8:
                om = BoxMesh(2, (n, n))
                disc = Discretisation(om, p)
                pr = ShallowWaterCN(disc, 1.0, dt)
                U = W.swe_standing_wave(ihdg.node_points(mesh, co), 0.0)
                for _ in range(2):
                    U, T, K, r, st = pr.step(U, 1e-9)
                assert abs(row[-1] - K) <= 1, (n_el, p, row[-1], K)
        got[n_el] = row
    assert got["16"] == gold["rows_n_el"]["16"], got
    for n_el, paper in gold["rows_n_el"].items():
        bar = 2 if n_el == "1024" else 1
        assert max(abs(a - b) for a, b in zip(got[n_el], paper)) <= bar, (got, gold["rows_n_el"])


# ------------------------------------------------------------------------------ mixed precision
@pytest.mark.parametrize("prec_name", ["MIXED_FP32", "MIXED_BF16"])
def test_mixed_transport2d(ctx, prec_name):
    ihdg = ih()
    n, p, beta = (24, 24), 2, (1.0, 0.5)
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.transport2d_forcing(vol), W.transport2d_exact(bnd)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-10, prec=getattr(ihdg, prec_name)))
    om = BoxMesh(2, n)
    disc = Discretisation(om, p)
    U, T, K, r, st = Transport(disc, np.array(beta)).iterate(f, g, 1e-10)
    assert res.status == ihdg.OK, res.as_dict()
    assert res.fp64_sweeps >= 2 and res.lowp_sweeps > 0
    assert rel(u, U.reshape(om.nel, -1)) < 1e-6
    assert rel(tr, oracle_trace_at_nodes(disc, T)) < 1e-6


@pytest.mark.parametrize("prec_name", ["MIXED_FP32", "MIXED_BF16"])
def test_mixed_transport3d(ctx, prec_name):
    ihdg = ih()
    n, p = (6, 6, 6), 2
    b = tuple(np.ones(3) / np.sqrt(3))
    mesh = ihdg.make_mesh(3, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=b)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.transport3d_forcing(vol, b), W.transport3d_exact(bnd)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-8, prec=getattr(ihdg, prec_name)))
    om = BoxMesh(3, n)
    disc = Discretisation(om, p)
    U, T, K, r, st = Transport(disc, np.array(b)).iterate(f, g, 1e-8)
    assert res.status == ihdg.OK, res.as_dict()
    assert rel(u, U.reshape(om.nel, -1)) < 1e-6


@pytest.mark.parametrize("kernel,grid,lpe", [("tile", "2", "1"), ("tile", "", "1"), ("global", "2", "1"),
                                             ("global", "", "1"), ("tile", "", "4")])
def test_mixed_inner_kernel_variants(ctx, monkeypatch, kernel, grid, lpe):
    """The inner loop's kernel variants (register-resident 4-lanes-per-element state, the
    default on 2D meshes; block-resident tile state; global state) and grid
    sizes far smaller than the element count (every thread loops over several elements)
    reach the same solution as the default launch.  The inner stopping test sums per-block
    partials, so the inner sweep count may differ by a sweep: compare at 1e-9."""
    ihdg = ih()
    n, p, beta = (40, 30), 2, (0.8, 1.0)
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.transport2d_forcing(vol, beta), W.transport2d_exact(bnd)
    opts = ihdg.make_options(1e-11, prec=ihdg.MIXED_FP32)
    u_a, _, ra = ctx.solve(mesh, co, f, g, opts)
    if grid:
        monkeypatch.setenv("IHDG_PERSISTENT_GRID", grid)
    monkeypatch.setenv("IHDG_INNER_KERNEL", kernel)
    monkeypatch.setenv("IHDG_TILE_LPE", lpe)
    if lpe == "4":
        monkeypatch.setenv("IHDG_REG_NT", "512")      # the register kernel's two-blocks-per-SM shape
    u_b, _, rb = ctx.solve(mesh, co, f, g, opts)
    assert ra.status == rb.status == ihdg.OK
    assert rel(u_b, u_a) < 1e-9
    # the result names the kernel that ran: global state, or a tile kernel (temporally
    # blocked, register-resident or shared-memory tile)
    used = rb.inner_kernel_used
    assert (used == 5) if kernel == "global" else (used in (2, 3, 4)), used


TC_CASES = [("t3d_p1", "", "tc", "MIXED_BF16"), ("t3d_p2", "", "tc", "MIXED_BF16"), ("cd2d_p3", "", "tc", "MIXED_BF16"),
            ("t2d_p2", "1", "tc", "MIXED_BF16"), ("t3d_p1", "", "tile", "MIXED_BF16"), ("cd2d_p3", "", "tile", "MIXED_BF16"),
            ("t3d_p1", "", "tc", "MIXED_FP32"), ("t3d_p2", "", "tc", "MIXED_FP32"), ("cd2d_p3", "", "tc", "MIXED_FP32"),
            ("t2d_p2", "1", "tc", "MIXED_FP32"), ("t3d_p2", "", "tc", "MIXED_TF32"), ("cd2d_p3", "", "tc", "MIXED_TF32"),
            ("cd2d_p3", "", "global", "MIXED_FP32"), ("cd2d_p3", "3", "global", "MIXED_BF16"),
            ("t3d_p2", "", "global", "MIXED_FP32"), ("t3d_p1", "2", "global", "MIXED_BF16"),
            ("t2d_p2", "", "global", "MIXED_FP32")]


@pytest.mark.parametrize("case,grid,kernel,prec_name", TC_CASES)
def test_mixed_tensor_core_inner(ctx, monkeypatch, case, grid, kernel, prec_name):
    """Inner sweeps with the local apply on the tensor cores (kernel "tc": tcgen05 MMA over
    tiles of 128 elements with a float32 accumulator in tensor memory) reach the oracle's
    float64 solution at the mixed bar, for every operand mode: bf16 (kind::f16), float32 as
    four tf32 passes on hi/lo splits, and one tf32 pass; and so do bf16 sweeps on the CUDA
    cores (kernel "tile") and the global-state kernel (kernel "global": per-face and per-axis
    export layouts, 2D and 3D, float32 and bf16 state, grids of 2 and 3 blocks looping over
    the elements).  The meshes leave a ragged last tile
    (element counts not multiples of 128) and some of a block's four tile groups without a
    tile; a grid of one block makes its groups loop over several tiles per sweep."""
    ihdg = ih()
    if case.startswith("t3d"):
        n, p = ((9, 7, 11), 1) if case == "t3d_p1" else ((6, 5, 7), 2)
        beta = tuple(np.ones(3) / np.sqrt(3))
        mesh = ihdg.make_mesh(3, n, p)
        co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta)
        vol, bnd = ihdg.quadrature_points(mesh, co)
        f, g = W.transport3d_forcing(vol, beta), W.transport3d_exact(bnd)
        pr = Transport(Discretisation(BoxMesh(3, n), p), np.array(beta))
    elif case == "cd2d_p3":
        n, p, kappa = (13, 11), 3, 1e-4
        mesh = ihdg.make_mesh(2, n, p)
        co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1.0, 1.0), kappa=kappa)
        vol, bnd = ihdg.quadrature_points(mesh, co)
        f, g = W.convdiff_forcing(vol, kappa), W.convdiff_exact(bnd)
        pr = ConvDiff(Discretisation(BoxMesh(2, n), p), np.array([1.0, 1.0]), kappa)
    else:
        n, p, beta = (29, 23), 2, (0.8, 1.0)
        mesh = ihdg.make_mesh(2, n, p)
        co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta)
        vol, bnd = ihdg.quadrature_points(mesh, co)
        f, g = W.transport2d_forcing(vol, beta), W.transport2d_exact(bnd)
        pr = Transport(Discretisation(BoxMesh(2, n), p), np.array(beta))
    tol = 1e-9
    U, T, K, r, st = pr.iterate(f, g, tol, max_iters=20000)
    assert st == STATUS_OK
    monkeypatch.setenv("IHDG_INNER_KERNEL", kernel)
    if grid:
        monkeypatch.setenv("IHDG_PERSISTENT_GRID", grid)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(tol, prec=getattr(ihdg, prec_name), max_iters=20000))
    assert res.status == ihdg.OK, res.as_dict()
    assert res.lowp_sweeps > 0
    if kernel == "tc":
        # transport in bf16 takes the staged-gather variant unless it is switched off
        staged = prec_name == "MIXED_BF16" and not case.startswith("cd") and os.environ.get("IHDG_TC_STAGED") != "0"
        assert res.inner_kernel_used == (6 if staged else 1), res.inner_kernel_used
    if kernel == "global":
        assert res.inner_kernel_used == 5
    if kernel == "tile":
        assert res.inner_kernel_used in (2, 3, 4)
    assert rel(u, U.reshape(pr.mesh.nel, -1)) < 1e-6



@pytest.mark.parametrize("n,p", [((9, 7, 11), 1), ((6, 5, 7), 2), ((16, 12, 10), 2)])
def test_tc_staged_gathers_equal_register_gathers(ctx, monkeypatch, n, p):
    """The tensor-core kernel with TMA-staged gathers (bf16 transport) computes exactly what
    the register-gather kernel computes: the same packed operands, tile assignment and
    reductions, so the solutions and sweep counts are bitwise equal; the meshes put windows
    into the guard bands (first and last layers) and leave a ragged last tile."""
    ihdg = ih()
    beta = tuple(np.array([1.0, -0.7, 0.5]) / np.linalg.norm([1.0, -0.7, 0.5]))
    mesh = ihdg.make_mesh(3, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.transport3d_forcing(vol, beta), W.transport3d_exact(bnd)
    opts = ihdg.make_options(1e-9, prec=ihdg.MIXED_BF16, max_iters=20000, inner_kernel=ihdg.KERNEL_TENSOR_CORES)
    u_s, t_s, r_s = ctx.solve(mesh, co, f, g, opts)
    monkeypatch.setenv("IHDG_TC_STAGED", "0")
    u_r, t_r, r_r = ctx.solve(mesh, co, f, g, opts)
    assert r_s.status == r_r.status == ihdg.OK
    assert r_s.inner_kernel_used == 6 and r_r.inner_kernel_used == 1
    assert r_s.iterations == r_r.iterations and r_s.lowp_sweeps == r_r.lowp_sweeps
    assert np.array_equal(u_s, u_r) and np.array_equal(t_s, t_r)


def _blocked_case(ihdg, pde):
    if pde == "convdiff":
        mesh = ihdg.make_mesh(2, (37, 29), 3)
        co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1.0, 0.7), kappa=1e-3)
        vol, bnd = ihdg.quadrature_points(mesh, co)
        return mesh, co, W.convdiff_forcing(vol, 1e-3, (1.0, 0.7)), W.convdiff_exact(bnd)
    if pde == "transport":
        mesh = ihdg.make_mesh(2, (41, 23), 2)
        co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(0.8, -0.6))
        vol, bnd = ihdg.quadrature_points(mesh, co)
        return mesh, co, W.transport2d_forcing(vol, (0.8, -0.6)), W.transport2d_exact(bnd)
    mesh = ihdg.make_mesh(2, (33, 27), 2)
    co = ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=0.5 / 33 / 12, coriolis_f=0.2, friction=0.01)
    return mesh, co, None, None


def _blocked_run(ctx, ihdg, pde, case, opts):
    mesh, co, f, g = case
    if pde == "swe":
        nodes = ihdg.node_points(mesh, co)
        q = W.swe_bump(nodes, seed=2, width=0.15)
        q = q.reshape(q.shape[0], -1).copy()
        its, res = ctx.swe_steps(mesh, co, q, 1, opts)
        return q, res
    u, tr, res = ctx.solve(mesh, co, f, g, opts)
    return u, res


@pytest.mark.parametrize("pde", ["convdiff", "transport", "swe"])
@pytest.mark.parametrize("H,grid", [(2, ""), (3, "6"), (4, "11")])
def test_blocked_inner_matches_one_barrier_per_sweep(ctx, monkeypatch, pde, H, grid):
    """Temporal blocking (H inner sweeps per grid barrier, halo recomputed in shared memory)
    must produce the iterates of the one-barrier-per-sweep kernel.  The float64 outer sweeps
    of the mixed path would repair a wrong inner correction, so the comparison fixes the
    schedule (tol 0, 7 inner sweeps per outer step, a sweep budget that ends right after the
    outer sweep that applies the second inner correction) and compares the results directly:
    float32 rounding of a different summation order differs by ~1e-6 relative, a stale or
    misplaced halo value by the size of the correction.  Grid caps give many small ragged
    tiles; the three PDEs cover the per-face layout with Dirichlet data (conv.-diff.), the
    per-axis layout (transport) and mirrored wall traces (shallow water)."""
    ihdg = ih()
    if grid:
        monkeypatch.setenv("IHDG_PERSISTENT_GRID", grid)
    case = _blocked_case(ihdg, pde)
    out = {}
    for sps in (1, H):
        opts = ihdg.make_options(0.0, prec=ihdg.MIXED_FP32, max_iters=19, inner_max=7, inner_rtol=1e-30,
                                 diverge_factor=-1.0, inner_kernel=ihdg.KERNEL_CUDA_CORES, sweeps_per_sync=sps)
        out[sps] = _blocked_run(ctx, ihdg, pde, case, opts)
    (u1, r1), (uh, rh) = out[1], out[H]
    assert r1.status == rh.status == ihdg.NOT_CONVERGED
    assert (r1.iterations, r1.fp64_sweeps, r1.lowp_sweeps) == (rh.iterations, rh.fp64_sweeps, rh.lowp_sweeps)
    assert rel(uh, u1) < 2e-5, rel(uh, u1)


@pytest.mark.parametrize("pde", ["convdiff", "transport"])
def test_blocked_tile_shapes_compute_the_same_iterates(ctx, pde):
    """The blocked kernel's tile shape (opts.tile_shape: 1 the smallest tile + halo area, 2
    and 3 the next ones, which the autotuner times) only changes which block computes an
    element: with a fixed schedule every shape gives bitwise the same result."""
    ihdg = ih()
    case = _blocked_case(ihdg, pde)
    out = []
    for shape in (1, 2, 3):
        opts = ihdg.make_options(0.0, prec=ihdg.MIXED_FP32, max_iters=19, inner_max=7, inner_rtol=1e-30,
                                 diverge_factor=-1.0, inner_kernel=ihdg.KERNEL_CUDA_CORES, sweeps_per_sync=4,
                                 tile_shape=shape)
        u, r = _blocked_run(ctx, ihdg, pde, case, opts)
        assert r.inner_kernel_used == 2
        out.append((u, r))
    for u, r in out[1:]:
        assert (r.iterations, r.lowp_sweeps) == (out[0][1].iterations, out[0][1].lowp_sweeps)
        assert np.array_equal(u, out[0][0])


@pytest.mark.parametrize("H", [2, 3, 4])
def test_blocked_inner_converges_to_oracle(ctx, H):
    """The blocked inner kernel in a complete mixed solve: the oracle's solution within the
    mixed bar (1e-6), and no more float64 outer steps than the one-barrier-per-sweep kernel
    needs plus one (a wrong inner solve would show as extra outer steps)."""
    ihdg = ih()
    n, p, kappa = (46, 38), 3, 1e-4
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1.0, 1.0), kappa=kappa)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.convdiff_forcing(vol, kappa), W.convdiff_exact(bnd)
    base = dict(prec=ihdg.MIXED_FP32, max_iters=20000, inner_kernel=ihdg.KERNEL_CUDA_CORES)
    u1, _, r1 = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-8, sweeps_per_sync=1, **base))
    uh, _, rh = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-8, sweeps_per_sync=H, **base))
    assert r1.status == rh.status == ihdg.OK, rh.as_dict()
    assert rh.fp64_sweeps <= r1.fp64_sweeps + 1, (rh.fp64_sweeps, r1.fp64_sweeps)
    om = BoxMesh(2, n)
    U = ConvDiff(Discretisation(om, p), np.array([1.0, 1.0]), kappa).iterate(f, g, 1e-8, max_iters=20000)[0]
    assert rel(uh, U.reshape(om.nel, -1)) < 1e-6

def test_mixed_convdiff(ctx):
    ihdg = ih()
    n, p, kappa = (12, 10), 3, 1e-4
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1.0, 1.0), kappa=kappa)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.convdiff_forcing(vol, kappa), W.convdiff_exact(bnd)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(1e-8, prec=ihdg.MIXED_FP32))
    om = BoxMesh(2, n)
    disc = Discretisation(om, p)
    U, T, K, r, st = ConvDiff(disc, np.array([1.0, 1.0]), kappa).iterate(f, g, 1e-8)
    assert res.status == ihdg.OK, res.as_dict()
    assert rel(u, U.reshape(om.nel, -1)) < 1e-6


# ------------------------------------------------------------------------------ device API
def test_device_api_matches_host_api(ctx):
    ihdg = ih()
    n, p, beta = (16, 12), 3, (0.7, 1.0)
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.transport2d_forcing(vol, beta), W.transport2d_exact(bnd)
    opts = ihdg.make_options(1e-10)
    u_h, tr_h, res_h = ctx.solve(mesh, co, f, g, opts)
    s = ihdg.problem_sizes(mesh, co)
    dev = torch.device("cuda:0")
    df = torch.from_numpy(np.ascontiguousarray(f)).to(dev)
    dg = torch.from_numpy(np.ascontiguousarray(g)).to(dev)
    du = torch.empty((s.n_el, s.nvol), dtype=torch.float64, device=dev)
    dt = torch.empty((s.n_face, s.nface_nodes), dtype=torch.float64, device=dev)
    nws = ihdg.workspace_bytes(mesh, co, opts)
    ws = torch.empty(nws + 256, dtype=torch.uint8, device=dev)
    base = (ws.data_ptr() + 255) // 256 * 256
    stream = torch.cuda.current_stream().cuda_stream
    res = ctx.solve_device(mesh, co, df.data_ptr(), dg.data_ptr(), opts, du.data_ptr(), dt.data_ptr(), base, nws, stream)
    assert res.iterations == res_h.iterations
    assert np.array_equal(du.cpu().numpy(), u_h) and np.array_equal(dt.cpu().numpy(), tr_h)


# ------------------------------------------------------------------------------ full size, sampled
def patch_oracle_sweeps(kind, nfull, p, h, k, centers, coeff, f_fun, g_fun):
    """u^k at sampled elements by the oracle on a patch that holds every element within k
    of the sample (after k sweeps nothing farther away can reach it)."""
    out = []
    d = len(nfull)
    for c in centers:
        lo_i = [max(0, c[a] - k - 1) for a in range(d)]
        hi_i = [min(nfull[a], c[a] + k + 2) for a in range(d)]
        nn = [hi_i[a] - lo_i[a] for a in range(d)]
        om = BoxMesh(d, nn, lo=[lo_i[a] * h for a in range(d)], hi=[hi_i[a] * h for a in range(d)])
        disc = Discretisation(om, p)
        pr = coeff(disc)
        f = f_fun(disc.volume_points())
        g = g_fun(disc.boundary_points())
        U, T, K, r, st = pr.iterate(f, g, 0.0, max_iters=k, diverge_factor=np.inf)
        loc = sum((c[a] - lo_i[a]) * int(np.prod(nn[:a])) for a in range(d))
        out.append(U[loc].ravel())
    return np.array(out)


def test_full_size_convdiff_sampled(ctx):
    """The 2D convection-diffusion workload at full size (256^2, p = 3), k float64 sweeps,
    sampled elements against the oracle on dependency patches."""
    ihdg = ih()
    n, p, kappa, k = (256, 256), 3, 1e-2, 4
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1.0, 1.0), kappa=kappa)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.convdiff_forcing(vol, kappa), W.convdiff_exact(bnd)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(0.0, max_iters=k, diverge_factor=-1.0))
    assert res.iterations == k
    rng = np.random.default_rng(0)
    centers = [(0, 0), (255, 255), (0, 200), (128, 3)] + [tuple(rng.integers(0, 256, 2)) for _ in range(4)]
    ref = patch_oracle_sweeps("cd", n, p, 1 / 256, k, centers,
                              lambda disc: ConvDiff(disc, np.array([1.0, 1.0]), kappa),
                              lambda X: W.convdiff_forcing(X, kappa), W.convdiff_exact)
    got = np.array([u[c[0] + 256 * c[1]] for c in centers])
    assert rel(got, ref) < 1e-10


def test_full_size_transport3d_sampled(ctx):
    """The 3D transport workload at full size (64^3, p = 2), k float64 sweeps, sampled."""
    ihdg = ih()
    n, p, k = (64, 64, 64), 2, 3
    b = tuple(np.ones(3) / np.sqrt(3))
    mesh = ihdg.make_mesh(3, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=b)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.transport3d_forcing(vol, b), W.transport3d_exact(bnd)
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(0.0, max_iters=k, diverge_factor=-1.0))
    centers = [(0, 0, 0), (63, 63, 63), (5, 40, 63), (31, 2, 17)]
    ref = patch_oracle_sweeps("tr", n, p, 1 / 64, k, centers, lambda disc: Transport(disc, np.array(b)),
                              lambda X: W.transport3d_forcing(X, b), W.transport3d_exact)
    got = np.array([u[c[0] + 64 * (c[1] + 64 * c[2])] for c in centers])
    assert rel(got, ref) < 1e-10


def test_full_size_convdiff_mixed_converged(ctx):
    """The headline solve itself: 2D convection-diffusion at 256^2, p = 3, kappa = 1e-4,
    mixed float32 inner sweeps with float64 outer sweeps, in the launch shape of the bench
    (the temporally blocked kernel: one 1024-thread block per SM, 152 tiles in its grid
    barrier), run to tolerance 1e-8 and compared with the float64 oracle's converged
    solution at 48 sampled elements (corners, edges, centre, seeded interior).  The oracle's
    values are stored in tests/golden/convdiff2d_256_p3.json, written by the committed script
    beside it from oracle/ alone.  Bar: the mixed path's 1e-6 relative L2 difference."""
    import json
    import os
    ihdg = ih()
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "convdiff2d_256_p3.json")))
    n, p, kappa, beta = tuple(gold["n"]), gold["p"], gold["kappa"], tuple(gold["beta"])
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=beta, kappa=kappa)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.convdiff_forcing(vol, kappa, beta), W.convdiff_exact(bnd)
    for kernel in ("KERNEL_AUTO", "KERNEL_TENSOR_CORES"):
        opts = ihdg.make_options(gold["tol"], prec=ihdg.MIXED_FP32, max_iters=4000,
                                 inner_kernel=getattr(ihdg, kernel))
        u, tr, res = ctx.solve(mesh, co, f, g, opts)
        assert res.status == ihdg.OK, res.as_dict()
        got = u[np.array(gold["elements"])]
        ref = np.array(gold["u"])
        assert rel(got, ref) < 1e-6, (kernel, rel(got, ref))
    # the float64 path stops at the oracle's sweep count on the same problem
    u64, _, r64 = ctx.solve(mesh, co, f, g, ihdg.make_options(gold["tol"], max_iters=4000))
    assert abs(r64.iterations - gold["iterations"]) <= 1
    assert rel(u64[np.array(gold["elements"])], np.array(gold["u"])) < 1e-10


def test_full_size_transport3d_mixed_converged(ctx):
    """The 3D transport workload itself: 64^3, p = 2, mixed bf16 inner sweeps on the tensor
    cores (TMA-staged gathers, the default for bf16 transport) with float64 outer sweeps, in
    the bench's launch shape, run to tolerance 1e-8 and compared with the float64 oracle's
    converged solution at 48 sampled elements (corners, face and edge centres, centre, seeded
    interior), stored in tests/golden/transport3d_64_p2.json by the committed script beside
    it from oracle/ alone.  The float64 path stops at the oracle's sweep count (to one) and
    matches it to 1e-10 at the samples, so it stands for the oracle's whole field: the mixed
    solution is within the mixed bar (1e-6 relative L2) of it over every node.  At the samples
    alone (which favour corners and edges, the outflow corner last to settle) the two
    converged solutions differ by more: each meets the stopping test ||u^k - u^(k-1)||_L2 <
    1e-8 at a different iterate, and near the outflow corner that leaves ~1e-6 per node, which
    the L2(Omega) norm weighs by the element volume h^3; the bar there is 1e-5."""
    import json
    import os
    ihdg = ih()
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "transport3d_64_p2.json")))
    n, p, beta = tuple(gold["n"]), gold["p"], tuple(gold["beta"])
    mesh = ihdg.make_mesh(3, n, p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.transport3d_forcing(vol, beta), W.transport3d_exact(bnd)
    els, ref = np.array(gold["elements"]), np.array(gold["u"])
    u, tr, res = ctx.solve(mesh, co, f, g, ihdg.make_options(gold["tol"], prec=ihdg.MIXED_BF16, max_iters=4000))
    assert res.status == ihdg.OK, res.as_dict()
    assert res.inner_kernel_used == 6
    u64, _, r64 = ctx.solve(mesh, co, f, g, ihdg.make_options(gold["tol"], max_iters=4000))
    assert abs(r64.iterations - gold["iterations"]) <= 1
    assert rel(u64[els], ref) < 1e-10
    assert rel(u, u64) < 1e-6, rel(u, u64)
    assert rel(u[els], ref) < 1e-5, rel(u[els], ref)


def test_full_size_swe_mixed_steps(ctx):
    """The shallow-water workload itself: 512^2, p = 2, dt = h/12, two backward-Euler steps
    from the seeded bump, mixed float32 inner sweeps with float64 outer sweeps in the bench's
    launch shape, against the float64 oracle's state after two steps at 48 sampled elements
    (tests/golden/swe_512_p2.json, written by the committed script beside it from oracle/
    alone).  The float64 path matches the samples to 1e-10 with the oracle's per-step counts
    (to one); the mixed state is within 1e-5 of them.  Both paths stop on ||q^k - q^(k-1)|| <
    1e-8 at different iterates of a slowly contracting first step (374 sweeps), which leaves
    them ~1e-6 apart; run to 1e-10 the mixed state is within the mixed bar (1e-6 relative L2)
    of the float64 state over every node, which is the precision claim."""
    import json
    import os
    ihdg = ih()
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "swe_512_p2.json")))
    n, p = tuple(gold["n"]), gold["p"]
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.SWE, Phi=gold["Phi"], dt=gold["dt"])
    q0 = W.swe_bump(ihdg.node_points(mesh, co), seed=gold["bump_seed"])
    q0 = q0.reshape(q0.shape[0], -1)
    els, ref = np.array(gold["elements"]), np.array(gold["q"])
    q64 = q0.copy()
    its64, r64 = ctx.swe_steps(mesh, co, q64, gold["steps"], ihdg.make_options(gold["tol"], max_iters=4000))
    assert r64.status == ihdg.OK
    assert all(abs(int(a) - b) <= 1 for a, b in zip(its64, gold["iterations_per_step"])), (list(its64), gold)
    assert rel(q64[els], ref) < 1e-10
    qm = q0.copy()
    itsm, rm = ctx.swe_steps(mesh, co, qm, gold["steps"], ihdg.make_options(gold["tol"], prec=ihdg.MIXED_FP32,
                                                                               max_iters=4000))
    assert rm.status == ihdg.OK and rm.lowp_sweeps > 0
    assert rel(qm[els], ref) < 1e-5, rel(qm[els], ref)
    tight = []
    for prec in (ihdg.FP64, ihdg.MIXED_FP32):
        q = q0.copy()
        _, r = ctx.swe_steps(mesh, co, q, gold["steps"], ihdg.make_options(1e-10, prec=prec, max_iters=40000))
        assert r.status == ihdg.OK, (prec, r.as_dict())
        tight.append(q)
    assert rel(tight[1], tight[0]) < 1e-6, rel(tight[1], tight[0])


# ------------------------------------------------------------------------------ autotuner
def test_autotune_choice_converges_and_is_cached(ctx):
    """ihdg_autotune times complete solves over the inner-kernel choices and a ladder of inner
    stopping ratios and returns the fastest.  Its options reach the oracle's solution at the
    mixed bar, and a later solve with automatic options on the same context uses the cached
    choice (bitwise the same result as passing the tuned options).  FP64 has nothing to tune."""
    ihdg = ih()
    n, p, kappa = (40, 36), 3, 1e-4
    mesh = ihdg.make_mesh(2, n, p)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1.0, 1.0), kappa=kappa)
    vol, bnd = ihdg.quadrature_points(mesh, co)
    f, g = W.convdiff_forcing(vol, kappa), W.convdiff_exact(bnd)
    opts = ihdg.make_options(1e-8, prec=ihdg.MIXED_FP32, max_iters=20000)
    tuned, best_ms = ctx.autotune(mesh, co, f, g, opts)
    assert tuned.inner_kernel in (ihdg.KERNEL_TENSOR_CORES, ihdg.KERNEL_CUDA_CORES)
    assert tuned.inner_rtol > 0 and best_ms > 0
    assert 1 <= tuned.tile_shape <= 3 and 1 <= tuned.sweeps_per_sync <= 4
    assert tuned.prec == ihdg.MIXED_FP32 and tuned.tol == opts.tol
    u_t, _, r_t = ctx.solve(mesh, co, f, g, tuned)
    u_a, _, r_a = ctx.solve(mesh, co, f, g, opts)
    assert r_t.status == r_a.status == ihdg.OK
    assert r_a.iterations == r_t.iterations and np.array_equal(u_a, u_t)
    om = BoxMesh(2, n)
    U, T, K, r, st = ConvDiff(Discretisation(om, p), np.array([1.0, 1.0]), kappa).iterate(f, g, 1e-8, max_iters=20000)
    assert rel(u_t, U.reshape(om.nel, -1)) < 1e-6
    t64, ms64 = ctx.autotune(mesh, co, f, g, ihdg.make_options(1e-8))
    assert t64.prec == ihdg.FP64 and t64.inner_kernel == ihdg.KERNEL_AUTO and ms64 == 0.0


# ------------------------------------------------------------------------------ grouped float64 solves
def _group_problems(ihdg, seed=3, n=14):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        if i % 5 == 4:
            d, p = 3, int(rng.integers(1, 3))
            side = int(rng.integers(3, 7))
            beta = tuple(np.array([1.0, 0.6, 0.8]) / np.linalg.norm([1.0, 0.6, 0.8]))
            mesh = ihdg.make_mesh(3, (side, side + 1, side), p)
            co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta)
            vol, bnd = ihdg.quadrature_points(mesh, co)
            f, g = W.transport3d_forcing(vol, beta), W.transport3d_exact(bnd)
        elif i % 2:
            p = int(rng.integers(1, 5))
            side = int(rng.integers(8, 40))
            kappa = float(10 ** rng.uniform(-3, -1))
            mesh = ihdg.make_mesh(2, (side, side + 3), p)
            co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1.0, 0.7), kappa=kappa)
            vol, bnd = ihdg.quadrature_points(mesh, co)
            f, g = W.convdiff_forcing(vol, kappa, (1.0, 0.7)), W.convdiff_exact(bnd)
        else:
            p = int(rng.integers(1, 5))
            side = int(rng.integers(6, 48))
            mesh = ihdg.make_mesh(2, (side, side + 2), p)
            co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(0.8, 0.6))
            vol, bnd = ihdg.quadrature_points(mesh, co)
            f, g = W.transport2d_forcing(vol, (0.8, 0.6)), W.transport2d_exact(bnd)
        out.append((mesh, co, f, g))
    return out


def test_group_fp64_equals_alone(ctx):
    """ihdg_solve_group_device: problems of different meshes, orders and PDEs (2D/3D
    transport, conv.-diff. at several diffusivities) in one call give bitwise the results,
    iteration counts and statuses of solving each alone with ihdg_solve_device."""
    ihdg = ih()
    probs = _group_problems(ihdg)
    dev = torch.device("cuda:0")
    opts = ihdg.make_options(1e-10, max_iters=3000)
    sizes = [ihdg.problem_sizes(m, c) for m, c, _, _ in probs]
    fs = [torch.from_numpy(np.ascontiguousarray(f)).to(dev) for _, _, f, _ in probs]
    gs = [torch.from_numpy(np.ascontiguousarray(g)).to(dev) for _, _, _, g in probs]
    ug = [torch.zeros((s.n_el, s.nvol), dtype=torch.float64, device=dev) for s in sizes]
    tg = [torch.zeros((s.n_face, s.nface_nodes), dtype=torch.float64, device=dev) for s in sizes]
    meshes, coeffs = [p[0] for p in probs], [p[1] for p in probs]
    nws = ctx.group_workspace_bytes(meshes, coeffs, opts)
    ws = torch.empty(nws + 256, dtype=torch.uint8, device=dev)
    wsp = (ws.data_ptr() + 255) // 256 * 256
    rg = ctx.solve_group_device(meshes, coeffs, [x.data_ptr() for x in fs], [x.data_ptr() for x in gs], opts,
                                [x.data_ptr() for x in ug], [x.data_ptr() for x in tg], wsp, nws)
    torch.cuda.synchronize()
    statuses = set()
    for i, (mesh, co, f, g) in enumerate(probs):
        s = sizes[i]
        nw = ihdg.workspace_bytes(mesh, co, opts)
        w1 = torch.empty(nw + 256, dtype=torch.uint8, device=dev)
        u1 = torch.zeros((s.n_el, s.nvol), dtype=torch.float64, device=dev)
        t1 = torch.zeros((s.n_face, s.nface_nodes), dtype=torch.float64, device=dev)
        r1 = ctx.solve_device(mesh, co, fs[i].data_ptr(), gs[i].data_ptr(), opts, u1.data_ptr(), t1.data_ptr(),
                              (w1.data_ptr() + 255) // 256 * 256, nw, 0)
        torch.cuda.synchronize()
        assert (rg[i].status, rg[i].iterations) == (r1.status, r1.iterations), (i, rg[i].as_dict(), r1.as_dict())
        assert torch.equal(ug[i], u1) and torch.equal(tg[i], t1), i
        statuses.add(r1.status)
    assert ihdg.OK in statuses


def test_group_rejects_mixed_and_small_workspace(ctx):
    ihdg = ih()
    probs = _group_problems(ihdg, seed=4, n=2)
    meshes, coeffs = [p[0] for p in probs], [p[1] for p in probs]
    dev = torch.device("cuda:0")
    opts = ihdg.make_options(1e-10)
    nws = ctx.group_workspace_bytes(meshes, coeffs, opts)
    ws = torch.empty(nws + 256, dtype=torch.uint8, device=dev)
    wsp = (ws.data_ptr() + 255) // 256 * 256
    dummy = [ws.data_ptr()] * 2
    with pytest.raises(ihdg.IHDGError) as e1:
        ctx.solve_group_device(meshes, coeffs, dummy, dummy, ihdg.make_options(1e-10, prec=ihdg.MIXED_FP32),
                               dummy, None, wsp, nws)
    assert e1.value.status == ihdg.ERR_UNSUPPORTED
    with pytest.raises(ihdg.IHDGError) as e2:
        ctx.solve_group_device(meshes, coeffs, dummy, dummy, opts, dummy, None, wsp, nws - 256)
    assert e2.value.status == ihdg.ERR_NOMEM
