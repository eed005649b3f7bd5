"""GPU parity of transport with a velocity field that varies in space (per-element local solves
and the warp-per-element batched GEMV), through the C ABI, against the float64 oracle
(TransportVar).

Bars (as for the constant-coefficient path): float64 -- the oracle's iteration count K (a
residual within 1e-9 relative of tol may land one sweep apart) and relative L2 difference of
u^K and of the trace <= 1e-10; mixed float32 / bf16 -- relative L2 difference <= 1e-6 from the
oracle's solution at the same tolerance.
"""
import numpy as np
import pytest

import workloads as W
from oracle import BoxMesh, Discretisation, TransportVar

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


FIELDS = {
    "e1": W.e1_beta,
    "e2": W.e2_beta,
    "swirl": lambda X: np.stack([1.2 + np.cos(2 * X[..., 1]), 0.8 + np.sin(3 * X[..., 0])], axis=-1),
    "neg": lambda X: np.stack([-(1.0 + 0.3 * np.sin(X[..., 1])), -0.5 - 0.2 * X[..., 0]], axis=-1),
    "zero_y": lambda X: np.stack([1.0 + 0.5 * X[..., 1], 0.0 * X[..., 0]], axis=-1),
}


def case(field, d, n, p):
    ihdg = ih()
    hi = (2.0, 2.0, 2.0) if field == "e1" else (1.0, 1.0, 1.0)
    mesh = ihdg.make_mesh(d, n, p, hi=hi)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1.0, 0.0, 0.0))
    vol, bnd = ihdg.quadrature_points(mesh, co)
    fpts = ihdg.face_quadrature_points(mesh)
    beta = FIELDS[field]
    if field == "e1":
        f, g = np.zeros(vol.shape[:2]), W.e1_inflow(bnd)
    elif d == 3:
        f, g = W.e2_forcing(vol), W.e2_exact(bnd)
    else:
        f, g = W.transport2d_forcing(vol), W.transport2d_exact(bnd)
    om = BoxMesh(d, n, lo=[0.0] * d, hi=list(hi[:d]))
    disc = Discretisation(om, p)
    return mesh, beta(vol), beta(fpts), f, g, TransportVar(disc, beta), disc


def oracle_trace_at_nodes(disc, T):
    from oracle.refelem import lagrange_matrix
    ref = disc.ref
    B1 = lagrange_matrix(ref.nodes1, ref.xq1)
    B = B1 if disc.d == 2 else np.kron(B1, B1)
    w = ref.face_w
    return np.linalg.solve(B.T @ (w[:, None] * B), B.T @ (w[:, None] * T.T)).T


@pytest.mark.parametrize("field,d,n,p", [("e1", 2, (8, 8), 3), ("swirl", 2, (7, 5), 2), ("neg", 2, (6, 7), 4),
                                         ("zero_y", 2, (5, 4), 1), ("e2", 3, (4, 3, 5), 2), ("e2", 3, (3, 3, 3), 1)])
def test_var_fp64_matches_oracle(ctx, field, d, n, p):
    ihdg = ih()
    mesh, bv, bf, f, g, pr, disc = case(field, d, n, p)
    plan = ctx.var_plan(mesh, bv, bf)
    try:
        u, tr, res = plan.solve(f, g, ihdg.make_options(1e-10, max_iters=5000))
    finally:
        plan.close()
    U, T, K, r, st, hist = pr.iterate(f, g, 1e-10, max_iters=5000, history=True)
    assert res.status == ihdg.OK and st == 0, res.as_dict()
    if res.iterations != K:
        assert abs(res.iterations - K) == 1 and abs(hist[min(K, res.iterations) - 1] - 1e-10) < 1e-19
    assert rel(u, U[:, 0, :]) < 1e-10
    assert rel(tr, oracle_trace_at_nodes(disc, T)) < 1e-10


@pytest.mark.parametrize("n,p", [(8, 3), (16, 4)])
def test_var_table1_counts_on_gpu(ctx, n, p):
    """The 2D experiment of Section 5.1 on the GPU float64 path: the upwind iteration counts of
    Table 1 (91 for 64 elements at p = 3, 129 for 256 elements at p = 4)."""
    ihdg = ih()
    mesh, bv, bf, f, g, pr, disc = case("e1", 2, (n, n), p)
    plan = ctx.var_plan(mesh, bv, bf)
    try:
        u, tr, res = plan.solve(f, g, ihdg.make_options(1e-10, max_iters=5000), want_trace=False)
    finally:
        plan.close()
    assert res.status == ihdg.OK
    assert abs(res.iterations - {(8, 3): 91, (16, 4): 129}[(n, p)]) <= 1


@pytest.mark.parametrize("prec_name", ["MIXED_FP32", "MIXED_BF16"])
@pytest.mark.parametrize("field,d,n,p", [("e1", 2, (16, 16), 3), ("e2", 3, (6, 6, 6), 2), ("swirl", 2, (13, 9), 2)])
def test_var_mixed_matches_oracle(ctx, prec_name, field, d, n, p):
    ihdg = ih()
    mesh, bv, bf, f, g, pr, disc = case(field, d, n, p)
    plan = ctx.var_plan(mesh, bv, bf)
    try:
        u, tr, res = plan.solve(f, g, ihdg.make_options(1e-10, max_iters=20000, prec=getattr(ihdg, prec_name)))
    finally:
        plan.close()
    U, T, K, r, st = pr.iterate(f, g, 1e-10, max_iters=5000)
    assert res.status == ihdg.OK, res.as_dict()
    assert res.fp64_sweeps >= 1 and res.lowp_sweeps > 0
    assert rel(u, U[:, 0, :]) < 1e-6
    assert rel(tr, oracle_trace_at_nodes(disc, T)) < 1e-6


def test_var_device_api_matches_host_api(ctx):
    ihdg = ih()
    mesh, bv, bf, f, g, pr, disc = case("swirl", 2, (9, 7), 3)
    plan = ctx.var_plan(mesh, bv, bf)
    try:
        opts = ihdg.make_options(1e-10, prec=ihdg.MIXED_FP32, max_iters=5000)
        u_h, tr_h, res_h = plan.solve(f, g, opts)
        dev = torch.device("cuda:0")
        df = torch.from_numpy(np.ascontiguousarray(f)).to(dev)
        dg = torch.from_numpy(np.ascontiguousarray(g)).to(dev)
        du = torch.empty(u_h.shape, dtype=torch.float64, device=dev)
        dt = torch.empty(tr_h.shape, dtype=torch.float64, device=dev)
        res = plan.solve_device(df.data_ptr(), dg.data_ptr(), opts, du.data_ptr(), dt.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
        assert res.iterations == res_h.iterations
        assert np.array_equal(du.cpu().numpy(), u_h) and np.array_equal(dt.cpu().numpy(), tr_h)
        nbytes, setup_ms = plan.info()
        assert nbytes > 0 and setup_ms > 0
    finally:
        plan.close()


def test_var_budget_and_initial_guess(ctx):
    """max_iters stops the float64 iteration with NOT_CONVERGED at exactly u^k of the oracle;
    started from the oracle's converged solution the iteration stops after one sweep."""
    ihdg = ih()
    mesh, bv, bf, f, g, pr, disc = case("e1", 2, (6, 6), 2)
    plan = ctx.var_plan(mesh, bv, bf)
    try:
        u5, _, r5 = plan.solve(f, g, ihdg.make_options(1e-10, max_iters=5), want_trace=False)
        U5 = pr.iterate(f, g, 0.0, max_iters=5, diverge_factor=np.inf)[0]
        assert r5.status == ihdg.NOT_CONVERGED and r5.iterations == 5
        assert rel(u5, U5[:, 0, :]) < 1e-12
        Uc = pr.iterate(f, g, 1e-13, max_iters=5000)[0][:, 0, :]
        u1, _, r1 = plan.solve(f, g, ihdg.make_options(1e-10, u0=np.ascontiguousarray(Uc).ctypes.data),
                               want_trace=False)
        assert r1.status == ihdg.OK and r1.iterations == 1
        assert rel(u1, Uc) < 1e-11
    finally:
        plan.close()


def test_var_rejects_sign_change_inside_faces(ctx):
    ihdg = ih()
    mesh = ihdg.make_mesh(2, (4, 4), 2)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1.0, 0.0, 0.0))
    vol, _ = ihdg.quadrature_points(mesh, co)
    fpts = ihdg.face_quadrature_points(mesh)
    beta = lambda X: np.stack([X[..., 1] - 0.45, np.ones_like(X[..., 0])], axis=-1)
    with pytest.raises(ihdg.IHDGError) as ei:
        ctx.var_plan(mesh, beta(vol), beta(fpts))
    assert ei.value.status == ihdg.ERR_UNSUPPORTED


def test_var_full_size_sampled(ctx):
    """The 3D experiment's field at 48^3, p = 2 (the bench workload's shape): k float64 sweeps
    on the GPU against the oracle on dependency patches around sampled elements (after k
    sweeps nothing farther than k elements away can reach an element)."""
    ihdg = ih()
    n, p, k = 48, 2, 3
    mesh, bv, bf, f, g, _, _ = case_big(n, p)
    plan = ctx.var_plan(mesh, bv, bf)
    try:
        u, _, res = plan.solve(f, g, ihdg.make_options(0.0, max_iters=k, diverge_factor=-1.0), want_trace=False)
    finally:
        plan.close()
    assert res.iterations == k
    h = 1.0 / n
    for c in [(0, 0, 0), (n - 1, n - 1, n - 1), (5, 30, n - 1), (20, 2, 17)]:
        lo = [max(0, c[a] - k - 1) for a in range(3)]
        hi = [min(n, c[a] + k + 2) for a in range(3)]
        nn = [hi[a] - lo[a] for a in range(3)]
        om = BoxMesh(3, nn, lo=[lo[a] * h for a in range(3)], hi=[hi[a] * h for a in range(3)])
        disc = Discretisation(om, p)
        pr = TransportVar(disc, W.e2_beta)
        U = pr.iterate(W.e2_forcing(disc.volume_points()), W.e2_exact(disc.boundary_points()), 0.0, max_iters=k,
                       diverge_factor=np.inf)[0]
        loc = (c[0] - lo[0]) + nn[0] * ((c[1] - lo[1]) + nn[1] * (c[2] - lo[2]))
        got = u[c[0] + n * (c[1] + n * c[2])]
        assert rel(got, U[loc, 0, :]) < 1e-10


def case_big(n, p):
    ihdg = ih()
    mesh = ihdg.make_mesh(3, (n, n, n), p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1.0, 0.0, 0.0))
    vol, bnd = ihdg.quadrature_points(mesh, co)
    fpts = ihdg.face_quadrature_points(mesh)
    return mesh, W.e2_beta(vol), W.e2_beta(fpts), W.e2_forcing(vol), W.e2_exact(bnd), None, None


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED_FP32", "MIXED_BF16"])
def test_var_group_equals_alone(ctx, prec_name):
    """Several plans of uneven size and order solved together (one grouped launch per shape
    class and sweep step) give bitwise the results of their own solves: each block of a
    grouped launch works for one plan as that block of the plan's own launch would."""
    ihdg = ih()
    cases = [("e1", 2, (8, 8), 3), ("swirl", 2, (13, 9), 3), ("e1", 2, (5, 7), 2), ("neg", 2, (6, 7), 4),
             ("e2", 3, (4, 3, 5), 2), ("e2", 3, (6, 6, 6), 2), ("e2", 3, (3, 3, 3), 1)]
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    opts = ihdg.make_options(1e-10, max_iters=20000, prec=getattr(ihdg, prec_name))
    plans, bufs, alone = [], [], []
    try:
        for field, d, n, p in cases:
            mesh, bv, bf, f, g, pr, disc = case(field, d, n, p)
            plan = ctx.var_plan(mesh, bv, bf)
            plans.append(plan)
            df = torch.from_numpy(np.ascontiguousarray(f)).to(dev)
            dg = torch.from_numpy(np.ascontiguousarray(g)).to(dev)
            s = plan.sizes
            nb = (p + 1) ** d
            du = torch.empty((s.n_el, nb), dtype=torch.float64, device=dev)
            dt = torch.empty((s.n_face, s.nface_nodes), dtype=torch.float64, device=dev)
            r = plan.solve_device(df.data_ptr(), dg.data_ptr(), opts, du.data_ptr(), dt.data_ptr(), stream)
            alone.append((du.cpu().numpy().copy(), dt.cpu().numpy().copy(), r.iterations, r.status))
            du.fill_(np.nan)
            dt.fill_(np.nan)
            bufs.append((df, dg, du, dt))
        res = ctx.var_solve_group(plans, [b[0].data_ptr() for b in bufs], [b[1].data_ptr() for b in bufs], opts,
                                  [b[2].data_ptr() for b in bufs], [b[3].data_ptr() for b in bufs], stream)
        for (u1, t1, it1, st1), (df, dg, du, dt), r in zip(alone, bufs, res):
            assert r.status == st1 == ihdg.OK and r.iterations == it1
            assert np.array_equal(du.cpu().numpy(), u1) and np.array_equal(dt.cpu().numpy(), t1)
    finally:
        for pl in plans:
            pl.close()
