"""Failure detection without a GPU fault.

* Every grid-barrier wait of the persistent kernels (the mixed path's inner loops and the
  float64 loop) is bounded.  A test-only hook set
  on the host (IHDG_TEST_STALL_BLOCK: that block never arrives) together with a short bound
  (IHDG_TEST_WAIT_CYCLES, ~10 ms) makes every block's wait run out: the kernels leave their
  loops (the tensor-core kernel also frees its tensor memory), the call returns
  IHDG_ERR_TIMEOUT, and the next solve on the same context gives the same result as before.
* Corrupted input: a NaN in the forcing is reported as DIVERGED (non-finite residual), on
  the float64 and the mixed path.
"""
import numpy as np
import pytest

import workloads as W

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


def problem(ih, case):
    if case == "cd2d":
        mesh = ih.make_mesh(2, (64, 48), 3)
        co = ih.make_coeffs(ih.CONVDIFF, beta=(1.0, 1.0), kappa=1e-4)
        vol, bnd = ih.quadrature_points(mesh, co)
        return mesh, co, W.convdiff_forcing(vol, 1e-4), W.convdiff_exact(bnd)
    b = tuple(np.ones(3) / np.sqrt(3))
    mesh = ih.make_mesh(3, (12, 12, 12), 2)
    co = ih.make_coeffs(ih.TRANSPORT, beta=b)
    vol, bnd = ih.quadrature_points(mesh, co)
    return mesh, co, W.transport3d_forcing(vol, b), W.transport3d_exact(bnd)


@pytest.mark.parametrize("case,prec,kernel", [("cd2d", "MIXED_FP32", ""), ("t3d", "MIXED_BF16", ""),
                                              ("t3d", "MIXED_FP32", "tile"), ("cd2d", "MIXED_FP32", "global"),
                                              ("cd2d", "FP64", "")])
def test_barrier_wait_runs_out_and_context_stays_usable(ctx, monkeypatch, case, prec, kernel):
    from paper_1605_03228_gb300 import ihdg as ih
    mesh, co, f, g = problem(ih, case)
    if kernel:
        monkeypatch.setenv("IHDG_INNER_KERNEL", kernel)
    opts = ih.make_options(1e-8, prec=getattr(ih, prec), max_iters=5000)
    u_ref, _, r_ref = ctx.solve(mesh, co, f, g, opts)
    assert r_ref.status == ih.OK
    monkeypatch.setenv("IHDG_TEST_WAIT_CYCLES", "20000000")
    monkeypatch.setenv("IHDG_TEST_STALL_BLOCK", "0")
    with pytest.raises(ih.IHDGError) as e:
        ctx.solve(mesh, co, f, g, opts)
    assert e.value.status == ih.ERR_TIMEOUT
    monkeypatch.delenv("IHDG_TEST_STALL_BLOCK")
    monkeypatch.delenv("IHDG_TEST_WAIT_CYCLES")
    u, _, r = ctx.solve(mesh, co, f, g, opts)
    assert r.status == ih.OK and r.iterations == r_ref.iterations
    assert np.array_equal(u, u_ref)


@pytest.mark.parametrize("prec", ["FP64", "MIXED_FP32"])
def test_nan_forcing_is_reported_as_diverged(ctx, prec):
    from paper_1605_03228_gb300 import ihdg as ih
    mesh, co, f, g = problem(ih, "cd2d")
    f = f.copy()
    f[100, 3] = np.nan
    u, _, r = ctx.solve(mesh, co, f, g, ih.make_options(1e-8, prec=getattr(ih, prec), max_iters=5000))
    assert r.status == ih.DIVERGED


@pytest.mark.parametrize("prec", ["MIXED_FP32", "MIXED_BF16"])
def test_operator_copy_wait_runs_out_and_plan_stays_usable(ctx, monkeypatch, prec):
    """Variable-coefficient transport: the inner sweep streams each element's operator into
    shared memory with bulk copies and waits for them with a bounded wait.  Under the test hook
    one warp issues no copy (IHDG_TEST_STALL_BLOCK) and the bound is ~10 ms: its wait runs out,
    the call returns IHDG_ERR_TIMEOUT, and the next solve on the same plan gives the same
    result as before."""
    from paper_1605_03228_gb300 import ihdg as ih
    mesh = ih.make_mesh(2, (40, 36), 3, hi=(2.0, 2.0))
    co = ih.make_coeffs(ih.TRANSPORT, beta=(1.0, 0.0, 0.0))
    vol, bnd = ih.quadrature_points(mesh, co)
    fpts = ih.face_quadrature_points(mesh)
    plan = ctx.var_plan(mesh, W.e1_beta(vol), W.e1_beta(fpts))
    try:
        f, g = np.zeros(vol.shape[:2]), W.e1_inflow(bnd)
        opts = ih.make_options(1e-10, prec=getattr(ih, prec), max_iters=20000)
        u_ref, _, r_ref = plan.solve(f, g, opts, want_trace=False)
        assert r_ref.status == ih.OK
        monkeypatch.setenv("IHDG_TEST_WAIT_CYCLES", "20000000")
        monkeypatch.setenv("IHDG_TEST_STALL_BLOCK", "0")
        with pytest.raises(ih.IHDGError) as e:
            plan.solve(f, g, opts, want_trace=False)
        assert e.value.status == ih.ERR_TIMEOUT
        monkeypatch.delenv("IHDG_TEST_STALL_BLOCK")
        monkeypatch.delenv("IHDG_TEST_WAIT_CYCLES")
        u, _, r = plan.solve(f, g, opts, want_trace=False)
        assert r.status == ih.OK and r.iterations == r_ref.iterations
        assert np.array_equal(u, u_ref)
    finally:
        plan.close()


def test_grouped_barrier_wait_runs_out_and_context_stays_usable(ctx, monkeypatch):
    """Grouped float64 solves: a block that never arrives at its problem's grid barrier makes
    that problem's bounded waits run out; the call returns IHDG_ERR_TIMEOUT, and the next
    grouped call on the same context and workspace solves normally."""
    import torch
    from paper_1605_03228_gb300 import ihdg as ih
    probs = [problem(ih, "cd2d"), problem(ih, "t3d")]
    dev = torch.device("cuda:0")
    opts = ih.make_options(1e-8, max_iters=5000)
    meshes, coeffs = [p[0] for p in probs], [p[1] for p in probs]
    fs = [torch.from_numpy(np.ascontiguousarray(p[2])).to(dev) for p in probs]
    gs = [torch.from_numpy(np.ascontiguousarray(p[3])).to(dev) for p in probs]
    sz = [ih.problem_sizes(m, c) for m, c in zip(meshes, coeffs)]
    us = [torch.zeros((s.n_el, s.nvol), dtype=torch.float64, device=dev) for s in sz]
    nws = ctx.group_workspace_bytes(meshes, coeffs, opts)
    ws = torch.empty(nws + 256, dtype=torch.uint8, device=dev)
    wsp = (ws.data_ptr() + 255) // 256 * 256
    args = ([x.data_ptr() for x in fs], [x.data_ptr() for x in gs], opts, [x.data_ptr() for x in us], None, wsp, nws)
    monkeypatch.setenv("IHDG_TEST_WAIT_CYCLES", "20000000")
    monkeypatch.setenv("IHDG_TEST_STALL_BLOCK", "0")
    with pytest.raises(ih.IHDGError) as e:
        ctx.solve_group_device(meshes, coeffs, *args)
    assert e.value.status == ih.ERR_TIMEOUT
    monkeypatch.delenv("IHDG_TEST_WAIT_CYCLES")
    monkeypatch.delenv("IHDG_TEST_STALL_BLOCK")
    res = ctx.solve_group_device(meshes, coeffs, *args)
    assert all(r.status == ih.OK for r in res)
