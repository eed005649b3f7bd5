"""The no-allocation solve (ihdg_solve_device_static) against the workspace solve.

Some callers cannot allocate device memory (an application whose allocator owns the whole
GPU, or a pipeline where a synchronising cudaMalloc is not allowed).  For them the library
keeps one static device array as scratch.  These tests call that entry point through the C
ABI twice in a row, on different problems and precisions, and compare each result with the
ordinary entry point that takes a caller workspace (same iteration count; relative L2
difference within the float64 bar of the parity tests, 1e-10).  A problem too large for the
array must be refused with IHDG_ERR_NOMEM before any GPU work.

This file is named to be collected last, so that a run stopping at its first failure has run
every other test already; it also passes alone in a fresh process.
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


def problem(ih, kind):
    if kind == "transport":
        mesh = ih.make_mesh(2, (24, 20), 3)
        co = ih.make_coeffs(ih.TRANSPORT, beta=(1.0, 0.5))
        vol, bnd = ih.quadrature_points(mesh, co)
        return mesh, co, W.transport2d_forcing(vol), W.transport2d_exact(bnd), ih.make_options(1e-10)
    mesh = ih.make_mesh(2, (32, 28), 2)
    co = ih.make_coeffs(ih.CONVDIFF, beta=(1.0, 1.0), kappa=1e-4)
    vol, bnd = ih.quadrature_points(mesh, co)
    return mesh, co, W.convdiff_forcing(vol, 1e-4), W.convdiff_exact(bnd), ih.make_options(1e-9, prec=ih.MIXED_FP32)


def run_both(ctx, ih, kind):
    mesh, co, f, g, opts = problem(ih, kind)
    s = ih.problem_sizes(mesh, co)
    dev = torch.device("cuda:0")
    df = torch.from_numpy(np.ascontiguousarray(f)).to(dev)
    dg = torch.from_numpy(np.ascontiguousarray(g)).to(dev)
    u_ref = torch.empty((s.n_el, s.nvol), dtype=torch.float64, device=dev)
    t_ref = torch.empty((s.n_face, s.nface_nodes), dtype=torch.float64, device=dev)
    u_st = torch.full_like(u_ref, float("nan"))
    t_st = torch.full_like(t_ref, float("nan"))
    nws = ih.workspace_bytes(mesh, co, opts)
    ws = torch.empty(nws + 256, dtype=torch.uint8, device=dev)
    wsp = (ws.data_ptr() + 255) // 256 * 256
    stream = torch.cuda.current_stream().cuda_stream
    r_ref = ctx.solve_device(mesh, co, df.data_ptr(), dg.data_ptr(), opts, u_ref.data_ptr(), t_ref.data_ptr(),
                             wsp, nws, stream)
    r_st = ctx.solve_device_static(mesh, co, df.data_ptr(), dg.data_ptr(), opts, u_st.data_ptr(), t_st.data_ptr(),
                                   stream)
    torch.cuda.synchronize()
    return r_ref, r_st, u_ref.cpu().numpy(), u_st.cpu().numpy(), t_ref.cpu().numpy(), t_st.cpu().numpy()


def test_static_solve_matches_workspace_solve_twice(ctx):
    from paper_1605_03228_gb300 import ihdg as ih
    for kind in ("transport", "convdiff"):          # two calls in a row, different problems
        r_ref, r_st, u_ref, u_st, t_ref, t_st = run_both(ctx, ih, kind)
        assert r_ref.status == r_st.status == ih.OK
        assert r_st.iterations == r_ref.iterations
        assert np.linalg.norm(u_st - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
        assert np.linalg.norm(t_st - t_ref) <= 1e-10 * np.linalg.norm(t_ref)


def test_static_solve_refuses_oversized_problem(ctx):
    from paper_1605_03228_gb300 import ihdg as ih
    mesh = ih.make_mesh(2, (512, 512), 3)          # ~270 MB of float64 exports: above the array
    co = ih.make_coeffs(ih.CONVDIFF, beta=(1.0, 1.0), kappa=1e-4)
    dev = torch.device("cuda:0")
    dummy = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises(ih.IHDGError) as e:
        ctx.solve_device_static(mesh, co, dummy.data_ptr(), dummy.data_ptr(), ih.make_options(1e-8),
                                dummy.data_ptr(), 0)
    assert e.value.status == ih.ERR_NOMEM
    assert "bytes of scratch" in str(e.value)
