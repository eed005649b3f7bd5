"""Serving (continuous batching) on the GPU: a mix of requests submitted together is admitted
by HBM footprint into a few slots whose work overlaps, and every result equals the same
request solved alone (the launch configuration depends only on the request itself)."""
import time

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


def make_request(ih, i):
    rng = np.random.default_rng(100 + i)
    side = int(rng.integers(8, 48))
    p = int(rng.integers(1, 5))
    if i % 3 == 0:
        beta = (float(rng.uniform(0.2, 1)), float(rng.uniform(-1, 1)))
        mesh = ih.make_mesh(2, (side, side + 3), p)
        co = ih.make_coeffs(ih.TRANSPORT, beta=beta)
        vol, bnd = ih.quadrature_points(mesh, co)
        f, g = W.transport2d_forcing(vol, beta), W.transport2d_exact(bnd)
    else:
        th = rng.uniform(0, 2 * np.pi)
        beta = (float(np.cos(th)), float(np.sin(th)))
        kappa = 1e-5
        mesh = ih.make_mesh(2, (side, side), p)
        co = ih.make_coeffs(ih.CONVDIFF, beta=beta, kappa=kappa)
        vol, bnd = ih.quadrature_points(mesh, co)
        a, b = rng.uniform(-1, 1, 2)
        f, g = W.convdiff_forcing(vol, kappa, beta, 0.0, a, b), W.convdiff_exact(bnd, a, b)
    prec = [ih.FP64, ih.MIXED_FP32, ih.MIXED_BF16][i % 3]
    return mesh, co, f, g, ih.make_options(1e-9 if prec == ih.FP64 else 1e-7, prec=prec, max_iters=3000)


def test_mix_equals_alone(ctx):
    from paper_1605_03228_gb300 import ihdg as ih
    reqs = [make_request(ih, i) for i in range(12)]
    alone = [ctx.solve(m, c, f, g, o) for (m, c, f, g, o) in reqs]
    ctx.server_start(96 * 1024 * 1024, 4)
    try:
        tickets = [ctx.submit(m, c, f, g, o) for (m, c, f, g, o) in reqs]
        results = [None] * len(reqs)
        t0 = time.time()
        while any(r is None for r in results):
            for k, t in enumerate(tickets):
                if results[k] is None:
                    results[k] = ctx.poll(t)
            assert time.time() - t0 < 120, "serving did not finish"
            time.sleep(0.005)
        for k, (t, (m, c, f, g, o)) in enumerate(zip(tickets, reqs)):
            u, tr = ctx.fetch(t, m, c)
            u_a, tr_a, r_a = alone[k]
            assert results[k].status == r_a.status
            assert results[k].iterations == r_a.iterations
            assert np.array_equal(u, u_a) and np.array_equal(tr, tr_a)
            assert results[k].latency_ms >= results[k].queue_ms >= 0.0
    finally:
        ctx.server_stop()


def test_admission_by_footprint(ctx):
    from paper_1605_03228_gb300 import ihdg as ih
    ctx.server_start(8 * 1024 * 1024, 2)
    try:
        big = ih.make_mesh(2, (256, 256), 3)
        co = ih.make_coeffs(ih.CONVDIFF, beta=(1.0, 1.0), kappa=1e-4)
        s = ih.problem_sizes(big, co)
        with pytest.raises(ih.IHDGError) as e:
            ctx.submit(big, co, np.zeros((s.n_el, s.nqv)), np.zeros((s.n_bface, s.nqf)), ih.make_options(1e-8))
        assert e.value.status == ih.ERR_NOMEM
        # several requests that fit one or two at a time all complete
        small = [make_request(ih, i) for i in (1, 4, 7, 10)]
        tickets = [ctx.submit(m, c, f, g, o) for (m, c, f, g, o) in small]
        t0 = time.time()
        for t, (m, c, f, g, o) in zip(tickets, small):
            while ctx.poll(t) is None:
                assert time.time() - t0 < 120
                time.sleep(0.005)
            ctx.fetch(t, m, c)
    finally:
        ctx.server_stop()
