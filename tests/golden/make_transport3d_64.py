#!/usr/bin/env python3
"""Writes transport3d_64_p2.json: the float64 oracle's converged solution of the 3D transport
workload at full size, at sampled elements.

Problem: beta.grad u = f on [0,1]^3, 64^3 uniform hexahedra, p = 2, beta = (1,1,1)/sqrt(3),
u = sin(pi x) sin(pi y) sin(pi z), g = u on the inflow boundary, the iHDG iteration
(Algorithm 1) with the upwind flux of Section 3 until ||u^k - u^(k-1)||_{L2} < 1e-8 (Section
5.1).  This is the mesh and launch shape of the bf16 tensor-core mixed solve; the full solution
takes the oracle about a quarter of an hour, so the test compares sampled elements.

Only oracle/ and the input generators in workloads/ are used.  Run from the repository root:
    python tests/golden/make_transport3d_64.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import BoxMesh, Discretisation, Transport  # noqa: E402

N, P, TOL = 64, 2, 1e-8
BETA = tuple(np.ones(3) / np.sqrt(3))


def sample_elements():
    """Corners, face and edge centres, the centre, and seeded interior elements."""
    c, m = N - 1, N // 2
    fixed = [(0, 0, 0), (c, 0, 0), (0, c, 0), (0, 0, c), (c, c, c), (m, 0, 0), (0, m, 0), (0, 0, m),
             (c, m, m), (m, c, m), (m, m, c), (m, m, m)]
    rng = np.random.default_rng(2025)
    rand = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(36)]
    return [i + N * (j + N * k) for i, j, k in fixed + rand]


def main():
    t0 = time.time()
    om = BoxMesh(3, (N, N, N))
    disc = Discretisation(om, P)
    pr = Transport(disc, np.array(BETA))
    f = W.transport3d_forcing(disc.volume_points(), BETA)
    g = W.transport3d_exact(disc.boundary_points())
    U, T, K, res, st = pr.iterate(f, g, TOL, max_iters=4000)
    assert st == 0, st
    els = sample_elements()
    Uf = U.reshape(om.nel, -1)
    out = {
        "what": "float64 oracle (Algorithm 1) solution u^K of 3D transport at sampled elements",
        "cite": "Section 3 (upwind HDG for transport), Algorithm 1, stopping test of Section 5.1",
        "n": [N, N, N], "p": P, "beta": list(BETA), "tol": TOL,
        "iterations": int(K), "residual": float(res),
        "elements": els,
        "u": [[float(v) for v in Uf[e]] for e in els],
        "u_l2_all_nodes": float(np.linalg.norm(Uf)),
        "written_by": "tests/golden/make_transport3d_64.py (oracle only)",
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "transport3d_64_p2.json")
    with open(path, "w") as fh:
        json.dump(out, fh)
    print(f"wrote {path}: K = {K}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
