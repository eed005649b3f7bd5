#!/usr/bin/env python3
"""Writes convdiff2d_256_p3.json: the float64 oracle's converged solution of the 2D
convection-diffusion workload at full size, at sampled elements.

Problem: -kappa Lap u + beta.grad u = f on [0,1]^2, 256 x 256 uniform quads, p = 3,
kappa = 1e-4, beta = (1, 1), u = exp(x+y) sin(pi x) sin(pi y), g = u on the boundary, the
iHDG iteration (Algorithm 1) with the upwind stabilisation of Section 4.1 until
||u^k - u^(k-1)||_{L2} < 1e-8 (Section 5.1).  This is the mesh and launch shape of the
headline mixed-precision solve; the full solution at this size takes the oracle minutes, so
the test compares sampled elements.

Only oracle/ and the input generators in workloads/ are used.  Run from the repository root:
    python tests/golden/make_convdiff2d_256.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import BoxMesh, ConvDiff, Discretisation  # noqa: E402

N, P, KAPPA, BETA, TOL = 256, 3, 1e-4, (1.0, 1.0), 1e-8


def sample_elements():
    """Corners, edge midpoints, the centre, and seeded interior elements (x index fastest)."""
    fixed = [(0, 0), (N - 1, 0), (0, N - 1), (N - 1, N - 1), (N // 2, 0), (0, N // 2), (N - 1, N // 2),
             (N // 2, N - 1), (N // 2, N // 2)]
    rng = np.random.default_rng(2024)
    rand = [tuple(int(v) for v in rng.integers(0, N, 2)) for _ in range(39)]
    return [i + N * j for i, j in fixed + rand]


def main():
    t0 = time.time()
    om = BoxMesh(2, (N, N))
    disc = Discretisation(om, P)
    pr = ConvDiff(disc, np.array(BETA), KAPPA)
    f = W.convdiff_forcing(disc.volume_points(), KAPPA, BETA)
    g = W.convdiff_exact(disc.boundary_points())
    U, T, K, res, st = pr.iterate(f, g, TOL, max_iters=4000)
    assert st == 0, st
    els = sample_elements()
    Uf = U.reshape(om.nel, -1)
    out = {
        "what": "float64 oracle (Algorithm 1) solution u^K of 2D convection-diffusion at sampled elements",
        "cite": "Section 4.1 (upwind HDG for convection-diffusion), Algorithm 1, stopping test of Section 5.1",
        "n": [N, N], "p": P, "kappa": KAPPA, "beta": list(BETA), "tol": TOL,
        "iterations": int(K), "residual": float(res),
        "elements": els,
        "u": [[float(v) for v in Uf[e]] for e in els],
        "u_l2_all_nodes": float(np.linalg.norm(Uf)),
        "written_by": "tests/golden/make_convdiff2d_256.py (oracle only)",
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "convdiff2d_256_p3.json"), "w") as fh:
        json.dump(out, fh, indent=0)
    print(f"K={K} res={res:.3e} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
