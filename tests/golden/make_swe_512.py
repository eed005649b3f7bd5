#!/usr/bin/env python3
"""Writes swe_512_p2.json: the float64 oracle's state after two backward-Euler steps of the
linearized shallow-water workload at full size, at sampled elements.

Problem: linearized shallow water (Section 3, Eq. localSolverDD), Phi = 1, no Coriolis or
friction, walls, 512 x 512 uniform quads on [0,1]^2, p = 2, dt = h/((p+1)(p+2)) = 1/6144, the
seeded Gaussian bump of the workload generators (seed 0) as q^0; each step runs the iHDG
iteration warm-started from the previous state until ||q^k - q^(k-1)|| < 1e-8 (phi and
Phi-weighted velocity, Section 5.1).  This is the mesh and launch shape of the 100-step
shallow-water workload; the full state takes the oracle about a quarter of an hour for two
steps, so the test compares sampled elements.

Only oracle/ and the input generators in workloads/ are used.  Run from the repository root:
    python tests/golden/make_swe_512.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import BoxMesh, Discretisation, ShallowWater  # noqa: E402

N, P, TOL, STEPS = 512, 2, 1e-8, 2
DT = 1.0 / (N * (P + 1) * (P + 2))


def sample_elements():
    """Corners, edge midpoints, the centre (the bump's neighbourhood), and seeded elements."""
    c, m = N - 1, N // 2
    fixed = [(0, 0), (c, 0), (0, c), (c, c), (m, 0), (0, m), (c, m), (m, c), (m, m)]
    rng = np.random.default_rng(2026)
    rand = [tuple(int(v) for v in rng.integers(0, N, 2)) for _ in range(39)]
    return [i + N * j for i, j in fixed + rand]


def main():
    t0 = time.time()
    om = BoxMesh(2, (N, N))
    disc = Discretisation(om, P)
    pr = ShallowWater(disc, 1.0, DT)
    U = W.swe_bump(disc.node_points(), seed=0)
    its = []
    for _ in range(STEPS):
        U, T, K, res, st = pr.step(U, TOL, max_iters=4000)
        assert st == 0, st
        its.append(int(K))
    els = sample_elements()
    Uf = U.reshape(om.nel, -1)
    out = {
        "what": "float64 oracle state q after two backward-Euler shallow-water steps at sampled elements",
        "cite": "Section 3 (Eq. localSolverDD, backward Euler), Algorithm 1 per step with warm start, Section 5.1 stopping test",
        "n": [N, N], "p": P, "Phi": 1.0, "dt": DT, "tol": TOL, "steps": STEPS, "bump_seed": 0,
        "iterations_per_step": its,
        "elements": els,
        "q": [[float(v) for v in Uf[e]] for e in els],
        "written_by": "tests/golden/make_swe_512.py (oracle only)",
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "swe_512_p2.json")
    with open(path, "w") as fh:
        json.dump(out, fh)
    print(f"wrote {path}: iterations {its}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
