"""Seeded synthetic inputs shared by the tests, the smoke check and bench.py.

This module holds none of the method's arithmetic.  It evaluates closed-form manufactured
solutions, forcings and boundary data at physical points that the caller supplies (from the
library's ihdg_quadrature_points / ihdg_node_points, or from the oracle's own point
generators), and draws the seeded random numbers the workloads call for.

Workloads (the sizes are the ones the benchmarks and parity tests use):
  transport2d   2D steady transport, beta = (1, 0.5), u = sin(pi x) cos(pi y) on [0,1]^2
  convdiff2d    2D convection-diffusion, -kappa Lap u + beta.grad u = f, beta = (1, 1),
                u = exp(x+y) sin(pi x) sin(pi y), homogeneous Dirichlet data
  transport3d   3D steady transport, beta = (1,1,1)/sqrt(3), u = sin(pi x) sin(pi y) sin(pi z)
  swe_bump      2D linearized shallow water, Gaussian bump in phi with seeded 1% amplitude
                noise per GLL node, zero velocity
  e1, e2        transport with velocity fields that vary in space: beta = (1 + sin(pi y/2), 2)
                on [0,2]^2 with discontinuous inflow data, and beta = (z, x, y) on [0,1]^3 with
                u = sin(pi x) cos(pi y) sin(pi z) / pi
  serving       a seeded stream of convection-diffusion requests with Poisson arrivals
"""
import math

import numpy as np

PI = math.pi


# ----------------------------------------------------------------------------- transport
def transport2d_exact(X):
    return np.sin(PI * X[..., 0]) * np.cos(PI * X[..., 1])


def transport2d_forcing(X, beta=(1.0, 0.5)):
    x, y = X[..., 0], X[..., 1]
    return beta[0] * PI * np.cos(PI * x) * np.cos(PI * y) - beta[1] * PI * np.sin(PI * x) * np.sin(PI * y)


def transport3d_exact(X):
    return np.sin(PI * X[..., 0]) * np.sin(PI * X[..., 1]) * np.sin(PI * X[..., 2])


def transport3d_forcing(X, beta=(1 / math.sqrt(3),) * 3):
    s = [np.sin(PI * X[..., a]) for a in range(3)]
    c = [np.cos(PI * X[..., a]) for a in range(3)]
    return PI * (beta[0] * c[0] * s[1] * s[2] + beta[1] * s[0] * c[1] * s[2] + beta[2] * s[0] * s[1] * c[2])


# ----------------------------------------------------------------------------- variable beta
# The two transport experiments of the paper's Section 5.1 (Table 1), with velocity fields
# that vary in space.
def e1_beta(X):
    """2D: beta = (1 + sin(pi y / 2), 2) on [0,2]^2 (divergence-free)."""
    y = X[..., 1]
    return np.stack([1.0 + np.sin(PI * y / 2.0), np.full_like(y, 2.0)], axis=-1)


def e1_inflow(X):
    """2D inflow data: 1 on x = 0; sin^6(pi x) on y = 0 for 0 < x <= 1; 0 on y = 0 for x >= 1;
    the forcing is zero.  Evaluated on boundary points (outflow points get values that the
    upwind flux never reads)."""
    x, y = X[..., 0], X[..., 1]
    return np.where(x <= 0.0, 1.0, np.where((y <= 0.0) & (x <= 1.0), np.sin(PI * x) ** 6, 0.0))


def e2_beta(X):
    """3D: beta = (z, x, y) on [0,1]^3 (divergence-free, inflow faces x = 0, y = 0, z = 0)."""
    return np.stack([X[..., 2], X[..., 0], X[..., 1]], axis=-1)


def e2_exact(X):
    """u = sin(pi x) cos(pi y) sin(pi z) / pi."""
    return np.sin(PI * X[..., 0]) * np.cos(PI * X[..., 1]) * np.sin(PI * X[..., 2]) / PI


def e2_forcing(X):
    """f = beta.grad u for beta = (z, x, y) and u = sin(pi x) cos(pi y) sin(pi z) / pi."""
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    sx, cx, sy, cy, sz, cz = (np.sin(PI * x), np.cos(PI * x), np.sin(PI * y), np.cos(PI * y), np.sin(PI * z),
                              np.cos(PI * z))
    return z * cx * cy * sz - x * sx * sy * sz + y * sx * cy * cz


# ----------------------------------------------------------------------------- conv.-diff.
def convdiff_exact(X, a=1.0, b=1.0):
    """u = exp(a x + b y) sin(pi x) sin(pi y) (the 2D workload has a = b = 1)."""
    x, y = X[..., 0], X[..., 1]
    return np.exp(a * x + b * y) * np.sin(PI * x) * np.sin(PI * y)


def convdiff_forcing(X, kappa, beta=(1.0, 1.0), nu=0.0, a=1.0, b=1.0):
    """f = -kappa (u_xx + u_yy) + beta.grad u + nu u for u = exp(a x + b y) sin(pi x) sin(pi y)."""
    x, y = X[..., 0], X[..., 1]
    E = np.exp(a * x + b * y)
    sx, cx, sy, cy = np.sin(PI * x), np.cos(PI * x), np.sin(PI * y), np.cos(PI * y)
    ux = E * sy * (a * sx + PI * cx)
    uy = E * sx * (b * sy + PI * cy)
    uxx = E * sy * ((a * a - PI * PI) * sx + 2 * a * PI * cx)
    uyy = E * sx * ((b * b - PI * PI) * sy + 2 * b * PI * cy)
    return -kappa * (uxx + uyy) + beta[0] * ux + beta[1] * uy + nu * E * sx * sy


# ----------------------------------------------------------------------------- shallow water
def swe_bump(node_xyz, seed=0, amp=0.1, width=0.05, noise=0.01, center=(0.5, 0.5)):
    """Initial state (phi, u, v) at GLL nodes, shape [n_el, 3, nb]: a Gaussian bump of height
    amp and width `width` times (1 + noise*xi), xi ~ U[-1, 1] per node from
    numpy.random.default_rng(seed); zero velocity."""
    x, y = node_xyz[..., 0], node_xyz[..., 1]
    rng = np.random.default_rng(seed)
    xi = rng.uniform(-1.0, 1.0, size=x.shape)
    q = np.zeros((x.shape[0], 3, x.shape[1]))
    q[:, 0] = amp * np.exp(-((x - center[0]) ** 2 + (y - center[1]) ** 2) / (2 * width ** 2)) * (1 + noise * xi)
    return q


def swe_standing_wave(node_xyz, t):
    """Exact standing wave with Phi = 1 in the unit square with walls (phi, u, v)."""
    x, y = node_xyz[..., 0], node_xyz[..., 1]
    s2 = math.sqrt(2.0)
    q = np.zeros((x.shape[0], 3, x.shape[1]))
    q[:, 0] = np.cos(PI * x) * np.cos(PI * y) * np.cos(s2 * PI * t)
    q[:, 1] = np.sin(PI * x) * np.cos(PI * y) * np.sin(s2 * PI * t) / s2
    q[:, 2] = np.cos(PI * x) * np.sin(PI * y) * np.sin(s2 * PI * t) / s2
    return q


# ----------------------------------------------------------------------------- serving
def serving_requests(n=10000, seed=12345):
    """The seeded request mix: side s = round(16 * 16^U), p ~ U{1..4}, kappa = 10^(-4 + 4U),
    beta = (cos t, sin t) with t ~ U[0, 2 pi), manufactured u = exp(a x + b y) sin sin with
    a, b ~ U[-1, 1]; request i draws from numpy.random.default_rng(i).  Arrival gaps are
    unit-rate exponentials from default_rng(seed); callers scale them to an offered load."""
    reqs = []
    for i in range(n):
        r = np.random.default_rng(i)
        side = int(round(16 * 16 ** r.uniform()))
        p = int(r.integers(1, 5))
        kappa = 10 ** (-4 + 4 * r.uniform())
        th = r.uniform(0, 2 * PI)
        a, b = r.uniform(-1, 1, size=2)
        reqs.append(dict(id=i, side=side, p=p, kappa=float(kappa), beta=(math.cos(th), math.sin(th)),
                         a=float(a), b=float(b)))
    gaps = np.random.default_rng(seed).exponential(1.0, size=n)
    return reqs, gaps
