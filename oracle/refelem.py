"""Reference-element machinery for the oracle: 1D node sets, quadrature, Lagrange bases.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper discretises each element with polynomials of degree p (Section 2, the spaces
V_h and Lambda_h) but does not name a basis or quadrature.  The oracle reads this as:
tensor-product Q^p on each box element, nodal Lagrange basis on the Gauss-Lobatto-Legendre
(GLL) points, and Gauss-Legendre quadrature with p+2 points per direction.  Nothing here is
shared with the CUDA library's own host-side operator builder.

Everything is float64 and written for clarity, not speed.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gll_nodes(p):
    """GLL points on [-1, 1]: the endpoints plus the roots of P_p' (p >= 1).

    p = 0 is given the single midpoint node 0 (piecewise constants), which the oracle uses
    only for the first-order finite-volume special case of the transport method.
    """
    if p == 0:
        return np.array([0.0])
    # coefficients of P_p in the Legendre basis, then its derivative's roots
    cp = np.zeros(p + 1)
    cp[p] = 1.0
    interior = np.sort(np.real(npleg.legroots(npleg.legder(cp)))) if p >= 2 else np.array([])
    return np.concatenate(([-1.0], interior, [1.0]))


def gauss_rule(q):
    """Gauss-Legendre rule with q points on [-1, 1] (exact for degree 2q-1)."""
    x, w = npleg.leggauss(q)
    return x, w


def lagrange_matrix(nodes, x):
    """L[a, i] = l_i(x_a), the i-th Lagrange polynomial on `nodes` evaluated at x_a."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for i in range(n):
        for j in range(n):
            if j != i:
                L[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return L


def lagrange_deriv_matrix(nodes, x):
    """D[a, i] = l_i'(x_a), by the product rule applied to the Lagrange product formula."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((len(x), n))
    for i in range(n):
        denom = 1.0
        for j in range(n):
            if j != i:
                denom *= nodes[i] - nodes[j]
        for m in range(n):
            if m == i:
                continue
            term = np.ones(len(x))
            for j in range(n):
                if j != i and j != m:
                    term *= x - nodes[j]
            D[:, i] += term
        D[:, i] /= denom
    return D


class RefElement:
    """Q^p reference element [-1,1]^d with GLL nodal basis and Gauss quadrature.

    Node and quadrature-point ordering is lexicographic with the x index fastest.
    Local faces are numbered 0:-x, 1:+x, 2:-y, 3:+y, 4:-z, 5:+z; the points on a face are
    ordered lexicographically over the remaining (tangential) axes in increasing axis order.
    """

    def __init__(self, d, p, q=None):
        self.d, self.p = d, p
        self.q = p + 2 if q is None else q
        self.nodes1 = gll_nodes(p)
        self.xq1, self.wq1 = gauss_rule(self.q)
        self.nb1 = p + 1
        self.nb = self.nb1 ** d
        # 1D tables at the Gauss points
        self.B1 = lagrange_matrix(self.nodes1, self.xq1)        # (q, p+1)
        self.D1 = lagrange_deriv_matrix(self.nodes1, self.xq1)  # (q, p+1)
        self.B1_end = lagrange_matrix(self.nodes1, np.array([-1.0, 1.0]))  # (2, p+1)
        self._build()

    @staticmethod
    def _kron_axes(mats):
        """Tensor product with the FIRST matrix varying fastest (x-fastest ordering)."""
        out = mats[0]
        for m in mats[1:]:
            out = np.kron(m, out)
        return out

    def _build(self):
        d = self.d
        self.Bq = self._kron_axes([self.B1] * d)                   # (q^d, nb)
        self.wq = self._kron_axes([self.wq1[:, None]] * d)[:, 0]    # (q^d,)
        # reference derivatives along each axis at the volume Gauss points
        self.Dq = []
        for a in range(d):
            mats = [self.D1 if ax == a else self.B1 for ax in range(d)]
            self.Dq.append(self._kron_axes(mats))
        # reference coordinates of the volume Gauss points, (q^d, d)
        grids = np.meshgrid(*([self.xq1] * d), indexing="ij")
        self.xq = np.stack([g.transpose(tuple(range(d))[::-1]).ravel() for g in grids], axis=1)
        # face tables: basis at face Gauss points and face weights
        self.face_B = []
        tang_w = self._kron_axes([self.wq1[:, None]] * (d - 1))[:, 0] if d > 1 else np.ones(1)
        self.face_w = tang_w
        for f in range(2 * d):
            a, side = f // 2, f % 2
            mats = [self.B1_end[side:side + 1] if ax == a else self.B1 for ax in range(d)]
            self.face_B.append(self._kron_axes(mats))               # (q^(d-1), nb)

    def physical_volume_points(self, lo_corner, h):
        """Physical coordinates of this element's volume Gauss points, (q^d, d)."""
        return lo_corner[None, :] + (self.xq + 1.0) * 0.5 * h[None, :]

    def face_ref_points(self, f):
        """Reference coordinates of the Gauss points on local face f, (q^(d-1), d)."""
        d = self.d
        a, side = f // 2, f % 2
        tang = [ax for ax in range(d) if ax != a]
        nq = self.q ** (d - 1)
        pts = np.zeros((nq, d))
        pts[:, a] = -1.0 if side == 0 else 1.0
        if d > 1:
            grids = np.meshgrid(*([self.xq1] * (d - 1)), indexing="ij")
            for t, ax in enumerate(tang):
                pts[:, ax] = grids[t].transpose(tuple(range(d - 1))[::-1]).ravel()
        return pts

    def node_ref_points(self):
        """Reference coordinates of the GLL nodes, (nb, d), x fastest."""
        d = self.d
        grids = np.meshgrid(*([self.nodes1] * d), indexing="ij")
        return np.stack([g.transpose(tuple(range(d))[::-1]).ravel() for g in grids], axis=1)
