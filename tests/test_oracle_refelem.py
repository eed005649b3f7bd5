"""Pins for the oracle's reference element: closed forms and exactness (test layer 1)."""
import numpy as np
import pytest

from oracle.refelem import RefElement, gauss_rule, gll_nodes, lagrange_deriv_matrix, lagrange_matrix


def test_gll_closed_forms():
    # GLL points: +-1 and the roots of P_p'
    assert np.allclose(gll_nodes(1), [-1, 1], atol=1e-15)
    assert np.allclose(gll_nodes(2), [-1, 0, 1], atol=1e-15)
    assert np.allclose(gll_nodes(3), [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1], atol=1e-14)
    assert np.allclose(gll_nodes(4), [-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1], atol=1e-14)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6])
def test_gauss_exactness(q):
    x, w = gauss_rule(q)
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_cardinal_and_derivative(p):
    nodes = gll_nodes(p)
    assert np.allclose(lagrange_matrix(nodes, nodes), np.eye(p + 1), atol=1e-14)
    x = np.linspace(-1, 1, 17)
    # interpolating x^k (k <= p) is exact, and so is its derivative
    for k in range(p + 1):
        assert np.allclose(lagrange_matrix(nodes, x) @ nodes ** k, x ** k, atol=1e-13)
        dk = k * x ** (k - 1) if k > 0 else 0 * x
        assert np.allclose(lagrange_deriv_matrix(nodes, x) @ nodes ** k, dk, atol=1e-12)


@pytest.mark.parametrize("d,p", [(1, 2), (2, 1), (2, 3), (3, 2)])
def test_tensor_mass_moments(d, p):
    ref = RefElement(d, p)
    M = ref.Bq.T @ (ref.wq[:, None] * ref.Bq)
    xn = ref.node_ref_points()
    # (1, 1) = 2^d ; (x_0, 1) = 0 ; (x_0^2, 1) = 2^d / 3  (exact moments on [-1,1]^d)
    one = np.ones(ref.nb)
    assert abs(one @ M @ one - 2.0 ** d) < 1e-13
    assert abs(xn[:, 0] @ M @ one) < 1e-13
    if p >= 1:
        assert abs(xn[:, 0] @ M @ xn[:, 0] - 2.0 ** d / 3) < 1e-13
    # face tables: restriction of the node coordinate to face 1 (+x) is identically +1
    assert np.allclose(ref.face_B[1] @ xn[:, 0], 1.0)
    assert np.allclose(ref.face_B[0] @ xn[:, 0], -1.0)
