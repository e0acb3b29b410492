"""Pins for the oracle's quadrature and barycentric basis (paper Sec. 4) against
library routines, textbook closed forms and polynomial exactness."""
import numpy as np
import pytest

from oracle import quadrature as qd


@pytest.mark.parametrize("q", range(1, 11))
def test_gauss_legendre_matches_library(q):
    x, w = qd.gauss_legendre(q)
    xr, wr = np.polynomial.legendre.leggauss(q)
    assert np.allclose(x, xr, atol=1e-15, rtol=0)
    assert np.allclose(w, wr, atol=1e-14, rtol=0)


@pytest.mark.parametrize("q", range(1, 9))
def test_gauss_legendre_exactness(q):
    x, w = qd.gauss_legendre(q)
    for deg in range(0, 2 * q):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(w @ x ** deg - exact) < 1e-14
    # degree 2q is not integrated exactly
    assert abs(w @ x ** (2 * q) - 2.0 / (2 * q + 1)) > 1e-6


def test_gauss_lobatto_closed_forms():
    x, w = qd.gauss_lobatto(3)
    assert np.allclose(x, [-1, 0, 1], atol=1e-16) and np.allclose(w, [1 / 3, 4 / 3, 1 / 3])
    x, w = qd.gauss_lobatto(4)
    s = 1 / np.sqrt(5)
    assert np.allclose(x, [-1, -s, s, 1], atol=1e-15)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    x, w = qd.gauss_lobatto(5)
    s = np.sqrt(3 / 7)
    assert np.allclose(x, [-1, -s, 0, s, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("n", range(2, 10))
def test_gauss_lobatto_exactness(n):
    x, w = qd.gauss_lobatto(n)
    for deg in range(0, 2 * n - 2):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(w @ x ** deg - exact) < 1e-14


@pytest.mark.parametrize("p", range(1, 8))
def test_barycentric_equals_direct_lagrange(p):
    nodes = qd.gauss_lobatto(p + 1)[0]
    pts = np.linspace(-1, 1, 37)
    L = qd.lagrange_matrix(nodes, pts)
    direct = np.ones((len(pts), p + 1))
    for j in range(p + 1):
        for m in range(p + 1):
            if m != j:
                direct[:, j] *= (pts - nodes[m]) / (nodes[j] - nodes[m])
    assert np.abs(L - direct).max() < 1e-14


@pytest.mark.parametrize("p", range(1, 8))
def test_derivative_matrix_exact_on_polynomials(p):
    nodes = qd.gauss_lobatto(p + 1)[0]
    pts = qd.gauss_legendre(p + 2)[0]
    Ld = qd.lagrange_derivative_matrix(nodes, pts)
    for deg in range(0, p + 1):
        vals = nodes ** deg
        d_exact = deg * pts ** (deg - 1) if deg else np.zeros_like(pts)
        assert np.abs(Ld @ vals - d_exact).max() < 1e-12


def test_trace_nodes_are_gl():
    assert np.allclose(qd.trace_nodes(0), [0.0])
    assert np.allclose(qd.trace_nodes(1), [-1 / np.sqrt(3), 1 / np.sqrt(3)])
