"""Pins for the oracle's reference element: closed-form integrals and the
Lagrange property (nodes/quadrature readings of Sec. 6, see oracle.refelem)."""
from math import factorial

import numpy as np
import pytest

from oracle import refelem


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_triangle_rule_exact_on_monomials(n):
    x, w = refelem.triangle_rule(n)
    assert abs(w.sum() - 0.5) < 1e-15
    for a in range(2 * n - 1):
        for b in range(2 * n - 1 - a):
            exact = factorial(a) * factorial(b) / factorial(a + b + 2)
            assert abs(np.sum(w * x[:, 0] ** a * x[:, 1] ** b) - exact) < 1e-15


@pytest.mark.parametrize("n", [2, 3, 5, 6])
def test_gauss_legendre_01(n):
    s, w = refelem.gauss_legendre_01(n)
    for k in range(2 * n):
        assert abs(np.sum(w * s**k) - 1.0 / (k + 1)) < 1e-15


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_basis(p):
    B = refelem.Basis(p)
    assert B.np == (p + 1) * (p + 2) // 2
    assert np.allclose(B.phi(B.nodes), np.eye(B.np), atol=1e-12)
    x, _ = refelem.triangle_rule(p + 2)
    assert np.allclose(B.phi(x).sum(1), 1.0, atol=1e-13)
    assert np.allclose(B.dphi(x).sum(1), 0.0, atol=1e-11)
    # derivative against central differences of phi
    h = 1e-6
    for d in range(2):
        e = np.zeros(2)
        e[d] = h
        fd = (B.phi(x + e) - B.phi(x - e)) / (2 * h)
        assert np.allclose(B.dphi(x)[:, :, d], fd, atol=1e-7)
    M = np.einsum("q,qi,qj->ij", *[refelem.triangle_rule(p + 2)[1], B.phi(x), B.phi(x)])
    assert abs(M.sum() - 0.5) < 1e-14
    assert np.all(np.linalg.eigvalsh(M) > 0)


def test_face_points_run_vertex_to_vertex():
    for f in range(3):
        pts = refelem.face_points(f, np.array([0.0, 1.0]))
        assert np.allclose(pts[0], refelem.CORNERS[f])
        assert np.allclose(pts[1], refelem.CORNERS[(f + 1) % 3])
