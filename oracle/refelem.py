"""Reference triangle: nodes, nodal Lagrange basis, quadrature (oracle).

The paper uses a nodal DG method on triangles (Sec. 6) without stating nodes
or quadrature.  Readings adopted:

* reference triangle (0,0), (1,0), (0,1); element vertex v_k maps to the k-th
  corner;
* equispaced nodes (i/p, j/p), ordered j-major: for j = 0..p, i = 0..p-j;
* Lagrange basis built from the monomial Vandermonde (phi_i(node_k) = delta_ik);
* volume quadrature: collapsed (Duffy) tensor Gauss-Legendre with n = p+2
  points per direction, exact for total degree 2n-2;
* face quadrature: n = p+2 Gauss-Legendre points on [0, 1];
* local face f runs from vertex f to vertex (f+1) % 3.
"""
import numpy as np

CORNERS = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])


def nodes(p):
    pts = [(i / p, j / p) for j in range(p + 1) for i in range(p + 1 - j)]
    return np.array(pts, dtype=np.float64)


def monomial_exponents(p):
    return [(a, b) for a in range(p + 1) for b in range(p + 1 - a)]


def _monomials(xi, p, deriv=None):
    """Monomials xi^a eta^b (and their first derivatives) at points xi [n, 2]."""
    x = xi[:, 0]
    y = xi[:, 1]
    cols = []
    for a, b in monomial_exponents(p):
        if deriv is None:
            cols.append(x**a * y**b)
        elif deriv == 0:
            cols.append(a * x ** max(a - 1, 0) * y**b if a > 0 else 0.0 * x)
        else:
            cols.append(b * x**a * y ** max(b - 1, 0) if b > 0 else 0.0 * x)
    return np.stack(cols, axis=1)


class Basis:
    def __init__(self, p):
        self.p = p
        self.nodes = nodes(p)
        self.np = len(self.nodes)
        V = _monomials(self.nodes, p)
        self.coef = np.linalg.solve(V, np.eye(self.np))  # columns: Lagrange coefficients

    def phi(self, xi):
        return _monomials(np.atleast_2d(xi), self.p) @ self.coef

    def dphi(self, xi):
        xi = np.atleast_2d(xi)
        return np.stack([_monomials(xi, self.p, 0) @ self.coef,
                         _monomials(xi, self.p, 1) @ self.coef], axis=-1)  # [n, Np, 2]


def gauss_legendre_01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def triangle_rule(n):
    """Collapsed-coordinate rule on the reference triangle; weights sum to 1/2."""
    a, wa = np.polynomial.legendre.leggauss(n)
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            xi = (1.0 + a[i]) * (1.0 - a[j]) / 4.0
            eta = (1.0 + a[j]) / 2.0
            pts.append((xi, eta))
            wts.append(wa[i] * wa[j] * (1.0 - a[j]) / 8.0)
    return np.array(pts), np.array(wts)


def face_points(f, s):
    """Reference coordinates of parameter s in [0,1] along local face f."""
    s = np.asarray(s, dtype=np.float64)
    a = CORNERS[f]
    b = CORNERS[(f + 1) % 3]
    return a[None, :] + s[:, None] * (b - a)[None, :]
