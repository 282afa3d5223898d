"""Reference-triangle tools for the oracle: quadrature rules and nodal (Lagrange) bases.

TEST INFRASTRUCTURE ONLY. This package is the slow, plain FP64 CPU statement of the method
that the CUDA path is checked against. Only tests/, the smoke check and the benchmark's CPU
baseline leg may import it; the product never does.

Reference triangle T = {(xi, eta): xi, eta >= 0, xi + eta <= 1}, vertices (0,0), (1,0), (0,1).
The spaces are the broken polynomial spaces of Sec. 2.2 (eq. function_spaces): P_{k+1} per
velocity component, P_k for the pressure and P_k on each facet for the trace (Sec. 2.4).
The oracle represents each of them by its Lagrange basis at the equispaced lattice nodes,
so a field's coefficients are its values at those nodes.
"""
import numpy as np
from scipy.special import roots_jacobi, roots_legendre


def lattice(m):
    """Equispaced lattice of degree m on the reference triangle: nodes (i/m, j/m) with
    i + j <= m, ordered with j outer and i inner. This is the exchange format for cell fields."""
    if m == 0:
        return np.array([[1.0 / 3.0, 1.0 / 3.0]])
    return np.array([(i / m, j / m) for j in range(m + 1) for i in range(m + 1 - j)], dtype=float)


def lattice_1d(m):
    """Equispaced nodes t = i/m on [0, 1] (the exchange format for facet fields)."""
    if m == 0:
        return np.array([0.5])
    return np.arange(m + 1, dtype=float) / m


def _exponents(m):
    return [(a, b) for b in range(m + 1) for a in range(m + 1 - b)]


def monomials(m, P):
    """xi^a eta^b for a + b <= m at points P (..., 2) -> (..., n_m)."""
    xi, eta = P[..., 0], P[..., 1]
    return np.stack([xi ** a * eta ** b for a, b in _exponents(m)], axis=-1)


def monomial_grads(m, P):
    """Gradients of the monomials at P: (..., n_m, 2)."""
    xi, eta = P[..., 0], P[..., 1]
    out = []
    for a, b in _exponents(m):
        dxi = a * xi ** (a - 1) * eta ** b if a > 0 else np.zeros_like(xi)
        deta = b * xi ** a * eta ** (b - 1) if b > 0 else np.zeros_like(xi)
        out.append(np.stack([dxi, deta], axis=-1))
    return np.stack(out, axis=-2)


class LagrangeTri:
    """Lagrange basis of P_m on the reference triangle at the lattice of degree m."""

    def __init__(self, m):
        self.m = m
        self.nodes = lattice(m)
        self.n = len(self.nodes)
        self.C = np.linalg.inv(monomials(m, self.nodes))   # monomial -> nodal coefficients

    def values(self, P):
        return monomials(self.m, P) @ self.C

    def grads(self, P):
        return np.einsum('...ms,mn->...ns', monomial_grads(self.m, P), self.C)


class Lagrange1D:
    """Lagrange basis of P_m on [0, 1] at t = i/m."""

    def __init__(self, m):
        self.m = m
        self.nodes = lattice_1d(m)
        self.n = len(self.nodes)
        V = np.stack([self.nodes ** j for j in range(m + 1)], axis=-1)
        self.C = np.linalg.inv(V)

    def values(self, t):
        t = np.asarray(t, dtype=float)
        return np.stack([t ** j for j in range(self.m + 1)], axis=-1) @ self.C


def triangle_quadrature(n):
    """Collapsed (Duffy) Gauss rule with n x n points on the reference triangle.

    xi = (1+u)(1-v)/4, eta = (1+v)/2 with Gauss-Legendre nodes in u and Gauss-Jacobi(1,0)
    nodes in v (weight 1-v absorbs the Jacobian). Exact for total degree 2n-1.
    """
    u, wu = roots_legendre(n)
    v, wv = roots_jacobi(n, 1.0, 0.0)
    U, V = np.meshgrid(u, v, indexing='ij')
    xi = (1.0 + U) * (1.0 - V) / 4.0
    eta = (1.0 + V) / 2.0
    W = np.outer(wu, wv) / 8.0
    return np.stack([xi.ravel(), eta.ravel()], axis=-1), W.ravel()


def line_quadrature(n):
    """n-point Gauss-Legendre rule on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1.0) / 2.0, w / 2.0


def volume_points(k):
    """Points per direction for cell integrals: exact for the advection integrand of degree
    3k+2 (w in P_{k+1}, Q* in P_{k+1}, grad Q in P_k)."""
    return (3 * k + 4) // 2


def facet_points(k):
    """Gauss-Legendre points on a facet: (3k+5)//2, exact for degree 3k+3 (Q*.n Q.w). The
    upwind integrand |Q*.n| is not a polynomial, so this rule is part of the discretisation
    and the CUDA path uses the same point count."""
    return (3 * k + 5) // 2
