"""Pins of the oracle's reference element and mesh against closed forms and the paper's table."""
import math
import os

import numpy as np
import pytest

from oracle import Mesh, dof_counts, LagrangeTri, Lagrange1D, triangle_quadrature, line_quadrature
from oracle.element import lattice, volume_points, facet_points
import hdg_workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden', 'stepsizes_table.txt')


@pytest.mark.parametrize('n', [1, 2, 4, 6, 8])
def test_triangle_quadrature_exact(n):
    # int_T xi^a eta^b = a! b! / (a + b + 2)!  (Dirichlet integral)
    P, w = triangle_quadrature(n)
    for a in range(2 * n):
        for b in range(2 * n - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(w * P[:, 0] ** a * P[:, 1] ** b) - exact) < 1e-15


def test_line_quadrature_exact():
    for n in range(1, 9):
        t, w = line_quadrature(n)
        for j in range(2 * n):
            assert abs(np.sum(w * t ** j) - 1.0 / (j + 1)) < 1e-15


def test_quadrature_degrees_cover_forms():
    for k in range(1, 5):
        assert 2 * volume_points(k) - 1 >= 3 * k + 2          # w (Q*.grad) Q
        assert 2 * facet_points(k) - 1 >= 3 * k + 3           # (Q*.n) Q.w on facets


@pytest.mark.parametrize('m', [1, 2, 3, 4, 5])
def test_lagrange_basis(m):
    V = LagrangeTri(m)
    assert np.allclose(V.values(V.nodes), np.eye(V.n), atol=1e-12)
    # reproduces an arbitrary polynomial of degree m and its gradient
    rng = np.random.default_rng(m)
    cf = rng.standard_normal((m + 1, m + 1))
    f = lambda x, y: sum(cf[a, b] * x ** a * y ** b for a in range(m + 1) for b in range(m + 1 - a))
    fx = lambda x, y: sum(cf[a, b] * a * x ** (a - 1) * y ** b for a in range(1, m + 1) for b in range(m + 1 - a))
    P = rng.random((20, 2)) * 0.5
    vals = V.values(P) @ f(V.nodes[:, 0], V.nodes[:, 1])
    assert np.allclose(vals, f(P[:, 0], P[:, 1]), atol=1e-11)
    g = np.einsum('pns,n->ps', V.grads(P), f(V.nodes[:, 0], V.nodes[:, 1]))
    assert np.allclose(g[:, 0], fx(P[:, 0], P[:, 1]), atol=1e-9)
    L = Lagrange1D(m)
    assert np.allclose(L.values(L.nodes), np.eye(m + 1), atol=1e-12)


def _table():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith('#')]
    return [(int(r[0]), float(r[1]), float(r[2]), [int(x) for x in r[3:6]], [int(x) for x in r[6:9]])
            for r in rows]


def test_dof_table_matches_paper():
    for n, h, dt, dg, tr in _table():
        m = Mesh(n)
        # the caption says "truncated", but the printed values are rounded to six decimals
        assert abs(round(math.sqrt(2.0) / n, 6) - h) < 1e-12
        assert abs(round(1.0 / n, 6) - dt) < 1e-12
        for k in (1, 2, 3):
            assert dof_counts(m, k) == (dg[k - 1], tr[k - 1])


@pytest.mark.parametrize('px,py', [(False, False), (True, False), (True, True)])
def test_mesh_geometry(px, py):
    n = 3
    m = Mesh(n, Lx=2.0, Ly=1.5, periodic_x=px, periodic_y=py)
    assert m.ncells == 2 * n * n
    assert m.nfacets == 3 * n * n + (0 if px else n) + (0 if py else n)
    assert np.all(m.detJ > 0)                                  # counter-clockwise cells
    assert abs(0.5 * m.detJ.sum() - 3.0) < 1e-13
    # every cell edge is a facet side with matching endpoints; outward normals
    for c in range(m.ncells):
        for e in range(3):
            f, s = m.cell_facet[c, e], m.cell_side[c, e]
            v1, v2 = m.cell_xy[c, (e + 1) % 3], m.cell_xy[c, (e + 2) % 3]
            ends = {tuple(np.round(m.f_a[f, s], 12)), tuple(np.round(m.f_b[f, s], 12))}
            assert ends == {tuple(np.round(v1, 12)), tuple(np.round(v2, 12))}
            nrm = m.f_normal[f] * (1 if s == 0 else -1)
            mid = 0.5 * (v1 + v2)
            assert np.dot(mid - m.cell_xy[c].mean(axis=0), nrm) > 0
    # divergence theorem per cell: sum of h n over its edges is zero
    tot = np.zeros((m.ncells, 2))
    for c in range(m.ncells):
        for e in range(3):
            f, s = m.cell_facet[c, e], m.cell_side[c, e]
            tot[c] += m.f_h[f] * m.f_normal[f] * (1 if s == 0 else -1)
    assert np.abs(tot).max() < 1e-13
    # periodic facets: both sides, the copies differ by the period
    if px:
        for f in range(m.nH, m.nH + m.nV):
            assert m.f_nsides[f] == 2
    assert (m.f_nsides == 1).sum() == (0 if px else 2 * n) + (0 if py else 2 * n)


def test_workload_nodes_match_oracle_mesh():
    # the shared input generator and the oracle agree on the exchange format
    for n, k in [(2, 1), (3, 3)]:
        m = Mesh(n)
        X = m.cell_points(np.arange(m.ncells), lattice(k + 1))
        assert np.allclose(X, W.cell_nodes(n, k + 1), atol=1e-14)
