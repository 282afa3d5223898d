"""Pins of the oracle's tracer advection (App. B): the continuous projection P_CG and the upwind
DG form a(chi, q, U), against what the mathematics fixes.

  * P_CG reproduces continuous polynomials of degree k+1, returns a continuous field (one value
    per lattice point) and is idempotent;
  * a(., 1, U) = 0 on a doubly periodic mesh for any continuous U (constants are transported
    unchanged: the facet flux of a constant cancels the volume term cell by cell);
  * a(1, q, U) = 0 for a constant U on a doubly periodic mesh (the tracer's mass is conserved);
  * upwinding: for q = 1 on one cell, 0 elsewhere, and a constant U, a(chi_K2, q, U) =
    h_F max(U.n1, 0) on the neighbour K2 across facet F (n1 outward of K1), and
    a(chi_K1, q, U) = -sum over K1's interior edges of h_e max(U.n_e, 0);
  * for a linear q and a constant U, M^-1 a(q) = -U.grad q exactly on the cells away from walls;
  * a smooth tracer translated by a constant U on a periodic mesh converges at rate k+1.
"""
import numpy as np
import pytest

from oracle import Mesh, HDG, Tracer, TABLEAUS
from oracle.element import lattice


def const_on(hdg, cell, value=1.0):
    q = np.zeros((hdg.mesh.ncells, hdg.npn))
    q[cell] = value
    return q.reshape(-1)


def const_velocity(hdg, U):
    Q = np.zeros((hdg.mesh.ncells, 2, hdg.mu))
    Q[:, 0], Q[:, 1] = U
    return Q.reshape(-1)


@pytest.mark.parametrize('k', [1, 2, 3, 4])
def test_cg_projection_reproduces_continuous_polynomials_and_is_continuous(k):
    h = HDG(Mesh(3, Lx=2.0), k)
    T = Tracer(h)
    m = h.mesh
    X = m.cell_points(np.arange(m.ncells), lattice(k + 1))
    f = lambda x, y: (x ** (k + 1) - 2 * x * y + 0.5, y ** k * x - y ** 2)
    Q = np.stack(f(X[..., 0], X[..., 1]), 1).reshape(-1)
    assert np.abs(T.cg_project(Q) - Q).max() < 1e-12 * 10 ** k
    rng = np.random.default_rng(k)
    U = T.cg_project(rng.standard_normal(h.nQ)).reshape(m.ncells, 2, h.mu)
    for d in range(2):                              # one value per continuous point
        vals = {}
        for c in range(m.ncells):
            for a in range(h.mu):
                vals.setdefault(T.gid[c, a], []).append(U[c, d, a])
        assert max(np.ptp(v) for v in vals.values()) < 1e-13
    assert np.abs(T.cg_project(U.reshape(-1)) - U.reshape(-1)).max() < 1e-13


@pytest.mark.parametrize('k', [1, 2, 3])
def test_constants_transported_and_mass_conserved_on_periodic_mesh(k):
    h = HDG(Mesh(4, periodic_x=True, periodic_y=True), k)
    T = Tracer(h)
    rng = np.random.default_rng(10 + k)
    U = T.cg_project(rng.standard_normal(h.nQ))
    ones = np.ones(h.nP)                            # the constant 1 (Lagrange coefficients)
    assert np.abs(T.form(U) @ ones).max() < 1e-13
    A = T.form(const_velocity(h, (0.7, -0.4)))
    assert np.abs(ones @ A).max() < 1e-13


@pytest.mark.parametrize('k', [1, 3])
def test_upwind_flux_closed_form(k):
    m = Mesh(3, Lx=2.0, Ly=1.0)
    h = HDG(m, k)
    T = Tracer(h)
    for U in ((0.8, 0.3), (-0.5, 1.1)):
        A = T.form(const_velocity(h, U))
        U = np.array(U)
        for f in np.nonzero(m.interior)[0][::2]:
            K1, K2 = m.f_cell[f]
            n1 = m.f_normal[f]
            got = const_on(h, K2) @ (A @ const_on(h, K1))
            assert abs(got - m.f_h[f] * max(U @ n1, 0.0)) < 1e-13
        for K1 in range(0, m.ncells, 3):
            want = 0.0
            for e in range(3):
                f = m.cell_facet[K1, e]
                if m.interior[f]:
                    ne = m.f_normal[f] * (1 if m.cell_side[K1, e] == 0 else -1)
                    want -= m.f_h[f] * max(U @ ne, 0.0)
            got = const_on(h, K1) @ (A @ const_on(h, K1))
            assert abs(got - want) < 1e-13


@pytest.mark.parametrize('k', [1, 2])
def test_linear_tracer_exact_away_from_walls(k):
    n = 4
    m = Mesh(n)
    h = HDG(m, k)
    T = Tracer(h)
    U = np.array([0.6, -0.9])
    X = m.cell_points(np.arange(m.ncells), lattice(k))
    q = (2.0 * X[..., 0] - 3.0 * X[..., 1] + 1.0).reshape(-1)
    dq = T.rhs(q, const_velocity(h, U)).reshape(m.ncells, h.npn)
    interior = [c for c in range(m.ncells) if all(m.interior[m.cell_facet[c, e]] for e in range(3))
                and all(all(m.interior[m.cell_facet[o, e]] for e in range(3)) for o in
                        [m.f_cell[m.cell_facet[c, e], 1 - m.cell_side[c, e]] for e in range(3)])]
    assert len(interior) > 0
    want = -(U[0] * 2.0 - U[1] * 3.0)
    assert np.abs(dq[interior] - want).max() < 1e-12


@pytest.mark.parametrize('k', [1, 2])
def test_translated_tracer_converges_at_rate_k_plus_1(k):
    from oracle.element import triangle_quadrature
    U = np.array([1.0, 0.5])
    f = lambda x, y: np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    tab = TABLEAUS['ARS343']()
    qp, qw = triangle_quadrature(k + 5)
    errs = []
    for n in (8, 16):
        m = Mesh(n, periodic_x=True, periodic_y=True)
        h = HDG(m, k)
        T = Tracer(h)
        Qc = const_velocity(h, U)
        X = m.cell_points(np.arange(m.ncells), lattice(k))
        q = f(X[..., 0], X[..., 1]).reshape(-1)
        dt, nt = 0.005, 8
        for s in range(nt):
            q = T.step(tab, dt, q, [Qc] * tab.s)
        t = dt * nt
        Xq = m.cell_points(np.arange(m.ncells), qp)
        num = np.einsum('qb,cb->cq', h.Vp.values(qp), q.reshape(m.ncells, h.npn))
        ex = f(Xq[..., 0] - U[0] * t, Xq[..., 1] - U[1] * t)
        errs.append(np.sqrt(np.sum(qw[None] * m.detJ[:, None] * (num - ex) ** 2)))
    rate = np.log2(errs[0] / errs[1])
    assert rate > k + 0.5, (errs, rate)
