"""Convergence pins of the oracle against the exact Taylor-Green solution (Sec. 3.3, 3.4).

The forced Taylor-Green problem of eq. taylor_green_Q0_f has the exact solution
Q = exp(-kappa t) Q0, p = exp(-2 kappa t)(cos 2 pi x + cos 2 pi y)/4 (the printed pressure is
replaced by the one that solves grad p = -(Q.grad)Q; see test_taylor_green_pressure_formula).
Measured rates of the L2 errors at t = T pin the whole oracle (forms, BDM projection, Alg. 1,
final update, pressure reconstruction) against the mathematics: a dropped term, a wrong sign or
weight anywhere breaks the rates.

  * Sec. 3.4's experiment: kappa = 0.5, T = 1, n_t = n (dt = 1/n), with the tableau of order k
    for pressure degree k; the paper observes L2 errors ~ h^k ~ dt^k in velocity and pressure.
    IMEX Euler for k = 1 and ARS(2,2,2) / ARS(3,4,3) for k = 2 / 3 (the paper's SSP2(3,3,2) and
    SSP3(4,3,3) do not fit Alg. 1's form, see the tableau tests).
  * Spatial order at small dt: with dt small enough that the time error is negligible, the
    errors fall as h^{k+1} (pressure degree k, velocity degree k+1).
  * The pressure reconstruction (Sec. 2.7) of the projected Taylor-Green velocity converges to
    the exact pressure.
  * The oracle's L2 projection reproduces its spaces and leaves a residual orthogonal to them.
"""
import numpy as np
import pytest

from oracle import Mesh, HDG, Oracle, TABLEAUS
from oracle.element import lattice, triangle_quadrature
import hdg_workloads as W

KAPPA = 0.5


def l2_error_Q(hdg, Q, fun):
    m = hdg.mesh
    qp, qw = triangle_quadrature(10)
    X = m.cell_points(np.arange(m.ncells), qp)
    ex = np.stack(fun(X[..., 0], X[..., 1]), -1)
    num = np.einsum('qa,cda->cqd', hdg.Vu.values(qp), Q.reshape(m.ncells, 2, hdg.mu))
    return np.sqrt(np.sum(qw[None, :, None] * m.detJ[:, None, None] * (num - ex) ** 2))


def l2_error_p(hdg, p, fun):
    m = hdg.mesh
    qp, qw = triangle_quadrature(10)
    X = m.cell_points(np.arange(m.ncells), qp)
    ex = fun(X[..., 0], X[..., 1])
    num = np.einsum('qb,cb->cq', hdg.Vp.values(qp), p.reshape(m.ncells, hdg.npn))
    return np.sqrt(np.sum(qw[None, :] * m.detJ[:, None] * (num - ex) ** 2))


def forced_taylor_green(n, k, tableau, T, nt):
    """Errors (velocity, pressure) at t = T of the forced Taylor-Green run with nt steps."""
    h = HDG(Mesh(n), k)
    o = Oracle(h)
    dt = T / nt
    Q = h.l2_project(W.taylor_green, 0)
    F0 = o.M @ Q                                     # dual vector of f / (-kappa e^{-kappa t})
    forcing = lambda t: -KAPPA * np.exp(-KAPPA * t) * F0
    _, p, lam = o.reconstruct_pressure(Q, forcing(0.0))
    tab = TABLEAUS[tableau]()
    for s in range(nt):
        Q, p, lam = o.imex_step(tab, dt, s * dt, Q, p, lam, forcing=forcing)
    eQ = l2_error_Q(h, Q, lambda x, y: tuple(np.exp(-KAPPA * T) * np.array(W.taylor_green(x, y))))
    ep = l2_error_p(h, p, lambda x, y: np.exp(-2 * KAPPA * T) * W.taylor_green_pressure(x, y))
    return eQ, ep


@pytest.mark.parametrize('k,tableau,meshes', [(1, 'IMEX_EULER', (8, 16)), (2, 'ARS222', (8, 16)),
                                              (3, 'ARS343', (4, 8))])
def test_taylor_green_kappa_convergence_rate_k(k, tableau, meshes):
    # Sec. 3.4: kappa = 0.5, T = 1, n_t = n; observed rates ~ k in velocity and pressure
    e = [forced_taylor_green(n, k, tableau, 1.0, n) for n in meshes]
    rate_Q = np.log2(e[0][0] / e[1][0])
    rate_p = np.log2(e[0][1] / e[1][1])
    assert rate_Q > k - 0.2 and rate_p > k - 0.2, (rate_Q, rate_p)
    assert e[1][0] < 5e-3 and e[1][1] < 5e-3


@pytest.mark.parametrize('k', [1, 2, 3])
def test_spatial_order_k_plus_1_at_small_dt(k):
    # dt = 0.005 with the third-order ARS(3,4,3): the time error is far below the space error;
    # velocity (degree k+1) and pressure (degree k) errors fall as h^{k+1}
    e = [forced_taylor_green(n, k, 'ARS343', 0.02, 4) for n in (4, 8)]
    rate_Q = np.log2(e[0][0] / e[1][0])
    rate_p = np.log2(e[0][1] / e[1][1])
    assert rate_Q > k + 0.6 and rate_p > k + 0.6, (rate_Q, rate_p)


@pytest.mark.parametrize('k', [1, 2])
def test_pressure_reconstruction_converges_to_taylor_green_pressure(k):
    # Sec. 2.7 applied to the projected steady vortex: p -> (cos 2 pi x + cos 2 pi y)/4
    errs = []
    for n in (4, 8, 16):
        h = HDG(Mesh(n), k)
        o = Oracle(h)
        _, p, _ = o.reconstruct_pressure(h.l2_project(W.taylor_green, 0))
        errs.append(l2_error_p(h, p, W.taylor_green_pressure))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > k + 0.6, rates


@pytest.mark.parametrize('k', [1, 2, 3, 4])
def test_l2_projection_reproduces_space_and_is_orthogonal(k):
    h = HDG(Mesh(3, Lx=2.0), k)
    m = h.mesh
    # reproduces polynomials of the space: nodal values equal the polynomial at the lattice
    poly = lambda x, y: (x ** (k + 1) - 2 * x * y + 1.0, y ** k * x - 0.5 * y)
    X = m.cell_points(np.arange(m.ncells), lattice(k + 1))
    Q = h.l2_project(poly, 0)
    ex = np.stack(poly(X[..., 0], X[..., 1]), 1).reshape(-1)
    assert np.abs(Q - ex).max() < 1e-13 * np.abs(ex).max() * 10 ** k
    Xp = m.cell_points(np.arange(m.ncells), lattice(k))
    pp = h.l2_project(lambda x, y: x ** k - y + 0.25, 1)
    assert np.abs(pp - (Xp[..., 0] ** k - Xp[..., 1] + 0.25).reshape(-1)).max() < 1e-12
    # the residual of smooth data is orthogonal to the space (checked with another rule)
    f = lambda x, y: np.exp(x) * np.sin(3 * y)
    pf = h.l2_project(f, 1, npts=k + 8)
    qp, qw = triangle_quadrature(k + 9)
    Xq = m.cell_points(np.arange(m.ncells), qp)
    B = h.Vp.values(qp)
    r = f(Xq[..., 0], Xq[..., 1]) - np.einsum('qb,cb->cq', B, pf.reshape(m.ncells, -1))
    assert np.abs(np.einsum('q,qb,cq->cb', qw, B, r)).max() < 1e-11
