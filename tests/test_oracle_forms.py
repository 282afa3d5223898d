"""Pins of the oracle's forms g, Gamma, f^impl and of the BDM projection (Sec. 2.3-2.4).

Each check is a consequence of the printed definitions and of calculus, not a re-typing of
them: the divergence theorem gives the kernels of g and Gamma, integration by parts gives the
skew-symmetry of the central advection term, the jump/average structure gives the +/- swap
invariance, and the BDM interpolant reproduces BDM fields."""
import numpy as np
import pytest

from oracle import Mesh, HDG, Oracle, bdm_project
from oracle.element import lattice

MESHES = [(False, False), (True, False), (True, True)]


def interp(hdg, fun):
    m = hdg.mesh
    X = m.cell_points(np.arange(m.ncells), lattice(hdg.k + 1))
    return np.stack(fun(X[..., 0], X[..., 1]), 1).reshape(-1)


def poly_stream(x, y):
    # curl of psi = x(1-x) y(1-y): a cubic, divergence-free field with n.Q = 0 on the walls
    return x * (1 - x) * (1 - 2 * y), -(1 - 2 * x) * y * (1 - y)


@pytest.mark.parametrize('per', MESHES)
@pytest.mark.parametrize('k', [1, 2, 3, 4])
def test_kernels_of_g_and_gamma(per, k):
    h = HDG(Mesh(2, periodic_x=per[0], periodic_y=per[1]), k)
    M, G, B, C = h.static()
    ones = np.ones(h.nP + h.nL)
    # g(w, 1, 1) = int div w - oint w.n = 0 ; Gamma(., ., 0, 1, 1) = 0
    assert np.abs(G @ ones).max() < 1e-13
    assert np.abs(C @ ones).max() < 1e-13
    # Gamma(1, -1, Q, p, lambda) = int div Q - oint Q.n + tau oint(p-l) - tau oint(p-l) = 0
    left = np.concatenate([np.ones(h.nP), -np.ones(h.nL)])
    assert np.abs(left @ B).max() < 1e-13
    assert np.abs(left @ C).max() < 1e-13
    # the pressure part of g is the adjoint of the divergence part of Gamma; the trace part of g
    # is minus the adjoint of the trace part of Gamma
    Gd, Bd = G.toarray(), B.toarray()
    assert np.abs(Bd[:h.nP] - Gd[:, :h.nP].T).max() < 1e-14
    assert np.abs(Bd[h.nP:] + Gd[:, h.nP:].T).max() < 1e-14
    # mass matrix: symmetric positive definite, total mass = area * 2 components
    assert np.abs((M - M.T).toarray()).max() < 1e-15
    assert abs(M.sum() - 2.0) < 1e-12


@pytest.mark.parametrize('per', MESHES)
def test_forms_invariant_under_side_swap(per):
    m = Mesh(3, periodic_x=per[0], periodic_y=per[1])
    for k in (1, 3):
        h, hs = HDG(m, k), HDG(m.swapped(), k)
        rng = np.random.default_rng(k)
        Qs = bdm_project(h, rng.standard_normal(h.nQ))
        assert np.abs(bdm_project(hs, Qs) - bdm_project(h, Qs)).max() < 1e-12
        for A, As in zip(h.static(), hs.static()):
            assert abs(A - As).max() < 1e-14
        assert abs(h.fimpl(Qs) - hs.fimpl(Qs)).max() < 1e-13


@pytest.mark.parametrize('k', [2, 3, 4])
def test_central_advection_skew_and_dissipation(k):
    m = Mesh(3)
    h = HDG(m, k)
    Qs = bdm_project(h, interp(h, poly_stream))
    central = HDG(m, k, alpha=0.0, delta_up=0.0).fimpl(Qs).toarray()
    full = h.fimpl(Qs).toarray()
    # volume + central facet term is skew when Q* is divergence free, normal-continuous and
    # tangential on the walls (integration by parts)
    assert np.abs(central + central.T).max() < 1e-12 * np.abs(central).max()
    # penalty and upwind terms are symmetric and non-positive
    diss = full - central
    assert np.abs(diss - diss.T).max() < 1e-13
    assert np.linalg.eigvalsh(0.5 * (diss + diss.T)).max() < 1e-12
    # with delta_up > 0 the upwind part is strictly present
    no_up = HDG(m, k, delta_up=0.0).fimpl(Qs).toarray()
    assert np.abs(full - no_up).max() > 1e-3


@pytest.mark.parametrize('k', [1, 2, 3, 4])
def test_advection_of_constant_and_linear_fields(k):
    # f^impl(w, Q, Q*) for Q constant: only the boundary penalty acts (jumps vanish, grad Q = 0);
    # on a doubly periodic mesh it vanishes identically
    m = Mesh(2, periodic_x=True, periodic_y=True)
    h = HDG(m, k)
    rng = np.random.default_rng(0)
    Qs = bdm_project(h, rng.standard_normal(h.nQ))
    Qc = interp(h, lambda x, y: (0 * x + 1.3, 0 * x - 0.4))
    assert np.abs(h.fimpl(Qs) @ Qc).max() < 1e-12
    # volume term against a closed form: Q = (x, 0), Q* = (1, 0) constant, walls off:
    # -(w.(Q*.grad)Q) = -int w_x, penalty/central/upwind vanish for continuous Q on a
    # doubly periodic mesh only if Q is periodic, so check the cell term directly
    Qs1 = interp(h, lambda x, y: (0 * x + 1.0, 0 * x))
    A = h.cell_advection(np.arange(m.ncells), Qs1)               # (c, mu, mu)
    X = m.cell_points(np.arange(m.ncells), lattice(k + 1))
    lin = X[..., 0]
    M1 = h.cell_mass(np.arange(m.ncells))
    got = np.einsum('cab,cb->ca', A, lin)
    assert np.allclose(got, -M1.sum(axis=2), atol=1e-13)


@pytest.mark.parametrize('k', [2, 3, 4])
def test_bdm_reproduces_bdm0_fields(k):
    h = HDG(Mesh(3), k)
    Q = interp(h, poly_stream)
    assert np.abs(bdm_project(h, Q) - Q).max() < 1e-12


@pytest.mark.parametrize('per', MESHES)
@pytest.mark.parametrize('k', [1, 2, 3, 4])
def test_bdm_normal_continuity_and_moments(per, k):
    m = Mesh(3, periodic_x=per[0], periodic_y=per[1])
    h = HDG(m, k)
    rng = np.random.default_rng(7)
    Q = rng.standard_normal(h.nQ)
    Qs = bdm_project(h, Q)
    it = np.nonzero(m.interior)[0]
    a, b = h.eval_Q_at_facet(Qs, it, 0), h.eval_Q_at_facet(Qs, it, 1)
    jump = np.einsum('fqd,fd->fq', a - b, m.f_normal[it])
    assert np.abs(jump).max() < 1e-11                   # single-valued normal component
    assert np.abs(a - b).max() > 1e-2                   # (the tangential part is not)
    bd = np.nonzero(~m.interior)[0]
    if len(bd):
        wall = np.einsum('fqd,fd->fq', h.eval_Q_at_facet(Qs, bd, 0), m.f_normal[bd])
        assert np.abs(wall).max() < 1e-11               # n.Q* = 0 on walls (BDM^0)
    # commuting property: (div P(Q), psi)_K = -(Q, grad psi)_K + <{Q}.n, psi>_dK for psi in P_k,
    # i.e. summed against the pressure basis: B_p P(Q) = Gamma-like weak divergence of Q
    M, G, B, C = h.static()
    div_star = (B @ Qs)[:h.nP]
    # weak divergence of Q with averaged normal traces: (psi div Q) + <psi ({Q} - Q_K).n>
    Qavg_flux = np.zeros(h.nP)
    for s in (0, 1):
        for f in range(m.nfacets):
            if s == 1 and not m.interior[f]:
                continue
            c, ph, ps = h.side_values(np.array([f]), s)
            n = h.side_normal(np.array([f]), s)[0]
            qK = h.eval_Q_at_facet(Q, np.array([f]), s)[0]
            if m.interior[f]:
                qavg = 0.5 * (h.eval_Q_at_facet(Q, np.array([f]), 0)[0] + h.eval_Q_at_facet(Q, np.array([f]), 1)[0])
            else:
                qavg = 0.0 * qK
            val = np.einsum('q,qd,d,qb->b', h.tw, qavg - qK, n, ps[0]) * m.f_h[f]
            Qavg_flux[h.iP(c)[0]] += val
    expect = (B @ Q)[:h.nP] + Qavg_flux
    assert np.abs(div_star - expect).max() < 1e-11 * max(1.0, np.abs(expect).max())


def test_trace_schur_complement_semidefinite_with_constant_kernel():
    for per in MESHES:
        for k in (1, 2, 4):
            h = HDG(Mesh(2, periodic_x=per[0], periodic_y=per[1]), k)
            o = Oracle(h)
            rng = np.random.default_rng(1)
            for c in (1e-3, 1.0):
                *_, S = o.condensed_mixed_solve(c, rng.standard_normal(h.nQ), np.zeros(o.nY))
                S = S.toarray()
                assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()
                ev = np.linalg.eigvalsh(-S)        # the mu-row sign makes S negative semidefinite
                assert abs(ev[0]) < 1e-10 * ev[-1] and ev[1] > 1e-8 * ev[-1]
                assert np.abs(S @ np.ones(h.nL)).max() < 1e-11 * np.abs(S).max()


def _const_field(h, cell, vec):
    """Nodal velocity that is the constant vector vec on one cell and zero elsewhere."""
    Q = np.zeros((h.mesh.ncells, 2, h.mu))
    Q[cell, 0, :], Q[cell, 1, :] = vec
    return Q.reshape(-1)


@pytest.mark.parametrize('per', MESHES)
@pytest.mark.parametrize('k', [1, 3])
def test_fimpl_penalty_and_upwind_weights_closed_form(per, k):
    # eq. f_impl with Q, w constant on single cells and a constant advecting velocity u: the volume
    # term vanishes and each facet integral is its constant integrand times |F| = h_F, so
    #   penalty  -alpha h_F^-1 <[[Q.n]][[w.n]]>  -> -alpha [[Q.n]][[w.n]]        (no h left)
    #   central  <(u.n+)(Q+ - Q-).{w}>           ->  h_F (u.n+)(Q+ - Q-).{w}
    #   upwind   -delta <|u.n+|(Q+ - Q-).(w+ - w-)> -> -delta h_F |u.n+|(Q+ - Q-).(w+ - w-)
    # For Q = a on K1, w = b on its neighbour K2 across F (n1 = outward normal of K1 on F):
    #   w^T F Q = alpha (a.n1)(b.n1) + h_F (u.n1)(a.b)/2 + delta h_F |u.n1| (a.b)
    # and for w = b on K1 itself (sum over K1's facets e, walls included in the penalty only):
    #   w^T F Q = -alpha sum_e (a.n_e)(b.n_e) + sum_{e interior} h_e ((u.n_e)/2 - delta |u.n_e|)(a.b)
    m = Mesh(3, Lx=2.0, Ly=1.0, periodic_x=per[0], periodic_y=per[1])   # facets of three lengths
    a, b, u = np.array([0.7, -1.3]), np.array([-0.4, 0.9]), np.array([1.1, 0.35])
    for alpha, delta in ((1.0, 0.0), (0.0, 1.0), (2.5, 0.6)):
        h = HDG(m, k, alpha=alpha, delta_up=delta)
        Qs = np.tile(np.repeat(u, h.mu), m.ncells)             # constant advecting velocity
        F = h.fimpl(Qs)
        for f in np.nonzero(m.interior)[0][::3]:
            K1, K2 = m.f_cell[f]
            n1, hf = m.f_normal[f], m.f_h[f]                   # outward from side 0 = K1
            got = _const_field(h, K2, b) @ (F @ _const_field(h, K1, a))
            want = alpha * (a @ n1) * (b @ n1) + hf * (u @ n1) * (a @ b) / 2 + delta * hf * abs(u @ n1) * (a @ b)
            assert abs(got - want) < 1e-12 * (1 + abs(want)), (f, got, want)
        for K1 in range(0, m.ncells, 5):
            want = 0.0
            for e in range(3):
                f = m.cell_facet[K1, e]
                ne = m.f_normal[f] * (1 if m.cell_side[K1, e] == 0 else -1)
                want -= alpha * (a @ ne) * (b @ ne)
                if m.interior[f]:
                    want += m.f_h[f] * ((u @ ne) / 2 - delta * abs(u @ ne)) * (a @ b)
            got = _const_field(h, K1, b) @ (F @ _const_field(h, K1, a))
            assert abs(got - want) < 1e-12 * (1 + abs(want)), (K1, got, want)
