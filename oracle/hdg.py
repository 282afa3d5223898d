"""The hybridised DG discretisation of Sec. 2 as global sparse matrices (FP64, plain SciPy).

TEST INFRASTRUCTURE ONLY (see oracle/element.py).

Unknowns: Q in V_Q = [DG_{k+1}]^2, p in V_p = DG_k, lambda in V_trace = P_k on every facet
(Sec. 2.2 eq. function_spaces, Sec. 2.4). Coefficients are nodal values (oracle/element.py).
Global numbering: Q index (K*2 + d)*mu + a (cell K, component d, node a); p index K*n_p + b;
lambda index F*(k+1) + j.

The forms follow Sec. 2.3-2.4 term by term, summing over interior and boundary facets as the
paper writes them (the two sides of an interior facet are the mesh's side 0 = "+" and
side 1 = "-"):

  M:  (w . Q)_Omega
  G:  g(w, p, lambda) = (p div w) - sum_int <[[w.n]] lambda> - sum_bdy <(w.n) lambda>
  B, C:  Gamma(psi, mu, Q, p, lambda) = (psi div Q) + 2 sum_int <{tau (p-lambda) psi}>
            + sum_bdy <tau (p-lambda) psi> + sum_int <([[Q.n]] + 2 tau {p-lambda}) mu>
            + sum_bdy <(Q.n + tau (p-lambda)) mu>
        split as Gamma = B Q + C (p, lambda); rows are (psi, mu) stacked.
  F(Q*):  f^impl(w, Q, Q*) of eq. f_impl (advection volume term, central facet term,
          alpha/h_F normal-jump penalty on interior and boundary facets, delta_up upwind term).

On interior facets Q*.n+ is read as {Q*}.n+: Q* = P(Q) has a single-valued normal component
(BDM), so the average only removes rounding differences between the two sides.
"""
import numpy as np
import scipy.sparse as sp

from .element import (LagrangeTri, Lagrange1D, triangle_quadrature, line_quadrature,
                       volume_points, facet_points)


def _coo(rows, cols, vals, shape):
    rows, cols, vals = np.broadcast_arrays(rows, cols, vals)
    return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=shape).tocsr()


class HDG:
    def __init__(self, mesh, k, alpha=1.0, tau=1.0, delta_up=1.0):
        self.mesh, self.k = mesh, k
        self.alpha, self.tau, self.delta_up = float(alpha), float(tau), float(delta_up)
        self.Vu, self.Vp, self.Vt = LagrangeTri(k + 1), LagrangeTri(k), Lagrange1D(k)
        self.mu, self.npn, self.nt = self.Vu.n, self.Vp.n, self.Vt.n
        self.nu = 2 * self.mu
        nc, nf = mesh.ncells, mesh.nfacets
        self.nQ, self.nP, self.nL = nc * self.nu, nc * self.npn, nf * self.nt
        self.qp, self.qw = triangle_quadrature(volume_points(k))
        self.tq, self.tw = line_quadrature(facet_points(k))
        self.phi = self.Vu.values(self.qp)            # (nq, mu)
        self.gphi = self.Vu.grads(self.qp)            # (nq, mu, 2) reference gradients
        self.psi = self.Vp.values(self.qp)            # (nq, npn)
        self.mut = self.Vt.values(self.tq)            # (nfq, nt)
        self._static = None

    # ----------------------------------------------------------------- index helpers
    def iQ(self, cells):
        return np.asarray(cells)[:, None] * self.nu + np.arange(self.nu)[None, :]

    def iP(self, cells):
        return np.asarray(cells)[:, None] * self.npn + np.arange(self.npn)[None, :]

    def iL(self, facets):
        return np.asarray(facets)[:, None] * self.nt + np.arange(self.nt)[None, :]

    # ----------------------------------------------------------------- geometry helpers
    def grad_phys(self, cells):
        """Physical gradients of the velocity basis at the volume points: (c, nq, mu, 2)."""
        return np.einsum('qar,cre->cqae', self.gphi, self.mesh.Jinv[cells])

    def side_values(self, facets, side):
        """Velocity and pressure basis of the side cell at the facet points: (f, nfq, .)."""
        m = self.mesh
        cells = m.f_cell[facets, side]
        X = m.facet_points(facets, side, self.tq)
        xi = m.to_reference(cells, X)
        return cells, self.Vu.values(xi), self.Vp.values(xi)

    def side_normal(self, facets, side):
        n = self.mesh.f_normal[facets]
        return n if side == 0 else -n

    def eval_Q_at_facet(self, Q, facets, side):
        """Vector field Q (nodal, global) at the facet points of a side: (f, nfq, 2)."""
        cells, ph, _ = self.side_values(facets, side)
        q = Q[self.iQ(cells)].reshape(len(facets), 2, self.mu)
        return np.einsum('fqa,fda->fqd', ph, q)

    # ----------------------------------------------------------------- cell blocks
    def cell_mass(self, cells):
        """(phi_a, phi_b)_K for one component: (c, mu, mu)."""
        m = np.einsum('q,qa,qb->ab', self.qw, self.phi, self.phi)
        return self.mesh.detJ[cells][:, None, None] * m[None]

    def cell_div(self, cells):
        """(psi_b, div(phi_a e_d))_K: (c, npn, nu) with column d*mu + a."""
        g = self.grad_phys(cells)
        D = np.einsum('q,qb,cqad->cbda', self.qw, self.psi, g)
        D *= self.mesh.detJ[cells][:, None, None, None]
        return D.reshape(len(cells), self.npn, self.nu)

    def cell_advection(self, cells, Qstar):
        """-(w . (Q* . grad) Q)_K for w = phi_a e_d, Q = phi_b e_d: (c, mu, mu)."""
        g = self.grad_phys(cells)
        qs = Qstar[self.iQ(cells)].reshape(len(cells), 2, self.mu)
        qsq = np.einsum('qa,cda->cqd', self.phi, qs)                 # Q* at points
        conv = np.einsum('cqd,cqbd->cqb', qsq, g)                     # Q* . grad phi_b
        A = -np.einsum('q,qa,cqb->cab', self.qw, self.phi, conv)
        return A * self.mesh.detJ[cells][:, None, None]

    # ----------------------------------------------------------------- global static forms
    def static(self):
        """M, G, B, C as CSR matrices (independent of the state)."""
        if self._static is not None:
            return self._static
        m, mu, nu, npn, nt = self.mesh, self.mu, self.nu, self.npn, self.nt
        cells = np.arange(m.ncells)
        nY = self.nP + self.nL
        # mass (w . Q): component-diagonal
        Ms = self.cell_mass(cells)
        Mfull = np.zeros((m.ncells, nu, nu))
        Mfull[:, :mu, :mu] = Ms
        Mfull[:, mu:, mu:] = Ms
        iq = self.iQ(cells)
        M = _coo(iq[:, :, None], iq[:, None, :], Mfull, (self.nQ, self.nQ))
        # volume parts: g: (p div w); Gamma: (psi div Q)
        D = self.cell_div(cells)
        ip = self.iP(cells)
        G = _coo(iq[:, :, None], ip[:, None, :], np.transpose(D, (0, 2, 1)), (self.nQ, nY))
        B = _coo(ip[:, :, None], iq[:, None, :], D, (nY, self.nQ))
        C = sp.csr_matrix((nY, nY))
        tau, tw = self.tau, self.tw
        for interior in (True, False):
            facets = np.nonzero(m.interior == interior)[0]
            if len(facets) == 0:
                continue
            h = m.f_h[facets]
            il = self.nP + self.iL(facets)
            nsides = 2 if interior else 1
            for s in range(nsides):
                c, ph, ps = self.side_values(facets, s)
                n = self.side_normal(facets, s)
                iqs, ips = self.iQ(c), self.iP(c)
                # <(w_s . n_s) mu_j>: (f, nu, nt)
                wn = np.einsum('q,fqa,fd,qj->fdaj', tw, ph, n, self.mut).reshape(len(facets), nu, nt)
                wn *= h[:, None, None]
                # g: - sum <[[w.n]] lambda>  (jump = sum over sides of w_s.n_s; boundary: w.n)
                G = G + _coo(iqs[:, :, None], il[:, None, :], -wn, (self.nQ, nY))
                # Gamma, mu-row: <[[Q.n]] mu> (boundary: <(Q.n) mu>)
                B = B + _coo(il[:, :, None], iqs[:, None, :], np.transpose(wn, (0, 2, 1)), (nY, self.nQ))
                # Gamma, tau terms. psi-row: tau <(p_s - lambda) psi_s> per side
                # (= 2 <{tau (p-lambda) psi}> on interior facets); mu-row: tau (p_s - lambda) per
                # side (= 2 tau {p - lambda} on interior facets).
                pp = tau * h[:, None, None] * np.einsum('q,fqa,fqb->fab', tw, ps, ps)
                pl = tau * h[:, None, None] * np.einsum('q,fqa,qj->faj', tw, ps, self.mut)
                ll = tau * h[:, None, None] * np.einsum('q,qi,qj->ij', tw, self.mut, self.mut)[None]
                C = C + _coo(ips[:, :, None], ips[:, None, :], pp, (nY, nY))
                C = C + _coo(ips[:, :, None], il[:, None, :], -pl, (nY, nY))
                C = C + _coo(il[:, :, None], ips[:, None, :], np.transpose(pl, (0, 2, 1)), (nY, nY))
                C = C + _coo(il[:, :, None], il[:, None, :], -ll * np.ones((len(facets), 1, 1)), (nY, nY))
        self._static = (M, G.tocsr(), B.tocsr(), C.tocsr())
        return self._static

    # ----------------------------------------------------------------- f^impl
    def fimpl(self, Qstar, chunk=4096):
        """f^impl(w, Q, Q*) = w^T F Q as a CSR matrix (eq. f_impl)."""
        m, mu, nu = self.mesh, self.mu, self.nu
        al, dup, tw = self.alpha, self.delta_up, self.tw
        cells = np.arange(m.ncells)
        A = self.cell_advection(cells, Qstar)
        Af = np.zeros((m.ncells, nu, nu))
        Af[:, :mu, :mu] = A
        Af[:, mu:, mu:] = A
        iq = self.iQ(cells)
        F = _coo(iq[:, :, None], iq[:, None, :], Af, (self.nQ, self.nQ))
        sigma = (1.0, -1.0)
        for interior in (True, False):
            allf = np.nonzero(m.interior == interior)[0]
            for c0 in range(0, len(allf), chunk):
                facets = allf[c0:c0 + chunk]
                nfc = len(facets)
                h = m.f_h[facets]
                nsides = 2 if interior else 1
                vals = [self.side_values(facets, s) for s in range(nsides)]
                nrm = [self.side_normal(facets, s) for s in range(nsides)]
                if interior:
                    qs0 = self.eval_Q_at_facet(Qstar, facets, 0)
                    qs1 = self.eval_Q_at_facet(Qstar, facets, 1)
                    qsn = 0.5 * np.einsum('fqd,fd->fq', qs0 + qs1, m.f_normal[facets])  # {Q*}.n+
                for s in range(nsides):          # test side
                    cs, phs, _ = vals[s]
                    for t in range(nsides):      # trial side
                        ct, pht, _ = vals[t]
                        blk = np.zeros((nfc, nu, nu))
                        # penalty: -alpha h^-1 <[[Q.n]][[w.n]]> (boundary: (Q.n)(w.n)); ds = h dt
                        pen = -al * np.einsum('q,fqa,fqb->fab', tw, phs, pht)
                        for d in range(2):
                            for e in range(2):
                                blk[:, d * mu:(d + 1) * mu, e * mu:(e + 1) * mu] += \
                                    (nrm[s][:, d] * nrm[t][:, e])[:, None, None] * pen
                        if interior:
                            # central: <(Q*.n+)(Q+ - Q-) . {w}>
                            cen = 0.5 * sigma[t] * h[:, None, None] * \
                                np.einsum('q,fq,fqa,fqb->fab', tw, qsn, phs, pht)
                            # upwind: -delta <|Q*.n+| (Q+ - Q-) . (w+ - w-)>
                            upw = -dup * sigma[s] * sigma[t] * h[:, None, None] * \
                                np.einsum('q,fq,fqa,fqb->fab', tw, np.abs(qsn), phs, pht)
                            for d in range(2):
                                blk[:, d * mu:(d + 1) * mu, d * mu:(d + 1) * mu] += cen + upw
                        F = F + _coo(self.iQ(cs)[:, :, None], self.iQ(ct)[:, None, :], blk,
                                     (self.nQ, self.nQ))
        return F.tocsr()

    # ----------------------------------------------------------------- L2 projection
    def l2_project(self, fun, field, npts=None):
        """L2 projection, cell by cell, of fun(x, y) onto V_Q (field 0; fun returns the pair of
        components) or V_p (field 1): the coefficients c of each cell solve
        (phi_a, phi_b)_K c_b = (f, phi_a)_K, the integrals taken by the collapsed Gauss rule with
        npts x npts points (default k + 4: exact to degree 2k + 7, i.e. the degree 2(k+1)+4 that
        non-polynomial data is projected with). Returns the nodal coefficients in the exchange
        layout ([cell][2][mu] or [cell][n_p], flattened)."""
        m = self.mesh
        qp, qw = triangle_quadrature(npts or self.k + 4)
        X = m.cell_points(np.arange(m.ncells), qp)                 # (c, nq, 2)
        V = self.Vu if field == 0 else self.Vp
        B = V.values(qp)                                           # (nq, nb)
        mass = np.einsum('q,qa,qb->ab', qw, B, B)                  # detJ cancels on both sides
        if field == 0:
            fx, fy = fun(X[..., 0], X[..., 1])
            f = np.stack([fx, fy], axis=1)                         # (c, 2, nq)
            rhs = np.einsum('q,qa,cdq->cda', qw, B, f)
        else:
            rhs = np.einsum('q,qa,cq->ca', qw, B, fun(X[..., 0], X[..., 1]))
        return np.linalg.solve(mass, rhs[..., None])[..., 0].reshape(-1)

    # ----------------------------------------------------------------- helpers on fields
    def mean_p(self, p):
        """(p)_Omega / |Omega| (the reference triangle has area 1/2)."""
        return self.p_integral_vector() @ p / (0.5 * self.mesh.detJ.sum())

    def p_integral_vector(self):
        """e with e . p = (p)_Omega."""
        m = self.mesh
        w = np.einsum('q,qb->b', self.qw, self.psi)
        return (m.detJ[:, None] * w[None, :]).ravel()
