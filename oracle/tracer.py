"""Passive tracer advection of App. B (explicit upwind DG), FP64, plain SciPy.

TEST INFRASTRUCTURE ONLY (see oracle/element.py).

  * P_CG: the L2 projection of a DG velocity (degree k+1) onto CG_{k+1} = DG_{k+1} cap C^0, a
    global mass-matrix solve. The continuous space is numbered by the points of the equispaced
    degree-(k+1) lattices of the cells, identified by their physical position (periodic
    directions wrapped).
  * a(chi, q, U) = (q, div(chi U))_Omega_h - sum over interior facets <q^up [[chi U.n]]>,
    q, chi in DG_k (the tracer degree k' = k, as in the paper's experiments), q^up the value on
    the side U.n points away from (U.n+ > 0: the + side). U is continuous; U.n+ at a facet point
    is evaluated as the average of the two sides' values (equal up to rounding).
  * time stepping with the explicit tableau of the IMEX method (eq. advection_update_stages,
    eq. advection_update_final): q_i = q^n + dt sum_{j<i} a^ex_ij M^-1 a(q_j, P_CG(Q_j)),
    q^{n+1} = q^n + dt sum_i b^ex_i M^-1 a(q_i, P_CG(Q_i)). The printed final sum starts at
    i = 1, which would leave the tracer of IMEX Euler (b^ex = (1, 0)) unchanged; it is read as
    starting at i = 0. The stage velocities Q_i are those of the IMEX step (Q_0 = Q^n when the
    first stage is explicit).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .element import lattice


def _coo(rows, cols, vals, shape):
    rows, cols, vals = np.broadcast_arrays(rows, cols, vals)
    return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=shape).tocsr()


class Tracer:
    def __init__(self, hdg):
        self.hdg = hdg
        m, k = hdg.mesh, hdg.k
        self.mcg = k + 1
        # continuous numbering: lattice points on the grid of spacing (Lx, Ly) / (n (k+1))
        X = m.cell_points(np.arange(m.ncells), lattice(self.mcg))          # (c, mu, 2)
        nx = m.n * self.mcg
        I = np.rint(X[..., 0] * nx / m.Lx).astype(int)
        J = np.rint(X[..., 1] * nx / m.Ly).astype(int)
        NX = nx if m.periodic_x else nx + 1
        NY = nx if m.periodic_y else nx + 1
        if m.periodic_x:
            I %= NX
        if m.periodic_y:
            J %= NY
        self.gid = J * NX + I                                              # (c, mu)
        self.ncg = NX * NY
        # CG mass matrix: sum of the cells' Lagrange mass matrices
        Mc = hdg.cell_mass(np.arange(m.ncells))                            # (c, mu, mu)
        self.Mcg = _coo(self.gid[:, :, None], self.gid[:, None, :], Mc, (self.ncg, self.ncg)).tocsc()
        self._lu = spla.splu(self.Mcg)
        self._forms = {}

    def cg_project(self, Q):
        """P_CG(Q) for a nodal DG velocity Q; returned as DG nodal values (equal at shared points)."""
        hdg, m = self.hdg, self.hdg.mesh
        mu = hdg.mu
        Mc = hdg.cell_mass(np.arange(m.ncells))
        Qc = Q.reshape(m.ncells, 2, mu)
        out = np.empty_like(Qc)
        for d in range(2):
            b = np.bincount(self.gid.ravel(), weights=np.einsum('cab,cb->ca', Mc, Qc[:, d]).ravel(),
                            minlength=self.ncg)
            u = self._lu.solve(b)
            for _ in range(2):                                             # iterative refinement
                u = u + self._lu.solve(b - self.Mcg @ u)
            out[:, d] = u[self.gid]
        return out.reshape(-1)

    def form(self, U):
        """a(chi, q, U) as a CSR matrix (rows chi, columns q; DG_k Lagrange coefficients) for a
        continuous velocity U given by nodal DG values."""
        hdg, m = self.hdg, self.hdg.mesh
        Vp, Vu = hdg.Vp, hdg.Vu
        npn, mu = hdg.npn, hdg.mu
        cells = np.arange(m.ncells)
        Uc = U.reshape(m.ncells, 2, mu)
        # volume: (q, grad chi . U + chi div U)_K
        psi = Vp.values(hdg.qp)                                            # (nq, np)
        gpsi = np.einsum('qar,cre->cqae', Vp.grads(hdg.qp), m.Jinv)        # (c, nq, np, 2)
        Uq = np.einsum('qa,cda->cqd', hdg.phi, Uc)
        gU = np.einsum('cqae,cda->cqde', hdg.grad_phys(cells), Uc)        # dU_d / dx_e
        divU = gU[..., 0, 0] + gU[..., 1, 1]
        vol = np.einsum('q,qb,cqae,cqe->cab', hdg.qw, psi, gpsi, Uq) + \
            np.einsum('q,qb,qa,cq->cab', hdg.qw, psi, psi, divU)
        vol *= m.detJ[:, None, None]
        ip = cells[:, None] * npn + np.arange(npn)[None, :]
        A = _coo(ip[:, :, None], ip[:, None, :], vol, (hdg.nP, hdg.nP))
        # interior facets: - <q^up [[chi U.n]]> with U.n+ from the average of the sides
        facets = np.nonzero(m.interior)[0]
        h = m.f_h[facets]
        sides = []
        for s in range(2):
            c = m.f_cell[facets, s]
            X = m.facet_points(facets, s, hdg.tq)
            xi = m.to_reference(c, X)
            sides.append((c, Vu.values(xi), Vp.values(xi)))
        Un = 0.5 * sum(np.einsum('fqa,fda->fqd', ph, Uc[c]) for c, ph, _ in sides)
        un = np.einsum('fqd,fd->fq', Un, m.f_normal[facets])               # U.n+
        up = (un > 0).astype(float)                                        # weight of the + side
        w = [up, 1.0 - up]
        sign = (1.0, -1.0)                                                 # [[chi U.n]] = (chi+ - chi-) U.n+
        for s in range(2):                                                 # test side
            cs, _, pss = sides[s]
            for t in range(2):                                             # side q^up comes from
                ct, _, pst = sides[t]
                blk = -sign[s] * np.einsum('q,fq,fq,fqa,fqb->fab', hdg.tw, w[t], un, pss, pst) * h[:, None, None]
                A = A + _coo((cs[:, None] * npn + np.arange(npn))[:, :, None],
                             (ct[:, None] * npn + np.arange(npn))[:, None, :], blk, (hdg.nP, hdg.nP))
        return A.tocsr()

    def mass(self):
        m, hdg = self.hdg.mesh, self.hdg
        Mp = np.einsum('q,qa,qb->ab', hdg.qw, hdg.psi, hdg.psi)
        blocks = m.detJ[:, None, None] * Mp[None]
        cells = np.arange(m.ncells)
        ip = cells[:, None] * hdg.npn + np.arange(hdg.npn)[None, :]
        return _coo(ip[:, :, None], ip[:, None, :], blocks, (hdg.nP, hdg.nP)).tocsc()

    def rhs(self, q, U):
        """M^-1 a(., q, U): the tracer's time derivative for velocity U (continuous)."""
        return spla.spsolve(self.mass(), self.form(U) @ q)

    def step(self, tab, dt, q, Qstages):
        """One explicit tracer step with the IMEX method's explicit tableau, advected by
        P_CG of the stage velocities Qstages[i] (i = 0..s-1)."""
        Ae, be, s = tab.A_ex, tab.b_ex, tab.s
        need = [np.any(Ae[i + 1:, i] != 0.0) or be[i] != 0.0 for i in range(s)]
        dq = [None] * s
        for i in range(s):
            qi = q.copy()
            for j in range(i):
                if Ae[i, j] != 0.0:
                    qi = qi + dt * Ae[i, j] * dq[j]
            if need[i]:
                dq[i] = self.rhs(qi, self.cg_project(Qstages[i]))
        out = q.copy()
        for i in range(s):
            if be[i] != 0.0:
                out = out + dt * be[i] * dq[i]
        return out
