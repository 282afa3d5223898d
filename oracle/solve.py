"""Stage solves, Alg. 2 and Alg. 1 of the paper with direct sparse solves (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/element.py).

Operators (oracle/hdg.py): A(c) = [[M - c F(Q*), -c G], [B, C]] acting on (Q, y), y = (p, lambda)
is the stage operator of eq. imex_implicit_solve + imex_implicit_solve_constraint with
c = a_ii dt; dropping F gives the mixed operator [[M, -c G], [B, C]] shared by Step II of
Alg. 2, the final update (eq. final_update, c = b_{s-1} dt) and the pressure reconstruction
(c = 1, Sec. 2.7). (p, lambda) = (1, 1) spans the kernel of g and Gamma; it is removed by the
pressure constraint (p)_Omega = 0 of eq. function_spaces: the last trace equation (implied by the
others for every compatible right-hand side, since (0, 1, -1) is a left null vector) and the
last trace unknown are dropped, and (p, lambda) is then shifted by the constant that gives
(p)_Omega = 0.

Readings of the paper used here:
  * Alg. 2 carries, besides the velocity residual it prints, the constraint residual
    rho = -Gamma(Q, p, lambda) of the current iterate, and Step II solves
    (U.w) - c g(w, dp, dl) = 0,  Gamma(psi, mu, U, dp, dl) = rho - Gamma(psi, mu, Qbar, 0, 0)
    with the update Q += Qbar + U (U = a_ii dt dQ in the paper's notation). The printed Step II
    puts the divergence of Qbar on the velocity row with a vector test function, which does
    not type-check; this is the Chorin split of A(c) it describes, and its fixed point is the
    monolithic stage solution.
  * The final update uses b^im_{s-1} (eq. final_update).
  * The pressure reconstruction solves eq. time_evolution with its constraint for
    (U = dQ/dt, p, lambda) given Q^{n+1}: (U.w) - g(w, p, lambda) = f^impl(w, Q, P(Q))
    + (w.f(t)), Gamma(psi, mu, U, p, lambda) = 0. The printed right-hand side of
    eq. pressure_reconstruction_compact has the same typing problem as Step II.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .bdm import bdm_project


class Oracle:
    def __init__(self, hdg):
        self.hdg = hdg
        self.M, self.G, self.B, self.C = hdg.static()
        self.nQ, self.nP, self.nL = hdg.nQ, hdg.nP, hdg.nL
        self.nY = self.nP + self.nL
        self._mixed = {}

    # ------------------------------------------------------------------ helpers
    def split(self, x):
        return x[:self.nQ], x[self.nQ:self.nQ + self.nP], x[self.nQ + self.nP:self.nQ + self.nY]

    REFINE = 2          # steps of iterative refinement after each direct solve

    def _pinned_factor(self, A):
        """LU of A without its last row and column (the last trace equation / unknown); the
        reduced matrix is kept for the refinement steps."""
        n = A.shape[0] - 1
        Ar = sp.csc_matrix(A)[:n, :n]
        lu = spla.splu(Ar)
        return lu, Ar

    def _pinned_solve(self, lu, rhs):
        """Solve with the pinned factorisation, then REFINE steps of iterative refinement
        (x += LU^{-1}(b - A x) with the residual in FP64): the stage and mixed solutions are
        defined as the exact solutions of their linear systems (eq. imex_implicit_solve), and the
        LU's backward error in the Lagrange basis leaves relative residuals ~1e-11 that the
        refinement removes (to ~1e-13)."""
        lu, Ar = lu
        b = rhs[:-1]
        y = lu.solve(b)
        for _ in range(self.REFINE):
            y = y + lu.solve(b - Ar @ y)
        x = np.zeros(len(rhs))
        x[:-1] = y
        Q, p, lam = self.split(x)
        shift = self.hdg.mean_p(p)
        return Q, p - shift, lam - shift

    def mixed_matrix(self, c):
        return sp.bmat([[self.M, -c * self.G], [self.B, self.C]], format='csr')

    def stage_matrix(self, c, F):
        return sp.bmat([[self.M - c * F, -c * self.G], [self.B, self.C]], format='csr')

    def fimpl(self, Qstar):
        return self.hdg.fimpl(Qstar)

    # ------------------------------------------------------------------ solves
    def mixed_solve(self, c, Ru, Ry):
        """[[M, -cG], [B, C]] (Q, p, lambda) = (Ru, Ry) with (p)_Omega = 0."""
        key = float(c)
        if key not in self._mixed:
            self._mixed[key] = self._pinned_factor(self.mixed_matrix(c))
        return self._pinned_solve(self._mixed[key], np.concatenate([Ru, Ry]))

    def stage_solve(self, c, r, Qstar):
        """Monolithic stage solve (eq. imex_implicit_solve + constraint) for right-hand side r
        (a dual vector on V_Q), advecting velocity Q*."""
        F = self.fimpl(Qstar)
        lu = self._pinned_factor(self.stage_matrix(c, F))
        return self._pinned_solve(lu, np.concatenate([r, np.zeros(self.nY)]))

    def constraint(self, Q, p, lam):
        """Gamma(psi, mu, Q, p, lambda) for all basis (psi, mu): vector of length nY."""
        return self.B @ Q + self.C @ np.concatenate([p, lam])

    def richardson(self, c, r, Qstar, Q0, p0, l0, n_iter=None, tol=None, max_iter=50,
                   history=None):
        """Alg. 2 with Step I and Step II solved directly (readings in the module docstring).
        Stops after n_iter iterations, or when ||Qbar + U||_M <= tol ||Q||_M."""
        F = self.fimpl(Qstar)
        Ms = (self.M - c * F).tocsc()
        lu1 = spla.splu(Ms)
        Q, y = Q0.copy(), np.concatenate([p0, l0])
        its = n_iter if n_iter is not None else max_iter
        for it in range(its):
            dr = r - self.M @ Q + c * (F @ Q + self.G @ y)
            rho = -(self.B @ Q + self.C @ y)
            Qbar = lu1.solve(dr)                                    # Step I
            for _ in range(self.REFINE):
                Qbar = Qbar + lu1.solve(dr - Ms @ Qbar)
            U, dp, dl = self.mixed_solve(c, np.zeros(self.nQ), rho - self.B @ Qbar)  # Step II
            dQ = Qbar + U                                           # Step III
            Q = Q + dQ
            y = y + np.concatenate([dp, dl])
            if history is not None:
                Qn, pn, ln = Q, y[:self.nP], y[self.nP:]
                history.append(dict(dQ=np.sqrt(dQ @ (self.M @ dQ)),
                                    gamma=np.linalg.norm(self.constraint(Qn, pn, ln))))
            if tol is not None and np.sqrt(dQ @ (self.M @ dQ)) <= tol * np.sqrt(Q @ (self.M @ Q)):
                break
        return Q, y[:self.nP], y[self.nP:], it + 1

    def condensed_mixed_solve(self, c, Ru, Ry):
        """The mixed solve by static condensation: eliminate (Q, p) cell by cell, solve the
        trace system S lambda = b, back-substitute (the SCPC route of Sec. 2.8)."""
        hdg = self.hdg
        A = self.mixed_matrix(c).tocsr()
        nI = self.nQ + self.nP
        Aii, Ail = A[:nI, :nI], A[:nI, nI:]
        Ali, All = A[nI:, :nI], A[nI:, nI:]
        # Aii is block diagonal: one (nu + npn) block per cell
        nc = hdg.mesh.ncells
        inv = []
        cells = np.arange(nc)
        for K in cells:
            idx = np.concatenate([hdg.iQ([K])[0], self.nQ + hdg.iP([K])[0]])
            inv.append((idx, np.linalg.inv(Aii[idx][:, idx].toarray())))
        rows = np.concatenate([np.repeat(i, len(i)) for i, _ in inv])
        cols = np.concatenate([np.tile(i, len(i)) for i, _ in inv])
        vals = np.concatenate([b.ravel() for _, b in inv])
        Ainv = sp.csr_matrix((vals, (rows, cols)), shape=(nI, nI))
        S = (All - Ali @ Ainv @ Ail).tocsr()
        Ri = np.concatenate([Ru, Ry[:self.nP]])
        b = Ry[self.nP:] - Ali @ (Ainv @ Ri)
        one = sp.csr_matrix(np.ones((self.nL, 1)))
        K = sp.bmat([[S, one], [one.T, None]], format='csc')
        lam = spla.spsolve(K, np.concatenate([b, [0.0]]))[:-1]
        xi = Ainv @ (Ri - Ail @ lam)
        Q, p = xi[:self.nQ], xi[self.nQ:]
        shift = hdg.mean_p(p)
        return Q, p - shift, lam - shift, S

    def div_free_project(self, Qbar):
        """Step II with c = 1 applied to Qbar: Qbar + U with Gamma(Qbar + U, p, lambda) = 0."""
        U, p, l = self.mixed_solve(1.0, np.zeros(self.nQ), -self.B @ Qbar)
        return Qbar + U, p, l

    def reconstruct_pressure(self, Q, forcing_dual=None):
        """Pressure reconstruction (reading in the module docstring): returns (U, p, lambda)."""
        F = self.fimpl(bdm_project(self.hdg, Q))
        Ru = F @ Q
        if forcing_dual is not None:
            Ru = Ru + forcing_dual
        return self.mixed_solve(1.0, Ru, np.zeros(self.nY))

    # ------------------------------------------------------------------ Alg. 1
    def imex_step(self, tab, dt, t, Q, p, lam, forcing=None, solver='direct',
                  richardson_kw=None, stats=None, stages=None):
        """One step of Alg. 1. forcing(t) returns the dual vector (w . f(t)) or None.
        solver='direct' solves each stage system monolithically (the definition);
        'richardson' uses Alg. 2 with the keyword arguments richardson_kw.

        Alg. 1 assumes an explicit first stage (a_00 = a_i0 = b_0 = 0, Q_0 = Q^n). The paper's
        SSP2(3,3,2) and SSP3(4,3,3) tableaus (App. A) have an implicit first stage (a_00 != 0);
        they are run with the same recursion extended to it: every stage i with a_ii != 0 is
        solved with coefficient a_ii dt (stage 0 advected by P(Q^n)), and the sums of
        eq. imex_residual and eq. final_residual run over every implicit stage j < i (or i),
        j = 0 included. For a_00 = 0 this is Alg. 1 exactly. stages (a list, optional) receives the
        stage velocities Q_0 .. Q_{s-1} (Q_0 = Q^n when the first stage is explicit)."""
        hdg, M = self.hdg, self.M
        A, Ae, b, be, cc, s = tab.A_im, tab.A_ex, tab.b_im, tab.b_ex, tab.c, tab.s
        fl = (lambda tt: forcing(tt)) if forcing is not None else (lambda tt: 0.0)
        MQn = M @ Q
        Qs, ps, ls, rs = [Q], [p], [lam], [None]
        implicit = [A[i, i] != 0.0 for i in range(s)]
        if not implicit[0]:
            assert np.all(A[:, 0] == 0.0) and b[0] == 0.0, 'explicit first stage needs a_i0 = b_0 = 0'
        for i in range(s):
            if i == 0 and not implicit[0]:
                continue                                            # Q_0 = Q^n
            assert implicit[i], 'only the first stage may be explicit'
            r = MQn.copy()
            for j in range(i):
                if implicit[j] and A[i, j] != 0.0:
                    r = r + (A[i, j] / A[j, j]) * (M @ Qs[j] - rs[j])
            for j in range(0, i):
                if Ae[i, j] != 0.0:
                    r = r + dt * Ae[i, j] * fl(t + cc[j] * dt)
            Qprev, pprev, lprev = (Qs[i - 1], ps[i - 1], ls[i - 1]) if i > 0 else (Q, p, lam)
            Qstar = bdm_project(hdg, Qprev)
            ci = A[i, i] * dt
            if solver == 'direct':
                Qi, pi, li = self.stage_solve(ci, r, Qstar)
            else:
                Qi, pi, li, nit = self.richardson(ci, r, Qstar, Qprev, pprev, lprev,
                                                  **(richardson_kw or {}))
                if stats is not None:
                    stats.setdefault('richardson', []).append(nit)
            if i == 0:
                Qs[0], ps[0], ls[0], rs[0] = Qi, pi, li, r
            else:
                Qs.append(Qi); ps.append(pi); ls.append(li); rs.append(r)
        if stages is not None:
            stages.extend(Qs)
        rn = MQn.copy()
        for i in range(s):
            if implicit[i] and b[i] != 0.0:
                rn = rn + (b[i] / A[i, i]) * (M @ Qs[i] - rs[i])
        for i in range(0, s):
            if be[i] != 0.0:
                rn = rn + dt * be[i] * fl(t + cc[i] * dt)
        Qn, _, _ = self.mixed_solve(dt * b[s - 1], rn, np.zeros(self.nY))
        fn = forcing(t + dt) if forcing is not None else None
        _, pn, ln = self.reconstruct_pressure(Qn, fn)
        return Qn, pn, ln
