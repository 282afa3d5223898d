"""Canonical structured triangulation for the oracle (Sec. 3.2, "Setup").

TEST INFRASTRUCTURE ONLY (see oracle/element.py).

The domain [0, Lx] x [0, Ly] is cut into n x n rectangles; rectangle (i, j) has corners
A=(i,j), B=(i+1,j), C=(i+1,j+1), D=(i,j+1) in units of (Lx/n, Ly/n) and is split along the
diagonal A-C into cell 2(jn+i) = (A, B, C) and cell 2(jn+i)+1 = (A, C, D), both
counter-clockwise. Local edge e of a cell is opposite its local vertex e.

Facets are numbered canonically: horizontal edges H(i,j) [(i,j)->(i+1,j)], then vertical
edges V(i,j) [(i,j)->(i,j+1)], then diagonals D(i,j) [(i,j)->(i+1,j+1)], each block ordered
j-major. Periodic directions drop the duplicate row/column of edges. The bracketed direction is
the facet parameter t in [0, 1] used by the trace exchange format.

Every cell keeps its own vertex coordinates (no wrap-around), so a periodic facet has a
different physical position on each side; each side stores its own copy of the endpoints.
"""
import numpy as np

from .element import lattice, lattice_1d


class Mesh:
    def __init__(self, n, Lx=1.0, Ly=1.0, periodic_x=False, periodic_y=False):
        self.n, self.Lx, self.Ly = n, float(Lx), float(Ly)
        self.periodic_x, self.periodic_y = bool(periodic_x), bool(periodic_y)
        hx, hy = self.Lx / n, self.Ly / n
        self.ncells = 2 * n * n
        xy = np.zeros((self.ncells, 3, 2))
        for j in range(n):
            for i in range(n):
                A = (i * hx, j * hy)
                B = ((i + 1) * hx, j * hy)
                C = ((i + 1) * hx, (j + 1) * hy)
                D = (i * hx, (j + 1) * hy)
                xy[2 * (j * n + i)] = (A, B, C)
                xy[2 * (j * n + i) + 1] = (A, C, D)
        self.cell_xy = xy
        # affine map x = v0 + J xi
        self.J = np.stack([xy[:, 1] - xy[:, 0], xy[:, 2] - xy[:, 0]], axis=-1)
        self.detJ = np.linalg.det(self.J)
        self.Jinv = np.linalg.inv(self.J)

        def cell(i, j, t):
            return 2 * (j * n + i) + t

        sides = []          # per facet: list of (cell, local edge, a_xy, b_xy)
        # horizontal edges
        jmax = n if self.periodic_y else n + 1
        for j in range(jmax):
            for i in range(n):
                s = []
                a = np.array([i * hx, j * hy]); b = np.array([(i + 1) * hx, j * hy])
                if j < n:
                    s.append((cell(i, j, 0), 2, a, b))
                if j > 0:
                    s.append((cell(i, j - 1, 1), 0, a, b))
                elif self.periodic_y:
                    s.append((cell(i, n - 1, 1), 0, a + [0, self.Ly], b + [0, self.Ly]))
                sides.append(s)
        self.nH = len(sides)
        imax = n if self.periodic_x else n + 1
        for j in range(n):
            for i in range(imax):
                s = []
                a = np.array([i * hx, j * hy]); b = np.array([i * hx, (j + 1) * hy])
                if i < n:
                    s.append((cell(i, j, 1), 1, a, b))
                if i > 0:
                    s.append((cell(i - 1, j, 0), 0, a, b))
                elif self.periodic_x:
                    s.append((cell(n - 1, j, 0), 0, a + [self.Lx, 0], b + [self.Lx, 0]))
                sides.append(s)
        self.nV = len(sides) - self.nH
        for j in range(n):
            for i in range(n):
                a = np.array([i * hx, j * hy]); b = np.array([(i + 1) * hx, (j + 1) * hy])
                sides.append([(cell(i, j, 0), 1, a, b), (cell(i, j, 1), 2, a, b)])
        self.nfacets = len(sides)

        nf = self.nfacets
        self.f_nsides = np.array([len(s) for s in sides])
        self.f_cell = -np.ones((nf, 2), dtype=int)
        self.f_a = np.zeros((nf, 2, 2))
        self.f_b = np.zeros((nf, 2, 2))
        self.cell_facet = -np.ones((self.ncells, 3), dtype=int)
        self.cell_side = -np.ones((self.ncells, 3), dtype=int)
        for f, s in enumerate(sides):
            for q, (c, e, a, b) in enumerate(s):
                self.f_cell[f, q] = c
                self.f_a[f, q] = a
                self.f_b[f, q] = b
                self.cell_facet[c, e] = f
                self.cell_side[c, e] = q
        assert (self.cell_facet >= 0).all()
        d = self.f_b[:, 0] - self.f_a[:, 0]
        self.f_h = np.linalg.norm(d, axis=1)
        nrm = np.stack([d[:, 1], -d[:, 0]], axis=1) / self.f_h[:, None]
        # orient n+ outward from side 0
        cen = self.cell_xy[self.f_cell[:, 0]].mean(axis=1)
        mid = 0.5 * (self.f_a[:, 0] + self.f_b[:, 0])
        sgn = np.sign(np.einsum('fi,fi->f', mid - cen, nrm))
        self.f_normal = nrm * sgn[:, None]
        self.interior = self.f_nsides == 2

    def swapped(self):
        """The same mesh with the two sides of every interior facet exchanged (n+ <-> n-)."""
        m = object.__new__(Mesh)
        m.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v)
                           for k, v in self.__dict__.items()})
        it = self.interior
        m.f_cell[it] = self.f_cell[it][:, ::-1]
        m.f_a[it] = self.f_a[it][:, ::-1]
        m.f_b[it] = self.f_b[it][:, ::-1]
        m.f_normal[it] = -self.f_normal[it]
        for c in range(self.ncells):
            for e in range(3):
                if it[m.cell_facet[c, e]]:
                    m.cell_side[c, e] = 1 - self.cell_side[c, e]
        return m

    def cell_points(self, cells, P):
        """Physical coordinates of reference points P (..., 2) in the given cells."""
        v0 = self.cell_xy[cells, 0]
        return v0[:, None, :] + np.einsum('cij,...j->c...i', self.J[cells], P)

    def to_reference(self, cells, X):
        """Reference coordinates of physical points X (c, q, 2) in cells (c,)."""
        v0 = self.cell_xy[cells, 0]
        return np.einsum('cij,cqj->cqi', self.Jinv[cells], X - v0[:, None, :])

    def facet_points(self, facets, side, t):
        """Physical points on a facet side at parameters t (q,), in that side cell's frame."""
        a = self.f_a[facets, side]; b = self.f_b[facets, side]
        return a[:, None, :] + t[None, :, None] * (b - a)[:, None, :]


def dof_counts(mesh, k):
    """(#DG unknowns in V_Q x V_p, #trace unknowns) of a mesh (Tab. stepsizes): two
    velocity components in P_{k+1} and a pressure in P_k per cell, P_k on each facet."""
    nu = 2 * len(lattice(k + 1))
    npp = len(lattice(k))
    return mesh.ncells * (nu + npp), mesh.nfacets * len(lattice_1d(k))
