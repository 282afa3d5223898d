"""Projection Q* = P(Q) onto BDM^0_{k+1} used by the advection operator (Sec. 2.3, Alg. 1).

TEST INFRASTRUCTURE ONLY (see oracle/element.py).

The paper refers to (2.25)-(2.26) of Guzman et al. (2016) for P without restating it. Reading
used here: the canonical BDM_{k+1} interpolant, cell by cell. Q*|_K in [P_{k+1}(K)]^2 is fixed
by
  * the normal moments <Q*.n_K, m>_e = <{Q}.n_K, m>_e for every m in P_{k+1}(e) on the three
    edges e of K; on boundary edges the right-hand side is 0 (the superscript 0: n.Q* = 0 on
    the wall);
  * the interior moments (Q*, v)_K = (Q, v)_K for every v in the first-kind Nedelec space
    N_k(K) = [P_{k-1}]^2 + (-y', x') P~_{k-1}  (x' = x - centroid, P~ homogeneous).
3(k+2) + k(k+2) = (k+2)(k+3) = dim [P_{k+1}]^2 conditions, so the local system is square. The
edge moments are shared by the two cells of a facet, so Q*.n is single-valued.
"""
import numpy as np


def _nedelec_values(k, Xc):
    """First-kind Nedelec N_k basis at points Xc (c, q, 2) (coordinates relative to the
    centroid): (c, q, dim, 2)."""
    x, y = Xc[..., 0], Xc[..., 1]
    out = []
    zero = np.zeros_like(x)
    for deg in range(k):                       # [P_{k-1}]^2
        for a in range(deg + 1):
            m = x ** (deg - a) * y ** a
            out.append(np.stack([m, zero], -1))
            out.append(np.stack([zero, m], -1))
    if k >= 1:
        for a in range(k):                     # (-y, x) times homogeneous degree k-1
            m = x ** (k - 1 - a) * y ** a
            out.append(np.stack([-y * m, x * m], -1))
    return np.stack(out, axis=-2)


def bdm_project(hdg, Q):
    """Q* = P(Q) for the nodal velocity Q (global vector) -> nodal Q* (global vector)."""
    m, k, mu, nu = hdg.mesh, hdg.k, hdg.mu, hdg.nu
    nc = m.ncells
    cells = np.arange(nc)
    A = np.zeros((nc, nu, nu))
    rhs = np.zeros((nc, nu))
    tj = np.stack([hdg.tq ** j for j in range(k + 2)], -1)       # P_{k+1}(e) basis (nfq, k+2)
    row = 0
    for e in range(3):
        F = m.cell_facet[:, e]
        s = m.cell_side[:, e]
        h = m.f_h[F]
        n = np.where((s == 0)[:, None], m.f_normal[F], -m.f_normal[F])
        a = m.f_a[F, s]; b = m.f_b[F, s]
        X = a[:, None, :] + hdg.tq[None, :, None] * (b - a)[:, None, :]
        ph = hdg.Vu.values(m.to_reference(cells, X))               # (c, q, mu)
        # rows: h sum_q w_q (phi_a e_d . n) t^j
        blk = np.einsum('q,cqa,cd,qj->cjda', hdg.tw, ph, n, tj) * h[:, None, None, None]
        A[:, row:row + k + 2, :] = blk.reshape(nc, k + 2, nu)
        # right-hand side with the average {Q} (zero on boundary edges)
        qK = np.einsum('cqa,cda->cqd', ph, Q[hdg.iQ(cells)].reshape(nc, 2, mu))
        inter = m.interior[F]
        so = 1 - s
        oc = np.where(inter, m.f_cell[F, np.where(inter, so, 0)], 0)
        ao = m.f_a[F, np.where(inter, so, 0)]; bo = m.f_b[F, np.where(inter, so, 0)]
        Xo = ao[:, None, :] + hdg.tq[None, :, None] * (bo - ao)[:, None, :]
        pho = hdg.Vu.values(m.to_reference(oc, Xo))
        qO = np.einsum('cqa,cda->cqd', pho, Q[hdg.iQ(oc)].reshape(nc, 2, mu))
        avg = 0.5 * (qK + qO)
        r = np.einsum('q,cqd,cd,qj->cj', hdg.tw, avg, n, tj) * h[:, None]
        rhs[:, row:row + k + 2] = np.where(inter[:, None], r, 0.0)
        row += k + 2
    # interior moments against N_k
    Xq = m.cell_points(cells, hdg.qp)                               # (c, q, 2)
    cen = m.cell_xy.mean(axis=1)
    V = _nedelec_values(k, Xq - cen[:, None, :])                    # (c, q, nv, 2)
    nv = V.shape[2]
    assert row + nv == nu
    blk = np.einsum('q,qa,cqvd->cvda', hdg.qw, hdg.phi, V) * m.detJ[:, None, None, None]
    A[:, row:, :] = blk.reshape(nc, nv, nu)
    qq = np.einsum('qa,cda->cqd', hdg.phi, Q[hdg.iQ(cells)].reshape(nc, 2, mu))
    rhs[:, row:] = np.einsum('q,cqd,cqvd->cv', hdg.qw, qq, V) * m.detJ[:, None]
    Qs = np.linalg.solve(A, rhs[..., None])[..., 0]
    return Qs.reshape(-1)
