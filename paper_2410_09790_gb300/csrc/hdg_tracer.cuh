// Passive tracer advection of App. B: explicit upwind DG for q in DG_k, advected by the L2
// projection U = P_CG(Q) of the velocity onto the continuous space CG_{k+1}.
//
//   P_CG:  M_CG u = b, b_i = (Q, phi_i) over the continuous Lagrange basis of the equispaced
//          lattices (point numbering: build_cg_numbering). Jacobi-preconditioned CG on the two
//          components at once (the same matrix for both), matrix-free: a cell's Lagrange mass is
//          detJ N^T N with N = nod_u (nodal -> orthonormal modal), applied per cell and summed per
//          point by gathering the point's (cell, node) entries (fixed order: deterministic).
//   a(chi, q, U) = (q, div(chi U))_K - sum over interior facets <q^up [[chi U.n]]>; U.n at a facet
//          point is the average of the two sides' values (identical on both sides, so the two
//          cells take the same upwind value), q^up the value on the side U.n points away from.
// Vectors on the continuous space are [component][point].
#pragma once
#include "hdg_kernels.cuh"

namespace hdg {

struct CGMap {
    const int *cell_gid;    // [cell][nl]
    const int *node_ptr;    // [npts + 1]
    const int *node_list;   // entries cell * nl + l
    const double *dinv;     // inverse diagonal of M_CG, [npts]
    int npts, nl, ncells;
};

// b[d][pt] = sum over the point's entries (c, l) of detJ_c sum_a N[a][l] Q[c][d][a]
__global__ void k_cgp_rhs(const CellGeo *__restrict__ geo, const double *__restrict__ nod_u, CGMap C,
                          const double *__restrict__ Qm, double *b) {
    wait_prior_kernel();
    const int nl = C.nl;
    GRID_STRIDE(i, 2LL * C.npts) {
        const int d = (int)(i / C.npts), pt = (int)(i % C.npts);
        double s = 0.0;
        for (int e = C.node_ptr[pt]; e < C.node_ptr[pt + 1]; ++e) {
            const int ent = C.node_list[e], c = ent / nl, l = ent % nl;
            const double *q = Qm + ((size_t)c * 2 + d) * nl;
            double t = 0.0;
            for (int a = 0; a < nl; ++a) t += __ldg(&nod_u[a * nl + l]) * q[a];
            s += geo[c].detJ * t;
        }
        b[i] = s;
    }
}

// u = 0; r = b; z = D^-1 r; rz = (r, z); the loop's scalars (beta = 0: the first direction is z)
__global__ void k_cgp_start(CGMap C, const double *__restrict__ b, double *u, double *r, double *z, RedBuf rb,
                            Scalars *sc, double rtol, int maxit) {
    wait_prior_kernel();
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, 2LL * C.npts) {
        const double bi = b[i], zi = C.dinv[i % C.npts] * bi;
        u[i] = 0.0;
        r[i] = bi;
        z[i] = zi;
        v[0] += bi * zi;
    }
    if (grid_sum<1>(rb, v, tot)) {
        sc->rz = tot[0];
        sc->rz0 = tot[0];
        sc->beta = 0.0;
        sc->iters = 0;
        sc->breakdown = 0;
        sc->rtol = rtol;
        sc->maxit = maxit;
        sc->relres = tot[0] > 0.0 ? 1.0 : 0.0;
        sc->done = !(tot[0] > 0.0);
        if (!isfinite(tot[0])) { sc->done = 1; sc->breakdown = 2; }
    }
}

// w[c][d][l] = detJ sum_a N[a][l] sum_m N[a][m] p[d][gid(c, m)] with p = z + beta pold formed at
// the gathered points (k_cgp_gather stores the same p)
template <int K>
__global__ void k_cgp_cell(MeshDev M, const double *__restrict__ nod_u, CGMap C, const double *__restrict__ z,
                           const double *__restrict__ pold, double *w, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU;
    constexpr int SCR = 4 * MU;
    CELL_TEAM(SCR)
    const double beta = sc->beta;
    double *pv = mine, *am = mine + 2 * MU;
    TFOR(i, 2 * MU) {
        const int d = i / MU, l = i % MU;
        const size_t g = (size_t)d * C.npts + C.cell_gid[(size_t)cell * MU + l];
        pv[i] = z[g] + beta * pold[g];
    }
    tm.sync();
    TFOR(i, 2 * MU) {
        const int d = i / MU, a = i % MU;
        double s = 0.0;
        for (int m = 0; m < MU; ++m) s += __ldg(&nod_u[a * MU + m]) * pv[d * MU + m];
        am[i] = s;
    }
    tm.sync();
    const double dj = M.geo[cell].detJ;
    TFOR(i, 2 * MU) {
        const int d = i / MU, l = i % MU;
        double s = 0.0;
        for (int a = 0; a < MU; ++a) s += __ldg(&nod_u[a * MU + l]) * am[d * MU + a];
        w[((size_t)cell * 2 + d) * MU + l] = dj * s;
    }
}

// p = z + beta pold (stored); Ap[d][pt] = sum of the point's w entries; alpha = rz / (p, Ap)
__global__ void k_cgp_gather(CGMap C, const double *__restrict__ w, const double *__restrict__ z, double *p,
                             double *Ap, RedBuf rb, Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const double beta = sc->beta;
    const int nl = C.nl;
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, 2LL * C.npts) {
        const int d = (int)(i / C.npts), pt = (int)(i % C.npts);
        double s = 0.0;
        for (int e = C.node_ptr[pt]; e < C.node_ptr[pt + 1]; ++e) {
            const int ent = C.node_list[e];
            s += w[((size_t)(ent / nl) * 2 + d) * nl + ent % nl];
        }
        const double pi = z[i] + beta * p[i];
        p[i] = pi;
        Ap[i] = s;
        v[0] += pi * s;
    }
    if (grid_sum<1>(rb, v, tot)) {
        sc->pAp = tot[0];
        if (tot[0] > 0.0 && isfinite(tot[0])) sc->alpha = sc->rz / tot[0];
        else { sc->alpha = 0.0; sc->done = 1; sc->breakdown = isfinite(tot[0]) ? 1 : 2; }
    }
}

// u += alpha p; r -= alpha Ap; z = D^-1 r; beta = (r, z) / rz; stop at sqrt(rz / rz0) <= rtol
__global__ void k_cgp_update(CGMap C, const double *__restrict__ p, const double *__restrict__ Ap, double *u,
                             double *r, double *z, RedBuf rb, Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const double alpha = sc->alpha;
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, 2LL * C.npts) {
        u[i] += alpha * p[i];
        const double ri = r[i] - alpha * Ap[i], zi = C.dinv[i % C.npts] * ri;
        r[i] = ri;
        z[i] = zi;
        v[0] += ri * zi;
    }
    if (grid_sum<1>(rb, v, tot)) {
        sc->beta = tot[0] / sc->rz;
        sc->rz = tot[0];
        sc->iters += 1;
        const double rel = sc->rz0 > 0 ? sqrt(fmax(tot[0], 0.0) / sc->rz0) : 0.0;
        sc->relres = rel;
        if (!isfinite(tot[0])) { sc->done = 1; sc->breakdown = 2; }
        else if (rel <= sc->rtol || sc->iters >= sc->maxit) sc->done = 1;
    }
}

// U[c][d][a] = sum_l N[a][l] u[d][gid(c, l)]: the continuous field in each cell's modal basis
template <int K>
__global__ void k_cgp_to_modal(const double *__restrict__ nod_u, CGMap C, const double *__restrict__ u, double *Um) {
    wait_prior_kernel();
    constexpr int MU = Dims<K>::MU;
    GRID_STRIDE(i, (long long)C.ncells * 2 * MU) {
        const int a = (int)(i % MU), d = (int)((i / MU) % 2);
        const long long c = i / (2 * MU);
        double s = 0.0;
        for (int l = 0; l < MU; ++l) s += __ldg(&nod_u[a * MU + l]) * u[(size_t)d * C.npts + C.cell_gid[c * MU + l]];
        Um[i] = s;
    }
}

// out = M^-1 a(., q, U) per cell (q: DG_k modal [c][NP]; U: modal velocity [c][2][MU], continuous)
template <int K>
__global__ void k_tracer_rhs(RefDev R, MeshDev M, const double *__restrict__ q, const double *__restrict__ U,
                             double *out) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NP = Dm::NP, NQ = Dm::NQ, NFQ = Dm::NFQ;
    constexpr int SCR = 3 * NQ + 3 * NFQ;
    CELL_TEAM(SCR)
    double *s1 = mine, *s2 = mine + 2 * NQ, *flux = s2 + NQ;
    const CellGeo g = M.geo[cell];
    const double *qK = q + (size_t)cell * NP, *UK = U + (size_t)cell * 2 * MU;
    TFOR(qq, NQ) {
        double qv = 0.0, u0 = 0.0, u1 = 0.0, d00 = 0.0, d01 = 0.0, d10 = 0.0, d11 = 0.0;
        for (int a = 0; a < MU; ++a) {
            const double f = ldg(&R.phi[qq * MU + a]);
            const double g0 = ldg(&R.dphi[(qq * MU + a) * 2]), g1 = ldg(&R.dphi[(qq * MU + a) * 2 + 1]);
            if (a < NP) qv += f * qK[a];
            u0 += f * UK[a]; u1 += f * UK[MU + a];
            d00 += g0 * UK[a]; d01 += g1 * UK[a];             // dUx / dxi, dUx / deta
            d10 += g0 * UK[MU + a]; d11 += g1 * UK[MU + a];   // dUy / dxi, dUy / deta
        }
        // div U = sum_d sum_r Jinv[r][d] dU_d / dxi_r; U . grad chi = sum_r beta_r dchi / dxi_r
        const double divU = g.Jinv[0] * d00 + g.Jinv[2] * d01 + g.Jinv[1] * d10 + g.Jinv[3] * d11;
        const double b0 = g.Jinv[0] * u0 + g.Jinv[1] * u1, b1 = g.Jinv[2] * u0 + g.Jinv[3] * u1;
        const double wq = ldg(&R.qw[qq]) * qv;
        s1[2 * qq] = wq * b0;
        s1[2 * qq + 1] = wq * b1;
        s2[qq] = wq * divU;
    }
    TFOR(i, 3 * NFQ) {
        const int e = i / NFQ, qq = i % NFQ;
        const int o = M.cell_nbr[3 * cell + e];
        double fl = 0.0;
        if (o >= 0) {
            const int eo = M.cell_nbr_edge[3 * cell + e], qo = NFQ - 1 - qq;
            const double *pk = &R.ephi[(e * NFQ + qq) * MU], *po = &R.ephi[(eo * NFQ + qo) * MU];
            const double *qO = q + (size_t)o * NP, *UO = U + (size_t)o * 2 * MU;
            double qk = 0.0, qn = 0.0, ux = 0.0, uy = 0.0;
            for (int a = 0; a < MU; ++a) {
                const double fk = ldg(pk + a), fo = ldg(po + a);
                if (a < NP) { qk += fk * qK[a]; qn += fo * qO[a]; }
                ux += fk * UK[a] + fo * UO[a];
                uy += fk * UK[MU + a] + fo * UO[MU + a];
            }
            const double un = 0.5 * (ux * g.nx[e] + uy * g.ny[e]);
            fl = -ldg(&R.fw[qq]) * g.h[e] * un * (un > 0.0 ? qk : qn);
        }
        flux[i] = fl;
    }
    tm.sync();
    TFOR(a, NP) {
        double v = 0.0, f = 0.0;
        for (int qq = 0; qq < NQ; ++qq)
            v += s1[2 * qq] * ldg(&R.dphi[(qq * MU + a) * 2]) + s1[2 * qq + 1] * ldg(&R.dphi[(qq * MU + a) * 2 + 1]) +
                 s2[qq] * ldg(&R.phi[qq * MU + a]);
        for (int i = 0; i < 3 * NFQ; ++i) f += ldg(&R.ephi[i * MU + a]) * flux[i];
        out[(size_t)cell * NP + a] = v + f / g.detJ;          // (the volume sums omit detJ: M = detJ I)
    }
}

}  // namespace hdg
