// Per-cell operations of the HDG stage solver, written for a "team" of threads that cooperates
// on one cell through a scratch buffer (shared memory on the GPU). Every function is
// __host__ __device__ and only uses team-strided loops and team barriers, so the same code runs
// inside the kernels of hdg_kernels.cuh.
//
// Conventions (see refelem.h, mesh.h):
//  * cell velocity Q|_K = sum_a q[d][a] phi_a e_d with phi_a = phi^_a o F_K^{-1} (orthonormal
//    Dubiner on the reference cell), so (phi_a, phi_b)_K = detJ delta_ab; coefficient index
//    d*MU + a. Pressure: first NP functions of the same basis. Dual vectors (one-forms on V_Q)
//    are stored by their values on the basis, r[d*MU + a] = r(phi_a e_d).
//  * trace on facet F: lambda_F = sum_j l[j] L_j(t), L_j orthonormal Legendre on [0,1] in the
//    facet's canonical direction t. A cell sees lambda in its local edge direction s; where the
//    two directions differ (flip), s = 1 - t and the coefficient picks up (-1)^j.
//  * mixed operator (Step II, eq. final_update, Sec. 2.7) with coefficient c, per cell:
//      M U - c (D^T p - E^T l) = Ru ,   D U + tau (Tpp p - Tpl l) = Rp ,
//      sum_K [E U + tau (Tlp p - Tll l)] = Rl
//    with D = (psi_b, div(phi_a e_d))_K, E = <(phi_a e_d).n, L_j>_dK, Tpp/Tpl/Tll the tau facet
//    masses (eq. implicit_HDG_scheme's g and Gamma, one cell at a time). Eliminating (U, p):
//      A = (c/detJ) D D^T + tau Tpp,  H = (c/detJ) D E^T + tau Tpl,  Z = A^{-1} H,
//      S_K = (c/detJ) E E^T + tau Tll - H^T Z    (symmetric positive semidefinite),
//      sum_K S_K l_K = sum_K [E Ru/detJ + Z^T w_K] - Rl,  w_K = Rp - D Ru/detJ,
//      p = A^{-1} w + Z l,  U = (Ru - c E^T l + c D^T p)/detJ.
#pragma once
#include <cmath>

#include "mesh.h"

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif
#ifdef __CUDACC__
#include "hdg_df64.cuh"
#endif

namespace hdg {

template <int K>
struct Dims {
    static constexpr int MU = (K + 2) * (K + 3) / 2;     // P_{k+1}
    static constexpr int NU = 2 * MU;
    static constexpr int NP = (K + 1) * (K + 2) / 2;     // P_k
    static constexpr int NT = K + 1;                     // trace per facet
    static constexpr int NL = 3 * NT;                    // trace per cell
    static constexpr int NB = K + 2;                     // BDM edge moments
    static constexpr int NV = K * (K + 2);               // BDM interior moments
    static constexpr int NQ1 = (3 * K + 4) / 2;
    static constexpr int NQ = NQ1 * (NQ1 + 1);           // volume points
    static constexpr int NFQ = (3 * K + 5) / 2;          // facet points
};

// Device copies of the reference tables (layouts as in RefTables).
struct RefDev {
    const double *qw, *phi, *dphi, *fw, *ephi, *leg, *Dhat, *Ehat, *Tpp, *bdm_inv, *Iv;
    const double *nod_u, *nod_p, *mod_u, *mod_p, *nod_t, *mod_t;
    const double *Sfac, *Tadv;
};

struct MeshDev {
    const CellGeo *geo;
    const int *cell_facet, *cell_flip, *cell_nbr, *cell_nbr_edge, *facet_cell, *facet_edge;
    const int *cell_vert, *facet_vert, *vert_facet, *vert_fsign, *vert_cell;   // P1 vertex maps
    int ncells, nfacets, nverts;
};

struct Team {
    int tid, nthr;
    __host__ __device__ __forceinline__ void sync() const {
#ifdef __CUDA_ARCH__
        if (nthr <= 32) __syncwarp(); else __syncthreads();
#endif
    }
};

#define TFOR(i, n) for (int i = tm.tid; i < (n); i += tm.nthr)

__host__ __device__ __forceinline__ double ldg(const double *p) {
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// sign of trace coefficient j on local edge e of a cell (flip = local edge against the facet)
__host__ __device__ __forceinline__ double tsign(int flip, int j) { return (flip && (j & 1)) ? -1.0 : 1.0; }

// ------------------------------------------------------------------------------------------
// Static condensation of the mixed operator for one cell (coefficient c).
// Outputs: S (NL x NL, canonical facet orientation), Z (NP x NL, local orientation),
// Ainv (NP x NP). Scratch: NP*NU + NL*NU + NP*NP*2 + NP*NL*2 + NL*NL doubles.
template <int K>
__host__ __device__ void cell_condense(const Team &tm, const RefDev &R, const CellGeo &g,
                                       const int *flip, double c, double tau, double *sm,
                                       double *S_out, double *Z_out, double *Ainv_out) {
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NP = Dm::NP, NT = Dm::NT, NL = Dm::NL;
    double *D = sm;                 // NP x NU
    double *E = D + NP * NU;        // NL x NU
    double *A = E + NL * NU;        // NP x NP  (Cholesky factor in place)
    double *Ai = A + NP * NP;       // NP x NP
    double *H = Ai + NP * NP;       // NP x NL
    double *Z = H + NP * NL;        // NP x NL
    double *S = Z + NP * NL;        // NL x NL
    const double cj = c / g.detJ;
    TFOR(i, NP * NU) {
        int b = i / NU, x = i % NU, d = x / MU, a = x % MU;
        D[i] = g.detJ * (g.Jinv[d] * ldg(&R.Dhat[(0 * NP + b) * MU + a]) +
                         g.Jinv[2 + d] * ldg(&R.Dhat[(1 * NP + b) * MU + a]));
    }
    TFOR(i, NL * NU) {
        int ej = i / NU, x = i % NU, e = ej / NT, j = ej % NT, d = x / MU, a = x % MU;
        double nd = d == 0 ? g.nx[e] : g.ny[e];
        E[i] = g.h[e] * nd * ldg(&R.Ehat[(e * NT + j) * MU + a]);
    }
    tm.sync();
    TFOR(i, NP * NP) {
        int b = i / NP, b2 = i % NP;
        double s = 0;
        for (int x = 0; x < NU; ++x) s += D[b * NU + x] * D[b2 * NU + x];
        double t = 0;
        for (int e = 0; e < 3; ++e) t += g.h[e] * ldg(&R.Tpp[(e * NP + b) * NP + b2]);
        A[i] = cj * s + tau * t;
    }
    TFOR(i, NP * NL) {
        int b = i / NL, ej = i % NL, e = ej / NT, j = ej % NT;
        double s = 0;
        for (int x = 0; x < NU; ++x) s += D[b * NU + x] * E[ej * NU + x];
        H[i] = cj * s + tau * g.h[e] * ldg(&R.Ehat[(e * NT + j) * MU + b]);
    }
    tm.sync();
    if (tm.tid == 0) {                        // Cholesky A = L L^T (lower part of A)
        for (int j = 0; j < NP; ++j) {
            double s = A[j * NP + j];
            for (int k = 0; k < j; ++k) s -= A[j * NP + k] * A[j * NP + k];
            s = sqrt(s);
            A[j * NP + j] = s;
            for (int i = j + 1; i < NP; ++i) {
                double t = A[i * NP + j];
                for (int k = 0; k < j; ++k) t -= A[i * NP + k] * A[j * NP + k];
                A[i * NP + j] = t / s;
            }
        }
    }
    tm.sync();
    TFOR(col, NP) {                           // column col of A^{-1}
        double y[NP];
        for (int i = 0; i < NP; ++i) {
            double t = (i == col) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= A[i * NP + k] * y[k];
            y[i] = t / A[i * NP + i];
        }
        for (int i = NP - 1; i >= 0; --i) {
            double t = y[i];
            for (int k = i + 1; k < NP; ++k) t -= A[k * NP + i] * y[k];
            y[i] = t / A[i * NP + i];
        }
        for (int i = 0; i < NP; ++i) Ai[i * NP + col] = y[i];
    }
    tm.sync();
    TFOR(i, NP * NL) {
        int b = i / NL, ej = i % NL;
        double s = 0;
        for (int k = 0; k < NP; ++k) s += Ai[b * NP + k] * H[k * NL + ej];
        Z[i] = s;
    }
    tm.sync();
    TFOR(i, NL * NL) {
        int r = i / NL, q = i % NL;
        double s = 0;
        for (int x = 0; x < NU; ++x) s += E[r * NU + x] * E[q * NU + x];
        double t = 0;
        for (int b = 0; b < NP; ++b) t += H[b * NL + r] * Z[b * NL + q];
        double v = cj * s - t + ((r == q) ? tau * g.h[r / NT] : 0.0);
        S[i] = v;
    }
    tm.sync();
    TFOR(i, NL * NL) {
        int r = i / NL, q = i % NL;
        S_out[i] = tsign(flip[r / NT], r % NT) * tsign(flip[q / NT], q % NT) * S[i];
    }
    TFOR(i, NP * NL) Z_out[i] = Z[i];
    TFOR(i, NP * NP) Ainv_out[i] = Ai[i];
}

// ------------------------------------------------------------------------------------------
// Right-hand side of the condensed trace system for one cell.
//   Ru: dual vector (NU) or null; X: velocity (NU) or null whose constraint residual enters
//   as Rp = -[D X + tau (Tpp p - Tpl l)] + Rp_add, Rl = -[E X + tau (Tlp p - Tll l)] (p, l of the
//   current iterate; pK/lK/Rp_add may be null = zero; a global Rl_add is subtracted by the
//   facet gather).
// Outputs: v (NL, canonical orientation) = E Ru/detJ + Z^T w - Rl,  w (NP) = Rp - D Ru/detJ.
// Scratch: 2*2*MU + NP + NL + NP doubles.
template <int K>
__host__ __device__ void cell_mixed_rhs(const Team &tm, const RefDev &R, const CellGeo &g,
                                        const int *flip, double tau, const double *Ru,
                                        const double *X, const double *pK, const double *lK_local,
                                        const double *Rp_add, const double *Z, double *sm,
                                        double *v_out, double *w_out) {
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NP = Dm::NP, NT = Dm::NT, NL = Dm::NL;
    double *xr = sm;              // 2 x MU  Jinv X (reference-frame components)
    double *ur = xr + 2 * MU;     // 2 x MU  Jinv Ru
    double *w = ur + 2 * MU;      // NP
    double *rl = w + NP;          // NL: -Rl + E Ru/detJ
    TFOR(a, MU) {
        double x0 = X ? X[a] : 0.0, x1 = X ? X[MU + a] : 0.0;
        xr[a] = g.Jinv[0] * x0 + g.Jinv[1] * x1;
        xr[MU + a] = g.Jinv[2] * x0 + g.Jinv[3] * x1;
        double u0 = Ru ? Ru[a] : 0.0, u1 = Ru ? Ru[MU + a] : 0.0;
        ur[a] = g.Jinv[0] * u0 + g.Jinv[1] * u1;
        ur[MU + a] = g.Jinv[2] * u0 + g.Jinv[3] * u1;
    }
    tm.sync();
    TFOR(b, NP) {
        double dx = 0, du = 0;
        for (int r = 0; r < 2; ++r)
            for (int a = 0; a < MU; ++a) {
                double dh = ldg(&R.Dhat[(r * NP + b) * MU + a]);
                dx += dh * xr[r * MU + a];
                du += dh * ur[r * MU + a];
            }
        double tp = 0, tl = 0;
        for (int e = 0; e < 3; ++e) {
            double s = 0;
            if (pK)
                for (int b2 = 0; b2 < NP; ++b2) s += ldg(&R.Tpp[(e * NP + b) * NP + b2]) * pK[b2];
            double s2 = 0;
            if (lK_local)
                for (int j = 0; j < NT; ++j) s2 += ldg(&R.Ehat[(e * NT + j) * MU + b]) * lK_local[e * NT + j];
            tp += g.h[e] * s;
            tl += g.h[e] * s2;
        }
        double Rp = -(g.detJ * dx + tau * (tp - tl)) + (Rp_add ? Rp_add[b] : 0.0);
        w[b] = Rp - du;                    // D Ru / detJ = du (detJ cancels)
    }
    TFOR(ej, NL) {
        int e = ej / NT, j = ej % NT;
        double ex = 0, eu = 0, ep = 0;
        for (int a = 0; a < MU; ++a) {
            double eh = ldg(&R.Ehat[(e * NT + j) * MU + a]);
            double xn = X ? (g.nx[e] * X[a] + g.ny[e] * X[MU + a]) : 0.0;
            double un = Ru ? (g.nx[e] * Ru[a] + g.ny[e] * Ru[MU + a]) : 0.0;
            ex += eh * xn;
            eu += eh * un;
            if (pK && a < NP) ep += eh * pK[a];
        }
        double ll = lK_local ? lK_local[ej] : 0.0;
        double Rl = -(g.h[e] * ex + tau * g.h[e] * (ep - ll));
        rl[ej] = g.h[e] * eu / g.detJ - Rl;
    }
    tm.sync();
    TFOR(ej, NL) {
        double s = rl[ej];
        for (int b = 0; b < NP; ++b) s += Z[b * NL + ej] * w[b];
        v_out[ej] = tsign(flip[ej / NT], ej % NT) * s;
    }
    TFOR(b, NP) w_out[b] = w[b];
    tm.sync();
}

// Constraint rows of one cell (eq. implicit_HDG_scheme's Gamma): psi-rows
//   yp = D Q + tau (Tpp p - Tpl l)  and the cell's contribution to the mu-rows
//   yl = E Q + tau (Tlp p - Tll l)  (canonical orientation; summed over the facet's cells).
template <int K>
__host__ __device__ void cell_constraint(const Team &tm, const RefDev &R, const CellGeo &g,
                                         const int *flip, double tau, const double *Q, const double *pK,
                                         const double *lK_local, double *sm, double *yp_out,
                                         double *yl_out) {
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NP = Dm::NP, NT = Dm::NT, NL = Dm::NL;
    double *xr = sm;              // 2 x MU
    TFOR(a, MU) {
        xr[a] = g.Jinv[0] * Q[a] + g.Jinv[1] * Q[MU + a];
        xr[MU + a] = g.Jinv[2] * Q[a] + g.Jinv[3] * Q[MU + a];
    }
    tm.sync();
    TFOR(b, NP) {
        double dx = 0;
        for (int r = 0; r < 2; ++r)
            for (int a = 0; a < MU; ++a) dx += ldg(&R.Dhat[(r * NP + b) * MU + a]) * xr[r * MU + a];
        double tp = 0, tl = 0;
        for (int e = 0; e < 3; ++e) {
            double s = 0, s2 = 0;
            for (int b2 = 0; b2 < NP; ++b2) s += ldg(&R.Tpp[(e * NP + b) * NP + b2]) * pK[b2];
            for (int j = 0; j < NT; ++j) s2 += ldg(&R.Ehat[(e * NT + j) * MU + b]) * lK_local[e * NT + j];
            tp += g.h[e] * s;
            tl += g.h[e] * s2;
        }
        yp_out[b] = g.detJ * dx + tau * (tp - tl);
    }
    TFOR(ej, NL) {
        int e = ej / NT, j = ej % NT;
        double ex = 0, ep = 0;
        for (int a = 0; a < MU; ++a) {
            double eh = ldg(&R.Ehat[(e * NT + j) * MU + a]);
            ex += eh * (g.nx[e] * Q[a] + g.ny[e] * Q[MU + a]);
            if (a < NP) ep += eh * pK[a];
        }
        yl_out[ej] = tsign(flip[e], j) * g.h[e] * (ex + tau * (ep - lK_local[ej]));
    }
    tm.sync();
}

// Back-substitution for one cell: p = Ainv w + Z l, U = (Ru - c E^T l + c D^T p)/detJ.
// lK_local: the cell's trace (local orientation). Ru may be null.
// Scratch: NP doubles.
template <int K>
__host__ __device__ void cell_mixed_backsub(const Team &tm, const RefDev &R, const CellGeo &g,
                                            double c, const double *Ru, const double *w,
                                            const double *lK_local, const double *Z,
                                            const double *Ainv, double *sm, double *U_out,
                                            double *p_out) {
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NP = Dm::NP, NT = Dm::NT, NL = Dm::NL;
    double *p = sm;
    TFOR(b, NP) {
        double s = 0;
        for (int k = 0; k < NP; ++k) s += Ainv[b * NP + k] * w[k];
        for (int q = 0; q < NL; ++q) s += Z[b * NL + q] * lK_local[q];
        p[b] = s;
    }
    tm.sync();
    TFOR(x, NU) {
        int d = x / MU, a = x % MU;
        double et = 0;
        for (int e = 0; e < 3; ++e) {
            double nd = d == 0 ? g.nx[e] : g.ny[e];
            double s = 0;
            for (int j = 0; j < NT; ++j) s += ldg(&R.Ehat[(e * NT + j) * MU + a]) * lK_local[e * NT + j];
            et += g.h[e] * nd * s;
        }
        double dt = 0;
        for (int r = 0; r < 2; ++r) {
            double s = 0;
            for (int b = 0; b < NP; ++b) s += ldg(&R.Dhat[(r * NP + b) * MU + a]) * p[b];
            dt += g.Jinv[r * 2 + d] * s;
        }
        double ru = Ru ? Ru[x] : 0.0;
        U_out[x] = (ru - c * et) / g.detJ + c * dt;     // c D^T p / detJ = c Jinv^T Dhat^T p
    }
    TFOR(b, NP) p_out[b] = p[b];
    tm.sync();
}

// ------------------------------------------------------------------------------------------
// BDM^0_{k+1} projection of one cell (Sec. 2.3, canonical interpolant): edge normal moments of
// the average {Q}.n (0 on walls) against L_j, j < k+2; interior moments against N_k; solved on
// the reference cell through the Piola map. QK, Qnbr[e] (null on walls): modal velocities.
// The normal average is evaluated once per facet point, then integrated against every L_j.
// Scratch: bdm_scratch<K>() doubles (moments, reference coefficients, the facet-point values).
template <int K>
constexpr int bdm_scratch() { return 2 * Dims<K>::NU + 3 * Dims<K>::NFQ; }

template <int K>
__host__ __device__ void cell_bdm(const Team &tm, const RefDev &R, const CellGeo &g,
                                  const double *QK, const double *const *Qnbr, const int *nbr_edge,
                                  double *sm, double *Qs_out) {
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NB = Dm::NB, NV = Dm::NV, NFQ = Dm::NFQ;
    double *m = sm;                 // NU moments
    double *qh = m + NU;            // NU reference coefficients
    double *an = qh + NU;           // 3 x NFQ: h_e fw_q {Q}.n at the facet points (0 on walls)
    TFOR(i, 3 * NFQ) {
        const int e = i / NFQ, q = i % NFQ;
        double s = 0;
        if (Qnbr[e]) {
            const double *Qo = Qnbr[e];
            const double *pk = &R.ephi[(e * NFQ + q) * MU];
            const double *po = &R.ephi[(nbr_edge[e] * NFQ + (NFQ - 1 - q)) * MU];
            double k0 = 0, k1 = 0, o0 = 0, o1 = 0;
            for (int a = 0; a < MU; ++a) {
                double fk = ldg(pk + a), fo = ldg(po + a);
                k0 += fk * QK[a]; k1 += fk * QK[MU + a];
                o0 += fo * Qo[a]; o1 += fo * Qo[MU + a];
            }
            s = g.h[e] * ldg(&R.fw[q]) * 0.5 * ((k0 + o0) * g.nx[e] + (k1 + o1) * g.ny[e]);
        }
        an[i] = s;
    }
    tm.sync();
    TFOR(i, 3 * NB) {               // edge moments against the Legendre polynomials
        const int e = i / NB, j = i % NB;
        double s = 0;
        for (int q = 0; q < NFQ; ++q) s += an[e * NFQ + q] * ldg(&R.leg[q * NB + j]);
        m[i] = s;
    }
    TFOR(v, NV) {
        double s = 0;
        for (int a = 0; a < MU; ++a) {
            double r0 = g.Jinv[0] * QK[a] + g.Jinv[1] * QK[MU + a];
            double r1 = g.Jinv[2] * QK[a] + g.Jinv[3] * QK[MU + a];
            s += r0 * ldg(&R.Iv[(a * NV + v) * 2]) + r1 * ldg(&R.Iv[(a * NV + v) * 2 + 1]);
        }
        m[3 * NB + v] = g.detJ * s;
    }
    tm.sync();
    TFOR(x, NU) {
        double s = 0;
        for (int k = 0; k < NU; ++k) s += ldg(&R.bdm_inv[x * NU + k]) * m[k];
        qh[x] = s;
    }
    tm.sync();
    TFOR(x, NU) {
        int d = x / MU, a = x % MU;
        Qs_out[x] = (g.J[2 * d] * qh[a] + g.J[2 * d + 1] * qh[MU + a]) / g.detJ;
    }
    tm.sync();
}

// ------------------------------------------------------------------------------------------
// The tentative-velocity operator M - c F(Q*) (eq. f_impl; Alg. 2 Step I) for one cell. F's
// facet terms with test functions on this cell (h = edge length, n = this cell's normal):
//   central  +<(Q*.n+)(Q+ - Q-).{w}>      -> diag +1/2 h (Q*.n_K) ,  neighbour -1/2 h (Q*.n_K)
//   upwind   -delta <|Q*.n+|(Q+-Q-).(w+-w-)> -> diag -delta h |Q*.n| , neighbour +delta h |Q*.n|
//   penalty  -alpha/h <[[Q.n]][[w.n]]>    -> diag -alpha n n^T ,     neighbour +alpha n n^T
// with Q*.n_K = {Q*}.n_K at the facet points (the two cells traverse a shared edge in opposite
// directions, so point q of one side is point NFQ-1-q of the other). The diagonal block (NU x
// NU, with the volume advection) is formed densely; the neighbour coupling only needs, per edge
// point, wq[e*NFQ + q] = -c fw_q h_e (-Q*.n_K/2 + delta |Q*.n_K|) (0 on walls) besides the
// penalty -c alpha fw_q n n^T, and is applied matrix-free (k_cell_apply_mf and friends).
// The sums are factored: the volume advection through the reference tensor Tadv (the block is
// sum_{r,c} g_rc Tadv[r][c] with g_rc the coefficients of (J^-1 Q*)_r: the quadrature sum over
// the volume points regrouped, 2 MU multiply-adds per entry), the penalty through the reference
// facet masses Sfac, and the central/upwind facet term through per-edge MU x MU weighted facet
// masses, so that each D entry combines a handful of precomputed numbers.
// Scratch: fimpl_diag_scratch<K>() doubles. D: row-major [row][col].
// The reference tables of the assembly's pair-arithmetic form (HDG_MIXED, device only): the
// advection tensor as an FP32 hi plane and lo plane, the facet-point values and the reference
// facet masses as pairs. All null: FP64.
struct AsmF2 {
    const float *Tadv2 = nullptr;
    const float2 *ephi2 = nullptr, *Sfac2 = nullptr;
};

template <int K>
constexpr int fimpl_diag_scratch() {
    typedef Dims<K> Dm;
    return 2 * Dm::MU + 3 * Dm::NFQ + Dm::MU * Dm::MU + 3 * Dm::MU * Dm::MU + 3 * Dm::NFQ * Dm::MU + 16 + 3 * Dm::NFQ;
}

#ifdef __CUDACC__
// The tail of cell_fimpl_diag in pairs (HDG_MIXED): the advection block adv and the weighted facet
// rows T2 arrive as pairs in their own bytes; the weighted facet masses Wa and the block entries
// are summed as pairs, the entries written to D in FP64.
template <int K>
__device__ void cell_fimpl_diag_f2(const Team &tm, const AsmF2 &F2, const double *adv_, double *Wa_,
                                   const double *T2_, const double *cst_, double *D) {
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NFQ = Dm::NFQ;
    const f2 *adv = reinterpret_cast<const f2 *>(adv_), *T2 = reinterpret_cast<const f2 *>(T2_);
    f2 *Wa = reinterpret_cast<f2 *>(Wa_);
    TFOR(i, 3 * MU * MU) {              // Wa = sum_q phi_a(e, q) T2[e][q][b]
        const int e = i / (MU * MU), a = (i / MU) % MU, b = i % MU;
        acc2 s;
#pragma unroll
        for (int q = 0; q < NFQ; ++q) s.fma(f2_of(__ldg(&F2.ephi2[(e * NFQ + q) * MU + a])), T2[(e * NFQ + q) * MU + b]);
        Wa[i] = s.get();
    }
    tm.sync();
    // the cell's constants as pairs (cst, formed once per cell): pk[k][e] = -alpha n_d n_d2 for
    // k = d + d2 (xx, xy = yx, yy) on edge e, the upwind weight h_e on interior edges, c, detJ
    const f2 *cst = reinterpret_cast<const f2 *>(cst_);
    const f2 *pk = cst, *hw = cst + 9, cf = cst[12], dj = cst[13];
    TFOR(i, NU * NU) {                  // diagonal block
        const int r = i / NU, x = i % NU, d = r / MU, a = r % MU, d2 = x / MU, b = x % MU;
        const int ab = a * MU + b, k = d + d2;
        acc2 F;
#pragma unroll
        for (int e = 0; e < 3; ++e)
            F.fma(pk[3 * k + e], f2_of(__ldg(&F2.Sfac2[e * MU * MU + ab])));
        if (d == d2) {
            F.add(adv[ab]);
#pragma unroll
            for (int e = 0; e < 3; ++e) F.fma(hw[e], Wa[e * MU * MU + ab]);
        }
        const f2 cF = f2_mul(cf, F.get());
        D[i] = f2_dbl(r == x ? f2_sub(dj, cF) : f2_neg(cF));
    }
    tm.sync();
}
#endif

template <int K>
__host__ __device__ void cell_fimpl_diag(const Team &tm, const RefDev &R, const CellGeo &g,
                                         const double *QsK, const double *const *Qsn,
                                         const int *nbr_edge, double c, double alpha,
                                         double dup, double *sm, double *D, double *wq,
                                         const AsmF2 F2 = AsmF2{}) {
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NFQ = Dm::NFQ;
    double *gc = sm;                 // 2 x MU: coefficients of (J^-1 Q*)_r
    double *qsn = gc + 2 * MU;       // 3 x NFQ: {Q*}.n_e
    double *adv = qsn + 3 * NFQ;     // MU x MU
    double *Wa = adv + MU * MU;      // 3 x MU x MU: sum_q fw phi_a phi_b (Q*.n/2 - delta |Q*.n|) on edge e
    double *T2 = Wa + 3 * MU * MU;   // 3 x NFQ x MU: fw_q phi_b(e, q) (Q*.n/2 - delta |Q*.n|) (0 on walls)
    double *cst = T2 + 3 * NFQ * MU; // 16: the pair form's per-cell constants (cell_fimpl_diag_f2)
    double *weq = cst + 16;          // 3 x NFQ: the pair form's facet-point weights fw_q (Q*.n/2 - delta |Q*.n|)
    // with Tadv2 (device): g_rc also split into FP32 pairs (hi, lo) at the start of Wa, which is
    // written only after the advection block is formed
    const float *Tadv2 = F2.Tadv2;
    float *gcf = reinterpret_cast<float *>(Wa);
#ifdef __CUDA_ARCH__
    if (Tadv2 && tm.tid < 15) {         // pair constants: pk[k][e] (9), hw[e] (3), c, detJ, -detJ
        const int i = tm.tid;
        double v;
        if (i < 9) {
            const int k = i / 3, e = i % 3;
            const double na = k == 2 ? g.ny[e] : g.nx[e], nb = k == 0 ? g.nx[e] : g.ny[e];
            v = -alpha * na * nb;
        } else if (i < 12) {
            v = Qsn[i - 9] ? g.h[i - 9] : 0.0;
        } else {
            v = i == 12 ? c : (i == 13 ? g.detJ : -g.detJ);
        }
        reinterpret_cast<f2 *>(cst)[i] = f2_of(v);
    }
#endif
    TFOR(i, 2 * MU) {
        const int r = i / MU, b = i % MU;
        const double v = g.Jinv[2 * r] * QsK[b] + g.Jinv[2 * r + 1] * QsK[MU + b];
        gc[i] = v;
        if (Tadv2) {
            const float h = (float)v;
            gcf[i] = h;
            gcf[2 * MU + i] = (float)(v - (double)h);
        }
    }
    TFOR(i, 3 * NFQ) {
        int e = i / NFQ, q = i % NFQ;
        double s = 0;
        if (Qsn[e]) {
            const double *pk = &R.ephi[(e * NFQ + q) * MU];
            const double *po = &R.ephi[(nbr_edge[e] * NFQ + (NFQ - 1 - q)) * MU];
            const double *Qo = Qsn[e];
            double k0 = 0, k1 = 0, o0 = 0, o1 = 0;
            for (int a = 0; a < MU; ++a) {
                double fk = ldg(pk + a), fo = ldg(po + a);
                k0 += fk * QsK[a]; k1 += fk * QsK[MU + a];
                o0 += fo * Qo[a]; o1 += fo * Qo[MU + a];
            }
            s = 0.5 * ((k0 + o0) * g.nx[e] + (k1 + o1) * g.ny[e]);
        }
        qsn[i] = s;
#ifdef __CUDA_ARCH__
        if (Tadv2) reinterpret_cast<f2 *>(weq)[i] = f2_of(Qsn[e] ? ldg(&R.fw[q]) * (0.5 * s - dup * fabs(s)) : 0.0);
#endif
    }
    tm.sync();
    TFOR(i, 3 * NFQ * MU) {             // facet masses as E^T diag(weights) E: the weighted rows first
        const int e = i / (NFQ * MU), q = (i / MU) % NFQ, b = i % MU;
        const double sq = qsn[e * NFQ + q];
#ifdef __CUDA_ARCH__
        if (Tadv2) {                    // (pairs in the same bytes)
            reinterpret_cast<f2 *>(T2)[i] = f2_mul(reinterpret_cast<const f2 *>(weq)[e * NFQ + q],
                                                   f2_of(__ldg(&F2.ephi2[(e * NFQ + q) * MU + b])));
            continue;
        }
#endif
        T2[i] = Qsn[e] ? ldg(&R.fw[q]) * ldg(&R.ephi[(e * NFQ + q) * MU + b]) * (0.5 * sq - dup * fabs(sq)) : 0.0;
    }
    TFOR(i, 3 * NFQ) {
        int e = i / NFQ, q = i % NFQ;
        wq[i] = Qsn[e] ? -c * ldg(&R.fw[q]) * g.h[e] * (-0.5 * qsn[i] + dup * fabs(qsn[i])) : 0.0;
    }
    if (Tadv2) {
#ifdef __CUDA_ARCH__
        // -(w.(Q*.grad)Q)_K in double-FP32 on the FP32 pipes (GB300's FP64 rate is 1/64 of its FP32
        // rate): T and g_rc as pairs hi + lo (48 significant bits), each hi*hi product split exactly
        // (TwoProduct by FMA), the cross terms hi*lo + lo*hi added in FP32, the sum kept as an
        // unevaluated pair (TwoSum; Dekker 1971, Ogita-Rump-Oishi's Dot2, SIAM J. Sci. Comput. 26
        // (2005)): about 2^-46 of sum |g T| against FP64's 2^-53 per operation. The _rn intrinsics
        // keep the compiler from fusing the products into the sums.
        const float *Tl = Tadv2 + (size_t)2 * MU * MU * MU;
        const f2 mdj = reinterpret_cast<const f2 *>(cst)[14];
        TFOR(i, MU * MU) {
            float sh = 0.f, sl = 0.f;
#pragma unroll 6
            for (int rc = 0; rc < 2 * MU; ++rc) {
                const float th = __ldg(&Tadv2[(size_t)rc * MU * MU + i]), tl = __ldg(&Tl[(size_t)rc * MU * MU + i]);
                const float gh = gcf[rc], gl = gcf[2 * MU + rc];
                const float p = __fmul_rn(gh, th);
                const float e = fmaf(gh, tl, fmaf(gl, th, fmaf(gh, th, -p)));
                const float sn = __fadd_rn(sh, p);
                const float bp = __fsub_rn(sn, sh);
                const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(sn, bp)), __fsub_rn(p, bp));
                sh = sn;
                sl = __fadd_rn(sl, __fadd_rn(t, e));
            }
            reinterpret_cast<f2 *>(adv)[i] = f2_mul(mdj, f2_norm(sh, sl));   // (pairs)
        }
        tm.sync();
        cell_fimpl_diag_f2<K>(tm, F2, adv, Wa, T2, cst, D);
        return;
#endif
    } else {
        TFOR(i, MU * MU) {              // -(w.(Q*.grad)Q)_K for one component
            double s = 0;
#pragma unroll 6
            for (int rc = 0; rc < 2 * MU; ++rc) s += gc[rc] * ldg(&R.Tadv[(size_t)rc * MU * MU + i]);
            adv[i] = -g.detJ * s;
        }
    }
    tm.sync();
    TFOR(i, 3 * MU * MU) {              // Wa = sum_q phi_a(e, q) T2[e][q][b]
        const int e = i / (MU * MU), a = (i / MU) % MU, b = i % MU;
        double sa = 0;
        for (int q = 0; q < NFQ; ++q) sa += ldg(&R.ephi[(e * NFQ + q) * MU + a]) * T2[(e * NFQ + q) * MU + b];
        Wa[i] = sa;
    }
    tm.sync();
    // per edge: -alpha n_d n_d2 for (d, d2) = (x, x), (x, y) = (y, x), (y, y); upwind weight h_e on
    // interior edges
    double pxx[3], pxy[3], pyy[3], hw[3];
    for (int e = 0; e < 3; ++e) {
        pxx[e] = -alpha * g.nx[e] * g.nx[e];
        pxy[e] = -alpha * g.nx[e] * g.ny[e];
        pyy[e] = -alpha * g.ny[e] * g.ny[e];
        hw[e] = Qsn[e] ? g.h[e] : 0.0;
    }
    TFOR(i, NU * NU) {                  // diagonal block
        const int r = i / NU, x = i % NU, d = r / MU, a = r % MU, d2 = x / MU, b = x % MU;
        const int ab = a * MU + b, k = d + d2;
        const double p0 = k == 0 ? pxx[0] : (k == 1 ? pxy[0] : pyy[0]);
        const double p1 = k == 0 ? pxx[1] : (k == 1 ? pxy[1] : pyy[1]);
        const double p2 = k == 0 ? pxx[2] : (k == 1 ? pxy[2] : pyy[2]);
        double F = p0 * ldg(&R.Sfac[ab]) + p1 * ldg(&R.Sfac[MU * MU + ab]) + p2 * ldg(&R.Sfac[2 * MU * MU + ab]);
        if (d == d2) F += adv[ab] + hw[0] * Wa[ab] + hw[1] * Wa[MU * MU + ab] + hw[2] * Wa[2 * MU * MU + ab];
        D[i] = ((r == x) ? g.detJ : 0.0) - c * F;
    }
    tm.sync();
}

// In-place inverse of an n x n row-major matrix A (Gauss-Jordan, partial pivoting) with the
// team, in the precision T; Inv receives the inverse. Scratch: 1 int (pivot). Returns false if
// singular.
template <int N, class T = double>
__host__ __device__ bool team_invert(const Team &tm, T *A, T *Inv, int *piv_sm) {
    TFOR(i, N * N) Inv[i] = (i / N == i % N) ? T(1) : T(0);
    tm.sync();
    bool ok = true;
    for (int col = 0; col < N; ++col) {
        if (tm.tid == 0) {
            int p = col;
            T best = fabs(A[col * N + col]);
            for (int r = col + 1; r < N; ++r)
                if (fabs(A[r * N + col]) > best) { best = fabs(A[r * N + col]); p = r; }
            *piv_sm = (best > T(0)) ? p : -1;
        }
        tm.sync();
        int p = *piv_sm;
        if (p < 0) { ok = false; break; }
        if (p != col) {
            TFOR(j, N) {
                T t = A[col * N + j]; A[col * N + j] = A[p * N + j]; A[p * N + j] = t;
                t = Inv[col * N + j]; Inv[col * N + j] = Inv[p * N + j]; Inv[p * N + j] = t;
            }
            tm.sync();
        }
        T inv_d = T(1) / A[col * N + col];
        tm.sync();
        TFOR(j, N) { A[col * N + j] *= inv_d; Inv[col * N + j] *= inv_d; }
        tm.sync();
        TFOR(i, (N - 1) * N) {
            int r = i / N, j = i % N;
            if (r >= col) ++r;
            T f = A[r * N + col];
            if (j != col) A[r * N + j] -= f * A[col * N + j];
            Inv[r * N + j] -= f * Inv[col * N + j];
        }
        tm.sync();
        TFOR(r, N) if (r != col) A[r * N + col] = T(0);
        tm.sync();
    }
    return ok;
}

}  // namespace hdg
