// FP32 stage operator for the relaxed Arnoldi steps of the stage flexible GMRES (HDG_MIXED).
//
// The stage system A(c) x = b (Sec. 2.7: velocity rows (M - cF)Q - c G(p, lambda), the cell's
// pressure rows and its contributions to the trace rows) is solved by FGMRES to a relative
// residual rtol. An Arnoldi product w_j = A z_j that carries an error e_j changes the final
// residual by at most sum_j |y_j| ||e_j||, and the late coefficients y_j shrink with the
// residual reached before step j (the inexact-Krylov bound of Simoncini and Szyld, SIAM J. Sci.
// Comput. 25 (2003), and Bouras and Fraysse, SIAM J. Matrix Anal. Appl. 26 (2005)): once the
// residual estimate r_j satisfies r_j * eta <= rtol * ||b|| the product may carry a relative
// error of order eta. The solver then takes the product below, in FP32 (eta ~ 1e-5 covers
// FP32's 6e-8 unit roundoff, the sums of up to 3,700 terms per cell and the preconditioner's
// gain on ||z_j||). The restart check always forms b - A x with the FP64 kernel, so an
// inaccurate late product can cost an extra cycle, never the tolerance.
//
// The FP32 and FP64 kernels are both recorded for every Arnoldi step; each reads the decision
// (GmresState::lowprec, set by the previous step's Givens update) and one of them returns at once.
// Inputs and outputs stay FP64 vectors (the Krylov basis is FP64): the kernel converts the
// cell's own and its three neighbours' coefficients to FP32 in shared memory once, and its
// stores widen back to FP64.
//
// The constraint rows are taken through the facet jump p - lambda: on edge e the trace of p is a
// polynomial of degree k, so it equals sum_j P_ej L_j with P_ej = (L_j, p)_e = sum_b Ehat[e j b]
// p_b, and with J_ej = P_ej - lambda_ej the rows are tau (Tpp p - Tpl lambda)_b = tau sum_e h_e
// sum_j Ehat[e j b] J_ej and tau (Tlp p - Tll lambda)_ej = tau h_e J_ej (the same numbers in exact
// arithmetic). The kernel forms J in FP64 (3 (k+1) dim P_k multiply-adds per cell) and the rest in
// FP32: in the preconditioned directions z_j = P^-1 v_j the pressure and trace are O(1/c) and
// nearly equal on the facets while the rows are O(1), so summing Tpp p and Tpl lambda separately
// in FP32 would leave an error of 1e-7 / c.
#pragma once
#include "hdg_kernels.cuh"

namespace hdg {

// FP32 copies of the reference tables the stage operator needs (layouts as in RefDev)
struct Ref32 {
    const float *Dhat, *Ehat;
};

// the diagonal blocks rounded to FP32 in the per-cell layout GsBlk (when no FP32 inverses are
// formed; else k_block_inv32 writes them): Dblk in the column-slice layout [col * nrows + cell *
// NU + row]
template <int K>
__global__ void k_blocks_to_f32(const double *__restrict__ Dblk, float *__restrict__ Dblk32, long long ncells) {
    wait_prior_kernel();
    typedef GsBlk<K> B;
    const long long nrows = ncells * B::NU;
    GRID_STRIDE(i, ncells * B::SIZE) {
        const long long cell = i / B::SIZE;
        const int o = (int)(i % B::SIZE), q = o / B::NUP, r = o % B::NUP;
        Dblk32[i] = (q < B::NU && r < B::NU) ? (float)Dblk[(size_t)q * nrows + (size_t)cell * B::NU + r] : 0.f;
    }
}

// per-cell geometry in FP32: Jinv[4], detJ, h[3]
constexpr int GEO32 = 8;

template <int K>
constexpr int stage32_scratch_floats() {
    typedef Dims<K> Dm;
    return 2 * (Dm::NP + Dm::NL) + 5 * Dm::NU + Dm::NP + Dm::NL + 6 * Dm::NFQ + 2 * Dm::MU + GEO32 + Dm::NL;
}

// a warp per cell, four cells per 128-thread block
constexpr int STAGE32_WARPS = 4;

// y = A(c) x with x = (Q, p, lambda) in FP64 memory, arithmetic in FP32; same outputs as
// k_stage_apply (yQ, yp, the cell's lambda-row contributions v, the FP32 shadows yQ32 / yp32,
// and the copy of x into the FGMRES's preconditioned-vector slot *zslot_j when set). Runs only
// when gs->lowprec is set; counts its launches in acc->products32 (when acc is set). A warp per
// cell: the diagonal block (Dblk, per-cell layout GsBlk) is applied by warp_block_apply with
// 16-byte loads of contiguous memory.
template <int K>
__global__ void __launch_bounds__(128) k_stage_apply32(RefDev R64, Ref32 R, EdgeTab<float> E, MeshDev M,
                                                       const float *__restrict__ geo32, const float *__restrict__ Dblk,
                                                       const float *__restrict__ wq, float c, float tau, const double *Q,
                                                       const double *p, const double *lam, double *yQ, double *yp,
                                                       double *v, float *yQ32, float *yp32, double *zslot,
                                                       const int *zslot_j, GmresState *gs, DevCount *acc) {
    wait_prior_kernel();
    if (!gs->lowprec) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        gs->used32 = 1;
        if (acc) acc->products32 += 1;
    }
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NP = Dm::NP, NT = Dm::NT, NL = Dm::NL, NFQ = Dm::NFQ;
    constexpr int SCR = (stage32_scratch_floats<K>() + 1) / 2;   // in doubles
    extern __shared__ double sm[];
    const int team = threadIdx.x >> 5;
    const int cell = blockIdx.x * STAGE32_WARPS + team;
    if (cell >= M.ncells) return;
    Team tm{(int)(threadIdx.x & 31), 32};
    double *pD = sm + team * SCR, *lD = pD + NP;             // p and lambda (local orientation) in FP64
    float *xK = reinterpret_cast<float *>(lD + NL);          // own Q (NU)
    float *xn = xK + NU;                                     // neighbours' Q (3 x NU)
    float *pK = xn + 3 * NU, *lK = pK + NP, *t = lK + NL, *xr = t + 6 * NFQ, *gg = xr + 2 * MU;
    float *jmp = gg + GEO32;                                 // J_ej = (L_j, p)_e - lambda_ej (NL)
    float *dq = jmp + NL;                                    // the diagonal block times Q (NU)
    const int *nbr = M.cell_nbr + 3 * cell;
    TFOR(i, NU) xK[i] = (float)Q[(size_t)cell * NU + i];
    TFOR(i, 3 * NU) {
        const int o = __ldg(&nbr[i / NU]);
        xn[i] = o >= 0 ? (float)Q[(size_t)o * NU + i % NU] : 0.f;
    }
    TFOR(b, NP) {
        const double pb = p[(size_t)cell * NP + b];
        pD[b] = pb;
        pK[b] = (float)pb;
    }
    TFOR(i, NL) {
        const int e = i / NT, j = i % NT;
        const int f = __ldg(&M.cell_facet[3 * cell + e]);
        const double l = (__ldg(&M.cell_flip[3 * cell + e]) && (j & 1)) ? -lam[(size_t)f * NT + j] : lam[(size_t)f * NT + j];
        lD[i] = l;
        lK[i] = (float)l;
    }
    TFOR(i, GEO32) gg[i] = __ldg(&geo32[(size_t)cell * GEO32 + i]);
    tm.sync();
    TFOR(i, NL) {                                            // the facet jumps, in FP64
        double s = -lD[i];
#pragma unroll
        for (int b = 0; b < NP; ++b) s += ldg(&R64.Ehat[i * MU + b]) * pD[b];
        jmp[i] = (float)s;
    }
    // neighbour coupling at this cell's edge points (team_nbr_flux, from the shared copies)
    TFOR(i, 3 * NFQ) {
        const int e = i / NFQ, q = i % NFQ;
        const int o = __ldg(&nbr[e]);
        float tx = 0.f, ty = 0.f;
        if (o >= 0) {
            const int eo = __ldg(&M.cell_nbr_edge[3 * cell + e]), qo = NFQ - 1 - q;
            const float *ph = &E.ephi[(eo * NFQ + qo) * MU];
            const float *xo = xn + e * NU;
            float ux = 0.f, uy = 0.f;
#pragma unroll 7
            for (int b = 0; b < MU; ++b) {
                const float f = __ldg(ph + b);
                ux = fmaf(f, xo[b], ux);
                uy = fmaf(f, xo[MU + b], uy);
            }
            const float nx = __ldg(&E.nrm[6 * cell + 2 * e]), ny = __ldg(&E.nrm[6 * cell + 2 * e + 1]);
            const float un = nx * ux + ny * uy, pen = __ldg(&E.pen[q]);
            const float w = __ldg(&wq[(size_t)cell * 3 * NFQ + i]);
            tx = pen * nx * un + w * ux;
            ty = pen * ny * un + w * uy;
        }
        t[2 * i] = tx;
        t[2 * i + 1] = ty;
    }
    TFOR(a, MU) {                                            // Jinv^T-mapped velocity for the p-rows
        xr[a] = gg[0] * xK[a] + gg[1] * xK[MU + a];
        xr[MU + a] = gg[2] * xK[a] + gg[3] * xK[MU + a];
    }
    tm.sync();
    warp_block_apply<K>(Dblk, cell, xK, dq);
    tm.sync();
    const float detJ = gg[4];
    // velocity rows: (M - cF) Q (diagonal block dense, neighbours from t) - c (detJ Jinv-mapped
    // Dhat^T p - sum_e h_e n_e Ehat^T lambda)
    TFOR(x, NU) {
        const int d = x / MU, a = x % MU;
        const size_t gi = (size_t)cell * NU + x;
        const float bq = nbr_row<K, float>(E, t, d, a) + dq[x];
        float et = 0.f;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float nd = __ldg(&E.nrm[6 * cell + 2 * e + d]);
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < NT; ++j) s = fmaf(__ldg(&R.Ehat[(e * NT + j) * MU + a]), lK[e * NT + j], s);
            et += gg[5 + e] * nd * s;
        }
        float dt = 0.f;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            float s = 0.f;
#pragma unroll
            for (int b = 0; b < NP; ++b) s = fmaf(__ldg(&R.Dhat[(rr * NP + b) * MU + a]), pK[b], s);
            dt += gg[rr * 2 + d] * s;
        }
        const float yv = bq - c * (detJ * dt - et);
        yQ[gi] = (double)yv;
        if (yQ32) yQ32[gi] = yv;
    }
    // the cell's pressure rows: yp = D Q + tau sum_e h_e sum_j Ehat[e j b] J_ej
    TFOR(b, NP) {
        float dx = 0.f;
        for (int r = 0; r < 2; ++r)
#pragma unroll 7
            for (int a = 0; a < MU; ++a) dx = fmaf(__ldg(&R.Dhat[(r * NP + b) * MU + a]), xr[r * MU + a], dx);
        float tj = 0.f;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < NT; ++j) s = fmaf(__ldg(&R.Ehat[(e * NT + j) * MU + b]), jmp[e * NT + j], s);
            tj += gg[5 + e] * s;
        }
        const float y = detJ * dx + tau * tj;
        yp[(size_t)cell * NP + b] = (double)y;
        if (yp32) yp32[(size_t)cell * NP + b] = y;
    }
    // the cell's contributions to its facets' trace rows (canonical orientation):
    // yl = h_e ((L_j, Q.n)_e + tau J_ej)
    TFOR(ej, NL) {
        const int e = ej / NT, j = ej % NT;
        const float nx = __ldg(&E.nrm[6 * cell + 2 * e]), ny = __ldg(&E.nrm[6 * cell + 2 * e + 1]);
        float ex = 0.f;
#pragma unroll 7
        for (int a = 0; a < MU; ++a)
            ex = fmaf(__ldg(&R.Ehat[(e * NT + j) * MU + a]), nx * xK[a] + ny * xK[MU + a], ex);
        const float s = (__ldg(&M.cell_flip[3 * cell + e]) && (j & 1)) ? -1.f : 1.f;
        v[(size_t)cell * NL + ej] = (double)(s * gg[5 + e] * (ex + tau * jmp[ej]));
    }
    if (zslot) {                        // the input x also stored as slot gs->j of the FGMRES's Z
        const long long nQ = (long long)M.ncells * NU, nPv = (long long)M.ncells * NP;
        double *zj = zslot + (size_t)*zslot_j * (size_t)(nQ + nPv + (long long)M.nfacets * NT);
        TFOR(x, NU) zj[(size_t)cell * NU + x] = Q[(size_t)cell * NU + x];
        TFOR(b, NP) zj[nQ + (size_t)cell * NP + b] = p[(size_t)cell * NP + b];
        TFOR(i, 3 * NT) {               // each facet's values once, by its first cell
            const int f = M.cell_facet[3 * cell + i / NT];
            if (M.facet_cell[2 * f] == cell) zj[nQ + nPv + (size_t)f * NT + i % NT] = lam[(size_t)f * NT + i % NT];
        }
    }
}

}  // namespace hdg
