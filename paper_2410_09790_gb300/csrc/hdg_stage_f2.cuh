// The stage operator y = A(c) x of the stage flexible GMRES (restart residuals and the Arnoldi
// products taken before the relaxed FP32 ones) in pair arithmetic (hdg_df64.cuh), HDG_MIXED.
//
// Same operator and outputs as the FP64 kernel k_stage_apply (Sec. 2.7: velocity rows
// (M - cF)Q - c G(p, lambda), the cell's pressure rows and its contributions to the trace rows),
// to about 2^-46 of the terms' magnitudes instead of FP64's 2^-53: far below the 1e-10 stage
// tolerance these products serve. A warp per cell as in k_stage_apply32: the FP64 inputs are split
// into pairs in shared memory once, the diagonal block is read as its FP32 rounding (hi) and the
// rest (lo) in the per-cell layout GsBlk with 16-byte loads, the reference tables as pairs, the
// geometry, normals, weights and penalty from their FP64 copies. The constraint rows are taken
// through the facet jumps J_ej = (L_j, p)_e - lambda_ej as in k_stage_apply32.
#pragma once
#include "hdg_df64.cuh"
#include "hdg_stage32.cuh"

namespace hdg {

// reference tables as pairs (layouts as in RefDev): facet-point values, Ehat, Dhat
struct RefF2 {
    const float2 *ephi, *Ehat, *Dhat;
};

// pairs of the per-cell scratch of k_stage_apply_f2 (a warp per cell)
template <int K>
constexpr int stage_f2_scratch() {
    typedef Dims<K> Dm;
    return 5 * Dm::NU + Dm::NP + 2 * Dm::NL + 6 * Dm::NFQ + 5 * Dm::MU + 14 + Dm::NFQ;
}

// z = D v for the block D = hi + lo of cell `cell` (GsBlk layout, slot = cell), in pairs: v in
// shared memory (NU pairs), z's NU pairs written to shared memory. Lane s*G + g sums the columns
// q = s, s + S, ... of rows 4g..4g+3; the S partial sums of a row group are added in order.
template <int K>
__device__ __forceinline__ void warp_block_apply_f2(const float *__restrict__ Dhi, const float *__restrict__ Dlo,
                                                    long long cell, const f2 *v, f2 *z) {
    typedef GsBlk<K> B;
    const int lane = (int)(threadIdx.x & 31), g = lane % B::G, s = lane / B::G;
    const float4 *bh = reinterpret_cast<const float4 *>(Dhi + (size_t)cell * B::SIZE);
    const float4 *bl = reinterpret_cast<const float4 *>(Dlo + (size_t)cell * B::SIZE);
    acc2 a0, a1, a2, a3;
    if (s < B::S) {
#pragma unroll 2
        for (int q = s; q < B::NU; q += B::S) {
            const float4 h = __ldg(bh + q * (B::NUP / 4) + g), l = __ldg(bl + q * (B::NUP / 4) + g);
            const f2 vq = v[q];
            a0.fma(f2{h.x, l.x}, vq); a1.fma(f2{h.y, l.y}, vq);
            a2.fma(f2{h.z, l.z}, vq); a3.fma(f2{h.w, l.w}, vq);
        }
    }
    acc2 t0, t1, t2, t3;
#pragma unroll
    for (int s2 = 0; s2 < B::S; ++s2) {             // the subsets' partial sums, in order
        const int src = s2 * B::G + g;
        t0.add(f2{__shfl_sync(0xffffffffu, a0.h, src), __shfl_sync(0xffffffffu, a0.l, src)});
        t1.add(f2{__shfl_sync(0xffffffffu, a1.h, src), __shfl_sync(0xffffffffu, a1.l, src)});
        t2.add(f2{__shfl_sync(0xffffffffu, a2.h, src), __shfl_sync(0xffffffffu, a2.l, src)});
        t3.add(f2{__shfl_sync(0xffffffffu, a3.h, src), __shfl_sync(0xffffffffu, a3.l, src)});
    }
    if (s == 0) {
        const int r = 4 * g;
        if (r < B::NU) z[r] = t0.get();
        if (r + 1 < B::NU) z[r + 1] = t1.get();
        if (r + 2 < B::NU) z[r + 2] = t2.get();
        if (r + 3 < B::NU) z[r + 3] = t3.get();
    }
}

// rest of the block's FP64 value: lo = D - fl32(D) in the layout of the FP32 copy (GsBlk, slot =
// cell); Dblk in the column-slice layout [col * nrows + cell * NU + row]
template <int K>
__global__ void k_blocks_lo(const double *__restrict__ Dblk, float *__restrict__ Dlo, long long ncells) {
    wait_prior_kernel();
    typedef GsBlk<K> B;
    const long long nrows = ncells * B::NU;
    GRID_STRIDE(i, ncells * B::SIZE) {
        const long long cell = i / B::SIZE;
        const int o = (int)(i % B::SIZE), q = o / B::NUP, r = o % B::NUP;
        float lo = 0.f;
        if (q < B::NU && r < B::NU) {
            const double d = Dblk[(size_t)q * nrows + (size_t)cell * B::NU + r];
            lo = (float)(d - (double)(float)d);
        }
        Dlo[i] = lo;
    }
}

// y = A(c) x in pairs; x = (Q, p, lambda) and the outputs in FP64 memory as in k_stage_apply (yQ,
// yp, the cell's lambda-row contributions v, the FP32 shadows yQ32 / yp32 when set, and the copy
// of x into the FGMRES's preconditioned-vector slot *zslot_j when set). skip (optional): return
// at once when *skip is set (k_stage_apply32 takes that product). Dhi, Dlo: the diagonal block's
// FP32 rounding and rest (GsBlk, slot = cell); wq, pen: the assembly's FP64 weights; cf, tf: the
// stage coefficient c and the stabilisation tau as pairs.
template <int K>
__global__ void __launch_bounds__(128) k_stage_apply_f2(RefF2 T, const double *__restrict__ pen, MeshDev M,
                                                        const float *__restrict__ Dhi, const float *__restrict__ Dlo,
                                                        const double *__restrict__ wq, f2 cf, f2 tf,
                                                        const double *Q, const double *p, const double *lam, double *yQ,
                                                        double *yp, double *v, float *yQ32, float *yp32, double *zslot,
                                                        const int *zslot_j, const int *skip) {
    wait_prior_kernel();
    if (skip && *skip) return;
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NP = Dm::NP, NT = Dm::NT, NL = Dm::NL, NFQ = Dm::NFQ;
    extern __shared__ double sm[];
    const int team = threadIdx.x >> 5;
    const int cell = blockIdx.x * STAGE32_WARPS + team;
    if (cell >= M.ncells) return;
    Team tm{(int)(threadIdx.x & 31), 32};
    f2 *xK = reinterpret_cast<f2 *>(sm) + (size_t)team * stage_f2_scratch<K>();   // own Q (NU)
    f2 *xn = xK + NU;                                        // neighbours' Q (3 x NU)
    f2 *pK = xn + 3 * NU, *lK = pK + NP, *t = lK + NL, *xr = t + 6 * NFQ;
    f2 *nq = xr + 2 * MU;                                    // n_e . Q at the coefficients (3 x MU)
    f2 *gg = nq + 3 * MU;                                    // Jinv[4], detJ, h[3], nx[3], ny[3]
    f2 *jmp = gg + 14, *dq = jmp + NL, *pn = dq + NU;
    const int *nbr = M.cell_nbr + 3 * cell;
    TFOR(i, NU) xK[i] = f2_of(Q[(size_t)cell * NU + i]);
    TFOR(i, 3 * NU) {
        const int o = __ldg(&nbr[i / NU]);
        xn[i] = o >= 0 ? f2_of(Q[(size_t)o * NU + i % NU]) : f2{0.f, 0.f};
    }
    TFOR(b, NP) pK[b] = f2_of(p[(size_t)cell * NP + b]);
    TFOR(i, NL) {
        const int e = i / NT, j = i % NT;
        const int f = __ldg(&M.cell_facet[3 * cell + e]);
        const double l = (__ldg(&M.cell_flip[3 * cell + e]) && (j & 1)) ? -lam[(size_t)f * NT + j] : lam[(size_t)f * NT + j];
        lK[i] = f2_of(l);
    }
    TFOR(q, NFQ) pn[q] = f2_of(__ldg(&pen[q]));
    if (tm.tid < 14) {
        const CellGeo &G = M.geo[cell];
        const int i = tm.tid;
        const double g = i < 4 ? G.Jinv[i] : (i == 4 ? G.detJ : (i < 8 ? G.h[i - 5] : (i < 11 ? G.nx[i - 8] : G.ny[i - 11])));
        gg[i] = f2_of(g);
    }
    tm.sync();
    TFOR(i, NL) {                                            // the facet jumps
        acc2 s;
        s.add(f2_neg(lK[i]));
#pragma unroll
        for (int b = 0; b < NP; ++b) s.fma(f2_of(__ldg(&T.Ehat[i * MU + b])), pK[b]);
        jmp[i] = s.get();
    }
    TFOR(i, 3 * NFQ) {                                       // neighbour coupling at the edge points
        const int e = i / NFQ, q = i % NFQ;
        const int o = __ldg(&nbr[e]);
        f2 tx{0.f, 0.f}, ty{0.f, 0.f};
        if (o >= 0) {
            const int eo = __ldg(&M.cell_nbr_edge[3 * cell + e]), qo = NFQ - 1 - q;
            const float2 *ph = &T.ephi[(eo * NFQ + qo) * MU];
            const f2 *xo = xn + e * NU;
            acc2 ux, uy;
#pragma unroll 7
            for (int b = 0; b < MU; ++b) {
                const f2 f = f2_of(__ldg(ph + b));
                ux.fma(f, xo[b]);
                uy.fma(f, xo[MU + b]);
            }
            const f2 uxv = ux.get(), uyv = uy.get(), nx = gg[8 + e], ny = gg[11 + e];
            const f2 un = f2_add(f2_mul(nx, uxv), f2_mul(ny, uyv));
            const f2 w = f2_of(__ldg(&wq[(size_t)cell * 3 * NFQ + i]));
            const f2 pu = f2_mul(pn[q], un);
            tx = f2_add(f2_mul(pu, nx), f2_mul(w, uxv));
            ty = f2_add(f2_mul(pu, ny), f2_mul(w, uyv));
        }
        t[2 * i] = tx;
        t[2 * i + 1] = ty;
    }
    TFOR(a, MU) {                                            // Jinv^T-mapped velocity for the p-rows
        xr[a] = f2_add(f2_mul(gg[0], xK[a]), f2_mul(gg[1], xK[MU + a]));
        xr[MU + a] = f2_add(f2_mul(gg[2], xK[a]), f2_mul(gg[3], xK[MU + a]));
    }
    TFOR(i, 3 * MU) {                                        // n_e . Q for the trace rows
        const int e = i / MU, a = i % MU;
        nq[i] = f2_add(f2_mul(gg[8 + e], xK[a]), f2_mul(gg[11 + e], xK[MU + a]));
    }
    tm.sync();
    warp_block_apply_f2<K>(Dhi, Dlo, cell, xK, dq);
    tm.sync();
    const f2 detJ = gg[4];
    // velocity rows: (M - cF) Q (diagonal block dense, neighbours from t) - c (detJ Jinv-mapped
    // Dhat^T p - sum_e h_e n_e Ehat^T lambda)
    TFOR(x, NU) {
        const int d = x / MU, a = x % MU;
        const size_t gi = (size_t)cell * NU + x;
        acc2 bq;
#pragma unroll 8
        for (int i = 0; i < 3 * NFQ; ++i) bq.fma(f2_of(__ldg(&T.ephi[i * MU + a])), t[2 * i + d]);
        bq.add(dq[x]);
        acc2 et;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            acc2 s;
#pragma unroll
            for (int j = 0; j < NT; ++j) s.fma(f2_of(__ldg(&T.Ehat[(e * NT + j) * MU + a])), lK[e * NT + j]);
            et.fma(f2_mul(gg[5 + e], gg[(d == 0 ? 8 : 11) + e]), s.get());
        }
        acc2 dt;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            acc2 s;
#pragma unroll
            for (int b = 0; b < NP; ++b) s.fma(f2_of(__ldg(&T.Dhat[(rr * NP + b) * MU + a])), pK[b]);
            dt.fma(gg[rr * 2 + d], s.get());
        }
        const f2 yv = f2_sub(bq.get(), f2_mul(cf, f2_sub(f2_mul(detJ, dt.get()), et.get())));
        const double yd = f2_dbl(yv);
        yQ[gi] = yd;
        if (yQ32) yQ32[gi] = (float)yd;
    }
    // the cell's pressure rows: yp = detJ D Q + tau sum_e h_e sum_j Ehat[e j b] J_ej
    TFOR(b, NP) {
        acc2 dx;
        for (int r = 0; r < 2; ++r)
#pragma unroll 7
            for (int a = 0; a < MU; ++a) dx.fma(f2_of(__ldg(&T.Dhat[(r * NP + b) * MU + a])), xr[r * MU + a]);
        acc2 tj;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            acc2 s;
#pragma unroll
            for (int j = 0; j < NT; ++j) s.fma(f2_of(__ldg(&T.Ehat[(e * NT + j) * MU + b])), jmp[e * NT + j]);
            tj.fma(gg[5 + e], s.get());
        }
        const double y = f2_dbl(f2_add(f2_mul(detJ, dx.get()), f2_mul(tf, tj.get())));
        yp[(size_t)cell * NP + b] = y;
        if (yp32) yp32[(size_t)cell * NP + b] = (float)y;
    }
    // the cell's contributions to its facets' trace rows (canonical orientation):
    // yl = h_e ((L_j, Q.n)_e + tau J_ej)
    TFOR(ej, NL) {
        const int e = ej / NT, j = ej % NT;
        acc2 ex;
#pragma unroll 7
        for (int a = 0; a < MU; ++a) ex.fma(f2_of(__ldg(&T.Ehat[(e * NT + j) * MU + a])), nq[e * MU + a]);
        const double s = (__ldg(&M.cell_flip[3 * cell + e]) && (j & 1)) ? -1.0 : 1.0;
        v[(size_t)cell * NL + ej] = s * f2_dbl(f2_mul(gg[5 + e], f2_add(ex.get(), f2_mul(tf, jmp[ej]))));
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

// ------------------------------------------------------------------ BDM projection in pairs
// The canonical BDM_{k+1} interpolant Q* = P(Q) per cell (Sec. 2.3; cell_bdm's steps) in pair
// arithmetic for HDG_MIXED: the normal averages {Q}.n at the facet points (own and neighbour
// traces), their moments against the Legendre polynomials, the interior Nedelec moments, the
// local solve through the reference inverse moment matrix and the Piola map back. Tables as pairs
// (layouts as in RefDev): facet-point values, facet weights, Legendre values, interior moment
// tensor, inverse moment matrix.
struct BdmF2 {
    const float2 *ephi, *fw, *leg, *Iv, *inv;
};

template <int K>
constexpr int bdm_f2_scratch() {
    typedef Dims<K> Dm;
    return 4 * Dm::NU + Dm::NU + Dm::NU + 3 * Dm::NFQ + 2 * Dm::MU + 20;
}

template <int K>
__global__ void k_bdm_f2(BdmF2 T, MeshDev M, const double *Q, double *Qs) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NB = Dm::NB, NV = Dm::NV, NFQ = Dm::NFQ;
    extern __shared__ double sm[];
    const int team = threadIdx.x / TEAM_LANES;
    const int cell = (blockIdx.x * blockDim.x + threadIdx.x) / TEAM_LANES;
    if (cell >= M.ncells) return;
    Team tm{(int)(threadIdx.x % TEAM_LANES), TEAM_LANES};
    f2 *xq = reinterpret_cast<f2 *>(sm) + (size_t)team * bdm_f2_scratch<K>();   // own Q (NU)
    f2 *xo = xq + NU;                   // neighbours' Q (3 x NU)
    f2 *m = xo + 3 * NU, *qh = m + NU, *an = qh + NU, *r = an + 3 * NFQ;
    f2 *gg = r + 2 * MU;                // J[4], Jinv[4], detJ, 1/detJ, h[3], nx[3], ny[3], (0)
    const int *nbr = M.cell_nbr + 3 * cell;
    TFOR(i, NU) xq[i] = f2_of(Q[(size_t)cell * NU + i]);
    TFOR(i, 3 * NU) {
        const int o = __ldg(&nbr[i / NU]);
        xo[i] = o >= 0 ? f2_of(Q[(size_t)o * NU + i % NU]) : f2{0.f, 0.f};
    }
    TFOR(i, 20) {                       // (a 16-lane team: some lanes take two)
        const CellGeo &G = M.geo[cell];
        double v;
        if (i < 4) v = G.J[i];
        else if (i < 8) v = G.Jinv[i - 4];
        else if (i == 8) v = G.detJ;
        else if (i == 9) v = 1.0 / G.detJ;
        else if (i < 13) v = G.h[i - 10];
        else if (i < 16) v = G.nx[i - 13];
        else if (i < 19) v = G.ny[i - 16];
        else v = 0.0;
        gg[i] = f2_of(v);
    }
    tm.sync();
    TFOR(i, 3 * NFQ) {                  // h_e fw_q {Q}.n at the facet points (0 on walls)
        const int e = i / NFQ, q = i % NFQ;
        const int o = __ldg(&nbr[e]);
        f2 sv{0.f, 0.f};
        if (o >= 0) {
            const int eo = __ldg(&M.cell_nbr_edge[3 * cell + e]);
            const float2 *pk = &T.ephi[(e * NFQ + q) * MU], *po = &T.ephi[(eo * NFQ + (NFQ - 1 - q)) * MU];
            const f2 *xe = xo + e * NU;
            acc2 s0, s1;
#pragma unroll 7
            for (int a = 0; a < MU; ++a) {
                const f2 fk = f2_of(__ldg(pk + a)), fo = f2_of(__ldg(po + a));
                s0.fma(fk, xq[a]); s1.fma(fk, xq[MU + a]);
                s0.fma(fo, xe[a]); s1.fma(fo, xe[MU + a]);
            }
            const f2 un = f2_add(f2_mul(s0.get(), gg[13 + e]), f2_mul(s1.get(), gg[16 + e]));
            const f2 w = f2_mul(gg[10 + e], f2_of(__ldg(&T.fw[q])));
            sv = f2_mul(w, f2{0.5f * un.h, 0.5f * un.l});
        }
        an[i] = sv;
    }
    TFOR(a, MU) {                       // Jinv-mapped velocity for the interior moments
        r[a] = f2_add(f2_mul(gg[4], xq[a]), f2_mul(gg[5], xq[MU + a]));
        r[MU + a] = f2_add(f2_mul(gg[6], xq[a]), f2_mul(gg[7], xq[MU + a]));
    }
    tm.sync();
    TFOR(i, 3 * NB) {                   // edge moments against the Legendre polynomials
        const int e = i / NB, j = i % NB;
        acc2 s;
#pragma unroll
        for (int q = 0; q < NFQ; ++q) s.fma(an[e * NFQ + q], f2_of(__ldg(&T.leg[q * NB + j])));
        m[i] = s.get();
    }
    TFOR(v, NV) {                       // interior moments
        acc2 s;
#pragma unroll 7
        for (int a = 0; a < MU; ++a) {
            s.fma(r[a], f2_of(__ldg(&T.Iv[(a * NV + v) * 2])));
            s.fma(r[MU + a], f2_of(__ldg(&T.Iv[(a * NV + v) * 2 + 1])));
        }
        m[3 * NB + v] = f2_mul(gg[8], s.get());
    }
    tm.sync();
    TFOR(x, NU) {                       // reference coefficients through the inverse moment matrix
        acc2 s;
#pragma unroll 6
        for (int k = 0; k < NU; ++k) s.fma(f2_of(__ldg(&T.inv[x * NU + k])), m[k]);
        qh[x] = s.get();
    }
    tm.sync();
    TFOR(x, NU) {                       // Piola map back
        const int d = x / MU, a = x % MU;
        const f2 v = f2_add(f2_mul(gg[2 * d], qh[a]), f2_mul(gg[2 * d + 1], qh[MU + a]));
        Qs[(size_t)cell * NU + x] = f2_dbl(f2_mul(v, gg[9]));
    }
}

}  // namespace hdg
