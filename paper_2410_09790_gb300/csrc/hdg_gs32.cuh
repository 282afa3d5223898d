// Red-black block Gauss-Seidel right preconditioner for the FP32 inner Step-I GMRES.
//
// The colour passes are bound by reading the FP32 block inverses (NU x NU per cell, 7 KB at
// k = 4). They are stored for these passes as one contiguous block per cell (GsBlk: column-major,
// rows padded to a multiple of 4, blocks padded to 128 bytes) in colour-major order (gs_slot),
// and a warp applies its cell's block with 16-byte loads: lane s*G + g holds row group g (rows
// 4g..4g+3) of the columns q = s, s + S, ..., so each load instruction of the warp covers
// consecutive columns of one block (352 contiguous bytes at k = 4), and the S partial sums of a
// row group are added by shuffles in a fixed order.
//
// On the structured triangulation every cell's three neighbours have the other index parity
// (each square's lower and upper triangle; checked on the host before use), so the even cells
// ("red") and the odd cells ("black") split the Step-I operator A = D + N (D: the cells' diagonal
// blocks, N: the neighbour coupling) into
//     A = [[D_R, N_RB], [N_BR, D_B]].
// The preconditioner solves the block lower triangle: z_R = D_R^-1 v_R, z_B = D_B^-1 (v_B - N_BR z_R).
// Then A z = v + [N_RB z_B; 0]: the Arnoldi product needs the coupling on the red rows only. The
// paper's Step I uses ILU(0) inside GMRES; this is the same idea (a triangular solve with the
// operator's blocks) in the form whose two halves are each fully parallel. Per Arnoldi step:
//   k_gs_diag(red), k_gs_diag(black), k_gs_apply, k_gm_finish_ctl
// and at the end of the cycle the same two-colour solve for x = P^-1 (V y) (k_gs_combine x2).
#pragma once
#include "hdg_kernels.cuh"

namespace hdg {

// the cell of colour col handled by this warp: the warps of a block take consecutive same-colour
// cells
#define GS_CELL(COL)                                                                 \
    const int team = threadIdx.x >> 5, tpb = blockDim.x >> 5;                        \
    const int cell = 2 * (blockIdx.x * tpb + team) + (COL);                          \
    Team tm{(int)(threadIdx.x & 31), 32};

// edge values of the cell's z (zK: its NU coefficients in shared memory) -> utr
template <int K>
__device__ __forceinline__ void team_edge_values(const Team &tm, const EdgeTab<float> &E, int cell, const float *zK,
                                                 float *utr) {
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NFQ = Dm::NFQ;
    TFOR(i, 3 * NFQ * 2) {
        const int d = i & 1, p = i >> 1;            // p = e*NFQ + q
        const float *ph = &E.ephi[p * MU];
        float s = 0.f;
#pragma unroll 5
        for (int b = 0; b < MU; ++b) s += __ldg(ph + b) * zK[d * MU + b];
        utr[(size_t)cell * 3 * NFQ * 2 + i] = s;
    }
}

// Colour col of the preconditioner at Arnoldi step j: v_j = (w - sum_{i<j} h_i V_i) / h on the
// colour's cells -> V_j; col 0: z = D^-1 v; col 1: z = D^-1 (v - N z_red) (the red neighbours'
// edge values from the col-0 pass); z's edge values -> utr.
template <int K>
__global__ void k_gs_diag(EdgeTab<float> E, MeshDev M, const float *__restrict__ Binv, const float *__restrict__ w,
                          float *V, float *utr, const float *__restrict__ wq, const GmresState *gs, int col) {
    wait_prior_kernel();
    if (gs->cycle_end) return;
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NFQ = Dm::NFQ;
    constexpr int SCR = 2 * NU + 6 * NFQ;
    __shared__ float hproj[GM_M + 2];
    GS_CELL(col)
    float4 pre[GsPre<K>::NC];                   // the block read ahead (small K)
    if constexpr (GsPre<K>::ON)
        if (cell < M.ncells) warp_block_prefetch<K>(Binv, gs_slot(cell, M.ncells), pre);
    const int j = gs->j;
    if ((int)threadIdx.x < j) hproj[threadIdx.x] = gs->hcol32[threadIdx.x];
    __syncthreads();
    extern __shared__ double smd[];
    if (cell >= M.ncells) return;
    float *vK = reinterpret_cast<float *>(smd) + team * SCR, *zK = vK + NU, *t = zK + NU;
    const float inv = gs->inv32;
    const long long nrows = (long long)M.ncells * NU;
    float *vj = V + (size_t)j * nrows;
    TFOR(r, NU) {
        const size_t gi = (size_t)cell * NU + r;
        float wv = w[gi];
        for (int i = 0; i < j; ++i) wv -= hproj[i] * V[(size_t)i * nrows + gi];
        const float v = wv * inv;
        vj[gi] = v;
        vK[r] = v;
    }
    if (col == 1) {                     // v_B - N_BR z_R
        tm.sync();
        team_nbr_flux<K, float>(tm, E, M, cell, wq, utr, nullptr, t);
        tm.sync();
        TFOR(r, NU) vK[r] -= nbr_row<K, float>(E, t, r / MU, r % MU);
    }
    tm.sync();
    if constexpr (GsPre<K>::ON) warp_block_apply_pre<K>(pre, vK, zK);
    else warp_block_apply<K>(Binv, gs_slot(cell, M.ncells), vK, zK);
    tm.sync();
    team_edge_values<K>(tm, E, cell, zK, utr);
}

// Arnoldi product for the Gauss-Seidel preconditioner: w = v_j + N_RB z_B on the red cells,
// w = v_j on the black cells; then the FP32 block partials of the dots with V_0..V_j and ||w||^2
// (summed by k_gm_finish_ctl). Teams take consecutive cells (their rows are the block's rows).
template <int K>
__global__ void k_gs_apply(EdgeTab<float> E, MeshDev M, const float *__restrict__ wq, const float *__restrict__ utr,
                           float *w, const float *__restrict__ V, RedBuf rb, GmresState *gs) {
    wait_prior_kernel();
    if (gs->cycle_end) return;
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NFQ = Dm::NFQ;
    extern __shared__ double smd[];
    const int team = threadIdx.x / TEAM_LANES, tpb = blockDim.x / TEAM_LANES;
    Team tm{(int)(threadIdx.x % TEAM_LANES), TEAM_LANES};
    float *t = reinterpret_cast<float *>(smd) + team * (6 * NFQ);
    const long long nrows = (long long)M.ncells * NU;
    const int j = gs->j;
    const float *vj = V + (size_t)j * nrows;
    for (int base = blockIdx.x * tpb; base < M.ncells; base += gridDim.x * tpb) {
        const int cell = base + team;
        if (cell < M.ncells) {
            // a warp holds one red and one black team: both execute the same barriers (a team
            // sync is a whole-warp __syncwarp)
            const bool red = (cell & 1) == 0;
            if (red) team_nbr_flux<K, float>(tm, E, M, cell, wq, utr, nullptr, t);
            tm.sync();
            TFOR(r, NU) {
                const size_t gi = (size_t)cell * NU + r;
                w[gi] = red ? vj[gi] + nbr_row<K, float>(E, t, r / MU, r % MU) : vj[gi];
            }
            tm.sync();
        }
    }
    constexpr int RPG = (128 / TEAM_LANES) * NU;                 // the rows of a 128-thread block's cells
    if (tpb * NU == RPG) multidot_groups_partials_f32<RPG>(rb, V, (const float *)w, nrows, j + 1, true);
    else multidot_groups_partials(rb, V, (const float *)w, nrows, (long long)tpb * NU, j + 1, true);
}

// End of an inner cycle, colour col: u = V y on the colour's cells; col 0: x = D^-1 u, x's edge
// values -> utr; col 1: x = D^-1 (u - N x_red); col 1 also counts the solve in acc.
template <int K>
__global__ void k_gs_combine(EdgeTab<float> E, MeshDev M, const float *__restrict__ V, const float *__restrict__ Binv,
                             const float *__restrict__ wq, float *utr, double *x, const GmresState *gs, DevCount *acc,
                             int col) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NFQ = Dm::NFQ;
    constexpr int SCR = 2 * NU + 6 * NFQ;
    __shared__ float ys[GM_M];
    const int m = gs->j;
    if ((int)threadIdx.x < m) ys[threadIdx.x] = gs->y32[threadIdx.x];
    if (col == 1 && acc && blockIdx.x == 0 && threadIdx.x == 0) { acc->stepI_iters += gs->total; acc->stepI_solves += 1; }
    __syncthreads();
    extern __shared__ double smd[];
    GS_CELL(col)
    if (cell >= M.ncells) return;
    float *uK = reinterpret_cast<float *>(smd) + team * SCR, *xK = uK + NU, *t = xK + NU;
    const long long nrows = (long long)M.ncells * NU;
    TFOR(r, NU) {
        const size_t gi = (size_t)cell * NU + r;
        float s = 0.f;
        for (int i = 0; i < m; ++i) s += ys[i] * V[(size_t)i * nrows + gi];
        uK[r] = s;
    }
    if (col == 1) {
        tm.sync();
        team_nbr_flux<K, float>(tm, E, M, cell, wq, utr, nullptr, t);
        tm.sync();
        TFOR(r, NU) uK[r] -= nbr_row<K, float>(E, t, r / MU, r % MU);
    }
    tm.sync();
    warp_block_apply<K>(Binv, gs_slot(cell, M.ncells), uK, xK);
    tm.sync();
    TFOR(r, NU) x[(size_t)cell * NU + r] = (double)xK[r];
    if (col == 0) {
        tm.sync();
        team_edge_values<K>(tm, E, cell, xK, utr);
    }
}

}  // namespace hdg
