// One inexact Step-I solve (Alg. 2 Step I inside the stage preconditioner) as a single persistent
// cooperative kernel: one GMRES(GM_M) cycle from x = 0 in FP32 with block-Jacobi right
// preconditioning and the matrix-free neighbour coupling, stopping at rtol or after GM_M steps.
// It computes what the multi-kernel FP32 path (k_gm_start<float> ... k_gm_update_x<K, float>)
// computes, with grid-wide barriers between the phases instead of kernel boundaries.
//
// Barriers. The kernel is launched cooperatively (all blocks resident; the launch fails instead
// of running if they cannot be). A barrier is an arrival counter and a generation word in global
// memory; waiting blocks poll the generation with a bounded number of polls. A block that runs
// out of polls raises the error flag, every block returns at its next barrier, and the host
// reports the flag as an error: no wait can be endless.
//
// Reductions. Every block writes its partial sums, passes a barrier, and then sums all blocks'
// partials in the same fixed order, so that every block holds bit-identical scalars (the
// Hessenberg column, norms, Givens rotations) without a further barrier. Deterministic.
#pragma once
#include "hdg_kernels.cuh"

namespace hdg {

struct GridBar {
    unsigned int count;
    unsigned int gen;
    int error;
    int pad;
};

constexpr long long GRID_BAR_POLLS = 1ll << 22;   // ~0.5 s of polling before giving up

// All threads of all blocks call it; returns false if the barrier failed (then return at once).
__device__ __forceinline__ bool grid_barrier(GridBar *bar) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile GridBar *vb = bar;
        const unsigned g = vb->gen;
        __threadfence();
        if (atomicAdd(&bar->count, 1u) == gridDim.x - 1) {
            bar->count = 0;
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            long long polls = 0;
            while (vb->gen == g) {
                if (vb->error || ++polls > GRID_BAR_POLLS) {
                    atomicExch(&bar->error, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

struct StepI32Args {
    EdgeTab<float> E;
    MeshDev M;
    const float *Binv, *wq;
    float *V, *utr, *w;
    const double *b;
    double *x;
    double *partials;          // >= gridDim.x * 32 doubles
    GridBar *bar;
    GmresState *gs;            // rtol, maxit in; statistics out (total, converged, breakdown)
};

// the cell groups (TEAMS_PER_BLOCK-cell groups blockIdx.x, blockIdx.x + gridDim.x, ...) of a block
#define FOR_MY_CELLS(cell, ncells)                                                                   \
    for (int base_ = blockIdx.x * (int)(blockDim.x / TEAM_LANES); base_ < (ncells);                 \
         base_ += gridDim.x * (int)(blockDim.x / TEAM_LANES))                                        \
        for (int cell = base_ + (int)(threadIdx.x / TEAM_LANES), once_ = 1; once_; once_ = 0)

// fixed-order sum over the blocks of partial slot i (every block calls it; one warp per value)
__device__ __forceinline__ void sum_partials(const double *partials, int nvals, double *out_sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < nvals; i += nw) {
        double a = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) a += __ldcg(&partials[b * 32 + i]);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) out_sm[i] = a;
    }
    __syncthreads();
}

// block-wide sum of one double (all threads call; result valid in every thread)
__device__ __forceinline__ double block_total(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += sh[i];
    return t;
}

template <int K>
__global__ void __launch_bounds__(128) k_stepI32_persistent(StepI32Args A) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NFQ = Dm::NFQ;
    constexpr int TPB = 128 / TEAM_LANES;
    constexpr int TS = (2 * NU > 6 * NFQ) ? 2 * NU : 6 * NFQ;
    __shared__ float tsm[TPB * TS];
    __shared__ double H[(GM_M + 1) * GM_M], cs[GM_M], sn[GM_M], gv[GM_M + 1], yv[GM_M], hc[32];
    __shared__ double scal[2];
    const int team = threadIdx.x / TEAM_LANES;
    const Team tm{(int)(threadIdx.x % TEAM_LANES), TEAM_LANES};
    float *ts = tsm + team * TS;
    const MeshDev &M = A.M;
    const int ncells = M.ncells;
    const long long n = (long long)ncells * NU;
    const long long rows_per_group = (long long)TPB * NU;
    const double rtol = A.gs->rtol;
    const int m = A.gs->maxit < GM_M ? (A.gs->maxit > 0 ? A.gs->maxit : 1) : GM_M;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;

    // w = b (FP32), beta = ||w||
    double part = 0.0;
    FOR_MY_CELLS(cell, ncells) if (cell < ncells) {
        TFOR(r, NU) {
            const size_t gi = (size_t)cell * NU + r;
            const float v = (float)A.b[gi];
            A.w[gi] = v;
            part += (double)v * (double)v;
        }
    }
    part = block_total(part);
    if (threadIdx.x == 0) A.partials[blockIdx.x * 32] = part;
    if (!grid_barrier(A.bar)) return;
    sum_partials(A.partials, 1, scal);
    const double beta = sqrt(scal[0]);
    if (threadIdx.x == 0) {
        for (int i = 0; i <= GM_M; ++i) gv[i] = 0.0;
        gv[0] = beta;
    }
    __syncthreads();
    int k = 0, breakdown = 0;
    bool done = !(beta > 0.0) || !isfinite(beta);
    if (!isfinite(beta)) breakdown = 2;
    double hprev = beta;
    for (int j = 0; j < m && !done; ++j) {
        const float *Vj = A.V + (size_t)j * n;
        // v_j = w / h; z = Binv v_j; z's edge values
        const float inv = (float)(1.0 / hprev);
        FOR_MY_CELLS(cell, ncells) if (cell < ncells) {
            float *vK = ts, *zK = ts + NU;
            TFOR(r, NU) {
                const size_t gi = (size_t)cell * NU + r;
                const float v = A.w[gi] * inv;
                A.V[(size_t)j * n + gi] = v;
                vK[r] = v;
            }
            tm.sync();
            TFOR(r, NU) {
                const size_t gi = (size_t)cell * NU + r;
                float acc = 0.f;
#pragma unroll 6
                for (int q = 0; q < NU; ++q) acc += __ldg(&A.Binv[(size_t)q * n + gi]) * vK[q];
                zK[r] = acc;
            }
            tm.sync();
            TFOR(i, 3 * NFQ * 2) {
                const int d = i & 1, p = i >> 1;
                const float *ph = &A.E.ephi[p * MU];
                float s = 0.f;
#pragma unroll 5
                for (int bb = 0; bb < MU; ++bb) s += __ldg(ph + bb) * zK[d * MU + bb];
                A.utr[(size_t)cell * 3 * NFQ * 2 + i] = s;
            }
            tm.sync();
        }
        if (!grid_barrier(A.bar)) return;
        // w = v_j + coupling(z); dots with V_0..V_j over this block's rows
        FOR_MY_CELLS(cell, ncells) if (cell < ncells) {
            team_nbr_flux<K, float>(tm, A.E, M, cell, A.wq, A.utr, nullptr, ts);
            tm.sync();
            TFOR(r, NU) {
                const size_t gi = (size_t)cell * NU + r;
                A.w[gi] = Vj[gi] + nbr_row<K, float>(A.E, ts, r / MU, r % MU);
            }
            tm.sync();
        }
        __syncthreads();
        for (int i = warp; i <= j; i += nw) {
            const float *Vi = A.V + (size_t)i * n;
            float at = 0.f;
            for (long long g0 = blockIdx.x * rows_per_group; g0 < n; g0 += gridDim.x * rows_per_group) {
                const long long g1 = g0 + rows_per_group < n ? g0 + rows_per_group : n;
                for (long long r = g0 + lane; r < g1; r += 32) at += Vi[r] * A.w[r];
            }
            double a = (double)at;
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) A.partials[blockIdx.x * 32 + i] = a;
        }
        if (!grid_barrier(A.bar)) return;
        sum_partials(A.partials, j + 1, hc);
        // w -= V hcol (one classical Gram-Schmidt pass), ||w||
        part = 0.0;
        for (long long g0 = blockIdx.x * rows_per_group; g0 < n; g0 += gridDim.x * rows_per_group) {
            const long long g1 = g0 + rows_per_group < n ? g0 + rows_per_group : n;
            for (long long r = g0 + threadIdx.x; r < g1; r += blockDim.x) {
                float s = A.w[r];
                for (int i = 0; i <= j; ++i) s -= (float)hc[i] * A.V[(size_t)i * n + r];
                A.w[r] = s;
                part += (double)s * (double)s;
            }
        }
        part = block_total(part);
        if (threadIdx.x == 0) A.partials[blockIdx.x * 32 + 31] = part;
        if (!grid_barrier(A.bar)) return;
        if (warp == 0) {
            double a = 0.0;
            for (int bb = lane; bb < (int)gridDim.x; bb += 32) a += __ldcg(&A.partials[bb * 32 + 31]);
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) scal[1] = a;
        }
        __syncthreads();
        const double hn = sqrt(scal[1]);
        if (threadIdx.x == 0) {             // Hessenberg column, Givens rotations (same in every block)
            double *Hc = H + j * (GM_M + 1);
            for (int i = 0; i <= j; ++i) Hc[i] = hc[i];
            Hc[j + 1] = hn;
            for (int i = 0; i < j; ++i) {
                const double a = Hc[i], b2 = Hc[i + 1];
                Hc[i] = cs[i] * a + sn[i] * b2;
                Hc[i + 1] = -sn[i] * a + cs[i] * b2;
            }
            const double a = Hc[j], b2 = Hc[j + 1];
            const double r = sqrt(a * a + b2 * b2);
            const double c_ = r > 0 ? a / r : 1.0, s_ = r > 0 ? b2 / r : 0.0;
            cs[j] = c_; sn[j] = s_;
            Hc[j] = r;
            Hc[j + 1] = 0.0;
            gv[j + 1] = -s_ * gv[j];
            gv[j] = c_ * gv[j];
        }
        __syncthreads();
        k = j + 1;
        hprev = hn;
        const double resid = fabs(gv[j + 1]);
        if (!isfinite(resid)) { breakdown = 2; done = true; }
        else if (resid <= rtol * beta || hn == 0.0) done = true;
    }
    // y = R^{-1} g; x = Binv (V y)
    if (threadIdx.x == 0) {
        for (int i = k - 1; i >= 0; --i) {
            double s = gv[i];
            for (int kk = i + 1; kk < k; ++kk) s -= H[kk * (GM_M + 1) + i] * yv[kk];
            const double d = H[i * (GM_M + 1) + i];
            yv[i] = d != 0.0 ? s / d : 0.0;
        }
    }
    __syncthreads();
    FOR_MY_CELLS(cell, ncells) if (cell < ncells) {
        TFOR(r, NU) {
            const size_t gi = (size_t)cell * NU + r;
            float s = 0.f;
            for (int i = 0; i < k; ++i) s += (float)yv[i] * A.V[(size_t)i * n + gi];
            ts[r] = s;
        }
        tm.sync();
        TFOR(r, NU) {
            const size_t gi = (size_t)cell * NU + r;
            float a = 0.f;
#pragma unroll 6
            for (int q = 0; q < NU; ++q) a += __ldg(&A.Binv[(size_t)q * n + gi]) * ts[q];
            A.x[gi] = (double)a;
        }
        tm.sync();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        GmresState *gs = A.gs;
        gs->bnorm = beta;
        gs->total = k;
        gs->j = k;
        gs->resid = k > 0 ? fabs(gv[k]) : beta;
        gs->converged = (k > 0 && fabs(gv[k]) <= rtol * beta) || !(beta > 0.0);
        gs->breakdown = breakdown;
        gs->cycle_end = 1;
    }
}

// barrier state before a launch; after it, a failed barrier counts as a breakdown
__global__ void k_bar_reset(GridBar *bar) {
    wait_prior_kernel();
    bar->count = 0;
    bar->error = 0;
}
__global__ void k_bar_check(const GridBar *bar, DevCount *acc) {
    wait_prior_kernel();
    if (bar->error) acc->breakdowns += 1;
}

}  // namespace hdg
