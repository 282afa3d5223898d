// CUDA kernels of the HDG stage solver (sm_103a).
//
// Layouts (FP64):
//  * velocity-like vectors: [cell][NU], modal (hdg_cell.cuh); pressure [cell][NP];
//    trace [facet][NT] (Legendre, canonical facet direction).
//  * trace operator S = sum_K S_K in ELL form with 5 block columns per facet row block
//    (the facet itself and the two other facets of each side cell):
//        Sell[((b*NT + col) * nrows) + f*NT + row],  tcol[b*nfacets + f] (facet or -1);
//    a warp reads 32 consecutive rows of one (b, col) slice: fully coalesced.
//  * tentative-velocity operator M - cF: the diagonal blocks Dblk[col*nrowsQ + cell*NU + row];
//    the neighbour coupling matrix-free from wq[(cell*3 + e)*NFQ + q] (hdg_cell.cuh,
//    cell_fimpl_diag) and the cells' velocity values at their edge points,
//    utr[((cell*3 + e)*NFQ + q)*2 + d]. The loose (inner) Step-I solves use FP32 copies
//    (Binv32, wq32, utr32) and FP32 Krylov vectors.
//  * block-Jacobi inverses: Dinv[col*nrows + f*NT + row], Binv[col*nrowsQ + cell*NU + row].
// Reductions are deterministic: each block writes a partial, the last block to finish (atomic
// ticket, no waiting) sums the partials in a fixed order and updates the solver scalars.
#pragma once
#include <cuda_runtime.h>

#include "hdg_cell.cuh"

namespace hdg {

// Every kernel here is launched with programmatic dependent launch (launch_k in hdg_solver.cu):
// its blocks may be scheduled while the previous kernel on the stream finishes, so that the launch
// overlaps that kernel's tail. Each kernel first waits until the previous kernel has completed
// and its writes are visible; only then does it touch memory.
__device__ __forceinline__ void wait_prior_kernel() { cudaGridDependencySynchronize(); }

constexpr int VEC_THREADS = 256;
constexpr int MAX_RED_BLOCKS = 2048;

struct Scalars {
    double rz, rz0, pAp, alpha, beta, omega, rho, bnorm, rr, rv, ts, tt;
    double bmean, red0, red1, red2, zmean;
    int done, iters, breakdown, maxit;
    double rtol, relres;
    double zmean_old;       // flexible CG: the mean removed from the previous z
};

struct RedBuf {
    double *partials;
    unsigned int *counter;
};

// ------------------------------------------------------------------ block / grid reductions
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double x = v[i];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[i][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double x = (lane < nw) ? sh[i][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            v[i] = x;                                   // valid in thread 0
        }
    }
    __syncthreads();
}

// Returns true in thread 0 of the last block (ALL: in every thread of the last block), with the
// grid totals in tot (valid in thread 0).
template <int NV, bool ALL = false>
__device__ bool grid_sum(const RedBuf rb, double (&v)[NV], double (&tot)[NV]) {
    __shared__ double sh[NV][32];
    __shared__ int last;
    block_sum<NV>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) rb.partials[blockIdx.x * NV + i] = v[i];
        __threadfence();
        unsigned t = atomicAdd(rb.counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += __ldcg(&rb.partials[b * NV + i]);
    block_sum<NV>(acc, sh);
    if (threadIdx.x == 0) {
        *rb.counter = 0u;
#pragma unroll
        for (int i = 0; i < NV; ++i) tot[i] = acc[i];
        return true;
    }
    return ALL;
}

inline int red_grid(long long n) {
    long long g = (n + VEC_THREADS - 1) / VEC_THREADS;
    if (g < 1) g = 1;
    if (g > MAX_RED_BLOCKS) g = MAX_RED_BLOCKS;
    return (int)g;
}

#define GRID_STRIDE(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// ------------------------------------------------------------------ nodal <-> modal
// out[item][blk][a] = sum_n T[a][n] in[item][blk][n]  (T is n x n)
__global__ void k_basis_change(const double *__restrict__ T, int n, const double *__restrict__ in,
                               double *__restrict__ out, long long nvec) {
    wait_prior_kernel();
    GRID_STRIDE(i, nvec * n) {
        long long v = i / n;
        int a = (int)(i % n);
        double s = 0;
        for (int m = 0; m < n; ++m) s += __ldg(&T[a * n + m]) * in[v * n + m];
        out[i] = s;
    }
}

// L2 projection of samples at the volume points onto the orthonormal cell basis: with
// int_T phi_a phi_b = delta_ab and M_K = detJ I, the coefficient of phi_a is
// (1/detJ) int_K f phi_a = sum_q w_q phi_a(xi_q) f(x_q). One thread per (vector v, basis a);
// vals: [v][nq] (v = cell, or cell * 2 + component), out: [v][n] modal.
__global__ void k_project_qp(const double *__restrict__ qw, const double *__restrict__ phi, int nq, int mu, int n,
                             const double *__restrict__ vals, double *__restrict__ out, long long nvec) {
    wait_prior_kernel();
    GRID_STRIDE(i, nvec * n) {
        const long long v = i / n;
        const int a = (int)(i % n);
        const double *f = vals + v * nq;
        double s = 0;
        for (int q = 0; q < nq; ++q) s += __ldg(&qw[q]) * __ldg(&phi[q * mu + a]) * f[q];
        out[i] = s;
    }
}

// dual <-> Riesz on V_Q: M = detJ I per cell. mode 0: out = detJ * in; mode 1: out = in / detJ.
__global__ void k_mass_scale(const CellGeo *__restrict__ geo, int nu, const double *in, double *out,
                             long long ncells, int mode) {
    wait_prior_kernel();
    GRID_STRIDE(i, ncells * nu) {
        double dj = geo[i / nu].detJ;
        out[i] = mode == 0 ? in[i] * dj : in[i] / dj;
    }
}

// trace dual -> Riesz: facet mass h_F I
__global__ void k_trace_riesz(const CellGeo *__restrict__ geo, const int *__restrict__ facet_cell,
                              const int *__restrict__ facet_edge, int nt, const double *in,
                              double *out, long long nfacets) {
    wait_prior_kernel();
    GRID_STRIDE(i, nfacets * nt) {
        long long f = i / nt;
        int c = facet_cell[2 * f], e = facet_edge[2 * f];
        out[i] = in[i] / geo[c].h[e];
    }
}

// out = sum_t coef[t] * (mass[t] ? detJ : 1) * vec[t]   (up to 12 terms; vec may alias out
// only for t = 0 when out is written after all reads of the element)
struct LinComb {
    int nterms;
    double coef[12];
    const double *vec[12];
    int mass[12];
    int fterm;              // >= 0: the coefficient of term fterm is also multiplied by *fscale
    const double *fscale;   // (device; the time factor of a forcing, refreshed between graph launches)
};
__global__ void k_lincomb(const CellGeo *__restrict__ geo, int nu, LinComb L, double *out, long long ncells) {
    wait_prior_kernel();
    if (L.fterm >= 0) L.coef[L.fterm] *= *L.fscale;
    GRID_STRIDE(i, ncells * nu) {
        double dj = geo[i / nu].detJ;
        double s = 0;
        for (int t = 0; t < L.nterms; ++t) s += L.coef[t] * (L.mass[t] ? dj : 1.0) * L.vec[t][i];
        out[i] = s;
    }
}

__global__ void k_axpby(double a, const double *x, double b, double *y, long long n) {
    wait_prior_kernel();
    GRID_STRIDE(i, n) y[i] = a * x[i] + b * y[i];
}

// Initial guesses of a step's stage solves from the previous step (one field: velocity, pressure
// or trace). With *hist set, stage k's guess is its solution in the previous step shifted by the
// state's change over that step, guess_k = H_k + (x - xprev): both are first-order accurate in
// time, so the guess is off by O(dt^2) where the previous stage's solution (the guess without
// history) is off by O(dt). S: dst_k the stage guesses, src_k the kept solutions. xprev is then
// set to x for the next step.
struct StageVecs {
    double *dst[8];
    const double *src[8];
    double *aux[8];
    int n;
};
__global__ void k_stage_guess(const int *hist, const double *x, double *xprev, StageVecs S, long long n) {
    wait_prior_kernel();
    const bool h = *hist != 0;
    GRID_STRIDE(i, n) {
        const double xv = x[i];
        if (h) {
            const double d = xv - xprev[i];
            for (int k = 0; k < S.n; ++k) S.dst[k][i] = S.src[k][i] + d;
        }
        xprev[i] = xv;
    }
}

// out[0] = max |a - b|, out[1] = max |b| (non-negative doubles compared by their bit patterns, whose
// order is theirs); out zeroed before the launch
__global__ void k_max_diff(const double *a, const double *b, long long n, unsigned long long *out) {
    wait_prior_kernel();
    double d = 0.0, m = 0.0;
    GRID_STRIDE(i, n) {
        const double bv = b[i];
        d = fmax(d, fabs(a[i] - bv));
        m = fmax(m, fabs(bv));
    }
    for (int o = 16; o > 0; o >>= 1) {
        d = fmax(d, __shfl_down_sync(0xffffffffu, d, o));
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(d));
        atomicMax(&out[1], (unsigned long long)__double_as_longlong(m));
    }
}

// the stage history is cleared unless out[0] <= rtol out[1] (see k_max_diff)
__global__ void k_keep_if_close(const unsigned long long *out, double rtol, int *hist) {
    wait_prior_kernel();
    const double d = __longlong_as_double((long long)out[0]), m = __longlong_as_double((long long)out[1]);
    if (!(d <= rtol * m)) *hist = 0;
}

// dst = src unless *hist is set (the stage guess without history: the previous stage's solution)
__global__ void k_copy_unless(const int *hist, const double *src, double *dst, long long n) {
    wait_prior_kernel();
    if (*hist) return;
    GRID_STRIDE(i, n) dst[i] = src[i];
}

// guess_k = 2 H1_k - H2_k once two steps are kept (*hist >= 2), H1_k after one step: each stage's
// own solutions in the last two steps, extrapolated linearly (dst: guesses, src: H1, aux: H2)
__global__ void k_stage_guess_self(const int *hist, StageVecs S, long long n) {
    wait_prior_kernel();
    const int h = *hist;
    if (h == 0) return;
    GRID_STRIDE(i, n)
        for (int k = 0; k < S.n; ++k) S.dst[k][i] = h >= 2 ? 2.0 * S.src[k][i] - S.aux[k][i] : S.src[k][i];
}

// the stage solutions of this step kept for the next step's guesses: aux_k = dst_k (the step
// before, when aux is set), dst_k = src_k; set_hist: *hist counts the kept steps (at most 2)
__global__ void k_stage_keep(StageVecs S, long long n, int *hist, int set_hist) {
    wait_prior_kernel();
    GRID_STRIDE(i, n)
        for (int k = 0; k < S.n; ++k) {
            if (S.aux[k]) S.aux[k][i] = S.dst[k][i];
            S.dst[k][i] = S.src[k][i];
        }
    if (set_hist && blockIdx.x == 0 && threadIdx.x == 0) *hist = *hist < 2 ? *hist + 1 : 2;
}

// ------------------------------------------------------------------ condensation (CTA / cell)
template <int K>
__global__ void k_condense(RefDev R, MeshDev M, double c, double tau, double *Scell, double *Zc,
                           double *Ac) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    extern __shared__ double sm[];
    const int cell = blockIdx.x;
    if (cell >= M.ncells) return;
    Team tm{(int)threadIdx.x, (int)blockDim.x};
    CellGeo g = M.geo[cell];
    int flip[3] = {M.cell_flip[3 * cell], M.cell_flip[3 * cell + 1], M.cell_flip[3 * cell + 2]};
    cell_condense<K>(tm, R, g, flip, c, tau, sm, Scell + (size_t)cell * Dm::NL * Dm::NL,
                     Zc + (size_t)cell * Dm::NP * Dm::NL, Ac + (size_t)cell * Dm::NP * Dm::NP);
}

// Assemble the ELL trace operator and its facet-block-Jacobi inverse (thread / facet).
template <int NT>
__global__ void k_assemble_trace(MeshDev M, const double *__restrict__ Scell, double *Sell,
                                 int *tcol, double *Dinv) {
    wait_prior_kernel();
    const int NL = 3 * NT;
    GRID_STRIDE(fl, M.nfacets) {
        int f = (int)fl;
        long long nrows = (long long)M.nfacets * NT;
        double blk[5][NT][NT];
        int col[5];
        for (int b = 0; b < 5; ++b) {
            col[b] = -1;
            for (int i = 0; i < NT; ++i)
                for (int j = 0; j < NT; ++j) blk[b][i][j] = 0.0;
        }
        col[0] = f;
        for (int s = 0; s < 2; ++s) {
            int c = M.facet_cell[2 * f + s];
            if (c < 0) continue;
            int e = M.facet_edge[2 * f + s];
            const double *S = Scell + (size_t)c * NL * NL;
            int ob = 1 + 2 * s;
            for (int e2 = 0; e2 < 3; ++e2) {
                int b = (e2 == e) ? 0 : ob++;
                if (b != 0) col[b] = M.cell_facet[3 * c + e2];
                for (int i = 0; i < NT; ++i)
                    for (int j = 0; j < NT; ++j) blk[b][i][j] += S[(e * NT + i) * NL + e2 * NT + j];
            }
        }
        for (int b = 0; b < 5; ++b) {
            tcol[b * M.nfacets + f] = col[b];
            for (int j = 0; j < NT; ++j)
                for (int i = 0; i < NT; ++i) Sell[((size_t)(b * NT + j)) * nrows + (size_t)f * NT + i] = blk[b][i][j];
        }
        // inverse of the diagonal block (symmetric positive definite): Gauss-Jordan
        double A[NT][NT], I[NT][NT];
        for (int i = 0; i < NT; ++i)
            for (int j = 0; j < NT; ++j) { A[i][j] = blk[0][i][j]; I[i][j] = (i == j) ? 1.0 : 0.0; }
        for (int k = 0; k < NT; ++k) {
            double d = 1.0 / A[k][k];
            for (int j = 0; j < NT; ++j) { A[k][j] *= d; I[k][j] *= d; }
            for (int i = 0; i < NT; ++i) {
                if (i == k) continue;
                double t = A[i][k];
                for (int j = 0; j < NT; ++j) { A[i][j] -= t * A[k][j]; I[i][j] -= t * I[k][j]; }
            }
        }
        for (int j = 0; j < NT; ++j)
            for (int i = 0; i < NT; ++i) Dinv[(size_t)j * nrows + (size_t)f * NT + i] = I[i][j];
    }
}

// y = S x (ELL, thread / row)
template <int NT>
__global__ void k_trace_apply(const double *__restrict__ Sell, const int *__restrict__ tcol,
                              const double *__restrict__ x, double *__restrict__ y, int nfacets) {
    wait_prior_kernel();
    long long nrows = (long long)nfacets * NT;
    GRID_STRIDE(g, nrows) {
        int f = (int)(g / NT);
        double s = 0;
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            int cf = __ldg(&tcol[b * nfacets + f]);
            if (cf < 0) continue;
#pragma unroll
            for (int j = 0; j < NT; ++j) s += __ldg(&Sell[(size_t)(b * NT + j) * nrows + g]) * x[(size_t)cf * NT + j];
        }
        y[g] = s;
    }
}

// ------------------------------------------------------------------ trace CG
// b -> sum of b_F[0] (constant-mode content), for the null-space projection
template <int NT>
__global__ void k_trace_mean(const double *__restrict__ b, int nfacets, RedBuf rb, Scalars *sc) {
    wait_prior_kernel();
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(f, nfacets) v[0] += b[(size_t)f * NT];
    if (grid_sum<1>(rb, v, tot)) sc->bmean = tot[0] / nfacets;
}

// r = b - mean e0, x = 0, pold = 0, z = Dinv r; rz = (r, z)
template <int NT>
__global__ void k_cg_setup(const double *__restrict__ b, const double *__restrict__ Dinv, double *x,
                           double *r, double *z, double *pold, int nfacets, RedBuf rb, Scalars *sc,
                           double rtol, int maxit) {
    wait_prior_kernel();
    long long nrows = (long long)nfacets * NT;
    const double mean = sc->bmean;
    double v[3] = {0.0, 0.0, 0.0}, tot[3];
    GRID_STRIDE(f, nfacets) {
        double rl[NT];
        for (int i = 0; i < NT; ++i) {
            rl[i] = b[f * NT + i] - (i == 0 ? mean : 0.0);
            r[f * NT + i] = rl[i];
            x[f * NT + i] = 0.0;
            pold[f * NT + i] = 0.0;
        }
        for (int i = 0; i < NT; ++i) {
            double s = 0;
            for (int j = 0; j < NT; ++j) s += __ldg(&Dinv[(size_t)j * nrows + f * NT + i]) * rl[j];
            z[f * NT + i] = s;
            v[0] += s * rl[i];
            if (i == 0) { v[1] += s; v[2] += rl[0]; }
        }
    }
    if (grid_sum<3>(rb, v, tot)) {
        sc->zmean = tot[1] / nfacets;
        tot[0] -= sc->zmean * tot[2];                 // (r, z - zmean e0)
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

// pnew = z' + beta pold with z' = z - zmean e0 (z projected off the constant trace mode, the
// kernel of S; without it the direction can drift into the kernel and p^T S p lose its sign);
// Ap = S pnew; pAp -> alpha = rz / pAp.
// A facet is handled by a group of NT lanes (32 / NT facets per warp; lane i of a group owns row
// i): for each of the facet's five block columns the group reads the neighbour facet's NT
// direction entries once (lane j forms p_j from z and pold) and passes them to every row by warp
// shuffles, so each row streams its 5 NT operator entries (consecutive rows at consecutive
// addresses: coalesced) and no vector entry is read twice by a group. Grid: cg_apply_grid.
template <int NT>
__global__ void __launch_bounds__(128) k_cg_apply(const double *__restrict__ Sell, const int *__restrict__ tcol,
                                                  const double *__restrict__ z, const double *__restrict__ pold,
                                                  double *__restrict__ pnew, double *__restrict__ Ap, int nfacets,
                                                  RedBuf rb, Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    constexpr int GPW = 32 / NT;                       // facets per warp
    const double beta = sc->beta, zm = sc->zmean;
    const long long nrows = (long long)nfacets * NT;
    const int lane = (int)(threadIdx.x & 31), q = lane / NT, i = lane - q * NT, base = q * NT;
    const long long wpb = blockDim.x >> 5, nw = (long long)gridDim.x * wpb;
    double v[1] = {0.0}, tot[1];
    for (long long w = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); w * GPW < nfacets; w += nw) {
        const long long f0 = w * GPW + q;
        const bool live = q < GPW && f0 < nfacets;
        const int f = live ? (int)f0 : 0;              // dead lanes read row 0 and store nothing
        const size_t g = (size_t)f * NT + i;
        double s = 0.0, pn = 0.0;
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const int cf = __ldg(&tcol[b * nfacets + f]);
            double pv = 0.0;
            if (cf >= 0) {
                const size_t k = (size_t)cf * NT + i;
                pv = z[k] - (i == 0 ? zm : 0.0) + beta * pold[k];
            }
            if (b == 0) pn = pv;                       // block 0 is the facet itself
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const double pj = __shfl_sync(0xffffffffu, pv, base + j);
                if (cf >= 0) s += __ldg(&Sell[(size_t)(b * NT + j) * nrows + g]) * pj;
            }
        }
        if (live) {
            pnew[g] = pn;
            Ap[g] = s;
            v[0] += pn * s;
        }
    }
    if (grid_sum<1>(rb, v, tot)) {
        sc->pAp = tot[0];
        if (tot[0] > 0.0 && isfinite(tot[0])) sc->alpha = sc->rz / tot[0];
        else { sc->alpha = 0.0; sc->done = 1; sc->breakdown = isfinite(tot[0]) ? 1 : 2; }
    }
}

// blocks of 128 threads for k_cg_apply: a warp per 32 / NT facets, at most MAX_RED_BLOCKS
template <int NT>
inline int cg_apply_grid(long long nfacets) {
    const long long warps = (nfacets + 32 / NT - 1) / (32 / NT);
    long long g = (warps + 3) / 4;
    if (g < 1) g = 1;
    if (g > MAX_RED_BLOCKS) g = MAX_RED_BLOCKS;
    return (int)g;
}

// x += alpha p; r -= alpha Ap; z = Dinv r; rz_new -> beta, convergence
template <int NT>
__global__ void k_cg_update(const double *__restrict__ Dinv, const double *__restrict__ p,
                            const double *__restrict__ Ap, double *x, double *r, double *z,
                            int nfacets, RedBuf rb, Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const double alpha = sc->alpha;
    long long nrows = (long long)nfacets * NT;
    double v[3] = {0.0, 0.0, 0.0}, tot[3];
    GRID_STRIDE(f, nfacets) {
        double rl[NT];
        for (int i = 0; i < NT; ++i) {
            size_t g = f * NT + i;
            x[g] += alpha * p[g];
            rl[i] = r[g] - alpha * Ap[g];
            r[g] = rl[i];
        }
        for (int i = 0; i < NT; ++i) {
            double s = 0;
            for (int j = 0; j < NT; ++j) s += __ldg(&Dinv[(size_t)j * nrows + f * NT + i]) * rl[j];
            z[f * NT + i] = s;
            v[0] += s * rl[i];
            if (i == 0) { v[1] += s; v[2] += rl[0]; }
        }
    }
    if (grid_sum<3>(rb, v, tot)) {
        sc->zmean = tot[1] / nfacets;
        double rz_new = tot[0] - sc->zmean * tot[2];  // (r, z - zmean e0)
        sc->beta = rz_new / sc->rz;
        sc->rz = rz_new;
        sc->iters += 1;
        double rel = sc->rz0 > 0 ? sqrt(fmax(rz_new, 0.0) / sc->rz0) : 0.0;
        sc->relres = rel;
        if (!isfinite(rz_new)) { sc->done = 1; sc->breakdown = 2; }
        else if (rel <= sc->rtol || sc->iters >= sc->maxit) sc->done = 1;
    }
}

// ------------------------------------------------------------------ Step-II per-cell kernels
template <int K>
__device__ __forceinline__ void gather_trace_local(const MeshDev &M, int cell, const double *lam,
                                                   double *lK, const Team &tm) {
    constexpr int NT = Dims<K>::NT;
    TFOR(i, 3 * NT) {
        int e = i / NT, j = i % NT;
        int f = M.cell_facet[3 * cell + e];
        lK[i] = lam ? tsign(M.cell_flip[3 * cell + e], j) * lam[(size_t)f * NT + j] : 0.0;
    }
    tm.sync();
}

// Per-cell kernels run one cell per TEAM_LANES lanes (two cells per warp: their row loops have
// 10..15 rows, so a full warp per cell would leave half of it idle). The mesh has an even number
// of cells, so both halves of a warp are either in range or out of range together.
constexpr int TEAM_LANES = 16;
#define CELL_TEAM(SCR)                                                              \
    extern __shared__ double sm[];                                                  \
    const int team = threadIdx.x / TEAM_LANES;                                      \
    const int cell = (blockIdx.x * blockDim.x + threadIdx.x) / TEAM_LANES;          \
    if (cell >= M.ncells) return;                                                   \
    Team tm{(int)(threadIdx.x % TEAM_LANES), TEAM_LANES};                           \
    double *mine = sm + team * (SCR);

template <int K>
__global__ void k_mixed_rhs(RefDev R, MeshDev M, double tau, const double *Ru, const double *X,
                            const double *p, const double *lam, const double *Rp_add,
                            const double *__restrict__ Zc, double *v, double *w) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int SCR = Dm::NL + 4 * Dm::MU + Dm::NP + Dm::NL;
    CELL_TEAM(SCR)
    double *lK = mine;
    gather_trace_local<K>(M, cell, lam, lK, tm);
    CellGeo g = M.geo[cell];
    int flip[3] = {M.cell_flip[3 * cell], M.cell_flip[3 * cell + 1], M.cell_flip[3 * cell + 2]};
    cell_mixed_rhs<K>(tm, R, g, flip, tau, Ru ? Ru + (size_t)cell * Dm::NU : nullptr,
                      X ? X + (size_t)cell * Dm::NU : nullptr, p ? p + (size_t)cell * Dm::NP : nullptr,
                      lam ? lK : nullptr, Rp_add ? Rp_add + (size_t)cell * Dm::NP : nullptr,
                      Zc + (size_t)cell * Dm::NP * Dm::NL, mine + Dm::NL,
                      v + (size_t)cell * Dm::NL, w + (size_t)cell * Dm::NP);
}

// b_F = sum over the facet's cells of v_K (canonical rows of the facet's local edge) - sub_F
template <int NT>
__global__ void k_facet_gather(MeshDev M, const double *__restrict__ v, const double *sub, double *b, float *b32) {
    wait_prior_kernel();
    GRID_STRIDE(g, (long long)M.nfacets * NT) {
        int f = (int)(g / NT), j = (int)(g % NT);
        double s = sub ? -sub[g] : 0.0;
        for (int side = 0; side < 2; ++side) {
            int c = M.facet_cell[2 * f + side];
            if (c < 0) continue;
            s += v[(size_t)c * 3 * NT + M.facet_edge[2 * f + side] * NT + j];
        }
        b[g] = s;
        if (b32) b32[g] = (float)s;
    }
}

// ------------------------------------------------------------------ Step II inside the preconditioner
// The stage preconditioner's Step II reads only (X, Rp_add) and the trace solution; its cell work
// is linear in them, so per coefficient c the two per-cell maps are formed once (by applying the
// FP64 cell routines to unit vectors) and stored in FP32:
//   Lrhs: (X (NU), Rp_add (NP)) -> (v (NL, facet orientation), w (NP))
//   Lbs:  (w (NP), lambda_local (NL)) -> (U (NU), p (NP))
// layout L[(col * ncells + cell) * ROWS + row].
template <int K>
__global__ void k_build_pre_maps(RefDev R, MeshDev M, double c, double tau, const double *__restrict__ Zc,
                                 const double *__restrict__ Ac, float *Lrhs, float *Lbs) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int NU = Dm::NU, NP = Dm::NP, NL = Dm::NL, MU = Dm::MU;
    constexpr int SCR = NU + NP + NL + NP + (NL + 4 * MU + NP + NL) + NU + NP + (NL + NP);
    CELL_TEAM(SCR)
    double *uin = mine;                 // NU + NP unit input (X, Rp_add)
    double *vo = uin + NU + NP;         // NL + NP outputs (v, w)
    double *scr = vo + NL + NP;         // scratch of cell_mixed_rhs
    double *bo = scr + NL + 4 * MU + NP + NL;   // NU + NP outputs (U, p)
    double *bscr = bo + NU + NP;        // scratch of cell_mixed_backsub
    const CellGeo g = M.geo[cell];
    int flip[3] = {M.cell_flip[3 * cell], M.cell_flip[3 * cell + 1], M.cell_flip[3 * cell + 2]};
    const double *Z = Zc + (size_t)cell * NP * NL, *A = Ac + (size_t)cell * NP * NP;
    constexpr int RR = NL + NP, RB = NU + NP;
    for (int col = 0; col < NU + NP; ++col) {
        TFOR(i, NU + NP) uin[i] = (i == col) ? 1.0 : 0.0;
        tm.sync();
        cell_mixed_rhs<K>(tm, R, g, flip, tau, nullptr, uin, nullptr, nullptr, uin + NU, Z, scr, vo, vo + NL);
        TFOR(r, RR) Lrhs[((size_t)col * M.ncells + cell) * RR + r] = (float)vo[r];
        tm.sync();
    }
    for (int col = 0; col < NP + NL; ++col) {
        TFOR(i, NU + NP) uin[i] = (i == col) ? 1.0 : 0.0;     // w = uin[0..NP), lambda = uin[NP..NP+NL)
        tm.sync();
        cell_mixed_backsub<K>(tm, R, g, c, nullptr, uin, uin + NP, Z, A, bscr, bo, bo + NU);
        TFOR(r, RB) Lbs[((size_t)col * M.ncells + cell) * RB + r] = (float)bo[r];
        tm.sync();
    }
}

// v, w of the preconditioner's Step II from X and Rp_add (FP32 map, FP64 in/out)
template <int K>
__global__ void k_pre_rhs(MeshDev M, const float *__restrict__ Lrhs, const double *__restrict__ X,
                          const double *__restrict__ Rp_add, double *v, double *w) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int NU = Dm::NU, NP = Dm::NP, NL = Dm::NL, RR = NL + NP;
    constexpr int SCR = NU + NP;
    CELL_TEAM(SCR)
    float *in = reinterpret_cast<float *>(mine);
    TFOR(i, NU + NP) in[i] = (float)(i < NU ? X[(size_t)cell * NU + i] : Rp_add[(size_t)cell * NP + i - NU]);
    tm.sync();
    TFOR(r, RR) {
        float s = 0.f;
        for (int col = 0; col < NU + NP; ++col) s += __ldg(&Lrhs[((size_t)col * M.ncells + cell) * RR + r]) * in[col];
        if (r < NL) v[(size_t)cell * NL + r] = s;
        else w[(size_t)cell * NP + r - NL] = s;
    }
}

// U, p of the preconditioner's Step II from w and the trace solution (FP32 map, FP64 in/out)
template <int K>
__global__ void k_pre_backsub(MeshDev M, const float *__restrict__ Lbs, const double *__restrict__ w,
                              const double *__restrict__ lam, double *U, double *p,
                              const double *__restrict__ Qbar = nullptr) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int NU = Dm::NU, NP = Dm::NP, NL = Dm::NL, NT = Dm::NT, RB = NU + NP;
    constexpr int SCR = NP + NL;
    CELL_TEAM(SCR)
    float *in = reinterpret_cast<float *>(mine);
    TFOR(i, NP + NL) {
        if (i < NP) {
            in[i] = (float)w[(size_t)cell * NP + i];
        } else {
            const int q = i - NP, e = q / NT, j = q % NT;
            const int f = M.cell_facet[3 * cell + e];
            in[i] = (float)(tsign(M.cell_flip[3 * cell + e], j) * lam[(size_t)f * NT + j]);
        }
    }
    tm.sync();
    TFOR(r, RB) {
        float s = 0.f;
        for (int col = 0; col < NP + NL; ++col) s += __ldg(&Lbs[((size_t)col * M.ncells + cell) * RB + r]) * in[col];
        if (r < NU) {                   // with Qbar: the preconditioner's velocity Qbar + U
            const size_t gi = (size_t)cell * NU + r;
            U[gi] = Qbar ? Qbar[gi] + (double)s : (double)s;
        } else {
            p[(size_t)cell * NP + r - NU] = s;
        }
    }
}

template <int K>
__global__ void k_mixed_backsub(RefDev R, MeshDev M, double c, const double *Ru,
                                const double *__restrict__ w, const double *lam,
                                const double *__restrict__ Zc, const double *__restrict__ Ac,
                                double *U, double *p) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int SCR = Dm::NL + Dm::NP;
    CELL_TEAM(SCR)
    double *lK = mine;
    gather_trace_local<K>(M, cell, lam, lK, tm);
    CellGeo g = M.geo[cell];
    cell_mixed_backsub<K>(tm, R, g, c, Ru ? Ru + (size_t)cell * Dm::NU : nullptr,
                          w + (size_t)cell * Dm::NP, lK, Zc + (size_t)cell * Dm::NP * Dm::NL,
                          Ac + (size_t)cell * Dm::NP * Dm::NP, lK + Dm::NL,
                          U + (size_t)cell * Dm::NU, p + (size_t)cell * Dm::NP);
}

// ------------------------------------------------------------------ BDM projection (warp / cell)
template <int K>
__global__ void k_bdm(RefDev R, MeshDev M, const double *Q, double *Qs) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int SCR = bdm_scratch<K>();
    CELL_TEAM(SCR)
    CellGeo g = M.geo[cell];
    const double *Qn[3];
    int ne[3];
    for (int e = 0; e < 3; ++e) {
        int o = M.cell_nbr[3 * cell + e];
        Qn[e] = o >= 0 ? Q + (size_t)o * Dm::NU : nullptr;
        ne[e] = M.cell_nbr_edge[3 * cell + e];
    }
    cell_bdm<K>(tm, R, g, Q + (size_t)cell * Dm::NU, Qn, ne, mine, Qs + (size_t)cell * Dm::NU);
}

// ------------------------------------------------------------------ tentative-velocity operator
template <int K>
constexpr int fimpl_smem_doubles() {
    typedef Dims<K> Dm;
    return fimpl_diag_scratch<K>() + 3 * Dm::NU * Dm::NU + 3 * Dm::NFQ + 2;
}
template <int K>
constexpr int fimpl_smem_noinv_doubles() {
    typedef Dims<K> Dm;
    return fimpl_diag_scratch<K>() + Dm::NU * Dm::NU + 3 * Dm::NFQ;
}

// Step-I operator of one stage, one block per cell: diagonal block -> Dblk, neighbour weights
// -> wq (and wq32 in FP32), the penalty weights -> pen / pen32 (cell 0), and the inverse of the
// diagonal block in FP64 -> Binv when non-null (dynamic shared memory: fimpl_smem_doubles, or
// fimpl_smem_noinv_doubles without Binv). The FP32 inverses come from k_block_inv32. F2 (tables
// non-null): the block formed in pair arithmetic (cell_fimpl_diag_f2), written in FP64.
template <int K>
__global__ void k_fimpl_assemble(RefDev R, MeshDev M, const double *Qs, double c, double alpha,
                                 double dup, double *Dblk, double *wq, float *wq32, double *pen, float *pen32,
                                 double *Binv, int *status, const AsmF2 F2) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int NU = Dm::NU, NFQ = Dm::NFQ;
    extern __shared__ double sm[];
    const int cell = blockIdx.x;
    if (cell >= M.ncells) return;
    Team tm{(int)threadIdx.x, (int)blockDim.x};
    if (cell == 0)
        TFOR(q, NFQ) {
            pen[q] = -c * alpha * ldg(&R.fw[q]);
            pen32[q] = (float)pen[q];
        }
    CellGeo g = M.geo[cell];
    const double *Qn[3];
    int ne[3];
    for (int e = 0; e < 3; ++e) {
        int o = M.cell_nbr[3 * cell + e];
        Qn[e] = o >= 0 ? Qs + (size_t)o * NU : nullptr;
        ne[e] = M.cell_nbr_edge[3 * cell + e];
    }
    double *D = sm + fimpl_diag_scratch<K>();
    double *wqs = D + NU * NU;
    cell_fimpl_diag<K>(tm, R, g, Qs + (size_t)cell * NU, Qn, ne, c, alpha, dup, sm, D, wqs, F2);
    const long long nrows = (long long)M.ncells * NU;
    TFOR(i, NU * NU) {
        int col = i / NU, row = i % NU;
        Dblk[(size_t)col * nrows + (size_t)cell * NU + row] = D[row * NU + col];
    }
    TFOR(i, 3 * NFQ) {
        wq[(size_t)cell * 3 * NFQ + i] = wqs[i];
        wq32[(size_t)cell * 3 * NFQ + i] = (float)wqs[i];
    }
    double *inv = wqs + 3 * NFQ;                    // NU^2 doubles (FP64 inverse only)
    int *piv = (int *)(inv + 2 * NU * NU);
    bool ok = true;
    if (Binv) {
        // the diagonal block is consumed by the inversion (in place)
        ok = team_invert<NU, double>(tm, D, inv, piv) && ok;
        TFOR(i, NU * NU) {
            int col = i / NU, row = i % NU;
            Binv[(size_t)col * nrows + (size_t)cell * NU + row] = inv[row * NU + col];
        }
    }
    if (!ok && tm.tid == 0) atomicExch(status, 1);
}

// storage slot of a cell's FP32 block inverse in the colour-major order of the red-black passes:
// even (red) cells first, then odd (black) cells (ncells is even)
__host__ __device__ __forceinline__ long long gs_slot(long long cell, long long ncells) {
    return (cell & 1) * (ncells >> 1) + (cell >> 1);
}

// per-cell block layout of the FP32 inverses for the red-black passes (hdg_gs32.cuh): the block
// of slot s at [s * SIZE], column-major with the rows padded to NUP (zeros), SIZE a multiple of
// 32 floats; G groups of 4 rows, S column subsets for a warp's lanes s * G + g
template <int K>
struct GsBlk {
    static constexpr int NU = Dims<K>::NU;
    static constexpr int NUP = (NU + 3) / 4 * 4;
    static constexpr int SIZE = (NU * NUP + 31) / 32 * 32;
    static constexpr int G = NUP / 4;
    static constexpr int S = 32 / G;
};

// z = B v for the block B of storage slot `slot` (a warp; v in shared memory, NU entries; z's NU
// entries written to shared memory)
template <int K>
__device__ __forceinline__ void warp_block_apply(const float *__restrict__ Binv, long long slot, const float *v,
                                                 float *z) {
    typedef GsBlk<K> B;
    const int lane = (int)(threadIdx.x & 31), g = lane % B::G, s = lane / B::G;
    const float4 *blk = reinterpret_cast<const float4 *>(Binv + (size_t)slot * B::SIZE);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (s < B::S) {
#pragma unroll 4
        for (int q = s; q < B::NU; q += B::S) {
            const float4 b = __ldg(blk + q * (B::NUP / 4) + g);
            const float vq = v[q];
            a0 = fmaf(b.x, vq, a0); a1 = fmaf(b.y, vq, a1);
            a2 = fmaf(b.z, vq, a2); a3 = fmaf(b.w, vq, a3);
        }
    }
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
#pragma unroll
    for (int s2 = 0; s2 < B::S; ++s2) {             // the subsets' partial sums, in order
        const int src = s2 * B::G + g;
        t0 += __shfl_sync(0xffffffffu, a0, src); t1 += __shfl_sync(0xffffffffu, a1, src);
        t2 += __shfl_sync(0xffffffffu, a2, src); t3 += __shfl_sync(0xffffffffu, a3, src);
    }
    if (s == 0) {
        const int r = 4 * g;
        if (r < B::NU) z[r] = t0;
        if (r + 1 < B::NU) z[r + 1] = t1;
        if (r + 2 < B::NU) z[r + 2] = t2;
        if (r + 3 < B::NU) z[r + 3] = t3;
    }
}

// The same product with the block read ahead into registers (warp_block_prefetch at the start of
// a kernel, so that its loads overlap the kernel's other loads; warp_block_apply_pre once v is
// ready): the same sums in the same order as warp_block_apply. Only for K <= 3, where a lane holds
// at most 8 of the block's 16-byte column pieces.
template <int K>
struct GsPre {
    static constexpr int NC = (GsBlk<K>::NU + GsBlk<K>::S - 1) / GsBlk<K>::S;   // columns per lane
    static constexpr bool ON = NC <= 8;
};

template <int K>
__device__ __forceinline__ void warp_block_prefetch(const float *__restrict__ Binv, long long slot,
                                                    float4 (&pre)[GsPre<K>::NC]) {
    typedef GsBlk<K> B;
    const int lane = (int)(threadIdx.x & 31), g = lane % B::G, s = lane / B::G;
    const float4 *blk = reinterpret_cast<const float4 *>(Binv + (size_t)slot * B::SIZE);
#pragma unroll
    for (int u = 0; u < GsPre<K>::NC; ++u) {
        const int q = s + u * B::S;
        pre[u] = (s < B::S && q < B::NU) ? __ldg(blk + q * (B::NUP / 4) + g) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <int K>
__device__ __forceinline__ void warp_block_apply_pre(const float4 (&pre)[GsPre<K>::NC], const float *v, float *z) {
    typedef GsBlk<K> B;
    const int lane = (int)(threadIdx.x & 31), g = lane % B::G, s = lane / B::G;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
    for (int u = 0; u < GsPre<K>::NC; ++u) {
        const int q = s + u * B::S;
        if (s < B::S && q < B::NU) {
            const float4 b = pre[u];
            const float vq = v[q];
            a0 = fmaf(b.x, vq, a0); a1 = fmaf(b.y, vq, a1);
            a2 = fmaf(b.z, vq, a2); a3 = fmaf(b.w, vq, a3);
        }
    }
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
#pragma unroll
    for (int s2 = 0; s2 < B::S; ++s2) {             // the subsets' partial sums, in order
        const int src = s2 * B::G + g;
        t0 += __shfl_sync(0xffffffffu, a0, src); t1 += __shfl_sync(0xffffffffu, a1, src);
        t2 += __shfl_sync(0xffffffffu, a2, src); t3 += __shfl_sync(0xffffffffu, a3, src);
    }
    if (s == 0) {
        const int r = 4 * g;
        if (r < B::NU) z[r] = t0;
        if (r + 1 < B::NU) z[r + 1] = t1;
        if (r + 2 < B::NU) z[r + 2] = t2;
        if (r + 3 < B::NU) z[r + 3] = t3;
    }
}

// FP32 inverses of the Step-I diagonal blocks for the inner (preconditioner) solves, one warp per
// cell with the block in registers: lane l holds rows l and l + 32 (< NU), Gauss-Jordan in place
// without pivoting, row k reaching the other lanes by shuffles. No pivoting is needed: the block
// M_K - c F_K has a positive definite symmetric part (mass plus the dissipative penalty and upwind
// terms; the advection's symmetric part is c (div Q*)/2 |Q|^2, far below the mass), so every
// leading block is nonsingular. A zero or non-finite pivot sets *status (singular block).
// Dblk32 (optional) receives the block itself rounded to FP32 for the relaxed stage products, in
// the per-cell block layout GsBlk (slot = cell). Dblk and Binv32 in the column-slice layout
// [col * nrows + cell * NU + row], or with by_colour set Binv32 in the red-black passes' layout
// (GsBlk, slot gs_slot(cell)).
template <int K>
__global__ void __launch_bounds__(128) k_block_inv32(const double *__restrict__ Dblk, float *__restrict__ Binv32,
                                                     float *__restrict__ Dblk32, long long ncells, int by_colour,
                                                     int *status) {
    wait_prior_kernel();
    constexpr int N = Dims<K>::NU;
    constexpr int R = (N + 31) / 32;
    const int lane = (int)(threadIdx.x & 31);
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // uniform per warp
    if (cell >= ncells) return;
    const long long nrows = ncells * N;
    float a[R][N];
#pragma unroll
    for (int s = 0; s < R; ++s) {
        const int r = lane + 32 * s;
#pragma unroll
        for (int j = 0; j < N; ++j) a[s][j] = r < N ? (float)__ldg(&Dblk[(size_t)j * nrows + (size_t)cell * N + r]) : 0.f;
    }
    if (Dblk32) {
        typedef GsBlk<K> B;
        float *blk = Dblk32 + (size_t)cell * B::SIZE;
#pragma unroll
        for (int s = 0; s < R; ++s) {
            const int r = lane + 32 * s;
            if (r < B::NUP)
#pragma unroll
                for (int j = 0; j < N; ++j) blk[j * B::NUP + r] = r < N ? a[s][j] : 0.f;
        }
        for (int i = N * B::NUP + lane; i < B::SIZE; i += 32) blk[i] = 0.f;
    }
    bool ok = true;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const int owner = k & 31, ks = k >> 5;
        const float piv = __shfl_sync(0xffffffffu, a[ks][k], owner);
        ok = ok && isfinite(piv) && piv != 0.f;
        const float inv = 1.f / piv;
        float f[R];
#pragma unroll
        for (int s = 0; s < R; ++s) f[s] = a[s][k];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const float rkj = __shfl_sync(0xffffffffu, a[ks][j], owner) * inv;   // row k, normalised
#pragma unroll
            for (int s = 0; s < R; ++s) {
                const bool pivot_row = lane + 32 * s == k;
                if (j == k) a[s][j] = pivot_row ? inv : -f[s] * inv;
                else a[s][j] = pivot_row ? rkj : a[s][j] - f[s] * rkj;
            }
        }
    }
    if (by_colour) {
        typedef GsBlk<K> B;
        float *blk = Binv32 + (size_t)gs_slot(cell, ncells) * B::SIZE;
#pragma unroll
        for (int s = 0; s < R; ++s) {
            const int r = lane + 32 * s;
            if (r < B::NUP)
#pragma unroll
                for (int j = 0; j < N; ++j) blk[j * B::NUP + r] = r < N ? a[s][j] : 0.f;
        }
        for (int i = N * B::NUP + lane; i < B::SIZE; i += 32) blk[i] = 0.f;
    } else {
#pragma unroll
        for (int s = 0; s < R; ++s) {
            const int r = lane + 32 * s;
            if (r < N)
#pragma unroll
                for (int j = 0; j < N; ++j) Binv32[(size_t)j * nrows + (size_t)cell * N + r] = a[s][j];
        }
    }
    if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicExch(status, 1);
}

// ------------------------------------------------------------ matrix-free neighbour coupling
// Tables the neighbour coupling needs, in the precision T of the solve: ephi (edge values of the
// velocity basis, [e][q][a]) and pen (the penalty weights -c alpha fw_q of the assembled operator,
// written by k_fimpl_assemble).
template <class T>
struct EdgeTab {
    const T *ephi, *pen;
    const T *nrm;           // optional: the cells' outward normals in T, nrm[6 cell + 2 e + d]
};

// t[(e*NFQ + q)*2 + d] = pen_q n_d (n . u) + wq(e, q) u_d at the points of this cell's edges,
// u = the neighbour's velocity at the matching point (its point NFQ-1-q on its edge), taken from
// the table utr of the cells' own edge values, or evaluated from the coefficients x when utr is
// null. Zero on walls.
template <int K, class T>
__device__ __forceinline__ void team_nbr_flux(const Team &tm, const EdgeTab<T> &E, const MeshDev &M, int cell,
                                              const T *__restrict__ wq, const T *utr, const T *x, T *t) {
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NFQ = Dm::NFQ;
    const CellGeo *gp = M.geo + cell;
    TFOR(i, 3 * NFQ) {
        const int e = i / NFQ, q = i % NFQ;
        const int o = __ldg(&M.cell_nbr[3 * cell + e]);
        T tx = 0, ty = 0;
        if (o >= 0) {
            const int eo = __ldg(&M.cell_nbr_edge[3 * cell + e]), qo = NFQ - 1 - q;
            T ux = 0, uy = 0;
            if (utr) {
                const T *u = utr + ((size_t)(o * 3 + eo) * NFQ + qo) * 2;
                ux = u[0]; uy = u[1];
            } else {
                const T *ph = &E.ephi[(eo * NFQ + qo) * MU];
                const T *xo = x + (size_t)o * NU;
#pragma unroll 5
                for (int b = 0; b < MU; ++b) {
                    const T f = __ldg(ph + b);
                    ux += f * xo[b]; uy += f * xo[MU + b];
                }
            }
            T nx, ny;
            if constexpr (sizeof(T) == 4) {     // FP32 tables: the normals always come in FP32
                nx = E.nrm[6 * cell + 2 * e];
                ny = E.nrm[6 * cell + 2 * e + 1];
            } else {
                nx = E.nrm ? E.nrm[6 * cell + 2 * e] : gp->nx[e];
                ny = E.nrm ? E.nrm[6 * cell + 2 * e + 1] : gp->ny[e];
            }
            const T un = nx * ux + ny * uy, pen = E.pen[q];
            const T w = __ldg(&wq[(size_t)cell * 3 * NFQ + i]);
            tx = pen * nx * un + w * ux;
            ty = pen * ny * un + w * uy;
        }
        t[2 * i] = tx;
        t[2 * i + 1] = ty;
    }
}

// row (d, a) of the neighbour coupling: sum over the edge points of phi_a(e, q) t[(e, q), d]
template <int K, class T>
__device__ __forceinline__ T nbr_row(const EdgeTab<T> &E, const T *t, int d, int a) {
    typedef Dims<K> Dm;
    T s = 0;
#pragma unroll 7
    for (int i = 0; i < 3 * Dm::NFQ; ++i) s += __ldg(&E.ephi[i * Dm::MU + a]) * t[2 * i + d];
    return s;
}

// y = (M - cF) x: diagonal block dense, neighbours matrix-free (team per cell)
template <int K>
__global__ void k_cell_apply_mf(EdgeTab<double> E, MeshDev M, const double *__restrict__ Dblk,
                                const double *__restrict__ wq, const double *__restrict__ x, double *__restrict__ y) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU;
    constexpr int SCR = 6 * Dm::NFQ;
    CELL_TEAM(SCR)
    double *t = mine;
    team_nbr_flux<K, double>(tm, E, M, cell, wq, nullptr, x, t);
    tm.sync();
    const long long nrows = (long long)M.ncells * NU;
    const double *xK = x + (size_t)cell * NU;
    TFOR(r, NU) {
        const size_t gi = (size_t)cell * NU + r;
        double s = nbr_row<K, double>(E, t, r / MU, r % MU);
#pragma unroll 6
        for (int j = 0; j < NU; ++j) s += __ldg(&Dblk[(size_t)j * nrows + gi]) * xK[j];
        y[gi] = s;
    }
}

// ------------------------------------------------------------------ stage operator, fused
// The stage operator A(c) applied to x = (Q, p, lambda) in one pass per cell (yQ32, yp32: FP32
// copies of the output for the FGMRES first-pass dots, when set; zslot: x also copied to slot
// *zslot_j (the FGMRES step) of the FGMRES's preconditioned vectors, when set): velocity rows
// (M - cF)Q - c G(p, lambda) (diagonal block dense, neighbours matrix-free), constraint rows of
// the cell (p-rows yp, the cell's lambda-row contributions v; summed per facet by k_facet_gather).
// skip (optional): return at once when *skip is set (k_stage_apply32 takes that product in FP32).
template <int K>
__global__ void k_stage_apply(RefDev R, EdgeTab<double> E, MeshDev M, const double *__restrict__ Dblk,
                              const double *__restrict__ wq, double c, double tau, const double *Q,
                              const double *p, const double *lam, double *yQ, double *yp, double *v,
                              float *yQ32, float *yp32, double *zslot, const int *zslot_j, const int *skip) {
    wait_prior_kernel();
    if (skip && *skip) return;
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NP = Dm::NP, NT = Dm::NT, NL = Dm::NL, NFQ = Dm::NFQ;
    constexpr int SCR = 6 * NFQ + NL + 2 * MU;
    CELL_TEAM(SCR)
    double *t = mine, *lK = mine + 6 * NFQ, *cs = lK + NL;
    team_nbr_flux<K, double>(tm, E, M, cell, wq, nullptr, Q, t);
    gather_trace_local<K>(M, cell, lam, lK, tm);          // (ends with a team sync)
    const CellGeo g = M.geo[cell];
    const long long nrows = (long long)M.ncells * NU;
    const double *QK = Q + (size_t)cell * NU, *pK = p + (size_t)cell * NP;
    TFOR(x, NU) {
        const int d = x / MU, a = x % MU;
        const size_t gi = (size_t)cell * NU + x;
        double bq = nbr_row<K, double>(E, t, d, a);
#pragma unroll 6
        for (int j = 0; j < NU; ++j) bq += __ldg(&Dblk[(size_t)j * nrows + gi]) * QK[j];
        double et = 0;
        for (int e = 0; e < 3; ++e) {
            const double nd = d == 0 ? g.nx[e] : g.ny[e];
            double s = 0;
            for (int j = 0; j < NT; ++j) s += ldg(&R.Ehat[(e * NT + j) * MU + a]) * lK[e * NT + j];
            et += g.h[e] * nd * s;
        }
        double dt = 0;
        for (int rr = 0; rr < 2; ++rr) {
            double s = 0;
            for (int b = 0; b < NP; ++b) s += ldg(&R.Dhat[(rr * NP + b) * MU + a]) * pK[b];
            dt += g.Jinv[rr * 2 + d] * s;
        }
        const double yv = bq - c * (g.detJ * dt - et);
        yQ[gi] = yv;
        if (yQ32) yQ32[gi] = (float)yv;
    }
    int flip[3] = {M.cell_flip[3 * cell], M.cell_flip[3 * cell + 1], M.cell_flip[3 * cell + 2]};
    cell_constraint<K>(tm, R, g, flip, tau, QK, pK, lK, cs, yp + (size_t)cell * NP, v + (size_t)cell * NL);
    if (yp32) TFOR(b, NP) yp32[(size_t)cell * NP + b] = (float)yp[(size_t)cell * NP + b];   // (team-synced)
    if (zslot) {                        // the input x also stored as slot gs->j of the FGMRES's Z
        const long long nQ = (long long)M.ncells * NU, nPv = (long long)M.ncells * NP;
        double *zj = zslot + (size_t)*zslot_j * (size_t)(nQ + nPv + (long long)M.nfacets * NT);
        TFOR(x, NU) zj[(size_t)cell * NU + x] = QK[x];
        TFOR(b, NP) zj[nQ + (size_t)cell * NP + b] = pK[b];
        TFOR(i, 3 * NT) {               // each facet's values once, by its first cell
            const int f = M.cell_facet[3 * cell + i / NT];
            if (M.facet_cell[2 * f] == cell) zj[nQ + nPv + (size_t)f * NT + i % NT] = lam[(size_t)f * NT + i % NT];
        }
    }
}


// ------------------------------------------------------------------ restarted GMRES (right block-Jacobi)
// Krylov basis V (GM_M+1 vectors of n), Hessenberg column / Givens rotations and the residual
// estimate live in device memory; the last block of each reduction does the small serial
// updates, so one host read per restart cycle suffices.
constexpr int GM_M = 30;        // restart length of the GMRES cycles
struct GmresState {
    double H[(GM_M + 1) * GM_M];     // column-major: H[j*(GM_M+1) + i]
    double cs[GM_M], sn[GM_M], g[GM_M + 1], y[GM_M], hcol[GM_M + 2], h2[GM_M + 2];
    double bnorm, beta, resid, rtol;
    int j, cycle_end, converged, total, maxit, breakdown, m;   // m: restart length of this cycle
    // FP32 copies for the FUSED inner kernels: 1 / (norm of the step's w) and the projections
    float inv32, hcol32[GM_M + 2];
    // the FP32 inner solves keep their Hessenberg matrix, rotations, residual estimates and
    // least-squares solution in FP32 (tol32 = rtol * bnorm)
    float H32[(GM_M + 1) * GM_M], cs32[GM_M], sn32[GM_M], g32[GM_M + 1], y32[GM_M], tol32;
    // relaxed products (stage FGMRES, HDG_MIXED): the next Arnoldi product may be taken in FP32
    // (lowprec) once resid * relax <= rtol * bnorm; relax = 0: never. used32: the current cycle
    // took an FP32 product (set by k_stage_apply32)
    double relax;
    int lowprec, used32;
};

__global__ void k_gm_set_cycle(GmresState *gs, int m) {
    wait_prior_kernel(); gs->m = m; }

// ------------------------------------------------------------------ device-side loops
// Control of a while loop that runs as a CUDA graph conditional node: one thread sets the
// node's condition. Every loop carries a guard counter with a hard limit, so that it ends
// even if the solver never raises its stop flag. Each pass also adds the number of kernels in
// the loop body (*nk, filled in after the body is recorded) to the launch counter.
struct LoopCtl {
    cudaGraphConditionalHandle h;
    int *guard;
    const int *nk;
    unsigned long long *launches;
};

__global__ void k_loop_init(LoopCtl L, const int *stop) {
    wait_prior_kernel();
    *L.guard = 0;
    cudaGraphSetConditional(L.h, *stop ? 0u : 1u);
}

// Last block of an FP64 Arnoldi step, called by all its threads: Hessenberg column (hcol, plus
// h2 after a second pass), norm hn = ||w|| (the value of thread 0), Givens rotations, residual
// estimate, step bookkeeping. The state it reads is first gathered into shared memory by the
// block in one round of independent loads; thread 0 then works on shared memory and only stores
// to the state.
__device__ void gm_finish_step(GmresState *gs, int j, double hn, bool with_h2) {
    __shared__ double Hc[GM_M + 2], cs[GM_M], sn[GM_M], dsc[4];
    __shared__ int isc[3];
    const int t = threadIdx.x;
    if (t <= j) Hc[t] = with_h2 ? gs->hcol[t] + gs->h2[t] : gs->hcol[t];
    if (t < j) { cs[t] = gs->cs[t]; sn[t] = gs->sn[t]; }
    const int tl = (int)blockDim.x - 1;               // scalars: the block's last threads
    if (t == tl) dsc[0] = gs->g[j];
    if (t == tl - 1) dsc[1] = gs->rtol;
    if (t == tl - 2) dsc[2] = gs->bnorm;
    if (t == tl - 3) isc[0] = gs->m;
    if (t == tl - 4) isc[1] = gs->total;
    if (t == tl - 5) isc[2] = gs->maxit;
    if (t == tl - 6) dsc[3] = gs->relax;
    __syncthreads();
    if (t != 0) return;
    Hc[j + 1] = hn;
    for (int i = 0; i < j; ++i) {                     // previous rotations
        const double a = Hc[i], b2 = Hc[i + 1];
        Hc[i] = cs[i] * a + sn[i] * b2;
        Hc[i + 1] = -sn[i] * a + cs[i] * b2;
    }
    const double a = Hc[j], b2 = Hc[j + 1];
    const double r = sqrt(a * a + b2 * b2);
    const double c_ = r > 0 ? a / r : 1.0, s_ = r > 0 ? b2 / r : 0.0;
    double *H = gs->H + j * (GM_M + 1);
    for (int i = 0; i < j; ++i) H[i] = Hc[i];
    H[j] = r;
    H[j + 1] = hn;                                    // the norm, kept for the next v (k_gm_precond_mf)
    gs->cs[j] = c_; gs->sn[j] = s_;
    const double gj = dsc[0], resid = fabs(-s_ * gj);
    gs->g[j + 1] = -s_ * gj;
    gs->g[j] = c_ * gj;
    gs->resid = resid;
    gs->lowprec = (dsc[3] > 0.0 && resid * dsc[3] <= dsc[1] * dsc[2]) ? 1 : 0;
    const int total = isc[1] + 1;
    gs->total = total;
    gs->hcol[GM_M + 1] = hn;
    gs->j = j + 1;
    if (!isfinite(resid)) { gs->breakdown = 2; gs->cycle_end = 1; }
    else if (resid <= dsc[1] * dsc[2]) { gs->converged = 1; gs->cycle_end = 1; }
    else if (j + 1 >= isc[0] || total >= isc[2] || hn == 0.0) gs->cycle_end = 1;
}


__global__ void k_loop_ctl(LoopCtl L, int limit, const int *stop) {
    wait_prior_kernel();
    const int gd = ++*L.guard;
    *L.launches += (unsigned long long)*L.nk;
    cudaGraphSetConditional(L.h, (!*stop && gd < limit) ? 1u : 0u);
}

// restart loop of a GMRES: continue while not converged, finite and under the iteration cap
__global__ void k_gm_loop_ctl(LoopCtl L, int limit, const GmresState *gs, int init) {
    wait_prior_kernel();
    int gd = 0;
    if (init) *L.guard = 0;
    else {
        gd = ++*L.guard;
        *L.launches += (unsigned long long)*L.nk;
    }
    const bool more = !gs->converged && gs->breakdown != 2 && gs->total < gs->maxit && gd < limit;
    cudaGraphSetConditional(L.h, more ? 1u : 0u);
}

// Solve counters kept on the device (DevCount fields: see the struct)
struct DevCount {
    long long stepI_iters, stepI_solves, trace_iters, trace_solves;
    long long outer_iters, stage_solves, stage_unconverged, breakdowns;
    unsigned long long launches;      // kernels run inside device-side loops
    long long products32;             // stage-operator products taken in FP32 (k_stage_apply32)
    long long pad[6];
};

__global__ void k_count_solve(DevCount *acc, const GmresState *gs, const Scalars *sc) {
    wait_prior_kernel();
    if (gs) { acc->stepI_iters += gs->total; acc->stepI_solves += 1; }
    if (sc) {
        acc->trace_iters += sc->iters; acc->trace_solves += 1;
        if (sc->breakdown == 2) acc->breakdowns += 1;
    }
}

// after a stage solve by flexible GMRES
__global__ void k_count_stage(DevCount *acc, const GmresState *fgs) {
    wait_prior_kernel();
    acc->outer_iters += fgs->total;
    acc->stage_solves += 1;
    if (!fgs->converged) acc->stage_unconverged += 1;
    if (fgs->breakdown == 2) acc->breakdowns += 1;
}

// Dots out[i] = (V_i, w), i < nvec, over the rows a block owns: `ranges` calls f(r0, r1) for each
// of the block's row ranges. Warp k of the block takes the vectors k, k + nwarps, ... (a warp reads
// 32 consecutive rows of one vector: coalesced; w is re-read from L1), writes its block partials,
// and the last block to arrive (atomic ticket, no waiting) adds the blocks' partials in a fixed
// order, a warp per value. Deterministic; no per-thread accumulator arrays (registers stay few).
// Lanes accumulate in T (FP32 for the inner solves: GB300's FP64 rate is low), warps and blocks
// combine in FP64. w must be visible to the whole block (written before a __syncthreads, or an
// input).
// The block's partials alone (no ticket): partials[block * (GM_M + 2) + i]; returns nvec (with
// the extra vector counted). With fence, each partial is fenced for a last-block reduction.
template <class T, class Ranges>
__device__ int block_dot_partials(const RedBuf rb, const T *V, const T *w, long long n, int nvec, Ranges ranges,
                                  const T *extra, bool fence, bool f32 = false) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (extra) ++nvec;                   // (extra, w) -> value nvec - 1
    for (int i = warp; i < nvec; i += nw) {
        const T *Vi = (extra && i == nvec - 1) ? extra : V + (size_t)i * n;
        T at = 0;
        ranges([&](long long r0, long long r1) {
            for (long long g = r0 + lane; g < r1; g += 32) at += Vi[g] * w[g];
        });
        for (int o = 16; o > 0; o >>= 1) at += __shfl_down_sync(0xffffffffu, at, o);
        if (lane == 0) {
            if (f32) reinterpret_cast<float *>(rb.partials)[blockIdx.x * (GM_M + 2) + i] = (float)at;
            else rb.partials[blockIdx.x * (GM_M + 2) + i] = (double)at;
            if (fence) __threadfence();
        }
    }
    return nvec;
}

template <class T, class Ranges>
__device__ bool block_multidot(const RedBuf rb, const T *V, const T *w, long long n, int nvec, Ranges ranges,
                               double *out, const T *extra = nullptr) {
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    nvec = block_dot_partials(rb, V, w, n, nvec, ranges, extra, true);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(rb.counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int i = warp; i < nvec; i += nw) {
        double a = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) a += __ldcg(&rb.partials[b * (GM_M + 2) + i]);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) out[i] = a;
    }
    if (threadIdx.x == 0) *rb.counter = 0u;
    return true;
}

// the contiguous row chunk of this block for n rows split over the grid
struct RowChunk {
    long long r0, r1;
    __device__ RowChunk(long long n) {
        const long long ch = (n + gridDim.x - 1) / gridDim.x;
        r0 = blockIdx.x * ch;
        r1 = r0 + ch < n ? r0 + ch : n;
    }
};

// out[i] = (V_i, w), i < nvec (rows split in contiguous chunks over the blocks); with_norm:
// also out[nvec] = (w, w)
template <class T>
__device__ void multidot_rows(const RedBuf rb, const T *V, const T *w, long long n, int nvec, double *out,
                              bool with_norm = false) {
    const RowChunk ch(n);
    block_multidot(rb, V, w, n, nvec, [&](auto f) { if (ch.r0 < ch.r1) f(ch.r0, ch.r1); }, out,
                   with_norm ? w : nullptr);
}

// the same over the rows of the cell groups a team-per-cell kernel assigns to this block (groups
// blockIdx.x, blockIdx.x + gridDim.x, ... of rows_per_group rows); w was written by this block
// before the call
template <class T>
__device__ bool multidot_groups(const RedBuf rb, const T *V, const T *w, long long nrows, long long rows_per_group,
                                int nvec, double *out, bool with_norm = false) {
    __syncthreads();
    return block_multidot(rb, V, w, nrows, nvec, [&](auto f) {
        for (long long g0 = blockIdx.x * rows_per_group; g0 < nrows; g0 += gridDim.x * rows_per_group)
            f(g0, g0 + rows_per_group < nrows ? g0 + rows_per_group : nrows);
    }, out, with_norm ? w : nullptr);
}

// the partials of multidot_groups only, in FP32 (reduced by k_gm_finish_ctl)
template <class T>
__device__ void multidot_groups_partials(const RedBuf rb, const T *V, const T *w, long long nrows,
                                         long long rows_per_group, int nvec, bool with_norm) {
    __syncthreads();
    block_dot_partials(rb, V, w, nrows, nvec, [&](auto f) {
        for (long long g0 = blockIdx.x * rows_per_group; g0 < nrows; g0 += gridDim.x * rows_per_group)
            f(g0, g0 + rows_per_group < nrows ? g0 + rows_per_group : nrows);
    }, with_norm ? w : nullptr, false, true);
}

// FP32 form (the inner solves' products): one pass over the block's rows with 16-byte loads, w
// read once and the nvec (+ 1) partial sums kept in registers, the block's sums added in a fixed
// order. Rows in groups of RPG (a compile-time multiple of 4, as is nrows; V, w 16-byte aligned);
// group g belongs to block g mod gridDim. w may have been written by this block before the call.
template <int RPG>
__device__ void multidot_groups_partials_f32(const RedBuf rb, const float *V, const float *w, long long nrows,
                                             int nvec, bool with_norm) {
    constexpr int NV = GM_M + 1;                 // V_0..V_j, j <= GM_M
    constexpr int Q4 = RPG / 4;
    __shared__ float red[GM_M + 2][32];          // per value, per warp
    __syncthreads();
    float acc[NV], an = 0.f;
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.f;
    const long long ngroups = (nrows + RPG - 1) / RPG;
    const int mine = (long long)blockIdx.x < ngroups ? (int)((ngroups - 1 - blockIdx.x) / gridDim.x) + 1 : 0;
    for (int it = threadIdx.x; it < mine * Q4; it += blockDim.x) {
        const long long r = ((long long)blockIdx.x + (long long)(it / Q4) * gridDim.x) * RPG + 4 * (it % Q4);
        if (r >= nrows) continue;
        const float4 wv = *reinterpret_cast<const float4 *>(w + r);
        if (with_norm) an = fmaf(wv.x, wv.x, fmaf(wv.y, wv.y, fmaf(wv.z, wv.z, fmaf(wv.w, wv.w, an))));
#pragma unroll
        for (int i = 0; i < NV; ++i)
            if (i < nvec) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(V + (size_t)i * nrows + r));
                acc[i] = fmaf(v.x, wv.x, fmaf(v.y, wv.y, fmaf(v.z, wv.z, fmaf(v.w, wv.w, acc[i]))));
            }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i)
        if (i < nvec) {
            float a = acc[i];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) red[i][warp] = a;
        }
    if (with_norm) {
        float a = an;
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) red[nvec][warp] = a;
    }
    __syncthreads();
    if ((int)threadIdx.x < nvec + (with_norm ? 1 : 0)) {
        float sum = 0.f;
        for (int k = 0; k < nw; ++k) sum += red[threadIdx.x][k];
        reinterpret_cast<float *>(rb.partials)[blockIdx.x * (GM_M + 2) + threadIdx.x] = sum;
    }
}

// start of a cycle: w = b - Bx (Bx = B x precomputed; null on the first cycle, x = 0: w = b);
// beta = ||w||
template <class T>
__global__ void k_gm_start(long long nrows, const double *__restrict__ b, const double *__restrict__ Bx,
                           T *w, int first, RedBuf rb, GmresState *gs, double rtol, int maxit, int m = 0) {
    wait_prior_kernel();
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(g, nrows) {
        const T r = (T)(b[g] - (Bx ? Bx[g] : 0.0));
        w[g] = r;
        v[0] += (double)r * (double)r;
    }
    if (grid_sum<1>(rb, v, tot)) {
        double beta = sqrt(tot[0]);
        if (first) {                    // (rtol, maxit: set when not captured, see k_gm_set_tol)
            gs->bnorm = beta;
            gs->total = 0;
            if (rtol > 0) { gs->rtol = rtol; gs->maxit = maxit; }
            gs->converged = 0;
            gs->breakdown = 0;
        }
        gs->beta = beta;
        gs->inv32 = (float)(1.0 / beta);
        gs->resid = beta;
        for (int i = 0; i <= GM_M; ++i) gs->g[i] = 0.0;
        gs->g[0] = beta;
        gs->g32[0] = (float)beta;
        gs->tol32 = (float)(gs->rtol * gs->bnorm);
        gs->j = 0;
        if (m > 0) gs->m = m;           // restart length of this cycle (else set by k_gm_set_cycle)
        if (!isfinite(beta)) { gs->breakdown = 2; gs->cycle_end = 1; }
        else if (beta <= rtol * gs->bnorm || beta == 0.0) { gs->converged = 1; gs->cycle_end = 1; }
        else gs->cycle_end = 0;
    }
}

// v_j = w / h (h = beta for j = 0, H[j, j-1] otherwise) -> V_j; z = Binv v_j (cell-local) and z's
// values at the cell's edge points -> utr (team per cell)
template <int K, class T, bool FUSED = false>
__global__ void k_gm_precond_mf(EdgeTab<T> E, MeshDev M, const T *__restrict__ Binv, const T *__restrict__ w,
                                T *V, T *utr, const GmresState *gs) {
    wait_prior_kernel();
    if (gs->cycle_end) return;
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NFQ = Dm::NFQ;
    constexpr int SCR = 2 * NU;
    extern __shared__ double smd[];
    T *sm = reinterpret_cast<T *>(smd);
    __shared__ float hproj[GM_M + 2];
    const int team = threadIdx.x / TEAM_LANES;
    const int cell = (blockIdx.x * blockDim.x + threadIdx.x) / TEAM_LANES;
    const int j = gs->j;
    if (FUSED) {                        // FP32 scalars of the step (no FP64 work in this kernel)
        if ((int)threadIdx.x < j) hproj[threadIdx.x] = gs->hcol32[threadIdx.x];
        __syncthreads();
    }
    if (cell >= M.ncells) return;
    Team tm{(int)(threadIdx.x % TEAM_LANES), TEAM_LANES};
    T *vK = sm + team * SCR, *zK = vK + NU;
    const T inv = FUSED ? (T)gs->inv32 : (T)(1.0 / (j == 0 ? gs->beta : gs->H[(j - 1) * (GM_M + 1) + j]));
    const long long nrows = (long long)M.ncells * NU;
    T *vj = V + (size_t)j * nrows;
    TFOR(r, NU) {
        const size_t gi = (size_t)cell * NU + r;
        T wv = w[gi];
        if (FUSED)                      // w of step j-1 minus its projections (one Gram-Schmidt pass)
            for (int i = 0; i < j; ++i) wv -= (T)hproj[i] * V[(size_t)i * nrows + gi];
        const T v = wv * inv;
        vj[gi] = v;
        vK[r] = v;
    }
    tm.sync();
    TFOR(r, NU) {
        const size_t gi = (size_t)cell * NU + r;
        T acc = 0;
#pragma unroll 6
        for (int q = 0; q < NU; ++q) acc += __ldg(&Binv[(size_t)q * nrows + gi]) * vK[q];
        zK[r] = acc;
    }
    tm.sync();
    TFOR(i, 3 * NFQ * 2) {
        const int d = i & 1, p = i >> 1;            // p = e*NFQ + q
        const T *ph = &E.ephi[p * MU];
        T s = 0;
#pragma unroll 5
        for (int b = 0; b < MU; ++b) s += __ldg(ph + b) * zK[d * MU + b];
        utr[(size_t)cell * 3 * NFQ * 2 + i] = s;
    }
}

// w = B z = v_j + (neighbour coupling) z for z = Binv v_j (the diagonal block returns v_j);
// hcol[i] = (V_i, w), i <= j. Team per cell over groups of cells; grid <= MAX_RED_BLOCKS.
// FUSED (FP32 inner solves): the same pass also gives ||w||^2; the blocks only write their
// partials, which k_gm_finish_ctl (one block, next in the loop) sums before it finishes the
// Arnoldi step with the norm of w - V hcol from Pythagoras, ||w||^2 - sum hcol_i^2 (V orthonormal),
// so that no separate orthogonalisation kernel runs; the next k_gm_precond_mf<.., true> subtracts
// the projections while it normalises.
template <int K, class T, bool FUSED = false>
__global__ void k_gm_apply_mf(EdgeTab<T> E, MeshDev M, const T *__restrict__ wq, const T *__restrict__ utr, T *w,
                              const T *__restrict__ V, RedBuf rb, GmresState *gs) {
    wait_prior_kernel();
    if (gs->cycle_end) return;
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NFQ = Dm::NFQ;
    extern __shared__ double smd[];
    const int team = threadIdx.x / TEAM_LANES, tpb = blockDim.x / TEAM_LANES;
    Team tm{(int)(threadIdx.x % TEAM_LANES), TEAM_LANES};
    T *t = reinterpret_cast<T *>(smd) + team * (6 * NFQ);
    const long long nrows = (long long)M.ncells * NU;
    const int j = gs->j;
    const T *vj = V + (size_t)j * nrows;
    // cells come in pairs (2 n^2 triangles) and groups start at multiples of tpb: both teams of
    // a warp are active or idle together
    for (int base = blockIdx.x * tpb; base < M.ncells; base += gridDim.x * tpb) {
        const int cell = base + team;
        if (cell < M.ncells) {
            team_nbr_flux<K, T>(tm, E, M, cell, wq, utr, nullptr, t);
            tm.sync();
            TFOR(r, NU) {
                const size_t gi = (size_t)cell * NU + r;
                w[gi] = vj[gi] + nbr_row<K, T>(E, t, r / MU, r % MU);
            }
            tm.sync();
        }
    }
    constexpr int RPG = (128 / TEAM_LANES) * NU;                 // the rows of a 128-thread block's cells
    if constexpr (FUSED && sizeof(T) == 4) {
        if (tpb * NU == RPG) multidot_groups_partials_f32<RPG>(rb, V, (const float *)w, nrows, j + 1, true);
        else multidot_groups_partials(rb, V, (const T *)w, nrows, (long long)tpb * NU, j + 1, true);
    } else if (FUSED) multidot_groups_partials(rb, V, (const T *)w, nrows, (long long)tpb * NU, j + 1, true);
    else multidot_groups(rb, V, (const T *)w, nrows, (long long)tpb * NU, j + 1, gs->hcol, false);
}

// The finishing work of an FP32 inner Arnoldi step for one whole block (see k_gm_finish_ctl);
// pf: the FP32 block partials of the product (nblocks rows of GM_M + 2).
__device__ void finish32_block(LoopCtl L, int limit, const float *pf, int nblocks, GmresState *gs, int ctl) {
    __shared__ float red[GM_M + 2][32];        // per value, per warp
    __shared__ float Hc[GM_M + 2], cs[GM_M], sn[GM_M], gv[GM_M + 1], tol;
    __shared__ int isc[8];
    __shared__ unsigned long long nlaunch;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = (int)(blockDim.x >> 5);
    if (t < GM_M) { cs[t] = gs->cs32[t]; sn[t] = gs->sn32[t]; }
    else if (t >= 32 && t < 32 + GM_M + 1) gv[t - 32] = gs->g32[t - 32];
    else if (t == 64) isc[0] = gs->cycle_end;
    else if (t == 65) isc[1] = gs->j;
    else if (t == 66) isc[2] = gs->m;
    else if (t == 67) isc[3] = gs->total;
    else if (t == 68) isc[4] = gs->maxit;
    else if (t == 69) isc[5] = ctl ? *L.guard : 0;           // (the loop state only when ctl)
    else if (t == 70) isc[6] = ctl ? *L.nk : 0;
    else if (t == 71) nlaunch = ctl ? *L.launches : 0ull;
    else if (t == 72) tol = gs->tol32;
    __syncthreads();
    const int j = isc[1];
    int end = isc[0];
    if (!end) {
        const int nvec = j + 2;
        for (int i0 = 0; i0 < nvec; i0 += 8) {
            float a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = 0.f;
#pragma unroll 4
            for (int b = t; b < nblocks; b += blockDim.x) {     // (unrolled: the loads of several
#pragma unroll                                                  // block rows in flight at once)
                for (int u = 0; u < 8; ++u)
                    if (i0 + u < nvec) a[u] += __ldcg(&pf[(size_t)b * (GM_M + 2) + i0 + u]);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float x = a[u];
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if (lane == 0 && i0 + u < nvec) red[i0 + u][warp] = x;
            }
        }
        __syncthreads();
        if (t < nvec) {
            float x = 0.f;
            for (int w2 = 0; w2 < nw; ++w2) x += red[t][w2];
            Hc[t] = x;
            gs->hcol32[t] = x;                          // projections for the next preconditioner pass
        }
        __syncthreads();
        if (t == 0) {                                   // FP32 throughout: GB300's FP64 pipe makes a
            float h2 = 0.f;                             // serial FP64 chain cost ~10 us here
            for (int i = 0; i <= j; ++i) h2 += Hc[i] * Hc[i];
            const float ww = Hc[j + 1], hn2 = ww - h2;
            const float hn = sqrtf(hn2 > 1e-10f * ww ? hn2 : 1e-10f * ww);
            Hc[j + 1] = hn;
            for (int i = 0; i < j; ++i) {              // previous rotations
                const float p = Hc[i], q = Hc[i + 1];
                Hc[i] = cs[i] * p + sn[i] * q;
                Hc[i + 1] = -sn[i] * p + cs[i] * q;
            }
            const float p = Hc[j], q = Hc[j + 1];
            const float r = sqrtf(p * p + q * q);
            const float c_ = r > 0.f ? p / r : 1.f, s_ = r > 0.f ? q / r : 0.f;
            float *H = gs->H32 + j * (GM_M + 1);
            for (int i = 0; i < j; ++i) H[i] = Hc[i];
            H[j] = r;
            gs->inv32 = 1.f / hn;
            gs->cs32[j] = c_; gs->sn32[j] = s_;
            const float gj = gv[j], resid = fabsf(s_ * gj);
            gs->g32[j + 1] = -s_ * gj;
            gs->g32[j] = c_ * gj;
            const int total = isc[3] + 1;
            gs->total = total;
            gs->j = j + 1;
            if (!isfinite(resid)) { gs->breakdown = 2; end = 1; }
            else if (resid <= tol) { gs->converged = 1; end = 1; }
            else if (j + 1 >= isc[2] || total >= isc[4] || hn == 0.f) end = 1;
            if (end) gs->cycle_end = 1;
        }
    }
    if (t == 0 && ctl) {
        const int gd = isc[5] + 1;
        *L.guard = gd;
        *L.launches = nlaunch + (unsigned long long)isc[6];
        cudaGraphSetConditional(L.h, (!end && gd < limit) ? 1u : 0u);
    }
}

// Step bookkeeping of the FP32 inner Arnoldi loop, one block (256 threads) after the FUSED
// k_gm_apply_mf: reads all the loop state it may need in one round of independent loads, sums the
// nblocks block partials of (V_i, w), i <= j, and ||w||^2 (each thread its blocks' rows, then a
// fixed tree: deterministic), finishes the step on shared memory (hn by Pythagoras with the
// 1e-10 ||w||^2 floor, all in FP32, previous rotations, new Givens rotation, residual estimate, convergence)
// and sets the condition of the loop whose body it ends: continue while the cycle has not ended
// and the pass guard is below limit.
// With ctl = 0 (an Arnoldi step inside an unrolled loop body, not its last) the loop's guard,
// counter and condition are left alone.
__global__ void __launch_bounds__(256) k_gm_finish_ctl(LoopCtl L, int limit, RedBuf rb, int nblocks, GmresState *gs,
                                                       int ctl) {
    wait_prior_kernel();
    finish32_block(L, limit, reinterpret_cast<const float *>(rb.partials), nblocks, gs, ctl);
}

// w -= V hcol; h2 = (V_i, w)  (second Gram-Schmidt pass); rows in contiguous chunks per block
template <class T>
__global__ void k_gm_orth1(T *w, const T *__restrict__ V, long long nrows, RedBuf rb, GmresState *gs) {
    wait_prior_kernel();
    if (gs->cycle_end) return;
    const int nvec = gs->j + 1;
    __shared__ double h[GM_M + 1];
    if ((int)threadIdx.x < nvec) h[threadIdx.x] = gs->hcol[threadIdx.x];
    __syncthreads();
    const RowChunk ch(nrows);
    for (long long g = ch.r0 + threadIdx.x; g < ch.r1; g += blockDim.x) {
        T s = w[g];
        for (int i = 0; i < nvec; ++i) s -= (T)h[i] * V[(size_t)i * nrows + g];
        w[g] = s;
    }
    __syncthreads();
    block_multidot(rb, V, (const T *)w, nrows, nvec, [&](auto f) { if (ch.r0 < ch.r1) f(ch.r0, ch.r1); }, gs->h2);
}

// w -= V h2; ||w|| -> H[j+1, j]; Givens rotations; residual estimate. CGS1: single classical
// Gram-Schmidt pass (w -= V hcol straight after the first dots; no orth1), used by the FP32 inner
// solves whose loose tolerance does not need the second pass.
template <class T, bool CGS1 = false>
__global__ void k_gm_orth2(T *w, const T *__restrict__ V, long long nrows, RedBuf rb, GmresState *gs) {
    wait_prior_kernel();
    if (gs->cycle_end) return;
    const int j = gs->j, nvec = j + 1;
    __shared__ double h[GM_M + 1];
    if ((int)threadIdx.x < nvec) h[threadIdx.x] = CGS1 ? gs->hcol[threadIdx.x] : gs->h2[threadIdx.x];
    __syncthreads();
    double v[1] = {0.0}, tot[1] = {0.0};
    T vt = 0;
    GRID_STRIDE(g, nrows) {
        T s = w[g];
        for (int i = 0; i < nvec; ++i) s -= (T)h[i] * V[(size_t)i * nrows + g];
        w[g] = s;
        vt += s * s;
    }
    v[0] = (double)vt;
    if (grid_sum<1, true>(rb, v, tot)) gm_finish_step(gs, j, sqrt(tot[0]), !CGS1);
}

// y = R^{-1} g (upper triangular part of the rotated H, without the subdiagonal); R and g are
// gathered into shared memory by the block first, then thread 0 substitutes
__global__ void k_gm_solve(GmresState *gs, const double *Hdiag_unused) {
    wait_prior_kernel();
    if (blockIdx.x != 0) return;
    __shared__ double R[GM_M * (GM_M + 1)], g[GM_M], y[GM_M];
    __shared__ int ms;
    if (threadIdx.x == 0) ms = gs->j;
    __syncthreads();
    const int m = ms;
    for (int q = threadIdx.x; q < m * (GM_M + 1); q += blockDim.x) R[q] = gs->H[q];
    for (int q = threadIdx.x; q < m; q += blockDim.x) g[q] = gs->g[q];
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = m - 1; i >= 0; --i) {
        double s = g[i];
        for (int k = i + 1; k < m; ++k) s -= R[k * (GM_M + 1) + i] * y[k];
        const double d = R[i * (GM_M + 1) + i];
        y[i] = d != 0.0 ? s / d : 0.0;
        gs->y[i] = y[i];
    }
}

// FP32 back substitution of an inner FP32 cycle: y32 = R^{-1} g32 (block 0; thread 0 substitutes
// after the block has gathered R and g into shared memory)
__global__ void k_gm_solve32(GmresState *gs) {
    wait_prior_kernel();
    if (blockIdx.x != 0) return;
    __shared__ float R[GM_M * (GM_M + 1)], g[GM_M], y[GM_M];
    __shared__ int ms;
    if (threadIdx.x == 0) ms = gs->j;
    __syncthreads();
    const int m = ms;
    for (int q = threadIdx.x; q < m * (GM_M + 1); q += blockDim.x) R[q] = gs->H32[q];
    for (int q = threadIdx.x; q < m; q += blockDim.x) g[q] = gs->g32[q];
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = m - 1; i >= 0; --i) {
        float s = g[i];
        for (int k = i + 1; k < m; ++k) s -= R[k * (GM_M + 1) + i] * y[k];
        const float d = R[i * (GM_M + 1) + i];
        y[i] = d != 0.f ? s / d : 0.f;
        gs->y32[i] = y[i];
    }
}

// u = V y (rows), then x += Binv u (cell-local)
template <class T>
__global__ void k_gm_combine(const T *__restrict__ V, T *u, long long nrows, const GmresState *gs) {
    wait_prior_kernel();
    const int m = gs->j;
    __shared__ double y[GM_M];
    if ((int)threadIdx.x < m) y[threadIdx.x] = gs->y[threadIdx.x];
    __syncthreads();
    GRID_STRIDE(g, nrows) {
        T s = 0;
        for (int i = 0; i < m; ++i) s += (T)y[i] * V[(size_t)i * nrows + g];
        u[g] = s;
    }
}

// End of an inner cycle from x = 0, team per cell: u = V y on the cell's rows, x = Binv u
// (cell-local), and the solve counted in acc (block 0). Replaces k_gm_combine + k_gm_update_x
// (first cycle) + k_count_solve.
template <int K, class T>
__global__ void k_gm_combine_update(const T *__restrict__ V, const T *__restrict__ Binv, double *x, MeshDev M,
                                    const GmresState *gs, DevCount *acc) {
    wait_prior_kernel();
    constexpr int NU = Dims<K>::NU;
    __shared__ float ys[GM_M];
    const int m = gs->j;
    if ((int)threadIdx.x < m) ys[threadIdx.x] = gs->y32[threadIdx.x];
    if (acc && blockIdx.x == 0 && threadIdx.x == 0) { acc->stepI_iters += gs->total; acc->stepI_solves += 1; }
    __syncthreads();
    extern __shared__ double smd[];
    const int team = threadIdx.x / TEAM_LANES;
    const int cell = (blockIdx.x * blockDim.x + threadIdx.x) / TEAM_LANES;
    if (cell >= M.ncells) return;
    Team tm{(int)(threadIdx.x % TEAM_LANES), TEAM_LANES};
    T *uK = reinterpret_cast<T *>(smd) + team * NU;
    const long long nrows = (long long)M.ncells * NU;
    TFOR(r, NU) {
        const size_t gi = (size_t)cell * NU + r;
        T s = 0;
        for (int i = 0; i < m; ++i) s += (T)ys[i] * V[(size_t)i * nrows + gi];
        uK[r] = s;
    }
    tm.sync();
    TFOR(r, NU) {
        const size_t gi = (size_t)cell * NU + r;
        T a = 0;
#pragma unroll 6
        for (int q = 0; q < NU; ++q) a += __ldg(&Binv[(size_t)q * nrows + gi]) * uK[q];
        x[gi] = (double)a;
    }
}

template <int K, class T>
__global__ void k_gm_update_x(const T *__restrict__ Binv, const T *__restrict__ u, double *x,
                              long long ncells, int first) {
    wait_prior_kernel();
    constexpr int NU = Dims<K>::NU;
    const long long nrows = ncells * NU;
    GRID_STRIDE(g, nrows) {
        long long base = (g / NU) * NU;
        T acc = 0;
#pragma unroll 6
        for (int q = 0; q < NU; ++q) acc += __ldg(&Binv[(size_t)q * nrows + g]) * u[base + q];
        x[g] = (first ? 0.0 : x[g]) + acc;
    }
}

// ------------------------------------------------------------------ Richardson pieces
// dr = sgn * (r - BQ + c (D^T p - E^T l))   (warp / cell; BQ precomputed; r may be null)
template <int K>
__global__ void k_rich_residual(RefDev R, MeshDev M, double c, const double *r, const double *BQ,
                                const double *p, const double *lam, double *dr, double sgn) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int MU = Dm::MU, NU = Dm::NU, NP = Dm::NP, NT = Dm::NT, NL = Dm::NL;
    constexpr int SCR = NL;
    CELL_TEAM(SCR)
    double *lK = mine;
    gather_trace_local<K>(M, cell, lam, lK, tm);
    CellGeo g = M.geo[cell];
    const double *pK = p + (size_t)cell * NP;
    TFOR(x, NU) {
        int d = x / MU, a = x % MU;
        double et = 0;
        for (int e = 0; e < 3; ++e) {
            double nd = d == 0 ? g.nx[e] : g.ny[e];
            double s = 0;
            for (int j = 0; j < NT; ++j) s += ldg(&R.Ehat[(e * NT + j) * MU + a]) * lK[e * NT + j];
            et += g.h[e] * nd * s;
        }
        double dt = 0;
        for (int rr = 0; rr < 2; ++rr) {
            double s = 0;
            for (int b = 0; b < NP; ++b) s += ldg(&R.Dhat[(rr * NP + b) * MU + a]) * pK[b];
            dt += g.Jinv[rr * 2 + d] * s;
        }
        size_t gi = (size_t)cell * NU + x;
        dr[gi] = sgn * ((r ? r[gi] : 0.0) - BQ[gi] + c * (g.detJ * dt - et));
    }
}


// Constraint rows of the stage operator: yp (per cell) and the cells' mu-row contributions
// (gathered per facet by k_facet_gather).
template <int K>
__global__ void k_constraint(RefDev R, MeshDev M, double tau, const double *Q, const double *p,
                             const double *lam, double *yp, double *v) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int SCR = Dm::NL + 2 * Dm::MU;
    CELL_TEAM(SCR)
    double *lK = mine;
    gather_trace_local<K>(M, cell, lam, lK, tm);
    CellGeo g = M.geo[cell];
    int flip[3] = {M.cell_flip[3 * cell], M.cell_flip[3 * cell + 1], M.cell_flip[3 * cell + 2]};
    cell_constraint<K>(tm, R, g, flip, tau, Q + (size_t)cell * Dm::NU, p + (size_t)cell * Dm::NP, lK,
                       lK + Dm::NL, yp + (size_t)cell * Dm::NP, v + (size_t)cell * Dm::NL);
}

// --------------------------------------------------------------- generic (flexible) GMRES pieces
// beta = ||r||, g = beta e1 (cycle start on an already formed residual r)
__global__ void k_vec_start(const double *__restrict__ r, long long n, int first, RedBuf rb, GmresState *gs,
                            double rtol, int maxit, double relax) {
    wait_prior_kernel();
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, n) v[0] += r[i] * r[i];
    if (grid_sum<1>(rb, v, tot)) {
        double beta = sqrt(tot[0]);
        const bool relaxed = !first && gs->used32;   // the cycle that just ended took FP32 products
        if (first) {
            gs->total = 0; gs->rtol = rtol; gs->maxit = maxit; gs->converged = 0; gs->breakdown = 0;
            gs->relax = relax;
            if (first == 1) gs->bnorm = beta;           // first == 2: bnorm set by the caller
        } else if (relaxed && !(beta < 0.5 * gs->beta)) {
            // a cycle with relaxed products that did not halve the FP64 residual: the products'
            // error is too large for this system, so the rest of the solve takes FP64 products
            gs->relax = 0.0;
        }
        gs->used32 = 0;
        gs->lowprec = (gs->relax > 0.0 && beta * gs->relax <= gs->rtol * gs->bnorm) ? 1 : 0;
        gs->beta = beta;
        gs->inv32 = (float)(1.0 / beta);
        gs->resid = beta;
        for (int i = 0; i <= GM_M; ++i) gs->g[i] = 0.0;
        gs->g[0] = beta;
        gs->j = 0;
        // convergence: the residual formed here in FP64 meets the tolerance, or the cycle that just
        // ended took FP64 products only and its estimate met it (the estimate is then exact up to
        // rounding, and an FP64 residual at the attainable-accuracy floor stays accepted); a cycle
        // with relaxed FP32 products is judged on the FP64 residual alone, its estimate can be
        // optimistic by the products' error
        if (!isfinite(beta)) { gs->breakdown = 2; gs->cycle_end = 1; }
        else if (beta <= gs->rtol * gs->bnorm || beta == 0.0) { gs->converged = 1; gs->cycle_end = 1; }
        else if (!relaxed && gs->converged) gs->cycle_end = 1;
        else { gs->converged = 0; gs->cycle_end = 0; }
    }
}

__global__ void k_vec_norm_into(const double *__restrict__ b, long long n, RedBuf rb, GmresState *gs) {
    wait_prior_kernel();
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, n) v[0] += b[i] * b[i];
    if (grid_sum<1>(rb, v, tot)) gs->bnorm = sqrt(tot[0]);
}

// V_j = w / h  (w = w0 and h = beta for j = 0, else w and H[j, j-1]); vfix (optional) gets a
// copy of V_j at a fixed address
__global__ void k_vec_normalize(const double *__restrict__ w0, const double *__restrict__ w, double *V,
                                double *vfix, long long n, const GmresState *gs, float *V32) {
    wait_prior_kernel();
    if (gs->cycle_end) return;
    const int j = gs->j;
    const double h = j == 0 ? gs->beta : gs->H[(j - 1) * (GM_M + 1) + j];
    const double inv = 1.0 / h;
    const double *src = j == 0 ? w0 : w;
    double *vj = V + (size_t)j * n;
    float *vj32 = V32 ? V32 + (size_t)j * n : nullptr;
    GRID_STRIDE(i, n) {
        double v = src[i] * inv;
        vj[i] = v;
        if (vfix) vfix[i] = v;
        if (vj32) vj32[i] = (float)v;
    }
}

// hcol = V^T w over V_0..V_j; T = float: in FP32 (FP32 shadows of the FGMRES basis and of w): the first
// classical Gram-Schmidt pass of the stage FGMRES. Its error (1e-7 of |w|) is removed by the FP64
// second pass, and H uses the same hcol as the update, so the Arnoldi relation stays FP64.
// (T = double: the same pass in FP64, for the all-FP64 precision mode.)
template <class T>
__global__ void k_vec_dot(const T *__restrict__ w, const T *__restrict__ V, long long n, RedBuf rb, GmresState *gs) {
    wait_prior_kernel();
    if (gs->cycle_end) return;
    multidot_rows(rb, V, w, n, gs->j + 1, gs->hcol, false);
}

// Second classical Gram-Schmidt pass of the stage FGMRES, first half: w' = w - V hcol; h2 =
// V^T w' and ||w'||^2 in the same sweep; the last block finishes the Arnoldi step with
// hn = sqrt(||w'||^2 - ||h2||^2) (exact for the w'' = w' - V h2 the next kernel forms, V
// orthonormal; no cancellation: h2 is small against w' after the first pass) and
// H[:, j] = hcol + h2.
__global__ void k_fgm_orth1(double *w, const double *__restrict__ V, long long nrows, RedBuf rb, GmresState *gs) {
    wait_prior_kernel();
    if (gs->cycle_end) return;
    const int j = gs->j, nvec = j + 1;
    __shared__ double h[GM_M + 1];
    if ((int)threadIdx.x < nvec) h[threadIdx.x] = gs->hcol[threadIdx.x];
    __syncthreads();
    const RowChunk ch(nrows);
    for (long long g = ch.r0 + threadIdx.x; g < ch.r1; g += blockDim.x) {
        double s = w[g];
        for (int i = 0; i < nvec; ++i) s -= h[i] * V[(size_t)i * nrows + g];
        w[g] = s;
    }
    __syncthreads();
    const bool last = block_multidot(rb, V, (const double *)w, nrows, nvec,
                                     [&](auto f) { if (ch.r0 < ch.r1) f(ch.r0, ch.r1); }, gs->h2, (const double *)w);
    if (!last) return;
    __syncthreads();
    __shared__ double hn_s;
    if (threadIdx.x == 0) {
        double q = 0.0;
        for (int i = 0; i <= j; ++i) q += gs->h2[i] * gs->h2[i];
        const double ww = gs->h2[j + 1], hn2 = ww - q;
        hn_s = sqrt(hn2 > 1e-24 * ww ? hn2 : 1e-24 * ww);
    }
    __syncthreads();
    gm_finish_step(gs, j, hn_s, true);
}

// Second half: v_{j+1} = (w' - V h2) / hn written to V_{j+1} (and vfix when set), for the step
// the previous kernel finished (gs->j already advanced; nothing when the cycle ended)
__global__ void k_fgm_orth2n(const double *__restrict__ w, double *V, double *vfix, long long nrows,
                             const GmresState *gs, float *V32) {
    wait_prior_kernel();
    if (gs->cycle_end) return;
    const int jn = gs->j;                        // the new basis slot
    __shared__ double h[GM_M + 1];
    __shared__ double inv;
    if ((int)threadIdx.x < jn) h[threadIdx.x] = gs->h2[threadIdx.x];
    if (threadIdx.x == 0) inv = 1.0 / gs->H[(jn - 1) * (GM_M + 1) + jn];
    __syncthreads();
    double *vn = V + (size_t)jn * nrows;
    float *vn32 = V32 ? V32 + (size_t)jn * nrows : nullptr;
    GRID_STRIDE(g, nrows) {
        double s = w[g];
        for (int i = 0; i < jn; ++i) s -= h[i] * V[(size_t)i * nrows + g];
        s *= inv;
        vn[g] = s;
        if (vfix) vfix[g] = s;
        if (vn32) vn32[g] = (float)s;
    }
}

// x += u
__global__ void k_vec_add(const double *__restrict__ u, double *x, long long n) {
    wait_prior_kernel();
    GRID_STRIDE(i, n) x[i] += u[i];
}

// Q += Qbar + U; p += dp; l += dl; norms ||Qbar+U||_M^2, ||Q||_M^2
template <int K>
__global__ void k_rich_update(MeshDev M, double *Q, const double *Qbar, const double *U, double *p,
                              const double *dp, double *lam, const double *dl, RedBuf rb, Scalars *sc) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    double v[2] = {0.0, 0.0}, tot[2];
    const long long nQ = (long long)M.ncells * Dm::NU;
    GRID_STRIDE(i, nQ) {
        double dj = M.geo[i / Dm::NU].detJ;
        double dq = Qbar[i] + U[i];
        double q = Q[i] + dq;
        Q[i] = q;
        v[0] += dj * dq * dq;
        v[1] += dj * q * q;
    }
    GRID_STRIDE(i, (long long)M.ncells * Dm::NP) p[i] += dp[i];
    GRID_STRIDE(i, (long long)M.nfacets * Dm::NT) lam[i] += dl[i];
    if (grid_sum<2>(rb, v, tot)) { sc->red0 = tot[0]; sc->red1 = tot[1]; }
}

// (p)_Omega: sum_K detJ p_K0 * int_T phi_0 = detJ p_K0 / sqrt(2)
template <int K>
__global__ void k_p_integral(MeshDev M, const double *p, RedBuf rb, Scalars *sc) {
    wait_prior_kernel();
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(cl, M.ncells) v[0] += M.geo[cl].detJ * p[(size_t)cl * Dims<K>::NP] * 0.70710678118654752440;
    if (grid_sum<1>(rb, v, tot)) sc->red2 = tot[0];
}

// p -= m (constant), lam -= m, with m = (p)_Omega / area
template <int K>
__global__ void k_p_shift(MeshDev M, double area, double *p, double *lam, const Scalars *sc) {
    wait_prior_kernel();
    const double m = sc->red2 / area;
    GRID_STRIDE(cl, M.ncells) p[(size_t)cl * Dims<K>::NP] -= m * 0.70710678118654752440;   // m = (m/sqrt2) phi_0
    if (lam) GRID_STRIDE(f, M.nfacets) lam[(size_t)f * Dims<K>::NT] -= m;
}

}  // namespace hdg
