// Kernels of the multigrid trace preconditioner (hdg_mg.cuh). Every V-cycle kernel returns at
// once when the CG it serves has converged (Scalars::done), so chunks of iterations can be
// launched ahead of the convergence test.
#pragma once
#include "hdg_kernels.cuh"
#include "hdg_mg.cuh"

namespace hdg {

// ---------------------------------------------------------------- setup
template <int NT>
__global__ void k_p1_cellop(const double *__restrict__ Scell, const int *__restrict__ cell_flip, int ncells,
                            double *cellA) {
    wait_prior_kernel();
    GRID_STRIDE(c, ncells) {
        int flip[3] = {cell_flip[3 * c], cell_flip[3 * c + 1], cell_flip[3 * c + 2]};
        p1_cellop<NT>(Scell + (size_t)c * 9 * NT * NT, flip, cellA + 9 * c);
    }
}

// bit pattern of a non-negative double orders like the value: atomicMax on it is a max
__device__ __forceinline__ void atomic_max_pos(unsigned long long *dst, double v) {
    if (v > 0) atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_p1_assemble(P1Grid G, const double *__restrict__ cellA, const int *__restrict__ vert_cell,
                              const int *__restrict__ cell_vert, double *A, double *dinv, unsigned long long *lmax) {
    wait_prior_kernel();
    GRID_STRIDE(v, G.nverts) {
        double row[P1_NS];
        p1_assemble_row((int)v, G, cellA, vert_cell, cell_vert, row);
        double s = 0;
        for (int o = 0; o < P1_NS; ++o) { A[P1_NS * v + o] = row[o]; s += fabs(row[o]); }
        dinv[v] = 1.0 / row[0];
        atomic_max_pos(lmax, s / row[0]);
    }
}

__global__ void k_p1_coarsen(P1Grid Gc, P1Grid Gf, const double *__restrict__ Af, double *Ac, double *dinv,
                             unsigned long long *lmax) {
    wait_prior_kernel();
    GRID_STRIDE(V, Gc.nverts) {
        double row[P1_NS];
        p1_galerkin_row((int)V, Gc, Gf, Af, row);
        double s = 0;
        for (int o = 0; o < P1_NS; ++o) { Ac[P1_NS * V + o] = row[o]; s += fabs(row[o]); }
        dinv[V] = 1.0 / row[0];
        atomic_max_pos(lmax, s / row[0]);
    }
}

// ||D^{-1} S||_inf over the facet rows (an upper bound of the largest eigenvalue of D^{-1} S)
template <int NT>
__global__ void k_trace_bound(const double *__restrict__ Sell, const int *__restrict__ tcol,
                              const double *__restrict__ Dinv, int nfacets, unsigned long long *lmax) {
    wait_prior_kernel();
    const long long nrows = (long long)nfacets * NT;
    GRID_STRIDE(fl, nfacets) {
        int f = (int)fl;
        double Di[NT][NT];
        for (int i = 0; i < NT; ++i)
            for (int m = 0; m < NT; ++m) Di[i][m] = Dinv[(size_t)m * nrows + (size_t)f * NT + i];
        double best = 0;
        for (int i = 0; i < NT; ++i) {
            double s = 0;
            for (int b = 0; b < 5; ++b) {
                if (tcol[b * nfacets + f] < 0) continue;
                for (int j = 0; j < NT; ++j) {
                    double t = 0;
                    for (int m = 0; m < NT; ++m) t += Di[i][m] * Sell[(size_t)(b * NT + j) * nrows + (size_t)f * NT + m];
                    s += fabs(t);
                }
            }
            best = fmax(best, s);
        }
        atomic_max_pos(lmax, best);
    }
}

// dense pseudo-inverse of the coarsest operator: Minv = (A + 1 1^T / N)^{-1} (one block)
__global__ void k_coarse_inverse(P1Grid G, const double *__restrict__ A, double *B, double *Minv, int *status) {
    wait_prior_kernel();
    const int N = G.nverts;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        B[i] = 1.0 / N;
        Minv[i] = (i / N == i % N) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < N; v += blockDim.x) {
        int i = v % G.nvx, j = v / G.nvx;
        for (int o = 0; o < P1_NS; ++o) {
            int w = p1_vid(G, i + p1_di(o), j + p1_dj(o));
            if (w >= 0) B[(size_t)v * N + w] += A[P1_NS * v + o];
        }
    }
    __syncthreads();
    __shared__ int piv;
    for (int col = 0; col < N; ++col) {             // Gauss-Jordan with partial pivoting
        if (threadIdx.x == 0) {
            int p = col;
            double best = fabs(B[(size_t)col * N + col]);
            for (int r = col + 1; r < N; ++r)
                if (fabs(B[(size_t)r * N + col]) > best) { best = fabs(B[(size_t)r * N + col]); p = r; }
            piv = best > 0 ? p : -1;
            if (piv < 0) *status = 1;
        }
        __syncthreads();
        if (piv < 0) return;
        if (piv != col)
            for (int j = threadIdx.x; j < N; j += blockDim.x) {
                double t = B[(size_t)col * N + j]; B[(size_t)col * N + j] = B[(size_t)piv * N + j]; B[(size_t)piv * N + j] = t;
                t = Minv[(size_t)col * N + j]; Minv[(size_t)col * N + j] = Minv[(size_t)piv * N + j]; Minv[(size_t)piv * N + j] = t;
            }
        __syncthreads();
        double inv = 1.0 / B[(size_t)col * N + col];
        __syncthreads();
        for (int j = threadIdx.x; j < N; j += blockDim.x) { B[(size_t)col * N + j] *= inv; Minv[(size_t)col * N + j] *= inv; }
        __syncthreads();
        for (int idx = threadIdx.x; idx < (N - 1) * N; idx += blockDim.x) {
            int r = idx / N, j = idx % N;
            if (r >= col) ++r;
            double f = B[(size_t)r * N + col];
            if (j != col) B[(size_t)r * N + j] -= f * B[(size_t)col * N + j];
            Minv[(size_t)r * N + j] -= f * Minv[(size_t)col * N + j];
        }
        __syncthreads();
        for (int r = threadIdx.x; r < N; r += blockDim.x)
            if (r != col) B[(size_t)r * N + col] = 0.0;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- V-cycle: trace level
template <int NT>
__global__ void k_tcheb0(const double *__restrict__ Dinv, const double *__restrict__ b, double *x, double *d,
                         double invth, int nfacets, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const long long nrows = (long long)nfacets * NT;
    GRID_STRIDE(fl, nfacets) {
        double bl[NT];
        for (int j = 0; j < NT; ++j) bl[j] = b[fl * NT + j];
        for (int i = 0; i < NT; ++i) {
            double s = 0;
            for (int j = 0; j < NT; ++j) s += Dinv[(size_t)j * nrows + fl * NT + i] * bl[j];
            s *= invth;
            d[fl * NT + i] = s;
            x[fl * NT + i] = s;
        }
    }
}

// r = b - S xin (facet rows); d = c1 d + c2 Dinv r; xout = xin + d
template <int NT>
__global__ void k_tcheb(const double *__restrict__ Sell, const int *__restrict__ tcol,
                        const double *__restrict__ Dinv, const double *__restrict__ b,
                        const double *__restrict__ xin, double *__restrict__ xout, double *d, double c1, double c2,
                        int nfacets, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const long long nrows = (long long)nfacets * NT;
    GRID_STRIDE(fl, nfacets) {
        int f = (int)fl;
        double r[NT];
        for (int i = 0; i < NT; ++i) r[i] = b[(size_t)f * NT + i];
        for (int bb = 0; bb < 5; ++bb) {
            int cf = __ldg(&tcol[bb * nfacets + f]);
            if (cf < 0) continue;
            for (int j = 0; j < NT; ++j) {
                double xv = xin[(size_t)cf * NT + j];
                for (int i = 0; i < NT; ++i) r[i] -= __ldg(&Sell[(size_t)(bb * NT + j) * nrows + (size_t)f * NT + i]) * xv;
            }
        }
        for (int i = 0; i < NT; ++i) {
            double s = 0;
            for (int j = 0; j < NT; ++j) s += Dinv[(size_t)j * nrows + (size_t)f * NT + i] * r[j];
            size_t g = (size_t)f * NT + i;
            double dn = c1 * d[g] + c2 * s;
            d[g] = dn;
            xout[g] = xin[g] + dn;
        }
    }
}

template <int NT>
__global__ void k_tresid(const double *__restrict__ Sell, const int *__restrict__ tcol, const double *__restrict__ b,
                         const double *__restrict__ x, double *__restrict__ t, int nfacets, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const long long nrows = (long long)nfacets * NT;
    GRID_STRIDE(g, nrows) {
        int f = (int)(g / NT);
        double s = b[g];
        for (int bb = 0; bb < 5; ++bb) {
            int cf = __ldg(&tcol[bb * nfacets + f]);
            if (cf < 0) continue;
            for (int j = 0; j < NT; ++j) s -= __ldg(&Sell[(size_t)(bb * NT + j) * nrows + g]) * x[(size_t)cf * NT + j];
        }
        t[g] = s;
    }
}

template <int NT>
__global__ void k_restrict_t(int nverts, const double *__restrict__ t, const int *__restrict__ vert_facet,
                             const int *__restrict__ vert_fsign, double *b1, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    GRID_STRIDE(v, nverts) b1[v] = restrict_trace<NT>((int)v, t, vert_facet, vert_fsign);
}

template <int NT>
__global__ void k_prolong_t(const int *__restrict__ facet_vert, const double *__restrict__ e1, double *x, int nfacets,
                            const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const double s3 = 0.28867513459481288225;
    GRID_STRIDE(f, nfacets) {
        double a = e1[facet_vert[2 * f]], b = e1[facet_vert[2 * f + 1]];
        x[(size_t)f * NT] += 0.5 * (a + b);
        x[(size_t)f * NT + 1] += s3 * (b - a);
    }
}

// ---------------------------------------------------------------- V-cycle: P1 levels
__global__ void k_pcheb0(const double *__restrict__ dinv, const double *__restrict__ b, double *x, double *d,
                         double invth, int n, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    GRID_STRIDE(v, n) {
        double s = dinv[v] * b[v] * invth;
        d[v] = s;
        x[v] = s;
    }
}

__global__ void k_pcheb(P1Grid G, const double *__restrict__ A, const double *__restrict__ dinv,
                        const double *__restrict__ b, const double *__restrict__ xin, double *__restrict__ xout,
                        double *d, double c1, double c2, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    GRID_STRIDE(v, G.nverts) {
        double r = b[v] - p1_apply((int)v, G, A, xin);
        double dn = c1 * d[v] + c2 * dinv[v] * r;
        d[v] = dn;
        xout[v] = xin[v] + dn;
    }
}

__global__ void k_presid(P1Grid G, const double *__restrict__ A, const double *__restrict__ b,
                         const double *__restrict__ x, double *t, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    GRID_STRIDE(v, G.nverts) t[v] = b[v] - p1_apply((int)v, G, A, x);
}

__global__ void k_prestrict(P1Grid Gc, P1Grid Gf, const double *__restrict__ tf, double *bc, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    GRID_STRIDE(V, Gc.nverts) bc[V] = restrict_p1((int)V, Gc, Gf, tf);
}

__global__ void k_pprolong(P1Grid Gf, P1Grid Gc, const double *__restrict__ ec, double *x, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    GRID_STRIDE(a, Gf.nverts) x[a] += prolong_p1((int)a, Gf, Gc, ec);
}

// x = Minv (b - mean(b))   (one block)
__global__ void k_coarse_solve(int N, const double *__restrict__ Minv, const double *__restrict__ b, double *x,
                               const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    __shared__ double sh[1][32];
    __shared__ double mean;
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < N; i += blockDim.x) v[0] += b[i];
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) mean = v[0] / N;
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double s = 0;
        for (int j = 0; j < N; ++j) s += Minv[(size_t)i * N + j] * (b[j] - mean);
        x[i] = s;
    }
}

// ---------------------------------------------------------------- CG with the V-cycle
// r = b - mean e0, x = 0, pold = 0 (z = M r follows)
template <int NT>
__global__ void k_cg_setup_mg(const double *__restrict__ b, double *x, double *r, double *pold, int nfacets,
                              Scalars *sc) {
    wait_prior_kernel();
    const double mean = sc->bmean;
    GRID_STRIDE(g, (long long)nfacets * NT) {
        r[g] = b[g] - ((g % NT) == 0 ? mean : 0.0);
        x[g] = 0.0;
        pold[g] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->done = 0; sc->beta = 0.0; sc->iters = 0; sc->breakdown = 0;      // rtol, maxit: k_set_tol
    }
}

// r = b - mean e0 - S x (stationary V-cycle iteration of the inner trace solves)
template <int NT>
__global__ void k_trace_resid(const double *__restrict__ Sell, const int *__restrict__ tcol,
                              const double *__restrict__ b, const double *__restrict__ x, double *r, int nfacets,
                              const Scalars *sc) {
    wait_prior_kernel();
    const double mean = sc->bmean;
    const long long nrows = (long long)nfacets * NT;
    GRID_STRIDE(g, nrows) {
        const int f = (int)(g / NT);
        double s = b[g] - ((g % NT) == 0 ? mean : 0.0);
        for (int bb = 0; bb < 5; ++bb) {
            const int cf = __ldg(&tcol[bb * nfacets + f]);
            if (cf < 0) continue;
            for (int j = 0; j < NT; ++j)
                s -= __ldg(&Sell[(size_t)(bb * NT + j) * nrows + g]) * x[(size_t)cf * NT + j];
        }
        r[g] = s;
    }
}

// x += z (the V-cycle correction)
__global__ void k_axpy_done(const double *__restrict__ z, double *x, long long n, const Scalars *sc) {
    wait_prior_kernel();
    GRID_STRIDE(i, n) x[i] += z[i];
}

// x += alpha p; r -= alpha Ap
__global__ void k_cg_update_nz(const double *__restrict__ p, const double *__restrict__ Ap, double *x, double *r,
                               long long n, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const double alpha = sc->alpha;
    GRID_STRIDE(i, n) {
        x[i] += alpha * p[i];
        r[i] -= alpha * Ap[i];
    }
}

// rz = (r, z) and the mean of z's constant trace mode (removed from the direction by
// k_cg_apply); first: rz0 = rz; else beta = rz_new / rz and convergence
template <int NT>
__global__ void k_cg_rz(const double *__restrict__ r, const double *__restrict__ z, int nfacets, int first,
                        RedBuf rb, Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    double v[3] = {0.0, 0.0, 0.0}, tot[3];
    GRID_STRIDE(i, (long long)nfacets * NT) {
        v[0] += r[i] * z[i];
        if (i % NT == 0) { v[1] += z[i]; v[2] += r[i]; }
    }
    if (grid_sum<3>(rb, v, tot)) {
        sc->zmean = tot[1] / nfacets;
        double rz = tot[0] - sc->zmean * tot[2];      // (r, z - zmean e0)
        if (first) {
            sc->rz = rz; sc->rz0 = rz; sc->relres = rz > 0 ? 1.0 : 0.0;
            if (!isfinite(rz)) { sc->done = 1; sc->breakdown = 2; }
            else if (!(rz > 0.0)) sc->done = 1;
        } else {
            sc->beta = rz / sc->rz;
            sc->rz = rz;
            sc->iters += 1;
            double rel = sc->rz0 > 0 ? sqrt(fmax(rz, 0.0) / sc->rz0) : 0.0;
            sc->relres = rel;
            if (!isfinite(rz)) { sc->done = 1; sc->breakdown = 2; }
            else if (rel <= sc->rtol || sc->iters >= sc->maxit) sc->done = 1;
        }
    }
}

// tolerances of the next solve (kept out of the captured graphs, which serve every tolerance)
__global__ void k_set_tol(Scalars *sc, double rtol, int maxit) {
    wait_prior_kernel();
    sc->rtol = rtol;
    sc->maxit = maxit;
}

__global__ void k_gm_set_tol(GmresState *gs, double rtol, int maxit) {
    wait_prior_kernel();
    gs->rtol = rtol;
    gs->maxit = maxit;
}

// instrumentation: put an Arnoldi step j of a live cycle in place (one kernel timed alone)
__global__ void k_gm_set_step(GmresState *gs, int j) {
    wait_prior_kernel();
    gs->j = j;
    gs->cycle_end = 0;
}

}  // namespace hdg

namespace hdg {

// ---------------------------------------------------------------- fused coarse part of the V-cycle
// The P1 levels from `first` down (their grids are small) and the coarsest solve run in one thread
// block, levels separated by __syncthreads (global writes of a block are visible to the block after
// the barrier). With first == 0 the kernel also restricts the trace residual to level 1 and
// prolongs the level-1 correction back to the trace.
constexpr int MG_MAX_LEVELS = 16;
struct MGTail {
    int first, L, Nc, nfacets;
    P1Grid G[MG_MAX_LEVELS];
    const double *A[MG_MAX_LEVELS];
    const double *dinv[MG_MAX_LEVELS];
    double invth[MG_MAX_LEVELS], c1[MG_MAX_LEVELS], c2[MG_MAX_LEVELS];
    double *b[MG_MAX_LEVELS], *xa[MG_MAX_LEVELS], *xb[MG_MAX_LEVELS], *d[MG_MAX_LEVELS], *t[MG_MAX_LEVELS];
    const double *Minv;
    const int *vert_facet, *vert_fsign, *facet_vert;
    const double *tres;      // trace residual (first == 0)
    double *z;               // trace iterate to correct (first == 0)
};

template <int NT>
__global__ void __launch_bounds__(1024) k_mg_tail(MGTail T, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const int tid = threadIdx.x, nth = blockDim.x;
    if (T.first == 0)
        for (int v = tid; v < T.G[0].nverts; v += nth) T.b[0][v] = restrict_trace<NT>(v, T.tres, T.vert_facet, T.vert_fsign);
    __syncthreads();
    for (int l = T.first; l < T.L - 1; ++l) {
        const P1Grid G = T.G[l];
        const double *A = T.A[l], *dv = T.dinv[l];
        double *b = T.b[l], *xa = T.xa[l], *xb = T.xb[l], *d = T.d[l], *t = T.t[l];
        for (int v = tid; v < G.nverts; v += nth) { double s = dv[v] * b[v] * T.invth[l]; d[v] = s; xa[v] = s; }
        __syncthreads();
        for (int v = tid; v < G.nverts; v += nth) {
            double dn = T.c1[l] * d[v] + T.c2[l] * dv[v] * (b[v] - p1_apply(v, G, A, xa));
            d[v] = dn;
            xb[v] = xa[v] + dn;
        }
        __syncthreads();
        for (int v = tid; v < G.nverts; v += nth) t[v] = b[v] - p1_apply(v, G, A, xb);
        __syncthreads();
        for (int V = tid; V < T.G[l + 1].nverts; V += nth) T.b[l + 1][V] = restrict_p1(V, T.G[l + 1], G, t);
        __syncthreads();
    }
    {   // coarsest: x = Minv (b - mean b)
        __shared__ double sh[1][32];
        __shared__ double mean;
        const int N = T.Nc;
        const double *b = T.b[T.L - 1];
        double v[1] = {0.0};
        for (int i = tid; i < N; i += nth) v[0] += b[i];
        block_sum<1>(v, sh);
        if (tid == 0) mean = v[0] / N;
        __syncthreads();
        for (int i = tid; i < N; i += nth) {
            double s = 0;
            for (int j = 0; j < N; ++j) s += T.Minv[(size_t)i * N + j] * (b[j] - mean);
            T.xb[T.L - 1][i] = s;
        }
        __syncthreads();
    }
    for (int l = T.L - 2; l >= T.first; --l) {
        const P1Grid G = T.G[l];
        const double *A = T.A[l], *dv = T.dinv[l];
        double *b = T.b[l], *xa = T.xa[l], *xb = T.xb[l], *d = T.d[l];
        for (int a = tid; a < G.nverts; a += nth) xb[a] += prolong_p1(a, G, T.G[l + 1], T.xb[l + 1]);
        __syncthreads();
        for (int v = tid; v < G.nverts; v += nth) {
            double dn = T.invth[l] * dv[v] * (b[v] - p1_apply(v, G, A, xb));
            d[v] = dn;
            xa[v] = xb[v] + dn;
        }
        __syncthreads();
        for (int v = tid; v < G.nverts; v += nth) {
            double dn = T.c1[l] * d[v] + T.c2[l] * dv[v] * (b[v] - p1_apply(v, G, A, xa));
            d[v] = dn;
            xb[v] = xa[v] + dn;
        }
        __syncthreads();
    }
    if (T.first == 0) {
        const double s3 = 0.28867513459481288225;
        const double *e1 = T.xb[0];
        for (int f = tid; f < T.nfacets; f += nth) {
            double a = e1[T.facet_vert[2 * f]], bb = e1[T.facet_vert[2 * f + 1]];
            T.z[(size_t)f * NT] += 0.5 * (a + bb);
            T.z[(size_t)f * NT + 1] += s3 * (bb - a);
        }
    }
}

// ---------------------------------------------------------------- fused CG steps
// x += alpha p; r -= alpha Ap; then the first Chebyshev step of the V-cycle on r:
// d = Dinv r / theta, z = d
template <int NT>
__global__ void k_cg_update_cheb0(const double *__restrict__ p, const double *__restrict__ Ap, double *x, double *r,
                                  const double *__restrict__ Dinv, double *z, double *d, double invth, int nfacets,
                                  const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const double alpha = sc->alpha;
    const long long nrows = (long long)nfacets * NT;
    GRID_STRIDE(fl, nfacets) {
        double rl[NT];
        for (int i = 0; i < NT; ++i) {
            size_t g = (size_t)fl * NT + i;
            x[g] += alpha * p[g];
            rl[i] = r[g] - alpha * Ap[g];
            r[g] = rl[i];
        }
        for (int i = 0; i < NT; ++i) {
            double s = 0;
            for (int j = 0; j < NT; ++j) s += Dinv[(size_t)j * nrows + fl * NT + i] * rl[j];
            s *= invth;
            d[fl * NT + i] = s;
            z[fl * NT + i] = s;
        }
    }
}

// last Chebyshev step of the V-cycle (b = the CG residual r) fused with the CG reduction:
// xout = z; rz = (r, z - zmean e0), zmean; first: rz0, else beta and convergence
template <int NT>
__global__ void k_tcheb_rz(const double *__restrict__ Sell, const int *__restrict__ tcol,
                           const double *__restrict__ Dinv, const double *__restrict__ b,
                           const double *__restrict__ xin, double *__restrict__ xout, double *d, double c1, double c2,
                           int nfacets, int first, RedBuf rb, Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const long long nrows = (long long)nfacets * NT;
    double v[3] = {0.0, 0.0, 0.0}, tot[3];
    GRID_STRIDE(fl, nfacets) {
        int f = (int)fl;
        double r[NT], bl[NT];
        for (int i = 0; i < NT; ++i) { bl[i] = b[(size_t)f * NT + i]; r[i] = bl[i]; }
        for (int bb = 0; bb < 5; ++bb) {
            int cf = __ldg(&tcol[bb * nfacets + f]);
            if (cf < 0) continue;
            for (int j = 0; j < NT; ++j) {
                double xv = xin[(size_t)cf * NT + j];
                for (int i = 0; i < NT; ++i) r[i] -= __ldg(&Sell[(size_t)(bb * NT + j) * nrows + (size_t)f * NT + i]) * xv;
            }
        }
        for (int i = 0; i < NT; ++i) {
            double s = 0;
            for (int j = 0; j < NT; ++j) s += Dinv[(size_t)j * nrows + (size_t)f * NT + i] * r[j];
            size_t g = (size_t)f * NT + i;
            double dn = c1 * d[g] + c2 * s;
            d[g] = dn;
            double zn = xin[g] + dn;
            xout[g] = zn;
            v[0] += bl[i] * zn;
            if (i == 0) { v[1] += zn; v[2] += bl[0]; }
        }
    }
    if (grid_sum<3>(rb, v, tot)) {
        sc->zmean = tot[1] / nfacets;
        double rz = tot[0] - sc->zmean * tot[2];
        if (first) {
            sc->rz = rz; sc->rz0 = rz; sc->relres = rz > 0 ? 1.0 : 0.0;
            if (!isfinite(rz)) { sc->done = 1; sc->breakdown = 2; }
            else if (!(rz > 0.0)) sc->done = 1;
        } else {
            sc->beta = rz / sc->rz;
            sc->rz = rz;
            sc->iters += 1;
            double rel = sc->rz0 > 0 ? sqrt(fmax(rz, 0.0) / sc->rz0) : 0.0;
            sc->relres = rel;
            if (!isfinite(rz)) { sc->done = 1; sc->breakdown = 2; }
            else if (rel <= sc->rtol || sc->iters >= sc->maxit) sc->done = 1;
        }
    }
}

}  // namespace hdg
