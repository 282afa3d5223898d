// FP32 V-cycle of the trace multigrid (Sec. 2.8), used as the preconditioner's inner Step II
// (one V-cycle on the condensed trace system inside the flexible outer iteration). Same cycle as
// the FP64 one in hdg_mg_kernels.cuh — degree-2 Chebyshev on the facet block-Jacobi
// preconditioner, P1 Galerkin levels with degree-2 Chebyshev smoothing, dense pseudo-inverse on
// the coarsest grid — with operators rounded to FP32 once per stage coefficient. In six kernels:
//   k_tv_gather  : b = (sum of the cells' lambda-row contributions) - v_lambda, mean of b_0
//   k_tv_cheb01  : r = b - mean e0; the first two Chebyshev steps from x = 0
//   k_tv_resid   : t = r - S x
//   k_tv_tail    : one block: t -> P1 level 1, the whole P1 hierarchy in shared memory, x += P e
//   k_tv_cheb x2 : the two post-smoothing steps; the last writes the FP64 result
// A trace-level thread owns one row (facet f, component i) and works in a group of G lanes per
// facet (G = NT rounded up to a power of two), so the facet block-Jacobi product is a
// shuffle within the group. GB300's FP32 rate is 64x its FP64 rate: these kernels are bound by
// latency, not arithmetic.
#pragma once
#include "hdg_mg_kernels.cuh"

namespace hdg {

template <int NT>
struct TGrp {
    static constexpr int G = NT <= 2 ? 2 : (NT <= 4 ? 4 : 8);
};

struct TraceOp32 {
    const float *Sell, *Dinv;   // as the FP64 operator: Sell[(b NT + j) nrows + f NT + i], Dinv[j nrows + f NT + i]
    const int *tcol;            // tcol[b nfacets + f]: facet of block b (b = 0: f itself), -1: none
    int nfacets;
};

// (row ic of the facet block D_f^{-1}) . r, r spread over the group (lane i holds r_i, 0 past NT)
template <int NT>
__device__ __forceinline__ float grp_dinv(const float *__restrict__ Dinv, long long nrows, int f, int ic, float r) {
    constexpr int G = TGrp<NT>::G;
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const float rj = __shfl_sync(0xffffffffu, r, j, G);
        s += __ldg(&Dinv[(size_t)j * nrows + (size_t)f * NT + ic]) * rj;
    }
    return s;
}

// row (f, ic) of S x: x read per neighbour facet (the group's lanes read the same values)
template <int NT>
__device__ __forceinline__ float row_S(const TraceOp32 &T, long long nrows, int f, int ic, const float *__restrict__ x) {
    float s = 0.f;
#pragma unroll
    for (int bb = 0; bb < 5; ++bb) {
        const int cf = __ldg(&T.tcol[bb * T.nfacets + f]);
        if (cf < 0) continue;                                  // uniform over the group
#pragma unroll
        for (int j = 0; j < NT; ++j)
            s += __ldg(&T.Sell[(size_t)(bb * NT + j) * nrows + (size_t)f * NT + ic]) * __ldcg(&x[(size_t)cf * NT + j]);
    }
    return s;
}

// thread -> (facet, row) of the group layout; live = a row that exists
#define TV_ROW(NT_)                                                                    \
    constexpr int G = TGrp<NT_>::G;                                                    \
    const long long t_ = (long long)blockIdx.x * blockDim.x + threadIdx.x;             \
    const int i = (int)(t_ % G);                                                       \
    int f = (int)(t_ / G);                                                             \
    const bool live = f < T.nfacets && i < NT_;                                        \
    if (f >= T.nfacets) f = T.nfacets - 1;                                             \
    const int ic = i < NT_ ? i : 0;                                                    \
    const long long nrows = (long long)T.nfacets * NT_;                                \
    const size_t g = (size_t)f * NT_ + ic;

inline unsigned tv_blocks(long long nfacets, int G) { return (unsigned)((nfacets * G + 127) / 128); }

// b = sum over the facet's cells of v (cell lambda rows) - sub, in FP32; the last block stores
// the mean of the b_0 components in sc->bmean and counts the solve (acc non-null).
template <int NT>
__global__ void k_tv_gather(MeshDev M, const double *__restrict__ v, const double *__restrict__ sub, float *b32,
                            RedBuf rb, Scalars *sc, DevCount *acc) {
    wait_prior_kernel();
    double s0[1] = {0.0}, tot[1];
    GRID_STRIDE(gi, (long long)M.nfacets * NT) {
        const int f = (int)(gi / NT), j = (int)(gi % NT);
        double s = sub ? -sub[gi] : 0.0;
        for (int side = 0; side < 2; ++side) {
            const int c = M.facet_cell[2 * f + side];
            if (c < 0) continue;
            s += v[(size_t)c * 3 * NT + M.facet_edge[2 * f + side] * NT + j];
        }
        b32[gi] = (float)s;
        if (j == 0) s0[0] += s;
    }
    if (grid_sum<1>(rb, s0, tot)) {
        sc->bmean = tot[0] / M.nfacets;
        if (acc) acc->trace_solves += 1;
    }
}

// r = b - mean e0; x0 = d0 = invth D^{-1} r; r1 = r - S x0 (x0 of the neighbours formed here from
// their b); d1 = c1 d0 + c2 D^{-1} r1; x1 = x0 + d1.  Writes r, x1, d1.
template <int NT>
__global__ void k_tv_cheb01(TraceOp32 T, const float *__restrict__ b, const Scalars *sc, float invth, float c1,
                            float c2, float *r, float *x, float *d) {
    wait_prior_kernel();
    TV_ROW(NT)
    const float mean = (float)sc->bmean;
    const float rown = i < NT ? __ldcg(&b[g]) - (i == 0 ? mean : 0.f) : 0.f;
    float sx = 0.f;
#pragma unroll
    for (int bb = 0; bb < 5; ++bb) {
        const int cf = __ldg(&T.tcol[bb * T.nfacets + f]);
        const int cfc = cf >= 0 ? cf : f;
        const float rn = i < NT ? __ldcg(&b[(size_t)cfc * NT + ic]) - (i == 0 ? mean : 0.f) : 0.f;
        float xn = invth * grp_dinv<NT>(T.Dinv, nrows, cfc, ic, rn);
        if (cf < 0) xn = 0.f;
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const float xj = __shfl_sync(0xffffffffu, xn, j, G);
            s += __ldg(&T.Sell[(size_t)(bb * NT + j) * nrows + g]) * xj;
        }
        sx += s;
    }
    const float x0 = invth * grp_dinv<NT>(T.Dinv, nrows, f, ic, rown);
    const float d1 = c1 * x0 + c2 * grp_dinv<NT>(T.Dinv, nrows, f, ic, rown - sx);
    if (live) {
        r[g] = rown;
        x[g] = x0 + d1;
        d[g] = d1;
    }
}

// t = r - S x
template <int NT>
__global__ void k_tv_resid(TraceOp32 T, const float *__restrict__ r, const float *__restrict__ x, float *t) {
    wait_prior_kernel();
    TV_ROW(NT)
    (void)G;
    const float s = __ldcg(&r[g]) - row_S<NT>(T, nrows, f, ic, x);
    if (live) t[g] = s;
}

// d = c1 d + c2 D^{-1} (r - S xin); xout = xin + d (FP32), or out64 = xin + d when out64 is set
template <int NT>
__global__ void k_tv_cheb(TraceOp32 T, const float *__restrict__ r, const float *__restrict__ xin, float *xout,
                          float *d, float c1, float c2, double *out64) {
    wait_prior_kernel();
    TV_ROW(NT)
    (void)G;
    const float res = i < NT ? __ldcg(&r[g]) - row_S<NT>(T, nrows, f, ic, xin) : 0.f;
    const float dn = (c1 != 0.f ? c1 * __ldcg(&d[g]) : 0.f) + c2 * grp_dinv<NT>(T.Dinv, nrows, f, ic, res);
    if (live) {
        const float xo = __ldcg(&xin[g]) + dn;
        d[g] = dn;
        if (out64) out64[g] = (double)xo;
        else xout[g] = xo;
    }
}

// ---------------------------------------------------------------- P1 levels in one block
// Neighbour of grid point (i, j) at offset (di, dj), |di|, |dj| <= 1: vertex id, or -1 outside
// a non-periodic grid (no division: the offsets are one step)
__device__ __forceinline__ int p1_nb32(const P1Grid &G, int i, int j, int di, int dj) {
    i += di; j += dj;
    if (i < 0) { if (!G.px) return -1; i += G.nvx; }
    else if (i >= G.nvx) { if (!G.px) return -1; i -= G.nvx; }
    if (j < 0) { if (!G.py) return -1; j += G.nvy; }
    else if (j >= G.nvy) { if (!G.py) return -1; j -= G.nvy; }
    return j * G.nvx + i;
}

// (A x)(v) for the 7-point stencil (entries of missing neighbours are zero)
__device__ __forceinline__ float p1_apply32(const P1Grid &G, const float *__restrict__ A, int v, int i, int j,
                                            const float *x) {
    float s = 0.f;
#pragma unroll
    for (int o = 0; o < P1_NS; ++o) {
        const int w = p1_nb32(G, i, j, p1_di(o), p1_dj(o));
        if (w >= 0) s += __ldg(&A[P1_NS * v + o]) * x[w];
    }
    return s;
}

struct Tail32 {
    int L, Nc, nfacets;
    P1Grid G[MG_MAX_LEVELS];
    const float *A[MG_MAX_LEVELS], *dinv[MG_MAX_LEVELS];
    float invth[MG_MAX_LEVELS], c1[MG_MAX_LEVELS], c2[MG_MAX_LEVELS];
    int off[MG_MAX_LEVELS];        // shared-memory offset (floats) of the level's 4 vectors b, xa, xb, d
    const float *Minv;             // coarsest grid: (A + 1 1^T / N)^{-1}, row-major
    const int *vert_facet, *vert_fsign, *facet_vert;
    const float *tres;             // trace residual t
    float *z;                      // trace iterate corrected by P e (components 0 and 1 of each facet)
};

// shared floats the tail needs for the grids G[0..L-1]
inline size_t tail32_floats(const P1Grid *G, int L) {
    size_t n = 0;
    for (int l = 0; l < L; ++l) n += 4 * (size_t)G[l].nverts;
    return n;
}

#define TAIL_FOR(v_, n_) for (int v_ = threadIdx.x; v_ < (n_); v_ += blockDim.x)

template <int NT>
__global__ void __launch_bounds__(1024) k_tv_tail(Tail32 T) {
    wait_prior_kernel();
    extern __shared__ float tsm[];
    const float s3 = 0.28867513459481288225f;              // 1 / (2 sqrt 3)
    {   // b_1 = P^T t: a facet gives 0.5 t_0 +- t_1 / (2 sqrt 3) to each of its vertices
        float *b = tsm + T.off[0];
        TAIL_FOR(v, T.G[0].nverts) {
            float s = 0.f;
            for (int q = 0; q < 6; ++q) {
                const int f = __ldg(&T.vert_facet[6 * v + q]);
                if (f < 0) continue;
                s += 0.5f * __ldcg(&T.tres[(size_t)f * NT]) +
                     (float)__ldg(&T.vert_fsign[6 * v + q]) * s3 * __ldcg(&T.tres[(size_t)f * NT + 1]);
            }
            b[v] = s;
        }
    }
    __syncthreads();
    for (int l = 0; l < T.L - 1; ++l) {                    // down: two Chebyshev steps, restrict
        const P1Grid G = T.G[l];
        const float *A = T.A[l], *dv = T.dinv[l];
        float *b = tsm + T.off[l], *xa = b + G.nverts, *xb = xa + G.nverts, *d = xb + G.nverts;
        const float invth = T.invth[l], c1 = T.c1[l], c2 = T.c2[l];
        TAIL_FOR(v, G.nverts) {
            const float s = __ldg(&dv[v]) * b[v] * invth;
            d[v] = s;
            xa[v] = s;
        }
        __syncthreads();
        TAIL_FOR(v, G.nverts) {
            const int i = v % G.nvx, j = v / G.nvx;
            const float dn = c1 * d[v] + c2 * __ldg(&dv[v]) * (b[v] - p1_apply32(G, A, v, i, j, xa));
            d[v] = dn;
            xb[v] = xa[v] + dn;
        }
        __syncthreads();
        TAIL_FOR(v, G.nverts) {                             // residual into d (not needed again)
            const int i = v % G.nvx, j = v / G.nvx;
            d[v] = b[v] - p1_apply32(G, A, v, i, j, xb);
        }
        __syncthreads();
        const P1Grid Gc = T.G[l + 1];
        float *bc = tsm + T.off[l + 1];
        TAIL_FOR(V, Gc.nverts) {                            // (I^T r)(V), I = linear interpolation
            const int I = V % Gc.nvx, J = V / Gc.nvx;
            float s = 0.f;
#pragma unroll
            for (int o = 0; o < P1_NS; ++o) {
                const int a = p1_nb32(G, 2 * I, 2 * J, p1_di(o), p1_dj(o));
                if (a >= 0) s += (o == 0 ? 1.f : 0.5f) * d[a];
            }
            bc[V] = s;
        }
        __syncthreads();
    }
    {   // coarsest: x = Minv (b - mean b)
        const int N = T.Nc;
        float *b = tsm + T.off[T.L - 1], *xb = b + 2 * N;
        __shared__ float part[32];
        __shared__ float mean;
        float s = 0.f;
        TAIL_FOR(v, N) s += b[v];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = 0.f;
            for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) m += part[w];
            mean = m / N;
        }
        __syncthreads();
        TAIL_FOR(v, N) {
            float acc = 0.f;
            for (int c = 0; c < N; ++c) acc += __ldg(&T.Minv[(size_t)v * N + c]) * (b[c] - mean);
            xb[v] = acc;
        }
        __syncthreads();
    }
    for (int l = T.L - 2; l >= 0; --l) {                   // up: prolong, two Chebyshev steps
        const P1Grid G = T.G[l], Gc = T.G[l + 1];
        const float *A = T.A[l], *dv = T.dinv[l];
        float *b = tsm + T.off[l], *xa = b + G.nverts, *xb = xa + G.nverts, *d = xb + G.nverts;
        const float *ec = tsm + T.off[l + 1] + 2 * Gc.nverts;
        const float invth = T.invth[l], c1 = T.c1[l], c2 = T.c2[l];
        TAIL_FOR(a, G.nverts) {                             // xb += I e (linear interpolation)
            const int i = a % G.nvx, j = a / G.nvx, i0 = i >> 1, j0 = j >> 1;
            const int oi = i & 1, oj = j & 1;
            float e = ec[p1_nb32(Gc, i0, j0, 0, 0)];
            if (oi || oj) e = 0.5f * (e + ec[p1_nb32(Gc, i0, j0, oi, oj)]);
            xb[a] += e;
        }
        __syncthreads();
        TAIL_FOR(v, G.nverts) {
            const int i = v % G.nvx, j = v / G.nvx;
            const float dn = invth * __ldg(&dv[v]) * (b[v] - p1_apply32(G, A, v, i, j, xb));
            d[v] = dn;
            xa[v] = xb[v] + dn;
        }
        __syncthreads();
        TAIL_FOR(v, G.nverts) {
            const int i = v % G.nvx, j = v / G.nvx;
            const float dn = c1 * d[v] + c2 * __ldg(&dv[v]) * (b[v] - p1_apply32(G, A, v, i, j, xa));
            d[v] = dn;
            xb[v] = xa[v] + dn;
        }
        __syncthreads();
    }
    {   // z += P e_1: components 0 and 1 of each facet from its two vertices
        const float *e1 = tsm + T.off[0] + 2 * T.G[0].nverts;
        TAIL_FOR(f, T.nfacets) {
            const float a = e1[__ldg(&T.facet_vert[2 * f])], bb = e1[__ldg(&T.facet_vert[2 * f + 1])];
            T.z[(size_t)f * NT] += 0.5f * (a + bb);
            T.z[(size_t)f * NT + 1] += s3 * (bb - a);
        }
    }
}

__global__ void k_f64_to_f32(const double *__restrict__ a, float *b, long long n) {
    wait_prior_kernel();
    GRID_STRIDE(i, n) b[i] = (float)a[i];
}

}  // namespace hdg
