// FP32 V-cycle of the trace multigrid (Sec. 2.8), used as the preconditioner's inner Step II
// (one V-cycle on the condensed trace system inside the flexible outer iteration). Same cycle as
// the FP64 one in hdg_mg_kernels.cuh — degree-2 Chebyshev on the facet block-Jacobi
// preconditioner, P1 Galerkin levels with degree-2 Chebyshev smoothing, dense pseudo-inverse on
// the coarsest grid — with operators rounded to FP32 once per stage coefficient. In six kernels:
//   k_tv_gather  : b = (sum of the cells' lambda-row contributions) - v_lambda, mean of b_0
//   k_tv_cheb01  : r = b - mean e0; the first two Chebyshev steps from x = 0
//   k_tv_restrict: b_1 = P^T (r - S x) at the mesh vertices (rows 0 and 1 of the residual at
//                  the vertex's facets, a 16-lane group per vertex)
//   k_tv_tail    : one block: the whole P1 hierarchy in shared memory, e_1 out
//   k_tv_cheb x2 : the two post-smoothing steps (the first from x + P e_1, formed on the fly;
//                  the last writes the FP64 result)
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
// b64 (when set, in place of b): an FP64 right-hand side; sc null: no mean removed.
template <int NT>
__global__ void k_tv_cheb01(TraceOp32 T, const float *__restrict__ b, const double *__restrict__ b64,
                            const Scalars *sc, float invth, float c1, float c2, float *r, float *x, float *d) {
    wait_prior_kernel();
    TV_ROW(NT)
    const float mean = sc ? (float)sc->bmean : 0.f;
    auto bv = [&](size_t k) { return b64 ? (float)__ldcg(&b64[k]) : __ldcg(&b[k]); };
    const float rown = i < NT ? bv(g) - (i == 0 ? mean : 0.f) : 0.f;
    float sx = 0.f;
#pragma unroll
    for (int bb = 0; bb < 5; ++bb) {
        const int cf = __ldg(&T.tcol[bb * T.nfacets + f]);
        const int cfc = cf >= 0 ? cf : f;
        const float rn = i < NT ? bv((size_t)cfc * NT + ic) - (i == 0 ? mean : 0.f) : 0.f;
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

// b_1(v) = sum over the facets f of vertex v of 0.5 t_f0 + sign(v, f) t_f1 / (2 sqrt 3), t = r - S x:
// lane (q, row) of a vertex's 16-lane group forms row `row` of t at its q-th facet; the group sums
// in a fixed tree (deterministic)
template <int NT>
__global__ void k_tv_restrict(TraceOp32 T, const float *__restrict__ r, const float *__restrict__ x,
                              const int *__restrict__ vert_facet, const int *__restrict__ vert_fsign, int nverts,
                              float *b1) {
    wait_prior_kernel();
    const float s3 = 0.28867513459481288225f;              // 1 / (2 sqrt 3)
    const long long t_ = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = (int)(t_ & 15), q = lane >> 1, row = lane & 1;
    int v = (int)(t_ >> 4);
    const bool vlive = v < nverts;
    if (!vlive) v = nverts - 1;
    const long long nrows = (long long)T.nfacets * NT;
    float c = 0.f;
    const int f = q < 6 ? __ldg(&vert_facet[6 * v + q]) : -1;
    if (f >= 0) {
        const float t = __ldcg(&r[(size_t)f * NT + row]) - row_S<NT>(T, nrows, f, row, x);
        c = row == 0 ? 0.5f * t : (float)__ldg(&vert_fsign[6 * v + q]) * s3 * t;
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o, 16);
    if (vlive && lane == 0) b1[v] = c;
}

// component j of x + P e_1 at facet cf (P e_1: the linear interpolant of the vertex values e_1,
// components 0 and 1 of each facet)
template <int NT>
__device__ __forceinline__ float x_plus_pe(const float *__restrict__ x, const float *__restrict__ e1,
                                           const int *__restrict__ facet_vert, int cf, int j) {
    float v = __ldcg(&x[(size_t)cf * NT + j]);
    if (e1 && j < 2) {
        const float a = __ldcg(&e1[__ldg(&facet_vert[2 * cf])]), b = __ldcg(&e1[__ldg(&facet_vert[2 * cf + 1])]);
        v += j == 0 ? 0.5f * (a + b) : 0.28867513459481288225f * (b - a);
    }
    return v;
}

// d = c1 d + c2 D^{-1} (r - S xin); xout = xin + d (FP32), or out64 = xin + d when out64 is set;
// xin = x + P e_1 when e1 is set
template <int NT>
__global__ void k_tv_cheb(TraceOp32 T, const float *__restrict__ r, const float *__restrict__ x,
                          const float *__restrict__ e1, const int *__restrict__ facet_vert, float *xout, float *d,
                          float c1, float c2, double *out64) {
    wait_prior_kernel();
    TV_ROW(NT)
    (void)G;
    float res = 0.f;
    if (i < NT) {
        float s = 0.f;
#pragma unroll
        for (int bb = 0; bb < 5; ++bb) {
            const int cf = __ldg(&T.tcol[bb * T.nfacets + f]);
            if (cf < 0) continue;                              // uniform over the group
#pragma unroll
            for (int j = 0; j < NT; ++j)
                s += __ldg(&T.Sell[(size_t)(bb * NT + j) * nrows + g]) * x_plus_pe<NT>(x, e1, facet_vert, cf, j);
        }
        res = __ldcg(&r[g]) - s;
    }
    const float dn = (c1 != 0.f ? c1 * __ldcg(&d[g]) : 0.f) + c2 * grp_dinv<NT>(T.Dinv, nrows, f, ic, res);
    if (live) {
        const float xo = x_plus_pe<NT>(x, e1, facet_vert, f, ic) + dn;
        d[g] = dn;
        if (out64) out64[g] = (double)xo;
        else xout[g] = xo;
    }
}

// ---------------------------------------------------------------- P1 levels in one block
// Shared-memory layout of P1 level l (l = 0: the tail's first level) at off[l]: b, xa, xb, d, dinv
// (nv floats each), then the stencil A (7 nv floats, by vertex). The constant parts (dinv, A) come
// from an image of the whole layout in global memory (img, built once per coefficient: zeros in
// the vector parts), copied in with 16-byte loads at the kernel's start. Threads take the points of
// a level as rows of nvx columns, so a thread's column and its neighbours' columns are fixed and
// rows step without a division.
struct Tail32 {
    int L, Nc, nfacets;
    P1Grid G[MG_MAX_LEVELS];
    const float *A[MG_MAX_LEVELS], *dinv[MG_MAX_LEVELS];
    float invth[MG_MAX_LEVELS], c1[MG_MAX_LEVELS], c2[MG_MAX_LEVELS];
    int off[MG_MAX_LEVELS];
    const float *Minv;             // coarsest grid: (A + 1 1^T / N)^{-1}, row-major
    const float *b1;               // right-hand side on level 0 (P^T of the trace residual)
    float *e1;                     // correction on level 0 (out)
    const float4 *img;             // the shared-memory image (tail32_floats, padded to 4 floats)
    int nimg4;                     // its length in float4
};

// shared floats the tail needs for the grids G[0..L-1]
inline size_t tail32_floats(const P1Grid *G, int L) {
    size_t n = 0;
    for (int l = 0; l < L; ++l) n += (size_t)12 * G[l].nverts;
    return (n + 3) / 4 * 4;
}

// index k + one step on a line of n points: wrapped when periodic, -1 outside otherwise
__device__ __forceinline__ int step1(int k, int n, int per) {
    return k < 0 ? (per ? k + n : -1) : (k >= n ? (per ? k - n : -1) : k);
}

// A level seen by the tail: vectors in shared memory, threads laid out as rows of nvx
struct TLevel {
    int nvx, nvy, px, py, nv;
    float *b, *xa, *xb, *d, *dv;
    const float *A;
    float invth, c1, c2;
};

__device__ __forceinline__ TLevel tail_level(const Tail32 &T, float *tsm, int l) {
    TLevel V;
    const P1Grid &G = T.G[l];
    V.nvx = G.nvx; V.nvy = G.nvy; V.px = G.px; V.py = G.py; V.nv = G.nverts;
    V.b = tsm + T.off[l]; V.xa = V.b + V.nv; V.xb = V.xa + V.nv; V.d = V.xb + V.nv; V.dv = V.d + V.nv;
    V.A = V.dv + V.nv;
    V.invth = T.invth[l]; V.c1 = T.c1[l]; V.c2 = T.c2[l];
    return V;
}

// the 7 stencil points of (i, j) in the order of P1_NS; absent neighbours (non-periodic edges)
// are replaced by the point itself, whose stencil entry for that offset is zero
struct Stencil {
    int p[P1_NS];
};

__device__ __forceinline__ Stencil stencil(const TLevel &V, int i, int j, int ip, int im) {
    const int jp = step1(j + 1, V.nvy, V.py), jm = step1(j - 1, V.nvy, V.py);
    const int c = j * V.nvx + i;
    Stencil S;
    S.p[0] = c;
    S.p[1] = ip >= 0 ? j * V.nvx + ip : c;
    S.p[2] = im >= 0 ? j * V.nvx + im : c;
    S.p[3] = jp >= 0 ? jp * V.nvx + i : c;
    S.p[4] = jm >= 0 ? jm * V.nvx + i : c;
    S.p[5] = ip >= 0 && jp >= 0 ? jp * V.nvx + ip : c;
    S.p[6] = im >= 0 && jm >= 0 ? jm * V.nvx + im : c;
    return S;
}

__device__ __forceinline__ float apply_st(const TLevel &V, const Stencil &S, const float *x) {
    const float *a = V.A + P1_NS * S.p[0];
    float s = 0.f;
#pragma unroll
    for (int o = 0; o < P1_NS; ++o) s += a[o] * x[S.p[o]];
    return s;
}

// loop over the level's points, threads as rows of nvx columns (nvx <= blockDim.x)
#define TL_FOR(V, ...)                                                                       \
    {                                                                                        \
        const int rows_ = (int)blockDim.x / (V).nvx;                                         \
        const int i = (int)threadIdx.x % (V).nvx, j0_ = (int)threadIdx.x / (V).nvx;          \
        const int ip = step1(i + 1, (V).nvx, (V).px), im = step1(i - 1, (V).nvx, (V).px);    \
        (void)ip; (void)im;                                                                  \
        if (j0_ < rows_)                                                                     \
            for (int j = j0_; j < (V).nvy; j += rows_) {                                     \
                const int v = j * (V).nvx + i;                                               \
                __VA_ARGS__                                                                  \
            }                                                                                \
    }

template <int NT>
__global__ void __launch_bounds__(1024) k_tv_tail(Tail32 T) {
    wait_prior_kernel();
    extern __shared__ float tsm[];
    const int tid = threadIdx.x, nth = blockDim.x;
    {                                                      // diagonals and stencils: the image
        float4 *dst = reinterpret_cast<float4 *>(tsm);
#pragma unroll 4
        for (int i = tid; i < T.nimg4; i += nth) dst[i] = __ldg(&T.img[i]);
    }
    __syncthreads();
    {
        float *b = tsm + T.off[0];
        for (int v = tid; v < T.G[0].nverts; v += nth) b[v] = __ldcg(&T.b1[v]);
    }
    __syncthreads();
    for (int l = 0; l < T.L - 1; ++l) {                    // down
        const TLevel V = tail_level(T, tsm, l);
        // two Chebyshev steps from 0: x0 = invth D^-1 b (formed at the stencil points), then
        // d = c1 x0 + c2 D^-1 (b - A x0), xb = x0 + d
        TL_FOR(V, {
            const Stencil S = stencil(V, i, j, ip, im);
            const float *a = V.A + P1_NS * v;
            float ax = 0.f;
_Pragma("unroll")
            for (int o = 0; o < P1_NS; ++o) {
                const int w = S.p[o];
                ax += a[o] * (V.invth * V.dv[w] * V.b[w]);
            }
            const float x0 = V.invth * V.dv[v] * V.b[v];
            const float dn = V.c1 * x0 + V.c2 * V.dv[v] * (V.b[v] - ax);
            V.d[v] = dn;
            V.xb[v] = x0 + dn;
        })
        __syncthreads();
        TL_FOR(V, {                                        // residual, kept in xa
            const Stencil S = stencil(V, i, j, ip, im);
            V.xa[v] = V.b[v] - apply_st(V, S, V.xb);
        })
        __syncthreads();
        const TLevel C = tail_level(T, tsm, l + 1);
        TL_FOR(C, {                                        // (I^T r)(V): fine points 2I + o
            const int fi = 2 * i, fj = 2 * j;
            const int fip = step1(fi + 1, V.nvx, V.px), fim = step1(fi - 1, V.nvx, V.px);
            const Stencil S = stencil(V, fi, fj, fip, fim);
            float s = V.xa[S.p[0]];
            const int fjp = step1(fj + 1, V.nvy, V.py), fjm = step1(fj - 1, V.nvy, V.py);
            const bool has[P1_NS] = {true, fip >= 0, fim >= 0, fjp >= 0, fjm >= 0, fip >= 0 && fjp >= 0,
                                     fim >= 0 && fjm >= 0};
_Pragma("unroll")
            for (int o = 1; o < P1_NS; ++o) s += has[o] ? 0.5f * V.xa[S.p[o]] : 0.f;
            C.b[v] = s;
        })
        __syncthreads();
    }
    {   // coarsest: x = Minv (b - mean b)
        const TLevel V = tail_level(T, tsm, T.L - 1);
        const int N = T.Nc;
        __shared__ float part[32];
        __shared__ float mean;
        float s = 0.f;
        for (int v = tid; v < N; v += nth) s += V.b[v];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((tid & 31) == 0) part[tid >> 5] = s;
        __syncthreads();
        if (tid == 0) {
            float m = 0.f;
            for (int w = 0; w < (nth + 31) / 32; ++w) m += part[w];
            mean = m / N;
        }
        __syncthreads();
        for (int v = tid; v < N; v += nth) {
            float acc = 0.f;
            for (int c = 0; c < N; ++c) acc += __ldg(&T.Minv[(size_t)v * N + c]) * (V.b[c] - mean);
            V.xb[v] = acc;
        }
        __syncthreads();
    }
    for (int l = T.L - 2; l >= 0; --l) {                   // up
        const TLevel V = tail_level(T, tsm, l), C = tail_level(T, tsm, l + 1);
        TL_FOR(V, {                                        // xb += I e (linear interpolation)
            const int i0 = i >> 1, j0 = j >> 1, oi = i & 1, oj = j & 1;
            float e = C.xb[j0 * C.nvx + i0];
            if (oi || oj) {
                const int in = oi ? step1(i0 + 1, C.nvx, C.px) : i0, jn = oj ? step1(j0 + 1, C.nvy, C.py) : j0;
                e = 0.5f * (e + C.xb[jn * C.nvx + in]);
            }
            V.xb[v] += e;
        })
        __syncthreads();
        TL_FOR(V, {
            const Stencil S = stencil(V, i, j, ip, im);
            const float dn = V.invth * V.dv[v] * (V.b[v] - apply_st(V, S, V.xb));
            V.d[v] = dn;
            V.xa[v] = V.xb[v] + dn;
        })
        __syncthreads();
        TL_FOR(V, {
            const Stencil S = stencil(V, i, j, ip, im);
            const float dn = V.c1 * V.d[v] + V.c2 * V.dv[v] * (V.b[v] - apply_st(V, S, V.xa));
            V.d[v] = dn;
            V.xb[v] = V.xa[v] + dn;
        })
        __syncthreads();
    }
    {
        const float *e = tail_level(T, tsm, 0).xb;
        for (int v = tid; v < T.G[0].nverts; v += nth) T.e1[v] = e[v];
    }
}

// ---------------------------------------------------------------- large P1 levels, grid-wide
// The P1 levels with more vertices than the one-block tail takes run as grid-wide FP32 kernels,
// a thread per vertex, with the same smoothing as the tail: down, two Chebyshev steps from 0 and
// the restriction of the residual; up, the prolongation and two Chebyshev steps.
// x = d = invth D^{-1} b
__global__ void k_p32_cheb0(const float *__restrict__ dinv, const float *__restrict__ b, float *x, float *d,
                            float invth, int n) {
    wait_prior_kernel();
    GRID_STRIDE(v, n) {
        const float s = invth * __ldg(&dinv[v]) * __ldcg(&b[v]);
        d[v] = s;
        x[v] = s;
    }
}

// d = c1 d + c2 D^{-1} (b - A xin); xout = xin + d
__global__ void k_p32_cheb(P1Grid G, const float *__restrict__ A, const float *__restrict__ dinv,
                           const float *__restrict__ b, const float *__restrict__ xin, float *__restrict__ xout,
                           float *d, float c1, float c2) {
    wait_prior_kernel();
    GRID_STRIDE(v, G.nverts) {
        const float r = __ldcg(&b[v]) - p1_apply<float>((int)v, G, A, xin);
        const float dn = (c1 != 0.f ? c1 * d[v] : 0.f) + c2 * __ldg(&dinv[v]) * r;
        d[v] = dn;
        xout[v] = xin[v] + dn;
    }
}

// t = b - A x
__global__ void k_p32_resid(P1Grid G, const float *__restrict__ A, const float *__restrict__ b,
                            const float *__restrict__ x, float *t) {
    wait_prior_kernel();
    GRID_STRIDE(v, G.nverts) t[v] = __ldcg(&b[v]) - p1_apply<float>((int)v, G, A, x);
}

// b_coarse = I^T t_fine
__global__ void k_p32_restrict(P1Grid Gc, P1Grid Gf, const float *__restrict__ tf, float *bc) {
    wait_prior_kernel();
    GRID_STRIDE(V, Gc.nverts) bc[V] = restrict_p1<float>((int)V, Gc, Gf, tf);
}

// x_fine += I e_coarse
__global__ void k_p32_prolong(P1Grid Gf, P1Grid Gc, const float *__restrict__ ec, float *x) {
    wait_prior_kernel();
    GRID_STRIDE(a, Gf.nverts) x[a] += prolong_p1<float>((int)a, Gf, Gc, ec);
}

// ---------------------------------------------------------------- flexible CG with the FP32 V-cycle
// x += alpha p; r -= alpha Ap (the preconditioner follows as separate kernels)
template <int NT>
__global__ void k_cg_update_xr(const double *__restrict__ p, const double *__restrict__ Ap, double *x, double *r,
                               int nfacets, const Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    const double alpha = sc->alpha;
    GRID_STRIDE(g, (long long)nfacets * NT) {
        x[g] += alpha * p[g];
        r[g] -= alpha * Ap[g];
    }
}

// Reduction of flexible CG (Polak-Ribiere beta; the FP32 V-cycle is not exactly the same linear
// map twice): z is taken off the constant mode, z - zmean e0; rz = (r, z - zmean e0);
// beta = (r, (z - zmean e0) - (zold - zmean_old e0)) / rz_old; zold = z. first: rz0. Convergence
// on sqrt(rz / rz0), as the CG with the FP64 V-cycle.
template <int NT>
__global__ void k_fcg_rz(const double *__restrict__ r, const double *__restrict__ z, double *zold, int nfacets,
                         int first, RedBuf rb, Scalars *sc) {
    wait_prior_kernel();
    if (sc->done) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0}, tot[4];
    GRID_STRIDE(g, (long long)nfacets * NT) {
        const double rg = r[g], zg = z[g];
        v[0] += rg * zg;
        if (g % NT == 0) { v[1] += zg; v[2] += rg; }
        if (!first) v[3] += rg * zold[g];
        zold[g] = zg;
    }
    if (grid_sum<4>(rb, v, tot)) {
        const double zm = tot[1] / nfacets, rz = tot[0] - zm * tot[2];
        if (first) {
            sc->rz = rz; sc->rz0 = rz; sc->relres = rz > 0 ? 1.0 : 0.0;
            if (!isfinite(rz)) { sc->done = 1; sc->breakdown = 2; }
            else if (!(rz > 0.0)) sc->done = 1;
        } else {
            const double rzo = tot[3] - sc->zmean_old * tot[2];
            sc->beta = (rz - rzo) / sc->rz;
            sc->rz = rz;
            sc->iters += 1;
            const double rel = sc->rz0 > 0 ? sqrt(fmax(rz, 0.0) / sc->rz0) : 0.0;
            sc->relres = rel;
            if (!isfinite(rz)) { sc->done = 1; sc->breakdown = 2; }
            else if (rel <= sc->rtol || sc->iters >= sc->maxit) sc->done = 1;
        }
        sc->zmean = zm;
        sc->zmean_old = zm;
    }
}

__global__ void k_f64_to_f32(const double *__restrict__ a, float *b, long long n) {
    wait_prior_kernel();
    GRID_STRIDE(i, n) b[i] = (float)a[i];
}

}  // namespace hdg
