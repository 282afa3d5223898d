// Non-nested multigrid preconditioner for the trace system (Sec. 2.8, after Cockburn et al.
// 2014): fine level = the trace space with a degree-2 Chebyshev smoother on the facet
// block-Jacobi preconditioner; next level = continuous P1 on the mesh vertices, reached by the
// injection P of a P1 function into the trace space (its facet traces are linear, so exact for
// k >= 1), with the Galerkin operator A1 = P^T S P; then a geometric hierarchy of P1 spaces on
// the nested structured meshes (n -> n/2, Galerkin coarsening with linear interpolation),
// degree-2 Chebyshev / Jacobi smoothing, and a dense pseudo-inverse on the coarsest grid. All
// P1 operators are 7-point stencils on the vertex grid (the triangulation's diagonals run from
// (i,j) to (i+1,j+1)); the constant is their one-dimensional kernel.
#pragma once
#include "hdg_cell.cuh"

namespace hdg {

constexpr int P1_NS = 7;    // stencil offsets: (0,0) (1,0) (-1,0) (0,1) (0,-1) (1,1) (-1,-1)

__host__ __device__ __forceinline__ int p1_di(int o) { return o == 1 || o == 5 ? 1 : (o == 2 || o == 6 ? -1 : 0); }
__host__ __device__ __forceinline__ int p1_dj(int o) { return o == 3 || o == 5 ? 1 : (o == 4 || o == 6 ? -1 : 0); }
__host__ __device__ __forceinline__ int p1_off(int di, int dj) {
    for (int o = 0; o < P1_NS; ++o)
        if (p1_di(o) == di && p1_dj(o) == dj) return o;
    return -1;
}

struct P1Grid {
    int n, px, py, nvx, nvy, nverts;
};

inline P1Grid make_p1grid(int n, int px, int py) {
    P1Grid G;
    G.n = n; G.px = px; G.py = py;
    G.nvx = px ? n : n + 1;
    G.nvy = py ? n : n + 1;
    G.nverts = G.nvx * G.nvy;
    return G;
}

// vertex id of grid point (i, j) (unwrapped coordinates), -1 outside a non-periodic grid
__host__ __device__ __forceinline__ int p1_vid(const P1Grid &G, int i, int j) {
    if (G.px) { i %= G.n; if (i < 0) i += G.n; } else if (i < 0 || i > G.n) return -1;
    if (G.py) { j %= G.n; if (j < 0) j += G.n; } else if (j < 0 || j > G.n) return -1;
    return j * G.nvx + i;
}

// A_K = P_K^T S_K P_K for one cell (3 x 3, local vertex order). S: NL x NL, canonical orientation.
template <int NT>
__host__ __device__ void p1_cellop(const double *S, const int *flip, double *A3) {
    const int NL = 3 * NT;
    const double s3 = 0.28867513459481288225;           // 1 / (2 sqrt 3)
    double P[3 * NT][3];
    for (int r = 0; r < NL; ++r)
        for (int a = 0; a < 3; ++a) P[r][a] = 0.0;
    for (int e = 0; e < 3; ++e) {
        int a = (e + 1) % 3, b = (e + 2) % 3;
        int st = flip[e] ? b : a, en = flip[e] ? a : b;
        P[e * NT][st] += 0.5;
        P[e * NT][en] += 0.5;
        P[e * NT + 1][en] += s3;
        P[e * NT + 1][st] -= s3;
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (int r = 0; r < NL; ++r) {
                if (P[r][a] == 0.0) continue;
                double t = 0;
                for (int q = 0; q < NL; ++q) t += S[r * NL + q] * P[q][b];
                s += P[r][a] * t;
            }
            A3[a * 3 + b] = s;
        }
}

// stencil row of the level-1 operator at vertex v, gathered from its (up to 6) cells
__host__ __device__ inline void p1_assemble_row(int v, const P1Grid &G, const double *cellA, const int *vert_cell,
                                                const int *cell_vert, double *row) {
    int i = v % G.nvx, j = v / G.nvx;
    int nb[P1_NS];
    for (int o = 0; o < P1_NS; ++o) { nb[o] = p1_vid(G, i + p1_di(o), j + p1_dj(o)); row[o] = 0.0; }
    for (int s = 0; s < 6; ++s) {
        int ca = vert_cell[6 * v + s];
        if (ca < 0) continue;
        int c = ca / 3, a = ca % 3;
        for (int b = 0; b < 3; ++b) {
            int w = cell_vert[3 * c + b];
            for (int o = 0; o < P1_NS; ++o)
                if (nb[o] == w) { row[o] += cellA[9 * c + 3 * a + b]; break; }
        }
    }
}

// Galerkin row of the coarse operator at coarse vertex V: sum_{a,b} phi_V(a) A_f(a,b) phi_W(b)
__host__ __device__ inline void p1_galerkin_row(int V, const P1Grid &Gc, const P1Grid &Gf, const double *Af,
                                                double *row) {
    const int I = V % Gc.nvx, J = V / Gc.nvx;
    for (int o = 0; o < P1_NS; ++o) row[o] = 0.0;
    for (int sa = 0; sa < P1_NS; ++sa) {                 // support of phi_V on the fine grid
        int fi = 2 * I + p1_di(sa), fj = 2 * J + p1_dj(sa);
        double wa = sa == 0 ? 1.0 : 0.5;
        int a = p1_vid(Gf, fi, fj);
        if (a < 0) continue;
        for (int o = 0; o < P1_NS; ++o) {
            double Aab = Af[P1_NS * a + o];
            if (Aab == 0.0) continue;
            int bi = fi + p1_di(o), bj = fj + p1_dj(o);
            // coarse parents of fine vertex b (unwrapped coordinates)
            int wi[2], wj[2], nw = 0;
            double wb;
            bool oi = (bi & 1) != 0, oj = (bj & 1) != 0;
            if (!oi && !oj) { wi[0] = bi / 2; wj[0] = bj / 2; nw = 1; wb = 1.0; }
            else {
                wb = 0.5; nw = 2;
                int bi0 = oi ? (bi - 1) : bi, bj0 = oj ? (bj - 1) : bj;   // even lower corner
                wi[0] = bi0 / 2; wj[0] = bj0 / 2;                        // exact: bi0, bj0 even
                wi[1] = wi[0] + (oi ? 1 : 0); wj[1] = wj[0] + (oj ? 1 : 0);
            }
            for (int q = 0; q < nw; ++q) {
                int off = p1_off(wi[q] - I, wj[q] - J);
                if (off >= 0) row[off] += wa * Aab * wb;
            }
        }
    }
}

// y(v) = sum_o A(v, o) x(nb)   (T = double, or float for the FP32 V-cycle)
template <class T>
__host__ __device__ __forceinline__ T p1_apply(int v, const P1Grid &G, const T *A, const T *x) {
    int i = v % G.nvx, j = v / G.nvx;
    T s = 0;
    for (int o = 0; o < P1_NS; ++o) {
        int w = p1_vid(G, i + p1_di(o), j + p1_dj(o));
        if (w >= 0) s += A[P1_NS * v + o] * x[w];
    }
    return s;
}

// (P^T r)(v) for a trace vector r: a facet contributes 0.5 r_0 +- r_1 / (2 sqrt 3)
template <int NT>
__host__ __device__ __forceinline__ double restrict_trace(int v, const double *r, const int *vert_facet,
                                                          const int *vert_fsign) {
    const double s3 = 0.28867513459481288225;
    double s = 0;
    for (int q = 0; q < 6; ++q) {
        int f = vert_facet[6 * v + q];
        if (f < 0) continue;
        s += 0.5 * r[(size_t)f * NT] + vert_fsign[6 * v + q] * s3 * r[(size_t)f * NT + 1];
    }
    return s;
}

// (I^T r)(V): restriction between P1 levels
template <class T>
__host__ __device__ __forceinline__ T restrict_p1(int V, const P1Grid &Gc, const P1Grid &Gf, const T *rf) {
    const int I = V % Gc.nvx, J = V / Gc.nvx;
    T s = 0;
    for (int sa = 0; sa < P1_NS; ++sa) {
        int a = p1_vid(Gf, 2 * I + p1_di(sa), 2 * J + p1_dj(sa));
        if (a >= 0) s += (sa == 0 ? T(1) : T(0.5)) * rf[a];
    }
    return s;
}

// (I e)(a): linear interpolation from the coarse P1 grid to fine vertex a
template <class T>
__host__ __device__ __forceinline__ T prolong_p1(int a, const P1Grid &Gf, const P1Grid &Gc, const T *ec) {
    int i = a % Gf.nvx, j = a / Gf.nvx;
    int i0 = i >> 1, j0 = j >> 1;
    bool oi = i & 1, oj = j & 1;
    T v0 = ec[p1_vid(Gc, i0, j0)];
    if (!oi && !oj) return v0;
    return T(0.5) * (v0 + ec[p1_vid(Gc, i0 + (oi ? 1 : 0), j0 + (oj ? 1 : 0))]);
}

}  // namespace hdg
