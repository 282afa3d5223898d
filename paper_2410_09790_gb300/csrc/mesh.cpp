// Structured triangulation (host). See mesh.h.
#include "mesh.h"

#include <cmath>
#include <stdexcept>

namespace hdg {

int64_t mesh_facet_count(int n, bool px, bool py) {
    int64_t N = n;
    return N * (py ? N : N + 1) + N * (px ? N : N + 1) + N * N;
}

HostMesh build_mesh(int n, double Lx, double Ly, bool px, bool py) {
    if (n < 1) throw std::runtime_error("n must be >= 1");
    HostMesh M;
    M.n = n; M.Lx = Lx; M.Ly = Ly; M.px = px; M.py = py;
    M.ncells = 2 * n * n;
    M.nfacets = (int)mesh_facet_count(n, px, py);
    const double hx = Lx / n, hy = Ly / n;
    M.vxy.resize(M.ncells * 6);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double A[2] = {i * hx, j * hy}, B[2] = {(i + 1) * hx, j * hy};
            double C[2] = {(i + 1) * hx, (j + 1) * hy}, D[2] = {i * hx, (j + 1) * hy};
            double *c0 = &M.vxy[(2 * (j * n + i)) * 6], *c1 = &M.vxy[(2 * (j * n + i) + 1) * 6];
            const double *t0[3] = {A, B, C}, *t1[3] = {A, C, D};
            for (int v = 0; v < 3; ++v) {
                c0[2 * v] = t0[v][0]; c0[2 * v + 1] = t0[v][1];
                c1[2 * v] = t1[v][0]; c1[2 * v + 1] = t1[v][1];
            }
        }
    M.geo.resize(M.ncells);
    for (int c = 0; c < M.ncells; ++c) {
        const double *v = &M.vxy[c * 6];
        CellGeo &g = M.geo[c];
        g.J[0] = v[2] - v[0]; g.J[1] = v[4] - v[0];
        g.J[2] = v[3] - v[1]; g.J[3] = v[5] - v[1];
        g.detJ = g.J[0] * g.J[3] - g.J[1] * g.J[2];
        if (!(g.detJ > 0)) throw std::runtime_error("cell not counter-clockwise");
        g.Jinv[0] = g.J[3] / g.detJ; g.Jinv[1] = -g.J[1] / g.detJ;
        g.Jinv[2] = -g.J[2] / g.detJ; g.Jinv[3] = g.J[0] / g.detJ;
        for (int e = 0; e < 3; ++e) {
            int a = (e + 1) % 3, b = (e + 2) % 3;
            double dx = v[2 * b] - v[2 * a], dy = v[2 * b + 1] - v[2 * a + 1];
            g.h[e] = std::sqrt(dx * dx + dy * dy);
            g.nx[e] = dy / g.h[e];
            g.ny[e] = -dx / g.h[e];
        }
        g.pad = 0;
    }
    M.cell_facet.assign(M.ncells * 3, -1);
    M.cell_flip.assign(M.ncells * 3, 0);
    M.cell_nbr.assign(M.ncells * 3, -1);
    M.cell_nbr_edge.assign(M.ncells * 3, -1);
    M.facet_cell.assign(M.nfacets * 2, -1);
    M.facet_edge.assign(M.nfacets * 2, -1);
    auto cell = [n](int i, int j, int t) { return 2 * (j * n + i) + t; };
    int f = 0;
    auto add_side = [&](int fac, int side, int c, int e, int flip) {
        M.facet_cell[fac * 2 + side] = c;
        M.facet_edge[fac * 2 + side] = e;
        M.cell_facet[c * 3 + e] = fac;
        M.cell_flip[c * 3 + e] = flip;
    };
    // horizontal H(i,j): above = (i,j) lower-right cell, local edge 2 (A->B, same direction);
    // below = (i,j-1) upper-left cell, local edge 0 (C->D, opposite)
    const int jmax = py ? n : n + 1;
    for (int j = 0; j < jmax; ++j)
        for (int i = 0; i < n; ++i, ++f) {
            int s = 0;
            if (j < n) add_side(f, s++, cell(i, j, 0), 2, 0);
            if (j > 0) add_side(f, s++, cell(i, j - 1, 1), 0, 1);
            else if (py) add_side(f, s++, cell(i, n - 1, 1), 0, 1);
        }
    // vertical V(i,j): right = (i,j) upper-left cell, local edge 1 (D->A, opposite);
    // left = (i-1,j) lower-right cell, local edge 0 (B->C, same)
    const int imax = px ? n : n + 1;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < imax; ++i, ++f) {
            int s = 0;
            if (i < n) add_side(f, s++, cell(i, j, 1), 1, 1);
            if (i > 0) add_side(f, s++, cell(i - 1, j, 0), 0, 0);
            else if (px) add_side(f, s++, cell(n - 1, j, 0), 0, 0);
        }
    // diagonal D(i,j): lower-right cell local edge 1 (C->A, opposite), upper-left local edge 2 (A->C, same)
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i, ++f) {
            add_side(f, 0, cell(i, j, 0), 1, 1);
            add_side(f, 1, cell(i, j, 1), 2, 0);
        }
    if (f != M.nfacets) throw std::runtime_error("facet count mismatch");
    for (int fac = 0; fac < M.nfacets; ++fac) {
        int c0 = M.facet_cell[fac * 2], c1 = M.facet_cell[fac * 2 + 1];
        int e0 = M.facet_edge[fac * 2], e1 = M.facet_edge[fac * 2 + 1];
        if (c1 >= 0) {
            M.cell_nbr[c0 * 3 + e0] = c1; M.cell_nbr_edge[c0 * 3 + e0] = e1;
            M.cell_nbr[c1 * 3 + e1] = c0; M.cell_nbr_edge[c1 * 3 + e1] = e0;
        }
    }
    for (int i = 0; i < M.ncells * 3; ++i)
        if (M.cell_facet[i] < 0) throw std::runtime_error("unassigned cell edge");
    // P1 vertices
    M.nvx = px ? n : n + 1;
    M.nvy = py ? n : n + 1;
    M.nverts = M.nvx * M.nvy;
    auto vid = [&](int i, int j) {
        if (px) i %= n;
        if (py) j %= n;
        return j * M.nvx + i;
    };
    M.cell_vert.assign(M.ncells * 3, -1);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            int c0 = cell(i, j, 0), c1 = cell(i, j, 1);
            M.cell_vert[3 * c0] = vid(i, j); M.cell_vert[3 * c0 + 1] = vid(i + 1, j); M.cell_vert[3 * c0 + 2] = vid(i + 1, j + 1);
            M.cell_vert[3 * c1] = vid(i, j); M.cell_vert[3 * c1 + 1] = vid(i + 1, j + 1); M.cell_vert[3 * c1 + 2] = vid(i, j + 1);
        }
    M.facet_vert.assign(M.nfacets * 2, -1);
    for (int fac = 0; fac < M.nfacets; ++fac) {
        int c = M.facet_cell[2 * fac], e = M.facet_edge[2 * fac];
        int a = M.cell_vert[3 * c + (e + 1) % 3], b = M.cell_vert[3 * c + (e + 2) % 3];
        if (M.cell_flip[3 * c + e]) std::swap(a, b);
        M.facet_vert[2 * fac] = a;
        M.facet_vert[2 * fac + 1] = b;
    }
    M.vert_facet.assign(M.nverts * 6, -1);
    M.vert_fsign.assign(M.nverts * 6, 0);
    M.vert_cell.assign(M.nverts * 6, -1);
    std::vector<int> nf(M.nverts, 0), ncl(M.nverts, 0);
    M.p1_ok = n >= 3;
    for (int fac = 0; fac < M.nfacets && M.p1_ok; ++fac)
        for (int s = 0; s < 2; ++s) {
            int v = M.facet_vert[2 * fac + s];
            if (nf[v] >= 6) { M.p1_ok = false; break; }
            M.vert_facet[6 * v + nf[v]] = fac;
            M.vert_fsign[6 * v + nf[v]] = s == 0 ? -1 : 1;
            ++nf[v];
        }
    for (int c = 0; c < M.ncells && M.p1_ok; ++c)
        for (int a = 0; a < 3; ++a) {
            int v = M.cell_vert[3 * c + a];
            if (ncl[v] >= 6) { M.p1_ok = false; break; }
            M.vert_cell[6 * v + ncl[v]++] = 3 * c + a;
        }
    return M;
}

CGNumbering build_cg_numbering(const HostMesh &M, int m) {
    if (m < 1) throw std::runtime_error("CG degree must be >= 1");
    CGNumbering C;
    const int n = M.n, nm = n * m;
    const int NX = M.px ? nm : nm + 1, NY = M.py ? nm : nm + 1;
    C.m = m;
    C.nl = (m + 1) * (m + 2) / 2;
    C.npts = NX * NY;
    C.cell_gid.resize((size_t)M.ncells * C.nl);
    for (int cj = 0; cj < n; ++cj)
        for (int ci = 0; ci < n; ++ci)
            for (int t = 0; t < 2; ++t) {
                const int c = 2 * (cj * n + ci) + t;
                int l = 0;
                for (int j = 0; j <= m; ++j)
                    for (int i = 0; i + j <= m; ++i, ++l) {
                        // lower cell (A, B, C): A + h ((i + j)/m, j/m); upper (A, C, D): A + h (i/m, (i + j)/m)
                        int I = m * ci + (t == 0 ? i + j : i), J = m * cj + (t == 0 ? j : i + j);
                        if (M.px) I %= NX;
                        if (M.py) J %= NY;
                        C.cell_gid[(size_t)c * C.nl + l] = J * NX + I;
                    }
            }
    std::vector<int> count(C.npts + 1, 0);
    for (int g : C.cell_gid) ++count[g + 1];
    for (int p = 0; p < C.npts; ++p) count[p + 1] += count[p];
    C.node_ptr = count;
    C.node_list.resize(C.cell_gid.size());
    std::vector<int> fill(count.begin(), count.end() - 1);
    for (size_t e = 0; e < C.cell_gid.size(); ++e) C.node_list[fill[C.cell_gid[e]]++] = (int)e;
    return C;
}

}  // namespace hdg
