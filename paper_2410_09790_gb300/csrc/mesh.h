// Structured triangulation of [0,Lx]x[0,Ly] (Sec. 3.2 "Setup") with the canonical numbering of
// the exchange format (hdg.h): n x n rectangles, rectangle (i,j) split along its (i,j)-(i+1,j+1)
// diagonal into cells 2(jn+i) = (A,B,C) and 2(jn+i)+1 = (A,C,D), both counter-clockwise.
// Local edge e of a cell runs from its vertex (e+1)%3 to (e+2)%3. Facets: H(i,j), V(i,j), D(i,j).
#pragma once
#include <cstdint>
#include <vector>

namespace hdg {

struct CellGeo {          // per-cell affine geometry, x = v0 + J xi (J column-major: J[0]=dx/dxi...)
    double J[4];          // J = [[J0, J1], [J2, J3]] row-major: x = v0 + (J0 xi + J1 eta, J2 xi + J3 eta)
    double Jinv[4];       // inverse, row-major
    double detJ;
    double h[3];          // edge lengths
    double nx[3], ny[3];  // outward unit normals
    double pad;
};

struct HostMesh {
    int n = 0;
    double Lx = 1, Ly = 1;
    bool px = false, py = false;
    int ncells = 0, nfacets = 0;
    std::vector<double> vxy;            // [c][3][2] vertex coordinates (own copy, unwrapped)
    std::vector<CellGeo> geo;           // [c]
    std::vector<int> cell_facet;        // [c][3]
    std::vector<int> cell_flip;         // [c][3]: 1 if the local edge runs against the facet's canonical direction
    std::vector<int> cell_nbr;          // [c][3]: neighbour across the edge or -1 (wall)
    std::vector<int> cell_nbr_edge;     // [c][3]: the neighbour's local edge index
    std::vector<int> facet_cell;        // [f][2]: side cells (second -1 on walls)
    std::vector<int> facet_edge;        // [f][2]: local edge index in each side cell
    // vertices of the P1 coarse space: (i,j), i < nvx, j < nvy (periodic directions wrap)
    int nvx = 0, nvy = 0, nverts = 0;
    std::vector<int> cell_vert;         // [c][3]
    std::vector<int> facet_vert;        // [f][2]: canonical start / end vertex
    std::vector<int> vert_facet;        // [v][6]: incident facets (-1 padded)
    std::vector<int> vert_fsign;        // [v][6]: -1 if v starts the facet, +1 if it ends it
    std::vector<int> vert_cell;         // [v][6]: incident cell*3 + local vertex (-1 padded)
    bool p1_ok = false;                 // vertex maps valid (n >= 3: distinct stencil neighbours)
};

int64_t mesh_facet_count(int n, bool px, bool py);
HostMesh build_mesh(int n, double Lx, double Ly, bool px, bool py);

// The continuous space CG_m on the mesh (App. B: the tracer's advecting velocity). The points of
// the cells' equispaced degree-m lattices lie on the grid of spacing (Lx, Ly) / (n m); a point is
// numbered J * NX + I (periodic directions wrapped, NX = n m or n m + 1). cell_gid[c][l]: the
// point of lattice node l of cell c (nodes j outer, i inner, i + j <= m); node_ptr / node_list:
// for every point the entries c * nl + l that share it (CSR, ascending).
struct CGNumbering {
    int m = 0, nl = 0, npts = 0;
    std::vector<int> cell_gid, node_ptr, node_list;
};
CGNumbering build_cg_numbering(const HostMesh &M, int m);

}  // namespace hdg
