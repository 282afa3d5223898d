// Reference-element tables of the GB300 HDG solver (host side).
//
// Reference triangle T = (0,0), (1,0), (0,1); local edge e runs from vertex (e+1)%3 to
// vertex (e+2)%3 (counter-clockwise), parameter s in [0,1]. Cell spaces use the orthonormal
// Dubiner basis (int_T phi_a phi_b = delta_ab), ordered by total degree so that the first
// dim P_k functions of the P_{k+1} basis span P_k (the pressure basis is a prefix of the
// velocity basis). Facet spaces use orthonormal Legendre polynomials on [0,1].
#pragma once
#include <vector>

namespace hdg {

struct RefTables {
    int k = 0;
    int mu = 0;     // dim P_{k+1}: scalar velocity basis
    int np = 0;     // dim P_k: pressure basis (prefix of the velocity basis)
    int nt = 0;     // k+1: trace basis on a facet
    int nq = 0;     // volume quadrature points
    int nfq = 0;    // facet quadrature points (Gauss-Legendre, (3k+5)/2)
    int nv = 0;     // interior BDM moments k(k+2)
    int nb = 0;     // k+2 edge BDM moments per edge
    int nnu = 0;    // lattice nodes of P_{k+1} (== mu)
    int nnp = 0;    // lattice nodes of P_k (== np)

    std::vector<double> qx, qy, qw;       // volume rule
    std::vector<double> phi;              // [q][a]           nq x mu
    std::vector<double> dphi;             // [q][a][r]        nq x mu x 2 (reference gradient)
    std::vector<double> fs, fw;           // facet rule on [0,1]
    std::vector<double> ephi;             // [e][q][a]        3 x nfq x mu (edge e, local s)
    std::vector<double> leg;              // [q][j]           nfq x nb     (orthonormal Legendre, j < k+2)
    std::vector<double> Dhat;             // [r][b][a]        2 x np x mu  = int psi_b d_r phi_a
    std::vector<double> Ehat;             // [e][j][a]        3 x nt x mu  = int_0^1 phi_a(x_e(s)) L_j(s) ds
    std::vector<double> Tpp;              // [e][b][c]        3 x np x np  = int_0^1 psi_b psi_c ds
    std::vector<double> Sfac;             // [e][a][b]        3 x mu x mu  = sum_q fw_q phi_a(e,q) phi_b(e,q)
    std::vector<double> Tadv;             // [r][c][a][b]     2 x mu^3     = sum_q w_q phi_a phi_c d_r phi_b
    std::vector<double> bdm_inv;          // [(d,a)][dof]     nu x nu      inverse BDM moment matrix
    std::vector<double> Iv;               // [a][v][d]        mu x nv x 2  = int_T phi_a v_d (Nedelec N_k)
    std::vector<double> nod_u, nod_p;     // nodal -> modal: [a][node]
    std::vector<double> mod_u, mod_p;     // modal -> nodal: [node][a]
    std::vector<double> nod_t, mod_t;     // trace nodal <-> modal: [j][node], [node][j]
    double en[3][2];                      // reference outward edge normals
    double eh[3];                         // reference edge lengths
};

int dim_P(int m);
// Orthonormal Dubiner basis of P_m at (x, y): values[dim_P(m)], optional grads[dim_P(m)][2].
void dubiner(int m, double x, double y, double *vals, double *grads);
// Orthonormal Legendre on [0,1]: L_j(s), j = 0..m.
void legendre01(int m, double s, double *vals);
// Gauss-Legendre rule on [0,1].
void gauss_legendre01(int n, double *x, double *w);
// Volume rule exact for total degree 2n-1 on the reference triangle (collapsed GL x GL with
// n and n+1 points); returns the number of points.
int triangle_rule(int n, std::vector<double> &x, std::vector<double> &y, std::vector<double> &w);
int volume_points_1d(int k);   // (3k+4)/2
int facet_points(int k);       // (3k+5)/2

RefTables build_tables(int k);

}  // namespace hdg
