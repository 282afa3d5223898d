// Reference-element tables (host). See refelem.h.
#include "refelem.h"

#include <cmath>
#include <stdexcept>

namespace hdg {

namespace {
typedef long double ld;

struct Dual {            // value and gradient in (x, y)
    ld v, dx, dy;
};
inline Dual dmul(const Dual &a, const Dual &b) {
    return {a.v * b.v, a.dx * b.v + a.v * b.dx, a.dy * b.v + a.v * b.dy};
}
inline Dual dlin(ld ca, const Dual &a, ld cb, const Dual &b) {
    return {ca * a.v + cb * b.v, ca * a.dx + cb * b.dx, ca * a.dy + cb * b.dy};
}

// In-place inverse of an n x n matrix (row-major) with partial pivoting.
void invert(int n, std::vector<ld> &A) {
    std::vector<ld> I(n * n, 0.0L);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0L;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabsl(A[r * n + c]) > fabsl(A[piv * n + c])) piv = r;
        if (fabsl(A[piv * n + c]) < 1e-30L) throw std::runtime_error("singular reference matrix");
        if (piv != c)
            for (int j = 0; j < n; ++j) {
                std::swap(A[c * n + j], A[piv * n + j]);
                std::swap(I[c * n + j], I[piv * n + j]);
            }
        ld d = A[c * n + c];
        for (int j = 0; j < n; ++j) { A[c * n + j] /= d; I[c * n + j] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            ld f = A[r * n + c];
            if (f == 0.0L) continue;
            for (int j = 0; j < n; ++j) { A[r * n + j] -= f * A[c * n + j]; I[r * n + j] -= f * I[c * n + j]; }
        }
    }
    A = I;
}

void gl_ld(int n, std::vector<ld> &x, std::vector<ld> &w) {   // Gauss-Legendre on [-1,1]
    x.assign(n, 0); w.assign(n, 0);
    const ld pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        ld z = cosl(pi * (i + 0.75L) / (n + 0.5L));
        ld dp = 0;
        for (int it = 0; it < 100; ++it) {
            ld p0 = 1, p1 = z;
            for (int m = 2; m <= n; ++m) { ld p2 = ((2 * m - 1) * z * p1 - (m - 1) * p0) / m; p0 = p1; p1 = p2; }
            if (n == 1) { p1 = z; p0 = 1; }
            dp = n * (z * p1 - p0) / (z * z - 1);
            ld dz = p1 / dp;
            z -= dz;
            if (fabsl(dz) < 1e-21L) break;
        }
        ld p0 = 1, p1 = z;
        for (int m = 2; m <= n; ++m) { ld p2 = ((2 * m - 1) * z * p1 - (m - 1) * p0) / m; p0 = p1; p1 = p2; }
        dp = n * (z * p1 - p0) / (z * z - 1);
        x[i] = z;
        w[i] = 2 / ((1 - z * z) * dp * dp);
    }
}

void dubiner_ld(int m, ld x, ld y, std::vector<Dual> &out) {
    // phi_{ij} = sqrt(2(2i+1)(i+j+1)) Q_i(X, Y) P_j^{(2i+1,0)}(2y-1), with X = 2x+y-1,
    // Y = 1-y and Q_i = Y^i P_i(X/Y) from the scaled Legendre recursion (no collapse singularity).
    Dual X = {2 * x + y - 1, 2, 1}, Y = {1 - y, 0, -1}, Bv = {2 * y - 1, 0, 2};
    Dual one = {1, 0, 0};
    std::vector<Dual> Qi(m + 1);
    Qi[0] = one;
    if (m >= 1) Qi[1] = X;
    Dual Y2 = dmul(Y, Y);
    for (int i = 1; i < m; ++i)
        Qi[i + 1] = dlin(ld(2 * i + 1) / (i + 1), dmul(X, Qi[i]), -ld(i) / (i + 1), dmul(Y2, Qi[i - 1]));
    std::vector<std::vector<Dual>> P(m + 1);
    for (int i = 0; i <= m; ++i) {
        int jm = m - i;
        ld al = 2 * i + 1;
        P[i].resize(jm + 1);
        P[i][0] = one;
        if (jm >= 1) P[i][1] = dlin((al + 2) / 2, Bv, al / 2, one);
        for (int n = 2; n <= jm; ++n) {
            ld a1 = 2 * n * (n + al) * (2 * n + al - 2);
            ld a2 = (2 * n + al - 1) * al * al;
            ld a3 = (2 * n + al - 1) * (2 * n + al) * (2 * n + al - 2);
            ld a4 = 2 * (n + al - 1) * (n - 1) * (2 * n + al);
            Dual t = dlin(a3, dmul(Bv, P[i][n - 1]), a2, P[i][n - 1]);
            P[i][n] = dlin(1 / a1, t, -a4 / a1, P[i][n - 2]);
        }
    }
    out.clear();
    for (int d = 0; d <= m; ++d)
        for (int i = d; i >= 0; --i) {
            int j = d - i;
            ld nrm = sqrtl(2.0L * (2 * i + 1) * (i + j + 1));
            Dual v = dmul(Qi[i], P[i][j]);
            out.push_back({nrm * v.v, nrm * v.dx, nrm * v.dy});
        }
}

void legendre01_ld(int m, ld s, std::vector<ld> &out) {
    out.assign(m + 1, 0);
    ld z = 2 * s - 1, p0 = 1, p1 = z;
    out[0] = 1;
    if (m >= 1) out[1] = sqrtl(3.0L) * z;
    for (int n = 2; n <= m; ++n) {
        ld p2 = ((2 * n - 1) * z * p1 - (n - 1) * p0) / n;
        p0 = p1; p1 = p2;
        out[n] = sqrtl(ld(2 * n + 1)) * p2;
    }
}
}  // namespace

int dim_P(int m) { return (m + 1) * (m + 2) / 2; }
int volume_points_1d(int k) { return (3 * k + 4) / 2; }
int facet_points(int k) { return (3 * k + 5) / 2; }

void dubiner(int m, double x, double y, double *vals, double *grads) {
    std::vector<Dual> v;
    dubiner_ld(m, x, y, v);
    for (size_t a = 0; a < v.size(); ++a) {
        vals[a] = (double)v[a].v;
        if (grads) { grads[2 * a] = (double)v[a].dx; grads[2 * a + 1] = (double)v[a].dy; }
    }
}

void legendre01(int m, double s, double *vals) {
    std::vector<ld> v;
    legendre01_ld(m, s, v);
    for (int j = 0; j <= m; ++j) vals[j] = (double)v[j];
}

void gauss_legendre01(int n, double *x, double *w) {
    std::vector<ld> xs, ws;
    gl_ld(n, xs, ws);
    for (int i = 0; i < n; ++i) { x[i] = (double)((xs[i] + 1) / 2); w[i] = (double)(ws[i] / 2); }
}

int triangle_rule(int n, std::vector<double> &x, std::vector<double> &y, std::vector<double> &w) {
    std::vector<ld> u, wu, v, wv;
    gl_ld(n, u, wu);
    gl_ld(n + 1, v, wv);
    x.clear(); y.clear(); w.clear();
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= n; ++j) {
            x.push_back((double)((1 + u[i]) * (1 - v[j]) / 4));
            y.push_back((double)((1 + v[j]) / 2));
            w.push_back((double)(wu[i] * wv[j] * (1 - v[j]) / 8));
        }
    return (int)w.size();
}

RefTables build_tables(int k) {
    if (k < 1 || k > 4) throw std::runtime_error("degree k must be 1..4");
    RefTables T;
    T.k = k;
    T.mu = dim_P(k + 1);
    T.np = dim_P(k);
    T.nt = k + 1;
    T.nb = k + 2;
    T.nv = k * (k + 2);
    T.nnu = T.mu;
    T.nnp = T.np;
    const int mu = T.mu, np = T.np, nt = T.nt, nb = T.nb, nu = 2 * mu;
    // reference edges
    const double vx[3] = {0, 1, 0}, vy[3] = {0, 0, 1};
    for (int e = 0; e < 3; ++e) {
        int a = (e + 1) % 3, b = (e + 2) % 3;
        double dx = vx[b] - vx[a], dy = vy[b] - vy[a];
        T.eh[e] = std::sqrt(dx * dx + dy * dy);
        T.en[e][0] = dy / T.eh[e];
        T.en[e][1] = -dx / T.eh[e];
    }
    // volume rule and basis
    T.nq = triangle_rule(volume_points_1d(k), T.qx, T.qy, T.qw);
    T.phi.resize(T.nq * mu);
    T.dphi.resize(T.nq * mu * 2);
    std::vector<long double> phiL(T.nq * mu), dphiL(T.nq * mu * 2);
    std::vector<Dual> tmp;
    for (int q = 0; q < T.nq; ++q) {
        dubiner_ld(k + 1, T.qx[q], T.qy[q], tmp);
        for (int a = 0; a < mu; ++a) {
            phiL[q * mu + a] = tmp[a].v;
            dphiL[(q * mu + a) * 2] = tmp[a].dx;
            dphiL[(q * mu + a) * 2 + 1] = tmp[a].dy;
            T.phi[q * mu + a] = (double)tmp[a].v;
            T.dphi[(q * mu + a) * 2] = (double)tmp[a].dx;
            T.dphi[(q * mu + a) * 2 + 1] = (double)tmp[a].dy;
        }
    }
    // facet rule, edge values, Legendre
    T.nfq = facet_points(k);
    T.fs.resize(T.nfq); T.fw.resize(T.nfq);
    std::vector<ld> fsL, fwL;
    gl_ld(T.nfq, fsL, fwL);
    for (int q = 0; q < T.nfq; ++q) { fsL[q] = (fsL[q] + 1) / 2; fwL[q] /= 2; T.fs[q] = (double)fsL[q]; T.fw[q] = (double)fwL[q]; }
    T.ephi.resize(3 * T.nfq * mu);
    std::vector<ld> ephiL(3 * T.nfq * mu);
    T.leg.resize(T.nfq * nb);
    std::vector<ld> legL(T.nfq * nb), lv;
    for (int q = 0; q < T.nfq; ++q) {
        legendre01_ld(nb - 1, fsL[q], lv);
        for (int j = 0; j < nb; ++j) { legL[q * nb + j] = lv[j]; T.leg[q * nb + j] = (double)lv[j]; }
    }
    for (int e = 0; e < 3; ++e) {
        int a0 = (e + 1) % 3, b0 = (e + 2) % 3;
        for (int q = 0; q < T.nfq; ++q) {
            ld s = fsL[q];
            ld x = vx[a0] + s * (vx[b0] - vx[a0]), y = vy[a0] + s * (vy[b0] - vy[a0]);
            dubiner_ld(k + 1, x, y, tmp);
            for (int a = 0; a < mu; ++a) {
                ephiL[(e * T.nfq + q) * mu + a] = tmp[a].v;
                T.ephi[(e * T.nfq + q) * mu + a] = (double)tmp[a].v;
            }
        }
    }
    // Dhat, Ehat, Tpp
    T.Dhat.assign(2 * np * mu, 0.0);
    for (int r = 0; r < 2; ++r)
        for (int b = 0; b < np; ++b)
            for (int a = 0; a < mu; ++a) {
                ld s = 0;
                for (int q = 0; q < T.nq; ++q) s += (ld)T.qw[q] * phiL[q * mu + b] * dphiL[(q * mu + a) * 2 + r];
                T.Dhat[(r * np + b) * mu + a] = (double)s;
            }
    T.Ehat.assign(3 * nt * mu, 0.0);
    T.Tpp.assign(3 * np * np, 0.0);
    for (int e = 0; e < 3; ++e) {
        for (int j = 0; j < nt; ++j)
            for (int a = 0; a < mu; ++a) {
                ld s = 0;
                for (int q = 0; q < T.nfq; ++q) s += fwL[q] * ephiL[(e * T.nfq + q) * mu + a] * legL[q * nb + j];
                T.Ehat[(e * nt + j) * mu + a] = (double)s;
            }
        for (int b = 0; b < np; ++b)
            for (int c = 0; c < np; ++c) {
                ld s = 0;
                for (int q = 0; q < T.nfq; ++q)
                    s += fwL[q] * ephiL[(e * T.nfq + q) * mu + b] * ephiL[(e * T.nfq + q) * mu + c];
                T.Tpp[(e * np + b) * np + c] = (double)s;
            }
    }
    // facet mass of each reference edge (the penalty term's matrices) and the volume advection
    // tensor: the advection block of a cell is sum_{r,c} g_rc Tadv[r][c] with g_rc the
    // coefficients of (J^-1 Q*)_r, the same quadrature sum regrouped (exact in exact arithmetic)
    T.Sfac.assign(3 * mu * mu, 0.0);
    for (int e = 0; e < 3; ++e)
        for (int a = 0; a < mu; ++a)
            for (int b = 0; b < mu; ++b) {
                ld s = 0;
                for (int q = 0; q < T.nfq; ++q)
                    s += fwL[q] * ephiL[(e * T.nfq + q) * mu + a] * ephiL[(e * T.nfq + q) * mu + b];
                T.Sfac[(e * mu + a) * mu + b] = (double)s;
            }
    T.Tadv.assign(2 * mu * mu * mu, 0.0);
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < mu; ++c)
            for (int a = 0; a < mu; ++a)
                for (int b = 0; b < mu; ++b) {
                    ld s = 0;
                    for (int q = 0; q < T.nq; ++q)
                        s += (ld)T.qw[q] * phiL[q * mu + a] * phiL[q * mu + c] * dphiL[(q * mu + b) * 2 + r];
                    T.Tadv[((r * mu + c) * mu + a) * mu + b] = (double)s;
                }
    // interior BDM moments against the first-kind Nedelec space N_k on T:
    // [P_{k-1}]^2 (monomials x^i y^j) and (-y, x) * homogeneous degree k-1
    const int nv = T.nv;
    T.Iv.assign(mu * nv * 2, 0.0);
    std::vector<ld> IvL(mu * nv * 2, 0.0L);
    for (int q = 0; q < T.nq; ++q) {
        ld x = T.qx[q], y = T.qy[q];
        std::vector<std::pair<ld, ld>> V;
        for (int deg = 0; deg < k; ++deg)
            for (int i = 0; i <= deg; ++i) {
                ld m = powl(x, deg - i) * powl(y, i);
                V.push_back({m, 0}); V.push_back({0, m});
            }
        for (int i = 0; i < k; ++i) {
            ld m = powl(x, k - 1 - i) * powl(y, i);
            V.push_back({-y * m, x * m});
        }
        if ((int)V.size() != nv) throw std::runtime_error("Nedelec basis size");
        for (int a = 0; a < mu; ++a)
            for (int v = 0; v < nv; ++v) {
                IvL[(a * nv + v) * 2] += (ld)T.qw[q] * phiL[q * mu + a] * V[v].first;
                IvL[(a * nv + v) * 2 + 1] += (ld)T.qw[q] * phiL[q * mu + a] * V[v].second;
            }
    }
    for (size_t i = 0; i < IvL.size(); ++i) T.Iv[i] = (double)IvL[i];
    // BDM moment matrix: rows = dofs (edge e, j < k+2; then interior v), cols = (d, a)
    std::vector<ld> Vb(nu * nu, 0.0L);
    for (int e = 0; e < 3; ++e)
        for (int j = 0; j < nb; ++j)
            for (int d = 0; d < 2; ++d)
                for (int a = 0; a < mu; ++a) {
                    ld s = 0;
                    for (int q = 0; q < T.nfq; ++q) s += fwL[q] * ephiL[(e * T.nfq + q) * mu + a] * legL[q * nb + j];
                    Vb[(e * nb + j) * nu + d * mu + a] = (ld)T.eh[e] * (ld)T.en[e][d] * s;
                }
    for (int v = 0; v < nv; ++v)
        for (int d = 0; d < 2; ++d)
            for (int a = 0; a < mu; ++a) Vb[(3 * nb + v) * nu + d * mu + a] = IvL[(a * nv + v) * 2 + d];
    invert(nu, Vb);
    T.bdm_inv.resize(nu * nu);
    for (int i = 0; i < nu * nu; ++i) T.bdm_inv[i] = (double)Vb[i];
    // nodal <-> modal on the lattices
    auto lattice_maps = [&](int m, int n, std::vector<double> &nod, std::vector<double> &mod) {
        std::vector<ld> V(n * n);
        int node = 0;
        for (int j = 0; j <= m; ++j)
            for (int i = 0; i <= m - j; ++i, ++node) {
                dubiner_ld(m, ld(i) / m, ld(j) / m, tmp);
                for (int a = 0; a < n; ++a) V[node * n + a] = tmp[a].v;
            }
        mod.resize(n * n);
        for (int i = 0; i < n * n; ++i) mod[i] = (double)V[i];
        invert(n, V);
        nod.resize(n * n);
        for (int i = 0; i < n * n; ++i) nod[i] = (double)V[i];
    };
    lattice_maps(k + 1, mu, T.nod_u, T.mod_u);
    lattice_maps(k, np, T.nod_p, T.mod_p);
    {
        std::vector<ld> V(nt * nt);
        for (int i = 0; i < nt; ++i) {
            legendre01_ld(nt - 1, ld(i) / k, lv);
            for (int j = 0; j < nt; ++j) V[i * nt + j] = lv[j];
        }
        T.mod_t.resize(nt * nt);
        for (int i = 0; i < nt * nt; ++i) T.mod_t[i] = (double)V[i];
        invert(nt, V);
        T.nod_t.resize(nt * nt);
        for (int i = 0; i < nt * nt; ++i) T.nod_t[i] = (double)V[i];
    }
    return T;
}

}  // namespace hdg
