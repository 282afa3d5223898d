"""Seeded synthetic inputs for the hybridised DG IMEX solver (shared by tests, bench and the
oracle; holds none of the method's arithmetic).

Exchange format. Fields are passed as nodal values on the canonical structured mesh: n x n
rectangles over [0, Lx] x [0, Ly], rectangle (i, j) split along its (i,j)-(i+1,j+1) diagonal
into cell 2(jn+i) with vertices (A, B, C) and cell 2(jn+i)+1 with vertices (A, C, D), where
A=(i,j), B=(i+1,j), C=(i+1,j+1), D=(i,j+1). A degree-m cell field is given at the lattice
nodes v0 + (i/m)(v1 - v0) + (j/m)(v2 - v0), i + j <= m, j outer / i inner. A velocity is an
array (ncells, 2, n_nodes(k+1)), a pressure (ncells, n_nodes(k)), a trace (nfacets, k+1) at
t = i/k along each facet in its canonical direction. Facets: horizontal H(i,j), then vertical
V(i,j), then diagonal D(i,j), j-major; periodic directions drop the duplicate edges.
"""
import numpy as np


def lattice(m):
    if m == 0:
        return np.array([[1.0 / 3.0, 1.0 / 3.0]])
    return np.array([(i / m, j / m) for j in range(m + 1) for i in range(m + 1 - j)], float)


def cell_vertices(n, Lx=1.0, Ly=1.0):
    hx, hy = Lx / n, Ly / n
    v = np.zeros((2 * n * n, 3, 2))
    for j in range(n):
        for i in range(n):
            A = (i * hx, j * hy); B = ((i + 1) * hx, j * hy)
            C = ((i + 1) * hx, (j + 1) * hy); D = (i * hx, (j + 1) * hy)
            v[2 * (j * n + i)] = (A, B, C)
            v[2 * (j * n + i) + 1] = (A, C, D)
    return v


def cell_nodes(n, m, Lx=1.0, Ly=1.0):
    """Physical coordinates (ncells, n_nodes(m), 2) of the degree-m lattice of every cell."""
    v = cell_vertices(n, Lx, Ly)
    L = lattice(m)
    return (v[:, None, 0, :] + L[None, :, 0, None] * (v[:, None, 1] - v[:, None, 0])
            + L[None, :, 1, None] * (v[:, None, 2] - v[:, None, 0]))


# ---------------------------------------------------------------- analytic fields
def taylor_green(x, y, scale=np.pi):
    """u = (sin(s x) cos(s y), -cos(s x) sin(s y)) (s = pi on the unit square)."""
    return np.sin(scale * x) * np.cos(scale * y), -np.cos(scale * x) * np.sin(scale * y)


def taylor_green_pressure(x, y, scale=np.pi):
    """p with grad p = -(u.grad)u for taylor_green: (cos 2sx + cos 2sy) / 4."""
    return 0.25 * (np.cos(2 * scale * x) + np.cos(2 * scale * y))


def shear_layer(x, y, width=0.05, amp=1e-3):
    """(tanh((y - 1/2)/width), amp sin(2 pi x)) on the unit channel."""
    return np.tanh((y - 0.5) / width), amp * np.sin(2 * np.pi * x)


def double_shear_layer(x, y, rho=np.pi / 15, delta=0.05):
    """The doubly periodic double shear layer on [0, 2 pi]^2: u = tanh((y - pi/2)/rho) for
    y <= pi, tanh((3 pi/2 - y)/rho) above; v = delta sin x."""
    u = np.where(y <= np.pi, np.tanh((y - 0.5 * np.pi) / rho), np.tanh((1.5 * np.pi - y) / rho))
    return u, delta * np.sin(x)


def stream_function_modes(seed, n_modes=8, kmax=4):
    """(m1, m2, a) for psi = sum a sin(m1 pi x) sin(m2 pi y), a ~ N(0,1)/|m|^2."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(1, kmax + 1, size=(n_modes, 2))
    a = rng.standard_normal(n_modes) / (ms[:, 0] ** 2 + ms[:, 1] ** 2)
    return ms, a


def stream_velocity(x, y, modes):
    """u = (d psi/dy, -d psi/dx) for the stream function of stream_function_modes."""
    ms, a = modes
    u = np.zeros_like(x); v = np.zeros_like(x)
    for (m1, m2), am in zip(ms, a):
        u += am * m2 * np.pi * np.sin(m1 * np.pi * x) * np.cos(m2 * np.pi * y)
        v -= am * m1 * np.pi * np.cos(m1 * np.pi * x) * np.sin(m2 * np.pi * y)
    return u, v


def nodal_velocity(n, k, fun, Lx=1.0, Ly=1.0, noise=0.0, seed=0):
    """Velocity nodal values (ncells, 2, n_nodes(k+1)) of fun, plus optional N(0,1)*noise
    per nodal value."""
    X = cell_nodes(n, k + 1, Lx, Ly)
    u, v = fun(X[..., 0], X[..., 1])
    Q = np.stack([u, v], axis=1)
    if noise:
        Q = Q + noise * np.random.default_rng(seed).standard_normal(Q.shape)
    return np.ascontiguousarray(Q)


def nodal_scalar(n, m, fun, Lx=1.0, Ly=1.0):
    X = cell_nodes(n, m, Lx, Ly)
    return np.ascontiguousarray(fun(X[..., 0], X[..., 1]))


def random_nodal_velocity(n, k, seed):
    nn = len(lattice(k + 1))
    return np.random.default_rng(seed).standard_normal((2 * n * n, 2, nn))


def cell_points(n, ref_pts, Lx=1.0, Ly=1.0):
    """Physical coordinates (ncells, npts, 2) of reference points (npts, 2) (xi, eta) in every
    cell: v0 + xi (v1 - v0) + eta (v2 - v0)."""
    v = cell_vertices(n, Lx, Ly)
    P = np.asarray(ref_pts, float)
    return (v[:, None, 0, :] + P[None, :, 0, None] * (v[:, None, 1] - v[:, None, 0])
            + P[None, :, 1, None] * (v[:, None, 2] - v[:, None, 0]))


def sampled_velocity(n, ref_pts, fun, Lx=1.0, Ly=1.0):
    """fun sampled at reference points of every cell: (ncells, 2, npts), the layout of a
    velocity sample for the library's L2 projection."""
    X = cell_points(n, ref_pts, Lx, Ly)
    u, v = fun(X[..., 0], X[..., 1])
    return np.ascontiguousarray(np.stack([u, v], axis=1))


# ---------------------------------------------------------------- named workloads
# The benchmark's configurations (data only). c2: the shear layer in the periodic channel, every
# stage solved to a relative stage residual of 1e-10. c3: the forced Taylor-Green vortex on the
# unit square with walls (f = -kappa exp(-kappa t) Q0, exact solution exp(-kappa t) Q0); its time
# step keeps the stage stiffness c/h^2 = a_ii dt n^2 of c2 (dt scaled by h^2).
WORKLOADS = {
    'c2': dict(n=64, k=3, periodic_x=True, tableau='ARS343', dt=2e-3, steps=100,
               init='shear_layer', width=0.05, amp=1e-3, noise=1e-4, seed=0, stage_rtol=1e-10,
               name='shear-layer channel 64x64, k=3, ARS(3,4,3), dt=2e-3, stages to 1e-10'),
    'c3': dict(n=256, k=4, periodic_x=False, tableau='ARS343', dt=1.25e-4, steps=50,
               init='taylor_green', kappa=1.0, stage_rtol=1e-10,
               name='forced Taylor-Green 256x256 walls, k=4, ARS(3,4,3), dt=1.25e-4, stages to 1e-10'),
}
