"""The C-ABI's boundary entry points beyond the hot-path rows: hdg_project (L2 projection of data
sampled at the library's quadrature points) and the wait bound hdg_params.timeout_ms
(HDG_ERR_TIMEOUT).

hdg_project is checked against what the mathematics fixes (it reproduces every polynomial of the
space: the nodal values equal the polynomial at the lattice) and against the oracle's own L2
projection (oracle/hdg.py, its own Gauss rule) on data both rules integrate exactly.
timeout_ms is checked by a wait that runs out on the host: the step stays queued on the stream,
and the state the next call reads is the one a run without the bound reaches.
"""
import numpy as np
import pytest

import hdg_workloads as W
from oracle import Mesh, HDG

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


def H():
    import paper_2410_09790_gb300 as mod
    return mod


def qp_values(ctx, n, k, fun, field, Lx=1.0, Ly=1.0):
    """fun sampled at the library's volume points of every cell (host numpy -> device)."""
    pts, _ = H().hdg_reference_rule(k, 0)
    v = W.cell_vertices(n, Lx, Ly)                                      # (c, 3, 2)
    X = v[:, None, 0, :] + pts[None, :, 0, None] * (v[:, None, 1] - v[:, None, 0]) \
        + pts[None, :, 1, None] * (v[:, None, 2] - v[:, None, 0])       # (c, nq, 2)
    if field == 0:
        vals = np.stack(fun(X[..., 0], X[..., 1]), axis=1)              # (c, 2, nq)
    else:
        vals = fun(X[..., 0], X[..., 1])
    return torch.from_numpy(np.ascontiguousarray(vals, dtype=np.float64)).cuda()


@pytest.mark.parametrize('px', [False, True])
@pytest.mark.parametrize('k', [1, 2, 3, 4])
def test_project_reproduces_the_space_and_matches_the_oracle(k, px):
    n, Lx = 5, 2.0
    ctx = H().Context(n, k, periodic_x=px, Lx=Lx)
    # a velocity of degree k+1 and a pressure of degree k: reproduced exactly at the lattice
    vel = lambda x, y: (x ** (k + 1) - 2 * x * y + 1.0, y ** k * x - 0.5 * y)
    pre = lambda x, y: x ** k - y + 0.25
    Q = ctx.hdg_project(0, qp_values(ctx, n, k, vel, 0, Lx)).cpu().numpy().reshape(-1)
    p = ctx.hdg_project(1, qp_values(ctx, n, k, pre, 1, Lx)).cpu().numpy().reshape(-1)
    X = W.cell_nodes(n, k + 1, Lx)
    Xp = W.cell_nodes(n, k, Lx)
    exQ = np.stack(vel(X[..., 0], X[..., 1]), 1).reshape(-1)
    exp_ = pre(Xp[..., 0], Xp[..., 1]).reshape(-1)
    assert np.abs(Q - exQ).max() <= 1e-12 * np.abs(exQ).max() * 10 ** k
    assert np.abs(p - exp_).max() <= 1e-12 * np.abs(exp_).max() * 10 ** k
    # data of degree k+2 (the library's rule is exact to degree 2 floor((3k+4)/2) - 1 >= 2k+3,
    # the degree of its product with the velocity basis) against the oracle's projection with its
    # own rule
    hq = HDG(Mesh(n, Lx=Lx, periodic_x=px), k)
    g = lambda x, y: (x ** (k + 1) * y - 3 * y ** 2, x * y ** (k + 1) + x ** 2)
    Qg = ctx.hdg_project(0, qp_values(ctx, n, k, g, 0, Lx)).cpu().numpy().reshape(-1)
    Qo = hq.l2_project(g, 0)
    assert np.linalg.norm(Qg - Qo) <= 1e-11 * np.linalg.norm(Qo)
    ctx.close()


def test_project_rejects_bad_field():
    ctx = H().Context(3, 2)
    v = torch.zeros(ctx.ncells * 64, dtype=torch.float64, device='cuda')
    st = H().load().hdg_project(ctx._ctx, 2, H().hdg._ptr(v), H().hdg._ptr(v))
    assert st == H().hdg.HDG_ERR_INVALID_ARG
    ctx.close()


def test_timeout_returns_at_once_and_the_step_completes_on_the_stream():
    n, k = 32, 3
    Q0 = W.nodal_velocity(n, k, lambda x, y: W.shear_layer(x, y, width=0.1, amp=0.05), noise=1e-3, seed=12)
    kw = dict(periodic_x=True, tableau='ARS343', dt=2e-3, n_richardson=0, richardson_rtol=1e-10,
              richardson_max=600)
    ref = H().Context(n, k, **kw)
    ref.hdg_set_state(torch.from_numpy(Q0).cuda())
    ref.hdg_div_free_project()
    ref.hdg_imex_step(1)
    ref.hdg_imex_step(1)
    Qr, pr, lr, tr = [x.cpu().numpy() if hasattr(x, 'cpu') else x for x in ref.hdg_get_state()]
    ref.close()
    ctx = H().Context(n, k, timeout_ms=0.001, **kw)          # a bound no step can meet
    ctx.hdg_set_state(torch.from_numpy(Q0).cuda())
    ctx.hdg_div_free_project()
    st1 = ctx.hdg_imex_step(1, check=False)   # set-up is not bounded; the step's wait is
    st2 = ctx.hdg_imex_step(1, check=False)   # waits for step 1 first, then times out on step 2
    assert st1['status'] == H().hdg.HDG_ERR_TIMEOUT and st2['status'] == H().hdg.HDG_ERR_TIMEOUT
    Q, p, lam, t = ctx.hdg_get_state()                        # waits for the queued step
    assert abs(t - tr) < 1e-15 and abs(t - 2 * 2e-3) < 1e-15
    assert np.array_equal(Q.cpu().numpy(), Qr) and np.array_equal(p.cpu().numpy(), pr)
    assert np.array_equal(lam.cpu().numpy(), lr)
    ctx.close()
