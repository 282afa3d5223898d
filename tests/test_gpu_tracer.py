"""Parity of the GPU tracer advection (App. B) with the oracle, through the C-ABI: the continuous
projection P_CG (hdg_cg_project), the upwind DG operator M^-1 a(., q, U) (hdg_tracer_rhs) and the
tracer carried through IMEX steps (hdg_set_tracer / hdg_imex_step / hdg_get_tracer), on meshes with
walls and periodic directions, k = 1..4. Bar: relative L2 <= 1e-10 (FP64 path)."""
import numpy as np
import pytest

import hdg_workloads as W
from oracle import Mesh, HDG, Oracle, Tracer, TABLEAUS

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

MESHES = [(4, False, False), (4, True, False), (3, True, True)]


def H():
    import paper_2410_09790_gb300 as mod
    return mod


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy().reshape(-1)


def assert_close(got, ref, tol, name):
    l2 = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    mx = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert l2 <= tol and mx <= 10 * tol, f'{name}: rel L2 {l2:.3e}, rel max {mx:.3e}'


@pytest.mark.parametrize('n,px,py', MESHES)
@pytest.mark.parametrize('k', [1, 2, 3, 4])
def test_cg_projection_matches_oracle(n, px, py, k):
    h = HDG(Mesh(n, periodic_x=px, periodic_y=py), k)
    T = Tracer(h)
    ctx = H().Context(n, k, periodic_x=px, periodic_y=py)
    Q = np.random.default_rng(100 + k).standard_normal((h.mesh.ncells, 2, h.mu))
    got = host(ctx.hdg_cg_project(cuda(Q)))
    ctx.close()
    assert_close(got, T.cg_project(Q.reshape(-1)), 1e-11, 'P_CG')


@pytest.mark.parametrize('n,px,py', MESHES)
@pytest.mark.parametrize('k', [1, 2, 3, 4])
def test_tracer_operator_matches_oracle(n, px, py, k):
    h = HDG(Mesh(n, periodic_x=px, periodic_y=py), k)
    T = Tracer(h)
    rng = np.random.default_rng(200 + k)
    U = T.cg_project(rng.standard_normal(h.nQ))
    q = rng.standard_normal(h.nP)
    ctx = H().Context(n, k, periodic_x=px, periodic_y=py)
    got = host(ctx.hdg_tracer_rhs(cuda(q.reshape(ctx.shapes()[1])), cuda(U.reshape(ctx.shapes()[0]))))
    ctx.close()
    assert_close(got, T.rhs(q, U), 1e-11, 'M^-1 a(q, U)')


@pytest.mark.parametrize('tab,k', [('ARS222', 2), ('IMEX_EULER', 1), ('SSP2_332', 2), ('ARS343', 3)])
@pytest.mark.parametrize('mode', ['graph', 'host'])
def test_tracer_through_imex_steps_matches_oracle(tab, k, mode):
    # the tracer advected by the step's stage velocities, explicit tableau (App. B), stages to
    # tolerance; the velocity is a Taylor-Green field with noise, the tracer a smooth bump
    n, dt = 4, 0.02
    Q0 = W.nodal_velocity(n, k, W.taylor_green, noise=1e-2, seed=31)
    q0 = W.nodal_scalar(n, k, lambda x, y: np.exp(-10 * ((x - 0.4) ** 2 + (y - 0.6) ** 2)))
    ctx = H().Context(n, k, tableau=tab, dt=dt, n_richardson=0, stage_krylov=1, richardson_rtol=1e-13,
                      richardson_max=600, trace_rtol=1e-14, stepI_rtol=1e-14, max_iters=20000,
                      device_loops=1 if mode == 'graph' else 0)
    ctx.hdg_set_state(cuda(Q0))
    ctx.hdg_reconstruct_pressure()
    ctx.hdg_set_tracer(cuda(q0))
    ctx.hdg_imex_step(2)
    q = host(ctx.hdg_get_tracer())
    Q = host(ctx.hdg_get_state()[0])
    ctx.close()
    h = HDG(Mesh(n), k)
    o, T = Oracle(h), Tracer(h)
    Qo, qo = Q0.reshape(-1), q0.reshape(-1)
    _, po, lo = o.reconstruct_pressure(Qo)
    for s in range(2):
        stages = []
        Qn, po, lo = o.imex_step(TABLEAUS[tab](), dt, s * dt, Qo, po, lo, stages=stages)
        qo = T.step(TABLEAUS[tab](), dt, qo, stages)
        Qo = Qn
    assert_close(Q, Qo, 1e-10, 'Q')
    assert_close(q, qo, 1e-10, 'tracer')
