"""Parity of the CUDA path (through the C-ABI) with the oracle, row by row of the hot path.

Bar: relative L2 difference <= 1e-10 and relative max difference <= 1e-9 per field (Q, p and
lambda alike; FP64 path),
with the iterative solves run at tight tolerances (the oracle's inner solves are direct).
Inputs: seeded random nodal fields (hdg_workloads) on meshes of several tiles with walls and
periodic directions, k = 1..4.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import hdg_workloads as W
from oracle import Mesh, HDG, Oracle, bdm_project, TABLEAUS

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TIGHT = dict(trace_rtol=1e-14, stepI_rtol=1e-14, max_iters=20000)
MESHES = [(3, False, False), (4, True, False), (3, True, True)]


def H():
    import paper_2410_09790_gb300 as mod
    return mod


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy().reshape(-1)


def assert_close(got, ref, tol=1e-10, name=''):
    got, ref = np.asarray(got).ravel(), np.asarray(ref).ravel()
    scale = max(np.linalg.norm(ref), 1e-300)
    l2 = np.linalg.norm(got - ref) / scale
    mx = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert l2 <= tol and mx <= 10 * tol, f'{name}: rel L2 {l2:.3e}, rel max {mx:.3e}'


def setup(n, px, py, k, **kw):
    m = Mesh(n, periodic_x=px, periodic_y=py)
    h = HDG(m, k)
    ctx = H().Context(n, k, periodic_x=px, periodic_y=py, **(TIGHT | kw))
    return m, h, ctx


def trace_mass(h):
    """Oracle trace mass matrix (block diagonal, nodal basis)."""
    m = h.mesh
    blk = np.einsum('q,qi,qj->ij', h.tw, h.mut, h.mut)
    return sp.block_diag([m.f_h[f] * blk for f in range(m.nfacets)], format='csc')


@pytest.mark.parametrize('k', [1, 2, 3, 4])
@pytest.mark.parametrize('mesh', MESHES)
def test_bdm_projection(k, mesh):
    m, h, ctx = setup(*mesh, k)
    Q = np.random.default_rng(k).standard_normal(h.nQ)
    got = host(ctx.hdg_bdm_project(cuda(Q.reshape(ctx.shapes()[0]))))
    assert_close(got, bdm_project(h, Q), 1e-11, 'Q*')


@pytest.mark.parametrize('k', [1, 2, 3, 4])
@pytest.mark.parametrize('mesh', MESHES)
def test_fimpl_apply(k, mesh):
    m, h, ctx = setup(*mesh, k)
    rng = np.random.default_rng(10 + k)
    Qs = bdm_project(h, rng.standard_normal(h.nQ))
    Q = rng.standard_normal(h.nQ)
    sQ = ctx.shapes()[0]
    got = host(ctx.hdg_fimpl_apply(cuda(Qs.reshape(sQ)), cuda(Q.reshape(sQ))))
    M = h.static()[0]
    ref = spla.spsolve(M.tocsc(), h.fimpl(Qs) @ Q)
    assert_close(got, ref, 1e-11, 'f_impl')


@pytest.mark.parametrize('k', [1, 2, 3, 4])
@pytest.mark.parametrize('mesh', MESHES)
def test_trace_operator(k, mesh):
    m, h, ctx = setup(*mesh, k)
    o = Oracle(h)
    lam = np.random.default_rng(20 + k).standard_normal(h.nL)
    for c in (2e-3, 1.0):
        got = host(ctx.hdg_trace_apply(c, cuda(lam.reshape(ctx.shapes()[2]))))
        *_, S = o.condensed_mixed_solve(c, np.zeros(h.nQ), np.zeros(o.nY))
        ref = -spla.spsolve(trace_mass(h), S @ lam)      # oracle's S is negative semidefinite
        assert_close(got, ref, 1e-11, f'S lambda (c={c})')


@pytest.mark.parametrize('mg', [0, 1])
@pytest.mark.parametrize('k', [1, 2, 3, 4])
@pytest.mark.parametrize('mesh', MESHES + [(8, True, False)])
def test_mixed_solve(k, mesh, mg):
    m, h, ctx = setup(*mesh, k, trace_mg=mg)
    o = Oracle(h)
    rng = np.random.default_rng(30 + k)
    R, X = rng.standard_normal(h.nQ), rng.standard_normal(h.nQ)
    sQ = ctx.shapes()[0]
    for c in (2e-3, 1.0):
        U, p, lam, st = ctx.hdg_mixed_solve(c, cuda(R.reshape(sQ)), cuda(X.reshape(sQ)))
        Uo, po, lo = o.mixed_solve(c, o.M @ R, -o.B @ X)
        assert_close(host(U), Uo, 1e-10, 'U')
        assert_close(host(p), po, 1e-10, 'p')
        assert_close(host(lam), lo, 1e-10, 'lambda')
        assert st['trace_iters'] > 0


@pytest.mark.parametrize('k', [1, 2, 3, 4])
@pytest.mark.parametrize('mesh', MESHES)
def test_tentative_solve(k, mesh):
    m, h, ctx = setup(*mesh, k)
    o = Oracle(h)
    rng = np.random.default_rng(40 + k)
    Qs = bdm_project(h, W.nodal_velocity(mesh[0], k, W.taylor_green).reshape(-1) + 0.3 * rng.standard_normal(h.nQ))
    R = rng.standard_normal(h.nQ)
    sQ = ctx.shapes()[0]
    c = 0.01
    got, st = ctx.hdg_tentative_solve(c, cuda(Qs.reshape(sQ)), cuda(R.reshape(sQ)))
    F = h.fimpl(Qs)
    ref = spla.spsolve((o.M - c * F).tocsc(), o.M @ R)
    assert_close(host(got), ref, 1e-10, 'Qbar')


@pytest.mark.parametrize('k', [2, 3])
@pytest.mark.parametrize('mesh', MESHES)
def test_solve_stage_fixed_richardson(k, mesh):
    # Alg. 2 with the paper's n_R = 2 against the oracle's Alg. 2 with direct inner solves
    m, h, ctx = setup(*mesh, k, n_richardson=2)
    o = Oracle(h)
    rng = np.random.default_rng(50 + k)
    Q0 = W.nodal_velocity(mesh[0], k, W.taylor_green).reshape(-1) + 0.05 * rng.standard_normal(h.nQ)
    p0, l0 = rng.standard_normal(h.nP), rng.standard_normal(h.nL)
    Qs = bdm_project(h, Q0)
    R = Q0 + 0.1 * rng.standard_normal(h.nQ)
    c = 0.004
    sQ, sP, sL = ctx.shapes()
    Q, p, lam = cuda(Q0.reshape(sQ)), cuda(p0.reshape(sP)), cuda(l0.reshape(sL))
    st = ctx.hdg_solve_stage(c, cuda(R.reshape(sQ)), cuda(Qs.reshape(sQ)), Q, p, lam)
    Qo, po, lo, it = o.richardson(c, o.M @ R, Qs, Q0, p0 - h.mean_p(p0), l0 - h.mean_p(p0), n_iter=2)
    assert st['richardson_iters'] == 2 and it == 2
    assert_close(host(Q), Qo, 1e-10, 'Q')
    assert_close(host(p), po, 1e-10, 'p')
    assert_close(host(lam), lo, 1e-10, 'lambda')


def test_solve_stage_tolerance_reaches_monolithic():
    # Alg. 2 iterated to tolerance (plain Richardson)
    m, h, ctx = setup(4, True, False, 2, n_richardson=0, stage_krylov=0, richardson_rtol=1e-13, richardson_max=200)
    o = Oracle(h)
    rng = np.random.default_rng(60)
    Q0 = W.nodal_velocity(4, 2, W.taylor_green).reshape(-1) + 0.05 * rng.standard_normal(h.nQ)
    Qs = bdm_project(h, Q0)
    c = 0.003
    sQ, sP, sL = ctx.shapes()
    Q, p, lam = cuda(Q0.reshape(sQ)), cuda(np.zeros(sP)), cuda(np.zeros(sL))
    st = ctx.hdg_solve_stage(c, cuda(Q0.reshape(sQ)), cuda(Qs.reshape(sQ)), Q, p, lam)
    Qd, pd, ld = o.stage_solve(c, o.M @ Q0, Qs)
    assert st['richardson_iters'] > 2
    assert_close(host(Q), Qd, 1e-10, 'Q')
    assert_close(host(p), pd, 1e-10, 'p')


@pytest.mark.parametrize('n,k,c', [(4, 2, 0.003), (16, 2, 3.6 / 256), (8, 3, 0.9 / 64), (8, 1, 0.9 / 64),
                                   (8, 4, 0.9 / 64)])
def test_solve_stage_krylov_reaches_monolithic(n, k, c):
    # Alg. 2's preconditioner inside flexible GMRES, including the stiff regime c/h^2 = 3.6 where
    # the plain Richardson iteration contracts slowly
    m, h, ctx = setup(n, True, False, k, n_richardson=0, stage_krylov=1, richardson_rtol=1e-12, richardson_max=400)
    o = Oracle(h)
    rng = np.random.default_rng(61)
    Q0 = W.nodal_velocity(n, k, lambda x, y: W.shear_layer(x, y, width=0.1, amp=0.05), noise=1e-3, seed=2).reshape(-1)
    Q0, p0, l0 = o.div_free_project(Q0)
    Qs = bdm_project(h, Q0)
    sQ, sP, sL = ctx.shapes()
    Q, p, lam = cuda(Q0.reshape(sQ)), cuda(p0.reshape(sP)), cuda(l0.reshape(sL))
    st = ctx.hdg_solve_stage(c, cuda(Q0.reshape(sQ)), cuda(Qs.reshape(sQ)), Q, p, lam)
    Qd, pd, ld = o.stage_solve(c, o.M @ Q0, Qs)
    assert st['richardson_iters'] >= 1
    assert_close(host(Q), Qd, 1e-10, 'Q')
    assert_close(host(p), pd, 1e-10, 'p')
    assert_close(host(lam), ld, 1e-10, 'lambda')


@pytest.mark.parametrize('mg', [0, 1])
def test_device_loops_match_host_loops(mg):
    # the stage solve recorded as one graph with device-side loops runs the same kernels in the same
    # order as the host-driven loops: identical results, bit for bit
    n, k = 8, 2
    Q0 = W.nodal_velocity(n, k, lambda x, y: W.shear_layer(x, y, width=0.1, amp=0.05), noise=1e-3, seed=4)
    outs, stats = [], []
    for dl in (0, 1):
        ctx = H().Context(n, k, periodic_x=True, tableau='ARS343', dt=0.01, n_richardson=0, stage_krylov=1,
                          richardson_rtol=1e-11, richardson_max=300, trace_mg=mg, device_loops=dl)
        ctx.hdg_set_state(cuda(Q0))
        ctx.hdg_reconstruct_pressure()
        stats.append(ctx.hdg_imex_step(2))
        outs.append([host(x) for x in ctx.hdg_get_state()[:3]])
        ctx.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    for key in ('richardson_iters', 'stepI_solves', 'stepI_iters', 'trace_solves', 'trace_iters',
                'stage_products32'):
        assert stats[0][key] == stats[1][key] > 0, key


@pytest.mark.parametrize('k', [1, 3, 4])
def test_precision_fp64_and_mixed_reach_the_same_stage_solutions(k):
    # HDG_FP64 runs every kernel of the path in FP64, HDG_MIXED the preconditioner in FP32: the
    # precision of the preconditioner changes neither the fixed point (the monolithic stage
    # solution) nor the FP64 stage tolerance both meet; the results agree to that tolerance
    n = 8
    Q0 = W.nodal_velocity(n, k, lambda x, y: W.shear_layer(x, y, width=0.1, amp=0.05), noise=1e-3, seed=6)
    outs, stats = [], []
    for prec in ('FP64', 'MIXED'):
        ctx = H().Context(n, k, periodic_x=True, tableau='ARS343', dt=0.01, n_richardson=0, stage_krylov=1,
                          richardson_rtol=1e-12, richardson_max=400, precision=prec)
        ctx.hdg_set_state(cuda(Q0))
        ctx.hdg_reconstruct_pressure()
        stats.append(ctx.hdg_imex_step(2))
        outs.append([host(x) for x in ctx.hdg_get_state()[:3]])
        ctx.close()
    assert_close(outs[1][0], outs[0][0], 1e-10, 'Q')
    assert_close(outs[1][1], outs[0][1], 1e-10, 'p')
    assert_close(outs[1][2], outs[0][2], 1e-10, 'lambda')
    for st in stats:
        assert st['status'] == 0 and st['stepI_solves'] > 0 and st['stepI_iters'] >= st['stepI_solves']


@pytest.mark.parametrize('n,px,k', [(8, True, 1), (8, True, 2), (8, True, 3), (8, True, 4), (16, False, 4),
                                    (3, True, 2)])
def test_relaxed_fp32_products_keep_the_stage_tolerance(n, px, k):
    # HDG_MIXED takes the late Arnoldi products of the stage FGMRES in FP32 (relax_eta): the
    # restart and final checks form the residual in FP64, so every eta meets the same stage
    # tolerance and the results agree to it; eta = 0 takes no FP32 product, the default some, and
    # a deliberately reckless eta = 1e-13 (the FP32 product assumed exact: FP32 products from the
    # first step on) still converges: a cycle that does not halve the FP64 residual switches the
    # rest of its solve to FP64 products
    Q0 = W.nodal_velocity(n, k, lambda x, y: W.shear_layer(x, y, width=0.1, amp=0.05), noise=1e-3, seed=9)
    outs, stats = [], []
    for eta in (0.0, 1e-4, 1e-13):
        ctx = H().Context(n, k, periodic_x=px, tableau='ARS343', dt=0.01, n_richardson=0, stage_krylov=1,
                          richardson_rtol=1e-12, richardson_max=400, relax_eta=eta)
        ctx.hdg_set_state(cuda(Q0))
        ctx.hdg_reconstruct_pressure()
        stats.append(ctx.hdg_imex_step(2))
        outs.append([host(x) for x in ctx.hdg_get_state()[:3]])
        ctx.close()
    for i in (1, 2):
        assert_close(outs[i][0], outs[0][0], 1e-10, 'Q')
        assert_close(outs[i][1], outs[0][1], 1e-10, 'p')
        assert_close(outs[i][2], outs[0][2], 1e-10, 'lambda')
    for st in stats:
        assert st['status'] == 0
    assert stats[0]['stage_products32'] == 0
    assert 0 < stats[1]['stage_products32'] < stats[1]['richardson_iters']
    assert stats[2]['stage_products32'] > 0
    assert stats[1]['richardson_iters'] <= stats[0]['richardson_iters'] + 2 * stats[0]['stage_solves'], \
        (stats[1]['richardson_iters'], stats[0]['richardson_iters'])


@pytest.mark.parametrize('n,px,k', [(8, True, 1), (8, True, 2), (8, True, 3), (8, True, 4), (16, False, 3),
                                    (3, True, 2)])
def test_inner_trace_vcycle_fp32_matches_fp64(n, px, k):
    # the preconditioner's one-V-cycle Step II in FP32 (group widths 2, 4, 4, 8 for k = 1..4; one to
    # three P1 levels) changes only the preconditioner: both runs meet the same stage tolerance,
    # agree to it, and need about as many outer iterations
    Q0 = W.nodal_velocity(n, k, lambda x, y: W.shear_layer(x, y, width=0.1, amp=0.05), noise=1e-3, seed=8)
    outs, stats = [], []
    for f32 in (0, 1):
        ctx = H().Context(n, k, periodic_x=px, tableau='ARS343', dt=0.01, n_richardson=0, stage_krylov=1,
                          richardson_rtol=1e-12, richardson_max=400, inner_trace_fp32=f32)
        ctx.hdg_set_state(cuda(Q0))
        ctx.hdg_reconstruct_pressure()
        stats.append(ctx.hdg_imex_step(2))
        outs.append([host(x) for x in ctx.hdg_get_state()[:3]])
        ctx.close()
    assert_close(outs[1][0], outs[0][0], 1e-10, 'Q')
    assert_close(outs[1][1], outs[0][1], 1e-10, 'p')
    for st in stats:
        assert st['status'] == 0 and st['trace_solves'] > 0
    it64, it32 = stats[0]['richardson_iters'], stats[1]['richardson_iters']
    assert it32 <= 1.1 * it64 + 3, (it32, it64)


@pytest.mark.parametrize('n,px,k', [(8, True, 1), (8, True, 2), (8, True, 3), (8, True, 4), (16, False, 3)])
def test_inner_gauss_seidel_matches_jacobi(n, px, k):
    # the red-black block Gauss-Seidel preconditioner of the inner Step-I solves changes only the
    # preconditioner: both runs meet the stage tolerance, agree to it, need about as many outer
    # iterations, and Gauss-Seidel fewer inner Arnoldi steps
    Q0 = W.nodal_velocity(n, k, lambda x, y: W.shear_layer(x, y, width=0.1, amp=0.05), noise=1e-3, seed=9)
    outs, stats = [], []
    for gsp in (0, 1):
        ctx = H().Context(n, k, periodic_x=px, tableau='ARS343', dt=0.01, n_richardson=0, stage_krylov=1,
                          richardson_rtol=1e-12, richardson_max=400, inner_gs=gsp)
        ctx.hdg_set_state(cuda(Q0))
        ctx.hdg_reconstruct_pressure()
        stats.append(ctx.hdg_imex_step(2))
        outs.append([host(x) for x in ctx.hdg_get_state()[:3]])
        ctx.close()
    assert_close(outs[1][0], outs[0][0], 1e-10, 'Q')
    assert_close(outs[1][1], outs[0][1], 1e-10, 'p')
    for st in stats:
        assert st['status'] == 0 and st['stepI_solves'] > 0
    assert stats[1]['richardson_iters'] <= 1.15 * stats[0]['richardson_iters'] + 3, stats
    assert stats[1]['stepI_iters'] < stats[0]['stepI_iters'], stats


@pytest.mark.parametrize('n,px,k', [(8, True, 2), (16, False, 3), (16, True, 4)])
def test_trace_cg_fp32_vcycle_matches_fp64(n, px, k):
    # the tight trace solves with the FP32 V-cycle inside flexible CG reach the same tolerance as
    # plain CG with the FP64 V-cycle, give the same solution to it, in about as many iterations
    rng = np.random.default_rng(71)
    R = rng.standard_normal((2 * n * n, 2, (k + 2) * (k + 3) // 2))
    outs, its = [], []
    for f32 in (0, 1):
        ctx = H().Context(n, k, periodic_x=px, trace_rtol=1e-12, max_iters=20000, trace_mg=1, trace_fp32_vcycle=f32)
        U, dp, dl, st = ctx.hdg_mixed_solve(1.0, cuda(R))
        outs.append([host(U), host(dp), host(dl)])
        its.append(st['trace_iters'])
        assert st['last_trace_relres'] <= 1e-12
        ctx.close()
    for a, b, name in zip(outs[1], outs[0], ('U', 'dp', 'dl')):
        assert_close(a, b, 1e-10, name)
    assert its[1] <= 1.5 * its[0] + 3, its


@pytest.mark.parametrize('n,k', [(128, 1), (128, 2)])
def test_large_mesh_fp32_vcycle_with_grid_levels_matches_fp64(n, k):
    # 128 x 128: the finest P1 level (129^2 vertices) is too large for the one-block tail, so the
    # FP32 V-cycle runs it with grid-wide kernels around the tail. FP32 and FP64 V-cycles (inner
    # Step II and the tight trace CG) change only the preconditioners: both runs reach the stage
    # tolerance, agree to it, and need about as many outer iterations
    Q0 = W.nodal_velocity(n, k, W.taylor_green, noise=1e-2, seed=3)      # pressure O(1), as velocity
    outs, its = [], []
    for f32 in (1, 0):
        ctx = H().Context(n, k, periodic_x=True, tableau='ARS222', dt=1e-3, n_richardson=0, stage_krylov=1,
                          richardson_rtol=1e-12, richardson_max=400, inner_trace_fp32=f32, trace_fp32_vcycle=f32)
        ctx.hdg_set_state(cuda(Q0))
        ctx.hdg_div_free_project()
        st = ctx.hdg_imex_step(1)
        assert st['status'] == 0 and st['stage_solves'] >= 2 and st['richardson_iters'] > 0, st
        its.append(st['richardson_iters'])
        outs.append([host(x) for x in ctx.hdg_get_state()[:3]])
        ctx.close()
    assert_close(outs[0][0], outs[1][0], 1e-10, 'Q')
    assert_close(outs[0][1], outs[1][1], 1e-10, 'p')
    assert_close(outs[0][2], outs[1][2], 1e-10, 'lambda')
    assert its[0] <= 1.1 * its[1] + 3, its


@pytest.mark.parametrize('n,px', [(16, True), (32, False)])
def test_multigrid_iterations_mesh_robust(n, px):
    # the V-cycle preconditioner keeps the trace CG iteration count small and nearly independent
    # of h, unlike facet block-Jacobi (Sec. 3.4.2 reports the same robustness for the paper's MG)
    k = 2
    rng = np.random.default_rng(70)
    R = rng.standard_normal((2 * n * n, 2, (k + 2) * (k + 3) // 2))
    its = {}
    for mg in (0, 1):
        ctx = H().Context(n, k, periodic_x=px, trace_rtol=1e-10, max_iters=20000, trace_mg=mg)
        *_, st = ctx.hdg_mixed_solve(1.0, cuda(R))
        its[mg] = st['trace_iters']
        ctx.close()
    assert its[1] <= 25 and its[0] > 4 * its[1], its


def _run_imex(n, k, px, tab, dt, steps, Q0, gpu_kw, oracle_solver, oracle_kw):
    m = Mesh(n, periodic_x=px)
    h = HDG(m, k)
    o = Oracle(h)
    ctx = H().Context(n, k, periodic_x=px, tableau=tab, dt=dt, **(TIGHT | gpu_kw))
    ctx.hdg_set_state(cuda(Q0))
    ctx.hdg_reconstruct_pressure()
    st = ctx.hdg_imex_step(steps)
    Q, p, lam, t = ctx.hdg_get_state()
    Qo = Q0.reshape(-1)
    _, po, lo = o.reconstruct_pressure(Qo)
    for s in range(steps):
        Qo, po, lo = o.imex_step(TABLEAUS[tab](), dt, s * dt, Qo, po, lo, solver=oracle_solver,
                                 richardson_kw=oracle_kw)
    return (host(Q), host(p), host(lam), t), (Qo, po, lo), st


def test_imex_taylor_green_8x8_k2_converged_stages():
    # the plain-FP64 Taylor-Green workload (8x8, k=2, ARS(2,2,2), dt=0.01, 10 steps); stages
    # iterated to 1e-13 against the oracle's monolithic (direct) stage solves
    Q0 = W.nodal_velocity(8, 2, W.taylor_green)
    (Q, p, lam, t), (Qo, po, lo), st = _run_imex(8, 2, False, 'ARS222', 0.01, 10, Q0,
                                                dict(n_richardson=0, richardson_rtol=1e-12, richardson_max=200),
                                                'direct', None)
    assert abs(t - 0.1) < 1e-14
    assert_close(Q, Qo, 1e-10, 'Q')
    assert_close(p, po, 1e-10, 'p')
    assert_close(lam, lo, 1e-10, 'lambda')


@pytest.mark.parametrize('k,tab', [(1, 'IMEX_EULER'), (3, 'ARS343')])
def test_imex_fixed_richardson_shear_channel(k, tab):
    # periodic channel, shear layer + noise, divergence-free projected, n_R = 2 (the paper's setting)
    n = 4
    Qb = W.nodal_velocity(n, k, lambda x, y: W.shear_layer(x, y, width=0.2, amp=0.1), noise=1e-3, seed=1)
    m = Mesh(n, periodic_x=True)
    o = Oracle(HDG(m, k))
    Q0, _, _ = o.div_free_project(Qb.reshape(-1))
    (Q, p, lam, t), (Qo, po, lo), st = _run_imex(n, k, True, tab, 0.02, 3, Q0.reshape(Qb.shape),
                                                dict(n_richardson=2), 'richardson', dict(n_iter=2))
    assert_close(Q, Qo, 1e-10, 'Q')
    assert_close(p, po, 1e-10, 'p')


def test_div_free_projection_and_forcing():
    n, k = 4, 2
    m = Mesh(n)
    h = HDG(m, k)
    o = Oracle(h)
    Qb = W.nodal_velocity(n, k, W.taylor_green, noise=0.05, seed=3)
    ctx = H().Context(n, k, tableau='ARS222', dt=0.02, n_richardson=3, **TIGHT)
    ctx.hdg_set_state(cuda(Qb))
    ctx.hdg_div_free_project()
    Q, p, lam, _ = ctx.hdg_get_state()
    Qo, _, _ = o.div_free_project(Qb.reshape(-1))
    _, po, lo = o.reconstruct_pressure(Qo)
    assert_close(host(Q), Qo, 1e-10, 'Q div-free')
    assert_close(host(p), po, 1e-10, 'p reconstructed')
    # forcing f = phi(t) F through the explicit tableau (eq. f_expl)
    F = W.nodal_velocity(n, k, W.taylor_green)
    phi = lambda t: np.exp(-t)
    ctx.hdg_set_forcing(cuda(F), phi)
    ctx.hdg_imex_step(2)
    Q, p, lam, _ = ctx.hdg_get_state()
    fd = o.M @ F.reshape(-1)
    forcing = lambda t: phi(t) * fd
    Qo2, po2, lo2 = Qo, *o.reconstruct_pressure(Qo)[1:]
    for s in range(2):
        Qo2, po2, lo2 = o.imex_step(TABLEAUS['ARS222'](), 0.02, s * 0.02, Qo2, po2, lo2, forcing=forcing,
                                    solver='richardson', richardson_kw=dict(n_iter=3))
    assert_close(host(Q), Qo2, 1e-10, 'Q forced')
    assert_close(host(p), po2, 1e-10, 'p forced')


def test_deterministic_bitwise():
    n, k = 6, 3
    Q0 = W.nodal_velocity(n, k, W.taylor_green, noise=1e-3, seed=5)
    outs = []
    for _ in range(2):
        ctx = H().Context(n, k, tableau='ARS343', dt=0.01, n_richardson=2)
        ctx.hdg_set_state(cuda(Q0))
        ctx.hdg_reconstruct_pressure()
        ctx.hdg_imex_step(2)
        outs.append([host(x) for x in ctx.hdg_get_state()[:3]])
        ctx.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_invalid_inputs_rejected_on_device():
    ctx = H().Context(3, 2)
    with pytest.raises(H().HdgError):
        ctx.hdg_mixed_solve(-1.0)
    with pytest.raises(ValueError):
        ctx.hdg_set_state(torch.zeros(3, device='cuda'))          # wrong dtype


def test_time_kernel_modes_and_algorithmic_bytes():
    # the instrumentation bench.py builds its roofline on: every mode runs, and modes 6, 8 and 9
    # report the algorithmic bytes their documentation states
    n, k = 8, 3
    Q0 = W.nodal_velocity(n, k, lambda x, y: W.shear_layer(x, y, width=0.1, amp=0.05), noise=1e-3, seed=12)
    ctx = H().Context(n, k, periodic_x=True, tableau='ARS343', dt=0.01, n_richardson=0, stage_krylov=1,
                      richardson_rtol=1e-10, richardson_max=400)
    ctx.hdg_set_state(cuda(Q0))
    ctx.hdg_reconstruct_pressure()
    ctx.hdg_imex_step(1)
    cstage = 0.43586652150845899942 * 0.01
    mu, npk, nt = (k + 2) * (k + 3) // 2, (k + 1) * (k + 2) // 2, k + 1
    nu, nfq = 2 * mu, (3 * k + 5) // 2
    nc = ctx.nQ // nu
    res = {}
    for which in range(12):
        ms, b = ctx.hdg_time_kernel(which, 1.0 if which == 1 else cstage, 3)
        assert ms > 0.0 and np.isfinite(ms), (which, ms)
        res[which] = b
    assert res[6] == 4.0 * (nc * 3 * nfq * 3 + 2 * ctx.nQ + 5 * ctx.nQ)
    assert res[9] == 4.0 * (nc * nu * nu + 6 * ctx.nQ + nc * 3 * nfq * 2)
    # HDG_MIXED (default) at this stage tolerance: the pair-arithmetic kernel, whose block is read as
    # its FP32 copy and rest in the padded per-cell layout (rows padded to 4, blocks to 32 floats)
    nup = (nu + 3) // 4 * 4
    size = (nu * nup + 31) // 32 * 32
    vec = 8.0 * (2 * ctx.nQ + 2 * ctx.nP + ctx.nL + nc * 3 * nt)
    assert res[8] == 8.0 * nc * (size + 3 * nfq) + 4.0 * 6 * nc + vec
    ctx.close()
    ctx = H().Context(n, k, periodic_x=True, tableau='ARS343', dt=0.01, n_richardson=0, stage_krylov=1,
                      richardson_rtol=1e-10, richardson_max=400, precision='FP64')
    ctx.hdg_set_state(cuda(Q0))
    ctx.hdg_reconstruct_pressure()
    ctx.hdg_imex_step(1)
    ms, b = ctx.hdg_time_kernel(8, cstage, 3)
    assert ms > 0.0 and b == 8.0 * nc * (nu * nu + 3 * nfq) + 4.0 * 6 * nc + vec
    ctx.close()


@pytest.mark.parametrize('prec', ['FP64', 'MIXED'])
def test_forced_taylor_green_step_graph_matches_oracle(prec):
    # the manufactured Taylor-Green forcing f = -kappa exp(-kappa t) Q0 (eq. taylor_green_Q0_f) in the
    # one-graph-per-step path (the forcing's time factors are device values refreshed per step),
    # against the oracle's monolithic stage solves
    n, k, dt, kappa = 6, 3, 0.02, 1.0
    Q0 = W.nodal_velocity(n, k, W.taylor_green)
    ctx = H().Context(n, k, tableau='ARS343', dt=dt, n_richardson=0, stage_krylov=1, device_loops=1,
                      richardson_rtol=1e-13, richardson_max=600, precision=prec, **TIGHT)
    ctx.hdg_set_state(cuda(Q0))
    ctx.hdg_set_forcing(cuda(Q0), lambda t: -kappa * np.exp(-kappa * t))
    ctx.hdg_reconstruct_pressure()
    st = ctx.hdg_imex_step(3)
    assert st['graph_kernels'] > 0
    Q, p, lam, t = ctx.hdg_get_state()
    ctx.close()
    o = Oracle(HDG(Mesh(n), k))
    fd = o.M @ Q0.reshape(-1)
    forcing = lambda tt: -kappa * np.exp(-kappa * tt) * fd
    Qo = Q0.reshape(-1)
    _, po, lo = o.reconstruct_pressure(Qo, forcing(0.0))
    for s in range(3):
        Qo, po, lo = o.imex_step(TABLEAUS['ARS343'](), dt, s * dt, Qo, po, lo, forcing=forcing)
    assert abs(t - 3 * dt) < 1e-15
    assert_close(host(Q), Qo, 1e-10, 'Q')
    assert_close(host(p), po, 1e-10, 'p')
    assert_close(host(lam), lo, 1e-10, 'lambda')


@pytest.mark.parametrize('tab,k,mode', [('SSP2_332', 2, 'krylov'), ('SSP3_433', 3, 'krylov'), ('SSP2_332', 2, 'nR2'),
                                        ('SSP3_433', 1, 'nR2'), ('IMEX_EULER', 1, 'krylov')])
def test_paper_tableaus_step_matches_oracle(tab, k, mode):
    # the paper's SSP2(3,3,2) / SSP3(4,3,3) (implicit first stage) and IMEX Euler, stages solved to
    # tolerance or by the paper's n_R = 2 Richardson iterations, against the oracle's recursion
    n, dt = 4, 0.02
    Q0 = W.nodal_velocity(n, k, W.taylor_green, noise=1e-2, seed=21)
    kw = dict(n_richardson=0, stage_krylov=1, richardson_rtol=1e-13, richardson_max=600) if mode == 'krylov' \
        else dict(n_richardson=2)
    ctx = H().Context(n, k, tableau=tab, dt=dt, **(TIGHT | kw))
    ctx.hdg_set_state(cuda(Q0))
    ctx.hdg_reconstruct_pressure()
    ctx.hdg_imex_step(2)
    Q, p, lam, _ = ctx.hdg_get_state()
    ctx.close()
    o = Oracle(HDG(Mesh(n), k))
    Qo = Q0.reshape(-1)
    _, po, lo = o.reconstruct_pressure(Qo)
    okw = dict(solver='direct') if mode == 'krylov' else dict(solver='richardson', richardson_kw=dict(n_iter=2))
    for s_ in range(2):
        Qo, po, lo = o.imex_step(TABLEAUS[tab](), dt, s_ * dt, Qo, po, lo, **okw)
    assert_close(host(Q), Qo, 1e-10, 'Q')
    assert_close(host(p), po, 1e-10, 'p')
    assert_close(host(lam), lo, 1e-10, 'lambda')


@pytest.mark.parametrize('k,tab', [(1, 'IMEX_EULER'), (2, 'SSP2_332'), (3, 'SSP3_433')])
def test_paper_convergence_experiment_rates(k, tab):
    # Sec. 3.4 on the GPU with the paper's own tableaus: forced Taylor-Green (eq. taylor_green_Q0_f),
    # kappa = 0.5, T = 1, n_t = n (dt = 1/n), stages solved to tolerance; L2 errors against the exact
    # solution at t = T fall at the rate ~ k the paper reports, in velocity and pressure
    import hdg_workloads as Wk
    kappa, errs = 0.5, []
    meshes = (8, 16) if k < 3 else (4, 8)
    for n in meshes:
        ctx = H().Context(n, k, tableau=tab, dt=1.0 / n, n_richardson=0, stage_krylov=1, richardson_rtol=1e-11,
                          richardson_max=900)
        pts, _ = H().hdg_reference_rule(k, 0)
        Q0 = ctx.hdg_project(0, cuda(Wk.sampled_velocity(n, pts, Wk.taylor_green)))
        ctx.hdg_set_state(Q0)
        ctx.hdg_set_forcing(Q0, lambda t: -kappa * np.exp(-kappa * t))
        ctx.hdg_reconstruct_pressure()
        ctx.hdg_imex_step(n)
        Q, p, _, t = ctx.hdg_get_state()
        ctx.close()
        h = HDG(Mesh(n), k)
        from oracle.element import triangle_quadrature
        qp, qw = triangle_quadrature(10)
        X = h.mesh.cell_points(np.arange(h.mesh.ncells), qp)
        exQ = np.exp(-kappa * t) * np.stack(Wk.taylor_green(X[..., 0], X[..., 1]), -1)
        exp_ = np.exp(-2 * kappa * t) * Wk.taylor_green_pressure(X[..., 0], X[..., 1])
        numQ = np.einsum('qa,cda->cqd', h.Vu.values(qp), host(Q).reshape(h.mesh.ncells, 2, h.mu))
        nump = np.einsum('qb,cb->cq', h.Vp.values(qp), host(p).reshape(h.mesh.ncells, h.npn))
        eQ = np.sqrt(np.sum(qw[None, :, None] * h.mesh.detJ[:, None, None] * (numQ - exQ) ** 2))
        ep = np.sqrt(np.sum(qw[None, :] * h.mesh.detJ[:, None] * (nump - exp_) ** 2))
        errs.append((eQ, ep))
    rQ, rp = np.log2(errs[0][0] / errs[1][0]), np.log2(errs[0][1] / errs[1][1])
    assert rQ > k - 0.3 and rp > k - 0.3, (errs, rQ, rp)


def test_double_shear_layer_matches_oracle():
    # Sec. 3.3: the doubly periodic double shear layer on [0, 2 pi]^2 (rho = pi/15, delta = 0.05),
    # SSP3(4,3,3), dt = 0.04 as in the paper, upwind flux; a coarse mesh against the oracle
    n, k, dt = 6, 3, 0.04
    L = 2 * np.pi
    Q0 = W.nodal_velocity(n, k, W.double_shear_layer, Lx=L, Ly=L)
    ctx = H().Context(n, k, periodic_x=True, periodic_y=True, Lx=L, Ly=L, tableau='SSP3_433', dt=dt,
                      n_richardson=0, stage_krylov=1, richardson_rtol=1e-13, richardson_max=900, **TIGHT)
    ctx.hdg_set_state(cuda(Q0))
    ctx.hdg_div_free_project()
    ctx.hdg_imex_step(2)
    Q, p, lam, _ = ctx.hdg_get_state()
    ctx.close()
    o = Oracle(HDG(Mesh(n, Lx=L, Ly=L, periodic_x=True, periodic_y=True), k))
    Qo, _, _ = o.div_free_project(Q0.reshape(-1))
    _, po, lo = o.reconstruct_pressure(Qo)
    for s_ in range(2):
        Qo, po, lo = o.imex_step(TABLEAUS['SSP3_433'](), dt, s_ * dt, Qo, po, lo)
    assert_close(host(Q), Qo, 1e-10, 'Q')
    assert_close(host(p), po, 1e-10, 'p')
    assert_close(host(lam), lo, 1e-10, 'lambda')
