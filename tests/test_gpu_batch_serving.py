"""Batched and served execution (hdg_batch_step, hdg_server_*): many independent instances of
different mesh sizes and degrees on the GPU at once, each giving exactly the result it gives alone.

  * hdg_batch_step over mixed (n, k, tableau, boundary) instances: every instance's fields after
    the batched steps are bitwise those of the same instance stepped alone (deterministic kernels,
    no shared buffers);
  * the memory estimate used for admission bounds the memory a context actually allocates;
  * the server: requests arriving while others run are admitted as slots and memory free up,
    contexts of finished requests are reused by requests of the same configuration, at most
    max_active requests run at once, and every request's result is bitwise its result alone.
"""
import numpy as np
import pytest

import hdg_workloads as W

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

KW = dict(n_richardson=0, stage_krylov=1, richardson_rtol=1e-10, richardson_max=600)
INSTANCES = [dict(n=8, k=1, tableau='ARS222', dt=0.01), dict(n=8, k=2, tableau='ARS343', dt=0.005, periodic_x=True),
             dict(n=6, k=3, tableau='SSP2_332', dt=0.01), dict(n=4, k=4, tableau='ARS343', dt=0.01, periodic_x=True,
                                                               periodic_y=True),
             dict(n=12, k=2, tableau='IMEX_EULER', dt=0.01), dict(n=16, k=1, tableau='ARS343', dt=0.004)]


def H():
    import paper_2410_09790_gb300 as mod
    return mod


def field(inst, seed):
    modes = W.stream_function_modes(seed)
    return W.nodal_velocity(inst['n'], inst['k'], lambda x, y: W.stream_velocity(x, y, modes))


def make(inst, Q0):
    kw = {key: v for key, v in inst.items() if key not in ('n', 'k')}
    ctx = H().Context(inst['n'], inst['k'], stream=torch.cuda.Stream(), **KW, **kw)
    ctx.hdg_set_state(torch.from_numpy(Q0).cuda())
    ctx.hdg_div_free_project()
    return ctx


def state(ctx):
    return [x.cpu().numpy() for x in ctx.hdg_get_state()[:3]]


def test_batch_step_matches_each_instance_alone():
    fields = [field(inst, 40 + i) for i, inst in enumerate(INSTANCES)]
    alone = []
    for inst, Q0 in zip(INSTANCES, fields):
        ctx = make(inst, Q0)
        ctx.hdg_imex_step(3)
        alone.append(state(ctx))
        ctx.close()
    ctxs = [make(inst, Q0) for inst, Q0 in zip(INSTANCES, fields)]
    stats, status = H().hdg_batch_step(ctxs, 3)
    assert status == 0 and all(s['stage_solves'] > 0 and s['graph_kernels'] > 0 for s in stats)
    for ctx, ref in zip(ctxs, alone):
        for a, b in zip(state(ctx), ref):
            assert np.array_equal(a, b)
        ctx.close()


@pytest.mark.parametrize('inst', INSTANCES[:4])
def test_memory_estimate_bounds_the_context(inst):
    ctx = make(inst, field(inst, 7))
    ctx.hdg_imex_step(2)
    used = ctx.hdg_ctx_bytes()
    kw = {key: v for key, v in inst.items() if key not in ('n', 'k')}
    est = H().hdg_estimate_bytes(inst['n'], inst['k'], **KW, **kw)
    ctx.close()
    assert used <= est <= 2.5 * used + (2 << 20), (used, est)


def test_server_continuous_batching_admission_and_reuse():
    reqs = [(INSTANCES[0], 3), (INSTANCES[1], 2), (INSTANCES[0], 4), (INSTANCES[2], 3), (INSTANCES[4], 2),
            (INSTANCES[1], 1), (INSTANCES[3], 2), (INSTANCES[0], 2)]
    fields = [field(inst, 60 + i) for i, (inst, _) in enumerate(reqs)]
    alone = []
    for (inst, steps), Q0 in zip(reqs, fields):
        ctx = make(inst, Q0)
        ctx.hdg_imex_step(steps)
        alone.append(state(ctx))
        ctx.close()
    # a budget that holds about three of these contexts, at most three requests at once
    est = [H().hdg_estimate_bytes(inst['n'], inst['k'], **KW, **{key: v for key, v in inst.items()
                                                                  if key not in ('n', 'k')}) for inst, _ in reqs]
    budget = 3.2 * max(est)
    srv = H().Server(budget, max_active=3)
    ids, rounds = [], 0
    pending = list(range(len(reqs)))
    while True:
        # two new arrivals per round while requests remain (they join the running batch)
        for _ in range(2):
            if pending:
                i = pending.pop(0)
                inst, steps = reqs[i]
                kw = {key: v for key, v in inst.items() if key not in ('n', 'k')}
                ids.append(srv.submit(inst['n'], inst['k'], fields[i], steps, **KW, **kw))
        st = srv.progress()
        rounds += 1
        assert st['active'] <= 3 and st['bytes_in_use'] <= budget * 1.01
        if st['completed'] == len(reqs):
            break
        assert rounds < 100
    assert st['submitted'] == st['admitted'] == st['completed'] == len(reqs)
    assert st['contexts_reused'] >= 1 and st['contexts_created'] + st['contexts_reused'] == len(reqs)
    for rid, ref in zip(ids, alone):
        out = srv.result(rid)
        assert out is not None and out[3] > 0
        for a, b in zip(out[:3], ref):
            assert np.array_equal(a, b.reshape(-1))
    srv.close()
