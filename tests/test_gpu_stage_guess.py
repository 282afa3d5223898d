"""Initial guesses of the stage solves carried from one IMEX step to the next.

A stage solved to a tolerance may start anywhere: its result is fixed by the tolerance. The
library starts each stage of a step from its solution in the previous step (velocity shifted by
the state's change over that step, pressure and trace extrapolated from the last two steps),
which is first-order closer than the previous stage's solution. These tests check that the
guesses change the results only within the stage tolerance, lower the outer iteration count,
survive a get_state / set_state round trip of the step's own output, and are dropped when the
state is set to something else.
"""
import numpy as np
import pytest

import hdg_workloads as W

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

N, K, DT, STEPS = 16, 2, 2e-3, 6


def _ctx():
    """The forced Taylor-Green vortex with walls (the flow decays in time as exp(-t))."""
    import paper_2410_09790_gb300 as H
    ctx = H.Context(N, K, tableau='ARS343', dt=DT, n_richardson=0, richardson_rtol=1e-10)
    Q0 = torch.from_numpy(W.nodal_velocity(N, K, W.taylor_green)).cuda()
    ctx.hdg_set_state(Q0)
    ctx.hdg_set_forcing(Q0, lambda t: -np.exp(-t))
    ctx.hdg_div_free_project()
    return ctx


def _host(t):
    return t.cpu().numpy().ravel()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _run(mode):
    """STEPS steps; mode 'straight': one call; 'roundtrip': get/set the state between steps;
    'cleared': the pressure reconstructed between steps (its call clears the history)."""
    ctx = _ctx()
    outer = 0
    if mode == 'straight':
        outer += ctx.hdg_imex_step(STEPS)['richardson_iters']
    else:
        for _ in range(STEPS):
            outer += ctx.hdg_imex_step(1)['richardson_iters']
            if mode == 'roundtrip':
                Q, p, lam, t = ctx.hdg_get_state()
                ctx.hdg_set_state(Q.clone(), p.clone(), lam.clone(), t)
            else:
                ctx.hdg_reconstruct_pressure()
    Q, p, lam, _ = ctx.hdg_get_state()
    ctx.close()
    return _host(Q), _host(p), _host(lam), outer


def test_stage_guesses_keep_results_and_cut_iterations():
    Qa, pa, la, na = _run('straight')
    Qc, pc, lc, nc = _run('cleared')
    # same solutions within the stage tolerance (1e-10 relative residual per stage)
    assert _rel(Qa, Qc) <= 1e-9, _rel(Qa, Qc)
    vel = np.linalg.norm(Qc)
    assert np.linalg.norm(pa - pc) <= 1e-9 * vel and np.linalg.norm(la - lc) <= 1e-9 * vel
    # the guesses start closer: fewer outer iterations over the same steps
    assert na < nc, (na, nc)


def test_stage_guesses_survive_a_state_round_trip():
    Qa, pa, la, na = _run('straight')
    Qb, pb, lb, nb = _run('roundtrip')
    assert abs(na - nb) <= 2, (na, nb)
    assert _rel(Qa, Qb) <= 1e-9, _rel(Qa, Qb)


def test_stage_guesses_dropped_for_another_state():
    ctx = _ctx()
    ctx.hdg_imex_step(3)
    Q, p, lam, t = ctx.hdg_get_state()
    Q2 = 0.5 * Q                                  # not the state the last step left
    ctx.hdg_set_state(Q2.clone(), None, None, t)
    ng = ctx.hdg_imex_step(2)['richardson_iters']
    Qg = _host(ctx.hdg_get_state()[0])
    ctx.close()
    # a fresh context from the same state takes the same steps without any history
    ref = _ctx()
    ref.hdg_set_state(Q2.clone(), None, None, t)
    nr = ref.hdg_imex_step(2)['richardson_iters']
    Qr = _host(ref.hdg_get_state()[0])
    ref.close()
    # (a kept history would move the result by the stage tolerance, ~1e-10)
    assert ng == nr and _rel(Qg, Qr) <= 1e-13, (ng, nr, _rel(Qg, Qr))
