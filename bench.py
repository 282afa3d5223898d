"""Benchmark: IMEX stage solves/s of the HDG incompressible-Euler stage solver on GB300.

Default workload (c2, the plain-method GPU configuration): periodic-in-x channel [0,1]^2 with
walls at y = 0, 1, 64 x 64 rectangles -> 8192 triangles, k = 3 (velocity P4, pressure/trace P3),
ARS(3,4,3), dt = 2e-3; every stage solved to a relative stage residual of 1e-10 (flexible GMRES
preconditioned by Alg. 2's Chorin split; inside it Step I by one FP32 GMRES cycle to 2e-2 and
Step II by one FP32 trace multigrid V-cycle: precision HDG_MIXED; the paper's fixed n_R = 2 is
unstable on this flow); final update and pressure reconstruction trace CG rtol 1e-12; initial
u = (tanh((y-1/2)/0.05), 1e-3 sin 2 pi x) + seeded N(0,1) 1e-4 noise per nodal value, projected to
divergence-free. One bench step = one IMEX time step of Alg. 1 (3 stage solves, final update,
pressure reconstruction) through hdg_imex_step. The same steps are also timed with every kernel in
FP64 (precision HDG_FP64; same stage tolerance) and the two results compared field by field.

--workload c3: the forced Taylor-Green vortex on 256 x 256 rectangles with walls, k = 4,
ARS(3,4,3), dt = 1.25e-4 (the stage stiffness c/h^2 of c2), f = -exp(-t) Q0, initial field and
forcing by the library's L2 projection (hdg_project); HDG_MIXED and HDG_FP64 timed in the same run,
errors against each other and against the exact solution exp(-t) Q0.

Output: one JSON line (rank 0). value = stage solves/s (whole job); trace_dof_per_s = trace
unknowns x trace solves / s. e2e: the same through the C-ABI with the state copied from pinned
host memory to the device and back every step. kernels: the path's main kernels, each timed
alone with CUDA events on the context's stream (time per launch), with launches per step from the
solver's own counters; roofline: the one of them with the largest device time per step. FP64
kernels are bound by GB300's FP64 pipe (achieved = algorithmic FP64 flops / time against the
nominal FP64 rate), FP32 ones by memory (algorithmic bytes / time against the measured HBM peak;
their data stays in L2 where it fits, 129 MB). trace_apply, condensation and stage_apply_fp64
report more kernels the same way.
cpu_baseline / --impl reference: the oracle (plain FP64 SciPy) on the host cores.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# solver settings of every bench context (the workloads themselves: hdg_workloads.WORKLOADS)
SOLVER = dict(n_richardson=0, stage_krylov=1, inner_stepI_rtol=2e-2, inner_trace_rtol=1e-1, trace_rtol=1e-12,
              stepI_rtol=1e-10, inner_trace_vcycles=1, inner_trace_fp32=1, trace_fp32_vcycle=1, inner_gs=1,
              richardson_max=600)
STAGES = {'ARS343': 3, 'ARS222': 2, 'IMEX_EULER': 1}
METRIC = 'IMEX stage solves/s (trace-DoF/s alongside)'


def measured_peaks():
    try:
        with open(os.path.join(ROOT, 'MEASURED_PEAKS.json')) as f:
            d = json.load(f)
        return float(d['hbm_gbs']), 'measured'
    except Exception:
        return 6800.0, 'fallback'


FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64 (vector pipe): 152 SMs x 2.07 GHz x 4 flops per clock


def profile_traffic(name):
    """DRAM bytes per launch of a kernel from its committed ncu summary profiles/<name> (None if
    the summary does not state them)."""
    import re
    try:
        with open(os.path.join(ROOT, 'profiles', name)) as f:
            m = re.search(r'^traffic_bytes_per_launch = (\d+)$', f.read(), re.M)
        return int(m.group(1)) if m else None
    except OSError:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(['nvidia-smi', '-i', str(self.idx), f'--query-gpu={self.Q}',
                                      '--format=csv,noheader,nounits'], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(',')])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['unavailable']}
        sm = sorted(float(s[1]) for s in self.samples if s[1].replace('.', '').isdigit())
        mx = max((float(s[2]) for s in self.samples if s[2].replace('.', '').isdigit()), default=None)
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        reasons = sorted({names[i] for s in self.samples for i in range(4) if len(s) > 5 + i and s[5 + i] == 'Active'})
        return {'sm_mhz': sm[len(sm) // 2] if sm else None, 'sm_max_mhz': mx, 'reasons': reasons,
                'samples': len(self.samples)}


def aggregate_ranks(total_ms, e2e_ms, world, device):
    """Whole-job timing over the ranks of a replica run: the slowest rank's time (MAX) for the
    timed steps and for the end-to-end steps. world == 1 returns the inputs."""
    if world == 1:
        return total_ms, e2e_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0]), float(t[1])


def job_rate(world, stages, steps, total_ms):
    """Stage solves per second of the whole job: every rank solves `stages` x `steps` stages."""
    return world * stages * steps / (total_ms / 1e3)


def workload(name):
    import hdg_workloads as W
    return dict(W.WORKLOADS[name])


def initial_velocity(w, n_override=None, seed_offset=0):
    import hdg_workloads as W
    n = n_override or w['n']
    return W.nodal_velocity(n, w['k'], lambda x, y: W.shear_layer(x, y, w['width'], w['amp']),
                            noise=w['noise'], seed=w['seed'] + seed_offset)


# ---------------------------------------------------------------------------------- oracle arm
def oracle_sample(w, n_sample=32):
    """The oracle (as it stands) on a bounded sample of the workload: the first stage solve of the
    first IMEX step (monolithic direct sparse LU, eq. imex_implicit_solve) of the same
    configuration on an n_sample x n_sample mesh, after the oracle's own divergence-free projection.
    Returns (stage solves/s scaled to the full mesh by the cell-count ratio, seconds of the timed
    stage solve, description, threads)."""
    os.environ.setdefault('OMP_NUM_THREADS', '1')
    os.environ.setdefault('OPENBLAS_NUM_THREADS', '1')
    from oracle import Mesh, HDG, Oracle, TABLEAUS, bdm_project
    m = Mesh(n_sample, periodic_x=w['periodic_x'])
    h = HDG(m, w['k'])
    o = Oracle(h)
    Q0 = initial_velocity(w, n_override=n_sample).reshape(-1)
    Q, _, _ = o.div_free_project(Q0)
    tab = TABLEAUS[w['tableau']]()
    c1 = tab.A_im[1, 1] * w['dt']
    t0 = time.perf_counter()
    o.stage_solve(c1, o.M @ Q, bdm_project(h, Q))
    sec = time.perf_counter() - t0
    scale = (n_sample / w['n']) ** 2
    rate = scale / sec
    desc = (f'the first stage solve (direct sparse LU of the monolithic stage system, with the f^impl assembly '
            f'and BDM projection) of the same workload on a {n_sample}x{n_sample} mesh: {sec:.1f} s; rate scaled by '
            f'the cell ratio ({n_sample}/{w["n"]})^2 to the {w["n"]}x{w["n"]} mesh (sparse LU grows faster than '
            f'the cell count, so this overstates the oracle at full size)')
    return rate, sec, desc, int(os.environ.get('OMP_NUM_THREADS', '1'))


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload('c2')
    for _ in range(min(args.warmup, 1)):
        oracle_sample(w)
    rates, secs = [], []
    for _ in range(args.steps):
        r, s, desc, cores = oracle_sample(w)
        rates.append(r)
        secs.append(s)
    value = len(rates) / sum(1.0 / r for r in rates)
    line = {'metric': METRIC, 'value': value, 'unit': 'stage_solves/s', 'impl': 'reference',
            'n_gpus': args.gpus, 'steps': args.steps, 'warmup': min(args.warmup, 1),
            'ms_per_step': 1e3 * sum(secs) / len(secs) * STAGES[w['tableau']], 'higher_is_better': True,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
            'config': {'workload': w['name'], 'n': w['n'], 'k': w['k'], 'periodic_x': True, 'sample_n': 32},
            'cpu_baseline': {'value': value, 'unit': 'stage_solves/s', 'cores': cores, 'kind': 'oracle',
                             'sample': desc},
            'e2e': {'value': value, 'unit': 'stage_solves/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------- batched / served
def c4_instances(count=64, seed=4):
    """The batching workload: `count` independent instances, mesh sizes from {16, 32, 64, 128}^2 and
    degrees from {1, 2, 3, 4} drawn with a seed, walls, ARS(3,4,3) with dt keeping the stage
    stiffness c/h^2 of the channel workload (dt = 2e-3 (64/n)^2), random divergence-free initial
    fields from a stream function of 8 Fourier modes (amplitudes N(0,1)/|m|^2)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    ns = rng.choice([16, 32, 64, 128], size=count)
    ks = rng.integers(1, 5, size=count)
    return [dict(n=int(n), k=int(k), dt=2e-3 * (64.0 / n) ** 2, seed=1000 + i) for i, (n, k) in enumerate(zip(ns, ks))]


def c5_requests(count, seed=5, rate=200.0, nmax=96, smax=30):
    """The serving workload: Poisson arrivals (mean `rate` per s), mesh sizes uniform over
    32..nmax, degrees from {2, 3, 4}, 10..smax steps each, the instances of c4_instances otherwise."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    ns = rng.integers(32, nmax + 1, size=count)
    ks = rng.integers(2, 5, size=count)
    steps = rng.integers(10, smax + 1, size=count)
    return [dict(t=float(ti), n=int(n), k=int(k), steps=int(st_), dt=2e-3 * (64.0 / n) ** 2, seed=2000 + i)
            for i, (ti, n, k, st_) in enumerate(zip(t, ns, ks, steps))]


def instance_field(inst):
    import hdg_workloads as W
    modes = W.stream_function_modes(inst['seed'])
    return W.nodal_velocity(inst['n'], inst['k'], lambda x, y: W.stream_velocity(x, y, modes))


def instance_context(H, inst, prec, kw):
    import torch
    ctx = H.Context(inst['n'], inst['k'], stream=torch.cuda.Stream(), tableau='ARS343', dt=inst['dt'],
                    precision=prec, **kw)
    ctx.hdg_set_state(torch.from_numpy(instance_field(inst)).cuda())
    ctx.hdg_div_free_project()
    return ctx


def run_batched(args, rank, world, local_rank):
    """c4: all instances advanced together (hdg_batch_step, HDG_MIXED) against the same instances
    stepped one at a time (HDG_MIXED, and every kernel in FP64: the plain GPU form)."""
    import numpy as np
    import torch
    import paper_2410_09790_gb300 as H
    torch.cuda.set_device(local_rank)
    insts = c4_instances(args.instances)
    kw = dict(SOLVER, richardson_rtol=1e-10)
    K = args.steps
    stages = STAGES['ARS343']

    def sync_time(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    out = {}
    # plain FP64 form, one instance at a time
    ctxs = [instance_context(H, inst, 'FP64', kw) for inst in insts]
    for c in ctxs:
        c.hdg_imex_step(1)
    sec64 = sync_time(lambda: [c.hdg_imex_step(K) for c in ctxs])
    for c in ctxs:
        c.close()
    # mixed precision: one at a time, then all together
    ctxs = [instance_context(H, inst, 'MIXED', kw) for inst in insts]
    H.hdg_batch_step(ctxs, 1)
    seqm = sync_time(lambda: [c.hdg_imex_step(K) for c in ctxs])
    with ClockSampler(local_rank) as clk:
        bat = sync_time(lambda: H.hdg_batch_step(ctxs, K))
    launches = sum(s['graph_kernels'] for s in H.hdg_batch_step(ctxs, 1)[0])
    for c in ctxs:
        c.close()
    n_stage = len(insts) * stages * K
    value = n_stage / bat
    line = {'metric': METRIC, 'value': value, 'unit': 'stage_solves/s', 'n_gpus': world, 'steps': K,
            'warmup': 1, 'ms_per_step': 1e3 * bat / K, 'higher_is_better': True, 'scaling': 'weak',
            'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic (seeded stream-function fields)',
            'config': {'workload': f'{len(insts)} instances, n from {{16,32,64,128}}^2, k from 1..4, walls, ARS(3,4,3), '
                                   f'dt = 2e-3 (64/n)^2, stages to 1e-10, HDG_MIXED, hdg_batch_step',
                       'instances': [[i['n'], i['k']] for i in insts], 'parallelism': 'one stream per instance',
                       'l2': 'inputs larger than L2 in total'},
            'sequential_mixed': {'value': n_stage / seqm, 'seconds': seqm},
            'sequential_fp64': {'value': n_stage / sec64, 'seconds': sec64,
                                'note': 'every kernel in FP64 (HDG_FP64), instances one at a time: the plain GPU form'},
            'speedup_vs_sequential_fp64': sec64 / bat, 'speedup_vs_sequential_mixed': seqm / bat,
            'gpu_launches': int(launches * K), 'clocks': clk.summary(),
            'e2e': {'value': None, 'unit': 'stage_solves/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_served(args, rank, world, local_rank):
    """c5: a Poisson stream of requests served by hdg_server (HDG_MIXED, continuous batching,
    admission by device memory) against the plain per-request loop (HDG_FP64, one request at a time,
    a new context each); latency = completion - arrival on the host clock."""
    import numpy as np
    import torch
    import paper_2410_09790_gb300 as H
    torch.cuda.set_device(local_rank)
    reqs = c5_requests(args.requests)
    kw = dict(SOLVER, richardson_rtol=1e-10)
    stages = STAGES['ARS343']
    fields = [instance_field(r) for r in reqs]
    free = torch.cuda.mem_get_info()[0]
    # served
    srv = H.Server(0.7 * free, max_active=args.max_active)
    ids, lat, done_t = {}, {}, {}
    t0 = time.perf_counter()
    nxt = 0
    with ClockSampler(local_rank) as clk:
        while len(lat) < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt]['t'] <= now:
                r = reqs[nxt]
                ids[srv.submit(r['n'], r['k'], fields[nxt], r['steps'], tableau='ARS343', dt=r['dt'], precision='MIXED',
                               **kw)] = nxt
                nxt += 1
            if not ids or all(i in lat for i in ids.values()):
                if nxt < len(reqs):
                    time.sleep(max(0.0, reqs[nxt]['t'] - (time.perf_counter() - t0)))
                continue
            st = srv.progress()
            tnow = time.perf_counter() - t0
            for rid, i in list(ids.items()):
                if i in lat:
                    continue
                res = srv.result(rid)
                if res is not None:
                    lat[i] = tnow - reqs[i]['t']
                    done_t[i] = res[0]
    span = time.perf_counter() - t0
    sst = srv.progress()
    srv.close()
    # the plain per-request loop
    lat64, fin64 = {}, {}
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        now = time.perf_counter() - t0
        if now < r['t']:
            time.sleep(r['t'] - now)
        ctx = instance_context(H, r, 'FP64', kw)
        ctx.hdg_imex_step(r['steps'])
        fin64[i] = ctx.hdg_get_state()[0].cpu().numpy().reshape(-1)
        ctx.close()
        torch.cuda.synchronize()
        lat64[i] = time.perf_counter() - t0 - r['t']
    span64 = time.perf_counter() - t0
    n_stage = sum(r['steps'] for r in reqs) * stages
    diff = max(float(np.linalg.norm(done_t[i] - fin64[i]) / np.linalg.norm(fin64[i])) for i in range(len(reqs)))
    pct = lambda d, q: 1e3 * float(np.percentile(np.array(list(d.values())), q))
    line = {'metric': METRIC, 'value': n_stage / span, 'unit': 'stage_solves/s', 'n_gpus': world,
            'steps': int(sum(r['steps'] for r in reqs)), 'warmup': 0, 'ms_per_step': None, 'higher_is_better': True,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic (seeded request stream)',
            'config': {'workload': f'{len(reqs)} requests, Poisson arrivals 200/s, n ~ U{{32..96}}, k in {{2,3,4}}, '
                                   f'10..30 steps, walls, ARS(3,4,3), dt = 2e-3 (64/n)^2, stages to 1e-10; '
                                   f'served by hdg_server (HDG_MIXED, continuous batching, admission by device memory)',
                       'scaled_down_from': '2,000 requests, n ~ U{32..256}, k in {2,3,4}, 10..100 steps',
                       'max_active': args.max_active, 'mem_budget_bytes': 0.7 * free},
            'latency_ms': {'p50': pct(lat, 50), 'p99': pct(lat, 99)},
            'server': sst,
            'plain_fp64_loop': {'value': n_stage / span64, 'latency_ms': {'p50': pct(lat64, 50), 'p99': pct(lat64, 99)},
                                'note': 'one request at a time in arrival order, a new HDG_FP64 context each'},
            'max_rel_diff_vs_plain_fp64': diff, 'clocks': clk.summary(), 'gpu_launches': None,
            'e2e': {'value': n_stage / span, 'unit': 'stage_solves/s', 'h2d_bytes_per_step': None,
                    'd2h_bytes_per_step': None}}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------- GPU arm
def rel_err(a, b):
    """Relative l2 difference of two nodal arrays (host numpy)."""
    import numpy as np
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


def solver_settings(args, w):
    kw = dict(SOLVER)
    for key in ('inner_trace_rtol', 'inner_stepI_rtol', 'inner_trace_vcycles', 'inner_trace_fp32', 'trace_fp32_vcycle',
                'inner_gs'):
        v = getattr(args, key)
        if v is not None:
            kw[key] = v
    kw['richardson_rtol'] = w['stage_rtol']
    kw['device_loops'] = 0 if args.host_loops else 1
    if getattr(args, 'relax_eta', None) is not None:
        kw['relax_eta'] = args.relax_eta
    return kw


def make_context(H, w, prec, stream, kw, seed_offset=0, n=None):
    """A context of workload w in precision prec, with its initial state (divergence-free)."""
    import numpy as np
    import torch
    import hdg_workloads as W
    n = n or w['n']
    ctx = H.Context(n, w['k'], periodic_x=w['periodic_x'], stream=stream, tableau=w['tableau'], dt=w['dt'],
                    precision=prec, **kw)
    if w['init'] == 'shear_layer':
        Q0 = torch.from_numpy(initial_velocity(w, n_override=n, seed_offset=seed_offset)).cuda()
        ctx.hdg_set_state(Q0)
    else:                                             # forced Taylor-Green: L2 projections
        pts, _ = H.hdg_reference_rule(w['k'], 0)
        vals = torch.from_numpy(W.sampled_velocity(n, pts, W.taylor_green)).cuda()
        Q0 = ctx.hdg_project(0, vals)
        ctx.hdg_set_state(Q0)
        kappa = w['kappa']
        ctx.hdg_set_forcing(Q0, lambda t: -kappa * np.exp(-kappa * t))
    ctx.hdg_div_free_project()
    return ctx


def timed_steps(ctx, stream, steps, warmup, flush, world=1, clk=None):
    """warmup untimed steps, then `steps` steps each between CUDA events on the context's stream
    (the L2 flushed before each). Returns (ms per step, stats per step)."""
    import torch
    for _ in range(warmup):
        ctx.hdg_imex_step(1)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stats = []

    def run():
        for i in range(steps):
            flush.fill_(float(i))                      # evict the previous step's working set
            ev[i][0].record(stream)
            stats.append(ctx.hdg_imex_step(1))
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    if clk is not None:
        with clk:
            run()
    else:
        run()
    return [a.elapsed_time(b) for a, b in ev], stats


def state_host(ctx):
    Q, p, lam, t = ctx.hdg_get_state()
    return Q.cpu().numpy(), p.cpu().numpy(), lam.cpu().numpy(), t


def e2e_steps(ctx, nsteps, flush, dev):
    """The metric end to end through the C-ABI: per step, the state from pinned host memory to the
    device, one step, the state back to pinned host memory. Returns (mean ms, bytes each way)."""
    import torch
    Qh, ph, lh, tsim = ctx.hdg_get_state()
    Qh, ph, lh = Qh.cpu().pin_memory(), ph.cpu().pin_memory(), lh.cpu().pin_memory()
    Qd, pd, ld = torch.empty_like(Qh, device=dev), torch.empty_like(ph, device=dev), torch.empty_like(lh, device=dev)
    ms = []
    for i in range(nsteps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Qd.copy_(Qh, non_blocking=True); pd.copy_(ph, non_blocking=True); ld.copy_(lh, non_blocking=True)
        ctx.hdg_set_state(Qd, pd, ld, tsim)
        ctx.hdg_imex_step(1)
        Qo, po, lo, tsim = ctx.hdg_get_state()
        Qh.copy_(Qo); ph.copy_(po); lh.copy_(lo)
        torch.cuda.synchronize()
        ms.append(1e3 * (time.perf_counter() - t0))
    return sum(ms) / max(len(ms), 1), (Qh.numel() + ph.numel() + lh.numel()) * 8


def golden_error(H, w, stream, kw):
    """Error of one step of the workload against the oracle's step stored by
    tests/golden/make_c2_golden.py (on the workload's own mesh, else 32 x 32), per field; None if
    no file is stored."""
    import numpy as np
    path = None
    for n in (w['n'], 32):                            # the workload's own mesh when stored
        cand = os.path.join(ROOT, 'tests', 'golden', f'c2_step1_{n}.npz')
        if os.path.exists(cand):
            path = cand
            break
    if path is None:
        return None
    g = np.load(path)
    n = int(g['meta'][0])
    ctx = make_context(H, w, 'MIXED', stream, kw, n=n)
    ctx.hdg_imex_step(1)
    Q, p, lam, _ = state_host(ctx)
    ctx.close()
    q_rms = float(np.linalg.norm(g['Q']) / np.sqrt(g['Q'].size))
    vs = lambda a, b: float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.sqrt(b.size) / q_rms)
    return {'mesh': f'{n}x{n} (same workload; oracle: monolithic direct stage solves)',
            'rel_l2': {'Q': rel_err(Q, g['Q']), 'p': rel_err(p, g['p']), 'lambda': rel_err(lam, g['lam'])},
            'rms_over_velocity_rms': {'Q': vs(Q, g['Q']), 'p': vs(p, g['p']), 'lambda': vs(lam, g['lam'])},
            'note': 'the flow\'s pressure is ~1e-3 of the velocity scale; the solver tolerances act at that scale'}


def stage_flops(k, ncells):
    """Algorithmic FP64 flops of one launch of the fused stage operator (k_stage_apply) and of the
    Step-I operator alone (k_cell_apply_mf)."""
    mu = (k + 2) * (k + 3) // 2
    nu, nfq = 2 * mu, (3 * k + 5) // 2
    npk, nt = (k + 1) * (k + 2) // 2, k + 1
    s_flop = 2.0 * (nu * nu + 3 * nfq * 2 * mu + 3 * nfq * 8 + nu * 3 * nfq) * ncells
    st_flop = s_flop + ncells * (nu * (3 * (2 * nt + 3) + 2 * (2 * npk + 2) + 3) + 6 * mu +
                                 npk * (4 * mu + 3 * (2 * npk + 2) + 3 * (2 * nt + 2) + 5) +
                                 3 * nt * (5 * mu + 2 * npk + 5))
    return st_flop, s_flop


def assembly_flops(k, ncells, df32=False):
    """Algorithmic flops of one launch of the Step-I assembly (k_fimpl_assemble, stage form): the
    coefficients of J^-1 Q*, {Q*}.n at the facet points (own and neighbour traces), the weighted
    facet rows, the volume advection block through the reference tensor (2 MU products per entry),
    the three weighted facet masses, and the NU x NU block entries (an FMA counts two). Returns
    (FP64 flops, flops of the parts that run in double-FP32 pairs on the FP32 pipes (df32,
    HDG_MIXED: the advection contraction, the weighted facet masses and the block entries), else 0)."""
    mu = (k + 2) * (k + 3) // 2
    nu, nfq = 2 * mu, (3 * k + 5) // 2
    fp64 = 4 * mu + 3 * nfq * 4 * mu + 3 * nfq * mu * 2 + 3 * nfq * 3
    pair = mu * mu * 2 * mu + 3 * mu * mu * nfq + nu * nu * 5
    if df32:
        return 2.0 * fp64 * ncells, 2.0 * pair * ncells
    return 2.0 * (fp64 + pair) * ncells, 0.0


def bdm_flops(k, ncells):
    """Algorithmic FP64 flops of one launch of the BDM projection (k_bdm): the normal average at the
    facet points (own and neighbour traces), the edge moments against L_j, the interior Nedelec
    moments, the NU x NU local solve through the precomputed inverse moment matrix and the Piola
    map back (an FMA counts two)."""
    mu = (k + 2) * (k + 3) // 2
    nu, nfq, nb, nv = 2 * mu, (3 * k + 5) // 2, k + 2, k * (k + 2)
    fma = 3 * nfq * 4 * mu + 3 * nb * nfq + nv * mu * 4 + nu * nu + 2 * nu
    return 2.0 * fma * ncells


def condense_flops(k, ncells):
    """Algorithmic FP64 flops of one launch of the per-cell condensation (k_condense): D and E
    formed, A = (c/detJ) D D^T + tau T_pp, H = (c/detJ) D E^T + tau E_hat^T, the Cholesky factor of
    A and its inverse, Z = A^-1 H, S_K = (c/detJ) E E^T + tau T_ll - H^T Z (an FMA counts two)."""
    mu = (k + 2) * (k + 3) // 2
    nu, npk, nl = 2 * mu, (k + 1) * (k + 2) // 2, 3 * (k + 1)
    per = (4 * npk * nu + 2 * nl * nu + npk * npk * (2 * nu + 8) + npk * nl * (2 * nu + 3) + 2 * npk ** 3 / 3
           + 2 * npk ** 3 + 2 * npk * npk * nl + nl * nl * (2 * nu + 2 * npk + 4))
    return per * ncells


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_2410_09790_gb300 as H

    torch.cuda.set_device(local_rank)
    dev = torch.device('cuda', local_rank)
    w = workload(args.workload)
    if args.n:
        w['n'] = args.n
    kw = solver_settings(args, w)
    stream = torch.cuda.Stream(device=dev)
    stages = STAGES[w['tableau']]
    gamma = 0.43586652150845899942                   # ARS(3,4,3) diagonal
    c_stage = gamma * w['dt']
    peak, peak_kind = measured_peaks()
    with torch.cuda.stream(stream):
        flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dev)   # > L2 (129 MB)
        ctx = make_context(H, w, args.precision, stream, kw, seed_offset=rank)
        if args.kernel_only is not None:
            ctx.hdg_imex_step(1)
            ms_k, b_k = ctx.hdg_time_kernel(args.kernel_only, c_stage, args.steps)
            print(json.dumps({'kernel': args.kernel_only, 'ms_per_launch': ms_k, 'bytes': b_k}), flush=True)
            ctx.close()
            return
        clk = ClockSampler(local_rank)
        ms, stats_all = timed_steps(ctx, stream, args.steps, args.warmup, flush, world, clk)
        # kernels timed alone on the same operators and stream (roofline and diagnostics)
        k_ms, k_bytes = ctx.hdg_time_kernel(0, c_stage, 50)
        s_ms, s_bytes = ctx.hdg_time_kernel(1, 1.0, 20)
        st_ms, st_bytes = ctx.hdg_time_kernel(8, c_stage, 20)
        cd_ms, cd_bytes = ctx.hdg_time_kernel(11, c_stage, 3)
        as_ms, as_bytes = ctx.hdg_time_kernel(15, c_stage, 5)
        bd_ms, bd_bytes = ctx.hdg_time_kernel(16, c_stage, 10)
        s32_ms = s32_bytes = gd_ms = gd_bytes = ga_ms = ga_bytes = None
        if args.precision == 'MIXED':
            if kw.get('relax_eta', 1e-4) > 0:
                s32_ms, s32_bytes = ctx.hdg_time_kernel(12, c_stage, 20)
            if kw.get('inner_gs', 1):
                gd_ms, gd_bytes = ctx.hdg_time_kernel(13, c_stage, 50)
                ga_ms, ga_bytes = ctx.hdg_time_kernel(14, c_stage, 50)
        e2e_ms, h2d = e2e_steps(ctx, args.e2e_steps, flush, dev)
        nsteps_done = args.warmup + args.steps + args.e2e_steps
        final = state_host(ctx)
        ntrace, nQ, nP = ctx.nL, ctx.nQ, ctx.nP
        ctx.close()
        # the same steps with every kernel in FP64 (the plain FP64 GPU form), and the two compared
        other = None
        if not args.no_compare:
            oprec = 'FP64' if args.precision == 'MIXED' else 'MIXED'
            ctx2 = make_context(H, w, oprec, stream, kw, seed_offset=rank)
            ms2, st2 = timed_steps(ctx2, stream, args.compare_steps, args.warmup, flush, world)
            for _ in range(nsteps_done - args.warmup - args.compare_steps):
                ctx2.hdg_imex_step(1)
            fin2 = state_host(ctx2)
            ctx2.close()
            other = {'precision': oprec, 'value': world * stages * len(ms2) / (sum(ms2) / 1e3),
                     'ms_per_step': float(np.mean(ms2)), 'steps': len(ms2),
                     'stage_outer_iters': sum(s['richardson_iters'] for s in st2) / len(st2),
                     'diff_after_steps': nsteps_done,
                     'rel_l2_diff': {'Q': rel_err(final[0], fin2[0]), 'p': rel_err(final[1], fin2[1]),
                                     'lambda': rel_err(final[2], fin2[2])}}
        gold = golden_error(H, w, stream, kw) if (rank == 0 and args.workload == 'c2' and not args.n) else None

    ms_step = float(np.mean(ms))
    total_ms, e2e_mean = aggregate_ranks(sum(ms), e2e_ms, world, dev)
    value = job_rate(world, stages, args.steps, total_ms)
    trace_solves = sum(s['trace_solves'] for s in stats_all)
    trace_iters = sum(s['trace_iters'] for s in stats_all)
    stepI_iters = sum(s['stepI_iters'] for s in stats_all)
    ncells = 2 * w['n'] * w['n']
    st_flop, s_flop = stage_flops(w['k'], ncells)
    host_loops = bool(args.host_loops)
    # the path's main kernels: time per launch alone (CUDA events, after the timed steps), launches
    # per step from the solver's counters, and the device time per step that gives; the roofline
    # object reports the kernel with the largest share
    outer = sum(s['richardson_iters'] for s in stats_all) / args.steps
    p32 = sum(s['stage_products32'] for s in stats_all) / args.steps
    inner = stepI_iters / args.steps
    as_flop = assembly_flops(w['k'], ncells, df32=args.precision == 'MIXED')
    if args.precision == 'MIXED':       # the pair-arithmetic kernel takes the FP64-accurate products
        st_name, st_entry = f"k_stage_apply_f2<{w['k']}>", {
            'what': 'stage operator in double-FP32 pairs, FP64-accurate (FGMRES products before the relaxed '
                    'ones, restart residuals)', 'bound': 'hbm', 'flop_fp64_equiv': st_flop}
    else:
        st_name, st_entry = f"k_stage_apply<{w['k']}>", {
            'what': 'FP64 stage operator (FGMRES products, restart residuals)', 'bound': 'alu', 'flop': st_flop}
    st_entry.update({'ms_per_launch': st_ms, 'launches_per_step': outer - p32 + 2 * stages, 'bytes': st_bytes})
    kernels = {
        st_name: st_entry,
        f"k_cg_apply<{w['k'] + 1}>": {'what': 'FP64 trace operator apply (tight trace CG)', 'ms_per_launch': k_ms,
                                      'launches_per_step': trace_iters / args.steps, 'bytes': k_bytes, 'bound': 'hbm'},
        f"k_fimpl_assemble<{w['k']}>": {'what': 'Step-I assembly (stage solves and the reconstruction f^impl): FP64; '
                                                'under HDG_MIXED the block (advection contraction, facet masses, '
                                                'entries) in double-FP32 pairs (flop: the FP64 part, df32_flop: '
                                                'the pair part)',
                                        'ms_per_launch': as_ms, 'launches_per_step': stages + 1, 'bytes': as_bytes,
                                        'flop': as_flop[0], 'df32_flop': as_flop[1], 'bound': 'alu'},
        (f"k_bdm_f2<{w['k']}>" if args.precision == 'MIXED' else f"k_bdm<{w['k']}>"): (
            {'what': 'BDM projection in double-FP32 pairs (stage advecting velocities and the reconstruction)',
             'ms_per_launch': bd_ms, 'launches_per_step': stages + 1, 'bytes': bd_bytes,
             'flop_fp64_equiv': bdm_flops(w['k'], ncells), 'bound': 'hbm'} if args.precision == 'MIXED' else
            {'what': 'FP64 BDM projection (stage advecting velocities and the reconstruction)',
             'ms_per_launch': bd_ms, 'launches_per_step': stages + 1, 'bytes': bd_bytes,
             'flop': bdm_flops(w['k'], ncells), 'bound': 'alu'})}
    if s32_ms is not None:
        kernels[f"k_stage_apply32<{w['k']}>"] = {'what': 'FP32 stage operator (relaxed FGMRES products)',
                                                 'ms_per_launch': s32_ms, 'launches_per_step': p32,
                                                 'bytes': s32_bytes, 'bound': 'hbm'}
    if gd_ms is not None:
        kernels[f"k_gs_diag<{w['k']}>"] = {'what': 'inner FP32 Step-I GMRES: red-black block Gauss-Seidel colour '
                                                   'pass (FP32 block inverses)', 'ms_per_launch': gd_ms,
                                           'launches_per_step': 2 * inner, 'bytes': gd_bytes, 'bound': 'hbm'}
        kernels[f"k_gs_apply<{w['k']}>"] = {'what': 'inner FP32 Step-I GMRES: Arnoldi product and dots',
                                            'ms_per_launch': ga_ms, 'launches_per_step': inner, 'bytes': ga_bytes,
                                            'bound': 'hbm'}
    for name, kd in kernels.items():
        kd['ms_per_step_est'] = kd['ms_per_launch'] * kd['launches_per_step']
        kd['share_of_step_est'] = kd['ms_per_step_est'] / float(np.mean(ms))
        kd['achieved_gbs'] = kd['bytes'] / (kd['ms_per_launch'] * 1e-3) / 1e9
        if kd['bound'] == 'hbm':
            kd['frac_of_hbm'] = kd['achieved_gbs'] / peak
        else:
            kd['achieved_tflops'] = kd['flop'] / (kd['ms_per_launch'] * 1e-3) / 1e12
            kd['frac_of_fp64_nominal'] = kd['achieved_tflops'] / FP64_NOMINAL_TFLOPS
    top = max(kernels, key=lambda n: kernels[n]['ms_per_step_est'])
    kt = kernels[top]
    # DRAM bytes per launch from a committed ncu summary of the same kernel: C2 captured at its own
    # size; C3's colour pass captured at 128x128 (the size rule for a full capture) and scaled by
    # the cell ratio (its traffic is proportional to the cells: one block inverse per cell)
    traffic_src = {('c2', 'k_stage_apply<3>'): ('k_stage_apply_fp64_c2.md', 1.0),
                   ('c2', 'k_stage_apply_f2<3>'): ('k_stage_apply_f2_pairs_c2.md', 1.0),
                   ('c2', 'k_gs_diag<3>'): ('k_gs_diag_fp32_c2.md', 1.0),
                   ('c3', 'k_gs_diag<4>'): ('k_gs_diag_fp32_tg128_k4.md', (w['n'] / 128.0) ** 2)}.get((args.workload, top))
    if kt['bound'] == 'alu':
        roofline = {'kernel': f"{top} ({kt['what']})", 'bound': 'alu', 'achieved': kt['achieved_tflops'],
                    'peak': FP64_NOMINAL_TFLOPS, 'unit': 'TFLOP/s', 'frac': kt['frac_of_fp64_nominal'],
                    'peak_kind': 'nominal FP64 vector rate (no measured FP64 peak exists for this pool)',
                    'algorithmic_flop': kt['flop']}
    else:
        roofline = {'kernel': f"{top} ({kt['what']})", 'bound': 'hbm', 'achieved': kt['achieved_gbs'], 'peak': peak,
                    'unit': 'GB/s', 'frac': kt['frac_of_hbm'], 'peak_kind': peak_kind}
    traffic = profile_traffic(traffic_src[0]) if traffic_src else None
    roofline.update({'traffic': traffic * traffic_src[1] if traffic is not None else None,
                     'ms_per_launch': kt['ms_per_launch'], 'algorithmic_bytes': kt['bytes'],
                     'launches_per_step': kt['launches_per_step'], 'share_of_step_est': kt['share_of_step_est'],
                     'note': 'the kernel with the largest estimated device time per step (time per launch alone x '
                             'launches per step from the solver counters)'})
    per_step = {'trace_solves': trace_solves / args.steps, 'trace_cg_iters': trace_iters / args.steps,
                'stage_outer_iters': sum(s['richardson_iters'] for s in stats_all) / args.steps,
                'stage_products_fp32': sum(s['stage_products32'] for s in stats_all) / args.steps,
                'gmres_iters': stepI_iters / args.steps}
    for key, name in (('ms_trace_solves', 'ms_trace'), ('ms_stepI_solves', 'ms_stepI'), ('ms_assembly', 'ms_assembly'),
                      ('ms_bdm', 'ms_bdm')):      # per-component device times exist only with host-driven loops
        per_step[key] = sum(s[name] for s in stats_all) / args.steps if host_loops else None
    cfg = {'workload': w['name'], 'n': w['n'], 'k': w['k'], 'periodic_x': w['periodic_x'], 'trace_dofs': ntrace,
           'dg_dofs': nQ + nP, 'precision': args.precision,
           'inner_rtol': [kw['inner_stepI_rtol'], kw['inner_trace_rtol']],
           'l2': 'flushed (256 MB write) between timed steps', 'parallelism': f'replicas x{world}',
           'loops': 'host' if host_loops else 'device (one CUDA graph per IMEX step)'}
    if gold is not None:
        cfg['error_vs_oracle'] = gold
    if w['init'] == 'taylor_green':                   # the exact solution exp(-kappa t) Q0 is known
        import hdg_workloads as W
        T = final[3]
        Qex = np.exp(-w['kappa'] * T) * W.nodal_velocity(w['n'], w['k'], W.taylor_green)
        pex = np.exp(-2 * w['kappa'] * T) * W.nodal_scalar(w['n'], w['k'], W.taylor_green_pressure)
        cfg['error_vs_exact'] = {'t': T, 'Q': rel_err(final[0], Qex), 'p': rel_err(final[1], pex)}
    line = {
        'metric': METRIC, 'value': value, 'unit': 'stage_solves/s', 'n_gpus': world, 'steps': args.steps,
        'warmup': args.warmup, 'ms_per_step': ms_step, 'higher_is_better': True, 'scaling': 'weak',
        'vs_baseline': None, 'dtype': 'f64',
        'data': 'synthetic (seeded shear layer + noise)' if w['init'] == 'shear_layer' else 'synthetic (analytic, forced)',
        'config': cfg,
        'trace_dof_per_s': world * ntrace * trace_solves / (total_ms / 1e3),
        'per_step': per_step,
        'e2e': {'value': world * stages / (e2e_mean / 1e3) if e2e_mean > 0 else None, 'unit': 'stage_solves/s',
                'h2d_bytes_per_step': h2d, 'd2h_bytes_per_step': h2d},
        'roofline': roofline,
        'kernels': kernels,
        'trace_apply': {'kernel': 'k_cg_apply', 'achieved_gbs': k_bytes / (k_ms * 1e-3) / 1e9, 'ms_per_launch': k_ms,
                        'bytes': k_bytes, 'frac_of_hbm': k_bytes / (k_ms * 1e-3) / 1e9 / peak, 'hbm_peak_kind': peak_kind},
        'condensation': {'kernel': f"k_condense<{w['k']}>", 'ms_per_launch': cd_ms,
                         'algorithmic_flop': condense_flops(w['k'], ncells), 'bytes': cd_bytes,
                         'achieved_tflops': condense_flops(w['k'], ncells) / (cd_ms * 1e-3) / 1e12,
                         'frac_of_fp64_nominal': condense_flops(w['k'], ncells) / (cd_ms * 1e-3) / 1e12 / FP64_NOMINAL_TFLOPS,
                         'achieved_gbs': cd_bytes / (cd_ms * 1e-3) / 1e9, 'frac_of_hbm': cd_bytes / (cd_ms * 1e-3) / 1e9 / peak,
                         'note': 'once per stage coefficient (setup); FP64, one block per cell, serial Cholesky'},
        'stage_apply_fp64': {'kernel': 'k_cell_apply_mf', 'achieved_gbs': s_bytes / (s_ms * 1e-3) / 1e9,
                             'achieved_tflops': s_flop / (s_ms * 1e-3) / 1e12, 'fp64_nominal_tflops': 1.25,
                             'ms_per_launch': s_ms, 'bytes': s_bytes, 'flop': s_flop},
        'clocks': clk.summary(),
        'gpu_launches': None,
    }
    if other is not None:
        line['compare_precision'] = other
    # kernels launched inside the timed steps: counted exactly by the library (graph kernel nodes
    # plus every pass of the device-side loops); with host-driven loops it is not counted (None)
    launches = sum(s['graph_kernels'] for s in stats_all)
    line['gpu_launches'] = int(launches) if launches > 0 else None
    if rank == 0 and not args.no_cpu_baseline and args.workload == 'c2':
        r, s_, desc, cores = oracle_sample(w)
        line['cpu_baseline'] = {'value': r, 'unit': 'stage_solves/s', 'cores': cores, 'kind': 'oracle', 'sample': desc}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=10)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='gpu', choices=['gpu', 'reference'])
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--e2e-steps', type=int, default=3)
    ap.add_argument('--workload', default='c2', choices=['c2', 'c3', 'c4', 'c5'],
                    help='c2: the shear channel (default); c3: forced Taylor-Green 256x256, k=4; '
                         'c4: batched instances; c5: served request stream')
    ap.add_argument('--instances', type=int, default=64, help='c4: number of instances')
    ap.add_argument('--requests', type=int, default=48, help='c5: number of requests')
    ap.add_argument('--max-active', type=int, default=64, help='c5: server slot limit')
    ap.add_argument('--precision', default='MIXED', choices=['MIXED', 'FP64'])
    ap.add_argument('--no-compare', action='store_true', help='skip the run in the other precision')
    ap.add_argument('--compare-steps', type=int, default=3, help='timed steps of the other precision')
    ap.add_argument('--n', type=int, default=None, help='mesh size override (profiling runs only)')
    ap.add_argument('--inner-trace-rtol', type=float, default=None, help='tuning: inner Step II tolerance')
    ap.add_argument('--inner-stepI-rtol', type=float, default=None, help='tuning: inner Step I tolerance')
    ap.add_argument('--inner-trace-vcycles', type=int, default=None,
                    help='tuning: Step II inside the preconditioner as n V-cycles (0: CG to the inner tolerance)')
    ap.add_argument('--inner-trace-fp32', type=int, default=None,
                    help='tuning: the one-V-cycle Step II inside the preconditioner in FP32 (1) or FP64 (0)')
    ap.add_argument('--trace-fp32-vcycle', type=int, default=None,
                    help='tuning: the tight trace CG preconditioned by the FP32 V-cycle (1) or the FP64 one (0)')
    ap.add_argument('--relax-eta', type=float, default=None,
                    help='tuning: relaxed FP32 stage-operator products once the FGMRES residual times this is '
                         'below the tolerance (0: all FP64; default: the library default)')
    ap.add_argument('--inner-gs', type=int, default=None,
                    help='tuning: inner Step-I preconditioner red-black block Gauss-Seidel (1) or block Jacobi (0)')
    ap.add_argument('--host-loops', action='store_true',
                    help='drive the Krylov loops from the host (fills the per-component timings)')
    ap.add_argument('--kernel-only', type=int, default=None,
                    help='profiling: set up the workload, take one step, then launch kernel K '
                         '(0 trace apply, 1 tentative-velocity apply) --steps times and exit')
    args = ap.parse_args()
    world = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local_rank = int(os.environ.get('LOCAL_RANK', '0'))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = 'nccl' if args.impl == 'gpu' else 'gloo'
        if args.impl == 'gpu':
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend)
    if args.impl == 'reference':
        run_reference(args, rank, world)
    elif args.workload == 'c4':
        run_batched(args, rank, world, local_rank)
    elif args.workload == 'c5':
        run_served(args, rank, world, local_rank)
    else:
        run_gpu(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == '__main__':
    main()
