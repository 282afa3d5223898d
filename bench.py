"""Benchmark: IMEX stage solves/s of the HDG incompressible-Euler stage solver on GB300.

Workload (the plain-FP64 GPU configuration): periodic-in-x channel [0,1]^2 with walls at
y = 0, 1, 64 x 64 rectangles -> 8192 triangles, k = 3 (velocity P4, pressure/trace P3),
ARS(3,4,3), dt = 2e-3; every stage solved to a relative stage residual of 1e-10 (flexible GMRES
preconditioned by Alg. 2's Chorin split; inside it Step I by one FP32 GMRES cycle to 2e-2 and
Step II by one trace multigrid V-cycle;
the paper's fixed n_R = 2 is unstable on this flow); final update and pressure reconstruction
trace CG rtol 1e-12; initial u = (tanh((y-1/2)/0.05), 1e-3 sin 2 pi x) + seeded N(0,1) 1e-4
noise per nodal value, projected to divergence-free. One bench step = one IMEX time step of
Alg. 1 (3 stage solves, final update, pressure reconstruction) through hdg_imex_step.

Output: one JSON line (rank 0). value = stage solves/s (whole job); trace_dof_per_s = trace
unknowns x trace solves / s. e2e: the same through the C-ABI with the state copied from pinned
host memory to the device and back every step. roofline: the kernel with the largest share of a
step, the fused FP64 stage-operator kernel (the flexible GMRES product), timed alone with CUDA
events on the context's stream; it is bound by GB300's FP64 pipe, so achieved = algorithmic
FP64 flops / time against the nominal FP64 rate. inner_stepI_fp32 (the two kernels of an inner
Arnoldi step, bytes / time vs the measured HBM peak), trace_apply and stage_apply_fp64 report
more kernels of the path the same way.
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

WORKLOAD = dict(n=64, k=3, periodic_x=True, tableau='ARS343', dt=2e-3, n_richardson=0, stage_rtol=1e-10,
                inner_stepI_rtol=2e-2, inner_trace_rtol=1e-1, trace_rtol=1e-12, stepI_rtol=1e-10,
                inner_trace_vcycles=1, inner_trace_fp32=1, trace_fp32_vcycle=1, inner_gs=1,
                init='shear_layer', width=0.05, amp=1e-3, noise=1e-4, seed=0)
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


def initial_velocity(w, n_override=None, seed_offset=0):
    import hdg_workloads as W
    n = n_override or w['n']
    return W.nodal_velocity(n, w['k'], lambda x, y: W.shear_layer(x, y, w['width'], w['amp']),
                            noise=w['noise'], seed=w['seed'] + seed_offset)


# ---------------------------------------------------------------------------------- oracle arm
def oracle_sample(w, n_sample=16, steps=1):
    """The oracle (as it stands) on a bounded sample of the workload: `steps` IMEX steps of the
    same configuration on an n_sample x n_sample mesh. Returns (stage solves/s scaled to the
    full mesh by the cell-count ratio, seconds, description, threads)."""
    os.environ.setdefault('OMP_NUM_THREADS', '1')
    os.environ.setdefault('OPENBLAS_NUM_THREADS', '1')
    from oracle import Mesh, HDG, Oracle, TABLEAUS
    m = Mesh(n_sample, periodic_x=w['periodic_x'])
    h = HDG(m, w['k'])
    o = Oracle(h)
    Q0 = initial_velocity(w, n_override=n_sample).reshape(-1)
    Q, _, _ = o.div_free_project(Q0)
    _, p, lam = o.reconstruct_pressure(Q)
    tab = TABLEAUS[w['tableau']]()
    t0 = time.perf_counter()
    for s in range(steps):
        Q, p, lam = o.imex_step(tab, w['dt'], s * w['dt'], Q, p, lam, solver='direct')
    sec = time.perf_counter() - t0
    stages = STAGES[w['tableau']] * steps
    scale = (n_sample / w['n']) ** 2
    rate = stages / sec * scale
    desc = (f'{steps} IMEX step(s) ({stages} stage solves by direct sparse LU of the monolithic stage system, '
            f'final update, reconstruction) of the same workload on a {n_sample}x{n_sample} mesh in {sec:.1f} s; '
            f'rate scaled by the cell ratio ({n_sample}/{w["n"]})^2 to the {w["n"]}x{w["n"]} mesh')
    return rate, sec, desc, int(os.environ.get('OMP_NUM_THREADS', '1'))


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = dict(WORKLOAD)
    for _ in range(args.warmup):
        oracle_sample(w, steps=1)
    rates, secs = [], []
    for _ in range(args.steps):
        r, s, desc, cores = oracle_sample(w, steps=1)
        rates.append(r)
        secs.append(s)
    value = len(rates) / sum(1.0 / r for r in rates)
    line = {'metric': METRIC, 'value': value, 'unit': 'stage_solves/s', 'impl': 'reference',
            'n_gpus': args.gpus, 'steps': args.steps, 'warmup': args.warmup,
            'ms_per_step': 1e3 * sum(secs) / len(secs), 'higher_is_better': True, 'scaling': 'weak',
            'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
            'config': {'workload': 'shear-layer channel 64x64, k=3, ARS(3,4,3), dt=2e-3, stages to 1e-10', 'n': w['n'],
                       'k': w['k'], 'periodic_x': True, 'sample_n': 16},
            'cpu_baseline': {'value': value, 'unit': 'stage_solves/s', 'cores': cores, 'kind': 'oracle',
                             'sample': desc},
            'e2e': {'value': value, 'unit': 'stage_solves/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_2410_09790_gb300 as H

    torch.cuda.set_device(local_rank)
    dev = torch.device('cuda', local_rank)
    w = dict(WORKLOAD)
    if args.n:
        w['n'] = args.n
    if args.inner_trace_rtol:
        w['inner_trace_rtol'] = args.inner_trace_rtol
    if args.inner_stepI_rtol:
        w['inner_stepI_rtol'] = args.inner_stepI_rtol
    if args.inner_trace_vcycles is not None:
        w['inner_trace_vcycles'] = args.inner_trace_vcycles
    if args.inner_trace_fp32 is not None:
        w['inner_trace_fp32'] = args.inner_trace_fp32
    if args.trace_fp32_vcycle is not None:
        w['trace_fp32_vcycle'] = args.trace_fp32_vcycle
    if args.inner_gs is not None:
        w['inner_gs'] = args.inner_gs
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        ctx = H.Context(w['n'], w['k'], periodic_x=w['periodic_x'], stream=stream, tableau=w['tableau'],
                        dt=w['dt'], n_richardson=w['n_richardson'], richardson_rtol=w['stage_rtol'],
                        richardson_max=600, stage_krylov=1, inner_stepI_rtol=w['inner_stepI_rtol'],
                        inner_trace_rtol=w['inner_trace_rtol'], trace_rtol=w['trace_rtol'],
                        stepI_rtol=w['stepI_rtol'], device_loops=0 if args.host_loops else 1,
                        inner_trace_vcycles=w['inner_trace_vcycles'], inner_trace_fp32=w['inner_trace_fp32'],
                        trace_fp32_vcycle=w['trace_fp32_vcycle'], inner_gs=w['inner_gs'])
        Q0 = torch.from_numpy(initial_velocity(w, seed_offset=rank)).to(dev)
        ctx.hdg_set_state(Q0)
        ctx.hdg_div_free_project()
        if args.kernel_only is not None:
            ctx.hdg_imex_step(1)
            gamma = 0.43586652150845899942
            ms_k, b_k = ctx.hdg_time_kernel(args.kernel_only, gamma * w['dt'], args.steps)
            print(json.dumps({'kernel': args.kernel_only, 'ms_per_launch': ms_k, 'bytes': b_k}), flush=True)
            ctx.close()
            return
        flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dev)   # > L2 (129 MB)
        stats_all = []
        for _ in range(args.warmup):
            ctx.hdg_imex_step(1)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with ClockSampler(local_rank) as clk:
            for i in range(args.steps):
                flush.fill_(float(i))                      # evict the previous step's working set
                torch.cuda.nvtx.range_push('bench_step')
                ev[i][0].record(stream)
                st = ctx.hdg_imex_step(1)
                ev[i][1].record(stream)
                torch.cuda.nvtx.range_pop()
                stats_all.append(st)
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        # kernels timed alone on the same operators and stream (roofline and two diagnostics)
        gamma = 0.43586652150845899942                   # ARS(3,4,3) diagonal
        c_stage = gamma * w['dt']
        k_ms, k_bytes = ctx.hdg_time_kernel(0, c_stage, 50)
        s_ms, s_bytes = ctx.hdg_time_kernel(1, 1.0, 20)
        a_ms, a_bytes = ctx.hdg_time_kernel(6, c_stage, 50)
        p_ms, p_bytes = ctx.hdg_time_kernel(9, c_stage, 50)
        st_ms, st_bytes = ctx.hdg_time_kernel(8, c_stage, 20)
        # end to end through the C-ABI with host buffers
        Qh, ph, lh, _ = ctx.hdg_get_state()
        Qh, ph, lh = Qh.cpu().pin_memory(), ph.cpu().pin_memory(), lh.cpu().pin_memory()
        Qd, pd, ld = torch.empty_like(Qh, device=dev), torch.empty_like(ph, device=dev), torch.empty_like(lh, device=dev)
        e2e_ms = []
        tsim = w['dt'] * (args.warmup + args.steps)
        for i in range(args.e2e_steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Qd.copy_(Qh, non_blocking=True); pd.copy_(ph, non_blocking=True); ld.copy_(lh, non_blocking=True)
            ctx.hdg_set_state(Qd, pd, ld, tsim)
            ctx.hdg_imex_step(1)
            Qo, po, lo, tsim = ctx.hdg_get_state()
            Qh.copy_(Qo); ph.copy_(po); lh.copy_(lo)
            torch.cuda.synchronize()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        h2d = (Qh.numel() + ph.numel() + lh.numel()) * 8
        ctx.close()

    stages = STAGES[w['tableau']]
    ms_step = float(np.mean(ms))
    total_ms, e2e_mean = aggregate_ranks(sum(ms), float(np.mean(e2e_ms)) if e2e_ms else float('nan'), world, dev)
    value = job_rate(world, stages, args.steps, total_ms)
    ntrace = ctx.nL
    trace_solves = sum(s['trace_solves'] for s in stats_all)
    trace_iters = sum(s['trace_iters'] for s in stats_all)
    stepI_iters = sum(s['stepI_iters'] for s in stats_all)
    peak, peak_kind = measured_peaks()
    # FP64 velocity-block apply: FMAs per cell = dense diagonal block + neighbour evaluation +
    # flux + test (interior edges; k = w['k'])
    mu = (w['k'] + 2) * (w['k'] + 3) // 2
    nu, nfq = 2 * mu, (3 * w['k'] + 5) // 2
    npk, nt = (w['k'] + 1) * (w['k'] + 2) // 2, w['k'] + 1
    ncells = ctx.nQ // nu
    s_flop = 2.0 * (nu * nu + 3 * nfq * 2 * mu + 3 * nfq * 8 + nu * 3 * nfq) * ncells
    # the fused stage operator: the velocity block above + the trace and pressure coupling of the
    # velocity rows + the cell's constraint rows (pressure rows, trace rows)
    st_flop = s_flop + ncells * (nu * (3 * (2 * nt + 3) + 2 * (2 * npk + 2) + 3) + 6 * mu +
                                 npk * (4 * mu + 3 * (2 * npk + 2) + 3 * (2 * nt + 2) + 5) +
                                 3 * nt * (5 * mu + 2 * npk + 5))
    st_tflops = st_flop / (st_ms * 1e-3) / 1e12
    line = {
        'metric': METRIC, 'value': value, 'unit': 'stage_solves/s', 'n_gpus': world, 'steps': args.steps,
        'warmup': args.warmup, 'ms_per_step': ms_step, 'higher_is_better': True, 'scaling': 'weak',
        'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic (seeded shear layer + noise)',
        'config': {'workload': 'shear-layer channel 64x64, k=3, ARS(3,4,3), dt=2e-3, stages to 1e-10', 'n': w['n'],
                   'k': w['k'], 'periodic_x': True, 'trace_dofs': ntrace, 'dg_dofs': ctx.nQ + ctx.nP,
                   'inner_rtol': [w['inner_stepI_rtol'], w['inner_trace_rtol']],
                   'inner_step2': f"{w['inner_trace_vcycles']} V-cycle(s), {'FP32' if w['inner_trace_fp32'] else 'FP64'}",
                   'l2': 'flushed (256 MB write) between timed steps', 'parallelism': f'replicas x{world}'},
        'trace_dof_per_s': world * ntrace * trace_solves / (total_ms / 1e3),
        'per_step': {'ms_trace_solves': sum(s['ms_trace'] for s in stats_all) / args.steps,
                     'ms_stepI_solves': sum(s['ms_stepI'] for s in stats_all) / args.steps,
                     'ms_assembly': sum(s['ms_assembly'] for s in stats_all) / args.steps,
                     'ms_bdm': sum(s['ms_bdm'] for s in stats_all) / args.steps,
                     'trace_solves': trace_solves / args.steps, 'trace_cg_iters': trace_iters / args.steps,
                     'stage_outer_iters': sum(s['richardson_iters'] for s in stats_all) / args.steps,
                     'gmres_iters': stepI_iters / args.steps},
        'e2e': {'value': world * stages / (e2e_mean / 1e3), 'unit': 'stage_solves/s', 'h2d_bytes_per_step': h2d,
                'd2h_bytes_per_step': h2d},
        'roofline': {'kernel': 'k_stage_apply<3> (fused FP64 stage operator, the flexible GMRES product)',
                     'bound': 'alu', 'achieved': st_tflops, 'peak': FP64_NOMINAL_TFLOPS, 'unit': 'TFLOP/s',
                     'frac': st_tflops / FP64_NOMINAL_TFLOPS,
                     'peak_kind': 'nominal FP64 vector rate (no measured FP64 peak exists for this pool)',
                     'traffic': profile_traffic('k_stage_apply_fp64_c2.md'), 'ms_per_launch': st_ms,
                     'algorithmic_flop': st_flop, 'algorithmic_bytes': st_bytes,
                     'achieved_gbs': st_bytes / (st_ms * 1e-3) / 1e9},
        'inner_stepI_fp32': {
            'apply': {'kernel': 'k_gm_apply_mf<3, float, 1> (Arnoldi product, step j = 4)', 'ms_per_launch': a_ms,
                      'bytes': a_bytes, 'achieved_gbs': a_bytes / (a_ms * 1e-3) / 1e9,
                      'frac_of_hbm': a_bytes / (a_ms * 1e-3) / 1e9 / peak,
                      'traffic': profile_traffic('k_gm_apply_mf_fp32_c2.md')},
            'precond': {'kernel': 'k_gm_precond_mf<3, float, 1> (block inverse pass, step j = 4)',
                        'ms_per_launch': p_ms, 'bytes': p_bytes, 'achieved_gbs': p_bytes / (p_ms * 1e-3) / 1e9,
                        'frac_of_hbm': p_bytes / (p_ms * 1e-3) / 1e9 / peak, 'hbm_peak_kind': peak_kind}},
        'trace_apply': {'kernel': 'k_cg_apply', 'achieved_gbs': k_bytes / (k_ms * 1e-3) / 1e9, 'ms_per_launch': k_ms,
                        'bytes': k_bytes},
        'stage_apply_fp64': {'kernel': 'k_cell_apply_mf', 'achieved_gbs': s_bytes / (s_ms * 1e-3) / 1e9,
                             'achieved_tflops': s_flop / (s_ms * 1e-3) / 1e12, 'fp64_nominal_tflops': 1.25,
                             'ms_per_launch': s_ms, 'bytes': s_bytes, 'flop': s_flop},
        'clocks': clk.summary(),
        'gpu_launches': None,
    }
    # kernels launched inside the timed steps: counted exactly by the library (graph kernel nodes
    # plus every pass of the device-side loops); with host-driven loops it is not counted (None)
    launches = sum(s['graph_kernels'] for s in stats_all)
    line['gpu_launches'] = int(launches) if launches > 0 else None
    line['config']['loops'] = 'host' if args.host_loops else 'device (one CUDA graph per IMEX step)'
    if rank == 0 and not args.no_cpu_baseline:
        r, s, desc, cores = oracle_sample(w, steps=1)
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
    ap.add_argument('--n', type=int, default=None, help='mesh size override (profiling runs only)')
    ap.add_argument('--inner-trace-rtol', type=float, default=None, help='tuning: inner Step II tolerance')
    ap.add_argument('--inner-stepI-rtol', type=float, default=None, help='tuning: inner Step I tolerance')
    ap.add_argument('--inner-trace-vcycles', type=int, default=None,
                    help='tuning: Step II inside the preconditioner as n V-cycles (0: CG to the inner tolerance)')
    ap.add_argument('--inner-trace-fp32', type=int, default=None,
                    help='tuning: the one-V-cycle Step II inside the preconditioner in FP32 (1) or FP64 (0)')
    ap.add_argument('--trace-fp32-vcycle', type=int, default=None,
                    help='tuning: the tight trace CG preconditioned by the FP32 V-cycle (1) or the FP64 one (0)')
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
    else:
        run_gpu(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == '__main__':
    main()
