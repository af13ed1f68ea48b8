"""Benchmark: explicit-step DOF-updates/s of the PW-tested heat step (Galerkin
comparator alongside), on the 3D workload 'heat3d': cubic C2 B-splines on
128^3 elements (131^3 = 2,248,091 coefficients), 4x4x4 Gauss points,
dt = 0.05 h^2, 50 explicit Euler steps per bench step, FP32 pairs (double-float
arithmetic) with one refinement per solve (FP64 banded factors; residual in
double-float, or FP64 with --residual fp64).

One bench step = one full 50-step run from the seeded initial state (reset
untimed before every step).  L2 (129 MB) is flushed before every timed step
by writing a 512 MB buffer.  Device time: CUDA events on the context stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun, one rank per GPU) every rank runs its own replica (the
path has no exchange step across instances: weak scaling, no collective on the
data path); the time is the max over ranks.  --impl reference times the FP64
CPU oracle on the same workload (bounded sample per step).

The line leads with the headline, the HBM roofline of one explicit step (16
bytes per coefficient and step: read u, write u', FP32 pairs) and the step
kernels in use; `rows` (keyed by the hot-path rows) follow: a4 the Table 1
source RHS (PW vs B-spline tests), a3 operator action and a6 refined
Kronecker solve (heat3d), a7 the heat2d workload and the size ladder past
L2 (3D and 2D, PW and Galerkin), a8 the error of every output against the
FP64 oracle (rel-L2, max-abs, max-abs relative to the largest entry; heat
states after steps 1, 10 and the last), f1 the 2D Poisson solve, f2 the
512-instance batched Poisson solve; then `serving`, the 2000-request mixed
stream (--no-serve skips it; --no-ladder skips the size ladder).
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = 'heat3d'
METRIC = 'explicit-step DOF-updates/s PW-const vs Galerkin (% HBM peak); served p50/p99 latency'


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=20)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='native', choices=['native', 'reference'])
    ap.add_argument('--residual', default='df', choices=['fp64', 'df'])
    ap.add_argument('--no-serve', action='store_true', help='skip the request-stream measurement')
    ap.add_argument('--no-ladder', action='store_true', help='skip the size ladder')
    return ap.parse_args()


def dist_setup(n):
    """(rank, world) from the torchrun environment; initialises a process
    group when world > 1 (NCCL with GPUs, gloo otherwise)."""
    rank = int(os.environ.get('RANK', '0'))
    world = int(os.environ.get('WORLD_SIZE', '1'))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = 'nccl' if torch.cuda.is_available() else 'gloo'
        if backend == 'nccl':
            torch.cuda.set_device(int(os.environ.get('LOCAL_RANK', '0')))
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Max of a float over all ranks (timing only; no data-path collective)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = 'cuda' if dist.get_backend() == 'nccl' else 'cpu'
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ('clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,'
         'clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,'
         'clocks_event_reasons.sw_power_cap')

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        import threading
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ['nvidia-smi', '-i', str(self.index), f'--query-gpu={self.Q}', '--format=csv,noheader,nounits',
                 '-lms', '20'], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self

        def reader():
            for l in self.proc.stdout:
                if l.strip():
                    self.lines.append(l)

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        # the timed region starts once the sampler is producing samples
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.skip = len(self.lines)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)
            self.lines = self.lines[max(self.skip - 1, 0):]

    def summary(self):
        import statistics
        sm, mx, reasons = [], [], set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for l in getattr(self, 'lines', []):
            f = [x.strip() for x in l.split(',')]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[3:7]):
                if v.lower().startswith('active'):
                    reasons.add(name)
        return {'sm_mhz': statistics.median(sm) if sm else None, 'sm_max_mhz': max(mx) if mx else None,
                'reasons': sorted(reasons), 'samples': len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, 'MEASURED_PEAKS.json')))
    except OSError:
        return {}


def peak_sources(pk):
    """Where each roofline denominator comes from: the machine's measured copy
    rate and maximum SM clock (MEASURED_PEAKS.json), else the fallbacks."""
    return {'hbm_gbs': pk.get('hbm_gbs', 6800.0),
            'hbm_source': 'measured' if 'hbm_gbs' in pk else 'fallback (6.8 TB/s)',
            'sm_max_mhz': pk.get('sm_max_mhz', 2070.0),
            'clock_source': 'measured' if 'sm_max_mhz' in pk else 'nominal (2070 MHz)'}


def rnd(x, sig=4):
    """Rounds floats (recursively) to `sig` significant digits for a compact line."""
    import math
    if isinstance(x, float):
        if x == 0.0 or not math.isfinite(x):
            return x
        return float(f'{x:.{sig}g}')
    if isinstance(x, dict):
        return {k: rnd(v, sig) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [rnd(v, sig) for v in x]
    return x


def errors(got, ref):
    """rel-L2, max-abs and max-abs relative to the largest reference entry."""
    import numpy as np
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.abs(got - ref)
    return {'rel_l2': float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)),
            'max_abs': float(d.max()), 'max_abs_rel': float(d.max() / max(np.abs(ref).max(), 1e-300))}


def oracle_heat(name, test, snaps, seed=0):
    """FP64 oracle run of a heat workload: the states after the steps listed
    in `snaps` (ascending), and the CPU seconds it took."""
    from oracle import systems, tensor
    from paper_1910_08535_gb300 import workloads
    w = workloads.WORKLOADS[name]
    axes = [systems.Axis(w['n_elem'], w['degree'], w['nq'], test) for _ in range(w['dim'])]
    M, L = tensor.mass_mats(axes), tensor.lap_mats(axes)
    u = workloads.initial_state(name, seed=seed)
    dt = workloads.dt_of(name)
    out = {}
    t0 = time.perf_counter()
    for s in range(1, max(snaps) + 1):
        u = tensor.ads_solve(M, tensor.apply_heat_system(axes, u, dt, M, L))
        if s in snaps:
            out[s] = u.copy()
    return out, time.perf_counter() - t0


def cpu_baseline_oracle(test='pw', steps=20):
    """The FP64 oracle on the same workload: `steps` explicit steps at full size."""
    import numpy as np  # noqa: F401
    from oracle import systems, tensor
    from paper_1910_08535_gb300 import workloads
    w = workloads.WORKLOADS[WORKLOAD]
    axes = [systems.Axis(w['n_elem'], w['degree'], w['nq'], test) for _ in range(3)]
    M, L = tensor.mass_mats(axes), tensor.lap_mats(axes)
    u = workloads.initial_state(WORKLOAD)
    dt = workloads.dt_of(WORKLOAD)
    t0 = time.perf_counter()
    for _ in range(steps):
        u = tensor.ads_solve(M, tensor.apply_heat_system(axes, u, dt, M, L))
    el = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get('num_threads', 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    return {'value': u.size * steps / el, 'unit': 'DOF-updates/s', 'cores': cores, 'kind': 'oracle',
            'sample': f'{steps} of the 50 explicit steps of heat3d at full size (131^3), FP64 numpy, PW tests',
            'seconds': el}


def run_reference(args, rank, world):
    if rank != 0:
        return
    samples = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline_oracle(steps=2)
        if i >= args.warmup:
            samples.append(r)
    val = sum(s['value'] for s in samples) / len(samples)
    sec = sum(s['seconds'] for s in samples) / len(samples)
    line = {'impl': 'reference', 'metric': METRIC, 'value': val, 'unit': 'DOF-updates/s', 'n_gpus': world,
            'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': sec * 1e3, 'higher_is_better': True,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic (seeded)',
            'config': {'workload': 'heat3d: 3D heat, p=3, 128^3 elements, 4^3 Gauss, 2 of 50 steps per bench step',
                       'test': 'pw'},
            'cpu_baseline': {'value': val, 'unit': 'DOF-updates/s', 'cores': samples[0]['cores'], 'kind': 'oracle',
                             'sample': '2 explicit steps of heat3d at full size (131^3) per bench step'},
            'e2e': {'value': val, 'unit': 'DOF-updates/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}
    print(json.dumps(line))


def _time_events(stream, fn, reps, flush=None, warm=3):
    """Average device time of fn() over reps calls (CUDA events on `stream`,
    L2 flushed before each call when a flush buffer is given)."""
    import torch
    out = []
    with torch.cuda.stream(stream):
        for i in range(warm + reps):
            if flush is not None:
                flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if i >= warm:
                out.append(e0.elapsed_time(e1) / 1e3)
    return sum(out) / len(out)


def source_sha(files):
    """Short hash of library sources (ties a stored ncu figure to the code it measured)."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), 'rb') as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


STEP_SOURCES = ('paper_1910_08535_gb300/csrc/chunkstep.cuh', 'paper_1910_08535_gb300/csrc/chunkstep_p3.cu',
                'paper_1910_08535_gb300/csrc/common.cuh')
TRAFFIC_PROFILE = 'profiles/chunk_step_kernel_heat3d.md'


def profiled_traffic():
    """DRAM bytes of one explicit step (three chunk_step_kernel launches) from
    the ncu summary under profiles/ (a line `traffic_bytes_per_step: B
    source_sha: S`), or None if there is none or the step kernel's sources
    changed since it was taken."""
    try:
        txt = open(os.path.join(ROOT, TRAFFIC_PROFILE)).read()
    except OSError:
        return None, 'no ncu summary'
    import re
    m = re.search(r'traffic_bytes_per_step:\s*([0-9.eE+]+)\s+source_sha:\s*([0-9a-f]+)', txt)
    if not m:
        return None, 'no traffic line in the ncu summary'
    if m.group(2) != source_sha(STEP_SOURCES):
        return None, 'step kernel changed since the ncu capture'
    return float(m.group(1)), TRAFFIC_PROFILE


def measure_rows(ctx, u, dt, stream, flush, hbm_peak):
    """Rows a3 (operator action) and a6 (refined Kronecker solve) on heat3d:
    device time per call, the algorithmic HBM fraction (read u, write r: 16
    bytes per coefficient), and the error of each output against the oracle
    (same input, timed on the host cores)."""
    from oracle import systems, tensor
    from paper_1910_08535_gb300 import workloads
    n = ctx.ntot
    r = ctx.empty()
    out = ctx.empty()
    t_apply = _time_events(stream, lambda: ctx.apply('heat', u, dt, out=r), 10, flush)
    t_solve = _time_events(stream, lambda: ctx.solve(r, out=out), 10, flush)
    ctx.sync()
    uin, rr, ss = ctx.to_numpy(u), ctx.to_numpy(r), ctx.to_numpy(out)
    w = workloads.WORKLOADS[WORKLOAD]
    axes = [systems.Axis(w['n_elem'], w['degree'], w['nq'], 'pw') for _ in range(3)]
    M, L = tensor.mass_mats(axes), tensor.lap_mats(axes)
    t0 = time.perf_counter()
    ref_r = tensor.apply_heat_system(axes, uin, dt, M, L)
    t1 = time.perf_counter()
    ref_s = tensor.ads_solve(M, rr)
    t2 = time.perf_counter()
    return {
        'a3_apply_heat': {'us': t_apply * 1e6, 'dof_per_s': n / t_apply,
                          'hbm_frac_16B_per_dof': 16.0 * n / t_apply / 1e9 / hbm_peak,
                          'kernel': 'contract_kernel (7 double-float banded passes)',
                          'vs_oracle': errors(rr, ref_r), 'oracle_cpu_s': t1 - t0},
        'a6_solve_refined': {'us': t_solve * 1e6, 'dof_per_s': n / t_solve,
                             'kernels': '3 FP32 line solves + double-float residual + 3 line solves',
                             'vs_oracle': errors(ss, ref_s), 'oracle_cpu_s': t2 - t1},
    }


def measure_source_table1(stream, flush, hbm_peak, reps=5):
    """Row a4 on the paper's Table 1 experiment (Sec. 4.1): 3D L2-projection
    RHS for a tensor-product cubic polynomial, quadratic C1 splines, 128^3
    elements; B-spline tests with 3 Gauss points per element, PW tests with 2
    (the cubic integrand on each cell needs only 2).  f is sampled at each
    rule's points (FP32), the RHS accumulates in double-float."""
    import numpy as np
    import torch
    from oracle import systems, tensor
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    ne, p = 128, 2
    cub = [lambda x: 2 * x ** 3 - x ** 2 + 0.5 * x + 1, lambda x: x ** 3 + 0.3 * x + 0.2,
           lambda x: -x ** 3 + 2 * x ** 2 + 1]
    res = {}
    for test, nq in (('pw', 2), ('galerkin', 3)):
        with torch.cuda.stream(stream):
            c = Context(dim=3, n_elem=ne, degree=p, nq=nq, test=test, precision='fp32r', op='mass', stream=stream)
            pts = [c.quad_points(a)[0] for a in range(3)]
            f = torch.from_numpy(workloads.tensor_samples(pts, [tuple(cub)]).astype(np.float32)).cuda()
            b = c.empty()
            t = _time_events(stream, lambda: c.rhs_source(f, out=b), reps, flush)
            c.sync()
        q = [len(x) for x in pts]
        alg = 4 * q[0] * q[1] * q[2] + 8 * c.ntot
        axes = [systems.Axis(ne, p, nq, test) for _ in range(3)]
        t0 = time.perf_counter()
        ref = tensor.rhs_source(axes, f.cpu().numpy().astype(np.float64))
        tcpu = time.perf_counter() - t0
        res[test] = {'us': t * 1e6, 'hbm_frac': alg / t / 1e9 / hbm_peak, 'achieved_gbs': alg / t / 1e9,
                     'nq': nq, 'points': q[0] * q[1] * q[2], 'dof_per_s': c.ntot / t, 'alg_bytes': alg,
                     'vs_oracle': errors(c.to_numpy(b), ref), 'oracle_cpu_s': tcpu}
        c.close()
        del f, b
    res['pw_speedup_over_galerkin'] = res['galerkin']['us'] / res['pw']['us']
    return res


def measure_heat(name, test, stream, flush, steps_timed, reps=3):
    """A heat workload on the device: DOF-updates/s over full runs (L2
    flushed before each), and the states after steps 1, 10 and the last,
    each against the FP64 oracle."""
    import torch
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    w = workloads.WORKLOADS[name]
    dt = workloads.dt_of(name)
    u0 = workloads.initial_state(name)
    with torch.cuda.stream(stream):
        c = Context(dim=w['dim'], n_elem=w['n_elem'], degree=w['degree'], nq=w['nq'], test=test,
                    precision='fp32r', stream=stream)
        init = c.from_numpy(u0)
        u = c.empty()

        def run():
            u.copy_(init)
            c.step(u, dt, steps_timed)
        t = _time_events(stream, run, reps, flush, warm=2)
        snaps = sorted({1, 10, w['steps']})
        u.copy_(init)
        got, done = {}, 0
        for s in snaps:
            c.step(u, dt, s - done)
            done = s
            c.sync()
            got[s] = c.to_numpy(u)
        shapes = [c.get_step_shape(a) for a in range(w['dim'])]
        c.close()
    ref, tcpu = oracle_heat(name, test, snaps)
    return {'dof_updates_per_s': (init.numel() // 2) * steps_timed / t, 'run_us': t * 1e6, 'steps': steps_timed,
            'step_kernels': [f'{k}/{nl}' for k, nl in shapes],
            'vs_oracle': {f'step_{s}': errors(got[s], ref[s]) for s in snaps}, 'oracle_cpu_s': tcpu}


LADDER_3D = ((128, 3), (192, 3), (256, 2), (256, 3), (256, 4), (384, 3), (512, 2), (512, 3))
LADDER_2D = ((1024, 3), (2048, 3), (4096, 3), (8192, 3))


def measure_ladder(stream, flush, hbm_peak, reps=5):
    """Size ladder of the explicit step (the a7 row past L2): one step of the
    3D and 2D heat problem (FP32 pairs, 1e-2 N(0,1) coefficients, dt = 0.05
    h^2), PW and Galerkin tests on the same grids, L2 flushed before each
    step.  Reports DOF-updates/s, the step's algorithmic HBM rate (read u,
    write u': 16 bytes per coefficient) and the PW / Galerkin ratio."""
    import torch
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    out = []
    for dim, sizes in ((3, LADDER_3D), (2, LADDER_2D)):
        for ne, p in sizes:
            row = {'dim': dim, 'n_elem': ne, 'degree': p}
            for test in ('pw', 'galerkin'):
                c = None
                try:
                    with torch.cuda.stream(stream):
                        c = Context(dim=dim, n_elem=ne, degree=p, nq=p + 1, test=test, precision='fp32r',
                                    stream=stream)
                        u = c.from_numpy(workloads.normal_coeffs(c.shape, seed=ne))
                        dt = 0.05 / ne ** 2
                        t = _time_events(stream, lambda: c.step(u, dt, 1), reps, flush)
                        c.sync()
                        shapes = [c.get_step_shape(a) for a in range(dim)]
                    row['dof'] = c.ntot
                    row[test] = {'step_us': t * 1e6, 'dof_updates_per_s': c.ntot / t,
                                 'alg_hbm_frac': 16 * c.ntot / t / 1e9 / hbm_peak,
                                 'kernels': '/'.join(f'{k}{nl}' for k, nl in shapes)}
                except Exception as ex:      # a grid no step kernel takes (lines too long)
                    row[test] = {'error': str(ex)[:160]}
                finally:
                    if c is not None:
                        c.close()
                    u = None
                    torch.cuda.empty_cache()
            if 'dof_updates_per_s' in row['pw'] and 'dof_updates_per_s' in row['galerkin']:
                row['pw_over_galerkin'] = row['pw']['dof_updates_per_s'] / row['galerkin']['dof_updates_per_s']
            out.append(row)
    return out


def measure_poisson(stream, flush, reps=10):
    """Row f1 (multi-D Poisson, Sec. 4.3 problem): 2D, 1024^2 elements, cubic
    PW tests, solve K u = b by fast diagonalisation (dense transforms per
    axis) inside iterative refinement; FP32 pairs (1 correction) and FP64 (3
    corrections); transforms on the library's tcgen05 split-TF32 kernel (the
    default), on cuBLAS FP32 GEMMs and on cuBLAS BF16x9 emulation.  The GEMM
    work of one transform application is 2 x sum_a 2 n_a N flops (W's then
    V's; N coefficients; counted once per FP32 product)."""
    import numpy as np
    import torch
    from paper_1910_08535_gb300 import igapw, workloads
    from paper_1910_08535_gb300.igapw import Context
    ne, p = 1024, 3
    res = {}
    for prec in ('fp32r', 'fp64'):
        for tag, flags in (('tc_split_tf32', 0), ('cublas_fp32', igapw.IGAPW_FLAG_FDM_CUBLAS),
                           ('cublas_bf16x9', igapw.IGAPW_FLAG_FDM_BF16X9)):
            with torch.cuda.stream(stream):
                t_create = time.perf_counter()
                c = Context(dim=2, n_elem=ne, degree=p, nq=p + 1, test='pw', precision=prec, op='poisson',
                            bc='dirichlet0', flags=flags, stream=stream)
                t_create = time.perf_counter() - t_create
                pts = [c.quad_points(a)[0] for a in range(2)]
                f = workloads.sine_product_source(pts, (1, 2))
                fd = torch.from_numpy(f.astype(np.float64 if prec == 'fp64' else np.float32)).cuda()
                b = c.rhs_source(fd)
                u = c.empty()
                t = _time_events(stream, lambda: c.solve(b, out=u), reps, flush)
                c.sync()
            applications = 2 if prec == 'fp32r' else 4
            flops = applications * 2 * sum(2 * c.n[a] * c.ntot for a in range(2))
            res[f'{prec}_{tag}'] = {'us': t * 1e6, 'dof_per_s': c.ntot / t, 'gemm_tflops': flops / t / 1e12,
                                    'fdm_applications': applications, 'create_s': t_create,
                                    'solution': c.to_numpy(u), 'rhs': c.to_numpy(b)}
            c.close()
    # the solution against the oracle's sparse direct solve on a 256^2 sample
    from oracle import poisson_nd, systems
    small = {}
    for prec in ('fp32r', 'fp64'):
        c = Context(dim=2, n_elem=256, degree=p, nq=p + 1, test='pw', precision=prec, op='poisson', bc='dirichlet0')
        bh = np.random.default_rng(0).standard_normal(c.shape)
        got = c.to_numpy(c.solve(c.from_numpy(bh)))
        c.sync()
        c.close()
        axes = [systems.Axis(256, p, p + 1, 'pw', 'dirichlet0') for _ in range(2)]
        t0 = time.perf_counter()
        ref = poisson_nd.solve(axes, bh, sparse=True)
        small[prec] = dict(errors(got, ref), oracle_sparse_direct_s=time.perf_counter() - t0)
    res['sample_256x256_vs_oracle'] = small
    return res


def measure_serving(requests=2000, seed=6, budget=120 * 10 ** 9):
    """Mixed request stream (Poisson solves and 20-step heat runs, 70% 2D
    64^2..1024^2 / 30% 3D 32^3..160^3, p in {2,3}, FP64 / FP32 pairs) through
    the continuous-batching server: slots for every shape created first
    (resident tables, factors and pencils), capacity from a closed-loop run of
    600 requests of the same mix, then `requests` Poisson arrivals at 80% of
    that capacity.
    A sample of the served results is checked against the oracle."""
    import numpy as np
    import torch
    from oracle import heat, poisson_nd, systems
    from paper_1910_08535_gb300 import serve
    torch.cuda.empty_cache()        # the rows before leave cached blocks of other sizes
    srv = serve.Server(budget_bytes=budget)
    stream = serve.make_stream(requests, rate=1.0, seed=seed)
    # capacity: closed loop (all at t = 0) over 600 requests drawn from the
    # stream's own distribution (same seed), so that it measures that mix
    probe = serve.make_stream(600, rate=None, seed=seed)
    t0 = time.perf_counter()
    srv.warm(sorted({r.shape for r in stream + probe}, key=str))
    torch.cuda.synchronize()
    t_warm = time.perf_counter() - t0
    recs, _ = srv.run(probe)
    srv.check()
    cap = serve.summarize(recs)['throughput_req_s']
    rate = 0.8 * cap
    stream = serve.make_stream(requests, rate=rate, seed=seed)
    recs, results = srv.run(stream, keep_results=True)
    srv.check()
    out = serve.summarize(recs)
    # precision of served results: the smallest requests of each kind and precision
    worst = {}
    byid = {r.rid: r for r in stream}
    for kind in ('heat', 'poisson'):
        for prec in ('fp32r', 'fp64'):
            cand = sorted((r for r in stream if r.shape.kind == kind and r.shape.precision == prec),
                          key=lambda r: r.shape.ntot)[:3]
            errs = []
            for r in cand:
                sh = r.shape
                axes = [systems.Axis(sh.n_elem, sh.degree, sh.nq, sh.test,
                                     'dirichlet0' if kind == 'poisson' else 'none') for _ in range(sh.dim)]
                if kind == 'heat':
                    ref = heat.run(axes, serve.base_state(sh), r.dt_h2 / (sh.n_elem ** 2 * sh.dim), r.steps)
                else:
                    from paper_1910_08535_gb300 import workloads
                    pts = [axes[a].points()[0] for a in range(sh.dim)]
                    f = workloads.sine_product_source(pts, r.k)
                    from oracle import tensor
                    ref = poisson_nd.solve(axes, tensor.rhs_source(axes, f), sparse=True)
                errs.append(errors(results[byid[r.rid].rid], ref))
            if errs:
                worst[f'{kind}_{prec}'] = {k: max(e[k] for e in errs) for k in errs[0]}
    out.update({'capacity_req_s': cap, 'arrival_rate_req_s': rate, 'budget_bytes': budget,
                'resident_bytes': srv.used, 'slots': sum(len(v) for v in srv.pools.values()),
                'warm_s': t_warm, 'evicted': srv.evicted, 'served_vs_oracle_worst_of_3': worst,
                'mix': '70% 2D (64..1024)^2 / 30% 3D (32..160)^3 on 16-rung geometric ladders, p in {2,3}, '
                       'Poisson solve / 20-step heat 50/50, FP64 / FP32 pairs 50/50, PW tests'})
    srv.close()
    return out


def measure_batch(stream, count=512, seed=0, reps=10):
    """Row f2 (batched 2D Poisson, 512 uneven instances): N log-uniform on 16
    rungs in [32, 512] per axis, p in {2, 3}, PW tests, FP32 pairs with one
    refinement; manufactured sources amp sin(k1 pi x) sin(k2 pi y), k uniform in
    1..4.  Times the fused source kernel and the graph-captured batch solve
    (grouped transforms on the tensor-core kernel; the cuBLAS grouped GEMMs
    beside it)."""
    import numpy as np
    import torch
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Batch
    shapes = workloads.batch_shapes(count, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.integers(1, 5, size=(count, 2))
    par = np.stack([np.pi ** 2 * (k[:, 0] ** 2 + k[:, 1] ** 2), k[:, 0], k[:, 1]], 1).astype(np.float64)
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        bt = Batch(shapes, stream=stream)
        t_create = time.perf_counter() - t0
        t_src = _time_events(stream, lambda: bt.source_sine(par), reps)
        t_solve = _time_events(stream, bt.solve, reps)
        bt.sync_status()
        bc = Batch(shapes, stream=stream, gemm='cublas')
        bc.source_sine(par)
        t_solve_cublas = _time_events(stream, bc.solve, reps)
        bc.close()
    dof = sum((a + p) * (b + p) for a, b, p in shapes)
    flops = sum(2 * 2 * 2 * ((a + p) + (b + p)) * (a + p) * (b + p) for a, b, p in shapes)
    out = {'instances': count, 'dof': dof, 'create_s': t_create, 'tiles_source_residual': bt.tiles(),
           'source_us': t_src * 1e6, 'solve_us': t_solve * 1e6, 'instances_per_s': count / t_solve,
           'dof_per_s': dof / t_solve, 'gemm_tflops': flops / t_solve / 1e12,
           'solve_us_cublas_grouped': t_solve_cublas * 1e6,
           'params': par, 'batch': bt}
    return out


def cpu_baseline_batch(res, sample=8):
    """Oracle side of row f2: sampled instances' solutions against the oracle
    (backward error, and the error against the oracle's sparse direct solve
    of the same right-hand side) and that solve timed per instance."""
    import numpy as np
    from oracle import poisson_nd, systems
    from paper_1910_08535_gb300 import workloads
    bt, par = res.pop('batch'), res.pop('params')
    shapes = workloads.batch_shapes(res['instances'], seed=0)
    idx = np.random.Generator(np.random.PCG64(1)).choice(len(shapes), size=sample, replace=False)
    etas, secs, errs = [], [], []
    for i in idx:
        nx, ny, p = shapes[i]
        axes = [systems.Axis(nx, p, p + 1, 'pw', 'dirichlet0'), systems.Axis(ny, p, p + 1, 'pw', 'dirichlet0')]
        b = bt.to_numpy(int(i), 0)
        u = bt.to_numpy(int(i), 1)
        etas.append(poisson_nd.backward_error(axes, u, b))
        if nx <= 200:        # the sparse direct solve of the largest grids takes minutes
            t0 = time.perf_counter()
            ref = poisson_nd.solve(axes, b, sparse=True)
            secs.append((time.perf_counter() - t0, (nx + p) * (ny + p)))
            errs.append(errors(u, ref))
    bt.close()
    res['max_backward_error_sample'] = float(max(etas))
    if errs:
        res['vs_oracle_worst_sample'] = {k: max(e[k] for e in errs) for k in errs[0]}
    res['oracle_sparse_direct_dof_per_s_sample'] = (float(sum(d for _, d in secs) / sum(t for t, _ in secs))
                                                    if secs else None)
    res['oracle_sample'] = f'{sample} random instances of the batch (sparse direct on those with N <= 200)'
    return res


def cpu_baseline_poisson(res):
    """Oracle side of row f1: the backward error of the GPU solutions at full
    size (the oracle applies K by per-axis contractions; a sparse direct
    solve at 1M unknowns is out of reach here)."""
    from oracle import poisson_nd, systems
    ne, p = 1024, 3
    axes = [systems.Axis(ne, p, p + 1, 'pw', 'dirichlet0') for _ in range(2)]
    out = {}
    for k, v in res.items():
        if k == 'sample_256x256_vs_oracle':
            out[k] = v
            continue
        out[k] = {kk: vv for kk, vv in v.items() if kk not in ('solution', 'rhs')}
        out[k]['backward_error_vs_oracle'] = poisson_nd.backward_error(axes, v['solution'], v['rhs'])
    return out


def window_width(ne, p, nq, test):
    """Padded window width (3, 5, 7 or 9) of the 1D tested mass and Laplacian
    rows: the number of coefficients a row of the step's banded passes reads."""
    import numpy as np
    from oracle import systems
    ax = systems.Axis(ne, p, nq, test)
    span = 0
    for M in (systems.mass(ax), systems.laplace(ax)):
        for row in M:
            nz = np.nonzero(row)[0]
            span = max(span, int(nz[-1] - nz[0] + 1))
    return next(x for x in (3, 5, 7, 9) if x >= span)


def run_native(args, rank, world):
    import numpy as np
    import torch
    from paper_1910_08535_gb300 import _build, igapw, workloads
    from paper_1910_08535_gb300.igapw import Context

    _build.build()
    dev = int(os.environ.get('LOCAL_RANK', '0')) if world > 1 else 0
    torch.cuda.set_device(dev)
    w = workloads.WORKLOADS[WORKLOAD]
    nsteps = w['steps']
    dt = workloads.dt_of(WORKLOAD)
    u0 = workloads.initial_state(WORKLOAD, seed=rank)
    flags = igapw.IGAPW_FLAG_FP64_RESIDUAL if args.residual == 'fp64' else 0
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device='cuda')

    def run_test(test):
        with torch.cuda.stream(stream):
            c = Context(dim=3, n_elem=w['n_elem'], degree=w['degree'], nq=w['nq'], test=test,
                        precision='fp32r', flags=flags, stream=stream)
            init = c.from_numpy(u0)
            u = c.empty()
            for _ in range(args.warmup):
                u.copy_(init)
                c.step(u, dt, nsteps)
            c.sync()
            barrier(world)
            torch.cuda.synchronize()
            times = []
            with ClockSampler(dev) as clk:
                for _ in range(args.steps):
                    u.copy_(init)
                    flush.fill_(1.0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    c.step(u, dt, nsteps)
                    e1.record(stream)
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1) / 1e3)
            torch.cuda.synchronize()
            barrier(world)
            c.sync()
            total = max_over_ranks(sum(times), world)
            return c, init, u, total, clk.summary()

    c, init, u, t_pw, clocks = run_test('pw')
    ntot = c.ntot
    value = world * ntot * nsteps * args.steps / t_pw
    step_kernels = [c.get_step_shape(a) for a in range(3)]
    # Galerkin comparator on the same mesh
    cg, _, _, t_g, _ = run_test('galerkin')
    value_g = world * ntot * nsteps * args.steps / t_g
    g_kernels = [cg.get_step_shape(a) for a in range(3)]
    cg.close()

    # dominant kernel: the explicit step, three per-axis launches of the step
    # kernel, timed as one step (a one-step graph) with CUDA events on the
    # context stream, L2 flushed before each.  Algorithmic bytes per step:
    # read u and write u' as FP32 pairs, 16 bytes per coefficient.
    one = []
    with torch.cuda.stream(stream):
        for i in range(23):
            u.copy_(init)
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c.step(u, dt, 1)
            e1.record(stream)
            e1.synchronize()
            if i >= 3:
                one.append(e0.elapsed_time(e1) / 1e3)
    t_one = sum(one) / len(one)
    pk = peaks()
    src = peak_sources(pk)
    hbm_peak = src['hbm_gbs']
    alg_bytes = 16.0 * ntot
    traffic, traffic_src = profiled_traffic()
    # ALU view (explanation, not the headline): FP32 operations per coefficient
    # and axis of the double-float step with the window width W and degree p
    # of the context: g = C u (W compensated products of 12 + 3), residual
    # g - A w0 (W of 11 + 2), two FP32 banded solves with spike corrections
    # (4p + 1 each), update 15; the method's own FP32 work is the banded
    # passes alone: 2 W (C, A) + 2 (2p + 1) flops.
    Wc, p = window_width(w['n_elem'], w['degree'], w['nq'], 'pw'), w['degree']
    emu_ops = 3 * ((12 * Wc + 3) + (11 * Wc + 2) + 2 * (4 * p + 1) + 15)
    method_flops = 3 * (2 * Wc + 2 * (2 * p + 1))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak_ops = sms * 128 * src['sm_max_mhz'] * 1e6
    roof = {'bound': 'hbm', 'achieved': alg_bytes / t_one / 1e9, 'peak': hbm_peak, 'unit': 'GB/s',
            'frac': alg_bytes / t_one / 1e9 / hbm_peak, 'traffic': traffic,
            'traffic_source': traffic_src,
            'kernel': 'chunk_step_kernel x3 per explicit step (x, y, z lines), heat3d PW',
            'alg_bytes_per_step': alg_bytes, 'step_us': t_one * 1e6, 'peak_source': src['hbm_source'],
            'note': 'heat3d state (18 MB) is L2-resident within a step; past-L2 grids in rows.a7_size_ladder',
            'alu_view': {'fp32_ops_per_dof_step_double_float': emu_ops,
                         'method_flops_per_dof_step': method_flops,
                         'ops_per_s': ntot * emu_ops / t_one,
                         'peak_ops_per_s': alu_peak_ops,
                         'frac': ntot * emu_ops / t_one / alu_peak_ops,
                         'peak_kind': f'{sms} SMs x 128 FP32 lanes x {src["sm_max_mhz"]:.0f} MHz'}}

    # end to end through the public C ABI with host buffers (pinned)
    host = torch.empty((2,) + c.shape, dtype=torch.float32).pin_memory()
    hb = host.numpy()
    e2e_t = []
    for i in range(args.warmup + args.steps):
        hb[...] = init.cpu().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        igapw.igapw_step_host(c.ctx, dt, nsteps, host)
        el = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_t.append(el)
    e2e_total = max_over_ranks(sum(e2e_t), world)
    e2e = {'value': world * ntot * nsteps * args.steps / e2e_total, 'unit': 'DOF-updates/s',
           'h2d_bytes_per_step': 8 * ntot, 'd2h_bytes_per_step': 8 * ntot}

    rows = {}
    rows['a4_source_table1'] = measure_source_table1(stream, flush, hbm_peak)
    rows.update(measure_rows(c, u, dt, stream, flush, hbm_peak))
    c.close()
    if rank == 0:
        rows['a8_heat3d_pw'] = measure_heat('heat3d', 'pw', stream, flush, nsteps)
        rows['a8_heat3d_galerkin'] = measure_heat('heat3d', 'galerkin', stream, flush, nsteps)
    rows['a7_heat2d_pw'] = measure_heat('heat2d', 'pw', stream, flush, 200)
    rows['a7_heat2d_galerkin'] = measure_heat('heat2d', 'galerkin', stream, flush, 200)
    rows['a7_heat2d_pw_over_galerkin'] = (rows['a7_heat2d_pw']['dof_updates_per_s'] /
                                          rows['a7_heat2d_galerkin']['dof_updates_per_s'])
    if not args.no_ladder:
        rows['a7_size_ladder'] = measure_ladder(stream, flush, hbm_peak)
    rows['f1_poisson_2d_1024'] = cpu_baseline_poisson(measure_poisson(stream, flush))
    rows['f2_batch_poisson_512'] = cpu_baseline_batch(measure_batch(stream))
    # the request server is a one-GPU process: measured at N = 1
    serving = measure_serving() if (world == 1 and not args.no_serve) else None

    cpu = None
    if rank == 0 and world == 1:
        cpu = cpu_baseline_oracle(steps=20)
        cpu.pop('seconds', None)
    launches_per_time_step = 3
    line = {'metric': METRIC, 'value': value, 'unit': 'DOF-updates/s', 'n_gpus': world, 'steps': args.steps,
            'warmup': args.warmup, 'ms_per_step': t_pw / args.steps * 1e3, 'higher_is_better': True,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32 pairs (double-float) + fp64 residual'
            if args.residual == 'fp64' else 'f32 pairs (double-float), double-float residual',
            'data': 'synthetic (seeded PCG64; coefficients 1e-2 N(0,1))',
            'config': {'workload': 'heat3d: 3D explicit heat, cubic C2, 128^3 elements (2,248,091 DOF), '
                                   '4x4x4 Gauss, dt=0.05h^2, 50 steps per bench step, PW tests',
                       'l2': 'flushed (512 MB write) before every timed step', 'residual': args.residual,
                       'step_kernels': [f'{k}/{nl}' for k, nl in step_kernels]},
            'roofline': roof,
            'galerkin': {'value': value_g, 'unit': 'DOF-updates/s', 'pw_over_galerkin': value / value_g,
                         'step_kernels': [f'{k}/{nl}' for k, nl in g_kernels],
                         'note': 'split form: both tests reduce to banded per-axis tables (PW width 5, '
                                 'Galerkin 7); the PW advantage is the narrower table'},
            'clocks': clocks, 'e2e': e2e,
            'gpu_launches': launches_per_time_step * nsteps * args.steps,
            'cpu_baseline': cpu, 'rows': rows, 'serving': serving}
    if rank == 0:
        print(json.dumps(rnd(line)))


def main():
    args = parse()
    rank, world = dist_setup(args.gpus)
    if args.impl == 'reference':
        run_reference(args, rank, world)
    else:
        run_native(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == '__main__':
    main()
