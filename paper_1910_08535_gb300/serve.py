"""Continuous-batching request loop for explicit heat runs.

Requests (2D or 3D explicit heat runs of different grid sizes and degrees)
arrive over time.  The server keeps, per problem shape, a pool of contexts:
each context owns its per-axis tables and factored 1D banded mass matrices
(built once, resident on the device), its scratch, a device state buffer and
its own CUDA stream.  A request that has arrived is admitted as soon as a slot
of its shape is free (or a new one fits the device-memory budget); its work is
enqueued on the slot's stream (host-to-device copy, the step graph,
device-to-host copy) and runs concurrently with the other admitted requests.
Completions are detected with CUDA events; latency = completion - arrival.

All computation runs in libigapw; this module only schedules.  Poisson-solve
requests need a multi-D Poisson solver, which is not part of the library yet,
so the request mix is heat runs only.
"""
import collections
import dataclasses
import heapq
import time

import numpy as np


@dataclasses.dataclass(frozen=True)
class Shape:
    dim: int
    n_elem: int
    degree: int
    test: str = 'pw'
    precision: str = 'fp32r'

    @property
    def nq(self):
        return self.degree + 1

    @property
    def ntot(self):
        return (self.n_elem + self.degree) ** self.dim


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the stream
    shape: Shape
    steps: int
    dt_h2: float
    seed: int


def make_stream(n_requests, rate, seed=0, frac_2d=0.7, n2d=(64, 1024), n3d=(32, 160), steps=20, dt_h2=0.05):
    """Seeded request stream: Poisson arrivals at `rate` per second; 70% 2D with
    n_elem log-uniform in n2d, 30% 3D log-uniform in n3d, degree uniform in {2, 3}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    out = []
    for k in range(n_requests):
        two = rng.uniform() < frac_2d
        lo, hi = n2d if two else n3d
        ne = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        p = int(rng.integers(2, 4))
        out.append(Request(k, float(t[k]), Shape(2 if two else 3, ne, p), steps, dt_h2 / (3 if not two else 2),
                           int(rng.integers(0, 2 ** 31))))
    return out


def initial_state(req):
    from . import workloads
    n = req.shape.n_elem + req.shape.degree
    return workloads.normal_coeffs((n,) * req.shape.dim, seed=req.seed)


def slot_bytes(shape):
    """Device bytes a slot holds: state + scratch (pair or FP64: 8 B/DOF each),
    the contexts' split-step accumulator, plus tables (small)."""
    return 3 * 8 * shape.ntot + (1 << 20)


class Slot:
    def __init__(self, shape, stream):
        import torch
        from .igapw import Context
        self.shape = shape
        self.stream = stream
        with torch.cuda.stream(stream):
            self.ctx = Context(dim=shape.dim, n_elem=shape.n_elem, degree=shape.degree, nq=shape.nq,
                               test=shape.test, precision=shape.precision, stream=stream)
            self.u = self.ctx.empty()
        n = self.ctx.ntot * (1 if shape.precision == 'fp64' else 2)
        dtype = torch.float64 if shape.precision == 'fp64' else torch.float32
        self.host_in = torch.empty(n, dtype=dtype).pin_memory()
        self.host_out = torch.empty(n, dtype=dtype).pin_memory()
        self.done = torch.cuda.Event()
        self.req = None

    def launch(self, req, u0):
        """Enqueue the whole request on the slot's stream (asynchronous)."""
        import torch
        arr = np.ascontiguousarray(u0, dtype=np.float64).ravel()
        if self.shape.precision == 'fp64':
            self.host_in.numpy()[:] = arr
        else:
            hi = arr.astype(np.float32)
            lo = (arr - hi.astype(np.float64)).astype(np.float32)
            self.host_in.numpy()[:] = np.concatenate([hi, lo])
        dt = req.dt_h2 / req.shape.n_elem ** 2
        with torch.cuda.stream(self.stream):
            self.u.view(-1).copy_(self.host_in, non_blocking=True)
            self.ctx.step(self.u, dt, req.steps)
            self.host_out.copy_(self.u.view(-1), non_blocking=True)
            self.done.record(self.stream)
        self.req = req

    def result(self):
        a = self.host_out.numpy()
        if self.shape.precision == 'fp64':
            return a.reshape(self.ctx.shape).copy()
        n = self.ctx.ntot
        return (a[:n].astype(np.float64) + a[n:].astype(np.float64)).reshape(self.ctx.shape)


class Server:
    """Continuous-batching scheduler over per-shape slot pools."""

    def __init__(self, budget_bytes, max_inflight=64):
        self.budget = budget_bytes
        self.max_inflight = max_inflight
        self.pools = collections.defaultdict(list)   # shape -> idle slots
        self.used_bytes = 0
        self.inflight = []
        self.streams = []

    def _slot_for(self, shape):
        import torch
        if self.pools[shape]:
            return self.pools[shape].pop()
        need = slot_bytes(shape)
        if self.used_bytes + need > self.budget:
            # evict idle slots of other shapes to make room
            for sh, lst in list(self.pools.items()):
                while lst and self.used_bytes + need > self.budget:
                    s = lst.pop()
                    s.ctx.close()
                    self.used_bytes -= slot_bytes(sh)
            if self.used_bytes + need > self.budget:
                return None
        s = Slot(shape, torch.cuda.Stream())
        self.used_bytes += need
        return s

    def run(self, requests, keep_results=False, clock=time.perf_counter):
        """Serve `requests` (sorted by arrival); returns per-request records."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        records = {}
        results = {}
        t0 = clock()
        while pending or self.inflight:
            now = clock() - t0
            # admit every arrived request that fits, in arrival order
            while pending and pending[0].arrival <= now and len(self.inflight) < self.max_inflight:
                req = pending[0]
                slot = self._slot_for(req.shape)
                if slot is None:
                    break
                pending.popleft()
                slot.launch(req, initial_state(req))
                records[req.rid] = {'arrival': req.arrival, 'admit': clock() - t0, 'dim': req.shape.dim,
                                    'n_elem': req.shape.n_elem, 'degree': req.shape.degree,
                                    'dof': req.shape.ntot, 'steps': req.steps}
                self.inflight.append(slot)
            # retire finished requests
            still = []
            for s in self.inflight:
                if s.done.query():
                    rec = records[s.req.rid]
                    rec['done'] = clock() - t0
                    rec['latency'] = rec['done'] - rec['arrival']
                    if keep_results:
                        results[s.req.rid] = s.result()
                    self.pools[s.shape].append(s)
                    s.req = None
                else:
                    still.append(s)
            self.inflight = still
            if not self.inflight and pending and pending[0].arrival > clock() - t0:
                time.sleep(min(0.001, pending[0].arrival - (clock() - t0)))
        return records, results

    def close(self):
        for lst in self.pools.values():
            for s in lst:
                s.ctx.close()
        self.pools.clear()
        self.used_bytes = 0


def summarize(records):
    lat = np.array([r['latency'] for r in records.values()])
    t_end = max(r['done'] for r in records.values())
    dof_upd = sum(r['dof'] * r['steps'] for r in records.values())
    return {'requests': len(records), 'p50_ms': float(np.percentile(lat, 50) * 1e3),
            'p99_ms': float(np.percentile(lat, 99) * 1e3), 'mean_ms': float(lat.mean() * 1e3),
            'throughput_req_s': len(records) / t_end, 'dof_updates_per_s': dof_upd / t_end,
            'makespan_s': t_end}
