"""Continuous-batching request loop for Poisson solves and explicit heat runs.

Requests (2D/3D, different grid sizes, degrees and precisions) arrive over
time.  The server keeps, per problem shape, a pool of slots.  A slot owns one
library context -- its per-axis tables, factored 1D banded mass matrices or
diagonalised 1D Poisson pencils, scratch -- plus the device tensors of one
request, pinned host buffers and its own CUDA stream; all of it stays resident
between requests.  An arrived request is admitted as soon as a slot of its
shape is idle, or a new slot fits the device-memory budget (idle slots of
other shapes are evicted to make room).  Its work is enqueued on the slot's
stream and overlaps on the GPU with every other admitted request:

  heat     host-to-device copy of the initial coefficients, `steps` explicit
           steps (one CUDA graph), device-to-host copy of the result;
  poisson  the source RHS of the manufactured source prod_a sin(k_a pi x_a)
           (evaluated by the library at the quadrature points), the multi-D
           Poisson solve, device-to-host copy of the solution.

Completion is detected by polling a CUDA event per slot; a request's latency
is completion time minus arrival time.  Every arithmetic step of a request
runs in libigapw (no torch kernel on the request path); this module
schedules and copies.
"""
import collections
import dataclasses
import time

import numpy as np

# grid-size ladders: log-uniform draws snap to 16 geometric rungs per range, so
# that shapes repeat and resident slots are reused
LADDER_2D = tuple(int(v) for v in np.unique(np.round(np.geomspace(64, 1024, 16))))
LADDER_3D = tuple(int(v) for v in np.unique(np.round(np.geomspace(32, 160, 16))))


@dataclasses.dataclass(frozen=True)
class Shape:
    kind: str            # 'heat' or 'poisson'
    dim: int
    n_elem: int
    degree: int
    precision: str       # 'fp64' or 'fp32r'
    test: str = 'pw'

    @property
    def nq(self):
        return self.degree + 1

    @property
    def ntot(self):
        return (self.n_elem + self.degree) ** self.dim

    @property
    def nquad(self):
        """Upper bound on the quadrature points of the tensor grid: a PW cell
        is split at the knots inside it, so an axis has at most 2 n_elem + p
        pieces (Galerkin: n_elem elements) of nq points."""
        pieces = 2 * self.n_elem + self.degree if self.test == 'pw' else self.n_elem
        return (pieces * self.nq) ** self.dim


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float       # seconds after the start of the stream
    shape: Shape
    steps: int = 20      # heat
    dt_h2: float = 0.05  # heat: dt = dt_h2 h^2 / dim
    k: tuple = ()        # poisson: source wave numbers per axis


def make_stream(n_requests, rate, seed=0, frac_2d=0.7, frac_poisson=0.5, frac_fp64=0.5, steps=20, test='pw',
                ladder_2d=LADDER_2D, ladder_3d=LADDER_3D):
    """Seeded mixed stream: Poisson arrivals at `rate` per second (rate None:
    all at t = 0); 70% 2D (n log-uniform on LADDER_2D), 30% 3D (LADDER_3D);
    degree uniform in {2, 3}; Poisson solve or `steps`-step heat run 50/50;
    FP64 or FP32 pairs 50/50; Poisson sources with k_a uniform in 1..4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if rate:
        t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    else:
        t = np.zeros(n_requests)
    out = []
    for r in range(n_requests):
        two = rng.uniform() < frac_2d
        ladder = ladder_2d if two else ladder_3d
        ne = ladder[int(rng.integers(0, len(ladder)))]
        p = int(rng.integers(2, 4))
        kind = 'poisson' if rng.uniform() < frac_poisson else 'heat'
        prec = 'fp64' if rng.uniform() < frac_fp64 else 'fp32r'
        dim = 2 if two else 3
        k = tuple(int(v) for v in rng.integers(1, 5, size=dim))
        out.append(Request(r, float(t[r]), Shape(kind, dim, ne, p, prec, test), steps=steps, k=k))
    return out


def base_state(shape):
    """Initial heat coefficients of a shape: seeded standard normal x 1e-2."""
    n = shape.n_elem + shape.degree
    seed = (shape.dim * 1000 + shape.n_elem) * 10 + shape.degree
    rng = np.random.Generator(np.random.PCG64(seed))
    return 1e-2 * rng.standard_normal((n,) * shape.dim)


def slot_bytes(shape):
    """Resident device bytes of a slot (estimate): the context's tables and
    scratch and the slot's tensors at 8 bytes per coefficient, plus, for a
    Poisson context, the dense 1D transforms (W and V per axis, FP32), their
    hi/lo tiles for the tensor-core GEMM (two FP32 parts per value, tiles of
    up to 128 rows and 32 columns, 1/8 layout gaps) and the GEMM's split-K
    partial tiles and counters (under 10 MB on the 2D ladder's largest grid)."""
    n = shape.n_elem + shape.degree
    b = 6 * 8 * shape.ntot + (4 << 20)
    if shape.kind == 'poisson':
        b += shape.dim * 2 * 4 * n * n
        b += shape.dim * 2 * 10 * (n + 128) * (n + 32)
        b += 16 << 20
    return b


def transient_bytes(shape):
    """Device bytes a request holds only while it runs, beyond its slot: none
    (a Poisson request's source is evaluated by the library into the slot's
    right-hand-side tensor; a heat request steps the slot's state).  The
    scheduler keeps the accounting for request kinds that would need some."""
    return 0


class Slot:
    """One resident context with the device and pinned host buffers of one
    request at a time."""

    def __init__(self, shape):
        import torch
        from .igapw import Context
        self.shape = shape
        self.stream = torch.cuda.Stream()
        op, bc = ('poisson', 'dirichlet0') if shape.kind == 'poisson' else ('heat', 'none')
        self.ctx = Context(dim=shape.dim, n_elem=shape.n_elem, degree=shape.degree, nq=shape.nq, test=shape.test,
                           precision=shape.precision, op=op, bc=bc, stream=self.stream)
        fp64 = shape.precision == 'fp64'
        planes = 1 if fp64 else 2
        hdtype = torch.float64 if fp64 else torch.float32
        with torch.cuda.stream(self.stream):
            self.u = self.ctx.empty()
            if shape.kind == 'poisson':
                self.b = self.ctx.empty()
        self.hdtype = hdtype
        self.host_out = torch.empty(planes * self.ctx.ntot, dtype=hdtype).pin_memory()
        if shape.kind == 'heat':
            u0 = base_state(shape).ravel()
            self.host_in = torch.empty(planes * self.ctx.ntot, dtype=hdtype).pin_memory()
            if fp64:
                self.host_in.numpy()[:] = u0
            else:
                hi = u0.astype(np.float32)
                self.host_in.numpy()[:] = np.concatenate([hi, (u0 - hi.astype(np.float64)).astype(np.float32)])
        self.h2d_bytes = self.host_in.numel() * self.host_in.element_size() if shape.kind == 'heat' else 0
        self.d2h_bytes = self.host_out.numel() * self.host_out.element_size()
        self.done = torch.cuda.Event()
        self.req = None

    def launch(self, req):
        """Enqueue the whole request on the slot's stream (returns at once)."""
        import torch
        sh = self.shape
        with torch.cuda.stream(self.stream):
            if sh.kind == 'heat':
                self.u.view(-1).copy_(self.host_in, non_blocking=True)
                self.ctx.step(self.u, req.dt_h2 / (sh.n_elem ** 2 * sh.dim), req.steps)
            else:
                amp = float(np.pi ** 2 * sum(k * k for k in req.k))
                self.ctx.rhs_source_sine(amp, req.k, out=self.b)
                self.ctx.solve(self.b, out=self.u)
            self.host_out.copy_(self.u.view(-1), non_blocking=True)
            self.done.record(self.stream)
        self.req = req

    def retire(self):
        """After completion: the slot is free for the next request."""
        self.req = None

    def result(self):
        a = self.host_out.numpy()
        if self.shape.precision == 'fp64':
            return a.reshape(self.ctx.shape).copy()
        n = self.ctx.ntot
        return (a[:n].astype(np.float64) + a[n:].astype(np.float64)).reshape(self.ctx.shape)

    def close(self):
        self.ctx.close()


class Server:
    """Continuous-batching scheduler over per-shape slot pools under a
    device-memory budget."""

    def __init__(self, budget_bytes=120 * 10 ** 9, max_inflight=32):
        self.budget = budget_bytes
        self.max_inflight = max_inflight
        self.pools = collections.defaultdict(list)   # shape -> idle slots
        self.used = 0                                # resident bytes of all slots
        self.transient = 0                           # bytes of the requests in flight
        self.inflight = []
        self.created = 0
        self.evicted = 0

    def _evict_idle(self, need):
        for sh in list(self.pools):
            lst = self.pools[sh]
            while lst and self.used + need > self.budget:
                lst.pop().close()
                self.used -= slot_bytes(sh)
                self.evicted += 1

    def acquire(self, shape, extra=0):
        """An idle slot of `shape`, a new one if the budget allows (with
        `extra` transient bytes on top of what is in flight), else None."""
        if self.pools[shape]:
            if self.used + self.transient + extra > self.budget:
                return None
            return self.pools[shape].pop()
        need = slot_bytes(shape)
        if need + extra > self.budget:
            raise ValueError(f'request needs {need + extra} bytes, above the whole budget')
        if self.used + self.transient + need + extra > self.budget:
            self._evict_idle(need + extra + self.transient)
            if self.used + self.transient + need + extra > self.budget:
                return None
        s = Slot(shape)
        self.used += need
        self.created += 1
        return s

    def warm(self, shapes, steps=20, dt_h2=0.05):
        """Create (and park) one slot per shape ahead of a stream, each running
        one dry request of the stream's kind (so that its step graph is captured
        and its buffers are allocated before the first real request)."""
        for sh in shapes:
            if not self.pools[sh] and self.used + slot_bytes(sh) + transient_bytes(sh) <= self.budget:
                slot = self.acquire(sh)
                slot.launch(Request(-1, 0.0, sh, steps=steps, dt_h2=dt_h2, k=(1,) * sh.dim))
                slot.done.synchronize()
                slot.retire()
                self.pools[sh].append(slot)

    def run(self, requests, keep_results=False, clock=time.perf_counter):
        """Serve `requests`; returns (records by rid, results by rid)."""
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        records, results = {}, {}
        t0 = clock()
        while pending or self.inflight:
            now = clock() - t0
            # admit arrived requests in order while slots and memory allow
            while pending and pending[0].arrival <= now and len(self.inflight) < self.max_inflight:
                req = pending[0]
                extra = transient_bytes(req.shape)
                slot = self.acquire(req.shape, extra)
                if slot is None:
                    break
                pending.popleft()
                admit = clock() - t0
                self.transient += extra
                slot.launch(req)
                records[req.rid] = {'arrival': req.arrival, 'admit': admit, 'kind': req.shape.kind,
                                    'dim': req.shape.dim, 'n_elem': req.shape.n_elem,
                                    'degree': req.shape.degree, 'precision': req.shape.precision,
                                    'dof': req.shape.ntot, 'steps': req.steps if req.shape.kind == 'heat' else 0,
                                    'h2d': slot.h2d_bytes, 'd2h': slot.d2h_bytes,
                                    'bytes': slot_bytes(req.shape) + extra}
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
                    self.transient -= transient_bytes(s.shape)
                    s.retire()
                    self.pools[s.shape].append(s)
                else:
                    still.append(s)
            self.inflight = still
            if not self.inflight and pending:
                wait = pending[0].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
        return records, results

    def check(self):
        """Raises if any context recorded an asynchronous error."""
        for lst in self.pools.values():
            for s in lst:
                s.ctx.sync()

    def close(self):
        for lst in self.pools.values():
            for s in lst:
                s.close()
        self.pools.clear()
        self.used = 0


def summarize(records):
    lat = np.array([r['latency'] for r in records.values()])
    t_end = max(r['done'] for r in records.values())
    t_start = min(r['arrival'] for r in records.values())
    span = max(t_end - t_start, 1e-9)
    heat_upd = sum(r['dof'] * r['steps'] for r in records.values())
    out = {'requests': len(records), 'p50_ms': float(np.percentile(lat, 50) * 1e3),
           'p99_ms': float(np.percentile(lat, 99) * 1e3), 'mean_ms': float(lat.mean() * 1e3),
           'max_ms': float(lat.max() * 1e3), 'throughput_req_s': len(records) / span,
           'heat_dof_updates_per_s': heat_upd / span, 'makespan_s': span,
           'h2d_bytes': int(sum(r['h2d'] for r in records.values())),
           'd2h_bytes': int(sum(r['d2h'] for r in records.values()))}
    for kind in ('heat', 'poisson'):
        l = np.array([r['latency'] for r in records.values() if r['kind'] == kind])
        if len(l):
            out[f'{kind}_p50_ms'] = float(np.percentile(l, 50) * 1e3)
            out[f'{kind}_p99_ms'] = float(np.percentile(l, 99) * 1e3)
    return out
