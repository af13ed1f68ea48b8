"""Host logic of the continuous-batching scheduler (serve.Server) with the
device slots replaced by fakes: admission in arrival order, the device-memory
budget (resident slot bytes + transient bytes of the requests in flight) never
exceeded, the in-flight limit, reuse of idle slots of the same shape, eviction
of idle slots of other shapes when memory is short, and the rejection of a
request larger than the whole budget."""
import itertools

import pytest

from paper_1910_08535_gb300 import serve


class _Done:
    """Completion event of a fake launch: done after a fixed number of polls."""

    def __init__(self, polls):
        self.left = polls

    def query(self):
        self.left -= 1
        return self.left < 0

    def synchronize(self):
        self.left = -1


class _Ctx:
    def sync(self):
        pass


def _fake_slot_class(server_ref, log, polls=2):
    class FakeSlot:
        def __init__(self, shape):
            self.shape, self.req, self.closed = shape, None, False
            self.h2d_bytes = self.d2h_bytes = 0
            self.done = _Done(0)
            self.ctx = _Ctx()
            log['created'].append(shape)

        def launch(self, req):
            srv = server_ref[0]
            assert not self.closed and self.req is None
            # admission happened just before: the budget holds with this request counted
            assert srv.used + srv.transient <= srv.budget
            log['order'].append(req.rid)
            log['live'] += 1
            log['peak'] = max(log['peak'], log['live'])
            self.req = req
            self.done = _Done(polls)

        def retire(self):
            log['live'] -= 1
            self.req = None

        def result(self):
            return self.req.rid

        def close(self):
            self.closed = True
            log['closed'] += 1

    return FakeSlot


def _clock():
    c = itertools.count()
    return lambda: next(c) * 1e-4


def _server(monkeypatch, budget, max_inflight=32, polls=2):
    ref = [None]
    log = {'created': [], 'order': [], 'live': 0, 'peak': 0, 'closed': 0}
    monkeypatch.setattr(serve, 'Slot', _fake_slot_class(ref, log, polls))
    srv = serve.Server(budget_bytes=budget, max_inflight=max_inflight)
    ref[0] = srv
    return srv, log


def _stream(n=300, seed=2):
    return serve.make_stream(n, None, seed=seed, ladder_2d=(64, 96, 128), ladder_3d=(32, 48))


def _largest(reqs):
    return max(serve.slot_bytes(r.shape) + serve.transient_bytes(r.shape) for r in reqs)


def test_tight_budget_admits_in_order_and_completes_everything(monkeypatch):
    reqs = _stream()
    srv, log = _server(monkeypatch, budget=2 * _largest(reqs))
    records, results = srv.run(reqs, keep_results=True, clock=_clock())
    assert sorted(records) == [r.rid for r in reqs]
    assert results == {r.rid: r.rid for r in reqs}
    assert log['order'] == [r.rid for r in reqs]          # all arrive at t = 0: rid order
    assert all(rec['latency'] >= rec['admit'] - rec['arrival'] >= 0 for rec in records.values())
    assert srv.evicted > 0 and log['closed'] == srv.evicted
    assert srv.transient == 0 and log['live'] == 0
    # resident bytes are exactly the parked slots'
    parked = sum(serve.slot_bytes(sh) * len(lst) for sh, lst in srv.pools.items())
    assert srv.used == parked <= srv.budget


def test_inflight_limit(monkeypatch):
    reqs = _stream(120)
    srv, log = _server(monkeypatch, budget=10 ** 13, max_inflight=5, polls=6)
    srv.run(reqs, clock=_clock())
    assert log['peak'] == 5


def test_one_at_a_time_reuses_one_slot_per_shape(monkeypatch):
    reqs = _stream(150)
    srv, log = _server(monkeypatch, budget=10 ** 13, max_inflight=1)
    srv.run(reqs, clock=_clock())
    shapes = {r.shape for r in reqs}
    assert len(log['created']) == len(shapes) and set(log['created']) == shapes
    assert srv.evicted == 0


def test_request_above_the_whole_budget_is_rejected(monkeypatch):
    reqs = _stream(10)
    srv, _ = _server(monkeypatch, budget=_largest(reqs) - 1)
    big = max(reqs, key=lambda r: serve.slot_bytes(r.shape) + serve.transient_bytes(r.shape))
    with pytest.raises(ValueError, match='above the whole budget'):
        srv.acquire(big.shape, serve.transient_bytes(big.shape))


def test_warm_parks_one_slot_per_shape(monkeypatch):
    reqs = _stream(60)
    srv, log = _server(monkeypatch, budget=10 ** 13)
    shapes = sorted({r.shape for r in reqs}, key=lambda s: (s.kind, s.dim, s.n_elem, s.degree, s.precision))
    srv.warm(shapes)
    assert all(len(srv.pools[sh]) == 1 for sh in shapes)
    assert srv.used == sum(serve.slot_bytes(sh) for sh in shapes)
    srv.close()
    assert srv.used == 0 and log['closed'] == len(shapes)
