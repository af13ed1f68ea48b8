"""The continuous-batching request loop on the GPU: every result is the same
alone and in the mix (within the stated tolerance), results match the oracle,
and admission respects the memory budget."""
import numpy as np
import pytest

from oracle import heat, poisson_nd
from tests._cases import TOL, oracle_axes, rel_err

pytestmark = pytest.mark.gpu

SMALL_2D = (16, 24, 40)
SMALL_3D = (8, 12)


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


def _stream(n, seed):
    from paper_1910_08535_gb300 import serve
    return serve.make_stream(n, rate=None, seed=seed, steps=4, ladder_2d=SMALL_2D, ladder_3d=SMALL_3D)


def _oracle(req):
    from paper_1910_08535_gb300 import serve, workloads
    sh = req.shape
    if sh.kind == 'heat':
        axes = oracle_axes(sh.dim, sh.n_elem, sh.degree, sh.nq, sh.test)
        u0 = serve.base_state(sh)
        return heat.run(axes, u0, req.dt_h2 / (sh.n_elem ** 2 * sh.dim), req.steps)
    axes = oracle_axes(sh.dim, sh.n_elem, sh.degree, sh.nq, sh.test, 'dirichlet0')
    pts = [ax.points()[0] for ax in axes]
    f = workloads.sine_product_source(pts, req.k)
    if sh.precision == 'fp32r':
        f = f.astype(np.float32).astype(np.float64)
    return poisson_nd.solve(axes, poisson_nd.rhs(axes, f))


def test_mix_equals_alone_and_oracle():
    from paper_1910_08535_gb300 import serve
    reqs = _stream(24, seed=7)
    srv = serve.Server(max_inflight=16)
    recs, mixed = srv.run(reqs, keep_results=True)
    srv.check()
    srv.close()
    assert sorted(mixed) == [r.rid for r in reqs]
    # several requests were on the GPU together
    overlap = sum(1 for r in recs.values() for q in recs.values()
                  if r is not q and q['admit'] < r['done'] and r['admit'] < q['done'])
    assert overlap > 0
    for req in reqs:
        solo = serve.Server()
        _, one = solo.run([req], keep_results=True)
        solo.check()
        solo.close()
        tol = TOL[req.shape.precision]
        assert rel_err(mixed[req.rid], one[req.rid]) <= tol, (req, rel_err(mixed[req.rid], one[req.rid]))
        ref = _oracle(req)
        assert rel_err(mixed[req.rid], ref) <= tol, (req, rel_err(mixed[req.rid], ref))


def test_budget_caps_resident_slots():
    from paper_1910_08535_gb300 import serve
    reqs = _stream(20, seed=11)
    biggest = max(serve.slot_bytes(r.shape) + serve.transient_bytes(r.shape) for r in reqs)
    srv = serve.Server(budget_bytes=2 * biggest, max_inflight=16)
    recs, _ = srv.run(reqs)
    srv.check()
    assert len(recs) == len(reqs)
    assert srv.used <= srv.budget
    # the slots of the requests in flight never exceeded the budget
    events = sorted([(r['admit'], r['bytes']) for r in recs.values()] +
                    [(r['done'], -r['bytes']) for r in recs.values()], key=lambda e: (e[0], e[1]))
    live = peak = 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak <= srv.budget
    assert srv.evicted > 0
    for r in recs.values():
        assert r['arrival'] <= r['admit'] <= r['done'] and r['latency'] >= 0
    srv.close()


def test_open_loop_stream_latency_summary():
    from paper_1910_08535_gb300 import serve
    reqs = serve.make_stream(40, rate=400.0, seed=2, steps=4, ladder_2d=SMALL_2D, ladder_3d=SMALL_3D)
    srv = serve.Server()
    srv.warm({r.shape for r in reqs})
    recs, _ = srv.run(reqs)
    srv.check()
    srv.close()
    s = serve.summarize(recs)
    assert s['requests'] == 40 and 0 < s['p50_ms'] <= s['p99_ms'] <= s['max_ms']
