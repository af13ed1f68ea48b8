"""Host logic of the request loop (no GPU): the seeded mixed stream, the
grid-size ladders and the memory estimate used for admission."""
import numpy as np

from paper_1910_08535_gb300 import serve


def test_ladders_are_geometric_and_cover_the_ranges():
    for lad, lo, hi in ((serve.LADDER_2D, 64, 1024), (serve.LADDER_3D, 32, 160)):
        assert lad[0] == lo and lad[-1] == hi
        r = np.diff(np.log(np.array(lad, dtype=float)))
        assert np.all(r > 0) and r.max() / r.min() < 1.6


def test_stream_is_seeded_and_mixed():
    a = serve.make_stream(2000, rate=100.0, seed=3)
    b = serve.make_stream(2000, rate=100.0, seed=3)
    assert [(r.arrival, r.shape, r.k) for r in a] == [(r.arrival, r.shape, r.k) for r in b]
    t = np.array([r.arrival for r in a])
    assert np.all(np.diff(t) >= 0)
    assert abs(len(a) / t[-1] - 100.0) < 10.0            # Poisson arrivals at the rate
    frac2 = np.mean([r.shape.dim == 2 for r in a])
    fracp = np.mean([r.shape.kind == 'poisson' for r in a])
    frac64 = np.mean([r.shape.precision == 'fp64' for r in a])
    assert abs(frac2 - 0.7) < 0.04 and abs(fracp - 0.5) < 0.04 and abs(frac64 - 0.5) < 0.04
    assert {r.shape.degree for r in a} == {2, 3}
    assert all(1 <= k <= 4 for r in a for k in r.k)
    assert all(len(r.k) == r.shape.dim for r in a)
    assert len({r.shape for r in a}) <= 2 * 16 * 2 * 2 * 2


def test_closed_loop_stream_arrives_at_once():
    s = serve.make_stream(10, rate=None, seed=1)
    assert all(r.arrival == 0.0 for r in s)


def test_slot_bytes_grow_with_size_and_cover_tensors():
    small = serve.Shape('heat', 2, 64, 2, 'fp64')
    big = serve.Shape('heat', 2, 1024, 2, 'fp64')
    assert serve.slot_bytes(big) > serve.slot_bytes(small) >= 8 * small.ntot
    assert serve.transient_bytes(big) == 0
    p = serve.Shape('poisson', 3, 160, 3, 'fp64')
    # resident: tensors plus the dense 1D transforms; nothing transient (the
    # library evaluates the source into the slot's right-hand-side tensor)
    assert serve.slot_bytes(p) >= 8 * p.ntot + 3 * 2 * 4 * (p.n_elem + p.degree) ** 2
    # ... and the transforms' hi/lo tiles for the tensor-core GEMM: per axis
    # and matrix ceil(n / 128) x ceil(n / 32) blocks of 2 x 128 x 32 values
    # (an A operand), each tile 8 x (128/8 x 144 + 16) bytes
    n = p.n_elem + p.degree
    blocks = -(-n // 128) * -(-n // 32)
    tiles = 3 * 2 * blocks * 2 * 8 * (128 // 8 * 144 + 16)
    assert serve.slot_bytes(p) >= 8 * p.ntot + 3 * 2 * 4 * n ** 2 + tiles
    assert serve.transient_bytes(p) == 0
    assert serve.transient_bytes(serve.Shape('poisson', 3, 160, 3, 'fp32r')) == 0
    # the largest request of the mixed stream fits the 120 GB budget several times over
    assert (serve.slot_bytes(p) + serve.transient_bytes(p)) * 5 < 120 * 10 ** 9


def test_summary_percentiles():
    recs = {i: {'latency': (i + 1) * 1e-3, 'done': 1.0 + i * 1e-3, 'arrival': i * 1e-3, 'dof': 10, 'steps': 2,
                'kind': 'heat' if i % 2 else 'poisson', 'h2d': 8, 'd2h': 8} for i in range(100)}
    s = serve.summarize(recs)
    assert abs(s['p50_ms'] - 50.5) < 1e-9 and abs(s['p99_ms'] - 99.01) < 1e-9
    assert s['requests'] == 100 and s['h2d_bytes'] == 800


def test_batch_shapes_ladder():
    from paper_1910_08535_gb300 import workloads
    s = workloads.batch_shapes(512, seed=0)
    assert len(s) == 512 and s == workloads.batch_shapes(512, seed=0)
    ns = sorted({a for a, _, _ in s})
    assert ns[0] == 32 and ns[-1] == 512 and len(ns) <= 16
    assert all(a == b for a, b, _ in s) and {p for _, _, p in s} == {2, 3}
