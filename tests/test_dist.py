"""Multi-rank logic of bench.py on CPU (gloo, world size 2): every rank runs its
own replica (no data-path collective); only the timing is reduced, as the max
over ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(('127.0.0.1', 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w = bench.dist_setup(world)
    assert (r, w) == (rank, world)
    bench.barrier(w)
    got = bench.max_over_ranks(1.5 + rank, w)
    q.put((rank, got))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res == [(0, 2.5), (1, 2.5)]


def test_single_rank_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ('RANK', 'WORLD_SIZE'):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup(1) == (0, 1)
    assert bench.max_over_ranks(3.0, 1) == 3.0


def test_reference_arm_under_torchrun_prints_one_line():
    """The reference arm launched as the driver launches it at N = 2 (torchrun,
    127.0.0.1, gloo on a machine without GPUs): rank 0 alone runs the oracle
    and prints one JSON line; the other rank exits 0 without work."""
    import json
    import subprocess
    cmd = [sys.executable, '-m', 'torch.distributed.run', '--nnodes=1', '--nproc-per-node', '2',
           '--master-addr', '127.0.0.1', '--master-port', str(_free_port()),
           os.path.join(ROOT, 'bench.py'), '--impl', 'reference', '--gpus', '2', '--steps', '1', '--warmup', '0']
    env = dict(os.environ, CUDA_VISIBLE_DEVICES='')
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith('{')]
    assert len(lines) == 1, res.stdout
    rec = json.loads(lines[0])
    assert rec['impl'] == 'reference' and rec['n_gpus'] == 2 and rec['value'] > 0
    assert rec['e2e']['h2d_bytes_per_step'] == 0 and rec['cpu_baseline']['kind'] == 'oracle'
