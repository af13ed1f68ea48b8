"""Launch planning of the tensor-core GEMM (csrc/tcgemm.cuh: tc_plan,
tc_makespan and the split workspace sizes), compiled for the CPU by
tests/c/tc_plan_check.cpp.  The plan must cover K with non-empty chunk ranges,
honour a fixed tile width, split only when allowed and only while the tiles
leave SMs idle, never be estimated slower than no split, split the
1032 x 1027 x 1032 transforms of the 1024^2 solve on 152 SMs, and size the
workspace for every partial tile; its estimated time is checked against a
list-scheduling simulation written here from the definition (CTAs start in
launch order, every tile of split 0 first, each on the first SM to free up)."""
import heapq
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, 'c', 'tc_plan_check.cpp')
BM, BK = 128, 32


@pytest.fixture(scope='module')
def planner():
    gxx = shutil.which('g++')
    cuda_inc = '/usr/local/cuda/include'
    if not gxx or not os.path.exists(os.path.join(cuda_inc, 'cuda.h')):
        pytest.skip('g++ and the CUDA headers are needed for the host build of the planner')
    d = tempfile.mkdtemp()
    exe = os.path.join(d, 'tc_plan_check')
    r = subprocess.run([gxx, '-std=c++20', '-O1', '-I' + cuda_inc, SRC, '-o', exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]

    def run(cases):
        inp = ''.join(' '.join(str(v) for v in c) + '\n' for c in cases)
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split('\n')
        res = []
        for line in out:
            if not line.strip():
                continue
            f = line.split()
            res.append({'bn': int(f[0]), 'splits': int(f[1]), 'kb': [int(v) for v in f[2:7]], 'time': float(f[7]),
                        'ws': int(f[8]), 'cnt': int(f[9]), 'tiles': int(f[10]), 'per_chunk': float(f[11]),
                        'over': float(f[12]), 'split_over': float(f[13])})
        assert len(res) == len(cases)
        return res

    yield run
    shutil.rmtree(d, ignore_errors=True)


def _simulate(tiles, kb, per_chunk, over, split_over, sms):
    S = len(kb) - 1
    extra = over + (split_over if S > 1 else 0.0)
    free = [0.0] * min(sms, tiles * S)
    heapq.heapify(free)
    end = 0.0
    for s in range(S):
        cost = per_chunk * (kb[s + 1] - kb[s] + extra)
        for _ in range(tiles):
            t0 = heapq.heappop(free)
            heapq.heappush(free, t0 + cost)
            end = max(end, t0 + cost)
    return end


def _cases(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        M, N = (int(v) for v in rng.integers(1, 2100, 2))
        K = int(rng.integers(1, 2100))
        batch = int(rng.choice([1, 1, 2, 3, 17]))
        sms = int(rng.choice([148, 152]))
        fixed = int(rng.choice([0, 0, 64, 96, 128]))
        out.append((M, N, K, batch, sms, fixed, 1))
    return out


def test_plans_cover_k_and_size_the_workspace(planner):
    cases = _cases(1, 300)
    for c, p in zip(cases, planner(cases)):
        M, N, K, batch, sms, fixed, _ = c
        nkc = -(-K // BK)
        S, kb = p['splits'], p['kb']
        assert 1 <= S <= 4
        assert p['bn'] in (64, 96, 128) and (fixed == 0 or p['bn'] == fixed)
        tiles = -(-M // BM) * -(-N // p['bn']) * batch
        assert p['tiles'] == tiles
        assert kb[0] == 0 and kb[S] == nkc and all(kb[i] < kb[i + 1] for i in range(S))
        assert all(v == nkc for v in kb[S + 1:])
        if S > 1:
            assert tiles < 2 * sms, (c, p)
            assert batch * S <= 65535
            assert p['ws'] == S * tiles * BM * p['bn'] and p['cnt'] == tiles
        else:
            assert p['ws'] == 0 and p['cnt'] == 0
        # the estimate is the list schedule of the plan's CTAs
        kb_used = kb[:S + 1]
        sim = _simulate(tiles, kb_used, p['per_chunk'], p['over'], p['split_over'], sms)
        assert abs(sim - p['time']) <= 1e-9 * sim, (c, p, sim)


def test_split_never_estimated_slower_and_only_when_allowed(planner):
    cases = _cases(2, 200)
    allowed = planner(cases)
    forbidden = planner([c[:6] + (0,) for c in cases])
    for c, a, f in zip(cases, allowed, forbidden):
        assert f['splits'] == 1
        assert a['time'] <= f['time'] * (1 + 1e-12), (c, a, f)
        if a['splits'] > 1:   # taken only when estimated at least 5% faster
            assert a['time'] * 1.05 < f['time'], (c, a, f)


def test_poisson_1024_transforms_are_split(planner):
    """99 tiles of 128 x 96 (33 chunks each) on 152 SMs leave 53 SMs idle:
    the plan splits K and is estimated well faster than no split."""
    a, f = planner([(1032, 1027, 1032, 1, 152, 0, 1), (1032, 1027, 1032, 1, 152, 0, 0)])
    assert a['splits'] >= 2 and f['splits'] == 1
    assert a['time'] < 0.85 * f['time']
    # large products (tiles >= 2 x SMs) are never split
    big = planner([(4104, 4099, 4104, 1, 152, 0, 1)])[0]
    assert big['splits'] == 1
