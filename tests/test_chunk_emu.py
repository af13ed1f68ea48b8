"""The chunked explicit-step kernel (csrc/chunkstep.cuh) and its table set-up
kernel (csrc/chunktables.cuh) run on the CPU: tests/c/chunk_emu.cpp compiles
them for the host, every CUDA thread a host thread and every buffer (global
tables, state tensors, the block's shared memory) allocated at its exact
size under AddressSanitizer, so that any access outside a buffer aborts the
run.  The stepped state is compared with the oracle's explicit steps
(Sec. 4.2, Eq. (6)) in 1D, 2D and 3D, PW and Galerkin tests, p = 2..4, with
lines of one chunk, several chunks, and a last chunk shorter than p, and
8, 16 and 32 lines per block (ragged last blocks)."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import heat, systems

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, 'c', 'chunk_emu.cpp')


@pytest.fixture(scope='module')
def emu():
    gxx = shutil.which('g++')
    cuda_inc = '/usr/local/cuda/include'
    if not gxx or not os.path.exists(os.path.join(cuda_inc, 'cuda_runtime.h')):
        pytest.skip('g++ and the CUDA headers are needed for the host emulator')
    d = tempfile.mkdtemp()
    exe = os.path.join(d, 'chunk_emu')
    r = subprocess.run([gxx, '-std=c++20', '-O1', '-g', '-fsanitize=address', '-fno-omit-frame-pointer',
                        '-I' + cuda_inc, SRC, '-o', exe, '-lpthread'], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def _windows(M, W):
    """Window format of a banded matrix: row i couples to columns fs[i] .. fs[i] + W - 1."""
    n = M.shape[0]
    fs = np.zeros(n, dtype=np.int32)
    tab = np.zeros((n, W))
    for i in range(n):
        nz = np.nonzero(M[i])[0]
        f = min(int(nz[0]), n - W) if len(nz) else 0
        f = max(f, 0)
        assert nz[-1] < f + W
        fs[i] = f
        for w in range(W):
            if f + w < n:
                tab[i, w] = M[i, f + w]
    return fs, tab


def _run(emu, dim, ne, p, test, nl, steps=2, seed=0):
    ax = systems.Axis(ne, p, p + 1, test, 'none')
    A, C = systems.mass(ax), systems.laplace(ax)
    n = A.shape[0]
    width = max(int(np.nonzero(A[i])[0][-1] - np.nonzero(A[i])[0][0] + 1) for i in range(n))
    width = max(width, max(int(np.nonzero(C[i])[0][-1] - np.nonzero(C[i])[0][0] + 1) for i in range(n)))
    W = next(w for w in (3, 5, 7, 9) if w >= width)
    fsA, At = _windows(A, W)
    fsC, Ct = _windows(C, W)
    # one window start per row for both tables
    fs = np.minimum(fsA, fsC)
    At = np.array([[A[i, fs[i] + w] if fs[i] + w < n else 0.0 for w in range(W)] for i in range(n)])
    Ct = np.array([[C[i, fs[i] + w] if fs[i] + w < n else 0.0 for w in range(W)] for i in range(n)])
    assert all(np.count_nonzero(A[i]) == np.count_nonzero(At[i]) for i in range(n))
    assert all(np.count_nonzero(C[i]) == np.count_nonzero(Ct[i]) for i in range(n))
    shape = (n,) * dim
    u0 = 1e-2 * np.random.default_rng(seed).standard_normal(shape)
    hi = u0.astype(np.float32)
    lo = (u0 - hi.astype(np.float64)).astype(np.float32)
    dt = 0.05 / ne ** 2
    nn = [n if a < dim else 1 for a in range(3)]
    with tempfile.TemporaryDirectory() as d:
        fin, fout = os.path.join(d, 'in.bin'), os.path.join(d, 'out.bin')
        with open(fin, 'wb') as f:
            f.write(np.array([dim, *nn, p, W, nl, steps], dtype=np.int32).tobytes())
            f.write(np.array([dt], dtype=np.float64).tobytes())
            for _ in range(dim):
                f.write(fs.astype(np.int32).tobytes())
                f.write(At.astype(np.float64).tobytes())
                f.write(Ct.astype(np.float64).tobytes())
            f.write(hi.tobytes())
            f.write(lo.tobytes())
        env = dict(os.environ, ASAN_OPTIONS='detect_leaks=0')
        r = subprocess.run([emu, fin, fout], capture_output=True, text=True, timeout=600, env=env)
        assert r.returncode == 0, r.stderr[-4000:]
        out = np.fromfile(fout, dtype=np.float32).reshape((2,) + shape)
    got = out[0].astype(np.float64) + out[1].astype(np.float64)
    ref = heat.run([ax] * dim, u0, dt, steps)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize('dim,ne,p,test,nl', [
    (1, 10, 2, 'pw', 8), (1, 40, 3, 'galerkin', 16), (1, 32, 3, 'pw', 32),
    (2, 12, 2, 'pw', 16), (2, 12, 2, 'pw', 32), (2, 14, 3, 'galerkin', 8), (2, 32, 3, 'pw', 16),
    (2, 33, 4, 'galerkin', 16), (2, 40, 2, 'pw', 8),
    (3, 8, 2, 'pw', 16), (3, 14, 3, 'galerkin', 32), (3, 20, 3, 'pw', 8), (3, 15, 4, 'pw', 16),
    (3, 40, 2, 'galerkin', 16), (2, 200, 3, 'galerkin', 32), (2, 300, 3, 'pw', 16), (1, 300, 4, 'pw', 16),
])
def test_chunk_kernel_host_emulation(emu, dim, ne, p, test, nl):
    err = _run(emu, dim, ne, p, test, nl)
    assert err < 1e-10, err
