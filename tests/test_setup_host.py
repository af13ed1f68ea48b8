"""CPU parity of the library's host set-up (setup.cpp: knots, Gauss rules, PW
cells, quadrature point sets, point windows, refined test weights, end
derivatives) with the oracle.  A small harness (tests/c/setup_dump.cpp)
compiled with g++ against setup.cpp prints one axis; no GPU is involved.

- Points and weights: the library's Newton-iterated Gauss-Legendre rules
  mapped to every element / PW piece / refined element, against the oracle's
  numpy rules, to 2 ulp-level absolute error.
- PW cells (Greville midpoints, Sec. 2 reading) equal the oracle's; every
  point belongs to the row the oracle's cell ownership gives, and each row's
  point window is exactly its cell's points.
- Galerkin and refined windows hold exactly the points where the oracle's test
  matrix row is non-zero; refined weights w_q T_i(x_q) equal the oracle's.
- Dirichlet rows are not free; end derivatives B_j'(0), B_j'(1) equal scipy's.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import quadrature, systems

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = {'galerkin': 0, 'pw': 1, 'refined': 2}
BCS = {'none': 0, 'dirichlet0': 1}


@pytest.fixture(scope='module')
def dump():
    if shutil.which('g++') is None:
        pytest.skip('g++ not available')
    out_dir = os.path.join(ROOT, 'tests', 'c', '_build')
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, 'setup_dump')
    csrc = os.path.join(ROOT, 'paper_1910_08535_gb300', 'csrc')
    subprocess.run(['g++', '-std=c++17', '-O1', '-Wall', '-Wextra', '-Werror', '-I', csrc,
                    os.path.join(ROOT, 'tests', 'c', 'setup_dump.cpp'), os.path.join(csrc, 'setup.cpp'),
                    '-o', exe], check=True)

    def run(ne, p, nq, test, bc, refine=0, knots=None):
        args = [exe, str(ne), str(p), str(nq), str(TESTS[test]), str(BCS[bc]), str(refine)]
        if knots is not None:
            args += [repr(float(k)) for k in knots]
        res = subprocess.run(args, check=True, capture_output=True, text=True)
        out = {}
        for line in res.stdout.splitlines():
            name, *vals = line.split(' ')
            out[name] = np.array([float(v) for v in vals]) if name != 'error' else ' '.join(vals)
        return out
    return run


def _knots(ne, p, uniform, seed=7):
    if uniform:
        return None
    rng = np.random.default_rng(seed)
    inner = np.concatenate([[0.0], np.sort(rng.uniform(0.05, 0.95, ne - 1)), [1.0]])
    return np.concatenate([np.zeros(p), inner, np.ones(p)])


def _cases():
    for test in ('pw', 'galerkin', 'refined'):
        for p in (2, 3, 4):
            for nq in (1, 2, 4):
                for bc in ('none', 'dirichlet0'):
                    for ne, uniform in ((1, True), (5, False), (9, True)):
                        if ne == 1 and (bc == 'dirichlet0' or test == 'refined'):
                            continue
                        yield test, p, nq, bc, ne, uniform


@pytest.mark.parametrize('test,p,nq,bc,ne,uniform', list(_cases()))
def test_host_setup_matches_oracle(dump, test, p, nq, bc, ne, uniform):
    _compare(dump, test, p, nq, bc, ne, _knots(ne, p, uniform))


@pytest.mark.parametrize('ratio', [1.05, 1.2, 1.5])
@pytest.mark.parametrize('test', ['pw', 'galerkin', 'refined'])
@pytest.mark.parametrize('p', [2, 3, 4])
def test_graded_meshes(dump, ratio, test, p):
    """Geometrically graded elements (each `ratio` times the previous, 50
    elements): built, and equal to the oracle."""
    h = ratio ** np.arange(50)
    inner = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
    inner[-1] = 1.0
    _compare(dump, test, p, p + 1, 'none', 50, np.concatenate([np.zeros(p), inner, np.ones(p)]))


def _compare(dump, test, p, nq, bc, ne, full):
    refine = 3 if test == 'refined' else 0
    got = dump(ne, p, nq, test, bc, refine, full)
    assert 'error' not in got, got.get('error')
    ax = systems.Axis(ne, p, nq, test, bc, knots=full, refine=max(refine, 2))
    n = ax.n
    assert int(got['n'][0]) == n
    assert np.max(np.abs(got['knots'] - ax.knots)) <= 1e-15
    x, w, owner = ax.points()
    assert len(got['qx']) == len(x)
    assert np.max(np.abs(got['qx'] - x)) <= 4e-16
    assert np.max(np.abs(got['qw'] - w)) <= 4e-16
    free = np.zeros(n)
    free[ax.rows()] = 1
    assert np.array_equal(got['is_free'], free)
    W = systems.test_matrix(ax)
    ps, pc = got['pstart'].astype(int), got['pcount'].astype(int)
    assert int(got['wq'][0]) == pc.max()
    for i in ax.rows():
        nz = np.nonzero(W[i])[0]
        assert np.array_equal(nz, np.arange(ps[i], ps[i] + pc[i])), (i, nz, ps[i], pc[i])
    if test == 'pw':
        assert np.max(np.abs(got['cells'] - quadrature.pw_cells(ax.knots, p, bc))) <= 1e-15
        rows = np.array(ax.rows())
        assert np.array_equal(got['qrow'].astype(int), rows[owner])
    if test == 'refined':
        tw = got['tw_refined'].reshape(n, -1)
        for i in ax.rows():
            ref = W[i, ps[i]: ps[i] + pc[i]]
            assert np.max(np.abs(tw[i, :pc[i]] - ref)) <= 1e-14 * np.max(np.abs(ref))
    for j in range(n):
        d = BSpline(ax.knots, np.eye(n)[j], p).derivative()
        scale = max(1.0, abs(d(0.0)), abs(d(1.0)))
        assert abs(got['dleft'][j] - d(0.0)) <= 1e-12 * scale
        assert abs(got['dright'][j] - d(1.0)) <= 1e-12 * scale


def test_rejected_setups_report_errors(dump):
    """Knots that are not an open knot vector on [0, 1] are refused with a
    message rather than built."""
    got = dump(3, 2, 3, 'pw', 'none', 0, [0.0, 0.0, 0.0, 0.6, 0.3, 1.0, 1.0, 1.0])
    assert 'error' in got and got['error']
