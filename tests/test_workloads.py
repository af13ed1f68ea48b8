"""Input recipes (paper_1910_08535_gb300/workloads.py): seeded and
deterministic, the stated shapes, sizes and distributions of the workloads,
and manufactured sources that are the negative Laplacian of their exact
solutions (checked by finite differences, independently of the method)."""
import numpy as np
import pytest

from oracle import bspline, quadrature
from paper_1910_08535_gb300 import workloads as W


def test_workload_constants():
    assert W.WORKLOADS['heat2d']['n_elem'] == 256 and W.WORKLOADS['heat2d']['steps'] == 200
    assert W.WORKLOADS['heat3d']['n_elem'] == 128 and W.WORKLOADS['heat3d']['steps'] == 50
    assert W.dt_of('heat2d') == 0.1 / 256 ** 2
    assert W.dt_of('heat3d') == 0.05 / 128 ** 2


@pytest.mark.parametrize('gen', [lambda s: W.normal_coeffs((7, 5), s), lambda s: W.uniform_coeffs((7, 5), s),
                                 lambda s: W.gaussian_bump_2d(8, 2, s), lambda s: np.array(W.batch_shapes(20, s))])
def test_seeded_and_deterministic(gen):
    assert np.array_equal(gen(3), gen(3))
    assert not np.array_equal(gen(3), gen(4))


def test_knot_averages_are_greville_abscissae():
    for ne, p in ((8, 2), (5, 3), (3, 4)):
        t = bspline.open_uniform_knots(ne, p)
        assert np.max(np.abs(W.knot_averages(ne, p) - quadrature.greville(t, p))) < 1e-15


def test_heat2d_initial_state():
    u = W.initial_state('heat2d')
    assert u.shape == (258, 258)
    xi = W.knot_averages(256, 2)
    X, Y = np.meshgrid(xi, xi, indexing='xy')
    bump = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * 0.1 ** 2))
    noise = u - bump
    assert np.max(np.abs(noise)) <= 1e-3
    assert 0.9e-3 < np.max(np.abs(noise))                         # the noise is there
    assert abs(np.mean(noise)) < 2e-5                            # and centred
    assert not np.array_equal(u, u.T)                            # the noise breaks the symmetry


def test_heat3d_initial_state():
    u = W.initial_state('heat3d')
    assert u.shape == (131, 131, 131)
    assert abs(np.std(u) - 1e-2) < 1e-4 and abs(np.mean(u)) < 2e-5


def test_tensor_samples_layout():
    x, y, z = np.linspace(0, 1, 4), np.linspace(0, 1, 3), np.linspace(0, 1, 2)
    f = W.tensor_samples([x, y, z], [(np.sin, np.cos, np.exp), (np.cos, np.exp, np.sin)])
    assert f.shape == (2, 3, 4)
    want = np.einsum('k,j,i->kji', np.exp(z), np.cos(y), np.sin(x)) + \
        np.einsum('k,j,i->kji', np.sin(z), np.exp(y), np.cos(x))
    assert np.max(np.abs(f - want)) < 1e-15


def _minus_laplacian_fd(u, pts, h=1e-4):
    d = pts.shape[1]
    out = np.zeros(len(pts))
    for a in range(d):
        e = np.zeros(d)
        e[a] = h
        out -= (u((pts + e).T) - 2 * u(pts.T) + u((pts - e).T)) / h ** 2
    return out


@pytest.mark.parametrize('k', [(1,), (2, 3), (1, 4, 2)])
def test_manufactured_sources_match_their_solutions(k):
    d = len(k)
    rng = np.random.default_rng(0)
    pts = rng.uniform(0.1, 0.9, size=(25, d))
    u = W.sine_product_exact(k)
    lap = _minus_laplacian_fd(u, pts)
    f = np.array([W.sine_product_source([np.array([c]) for c in p], k).ravel()[0] for p in pts])
    assert np.max(np.abs(f - lap)) < 1e-4 * np.max(np.abs(f))
    if d == 1:
        x = pts[:, 0]
        lap1 = -(W.sine_exact(x + 1e-4) - 2 * W.sine_exact(x) + W.sine_exact(x - 1e-4)) / 1e-8
        assert np.max(np.abs(W.sine_source(x) - lap1)) < 1e-4 * np.pi ** 2


def test_batch_shapes_recipe():
    s = W.batch_shapes(2000, seed=1)
    ns = np.array([a for a, b, p in s])
    assert all(a == b for a, b, p in s) and {p for _, _, p in s} == {2, 3}
    rungs = np.unique(ns)
    assert rungs[0] == 32 and rungs[-1] == 512 and len(rungs) == 16
    ratios = rungs[1:] / rungs[:-1]
    assert np.max(np.abs(ratios / np.exp(np.log(16) / 15) - 1)) < 0.05   # geometric rungs
    counts = np.array([np.sum(ns == r) for r in rungs])
    assert counts.min() > 0.6 * counts.mean()                                # uniform over the rungs
