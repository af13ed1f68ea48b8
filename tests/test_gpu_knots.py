"""General (random) knot vectors with piece-wise constant, refined and
B-spline tests (Sec. 2: any N independent intervals): 20 random open knot
vectors per test kind and degree, set on both axes of a 2D context, and a
geometrically graded (ratio 2) mesh.  Each context's operator action,
Kronecker solve, source RHS and explicit steps against the oracle built on the
same knots, element by element (rel-L2 and max-abs <= 1e-5 relative, FP32
pairs with refinement).  Row windows then start below their first non-zero
column where the padded width allows, and the widths reach 7 and 9."""
import numpy as np
import pytest

from oracle import heat, systems, tensor
from tests._cases import TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


def _random_knots(ne, p, seed):
    rng = np.random.default_rng(seed)
    inner = np.concatenate([[0.0], np.sort(rng.uniform(0.0, 1.0, ne - 1)), [1.0]])
    return np.concatenate([np.zeros(p), inner, np.ones(p)])


def _graded_knots(ne, p, ratio):
    h = ratio ** np.arange(ne)
    inner = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
    inner[-1] = 1.0
    return np.concatenate([np.zeros(p), inner, np.ones(p)])


def _check(test, p, ne, knots):
    import torch
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    refine = 3 if test == 'refined' else 0
    c = Context(dim=2, n_elem=[ne[0], ne[1]], degree=p, nq=p + 1, test=test, precision='fp32r', refine=refine)
    for a in range(2):
        c.set_knots(a, knots[a])
    axes = [systems.Axis(ne[a], p, p + 1, test, knots=knots[a], refine=max(refine, 2)) for a in range(2)]
    tol = TOL['fp32r']
    # the 1D tables
    for a in range(2):
        M = c.assemble_1d(a, 'mass')
        assert np.abs(M - systems.mass(axes[a])).max() < 1e-12 * np.abs(M).max()
    # operator action and solve
    u0 = workloads.normal_coeffs(c.shape, seed=5)
    dt = 1e-4
    Ms, Ls = tensor.mass_mats(axes), tensor.lap_mats(axes)
    r = c.apply('heat', c.from_numpy(u0), dt)
    assert rel_err(c.to_numpy(r), tensor.apply_heat_system(axes, u0, dt, Ms, Ls)) < tol
    s = c.solve(r)
    assert rel_err(c.to_numpy(s), tensor.ads_solve(Ms, c.to_numpy(r))) < tol
    # source RHS of a smooth f at the context's points
    pts = [c.quad_points(a)[0] for a in range(2)]
    f = workloads.tensor_samples(pts, [(np.sin, np.cos)])
    b = c.rhs_source(torch.from_numpy(f.astype(np.float32)).cuda())
    assert rel_err(c.to_numpy(b), tensor.rhs_source(axes, f.astype(np.float32).astype(np.float64))) < tol
    # explicit steps (the tuner picks the step kernels for these widths)
    u = c.from_numpy(u0)
    c.step(u, dt, 3)
    assert rel_err(c.to_numpy(u), heat.run(axes, u0, dt, 3)) < tol
    c.sync()
    c.close()


@pytest.mark.parametrize('test', ['pw', 'refined', 'galerkin'])
@pytest.mark.parametrize('p', [2, 3])
def test_twenty_random_knot_vectors(test, p):
    ne = (23, 17)
    for seed in range(20):
        _check(test, p, ne, [_random_knots(ne[0], p, seed), _random_knots(ne[1], p, 100 + seed)])


@pytest.mark.parametrize('test', ['pw', 'refined', 'galerkin'])
def test_graded_by_two(test):
    ne = (12, 9)
    _check(test, 3, ne, [_graded_knots(ne[0], 3, 2.0), _graded_knots(ne[1], 3, 0.5)])
