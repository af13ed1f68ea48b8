"""Pins of the refined-test-space variant (Sec. 2): tests that are sums of
B-splines of a test space refined r times, grouped by the PW cells.  Checked
against the paper's construction (summing rows of the rectangular
refined-tested system, integrated on its own quadrature), the partition of
unity, the limit r -> infinity (the PW rows) and a 1D Poisson solve."""
import numpy as np
import pytest

from oracle import bspline, poisson, quadrature, systems


def _row_sums_of_rectangular_system(ax, deriv):
    """Sec. 2: the B-spline-tested system over the refined test space (one row
    per refined test function, p+2 Gauss points per refined element), then
    the rows of J_k summed into row k."""
    tr = quadrature.refined_knots(ax.knots, ax.refine)
    br = bspline.unique_knots(tr)
    xs, ws = zip(*[quadrature.map_rule(ax.p + 2, br[e], br[e + 1]) for e in range(len(br) - 1)])
    x, w = np.concatenate(xs), np.concatenate(ws)
    G = (bspline.basis_matrix(tr, ax.p, x, 0).T * w) @ bspline.basis_matrix(ax.knots, ax.p, x, deriv)
    R = np.zeros((ax.n, ax.n))
    for k, i in enumerate(ax.rows()):
        R[i] = G[quadrature.refined_sets(ax.knots, ax.p, ax.refine, ax.bc)[k]].sum(axis=0)
    return R


@pytest.mark.parametrize('p', [2, 3])
@pytest.mark.parametrize('r', [2, 5])
@pytest.mark.parametrize('deriv', [0, 2])
def test_rows_are_sums_of_refined_rows(p, r, deriv):
    ax = systems.Axis(7, p, p + 1, 'refined', refine=r)
    W = systems.test_matrix(ax)
    got = W @ systems.eval_matrix(ax, deriv)
    want = _row_sums_of_rectangular_system(ax, deriv)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize('p', [2, 3])
def test_partition_of_unity_of_tests(p):
    """Every refined function joins exactly one set, so sum_i T_i = 1 and the
    column sums equal those of the B-spline-tested mass (int B_j)."""
    ax = systems.Axis(9, p, p + 1, 'refined', refine=3)
    sets = quadrature.refined_sets(ax.knots, p, 3, 'none')
    flat = sorted(m for s in sets for m in s)
    assert flat == list(range(len(flat)))
    g = systems.Axis(9, p, p + 1, 'galerkin')
    assert np.allclose(systems.mass(ax).sum(axis=0), systems.mass(g).sum(axis=0), rtol=0, atol=1e-13)
    W = systems.test_matrix(ax)
    x, w, _ = ax.points()
    assert np.allclose(W.sum(axis=0), w, rtol=1e-13, atol=0)


@pytest.mark.parametrize('p', [2, 3])
def test_limit_is_the_pw_test(p):
    ref = systems.mass(systems.Axis(6, p, p + 1, 'pw'))
    errs = [np.abs(systems.mass(systems.Axis(6, p, p + 1, 'refined', refine=r)) - ref).max() for r in (4, 8, 16, 32)]
    for a, b in zip(errs, errs[1:]):
        assert b < a / 1.5, errs
    assert errs[-1] < 0.02 * np.abs(ref).max()


@pytest.mark.parametrize('p', [2, 3])
def test_poisson_1d_converges(p):
    errs = []
    for ne in (8, 16, 32):
        ax = systems.Axis(ne, p, p + 1, 'refined', 'dirichlet0', refine=4)
        u = poisson.solve(ax, lambda x: np.pi ** 2 * np.sin(np.pi * x))
        errs.append(poisson.l2_error(ax, u, lambda x: np.sin(np.pi * x)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9), rates
