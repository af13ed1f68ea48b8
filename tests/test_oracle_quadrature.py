"""Pins of the oracle's quadrature and PW test cells (Sec. 2, Sec. 4.1)."""
import numpy as np
import pytest

from oracle import bspline, quadrature, systems


@pytest.mark.parametrize('nq', [1, 2, 3, 4, 5])
def test_gauss_exactness(nq):
    x, w = quadrature.map_rule(nq, 0.2, 0.9)
    for k in range(2 * nq):
        exact = (0.9 ** (k + 1) - 0.2 ** (k + 1)) / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14 * max(1, abs(exact)) * 10
    k = 2 * nq
    exact = (0.9 ** (k + 1) - 0.2 ** (k + 1)) / (k + 1)
    assert abs(np.sum(w * x ** k) - exact) > 1e-10 * exact


def _cubic(x):
    return 2.0 * x ** 3 - 0.7 * x ** 2 + 0.3 * x + 1.1


@pytest.mark.parametrize('test', ['galerkin', 'pw'])
def test_quadrature_order_claim(test):
    """Sec. 4.1: with a cubic RHS and quadratic trial space the B-spline-tested
    RHS (degree 5 integrand) needs 3 Gauss points per element, the PW-tested
    RHS (degree 3) only 2."""
    ref = systems.rhs_1d(systems.Axis(8, 2, 6, test), _cubic(systems.Axis(8, 2, 6, test).points()[0]))
    b2 = systems.rhs_1d(systems.Axis(8, 2, 2, test), _cubic(systems.Axis(8, 2, 2, test).points()[0]))
    b3 = systems.rhs_1d(systems.Axis(8, 2, 3, test), _cubic(systems.Axis(8, 2, 3, test).points()[0]))
    assert np.allclose(b3, ref, rtol=1e-13, atol=1e-15)
    if test == 'pw':
        assert np.allclose(b2, ref, rtol=1e-13, atol=1e-15)
    else:
        assert np.abs(b2 - ref).max() > 1e-7


@pytest.mark.parametrize('p', [2, 3, 4])
@pytest.mark.parametrize('bc', ['none', 'dirichlet0'])
def test_cells_partition_domain(p, bc):
    t = bspline.open_uniform_knots(10, p)
    c = quadrature.pw_cells(t, p, bc)
    n = bspline.n_basis(t, p)
    assert len(c) - 1 == len(quadrature.unknowns(n, bc))
    assert c[0] == 0.0 and c[-1] == 1.0 and np.all(np.diff(c) > 0)
    # every piece lies inside one element and no Gauss point sits on a cell bound
    pcs = quadrature.pw_points(t, p, 3, bc)
    br = bspline.unique_knots(t)
    for (x, w, k) in pcs:
        e = np.searchsorted(br, x.mean()) - 1
        assert np.all(x > br[e]) and np.all(x < br[e + 1])
        assert np.all(x > c[k]) and np.all(x < c[k + 1])
    assert abs(sum(pc[1].sum() for pc in pcs) - 1.0) < 1e-14


def test_cells_quadratic():
    """p=2: interior cells are the elements, the end elements are split at h/4."""
    ne = 8
    t = bspline.open_uniform_knots(ne, 2)
    c = quadrature.pw_cells(t, 2, 'none') * ne
    assert np.allclose(c, [0, 0.25] + list(range(1, ne)) + [ne - 0.25, ne])
    cd = quadrature.pw_cells(t, 2, 'dirichlet0') * ne
    assert np.allclose(cd, range(0, ne + 1))


def test_cells_cubic_straddle():
    """p=3: interior cells [(k-1/2)h, (k+1/2)h] straddle the knots."""
    ne = 8
    t = bspline.open_uniform_knots(ne, 3)
    c = quadrature.pw_cells(t, 3, 'none') * ne
    assert np.allclose(c, [0, 1 / 6, 2 / 3] + [k + 0.5 for k in range(1, ne - 1)] + [ne - 2 / 3, ne - 1 / 6, ne])
