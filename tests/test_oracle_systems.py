"""Pins of the oracle's 1D systems: integration-by-parts equality (Sec. 1),
row combination / partition of unity (Sec. 2), the refined-test-space limit
(Sec. 2), the divergence form of PW Laplacian rows, Dirichlet rows (Sec. 4.3)."""
import numpy as np
import pytest

from oracle import bspline, quadrature, systems


@pytest.mark.parametrize('p', [2, 3, 4])
def test_ibp_equality(p):
    """Sec. 1: for C^1 bases and exact quadrature int B_i B_j'' = -int B_i' B_j'
    on every row whose test function vanishes on the boundary; with zero
    Dirichlet rows the two matrices agree entirely."""
    ax = systems.Axis(12, p, p + 1, 'galerkin')
    L, Li = systems.laplace(ax), systems.laplace_ibp(ax)
    scale = np.abs(L).max()
    assert np.abs(L[1:-1] - Li[1:-1]).max() < 1e-13 * scale
    assert np.abs(L[0] - Li[0]).max() > 1e-3 * scale     # boundary flux term
    axd = systems.Axis(12, p, p + 1, 'galerkin', 'dirichlet0')
    assert np.abs(systems.laplace(axd) - systems.laplace_ibp(axd)).max() < 1e-13 * scale


@pytest.mark.parametrize('p', [2, 3, 4])
@pytest.mark.parametrize('deriv', [0, 2])
def test_row_combination_elementwise(p, deriv):
    """Sec. 2 black terms: on each element the p+1 B-spline tests supported
    there sum to 1 at every quadrature point, so the sum of their local rows
    equals the local row tested with 1."""
    ax = systems.Axis(7, p, p + 2, 'galerkin')
    x, w, owner = ax.points()
    W = systems.test_matrix(ax)
    V = systems.eval_matrix(ax, deriv)
    for e in range(ax.n_elem):
        sel = owner == e
        local = W[:, sel] @ V[sel]            # rows of every test restricted to element e
        combined = local[e:e + p + 1].sum(axis=0)
        ones = w[sel] @ V[sel]
        assert np.allclose(combined, ones, atol=1e-13 * max(1, np.abs(ones).max()))
        others = np.delete(local, range(e, e + p + 1), axis=0)
        assert np.all(others == 0.0)


@pytest.mark.parametrize('p', [2, 3])
def test_column_sums_equal(p):
    """Summing all rows of either system gives the test function 1: 1^T G = 1^T P."""
    g, w = systems.Axis(9, p, p + 1, 'galerkin'), systems.Axis(9, p, p + 1, 'pw')
    for f in (systems.mass, systems.laplace):
        assert np.allclose(f(g).sum(axis=0), f(w).sum(axis=0), atol=1e-12 * np.abs(f(g)).max())


def _refined_rows(ne, p, r, deriv):
    """Rows of the B-spline-tested system on a test space refined r times,
    summed over the refined tests whose Greville point lies in each PW cell."""
    t = bspline.open_uniform_knots(ne, p)
    tr = bspline.open_uniform_knots(ne * r, p)
    br = bspline.unique_knots(tr)
    xs, ws = zip(*[quadrature.map_rule(p + 2, br[e], br[e + 1]) for e in range(len(br) - 1)])
    x, w = np.concatenate(xs), np.concatenate(ws)
    G = (bspline.basis_matrix(tr, p, x, 0).T * w) @ bspline.basis_matrix(t, p, x, deriv)
    g = quadrature.greville(tr, p)
    c = quadrature.pw_cells(t, p, 'none')
    R = np.zeros((len(c) - 1, G.shape[1]))
    for k in range(len(c) - 1):
        hi = (g < c[k + 1]) if k < len(c) - 2 else (g <= c[k + 1])
        R[k] = G[(g >= c[k]) & hi].sum(axis=0)
    return R


@pytest.mark.parametrize('p', [2, 3])
@pytest.mark.parametrize('deriv', [0, 2])
def test_refined_test_space_limit(p, deriv):
    """Sec. 2 construction: refining the test space and summing the rows of
    the tests inside a cell converges to the PW-tested row as the refinement
    grows (the ramps at the cell ends shrink)."""
    ne = 6
    ax = systems.Axis(ne, p, p + 1, 'pw')
    ref = systems.mass(ax) if deriv == 0 else systems.laplace(ax)
    errs = [np.abs(_refined_rows(ne, p, r, deriv) - ref).max() / np.abs(ref).max() for r in (12, 24, 48, 96)]
    for a, b in zip(errs, errs[1:]):
        assert b < a / 1.5, errs
    assert errs[-1] < 0.025, errs


@pytest.mark.parametrize('p', [2, 3, 4])
def test_pw_laplace_divergence_form(p):
    """int_cell B_j'' = B_j'(c_{k+1}) - B_j'(c_k): quadrature-free check of PW rows."""
    ax = systems.Axis(9, p, p + 1, 'pw')
    C = systems.laplace(ax)
    c = quadrature.pw_cells(ax.knots, p, 'none')
    D = bspline.basis_matrix(ax.knots, p, c, 1)
    assert np.allclose(C, D[1:] - D[:-1], atol=1e-12 * np.abs(C).max())


@pytest.mark.parametrize('p', [2, 3])
def test_pw_mass_row_sums_are_cell_lengths(p):
    ax = systems.Axis(9, p, p + 1, 'pw')
    c = quadrature.pw_cells(ax.knots, p, 'none')
    assert np.allclose(systems.mass(ax).sum(axis=1), np.diff(c), rtol=1e-13)


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_dirichlet_rows(test):
    ax = systems.Axis(6, 2, 3, test, 'dirichlet0')
    M = systems.mass(ax)
    n = ax.n
    assert np.all(M[0] == np.eye(n)[0]) and np.all(M[-1] == np.eye(n)[-1])
    assert np.all(systems.test_matrix(ax)[[0, -1]] == 0.0)


@pytest.mark.parametrize('p', [2, 3, 4])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_mass_nonsingular(p, test):
    """Sec. 2: the tests must be linearly independent or the factorization
    breaks; with Greville-midpoint cells the PW mass stays well conditioned."""
    for ne in (4, 16, 64):
        M = systems.mass(systems.Axis(ne, p, p + 1, test))
        assert np.linalg.cond(M) < 100.0
