"""Pins of the oracle's 1D Poisson solve (Sec. 4.3, Eq. (7), zero Dirichlet
rows): exact polynomial solution, convergence on u = sin(pi x)."""
import numpy as np
import pytest

from oracle import bspline, poisson, quadrature, systems


@pytest.mark.parametrize('p', [2, 3, 4])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_quadratic_solution_exact(p, test):
    """-u'' = 2 has u = x(1-x), which lies in every spline space with p >= 2."""
    ax = systems.Axis(9, p, p + 1, test, 'dirichlet0')
    u = poisson.solve(ax, lambda x: 2.0 * np.ones_like(x))
    xi = quadrature.greville(ax.knots, p)
    want = np.linalg.solve(bspline.basis_matrix(ax.knots, p, xi, 0), xi * (1 - xi))
    assert np.abs(u - want).max() < 1e-12


@pytest.mark.parametrize('p', [2, 3])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_manufactured_sine_converges(p, test):
    """u = sin(pi x), f = pi^2 sin(pi x): Galerkin converges at the optimal L2
    rate p+1; the PW solution converges at least quadratically."""
    ex = lambda x: np.sin(np.pi * x)
    f = lambda x: np.pi ** 2 * np.sin(np.pi * x)
    errs = []
    for ne in (8, 16, 32, 64):
        ax = systems.Axis(ne, p, p + 1, test, 'dirichlet0')
        errs.append(poisson.l2_error(ax, poisson.solve(ax, f), ex))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    if test == 'galerkin':
        assert np.all(np.abs(rates - (p + 1)) < 0.15), rates
    else:
        assert np.all(rates > 1.9), rates
    assert errs[-1] < 2e-4


def test_config0_errors():
    """1D Poisson, p=2, 64 elements, 3 Gauss points: both solutions close to sin(pi x)."""
    ex = lambda x: np.sin(np.pi * x)
    f = lambda x: np.pi ** 2 * np.sin(np.pi * x)
    for test, tol in (('galerkin', 1e-6), ('pw', 2e-4)):
        ax = systems.Axis(64, 2, 3, test, 'dirichlet0')
        u = poisson.solve(ax, f)
        assert poisson.l2_error(ax, u, ex) < tol
        assert poisson.max_error(ax, u, ex) < 5 * tol
