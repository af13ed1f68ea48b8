"""Pins of the oracle's explicit heat step (Sec. 4.2, Eq. (6)): exact
reproduction of polynomials in the spline space, identity at dt = 0,
linearity, resume equivalence, quadrature route against system route."""
import numpy as np
import pytest

from oracle import bspline, heat, quadrature, systems


def _coeffs_1d(ax, g):
    """Spline coefficients of a polynomial g by interpolation at the Greville points."""
    xi = quadrature.greville(ax.knots, ax.p)
    return np.linalg.solve(bspline.basis_matrix(ax.knots, ax.p, xi, 0), g(xi))


def _coeffs(axes, terms):
    """Coefficients of sum_k prod_a g_{k,a}(x_a) (x-fastest tensor)."""
    out = 0.0
    for term in terms:
        c = np.ones(1)
        for a in reversed(range(len(axes))):
            c = np.multiply.outer(c, _coeffs_1d(axes[a], term[a])) if c.ndim else c
        out = out + c.reshape([ax.n for ax in reversed(axes)])
    return out


one = lambda x: np.ones_like(x)


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_polynomial_reproduced_2d(test):
    """u = x^2 y + 3 y^2 lies in the quadratic spline space and so does
    Lap u = 2y + 6, hence one step maps u to exactly u + dt (2y + 6)."""
    axes = [systems.Axis(5, 2, 3, test), systems.Axis(4, 2, 3, test)]
    u = _coeffs(axes, [(lambda x: x ** 2, lambda y: y), (one, lambda y: 3 * y ** 2)])
    dt = 0.01
    want = u + dt * _coeffs(axes, [(one, lambda y: 2 * y), (one, lambda y: 6 * one(y))])
    for route in ('system', 'quadrature'):
        got = heat.run(axes, u, dt, 1, route=route)
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_polynomial_reproduced_3d(test):
    """p=3: u = x^3 + y^2 z, Lap u = 6x + 2z."""
    axes = [systems.Axis(3, 3, 4, test), systems.Axis(4, 3, 4, test), systems.Axis(3, 3, 4, test)]
    u = _coeffs(axes, [(lambda x: x ** 3, one, one), (one, lambda y: y ** 2, lambda z: z)])
    dt = 0.003
    want = u + dt * _coeffs(axes, [(lambda x: 6 * x, one, one), (one, one, lambda z: 2 * z)])
    got = heat.run(axes, u, dt, 1)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_linear_fixed_point_many_steps(test):
    """Any global linear polynomial is a fixed point (its Laplacian vanishes)."""
    axes = [systems.Axis(6, 2, 3, test), systems.Axis(5, 2, 3, test)]
    u = _coeffs(axes, [(lambda x: 0.5 + 2 * x, one), (one, lambda y: -y)])
    got = heat.run(axes, u, 1e-3, 20)
    assert np.abs(got - u).max() < 1e-12


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_dt_zero_identity_and_linearity(test):
    axes = [systems.Axis(5, 3, 4, test), systems.Axis(6, 3, 4, test)]
    rng = np.random.default_rng(3)
    u, v = rng.standard_normal((2, axes[1].n, axes[0].n))
    assert np.abs(heat.run(axes, u, 0.0, 1) - u).max() < 1e-12
    dt = 0.2 / 36
    lhs = heat.run(axes, 2 * u - 3 * v, dt, 2)
    rhs = 2 * heat.run(axes, u, dt, 2) - 3 * heat.run(axes, v, dt, 2)
    assert np.abs(lhs - rhs).max() < 1e-11 * np.abs(lhs).max()


def test_resume_equivalence():
    axes = [systems.Axis(7, 2, 3, 'pw'), systems.Axis(7, 2, 3, 'pw')]
    u = np.random.default_rng(5).standard_normal((axes[1].n, axes[0].n))
    dt = 0.05 / 49
    a = heat.run(axes, u, dt, 5)
    b = heat.run(axes, heat.run(axes, u, dt, 2), dt, 3)
    assert np.array_equal(a, b)


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_smooth_mode_decays(test):
    """sin(pi x) sin(pi y) decays by about exp(-2 pi^2 t) (continuum rate)."""
    ne = 16
    axes = [systems.Axis(ne, 3, 4, test), systems.Axis(ne, 3, 4, test)]
    s = lambda x: np.sin(np.pi * x)
    u = _coeffs(axes, [(s, s)])
    dt, steps = 0.05 / ne ** 2, 40
    got = heat.run(axes, u, dt, steps)
    ratio = got[ne // 2, ne // 2] / u[ne // 2, ne // 2]
    assert abs(ratio - np.exp(-2 * np.pi ** 2 * dt * steps)) < 2e-3
