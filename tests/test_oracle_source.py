"""Pins of the oracle's source RHS (Sec. 4.1: the L2-projection right-hand side
b = T f from samples of f at the quadrature points) against values it does not
compute itself.  f is a spline of the trial space (piece-wise polynomial with
breaks at the knots, random coefficients), so

- PW: b_c is the exact integral of f over cell c, given here by scipy's
  B-spline antiderivative between cell break points rebuilt in this file from
  the Greville-midpoint definition.  This holds only if every cell is split at
  the knots inside it, each piece carries its own Gauss rule, and the weights
  are scaled to the piece;
- Galerkin: b_i = int B_i f, given here by a 10-point numpy Gauss rule per knot
  span with scipy's B-spline evaluation.

Tensor products in 2D/3D, uniform and non-uniform knots, zero Dirichlet rows,
and one negative control (one point per piece is not exact)."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import systems, tensor


def _knots(ne, p, uniform, seed=5):
    if uniform:
        inner = np.linspace(0.0, 1.0, ne + 1)
    else:
        rng = np.random.default_rng(seed)
        cuts = np.sort(rng.uniform(0.05, 0.95, ne - 1))
        inner = np.concatenate([[0.0], cuts, [1.0]])
    return np.concatenate([np.zeros(p), inner, np.ones(p)])


def _free(n, bc):
    return list(range(n)) if bc == 'none' else list(range(1, n - 1))


def _cells(t, p, bc):
    """Break points: the domain ends and the midpoints of consecutive Greville
    abscissae of the free coefficients."""
    n = len(t) - p - 1
    xi = np.array([np.mean(t[j + 1: j + p + 1]) for j in range(n)])[_free(n, bc)]
    return np.concatenate([[t[0]], 0.5 * (xi[:-1] + xi[1:]), [t[-1]]])


def _expected_1d(t, p, c, test, bc):
    n = len(t) - p - 1
    f = BSpline(t, c, p, extrapolate=False)
    out = np.zeros(n)
    if test == 'pw':
        F = f.antiderivative()
        br = _cells(t, p, bc)
        for k, i in enumerate(_free(n, bc)):
            out[i] = F(br[k + 1]) - F(br[k])
        return out
    g, gw = np.polynomial.legendre.leggauss(10)
    spans = np.unique(t)
    for i in _free(n, bc):
        Bi = BSpline(t, np.eye(n)[i], p, extrapolate=False)
        s = 0.0
        for a, b in zip(spans[:-1], spans[1:]):
            x = 0.5 * (b - a) * g + 0.5 * (a + b)
            s += 0.5 * (b - a) * np.sum(gw * Bi(x) * f(x))
        out[i] = s
    return out


def _case(d, ne, p, nq, test, bc, uniform, seed=0):
    rng = np.random.default_rng(seed)
    axes, coefs, want = [], [], []
    for a in range(d):
        t = _knots(ne[a], p, uniform, seed=5 + a)
        ax = systems.Axis(ne[a], p, nq, test, bc, knots=t)
        c = rng.uniform(-1.0, 1.0, ax.n)
        axes.append(ax)
        coefs.append(BSpline(t, c, p, extrapolate=False))
        want.append(_expected_1d(t, p, c, test, bc))
    # samples on the tensor grid (x fastest), then the tensor product of 1D results
    vals = [coefs[a](axes[a].points()[0]) for a in range(d)]
    f = vals[0]
    w = want[0]
    for a in range(1, d):
        f = np.multiply.outer(vals[a], f)
        w = np.multiply.outer(want[a], w)
    return tensor.rhs_source(axes, f), w


def _exact_rule(test, p, nq):
    """PW: f has degree p on a piece (nq >= (p + 1) / 2 points are exact);
    Galerkin: B_i f has degree 2p on a span (nq >= p + 1)."""
    return 2 * nq - 1 >= (p if test == 'pw' else 2 * p)


@pytest.mark.parametrize('p,nq', [(2, 2), (2, 3), (3, 2), (3, 4), (4, 3)])
@pytest.mark.parametrize('uniform', [True, False])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_source_1d_exact_for_splines(p, nq, uniform, test):
    if not _exact_rule(test, p, nq):
        pytest.skip('Gauss rule not exact for B_i f at this nq')
    got, want = _case(1, [9], p, nq, test, 'none', uniform)
    assert np.max(np.abs(got - want)) < 1e-14 * np.max(np.abs(want)) * 10


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_source_dirichlet_rows(test):
    got, want = _case(1, [8], 3, 4, test, 'dirichlet0', False)
    assert got[0] == 0.0 and got[-1] == 0.0
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize('d,ne', [(2, [6, 5]), (3, [4, 3, 5])])
@pytest.mark.parametrize('p,nq', [(2, 2), (2, 3), (3, 4)])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_source_tensor_product(d, ne, p, nq, test):
    if not _exact_rule(test, p, nq):
        pytest.skip('Gauss rule not exact for B_i f at this nq')
    got, want = _case(d, ne, p, nq, test, 'none', False)
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize('p', [2, 3])
def test_one_point_per_piece_is_not_exact(p):
    """Negative control: the midpoint rule misses the quadratic/cubic pieces."""
    got, want = _case(1, [9], p, 1, 'pw', 'none', True)
    assert np.max(np.abs(got - want)) > 1e-6 * np.max(np.abs(want))
