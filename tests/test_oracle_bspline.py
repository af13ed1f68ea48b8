"""Pins of the oracle's B-spline basis (Sec. 2): partition of unity, a library
B-spline routine, the paper's worked example, closed-form integrals."""
import os

import numpy as np
import pytest

from oracle import bspline, quadrature, systems

GOLD = os.path.join(os.path.dirname(__file__), 'golden')


def _nonuniform_knots(n_elem, p, seed):
    rng = np.random.default_rng(seed)
    inner = np.sort(rng.uniform(0.05, 0.95, n_elem - 1))
    return np.concatenate([[0.0] * (p + 1), inner, [1.0] * (p + 1)])


@pytest.mark.parametrize('p', [1, 2, 3, 4, 5])
@pytest.mark.parametrize('uniform', [True, False])
def test_partition_of_unity(p, uniform):
    t = bspline.open_uniform_knots(7, p) if uniform else _nonuniform_knots(7, p, p)
    x = np.concatenate([np.linspace(0, 1, 101), [0.0, 1.0], t])
    for deriv, target in ((0, 1.0), (1, 0.0), (2, 0.0)):
        if deriv > p:
            continue
        s = bspline.basis_matrix(t, p, x, deriv).sum(axis=1)
        scale = max(1.0, np.abs(bspline.basis_matrix(t, p, x, deriv)).max())
        assert np.allclose(s, target, atol=1e-12 * scale), (deriv, np.abs(s - target).max())


@pytest.mark.parametrize('p', [2, 3, 4])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_pou_at_quadrature_points(p, test):
    """Sec. 2 (black terms): the test B-splines non-zero at a quadrature point sum to 1."""
    ax = systems.Axis(9, p, p + 1, test)
    for deriv, target in ((0, 1.0), (1, 0.0), (2, 0.0)):
        V = systems.eval_matrix(ax, deriv)
        assert np.allclose(V.sum(axis=1), target, atol=1e-11 * max(1, np.abs(V).max()))


@pytest.mark.parametrize('p', [1, 2, 3, 4])
def test_against_scipy_bspline(p):
    from scipy.interpolate import BSpline
    t = _nonuniform_knots(6, p, 10 + p)
    n = bspline.n_basis(t, p)
    rng = np.random.default_rng(p)
    x = np.concatenate([rng.uniform(0, 1, 200), t[(t > 0) & (t < 1)] + 1e-3])
    for j in range(n):
        c = np.zeros(n)
        c[j] = 1.0
        spl = BSpline(t, c, p, extrapolate=False)
        for deriv in range(0, min(p, 2) + 1):
            ref = spl.derivative(deriv)(x) if deriv else spl(x)
            got = bspline.basis(t, p, j, x, deriv)
            assert np.allclose(got, np.nan_to_num(ref), atol=1e-10 * max(1, np.abs(ref).max()))


def test_right_end_point():
    for p in (1, 2, 3):
        t = bspline.open_uniform_knots(4, p)
        v = bspline.basis_matrix(t, p, np.array([1.0]), 0)[0]
        assert v[-1] == 1.0 and np.all(v[:-1] == 0.0)


def _read_worked():
    deg, knots, sup = None, None, []
    for line in open(os.path.join(GOLD, 'worked_example.txt')):
        if line.startswith('#') or not line.strip():
            continue
        tok = line.split()
        if tok[0] == 'degree':
            deg = int(tok[1])
        elif tok[0] == 'knots':
            knots = np.array([float(v) for v in tok[1:]])
        else:
            sup.append((int(tok[0]), float(tok[1]), float(tok[2])))
    return deg, knots, sup


def test_worked_example_supports():
    p, t, sup = _read_worked()
    assert bspline.n_basis(t, p) == len(sup) == 7
    x = np.linspace(0, 5, 5001)
    for (i, lo, hi) in sup:
        v = bspline.basis(t, p, i - 1, x, 0)
        nz = x[v > 1e-14]
        assert abs(nz.min() - lo) < 2e-3 and abs(nz.max() - hi) < 2e-3, (i, nz.min(), nz.max())
    # B_i + B_{i+1} + B_{i+2} = 1 on the element [i-1, i] (1-based i)
    for i in range(1, 6):
        xe = np.linspace(i - 1, i, 33)[1:-1]
        s = sum(bspline.basis(t, p, i - 1 + k, xe, 0) for k in range(3))
        assert np.allclose(s, 1.0, atol=1e-14)


def _closed_form_rows():
    rows = {}
    for line in open(os.path.join(GOLD, 'closed_form_rows.txt')):
        if line.startswith('#') or not line.strip():
            continue
        tok = line.split()
        rows[(tok[0], int(tok[1]))] = (tok[2], float(tok[3]), np.array([float(v) for v in tok[4:]]))
    return rows


@pytest.mark.parametrize('p', [2, 3])
def test_closed_form_interior_rows(p):
    """Interior rows of the 1D Galerkin and PW matrices equal the closed-form
    integrals of uniform B-spline pieces (independent of Cox--de Boor)."""
    rows = _closed_form_rows()
    ne = 16
    h = 1.0 / ne
    i = ne // 2
    mats = {
        'galerkin_mass': systems.mass(systems.Axis(ne, p, p + 1, 'galerkin')),
        'galerkin_lap': systems.laplace(systems.Axis(ne, p, p + 1, 'galerkin')),
        'pw_mass': systems.mass(systems.Axis(ne, p, p + 1, 'pw')),
        'pw_lap': systems.laplace(systems.Axis(ne, p, p + 1, 'pw')),
    }
    for name, M in mats.items():
        kind, den, ent = rows[(name, p)]
        ref = ent * h / den if kind == 'h' else ent / (h * den)
        got = M[i, i - p: i + p + 1]
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), (name, got, ref)
        # nothing outside the band
        assert np.all(M[i, :i - p] == 0) and np.all(M[i, i + p + 1:] == 0)


def test_integral_closed_form():
    """int_0^1 B_j = (t_{j+p+1} - t_j) / (p+1) on any knot vector."""
    for p in (2, 3):
        t = _nonuniform_knots(5, p, 3)
        ax = systems.Axis(5, p, p + 1, 'galerkin', knots=t)
        x, w, _ = ax.points()
        V = systems.eval_matrix(ax, 0)
        got = w @ V
        ref = np.array([(t[j + p + 1] - t[j]) / (p + 1) for j in range(ax.n)])
        assert np.allclose(got, ref, rtol=1e-13)
