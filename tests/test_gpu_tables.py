"""GPU parity of kernel (a) and the folded 1D tables against the oracle:
quadrature point sets, Cox--de Boor basis tables, tested mass / Laplacian
matrices, the 1D Poisson system with Dirichlet rows, non-uniform knots."""
import numpy as np
import pytest

from oracle import bspline, systems
from tests._cases import oracle_axes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


def _ctx(**kw):
    from paper_1910_08535_gb300.igapw import Context
    return Context(**kw)


@pytest.mark.parametrize('p', [2, 3, 4])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
@pytest.mark.parametrize('bc', ['none', 'dirichlet0'])
def test_points_basis_and_matrices_1d(p, test, bc):
    ne = 11
    op = 'poisson' if bc == 'dirichlet0' else 'heat'
    c = _ctx(dim=1, n_elem=ne, degree=p, nq=p + 1, test=test, bc=bc, op=op)
    ax = oracle_axes(1, ne, p, p + 1, test, bc)[0]
    x, w = c.quad_points(0)
    ox, ow, _ = ax.points()
    assert len(x) == len(ox)
    assert np.abs(x - ox).max() < 1e-15 and np.abs(w - ow).max() < 1e-15
    vals, first = c.basis_table(0)
    for d in (0, 1, 2):
        V = bspline.basis_matrix(ax.knots, p, ox, d)
        ref = np.stack([V[np.arange(len(ox)), first + a] for a in range(p + 1)], axis=1)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(vals[:, :, d] - ref).max() < 1e-12 * scale, d
    M = c.assemble_1d(0, 'mass')
    L = c.assemble_1d(0, 'laplace')
    assert np.abs(M - systems.mass(ax)).max() < 1e-14 * np.abs(M).max() * 10
    Lref = systems.laplace(ax)
    if bc == 'dirichlet0':
        Lref[[0, -1]] = 0.0        # the library's tested Laplacian has zero Dirichlet rows
    assert np.abs(L - Lref).max() < 1e-13 * np.abs(L).max()
    if bc == 'dirichlet0':
        K = c.assemble_1d(0, 'poisson')
        Kref = systems.dirichlet_rows(-systems.laplace(ax), ax)
        assert np.abs(K - Kref).max() < 1e-13 * np.abs(K).max()
    c.close()


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_nonuniform_knots(test):
    p, ne = 3, 9
    rng = np.random.default_rng(4)
    inner = np.sort(rng.uniform(0.05, 0.95, ne - 1))
    t = np.concatenate([[0.0] * (p + 1), inner, [1.0] * (p + 1)])
    c = _ctx(dim=1, n_elem=ne, degree=p, nq=p + 1, test=test)
    c.set_knots(0, t)   # row windows start below their first non-zero column where needed
    ax = systems.Axis(ne, p, p + 1, test, knots=t)
    assert np.abs(c.assemble_1d(0, 'mass') - systems.mass(ax)).max() < 1e-13
    x, _ = c.quad_points(0)
    assert np.abs(x - ax.points()[0]).max() < 1e-15


def test_bad_descriptors_rejected():
    from paper_1910_08535_gb300.igapw import IgapwError
    with pytest.raises(IgapwError):
        _ctx(dim=4, n_elem=4, degree=2, nq=3)
    with pytest.raises(IgapwError):
        _ctx(dim=1, n_elem=4, degree=1, nq=3)
    with pytest.raises(IgapwError):
        _ctx(dim=2, n_elem=4, degree=2, nq=3, bc='dirichlet0')
    with pytest.raises(IgapwError):
        _ctx(dim=1, n_elem=4, degree=2, nq=3, op='poisson')    # Poisson without Dirichlet rows is singular
