"""Pins of the multi-D Poisson oracle (Sec. 4.3) against what does not come
from the oracle's own Kronecker assembly: point-by-point brute-force
assembly, manufactured solutions and their convergence rates, symmetry of
the B-spline-tested system, and the 1D problem it must reduce to."""
import numpy as np
import pytest

from oracle import poisson, poisson_nd, systems, tensor


def _axes(ns, p, test, nq=None):
    return [systems.Axis(n, p, nq or p + 1, test, 'dirichlet0') for n in ns]


def _f_grid(axes, k):
    d = len(axes)
    g = np.ones([1] * d)
    for a, ax in enumerate(axes):
        x = ax.points()[0]
        shape = [1] * d
        shape[d - 1 - a] = len(x)
        g = g * np.sin(k[a] * np.pi * x).reshape(shape)
    return g * np.pi ** 2 * sum(kk * kk for kk in k)


def _exact(k):
    def f(coords):
        r = 1.0
        for a, x in enumerate(coords):
            r = r * np.sin(k[a] * np.pi * x)
        return r
    return f


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
@pytest.mark.parametrize('ns,p', [((3, 4), 2), ((2, 3), 3), ((2, 2, 3), 2)])
def test_matches_brute_force(test, ns, p):
    """Kronecker assembly == point-by-point d-D assembly of -Lap with the
    boundary identity rows."""
    axes = _axes(ns, p, test)
    lap = tensor.brute_force_system(axes, 1.0) - tensor.brute_force_system(axes, 0.0)
    Kb = -lap
    mask = poisson_nd.boundary_mask(axes).ravel()
    Kb[mask, :] = 0.0
    Kb[mask, mask] = 1.0
    K = poisson_nd.assemble(axes)
    assert np.max(np.abs(K - Kb)) < 1e-10 * np.max(np.abs(K))


def test_boundary_mask_counts():
    axes = _axes((4, 5, 3), 2, 'pw')
    m = poisson_nd.boundary_mask(axes)
    n = [ax.n for ax in axes]
    interior = (n[0] - 2) * (n[1] - 2) * (n[2] - 2)
    assert m.shape == (n[2], n[1], n[0])
    assert int((~m).sum()) == interior
    assert m[0, 3, 3] and m[2, 0, 1] and m[1, 2, n[0] - 1] and not m[1, 1, 1]


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_sparse_and_apply_agree_with_dense(test):
    axes = [systems.Axis(5, 3, 4, test, 'dirichlet0'), systems.Axis(4, 3, 4, test, 'dirichlet0'),
            systems.Axis(3, 3, 4, test, 'dirichlet0')]
    K = poisson_nd.assemble(axes)
    assert np.array_equal(poisson_nd.assemble_sparse(axes).toarray(), K)
    u = np.random.default_rng(1).standard_normal(tuple(ax.n for ax in reversed(axes)))
    assert np.max(np.abs(poisson_nd.apply(axes, u).ravel() - K @ u.ravel())) < 1e-12 * np.max(np.abs(K))


def test_galerkin_interior_block_symmetric_positive():
    axes = _axes((6, 5), 3, 'galerkin')
    K = poisson_nd.assemble(axes)
    free = ~poisson_nd.boundary_mask(axes).ravel()
    Kii = K[np.ix_(free, free)]
    assert np.max(np.abs(Kii - Kii.T)) < 1e-10 * np.max(np.abs(Kii))
    assert np.linalg.eigvalsh(0.5 * (Kii + Kii.T)).min() > 0


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_tensor_product_trial_recombines_1d_factors(test):
    """On a tensor product u = w(y) v(x) the 2D operator acts as
    (M_y w)(-L_x v) + (-L_y w)(M_x v) on the rows off the boundary: the 1D
    factors recombine exactly (Sec. 3 builds the 2D system from them)."""
    ax, ay = _axes((7, 6), 2, test)
    Mx, Lx = poisson_nd.raw_mats(ax)
    My, Ly = poisson_nd.raw_mats(ay)
    rng = np.random.default_rng(2)
    v = rng.standard_normal(ax.n)
    w = rng.standard_normal(ay.n)
    u = np.outer(w, v)                 # (n_y, n_x), x fastest
    got = poisson_nd.apply([ax, ay], u)
    want = np.outer(My @ w, -Lx @ v) + np.outer(-Ly @ w, Mx @ v)
    mask = poisson_nd.boundary_mask([ax, ay])
    assert np.max(np.abs(got[~mask] - want[~mask])) < 1e-10 * np.max(np.abs(want))


@pytest.mark.parametrize('test,p,lo', [('pw', 2, 1.9), ('pw', 3, 3.8), ('galerkin', 2, 2.9), ('galerkin', 3, 3.8)])
def test_manufactured_convergence_2d(test, p, lo):
    """u = sin(pi x) sin(2 pi y): L2 error rates under h-refinement (PW with
    even p loses one order, as in 1D)."""
    k = (1, 2)
    errs = []
    for ne in (4, 8, 16):
        axes = _axes((ne, ne), p, test)
        b = poisson_nd.rhs(axes, _f_grid(axes, k))
        u = poisson_nd.solve(axes, b)
        errs.append(poisson_nd.l2_error(axes, u, _exact(k)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > lo), rates
    assert errs[-1] < 6e-3


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_manufactured_3d(test):
    k = (1, 1, 1)
    errs = []
    for ne in (3, 6):
        axes = _axes((ne, ne, ne), 3, test)
        b = poisson_nd.rhs(axes, _f_grid(axes, k))
        u = poisson_nd.solve(axes, b)
        errs.append(poisson_nd.l2_error(axes, u, _exact(k), nq_err=4))
    assert errs[1] < errs[0] / 8
    assert errs[1] < 5e-3


def test_one_axis_mesh_reduces_to_1d_problem():
    """With d = 1 the assembled matrix is the 1D Poisson system of Sec. 4.3."""
    for test in ('pw', 'galerkin'):
        ax = systems.Axis(9, 3, 4, test, 'dirichlet0')
        K1, _ = poisson.assemble(ax, lambda x: np.sin(np.pi * x))
        assert np.max(np.abs(poisson_nd.assemble([ax]) - K1)) < 1e-12 * np.max(np.abs(K1))


def test_sparse_solve_matches_dense():
    axes = _axes((6, 5), 3, 'pw')
    b = poisson_nd.rhs(axes, _f_grid(axes, (2, 1)))
    assert np.max(np.abs(poisson_nd.solve(axes, b, sparse=True) - poisson_nd.solve(axes, b))) < 1e-12


def test_backward_error_of_exact_and_perturbed_solutions():
    """The dense solve is backward stable (error near eps); perturbing the
    solution by a relative 1e-6 raises the backward error to about that."""
    axes = _axes((7, 6), 3, 'pw')
    b = poisson_nd.rhs(axes, _f_grid(axes, (1, 1)))
    u = poisson_nd.solve(axes, b)
    assert poisson_nd.backward_error(axes, u, b) < 1e-15
    v = u * (1 + 1e-6 * np.random.default_rng(4).standard_normal(u.shape))
    eta = poisson_nd.backward_error(axes, v, b)
    assert 1e-8 < eta < 1e-5
    mask = poisson_nd.boundary_mask(axes).ravel()
    Kabs = sum(np.abs(tensor.kron_dense(t)) for t in poisson_nd.operator_terms(axes))
    Kabs[mask, :] = 0.0
    Kabs[mask, mask] = 1.0
    got = poisson_nd.apply_abs(axes, u).ravel()
    assert np.allclose(got, Kabs @ np.abs(u.ravel()), rtol=1e-12)
    assert np.all(got >= np.abs(poisson_nd.assemble(axes)) @ np.abs(u.ravel()) * (1 - 1e-12))
