"""Pins of the oracle's tensor-product layer (Sec. 3, Sec. 4.1): quadrature-grid
RHS against assembled systems, point-by-point d-D brute force against the
Kronecker structure, the ADS solve against a dense pivoted solve."""
import numpy as np
import pytest

from oracle import systems, tensor


def _axes(d, ne, p, test, nq=None):
    nq = p + 1 if nq is None else nq
    return [systems.Axis(ne + a, p, nq, test) for a in range(d)]


@pytest.mark.parametrize('d', [1, 2, 3])
@pytest.mark.parametrize('p', [2, 3])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_quadrature_route_equals_system_route(d, p, test):
    axes = _axes(d, 4, p, test)
    rng = np.random.default_rng(d * 10 + p)
    u = rng.standard_normal([ax.n for ax in reversed(axes)])
    dt = 0.013
    r1 = tensor.rhs_heat_quadrature(axes, u, dt)
    r2 = tensor.apply_heat_system(axes, u, dt)
    assert np.abs(r1 - r2).max() < 1e-13 * np.abs(r2).max()


@pytest.mark.parametrize('d', [2, 3])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_brute_force_matches_kronecker(d, test):
    axes = [systems.Axis(2 + (a % 2), 2, 3, test) for a in range(d)]
    dt = 0.05
    S = tensor.brute_force_system(axes, dt)
    M = tensor.mass_mats(axes)
    L = tensor.lap_mats(axes)
    K = tensor.kron_dense(M)
    for a in range(d):
        K = K + dt * tensor.kron_dense([L[b] if b == a else M[b] for b in range(d)])
    assert np.abs(S - K).max() < 1e-14 * np.abs(K).max() * 10
    # and the operator form agrees with the dense matrix on the x-fastest flattening
    u = np.random.default_rng(1).standard_normal([ax.n for ax in reversed(axes)])
    assert np.allclose(tensor.apply_heat_system(axes, u, dt).ravel(), S @ u.ravel(), atol=1e-14 * np.abs(S).max() * 50)


@pytest.mark.parametrize('d', [1, 2, 3])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_ads_matches_dense_solve(d, test):
    axes = _axes(d, 3, 3, test)
    M = tensor.mass_mats(axes)
    rng = np.random.default_rng(7)
    r = rng.standard_normal([ax.n for ax in reversed(axes)])
    u = tensor.ads_solve(M, r)
    ud = np.linalg.solve(tensor.kron_dense(M), r.ravel())
    assert np.allclose(u.ravel(), ud, rtol=1e-11, atol=1e-11 * np.abs(ud).max())
    # solve(apply_mass(u)) = u
    v = rng.standard_normal(r.shape)
    assert np.allclose(tensor.ads_solve(M, tensor.apply_heat_system(axes, v, 0.0)), v, atol=1e-11)


def test_source_rhs_constant():
    """T 1 = cell lengths (PW) or int B_i (Galerkin), as tensor products."""
    for test in ('pw', 'galerkin'):
        axes = _axes(2, 5, 2, test)
        Q = [len(ax.points()[0]) for ax in axes]
        b = tensor.rhs_source(axes, np.ones((Q[1], Q[0])))
        one = [systems.test_matrix(ax).sum(axis=1) for ax in axes]
        assert np.allclose(b, np.outer(one[1], one[0]), rtol=1e-14)
