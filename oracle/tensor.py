"""Tensor-product (d = 1, 2, 3) evaluation, testing and the alternating-
directions (ADS) Kronecker solve (oracle; test infrastructure only).

Sec. 3 builds the 2D system from products B^x B^y of 1D functions and
replaces the tests direction by direction with products of indicators;
Sec. 4.1 does the same in 3D and solves the mass matrix Mx (x) My (x) Mz as
three 1D systems with multiple right-hand sides.

Array convention: coefficient and RHS tensors are C-ordered with x fastest,
shape (n_z, n_y, n_x) in 3D, (n_y, n_x) in 2D, (n_x,) in 1D.  ``axes[0]`` is
x, ``axes[1]`` y, ``axes[2]`` z, so axis a lives in array dimension
ndim - 1 - a.
"""
import itertools

import numpy as np

from . import bspline, systems


def along(mat, arr, a):
    """Contract matrix ``mat`` (m x k) with tensor ``arr`` along coordinate a."""
    dim = arr.ndim - 1 - a
    out = np.tensordot(mat, arr, axes=([1], [dim]))   # new axis first
    return np.moveaxis(out, 0, dim)


def values_at_points(axes, u, derivs):
    """d^derivs[a] u / dx_a^... evaluated on the tensor grid of quadrature points:
    sum_j u_j prod_a d^{derivs[a]} B_{j_a}(x_{q_a})."""
    v = np.asarray(u, dtype=np.float64)
    for a, ax in enumerate(axes):
        v = along(systems.eval_matrix(ax, derivs[a]), v, a)
    return v


def heat_integrand(axes, u, dt):
    """u + dt * Laplacian(u) at every tensor quadrature point (Sec. 4.2, Eq. (6)
    with F = Laplacian and no source)."""
    d = len(axes)
    v = values_at_points(axes, u, [0] * d)
    for a in range(d):
        der = [0] * d
        der[a] = 2
        v = v + dt * values_at_points(axes, u, der)
    return v


def test_points(axes, v):
    """r = sum over the tensor quadrature grid of (product of 1D test weights) * v."""
    r = np.asarray(v, dtype=np.float64)
    for a, ax in enumerate(axes):
        r = along(systems.test_matrix(ax), r, a)
    return r


def rhs_heat_quadrature(axes, u, dt):
    """Explicit-step RHS by quadrature: T(u + dt Lap u) (tests at points)."""
    return test_points(axes, heat_integrand(axes, u, dt))


def rhs_source(axes, f_grid):
    """L2-projection / source RHS b = T f for f sampled on the tensor grid."""
    return test_points(axes, f_grid)


def mass_mats(axes):
    return [systems.mass(ax) for ax in axes]


def lap_mats(axes):
    return [systems.laplace(ax) for ax in axes]


def apply_heat_system(axes, u, dt, masses=None, laps=None):
    """Same RHS from the assembled 1D systems: (prod mass) u + dt sum_a
    (lap in direction a, mass elsewhere) u  (Sec. 3 tensor structure)."""
    masses = mass_mats(axes) if masses is None else masses
    laps = lap_mats(axes) if laps is None else laps
    u = np.asarray(u, dtype=np.float64)
    d = len(axes)
    r = u
    for a in range(d):
        r = along(masses[a], r, a)
    for a in range(d):
        t = u
        for b in range(d):
            t = along(laps[b] if b == a else masses[b], t, b)
        r = r + dt * t
    return r


def ads_solve(masses, r):
    """Solve (M_z (x) M_y (x) M_x) u = r as one batch of 1D systems per
    direction (Sec. 4.1), each by pivoted dense LU (numpy.linalg.solve)."""
    u = np.asarray(r, dtype=np.float64)
    for a, M in enumerate(masses):
        dim = u.ndim - 1 - a
        moved = np.moveaxis(u, dim, 0)
        shp = moved.shape
        sol = np.linalg.solve(M, moved.reshape(shp[0], -1)).reshape(shp)
        u = np.moveaxis(sol, 0, dim)
    return u


def kron_dense(mats_by_axis):
    """Dense d-D matrix of the operator that applies mats_by_axis[a] along axis a,
    for the x-fastest flattening (z slowest)."""
    K = np.ones((1, 1))
    for M in reversed(mats_by_axis):   # z first (slowest), x last (fastest)
        K = np.kron(K, M)
    return K


def brute_force_system(axes, dt):
    """Dense d-D system assembled point by point on the d-D quadrature grid:
    S[row, col] = sum_points (prod_a test weight_a) * (B_col + dt Lap B_col)(point),
    with the d-D trial function B_col = prod_a B_{j_a}(x_a) evaluated as a
    product of 1D Cox--de Boor values at each d-D point and
    Lap B_col = sum_a B''_{j_a} prod_{b != a} B_{j_b}.  Tiny meshes only."""
    d = len(axes)
    pts = [ax.points()[0] for ax in axes]
    Ws = [systems.test_matrix(ax) for ax in axes]
    ns = [ax.n for ax in axes]
    N = int(np.prod(ns))

    def flat(idx):                   # idx = (i_x, i_y, i_z) -> x-fastest index
        k = 0
        for a in reversed(range(d)):
            k = k * ns[a] + idx[a]
        return k

    S = np.zeros((N, N))
    for col in itertools.product(*[range(n) for n in ns]):
        vals = [[bspline.basis(axes[a].knots, axes[a].p, col[a], pts[a], m) for m in (0, 2)]
                for a in range(d)]
        c = flat(col)
        for qs in itertools.product(*[range(len(x)) for x in pts]):
            b0 = [vals[a][0][qs[a]] for a in range(d)]
            b2 = [vals[a][1][qs[a]] for a in range(d)]
            f = float(np.prod(b0))
            for a in range(d):
                f += dt * b2[a] * float(np.prod([b0[b] for b in range(d) if b != a]))
            if f == 0.0:
                continue
            # test weights of every row at this point, x-fastest flattening
            wrow = np.ones(1)
            for a in reversed(range(d)):
                wrow = np.kron(wrow, Ws[a][:, qs[a]])
            S[:, c] += wrow * f
    return S
