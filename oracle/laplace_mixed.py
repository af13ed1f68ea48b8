"""Laplace problem with zero Dirichlet and Neumann boundary conditions
(oracle; test infrastructure only).

Sec. 4.3 (the mixed-boundary example): -Lap u = RHS with u = 0 on Gamma_D and
du/dn = G on Gamma_N.  With C^1 trial B-splines the weak form can be
integrated back by parts on the discrete level, so the tested system keeps
the non-integrated operator plus a boundary term on the Neumann part:
  -int T Lap u + int_{Gamma_N} T du/dn = int T RHS + int_{Gamma_N} T G,
tested with products of 1D B-splines (Galerkin) or of 1D cell indicators
(PW); zero Dirichlet rows are replaced by identity rows with zero RHS.

Boundary parts are chosen per axis: a Dirichlet axis holds u = 0 at both of
its ends, a Neumann axis carries the flux data on both of its end faces.  On
a Neumann axis every coefficient is an unknown and the 1D factor of the
operator is -C + E with E_ij = T_i(b) B_j'(b) - T_i(a) B_j'(a) (outward
normal derivative at the ends a < b of the axis).
"""
import numpy as np

from . import bspline, quadrature, systems, tensor


def test_at(ax, x):
    """Values T_i(x) of every row's test function at one point x of the axis."""
    if ax.test == 'galerkin':
        return bspline.basis_matrix(ax.knots, ax.p, [x], 0)[0]
    c = quadrature.pw_cells(ax.knots, ax.p, ax.bc)
    rows = ax.rows()
    out = np.zeros(ax.n)
    for k in range(len(c) - 1):
        last = k == len(c) - 2
        if c[k] <= x < c[k + 1] or (last and x == c[k + 1]):
            out[rows[k]] = 1.0
            break
    return out


def boundary_matrix(ax):
    """E = T(b) B'(b)^T - T(a) B'(a)^T: the Neumann boundary term of one axis."""
    a, b = ax.knots[0], ax.knots[-1]
    da = bspline.basis_matrix(ax.knots, ax.p, [a], 1)[0]
    db = bspline.basis_matrix(ax.knots, ax.p, [b], 1)[0]
    return np.outer(test_at(ax, b), db) - np.outer(test_at(ax, a), da)


def _check(axes, neumann):
    assert len(axes) == len(neumann)
    for ax, nm in zip(axes, neumann):
        assert ax.bc == ('none' if nm else 'dirichlet0')
    assert not all(neumann), 'at least one Dirichlet axis (otherwise K is singular)'


def operator_terms(axes, neumann):
    """Per axis a: [(-C_a + E_a if Neumann) along a, M_b along b != a]."""
    _check(axes, neumann)
    from .poisson_nd import raw_mats
    mats = [raw_mats(ax) for ax in axes]
    terms = []
    for a in range(len(axes)):
        La = -mats[a][1] + (boundary_matrix(axes[a]) if neumann[a] else 0.0)
        terms.append([(La if b == a else mats[b][0]) for b in range(len(axes))])
    return terms


def assemble(axes, neumann):
    """Dense matrix with identity rows where a Dirichlet-axis index is an end."""
    from .poisson_nd import boundary_mask
    K = sum(tensor.kron_dense(t) for t in operator_terms(axes, neumann))
    mask = boundary_mask(axes).ravel()
    K[mask, :] = 0.0
    K[mask, mask] = 1.0
    return K


def assemble_sparse(axes, neumann):
    """The same matrix as a scipy CSR matrix (medium meshes)."""
    import scipy.sparse as sp
    from .poisson_nd import boundary_mask
    K = None
    for t in operator_terms(axes, neumann):
        term = sp.csr_matrix(np.ones((1, 1)))
        for M in reversed(t):
            term = sp.kron(term, sp.csr_matrix(M), format='csr')
        K = term if K is None else K + term
    mask = boundary_mask(axes).ravel()
    K = (sp.diags((~mask).astype(np.float64)) @ K + sp.diags(mask.astype(np.float64))).tocsr()
    K.eliminate_zeros()
    return K


def apply(axes, neumann, u):
    from .poisson_nd import boundary_mask
    u = np.asarray(u, dtype=np.float64)
    r = np.zeros_like(u)
    for t in operator_terms(axes, neumann):
        v = u
        for a, M in enumerate(t):
            v = tensor.along(M, v, a)
        r += v
    mask = boundary_mask(axes)
    r[mask] = u[mask]
    return r


def face_rhs(axes, axis, side, g):
    """int over the end face (side 0: a, 1: b) of `axis` of T G, for G sampled
    on the tensor grid of the other axes' quadrature points (x fastest):
    the 1D tests of the other axes applied to g, times T_axis(end)."""
    d = len(axes)
    others = [a for a in range(d) if a != axis]
    r = np.asarray(g, dtype=np.float64).reshape([len(axes[a].points()[0]) for a in reversed(others)])
    for k, a in enumerate(others):
        r = tensor.along(systems.test_matrix(axes[a]), r, k)
    ax = axes[axis]
    t = test_at(ax, ax.knots[-1] if side else ax.knots[0])
    return np.expand_dims(r, d - 1 - axis) * t.reshape([ax.n if b == axis else 1 for b in reversed(range(d))])


def rhs(axes, neumann, f_grid, faces):
    """int T f + sum over the Neumann faces of int T G; faces maps (axis, side)
    to the G samples of that face.  Dirichlet rows are zero."""
    from .poisson_nd import boundary_mask
    b = tensor.rhs_source(axes, f_grid)
    for (axis, side), g in faces.items():
        assert neumann[axis]
        b = b + face_rhs(axes, axis, side, g)
    b[boundary_mask(axes)] = 0.0
    return b


def solve(axes, neumann, b, sparse=False):
    b = np.asarray(b, dtype=np.float64)
    if sparse:
        import scipy.sparse.linalg as spl
        return spl.spsolve(assemble_sparse(axes, neumann).tocsc(), b.ravel()).reshape(b.shape)
    return np.linalg.solve(assemble(axes, neumann), b.ravel()).reshape(b.shape)
