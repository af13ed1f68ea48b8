"""Multi-dimensional Poisson problem -Lap u = f with zero Dirichlet rows
(oracle; test infrastructure only).

Sec. 4.3 (Eq. 7) tests -Lap u = f with the products of 1D tests (B-splines,
or the piece-wise constants of Sec. 3 direction by direction) and keeps the
operator in its non-integrated form.  In d dimensions the tested operator is
the sum over axes a of (-int T B'' along a) times (int T B along every other
axis); it is not a single Kronecker product, so Sec. 4.3 hands it to a
general sparse direct solver.  Every row whose multi-index touches the
boundary of any axis is replaced by the identity row with a zero right-hand
side (Sec. 4.3).  The oracle assembles that matrix densely and solves it with
pivoted dense LU (tiny and small meshes), or with a sparse direct solve
(medium meshes).
"""
import numpy as np

from . import bspline, quadrature, systems, tensor


def raw_mats(ax):
    """(mass, laplace) 1D matrices with zero rows at Dirichlet rows:
    int T_i B_j and int T_i B_j'' over the axis' quadrature points."""
    W = systems.test_matrix(ax)
    return W @ systems.eval_matrix(ax, 0), W @ systems.eval_matrix(ax, 2)


def boundary_mask(axes):
    """Boolean tensor (shape (n_z, n_y, n_x)[-d:]): True where any axis index is
    not an unknown of its axis."""
    d = len(axes)
    mask = np.zeros(tuple(ax.n for ax in reversed(axes)), dtype=bool)
    for a, ax in enumerate(axes):
        free = np.zeros(ax.n, dtype=bool)
        free[list(ax.rows())] = True
        shape = [1] * d
        shape[d - 1 - a] = ax.n
        mask |= ~free.reshape(shape)
    return mask


def operator_terms(axes):
    """The per-axis factors of the operator: for each axis a the list
    [-L_a along a, M_b along b != a] (1D matrices with zero Dirichlet rows)."""
    mats = [raw_mats(ax) for ax in axes]
    terms = []
    for a in range(len(axes)):
        terms.append([(-mats[b][1] if b == a else mats[b][0]) for b in range(len(axes))])
    return terms


def assemble(axes):
    """Dense d-D Poisson matrix (x-fastest flattening) with identity rows on the
    boundary."""
    K = sum(tensor.kron_dense(t) for t in operator_terms(axes))
    mask = boundary_mask(axes).ravel()
    K[mask, :] = 0.0
    K[mask, mask] = 1.0
    return K


def assemble_sparse(axes):
    """The same matrix as a scipy CSR matrix (medium meshes)."""
    import scipy.sparse as sp
    K = None
    for t in operator_terms(axes):
        term = sp.csr_matrix(np.ones((1, 1)))
        for M in reversed(t):
            term = sp.kron(term, sp.csr_matrix(M), format='csr')
        K = term if K is None else K + term
    mask = boundary_mask(axes).ravel()
    keep = sp.diags((~mask).astype(np.float64))
    K = (keep @ K + sp.diags(mask.astype(np.float64))).tocsr()
    K.eliminate_zeros()
    return K


def apply(axes, u):
    """K u by per-axis contractions (any size): sum_a (-L_a) (x) M_others on
    rows off the boundary, u itself on the boundary rows."""
    u = np.asarray(u, dtype=np.float64)
    r = np.zeros_like(u)
    for t in operator_terms(axes):
        v = u
        for a, M in enumerate(t):
            v = tensor.along(M, v, a)
        r += v
    mask = boundary_mask(axes)
    r[mask] = u[mask]
    return r


def apply_abs(axes, u):
    """sum_a |-L_a (x) M_others| |u| off the boundary, |u| on it: an upper
    bound on |K| |u| and the scale of the rounding in the per-axis evaluation
    of K u; used for normwise backward errors."""
    u = np.abs(np.asarray(u, dtype=np.float64))
    r = np.zeros_like(u)
    for t in operator_terms(axes):
        v = u
        for a, M in enumerate(t):
            v = tensor.along(np.abs(M), v, a)
        r += v
    mask = boundary_mask(axes)
    r[mask] = u[mask]
    return r


def backward_error(axes, u, b):
    """Normwise backward error ||b - K u|| / (||apply_abs(u)|| + ||b||) of an
    approximate solution u (2-norms)."""
    r = np.asarray(b, dtype=np.float64) - apply(axes, u)
    return float(np.linalg.norm(r) / (np.linalg.norm(apply_abs(axes, u)) + np.linalg.norm(b)))


def rhs(axes, f_grid):
    """b = T f on the tensor quadrature grid (zero on the boundary rows)."""
    return tensor.rhs_source(axes, f_grid)


def solve(axes, b, sparse=False):
    """u with K u = b."""
    b = np.asarray(b, dtype=np.float64)
    if sparse:
        import scipy.sparse.linalg as spl
        return spl.spsolve(assemble_sparse(axes).tocsc(), b.ravel()).reshape(b.shape)
    return np.linalg.solve(assemble(axes), b.ravel()).reshape(b.shape)


def l2_error(axes, u, exact, nq_err=6):
    """|| sum_j u_j B_j - exact ||_L2 over the box, an nq_err^d Gauss rule per
    d-D element; `exact` takes a list of coordinate arrays (x first) that
    broadcast against the (z, y, x)-ordered grid."""
    d = len(axes)
    xs, ws, Bs = [], [], []
    for ax in axes:
        br = bspline.unique_knots(ax.knots)
        x = []
        w = []
        for e in range(len(br) - 1):
            xe, we = quadrature.map_rule(nq_err, br[e], br[e + 1])
            x.append(xe)
            w.append(we)
        x = np.concatenate(x)
        xs.append(x)
        ws.append(np.concatenate(w))
        Bs.append(bspline.basis_matrix(ax.knots, ax.p, x, 0))
    uh = np.asarray(u, dtype=np.float64)
    for a in range(d):
        uh = tensor.along(Bs[a], uh, a)
    coords = []
    for a in range(d):
        shape = [1] * d
        shape[d - 1 - a] = len(xs[a])
        coords.append(xs[a].reshape(shape))
    wt = np.ones([1] * d)
    for a in range(d):
        shape = [1] * d
        shape[d - 1 - a] = len(ws[a])
        wt = wt * ws[a].reshape(shape)
    return float(np.sqrt(np.sum(wt * (uh - exact(coords)) ** 2)))
