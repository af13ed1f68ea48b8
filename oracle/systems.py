"""One-dimensional Galerkin and piece-wise-constant systems (oracle; test
infrastructure only).

Sec. 2 writes the B-spline-tested system entry by entry as
``int B_i F(B_j)`` (not integrated by parts) and the PW-tested Petrov--Galerkin
system as ``int I_i F(B_j)``; Sec. 4.1 lists the RHS generation loops, where
the PW loop multiplies the quadrature weight by 1.0 instead of a test
function.  Sec. 4.3: zero Dirichlet rows are replaced by identity rows with a
zero right-hand side.

An ``Axis`` bundles the 1D data of one coordinate direction.  Rows of every
matrix are test functions, columns trial functions; all entries are sums
over the quadrature points of the axis' point set, in increasing x.
"""
from dataclasses import dataclass, field

import numpy as np

from . import bspline, quadrature


@dataclass
class Axis:
    n_elem: int
    p: int
    nq: int
    test: str = 'pw'          # 'pw', 'galerkin' or 'refined'
    bc: str = 'none'          # 'none' or 'dirichlet0'
    knots: np.ndarray = field(default=None)
    refine: int = 4           # 'refined': elements of the test space per trial element

    def __post_init__(self):
        if self.knots is None:
            self.knots = bspline.open_uniform_knots(self.n_elem, self.p)
        self.knots = np.asarray(self.knots, dtype=np.float64)

    @property
    def n(self):
        return bspline.n_basis(self.knots, self.p)

    def pieces(self):
        if self.test == 'pw':
            return quadrature.pw_points(self.knots, self.p, self.nq, self.bc)
        if self.test == 'refined':
            return quadrature.refined_points(self.knots, self.p, self.nq, self.refine)
        return quadrature.galerkin_points(self.knots, self.p, self.nq)

    def points(self):
        """Flat quadrature points, weights, and owning element/cell index."""
        return quadrature.flat_points(self.pieces())

    def rows(self):
        """Row index (= unknown index) of each test function."""
        return quadrature.unknowns(self.n, self.bc)


def eval_matrix(ax, deriv=0):
    """V[q, j] = d^deriv B_j(x_q) on the axis' quadrature points."""
    x, _, _ = ax.points()
    return bspline.basis_matrix(ax.knots, ax.p, x, deriv)


def test_matrix(ax):
    """W[i, q]: quadrature weight times test function i at point q.

    Galerkin: W[i, q] = w_q B_i(x_q) (Sec. 4.1 standard loop).
    PW:       W[i, q] = w_q if q lies in the cell paired with row i, else 0
              (Sec. 4.1 PW loop: weight times 1.0).
    Refined: W[i, q] = w_q sum_{m in J_i} B^_m(x_q) with B^ the B-splines of the
              test space refined r times and J_i the refined functions whose
              Greville abscissa lies in cell i (Sec. 2: summing rows of the
              refined-tested system; the limit r -> inf is the PW test).
    Rows that are not unknowns (Dirichlet rows) stay zero: their RHS is 0.
    """
    x, w, owner = ax.points()
    n = ax.n
    W = np.zeros((n, len(x)), dtype=np.float64)
    rows = ax.rows()
    if ax.test == 'galerkin':
        for i in rows:
            W[i, :] = w * bspline.basis(ax.knots, ax.p, i, x, 0)
    elif ax.test == 'refined':
        tr = quadrature.refined_knots(ax.knots, ax.refine)
        sets = quadrature.refined_sets(ax.knots, ax.p, ax.refine, ax.bc)
        for k, i in enumerate(rows):
            W[i, :] = w * sum(bspline.basis(tr, ax.p, m, x, 0) for m in sets[k])
    else:
        for k, i in enumerate(rows):
            W[i, :] = np.where(owner == k, w, 0.0)
    return W


def dirichlet_rows(S, ax):
    """Replace every non-unknown row by the identity row (Sec. 4.3)."""
    S = S.copy()
    free = set(ax.rows())
    for i in range(S.shape[0]):
        if i not in free:
            S[i, :] = 0.0
            S[i, i] = 1.0
    return S


def mass(ax):
    """int T_i B_j: Galerkin mass or PW 'mass' (Sec. 4.1 first 1D ADS system)."""
    S = test_matrix(ax) @ eval_matrix(ax, 0)
    return dirichlet_rows(S, ax)


def laplace(ax):
    """int T_i B_j'' (not integrated by parts, Sec. 2)."""
    S = test_matrix(ax) @ eval_matrix(ax, 2)
    return dirichlet_rows(S, ax)


def laplace_ibp(ax):
    """-int B_i' B_j' (Galerkin only, integrated by parts; Sec. 1 equality)."""
    if ax.test != 'galerkin':
        raise ValueError('IBP form exists only for B-spline tests')
    x, w, _ = ax.points()
    D = bspline.basis_matrix(ax.knots, ax.p, x, 1)
    S = -(D.T * w) @ D
    return dirichlet_rows(S, ax)


def rhs_1d(ax, f_values):
    """b_i = sum_q W[i, q] f(x_q) for f sampled on the axis' points."""
    return test_matrix(ax) @ np.asarray(f_values, dtype=np.float64)
