"""1D Poisson problem -u'' = f with zero Dirichlet rows (oracle; test
infrastructure only).

Sec. 4.3, Eq. (7) (taken here in 1D, Dirichlet at both ends): the operator
rows are int T_i (-B_j'') (non-integrated form), the RHS int T_i f, and the
Dirichlet rows are replaced by identity rows with zero RHS.  Solved with
pivoted dense LU.
"""
import numpy as np

from . import bspline, quadrature, systems


def assemble(ax, f):
    """Operator K = -(int T_i B_j'') with Dirichlet rows, and RHS b = int T_i f."""
    K = -systems.laplace(ax)
    K = systems.dirichlet_rows(K, ax)
    x, _, _ = ax.points()
    b = systems.rhs_1d(ax, f(x))
    return K, b


def solve(ax, f):
    K, b = assemble(ax, f)
    return np.linalg.solve(K, b)


def l2_error(ax, u, exact, nq_err=8):
    """|| sum_j u_j B_j - exact ||_L2 with an nq_err-point Gauss rule per element."""
    err2 = 0.0
    br = bspline.unique_knots(ax.knots)
    for e in range(len(br) - 1):
        x, w = quadrature.map_rule(nq_err, br[e], br[e + 1])
        uh = bspline.basis_matrix(ax.knots, ax.p, x, 0) @ u
        err2 += float(np.sum(w * (uh - exact(x)) ** 2))
    return np.sqrt(err2)


def max_error(ax, u, exact, per_elem=16):
    br = bspline.unique_knots(ax.knots)
    x = np.concatenate([np.linspace(br[e], br[e + 1], per_elem) for e in range(len(br) - 1)])
    uh = bspline.basis_matrix(ax.knots, ax.p, x, 0) @ u
    return float(np.max(np.abs(uh - exact(x))))
