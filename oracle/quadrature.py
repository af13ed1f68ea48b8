"""Quadrature rules, Greville abscissae and piece-wise-constant test cells
(oracle; test infrastructure only).

Sec. 2: any quadrature exact for the integrand may be used; points and
weights are mapped to each element with the Jacobian len/2.  Sec. 4.1:
standard Gauss quadrature per element.

PW test cells (Sec. 2, closing paragraphs: N_x linearly independent
indicator functions, otherwise the factorization breaks).  The paper leaves
the choice of intervals open.  Reading adopted here (stated once, used
everywhere): the cells are bounded by the midpoints between consecutive
Greville abscissae of the unknowns, with the domain ends as outer bounds;
cell k is paired with the k-th unknown.  Each cell is split at the knots
into polynomial pieces, and every piece gets its own nq-point Gauss rule.
"""
import numpy as np

from . import bspline


def gauss_legendre(nq):
    """nq-point Gauss--Legendre rule on [-1, 1] (numpy's leggauss)."""
    xg, wg = np.polynomial.legendre.leggauss(nq)
    return xg.astype(np.float64), wg.astype(np.float64)


def map_rule(nq, a, b):
    """Gauss rule mapped affinely to [a, b]; weights carry Jac = (b-a)/2."""
    xg, wg = gauss_legendre(nq)
    jac = 0.5 * (b - a)
    return a + jac * (xg + 1.0), jac * wg


def greville(t, p):
    """Greville abscissae xi_j = (t_{j+1} + ... + t_{j+p}) / p."""
    n = bspline.n_basis(t, p)
    return np.array([sum(t[j + 1: j + p + 1]) / p for j in range(n)], dtype=np.float64)


def unknowns(n, bc):
    """Indices of the free coefficients along one axis.

    bc = 'none': all n; bc = 'dirichlet0': the first and last coefficients are
    held at zero (their rows are replaced by identity rows, Sec. 4.3)."""
    if bc == 'none':
        return list(range(n))
    if bc == 'dirichlet0':
        return list(range(1, n - 1))
    raise ValueError(bc)


def pw_cells(t, p, bc):
    """Break points c_0 < c_1 < ... < c_m of the PW test cells (m = #unknowns)."""
    xi = greville(t, p)
    idx = unknowns(bspline.n_basis(t, p), bc)
    a, b = t[0], t[-1]
    inner = [0.5 * (xi[idx[k]] + xi[idx[k + 1]]) for k in range(len(idx) - 1)]
    # a midpoint that equals a knot up to rounding is that knot (no sliver pieces)
    br = bspline.unique_knots(t)
    tol = 1e-12 * (b - a)
    inner = [min(br, key=lambda k: abs(k - c)) if np.min(np.abs(br - c)) < tol else c for c in inner]
    return np.array([a] + inner + [b], dtype=np.float64)


def split_at_knots(lo, hi, t):
    """Polynomial pieces of [lo, hi]: split at every distinct knot strictly inside."""
    cuts = [k for k in bspline.unique_knots(t) if lo < k < hi]
    pts = [lo] + cuts + [hi]
    return [(pts[i], pts[i + 1]) for i in range(len(pts) - 1)]


def galerkin_points(t, p, nq):
    """Element-wise Gauss points: list of (x, w, element) per element, left to right."""
    br = bspline.unique_knots(t)
    out = []
    for e in range(len(br) - 1):
        x, w = map_rule(nq, br[e], br[e + 1])
        out.append((x, w, e))
    return out


def pw_points(t, p, nq, bc):
    """Piece-wise Gauss points of the PW cells: list of (x, w, cell) per piece."""
    c = pw_cells(t, p, bc)
    out = []
    for k in range(len(c) - 1):
        for (lo, hi) in split_at_knots(c[k], c[k + 1], t):
            x, w = map_rule(nq, lo, hi)
            out.append((x, w, k))
    return out


def refined_knots(t, r):
    """Open knot vector with every element of t split into r equal parts
    (Sec. 2: the test space refined over the same trial functions)."""
    br = bspline.unique_knots(t)
    pts = [br[0]]
    for e in range(len(br) - 1):
        for k in range(1, r + 1):
            pts.append(br[e] + (br[e + 1] - br[e]) * k / r)
    p = sum(1 for x in t if x == t[0]) - 1
    return np.array([br[0]] * p + pts + [br[-1]] * p, dtype=np.float64)


def refined_points(t, p, nq, r):
    """Gauss points of the refined elements: list of (x, w, element) per element."""
    tr = refined_knots(t, r)
    br = bspline.unique_knots(tr)
    out = []
    for e in range(len(br) - 1):
        x, w = map_rule(nq, br[e], br[e + 1])
        out.append((x, w, e))
    return out


def refined_sets(t, p, r, bc):
    """Index sets J_k of the refined test B-splines summed into test k: the
    refined functions whose Greville abscissa lies in PW cell k (cells closed on
    the left, the last one closed on both sides)."""
    tr = refined_knots(t, r)
    g = greville(tr, p)
    c = pw_cells(t, p, bc)
    sets = []
    for k in range(len(c) - 1):
        last = k == len(c) - 2
        sets.append([m for m in range(len(g)) if c[k] <= g[m] < c[k + 1] or (last and g[m] == c[k + 1])])
    return sets


def flat_points(pieces):
    """Concatenate a piece list into flat arrays (x, w, owner) in increasing x."""
    x = np.concatenate([pc[0] for pc in pieces])
    w = np.concatenate([pc[1] for pc in pieces])
    owner = np.concatenate([np.full(len(pc[0]), pc[2], dtype=np.int64) for pc in pieces])
    return x, w, owner
