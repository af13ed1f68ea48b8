"""B-spline basis by the Cox--de Boor recursion (oracle; test infrastructure only).

The trial space of Sec. 2, Eq. (2): ``{B_{i,p}}, i = 1..N_x`` with
``N_x = N_e + p`` functions on an open knot vector (the paper's example knot
vector [0 0 0 1 2 3 4 5 5 5] in Sec. 2 has p+1 repeated end knots).  Indices
here are 0-based: function ``j`` lives on knots ``t[j] .. t[j+p+1]``.
"""
import numpy as np


def open_uniform_knots(n_elem, p, a=0.0, b=1.0):
    """Open knot vector with ``n_elem`` uniform elements on [a, b].

    p+1 copies of each end point, interior knots a + k (b-a)/n_elem.
    Length n_elem + 2p + 1, giving n_elem + p basis functions (Sec. 2).
    """
    inner = [a + (b - a) * k / n_elem for k in range(1, n_elem)]
    return np.array([a] * (p + 1) + inner + [b] * (p + 1), dtype=np.float64)


def n_basis(t, p):
    return len(t) - p - 1


def _span_indicator(t, j, x):
    """B_{j,0}: 1 on the half-open span [t_j, t_{j+1}); at the right end of the
    knot vector the last non-empty span is closed so that the basis still sums
    to one at x = b."""
    x = np.asarray(x, dtype=np.float64)
    lo, hi = t[j], t[j + 1]
    val = ((x >= lo) & (x < hi)).astype(np.float64)
    if hi > lo and hi == t[-1]:
        # last non-empty span: include its right end point
        last_nonempty = max(k for k in range(len(t) - 1) if t[k + 1] > t[k])
        if j == last_nonempty:
            val = np.where(x == hi, 1.0, val)
    return val


def _ratio(num, den):
    """Cox--de Boor convention 0/0 = 0 (repeated knots)."""
    return 0.0 if den == 0.0 else num / den


def basis(t, p, j, x, deriv=0):
    """Value of the ``deriv``-th derivative of B_{j,p} at points ``x``.

    Values: B_{j,k} = (x - t_j)/(t_{j+k} - t_j) B_{j,k-1}
                      + (t_{j+k+1} - x)/(t_{j+k+1} - t_{j+1}) B_{j+1,k-1}.
    Derivatives: d^m B_{j,k} = k [ d^{m-1} B_{j,k-1} / (t_{j+k} - t_j)
                                   - d^{m-1} B_{j+1,k-1} / (t_{j+k+1} - t_{j+1}) ].
    Plain recursion, no caching.
    """
    x = np.asarray(x, dtype=np.float64)
    if deriv > p:
        return np.zeros_like(x)
    if deriv > 0:
        left = _ratio(p, t[j + p] - t[j])
        right = _ratio(p, t[j + p + 1] - t[j + 1])
        out = np.zeros_like(x)
        if left != 0.0:
            out = out + left * basis(t, p - 1, j, x, deriv - 1)
        if right != 0.0:
            out = out - right * basis(t, p - 1, j + 1, x, deriv - 1)
        return out
    if p == 0:
        return _span_indicator(t, j, x)
    d1 = t[j + p] - t[j]
    d2 = t[j + p + 1] - t[j + 1]
    out = np.zeros_like(x)
    if d1 != 0.0:
        out = out + (x - t[j]) / d1 * basis(t, p - 1, j, x, 0)
    if d2 != 0.0:
        out = out + (t[j + p + 1] - x) / d2 * basis(t, p - 1, j + 1, x, 0)
    return out


def basis_matrix(t, p, x, deriv=0):
    """Dense matrix V[q, j] = d^deriv B_{j,p}(x_q) for all functions j."""
    x = np.asarray(x, dtype=np.float64)
    n = n_basis(t, p)
    return np.stack([basis(t, p, j, x, deriv) for j in range(n)], axis=1)


def unique_knots(t):
    """Break points (distinct knots) in increasing order."""
    return np.unique(np.asarray(t, dtype=np.float64))
