"""Shared helpers for the GPU parity tests: build the oracle's axes for a
library context and compare arrays."""
import numpy as np

from oracle import systems


def oracle_axes(dim, n_elem, p, nq, test, bc='none', refine=4):
    if isinstance(n_elem, int):
        n_elem = [n_elem] * dim
    return [systems.Axis(n_elem[a], p, nq, test, bc, refine=refine) for a in range(dim)]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_abs_rel(a, b):
    """Largest element-wise deviation relative to the largest reference entry."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# the element-wise bound allows ELEMENTWISE_SLACK times the norm-wise
# tolerance: rounding spreads unevenly over the entries (the unstable heat2d
# iteration, for one, concentrates it in its growing top mode), while a single
# wrong coefficient of a large tensor sits orders of magnitude above either
ELEMENTWISE_SLACK = 10.0


def rel_err(a, b):
    """Error measure checked against a tolerance tol: max(rel-L2,
    max-abs / (ELEMENTWISE_SLACK max|ref|)) < tol means rel-L2 < tol and
    max-abs < 10 tol max|ref|, so parity is checked both norm-wise and
    element-wise (a single wrong coefficient can hide in the L2 norm of a
    large tensor, not in the element-wise bound)."""
    return max(rel_l2(a, b), max_abs_rel(a, b) / ELEMENTWISE_SLACK)


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))))


# tolerances (relative L2) stated for the two precisions
TOL = {'fp64': 1e-12, 'fp32r': 1e-5}
