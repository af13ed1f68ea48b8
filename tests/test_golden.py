"""Degree-of-freedom counts printed in the paper's Tables 1, 1a and 2 equal
(n_elem + p)^d for the oracle's open knot vectors."""
import os

from oracle import bspline

GOLD = os.path.join(os.path.dirname(__file__), 'golden')


def test_nrdof_tables():
    rows = 0
    for line in open(os.path.join(GOLD, 'nrdof.txt')):
        if line.startswith('#') or not line.strip():
            continue
        _, d, p, ne, nrdof = line.split()
        d, p, ne, nrdof = int(d), int(p), int(ne), int(nrdof)
        n = bspline.n_basis(bspline.open_uniform_knots(ne, p), p)
        assert n ** d == nrdof
        rows += 1
    assert rows == 18
