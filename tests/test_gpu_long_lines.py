"""Long lines (n above ~800 per axis): the split-step kernel and the batched
line solves switch to fewer lines per block with the 1D tables read from
global memory once a line no longer fits shared memory next to them.  Parity
against the oracle at the largest 2D grid of the mixed request stream
(1024 x 1024 elements, cubic), a long 1D line, and columns of 8195 rows (the
y lines of an 8192^2 grid, one column per block)."""
import numpy as np
import pytest

from oracle import heat, tensor
from tests._cases import TOL, oracle_axes, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


def _ctx(**kw):
    from paper_1910_08535_gb300.igapw import Context
    return Context(**kw)


@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_heat_2d_1024_cubic(prec, test):
    from paper_1910_08535_gb300 import igapw, workloads
    ne, p = 1024, 3
    axes = oracle_axes(2, ne, p, p + 1, test)
    u = workloads.normal_coeffs((ne + p, ne + p), seed=4)
    dt = 0.05 / ne ** 2 / 2
    ref = heat.run(axes, u, dt, 3)
    for flags in (0, igapw.IGAPW_FLAG_STEP_RHS_SOLVE):
        c = _ctx(dim=2, n_elem=ne, degree=p, nq=p + 1, test=test, precision=prec, flags=flags)
        ud = c.from_numpy(u)
        c.step(ud, dt, 3)
        got = c.to_numpy(ud)
        c.sync()
        c.close()
        assert rel_err(got, ref) < TOL[prec], (flags, rel_err(got, ref))


@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_mass_solve_2d_1024(prec):
    from paper_1910_08535_gb300 import workloads
    ne, p = 1024, 3
    axes = oracle_axes(2, ne, p, p + 1, 'pw')
    c = _ctx(dim=2, n_elem=ne, degree=p, nq=p + 1, test='pw', precision=prec)
    r = workloads.uniform_coeffs(c.shape, seed=9)
    got = c.to_numpy(c.solve(c.from_numpy(r)))
    c.sync()
    c.close()
    ref = tensor.ads_solve(tensor.mass_mats(axes), r)
    assert rel_err(got, ref) < TOL[prec], rel_err(got, ref)


@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_long_1d_line(prec):
    from paper_1910_08535_gb300 import workloads
    ne, p = 1500, 3
    axes = oracle_axes(1, ne, p, p + 1, 'pw')
    u = workloads.uniform_coeffs((ne + p,), seed=2)
    dt = 0.05 / ne ** 2
    ref = heat.run(axes, u, dt, 4)
    c = _ctx(dim=1, n_elem=ne, degree=p, nq=p + 1, test='pw', precision=prec)
    ud = c.from_numpy(u)
    c.step(ud, dt, 4)
    got = c.to_numpy(ud)
    sol = c.to_numpy(c.solve(c.from_numpy(u)))
    c.sync()
    c.close()
    assert rel_err(got, ref) < TOL[prec], rel_err(got, ref)
    ref_s = tensor.ads_solve(tensor.mass_mats(axes), u)
    assert rel_err(sol, ref_s) < TOL[prec], rel_err(sol, ref_s)



@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_single_unpadded_column(prec, test):
    """The y step pinned to one column per block with the tables in global
    memory (the unpadded shape that lines of several thousand rows need), on
    8 x 1024 cubic elements, against the oracle."""
    from paper_1910_08535_gb300 import workloads
    ne, p = [8, 1024], 3
    axes = oracle_axes(2, ne, p, p + 1, test)
    c = _ctx(dim=2, n_elem=ne, degree=p, nq=p + 1, test=test, precision=prec)
    c.set_step_shape(1, 'global', 1)
    u = workloads.normal_coeffs(c.shape, seed=6)
    dt = 0.05 / ne[1] ** 2
    ud = c.from_numpy(u)
    c.step(ud, dt, 2)
    got = c.to_numpy(ud)
    c.sync()
    c.close()
    ref = heat.run(axes, u, dt, 2)
    assert rel_err(got, ref) < TOL[prec], rel_err(got, ref)


@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_columns_of_8192_elements(prec):
    """8 x 8192 cubic elements: its y lines are as long as those of the
    8192^2 grid (8195 rows), which only one unpadded column per block fits in
    shared memory; the tuner must find that shape, and the step must equal
    the step of the transposed 8192 x 8 grid, whose long lines run along x
    (the 1D tables and the per-line arithmetic are the same)."""
    from paper_1910_08535_gb300 import workloads
    p = 3
    dt = 0.05 / 8192 ** 2
    cy = _ctx(dim=2, n_elem=[8, 8192], degree=p, nq=p + 1, test='pw', precision=prec)
    u = workloads.normal_coeffs(cy.shape, seed=6)
    ud = cy.from_numpy(u)
    cy.step(ud, dt, 2)
    got = cy.to_numpy(ud)
    cy.sync()
    shape_y = cy.get_step_shape(1)
    cy.close()
    cx = _ctx(dim=2, n_elem=[8192, 8], degree=p, nq=p + 1, test='pw', precision=prec)
    assert tuple(cx.shape) == tuple(u.shape[::-1])
    vd = cx.from_numpy(np.ascontiguousarray(u.T))
    cx.step(vd, dt, 2)
    ref = cx.to_numpy(vd).T
    cx.sync()
    cx.close()
    assert shape_y == ('global', 1), shape_y
    assert rel_err(got, ref) < TOL[prec], rel_err(got, ref)
