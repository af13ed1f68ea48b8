"""Long lines (n above ~800 per axis): the split-step kernel and the batched
line solves switch to fewer lines per block with the 1D tables read from
global memory once a line no longer fits shared memory next to them.  Parity
against the oracle at the largest 2D grid of the mixed request stream
(1024 x 1024 elements, cubic) and a long 1D line."""
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
