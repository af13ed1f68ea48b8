"""GPU parity of the refined-test-space variant (Sec. 2, IGAPW_REFINED):
folded tables, operator action, source RHS, Kronecker solve, explicit steps
and the 2D Poisson solve against the oracle's refined-test axes."""
import numpy as np
import pytest

from oracle import heat, poisson_nd, systems, tensor
from tests._cases import TOL, oracle_axes, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


@pytest.mark.parametrize('d,ne', [(1, 23), (2, [9, 14]), (3, [5, 4, 6])])
@pytest.mark.parametrize('p,r', [(2, 4), (3, 6)])
@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_refined_apply_solve_step(d, ne, p, r, prec):
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    c = Context(dim=d, n_elem=ne, degree=p, nq=p + 1, test='refined', refine=r, precision=prec)
    axes = oracle_axes(d, ne, p, p + 1, 'refined', refine=r)
    tol = TOL[prec]
    # 1D tables
    for a in range(d):
        for which, ref in (('mass', systems.mass(axes[a])), ('laplace', systems.laplace(axes[a]))):
            got = c.assemble_1d(a, which)
            assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref)), (a, which)
    u = workloads.uniform_coeffs(c.shape, seed=13)
    ud = c.from_numpy(u)
    r_heat = c.to_numpy(c.apply('heat', ud, dt=0.01))
    ref = tensor.apply_heat_system(axes, u, 0.01)
    assert rel_err(r_heat, ref) < tol, rel_err(r_heat, ref)
    sol = c.to_numpy(c.solve(c.from_numpy(ref)))
    ref_s = tensor.ads_solve(tensor.mass_mats(axes), ref)
    assert rel_err(sol, ref_s) < tol, rel_err(sol, ref_s)
    h = 1.0 / (np.max(ne) if d > 1 else ne)
    dt = 0.05 * h * h / d
    c.step(ud, dt, 3)
    got = c.to_numpy(ud)
    ref = heat.run(axes, u, dt, 3)
    assert rel_err(got, ref) < tol, rel_err(got, ref)
    c.sync()
    c.close()


@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_refined_source_and_poisson_2d(prec):
    import torch
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    ne, p, r = [17, 12], 3, 5
    c = Context(dim=2, n_elem=ne, degree=p, nq=p + 1, test='refined', refine=r, bc='dirichlet0', op='poisson',
                precision=prec)
    axes = oracle_axes(2, ne, p, p + 1, 'refined', 'dirichlet0', refine=r)
    pts = [c.quad_points(a)[0] for a in range(2)]
    f = workloads.sine_product_source(pts, (1, 2))
    if prec == 'fp32r':
        f = f.astype(np.float32).astype(np.float64)
    fd = torch.from_numpy(f.astype(np.float64 if prec == 'fp64' else np.float32)).cuda()
    b = c.rhs_source(fd)
    b_ref = poisson_nd.rhs(axes, f)
    assert rel_err(c.to_numpy(b), b_ref) < TOL[prec], rel_err(c.to_numpy(b), b_ref)
    sol = c.to_numpy(c.solve(b))
    ref = poisson_nd.solve(axes, b_ref)
    assert rel_err(sol, ref) < TOL[prec], rel_err(sol, ref)
    c.sync()
    c.close()
