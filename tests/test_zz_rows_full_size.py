"""Full-size parity of the bench rows in the launch configurations bench.py
times, every coefficient against the oracle (rel-L2 <= 1e-5, FP32 pairs):

- the Table 1 source RHS (Sec. 4.1): 3D, quadratic C1 splines, 128^3
  elements, a tensor-product cubic sampled at each rule's points (PW: 2 points
  per piece, B-spline tests: 3 per element), FP32 samples, double-float sums;
- the heat3d operator action T(u + dt Lap u) and the refined Kronecker mass
  solve (Sec. 4.1-4.2): cubic C2, 128^3 elements, 4 points, PW tests;
- one explicit step (Sec. 4.2, Eq. (6)) at the size-ladder grids past L2
  (256^3 cubic and quadratic, 192^3 quartic; PW, 1e-2 N(0,1) coefficients,
  dt = 0.05 h^2)."""
import numpy as np
import pytest

from oracle import systems, tensor
from tests._cases import TOL, rel_err

pytestmark = pytest.mark.gpu

CUBICS = (lambda x: 2 * x ** 3 - x ** 2 + 0.5 * x + 1, lambda x: x ** 3 + 0.3 * x + 0.2,
          lambda x: -x ** 3 + 2 * x ** 2 + 1)


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


@pytest.mark.parametrize('test,nq', [('pw', 2), ('galerkin', 3)])
def test_table1_source_full_size(test, nq):
    import torch
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    ne, p = 128, 2
    c = Context(dim=3, n_elem=ne, degree=p, nq=nq, test=test, precision='fp32r', op='mass')
    pts = [c.quad_points(a)[0] for a in range(3)]
    f = workloads.tensor_samples(pts, [CUBICS]).astype(np.float32)
    b = c.rhs_source(torch.from_numpy(f).cuda())
    got = c.to_numpy(b)
    c.sync()
    c.close()
    ref = tensor.rhs_source([systems.Axis(ne, p, nq, test) for _ in range(3)], f.astype(np.float64))
    assert got.shape == ref.shape == (130, 130, 130)
    assert rel_err(got, ref) < TOL['fp32r'], rel_err(got, ref)


def test_heat3d_apply_and_solve_full_size():
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    w = workloads.WORKLOADS['heat3d']
    c = Context(dim=3, n_elem=w['n_elem'], degree=w['degree'], nq=w['nq'], test='pw', precision='fp32r')
    u0 = workloads.initial_state('heat3d')
    dt = workloads.dt_of('heat3d')
    r = c.apply('heat', c.from_numpy(u0), dt)
    got_r = c.to_numpy(r)
    got_s = c.to_numpy(c.solve(r))
    c.sync()
    c.close()
    axes = [systems.Axis(w['n_elem'], w['degree'], w['nq'], 'pw') for _ in range(3)]
    M, L = tensor.mass_mats(axes), tensor.lap_mats(axes)
    ref_r = tensor.apply_heat_system(axes, u0, dt, M, L)
    assert rel_err(got_r, ref_r) < TOL['fp32r'], rel_err(got_r, ref_r)
    ref_s = tensor.ads_solve(M, got_r)
    assert rel_err(got_s, ref_s) < TOL['fp32r'], rel_err(got_s, ref_s)


@pytest.mark.parametrize('ne,p', [(256, 3), (256, 2), (192, 4)])
def test_ladder_step_full_size(ne, p):
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    c = Context(dim=3, n_elem=ne, degree=p, nq=p + 1, test='pw', precision='fp32r')
    u0 = workloads.normal_coeffs(c.shape, seed=ne)
    dt = 0.05 / ne ** 2
    u = c.from_numpy(u0)
    c.step(u, dt, 1)
    c.sync()
    got = c.to_numpy(u)
    c.close()
    axes = [systems.Axis(ne, p, p + 1, 'pw') for _ in range(3)]
    M, L = tensor.mass_mats(axes), tensor.lap_mats(axes)
    ref = tensor.ads_solve(M, tensor.apply_heat_system(axes, u0, dt, M, L))
    assert rel_err(got, ref) < TOL['fp32r'], rel_err(got, ref)
