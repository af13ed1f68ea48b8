"""Full-size parity of the explicit heat workloads against the oracle, element
by element over every coefficient, in the launch configuration bench.py times:

  heat2d  quadratic, 256^2 elements, 3x3 Gauss, dt = 0.1 h^2, 200 steps,
          initial Gaussian bump + 1e-3 noise; FP64 and FP32 pairs.
  heat3d  cubic, 128^3 elements, 4^3 Gauss, dt = 0.05 h^2, 50 steps,
          coefficients 1e-2 N(0,1); FP32 pairs.
Step forms: flags 0 = split form (one kernel per axis), 2 = RHS then solve
(double-float residual), 3 = RHS then solve with an FP64 residual.

The quadratic PW step at dt = 0.1 h^2 lies beyond the forward-Euler limit
(the largest PW eigenvalue magnitude of the 1D operator is about 12/h^2, so
2 * 12 * 0.1 = 2.4 > 2): its top mode grows, and parity is checked in the
relative norm, which stays meaningful for a linear iteration."""
import numpy as np
import pytest

from oracle import heat
from tests._cases import TOL, oracle_axes, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


def _run(name, test, prec, flags=0):
    import torch
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    w = workloads.WORKLOADS[name]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        c = Context(dim=w['dim'], n_elem=w['n_elem'], degree=w['degree'], nq=w['nq'], test=test,
                    precision=prec, flags=flags, stream=stream)
        u0 = workloads.initial_state(name)
        u = c.from_numpy(u0)
        c.step(u, workloads.dt_of(name), w['steps'])
        c.sync()
        got = c.to_numpy(u)
        c.close()
    axes = oracle_axes(w['dim'], w['n_elem'], w['degree'], w['nq'], test)
    ref = heat.run(axes, u0, workloads.dt_of(name), w['steps'])
    return got, ref


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
@pytest.mark.parametrize('flags', [0, 2])
def test_heat2d_full(test, prec, flags):
    got, ref = _run('heat2d', test, prec, flags)
    err = rel_err(got, ref)
    print(f'heat2d {test} {prec} flags={flags}: rel-L2 {err:.3e} max-abs {np.abs(got - ref).max():.3e}')
    assert err < TOL[prec]


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
@pytest.mark.parametrize('flags', [0, 2, 3])
def test_heat3d_full(test, flags):
    got, ref = _run('heat3d', test, 'fp32r', flags)
    err = rel_err(got, ref)
    print(f'heat3d {test} flags={flags}: rel-L2 {err:.3e} max-abs {np.abs(got - ref).max():.3e}')
    assert err < TOL['fp32r']
