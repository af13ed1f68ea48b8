"""igapw_rhs_source_sine (the separable source amp prod_a sin(k_a pi x_a)
evaluated by the library) against the oracle's source RHS of the same
function sampled at the quadrature points (Sec. 4.1), and against the
library's general source RHS on those samples: 1D-3D, PW and Galerkin tests,
zero Dirichlet rows and no boundary condition, FP64 and FP32 pairs."""
import numpy as np
import pytest

from oracle import tensor
from tests._cases import TOL, oracle_axes, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


@pytest.mark.parametrize('dim,ne,p', [(1, [21], 2), (2, [17, 12], 3), (3, [9, 7, 11], 2), (3, [6, 8, 5], 4)])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
@pytest.mark.parametrize('bc', ['dirichlet0', 'none'])
@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_sine_source_matches_sampled_source(dim, ne, p, test, bc, prec):
    import torch
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    op = 'poisson' if bc == 'dirichlet0' else 'mass'
    c = Context(dim=dim, n_elem=ne, degree=p, nq=p + 1, test=test, bc=bc, op=op, precision=prec)
    k = [1 + a for a in range(dim)]
    amp = 2.5
    got = c.to_numpy(c.rhs_source_sine(amp, k))
    pts = [c.quad_points(a)[0] for a in range(dim)]
    f = amp * workloads.tensor_samples(pts, [tuple((lambda x, kk=kk: np.sin(kk * np.pi * x)) for kk in k)])
    lib = c.to_numpy(c.rhs_source(torch.from_numpy(f.astype(np.float64 if prec == 'fp64' else np.float32)).cuda()))
    c.sync()
    c.close()
    axes = oracle_axes(dim, ne, p, p + 1, test, bc)
    ref = tensor.rhs_source(axes, f)      # Dirichlet rows: no test, b = 0
    assert rel_err(got, ref) < TOL[prec], rel_err(got, ref)
    assert rel_err(got, lib) < TOL[prec], rel_err(got, lib)
