"""GPU test of igapw_rhs_source_noalloc, the allocation-free source RHS for
callers that cannot let the library allocate device memory at call time (its
intermediates live in a static device array instead of memory igapw_rhs_source
allocates on first use).  On a fresh context the first call must leave the
device's free memory unchanged; two calls in a row on different samples must
each match the allocating entry point; a problem whose intermediates exceed
the static array must be rejected.  Collected last so that a failure here
stops a run only after every other test has run; it also passes alone."""
import numpy as np
import pytest

from tests._cases import TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


def _samples(c, dim, seed, dtype):
    import torch
    from paper_1910_08535_gb300 import workloads
    pts = [c.quad_points(a)[0] for a in range(dim)]
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.5, 3.0, size=dim)
    f = workloads.tensor_samples(pts, [tuple((lambda x, kk=kk: np.sin(kk * x)) for kk in k)])
    return torch.from_numpy(f.astype(dtype)).cuda()


def test_noalloc_first_call_allocates_nothing():
    import torch
    from paper_1910_08535_gb300 import igapw
    from paper_1910_08535_gb300.igapw import Context
    # load the source kernels' module first (lazy module loading reserves
    # device memory for code on a module's first launch)
    w = Context(dim=3, n_elem=[13, 9, 11], degree=3, nq=4, test='galerkin', precision='fp32r')
    w.rhs_source(_samples(w, 3, seed=1, dtype=np.float32))
    w.sync()
    w.close()
    c = Context(dim=3, n_elem=[13, 9, 11], degree=3, nq=4, test='galerkin', precision='fp32r')
    f = _samples(c, 3, seed=2, dtype=np.float32)
    got = c.empty()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    igapw.igapw_rhs_source_noalloc(c.ctx, f, got)
    c.sync()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    ref = c.rhs_source(f)
    c.sync()
    assert rel_err(c.to_numpy(got), c.to_numpy(ref)) <= TOL['fp32r']
    c.close()


@pytest.mark.parametrize('dim,ne', [(1, [53]), (2, [37, 21]), (3, [13, 9, 11])])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_noalloc_matches_allocating_entry_point(dim, ne, test, prec):
    from paper_1910_08535_gb300 import igapw
    from paper_1910_08535_gb300.igapw import Context
    c = Context(dim=dim, n_elem=ne, degree=3, nq=4, test=test, precision=prec)
    dtype = np.float64 if prec == 'fp64' else np.float32
    for call in range(2):
        f = _samples(c, dim, seed=10 + call, dtype=dtype)
        ref = c.rhs_source(f)
        got = c.empty()
        igapw.igapw_rhs_source_noalloc(c.ctx, f, got)
        c.sync()
        err = rel_err(c.to_numpy(got), c.to_numpy(ref))
        assert err <= TOL[prec], (call, err)
    c.close()


def test_noalloc_rejects_oversized_problem():
    import torch
    from paper_1910_08535_gb300 import igapw
    from paper_1910_08535_gb300.igapw import Context, IgapwError
    # Galerkin, p = 3, 4 points per element, 64^3 elements: each intermediate
    # needs 8 * 256 * 256 * 67 bytes = 35 MB, beyond half of the 8 MiB array
    c = Context(dim=3, n_elem=64, degree=3, nq=4, test='galerkin', precision='fp32r')
    q = [len(c.quad_points(a)[0]) for a in range(3)]
    f = torch.zeros((q[2], q[1], q[0]), dtype=torch.float32, device='cuda')
    b = c.empty()
    with pytest.raises(IgapwError) as ei:
        igapw.igapw_rhs_source_noalloc(c.ctx, f, b)
    assert ei.value.code == igapw.IGAPW_ERR_ARG
    assert 'static scratch' in str(ei.value)
    c.close()
