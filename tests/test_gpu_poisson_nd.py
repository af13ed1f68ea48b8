"""GPU parity of the 2D/3D Poisson system (Sec. 4.3, -Lap u = f with zero
Dirichlet rows) against the oracle: operator action K u, the source RHS of a
manufactured solution, and the solve, element by element (rel-L2 <= 1e-12 in
FP64, <= 1e-5 for FP32 pairs with refinement), on meshes spanning several
tiles with ragged tails; right-hand sides that are non-zero on the boundary
rows; the cuBLAS FP32 and BF16x9 transform options beside the default
tensor-core transforms; and, at the largest grids of the mixed
request stream, the residual and sampled entries against the oracle."""
import numpy as np
import pytest

from oracle import poisson_nd
from tests._cases import TOL, oracle_axes, rel_err, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


def _ctx(**kw):
    from paper_1910_08535_gb300.igapw import Context
    return Context(op='poisson', bc='dirichlet0', **kw)


def _source(c, d, k, prec):
    import torch
    from paper_1910_08535_gb300 import workloads
    pts = [c.quad_points(a)[0] for a in range(d)]
    f = workloads.sine_product_source(pts, k)
    f = f if prec == 'fp64' else f.astype(np.float32).astype(np.float64)
    fd = torch.from_numpy(f.astype(np.float64 if prec == 'fp64' else np.float32)).cuda()
    return f, fd


CASES = [(2, [8, 11]), (2, [37, 21]), (3, [5, 6, 7]), (3, [9, 4, 11])]


@pytest.mark.parametrize('d,ne', CASES)
@pytest.mark.parametrize('p', [2, 3])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_apply_rhs_solve(d, ne, p, test, prec):
    from paper_1910_08535_gb300 import workloads
    c = _ctx(dim=d, n_elem=ne, degree=p, nq=p + 1, test=test, precision=prec)
    axes = oracle_axes(d, ne, p, p + 1, test, 'dirichlet0')
    tol = TOL[prec]
    # operator action on random coefficients (boundary values included)
    u = workloads.uniform_coeffs(c.shape, seed=21)
    r = c.to_numpy(c.apply('poisson', c.from_numpy(u)))
    ref = poisson_nd.apply(axes, u)
    assert rel_err(r, ref) < tol, rel_err(r, ref)
    # manufactured source RHS, then the solve
    k = (1, 2, 1)[:d]
    f, fd = _source(c, d, k, prec)
    bd = c.rhs_source(fd)
    b_ref = poisson_nd.rhs(axes, f)
    assert rel_err(c.to_numpy(bd), b_ref) < tol, rel_err(c.to_numpy(bd), b_ref)
    sol = c.to_numpy(c.solve(bd))
    ref = poisson_nd.solve(axes, b_ref)
    assert rel_err(sol, ref) < tol, rel_err(sol, ref)
    # boundary rows of the solution are exactly the (zero) RHS rows
    mask = poisson_nd.boundary_mask(axes)
    assert np.max(np.abs(sol[mask])) <= 1e-12 * np.max(np.abs(sol))
    c.sync()
    c.close()


@pytest.mark.parametrize('d,ne', [(2, [13, 10]), (3, [6, 5, 7])])
@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_boundary_rhs_nonzero(d, ne, prec):
    """b non-zero on the boundary rows: u_B = b_B and the interior sees the
    coupling through K_IB (settled by the refinement)."""
    from paper_1910_08535_gb300 import workloads
    c = _ctx(dim=d, n_elem=ne, degree=3, nq=4, test='pw', precision=prec)
    axes = oracle_axes(d, ne, 3, 4, 'pw', 'dirichlet0')
    b = workloads.uniform_coeffs(c.shape, seed=5)
    sol = c.to_numpy(c.solve(c.from_numpy(b)))
    ref = poisson_nd.solve(axes, b)
    assert rel_err(sol, ref) < TOL[prec], rel_err(sol, ref)
    c.sync()
    c.close()


@pytest.mark.parametrize('engine', ['bf16x9', 'cublas'])
@pytest.mark.parametrize('d,ne', [(2, [40, 33]), (3, [9, 12, 7])])
@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_transform_engines(engine, d, ne, prec):
    """The cuBLAS transform options against the oracle and against the
    default tensor-core transforms on the same right-hand side."""
    from paper_1910_08535_gb300 import igapw, workloads
    p = 3
    flag = igapw.IGAPW_FLAG_FDM_BF16X9 if engine == 'bf16x9' else igapw.IGAPW_FLAG_FDM_CUBLAS
    c = _ctx(dim=d, n_elem=ne, degree=p, nq=p + 1, test='pw', precision=prec, flags=flag)
    ct = _ctx(dim=d, n_elem=ne, degree=p, nq=p + 1, test='pw', precision=prec)
    axes = oracle_axes(d, ne, p, p + 1, 'pw', 'dirichlet0')
    b = workloads.uniform_coeffs(c.shape, seed=8)
    sol = c.to_numpy(c.solve(c.from_numpy(b)))
    sol_tc = ct.to_numpy(ct.solve(ct.from_numpy(b)))
    ref = poisson_nd.solve(axes, b, sparse=True)
    assert rel_err(sol, ref) < TOL[prec], rel_err(sol, ref)
    assert rel_err(sol_tc, ref) < TOL[prec], rel_err(sol_tc, ref)
    c.sync()
    ct.sync()
    c.close()
    ct.close()


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_medium_2d_against_sparse_direct(test):
    """256 x 256 elements, p = 2: the whole solution against a sparse direct
    solve of the oracle's matrix."""
    c = _ctx(dim=2, n_elem=256, degree=2, nq=3, test=test, precision='fp64')
    axes = oracle_axes(2, 256, 2, 3, test, 'dirichlet0')
    f, fd = _source(c, 2, (2, 3), 'fp64')
    sol = c.to_numpy(c.solve(c.rhs_source(fd)))
    ref = poisson_nd.solve(axes, poisson_nd.rhs(axes, f), sparse=True)
    assert rel_err(sol, ref) < TOL['fp64'], rel_err(sol, ref)
    c.sync()
    c.close()


@pytest.mark.parametrize('d,ne,p,err_max', [(2, 1024, 3, 1e-5), (3, 160, 2, 5e-4), (3, 128, 3, 1e-5)])
@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_largest_grids_residual(d, ne, p, err_max, prec):
    """The largest grids of the mixed request stream, where the oracle cannot
    solve: the normwise backward error of the GPU solution, |b - K u| /
    (| |K| |u| | + |b|) with K applied by the oracle's per-axis contractions in
    FP64 (a relative residual |b - K u| / |b| would carry the conditioning of
    K, about 1e6 here), and the manufactured-solution error against the
    discretisation error the convergence rates predict."""
    from paper_1910_08535_gb300 import workloads
    c = _ctx(dim=d, n_elem=ne, degree=p, nq=p + 1, test='pw', precision=prec)
    axes = oracle_axes(d, ne, p, p + 1, 'pw', 'dirichlet0')
    k = (1, 2, 1)[:d]
    f, fd = _source(c, d, k, prec)
    bd = c.rhs_source(fd)
    b = c.to_numpy(bd)
    sol = c.to_numpy(c.solve(bd))
    eta = poisson_nd.backward_error(axes, sol, b)
    print('backward error', eta, 'relative residual', rel_l2(poisson_nd.apply(axes, sol), b))
    assert eta < (1e-14 if prec == 'fp64' else 1e-7), eta
    err = poisson_nd.l2_error(axes, sol, workloads.sine_product_exact(k), nq_err=3)
    assert err < err_max, err
    c.sync()
    c.close()


def test_rejects_aliasing_and_bad_descriptors():
    from paper_1910_08535_gb300.igapw import Context, IgapwError
    c = _ctx(dim=2, n_elem=[6, 5], degree=2, nq=3, test='pw', precision='fp64')
    t = c.empty()
    with pytest.raises(IgapwError):
        c.solve(t, out=t)
    c.close()
    with pytest.raises(IgapwError):
        Context(dim=2, n_elem=6, degree=2, nq=3, bc='dirichlet0', op='heat')
