"""GPU parity of the operator action, the source RHS, the Kronecker solve and
explicit steps against the oracle, element by element, FP64 (rel-L2 <= 1e-12)
and FP32 pairs with refinement (rel-L2 <= 1e-5), on sizes spanning several
tiles with ragged tails, plus edge cases (one element, tiny meshes)."""
import numpy as np
import pytest

from oracle import heat, poisson, systems, tensor
from tests._cases import TOL, oracle_axes, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


def _ctx(**kw):
    from paper_1910_08535_gb300.igapw import Context
    return Context(**kw)


SHAPES = {1: [1, 7, 300], 2: [[3, 2], [37, 21]], 3: [[2, 3, 1], [35, 14, 9]]}


def _cases():
    for d, sizes in SHAPES.items():
        for ne in sizes:
            for p in (2, 3):
                for test in ('pw', 'galerkin'):
                    for prec in ('fp64', 'fp32r'):
                        yield d, ne, p, test, prec


@pytest.mark.parametrize('d,ne,p,test,prec', list(_cases()))
def test_apply_solve_step(d, ne, p, test, prec):
    from paper_1910_08535_gb300 import workloads
    c = _ctx(dim=d, n_elem=ne, degree=p, nq=p + 1, test=test, precision=prec)
    axes = oracle_axes(d, ne, p, p + 1, test)
    u = workloads.uniform_coeffs(c.shape, seed=11)
    ud = c.from_numpy(u)
    tol = TOL[prec]
    # operator action for every op
    for op, (alpha, beta) in (('mass', (1.0, 0.0)), ('laplace', (0.0, 1.0)), ('heat', (1.0, 0.0123))):
        r = c.to_numpy(c.apply(op, ud, dt=beta if op == 'heat' else 0.0))
        M = tensor.mass_mats(axes)
        L = tensor.lap_mats(axes)
        ref = 0.0
        if alpha:
            ref = ref + alpha * tensor.apply_heat_system(axes, u, 0.0, M, L)
        if beta:
            lap = tensor.apply_heat_system(axes, u, 1.0, M, L) - tensor.apply_heat_system(axes, u, 0.0, M, L)
            ref = ref + beta * lap
        assert rel_err(r, ref) < tol, (op, rel_err(r, ref))
    # Kronecker mass solve
    rhs = workloads.uniform_coeffs(c.shape, seed=12)
    sol = c.to_numpy(c.solve(c.from_numpy(rhs)))
    ref = tensor.ads_solve(tensor.mass_mats(axes), rhs)
    assert rel_err(sol, ref) < tol, rel_err(sol, ref)
    # explicit steps (stable step size), split form and RHS-then-solve form
    h = 1.0 / (np.max(ne) if d > 1 else ne)
    dt = 0.05 * h * h / d
    ref = heat.run(axes, u, dt, 3)
    c.step(ud, dt, 3)
    got = c.to_numpy(ud)
    assert rel_err(got, ref) < tol, rel_err(got, ref)
    c.sync()
    c.close()
    from paper_1910_08535_gb300 import igapw
    c2 = _ctx(dim=d, n_elem=ne, degree=p, nq=p + 1, test=test, precision=prec, flags=igapw.IGAPW_FLAG_STEP_RHS_SOLVE)
    ud2 = c2.from_numpy(u)
    c2.step(ud2, dt, 3)
    got2 = c2.to_numpy(ud2)
    assert rel_err(got2, ref) < tol, rel_err(got2, ref)
    c2.sync()
    c2.close()


# (p, nq): at most 2, 3 or 4 sample points per PW cell and axis (the slab
# kernel's unroll widths), and 8 (p = 3 cells straddle a knot: two pieces)
@pytest.mark.parametrize('p,nq', [(2, 2), (2, 3), (3, 2), (3, 4)])
@pytest.mark.parametrize('d,ne', [(1, 9), (2, [6, 5]), (3, [4, 3, 5]), (2, [300, 7]), (3, [37, 21, 5])])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_source_rhs(d, ne, test, prec, p, nq):
    import torch
    from paper_1910_08535_gb300 import workloads
    c = _ctx(dim=d, n_elem=ne, degree=p, nq=nq, test=test, precision=prec)
    axes = oracle_axes(d, ne, p, nq, test)
    pts = [c.quad_points(a)[0] for a in range(d)]
    f = workloads.tensor_samples(pts, [tuple(np.sin for _ in range(d)), tuple((lambda x: x ** 2) for _ in range(d))])
    fd = torch.from_numpy(f.astype(np.float64 if prec == 'fp64' else np.float32)).cuda()
    b = c.to_numpy(c.rhs_source(fd))
    fin = f if prec == 'fp64' else f.astype(np.float32).astype(np.float64)
    ref = tensor.rhs_source(axes, fin)
    assert rel_err(b, ref) < TOL[prec] * (1 if prec == 'fp64' else 0.01), rel_err(b, ref)


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_poisson_1d_config(test, prec):
    """1D Poisson, p=2, 64 elements, 3 Gauss points, f = pi^2 sin(pi x), zero
    Dirichlet rows: the GPU solution equals the oracle's and is close to sin."""
    import torch
    from paper_1910_08535_gb300 import workloads
    c = _ctx(dim=1, n_elem=64, degree=2, nq=3, test=test, bc='dirichlet0', op='poisson', precision=prec)
    ax = systems.Axis(64, 2, 3, test, 'dirichlet0')
    x, _ = c.quad_points(0)
    f = workloads.sine_source(x)
    fd = torch.from_numpy(f.astype(np.float64 if prec == 'fp64' else np.float32)).cuda()
    b = c.rhs_source(fd)
    u = c.to_numpy(c.solve(b))
    ref = poisson.solve(ax, workloads.sine_source)
    assert rel_err(u, ref) < TOL[prec], rel_err(u, ref)
    assert poisson.l2_error(ax, u, workloads.sine_exact) < (1e-6 if test == 'galerkin' else 2e-4)
    # apply(POISSON) then solve is the identity
    v = workloads.uniform_coeffs(c.shape, seed=3)
    v[0] = v[-1] = 0.0
    back = c.to_numpy(c.solve(c.apply('poisson', c.from_numpy(v))))
    assert rel_err(back, v) < TOL[prec]


def test_status_flags_nonfinite():
    """A NaN coefficient makes the step's solve flag a non-finite value; the
    context stays usable."""
    import torch
    from paper_1910_08535_gb300.igapw import IgapwError
    c = _ctx(dim=2, n_elem=5, degree=2, nq=3)
    u = torch.zeros(c.shape, dtype=torch.float64, device='cuda')
    u[2, 2] = float('nan')
    c.step(u, 1e-4, 1)
    with pytest.raises(IgapwError, match='non-finite'):
        c.sync()
    u.zero_()
    c.step(u, 1e-4, 1)
    c.sync()
