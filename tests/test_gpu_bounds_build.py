"""The debug build (lib/libigapw_bounds.so, -DIGAPW_BOUNDS_CHECK): every kernel
checks its indices, skips an out-of-range access and records it, and
igapw_sync_status reports it as IGAPW_ERR_DEVICE_STATUS.  A child process
loads that build and runs the hot-path calls on small ragged problems --
explicit steps with every step kernel shape, operator action, Kronecker
solve, PW and Galerkin source RHS, 2D Poisson, a small batch -- and checks
that no access was out of range and that the results match the oracle."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent('''
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch
    from paper_1910_08535_gb300 import _build, igapw, workloads
    lib = _build.build(bounds=True)
    igapw.load(lib)
    from paper_1910_08535_gb300.igapw import Context, Batch
    from oracle import heat, poisson_nd, systems, tensor
    from tests._cases import TOL, oracle_axes, rel_err

    def check(c, what):
        c.sync()   # raises IgapwError(IGAPW_ERR_DEVICE_STATUS) on a recorded access

    for dim, ne, p, test in ((2, [23, 17], 2, 'pw'), (3, [11, 9, 13], 3, 'galerkin'), (3, [20, 7, 5], 3, 'pw')):
        for kind, nl in (('chunked', 32), ('chunked', 8), ('staged', 32), ('global', 8), (None, 0)):
            c = Context(dim=dim, n_elem=ne, degree=p, nq=p + 1, test=test, precision='fp32r')
            shape = c.shape
            if kind is not None:
                for a in range(dim):
                    # a block of x lines takes at most as many lines as there are (shape is z, y, x)
                    nl_a = min(nl, int(np.prod(shape[:-1]))) if (a == 0 and kind != 'chunked') else nl
                    c.set_step_shape(a, kind, nl_a)
            u0 = workloads.normal_coeffs(shape, seed=3)
            u = c.from_numpy(u0)
            dt = 0.05 / max(ne) ** 2
            c.step(u, dt, 2)
            check(c, 'step')
            ref = heat.run(oracle_axes(dim, ne, p, p + 1, test), u0, dt, 2)
            assert rel_err(c.to_numpy(u), ref) < TOL['fp32r'], (dim, ne, kind)
            r = c.apply('heat', c.from_numpy(u0), dt)
            s = c.solve(r)
            check(c, 'apply/solve')
            axes = oracle_axes(dim, ne, p, p + 1, test)
            M, L = tensor.mass_mats(axes), tensor.lap_mats(axes)
            assert rel_err(c.to_numpy(r), tensor.apply_heat_system(axes, u0, dt, M, L)) < TOL['fp32r']
            assert rel_err(c.to_numpy(s), tensor.ads_solve(M, c.to_numpy(r))) < TOL['fp32r']
            pts = [c.quad_points(a)[0] for a in range(dim)]
            f = workloads.tensor_samples(pts, [tuple(np.sin for _ in range(dim))])
            b = c.rhs_source(torch.from_numpy(f.astype(np.float32)).cuda())
            check(c, 'source')
            assert rel_err(c.to_numpy(b), tensor.rhs_source(axes, f.astype(np.float32).astype(np.float64))) < TOL['fp32r']
            c.close()
    c = Context(dim=2, n_elem=[19, 14], degree=3, nq=4, test='pw', bc='dirichlet0', op='poisson', precision='fp32r')
    bh = workloads.uniform_coeffs(c.shape, seed=2)
    sol = c.to_numpy(c.solve(c.from_numpy(bh)))
    check(c, 'poisson')
    c.close()
    axes = [systems.Axis(19, 3, 4, 'pw', 'dirichlet0'), systems.Axis(14, 3, 4, 'pw', 'dirichlet0')]
    assert rel_err(sol, poisson_nd.solve(axes, bh)) < TOL['fp32r']
    shapes = [(17, 17, 2), (24, 24, 3), (9, 9, 2)]
    bt = Batch(shapes)
    par = np.array([[2 * np.pi ** 2, 1, 1], [5 * np.pi ** 2, 1, 2], [8 * np.pi ** 2, 2, 2]], dtype=np.float64)
    bt.source_sine(par)
    bt.solve()
    torch.cuda.synchronize()
    for i, (nx, ny, p) in enumerate(shapes):
        axes = [systems.Axis(nx, p, p + 1, 'pw', 'dirichlet0'), systems.Axis(ny, p, p + 1, 'pw', 'dirichlet0')]
        assert rel_err(bt.to_numpy(i, 1), poisson_nd.solve(axes, bt.to_numpy(i, 0))) < TOL['fp32r']
    bt.close()
    print('bounds build ok')
''')


def test_bounds_checked_build_runs_clean():
    r = subprocess.run([sys.executable, '-c', CHILD.format(root=ROOT)], capture_output=True, text=True, cwd=ROOT,
                       timeout=1500)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert 'bounds build ok' in r.stdout
