"""Batched 2D Poisson over uneven instances: every instance's RHS and solution
against the oracle (rel-L2 <= 1e-5, FP32 pairs with refinement) and against a
single-instance context solving the same RHS; a full-size batch of the
512-instance configuration checked by sampled instances."""
import numpy as np
import pytest

from oracle import poisson_nd
from tests._cases import TOL, oracle_axes, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


def _params(shapes, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.integers(1, 5, size=(len(shapes), 2))
    amp = np.pi ** 2 * (k[:, 0] ** 2 + k[:, 1] ** 2)
    return np.stack([amp, k[:, 0], k[:, 1]], axis=1).astype(np.float64)


def _oracle(shape, par, test):
    from paper_1910_08535_gb300 import workloads
    nx, ny, p = shape
    axes = [oracle_axes(1, nx, p, p + 1, test, 'dirichlet0')[0], oracle_axes(1, ny, p, p + 1, test, 'dirichlet0')[0]]
    pts = [ax.points()[0] for ax in axes]
    f = par[0] / (np.pi ** 2 * (par[1] ** 2 + par[2] ** 2)) * workloads.sine_product_source(pts, (int(par[1]), int(par[2])))
    b = poisson_nd.rhs(axes, f)
    return axes, b


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_small_batch_against_oracle_and_single(test):
    from paper_1910_08535_gb300.igapw import Batch, Context
    shapes = [(8, 8, 2), (13, 9, 3), (40, 17, 2), (21, 33, 3), (5, 6, 2), (64, 48, 3), (33, 33, 2), (9, 50, 3)]
    par = _params(shapes, seed=3)
    bt = Batch(shapes, test=test)
    tx, ty, rx, ry = bt.tiles()
    assert (tx, ty) in ((32, 8), (64, 4), (16, 16)) and (rx, ry) in ((32, 8), (64, 4), (16, 16))
    bt.source_sine(par)
    bt.solve()
    for i, sh in enumerate(shapes):
        axes, b_ref = _oracle(sh, par[i], test)
        b = bt.to_numpy(i, 0)
        assert rel_err(b, b_ref) < TOL['fp32r'], (sh, rel_err(b, b_ref))
        u = bt.to_numpy(i, 1)
        u_ref = poisson_nd.solve(axes, b_ref)
        assert rel_err(u, u_ref) < TOL['fp32r'], (sh, rel_err(u, u_ref))
        # a single context on the same right-hand side
        c = Context(dim=2, n_elem=[sh[0], sh[1]], degree=sh[2], nq=sh[2] + 1, test=test, bc='dirichlet0',
                    precision='fp32r', op='poisson')
        us = c.to_numpy(c.solve(bt.tensor(i, 0).clone()))
        c.close()
        assert rel_err(u, us) < 1e-7, (sh, rel_err(u, us))


def test_cublas_transforms_match_tensor_cores():
    """The batch with cuBLAS grouped GEMMs and with the tensor-core grouped
    GEMMs on the same sources: both against the oracle, and the device status
    word clear after the solves."""
    from paper_1910_08535_gb300.igapw import Batch
    shapes = [(30, 20, 2), (17, 44, 3), (64, 64, 3), (9, 9, 2)]
    par = _params(shapes, seed=4)
    out = {}
    for gemm in ('tc', 'cublas'):
        bt = Batch(shapes, gemm=gemm)
        bt.source_sine(par)
        bt.solve()
        bt.sync_status()
        out[gemm] = [bt.to_numpy(i, 1) for i in range(len(shapes))]
        bt.close()
    for i, sh in enumerate(shapes):
        axes, b_ref = _oracle(sh, par[i], 'pw')
        u_ref = poisson_nd.solve(axes, b_ref)
        for gemm in ('tc', 'cublas'):
            assert rel_err(out[gemm][i], u_ref) < TOL['fp32r'], (gemm, sh, rel_err(out[gemm][i], u_ref))


def test_resolve_after_rhs_update():
    """A second source and solve through the captured graph gives the new solution."""
    from paper_1910_08535_gb300.igapw import Batch
    shapes = [(16, 12, 2), (24, 24, 3)]
    bt = Batch(shapes)
    for seed in (1, 2):
        par = _params(shapes, seed)
        bt.source_sine(par)
        bt.solve()
        for i, sh in enumerate(shapes):
            axes, b_ref = _oracle(sh, par[i], 'pw')
            u_ref = poisson_nd.solve(axes, b_ref)
            assert rel_err(bt.to_numpy(i, 1), u_ref) < TOL['fp32r']
    bt.close()


def test_full_batch_512_sampled():
    """512 instances, grids log-uniform on 16 rungs from 32^2 to 512^2, p in
    {2, 3}: backward error of sampled instances with the oracle's operator,
    and the smallest instances against the dense oracle solve."""
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Batch
    shapes = workloads.batch_shapes(512, seed=0)
    par = _params(shapes, seed=0)
    bt = Batch(shapes)
    bt.source_sine(par)
    bt.solve()
    bt.sync_status()
    order = np.argsort([s[0] * s[1] for s in shapes])
    for i in list(order[:3]):
        axes, b_ref = _oracle(shapes[i], par[i], 'pw')
        assert rel_err(bt.to_numpy(i, 1), poisson_nd.solve(axes, b_ref)) < TOL['fp32r']
    for i in list(order[-2:]) + list(order[250:252]):
        axes, _ = _oracle(shapes[i], par[i], 'pw')
        eta = poisson_nd.backward_error(axes, bt.to_numpy(i, 1), bt.to_numpy(i, 0))
        assert eta < 1e-7, (shapes[i], eta)
    bt.close()
