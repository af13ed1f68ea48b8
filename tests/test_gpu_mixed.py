"""GPU parity of the mixed Dirichlet/Neumann Laplace problem (Sec. 4.3):
operator action with the Neumann boundary term, source plus face-data RHS,
and the solve (fast diagonalisation with a zero-mode Neumann pencil), against
the oracle element by element (rel-L2 <= 1e-12 FP64, <= 1e-5 FP32 pairs)."""
import numpy as np
import pytest

from oracle import laplace_mixed as LM, poisson_nd
from tests._cases import TOL, oracle_axes, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


def _axes(ne, p, test, neumann):
    out = []
    for a, n in enumerate(ne):
        bc = 'none' if (neumann >> a) & 1 else 'dirichlet0'
        out.append(oracle_axes(1, n, p, p + 1, test, bc)[0])
    return out


def _data(pts, d):
    """u = sin(pi x) e^y (sin(pi z)): f = -Lap u, G on the y faces."""
    sx, ey = np.sin(np.pi * pts[0]), np.exp(pts[1])
    if d == 2:
        f = (np.pi ** 2 - 1) * np.outer(ey, sx)
        faces = {(1, 0): -sx, (1, 1): np.e * sx}
    else:
        sz = np.sin(np.pi * pts[2])
        f = (2 * np.pi ** 2 - 1) * np.einsum('k,j,i->kji', sz, ey, sx)
        faces = {(1, 0): -np.outer(sz, sx), (1, 1): np.e * np.outer(sz, sx)}
    return f, faces


CASES = [(2, [12, 9]), (2, [37, 21]), (3, [6, 7, 5])]


@pytest.mark.parametrize('d,ne', CASES)
@pytest.mark.parametrize('p', [2, 3])
@pytest.mark.parametrize('test', ['pw', 'galerkin'])
@pytest.mark.parametrize('prec', ['fp64', 'fp32r'])
def test_mixed_apply_rhs_solve(d, ne, p, test, prec):
    import torch
    from paper_1910_08535_gb300 import workloads
    from paper_1910_08535_gb300.igapw import Context
    neumann = 2                                      # the y axis carries the flux data
    nm = [bool((neumann >> a) & 1) for a in range(d)]
    c = Context(dim=d, n_elem=ne, degree=p, nq=p + 1, test=test, bc='dirichlet0', precision=prec, op='poisson',
                neumann_axes=neumann)
    axes = _axes(ne, p, test, neumann)
    tol = TOL[prec]
    u = workloads.uniform_coeffs(c.shape, seed=31)
    r = c.to_numpy(c.apply('poisson', c.from_numpy(u)))
    ref = LM.apply(axes, nm, u)
    assert rel_err(r, ref) < tol, rel_err(r, ref)
    pts = [c.quad_points(a)[0] for a in range(d)]
    f, faces = _data(pts, d)
    dt = np.float64 if prec == 'fp64' else np.float32
    if prec == 'fp32r':
        f = f.astype(np.float32).astype(np.float64)
        faces = {k: v.astype(np.float32).astype(np.float64) for k, v in faces.items()}
    b = c.rhs_source(torch.from_numpy(f.astype(dt)).cuda())
    for (axis, side), g in faces.items():
        c.rhs_neumann(axis, side, torch.from_numpy(np.ascontiguousarray(g, dtype=dt)).cuda(), b)
    b_ref = LM.rhs(axes, nm, f, faces)
    assert rel_err(c.to_numpy(b), b_ref) < tol, rel_err(c.to_numpy(b), b_ref)
    sol = c.to_numpy(c.solve(b))
    s_ref = LM.solve(axes, nm, b_ref)
    assert rel_err(sol, s_ref) < tol, rel_err(sol, s_ref)
    c.sync()
    c.close()


def test_mixed_2d_256_converges():
    """256^2 cubic PW: the manufactured error is at the discretisation level
    (rate-4 prediction from the coarse meshes) and matches a sparse direct
    solve of the oracle's matrix."""
    import torch
    from paper_1910_08535_gb300.igapw import Context
    ne, p = [256, 256], 3
    c = Context(dim=2, n_elem=ne, degree=p, nq=4, test='pw', bc='dirichlet0', precision='fp64', op='poisson',
                neumann_axes=2)
    axes = _axes(ne, p, 'pw', 2)
    pts = [c.quad_points(a)[0] for a in range(2)]
    f, faces = _data(pts, 2)
    b = c.rhs_source(torch.from_numpy(f).cuda())
    for (axis, side), g in faces.items():
        c.rhs_neumann(axis, side, torch.from_numpy(np.ascontiguousarray(g)).cuda(), b)
    sol = c.to_numpy(c.solve(b))
    c.close()
    ref = LM.solve(axes, [False, True], LM.rhs(axes, [False, True], f, faces), sparse=True)
    assert rel_err(sol, ref) < TOL['fp64'], rel_err(sol, ref)
    err = poisson_nd.l2_error(axes, sol, lambda cc: np.sin(np.pi * cc[0]) * np.exp(cc[1]), nq_err=3)
    assert err < 1e-8, err


def test_neumann_descriptor_errors():
    from paper_1910_08535_gb300.igapw import Context, IgapwError
    with pytest.raises(IgapwError):       # every axis Neumann: singular
        Context(dim=2, n_elem=6, degree=2, nq=3, bc='dirichlet0', op='poisson', neumann_axes=3)
    with pytest.raises(IgapwError):       # Neumann data needs the POISSON system
        Context(dim=2, n_elem=6, degree=2, nq=3, bc='dirichlet0', op='heat', neumann_axes=1)
    c = Context(dim=2, n_elem=6, degree=2, nq=3, bc='dirichlet0', op='poisson', neumann_axes=2)
    with pytest.raises(IgapwError):       # axis 0 is a Dirichlet axis
        c.rhs_neumann(0, 1, c.empty(), c.empty())
    c.close()
