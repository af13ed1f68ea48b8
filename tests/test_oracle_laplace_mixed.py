"""Pins of the mixed Dirichlet/Neumann Laplace oracle (Sec. 4.3): the
integrate-back-by-parts identity for B-spline tests, the flux of linear
functions, closed forms of the boundary data term, and manufactured solutions
with Neumann data converging at the expected rates."""
import numpy as np
import pytest

from oracle import bspline, laplace_mixed as LM, poisson_nd, quadrature, systems, tensor


@pytest.mark.parametrize('p', [2, 3, 4])
def test_galerkin_boundary_term_gives_ibp_stiffness(p):
    """-int B_i B_j'' + [B_i B_j']_a^b = int B_i' B_j' (Sec. 4.3: integrating
    back by parts on the discrete level)."""
    ax = systems.Axis(7, p, p + 1, 'galerkin', 'none')
    _, C = poisson_nd.raw_mats(ax)
    L = -C + LM.boundary_matrix(ax)
    S = -systems.laplace_ibp(ax)
    assert np.max(np.abs(L - S)) < 1e-12 * np.max(np.abs(S))


def test_galerkin_mixed_2d_equals_ibp_assembly():
    """2D: the assembled mixed system on the rows off the Dirichlet boundary
    equals the IBP stiffness S_x (x) M_y + M_x (x) S_y."""
    axes = [systems.Axis(5, 3, 4, 'galerkin', 'dirichlet0'), systems.Axis(6, 3, 4, 'galerkin', 'none')]
    K = LM.assemble(axes, [False, True])
    mats = [poisson_nd.raw_mats(ax)[0] for ax in axes]
    S = [-systems.laplace_ibp(ax) for ax in axes]
    ref = tensor.kron_dense([S[0], mats[1]]) + tensor.kron_dense([mats[0], S[1]])
    free = ~poisson_nd.boundary_mask(axes).ravel()
    assert np.max(np.abs(K[free] - ref[free])) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
@pytest.mark.parametrize('p', [2, 3])
def test_neumann_axis_flux_of_linear_functions(test, p):
    """On a Neumann axis, -C + E annihilates constants and maps u = x (Greville
    coefficients) to the boundary flux T(b) - T(a)."""
    ax = systems.Axis(9, p, p + 1, test, 'none')
    _, C = poisson_nd.raw_mats(ax)
    L = -C + LM.boundary_matrix(ax)
    one = np.ones(ax.n)
    assert np.max(np.abs(L @ one)) < 1e-10 * np.max(np.abs(L))
    g = quadrature.greville(ax.knots, p)
    flux = LM.test_at(ax, ax.knots[-1]) - LM.test_at(ax, ax.knots[0])
    assert np.max(np.abs(L @ g - flux)) < 1e-10 * np.max(np.abs(L))


@pytest.mark.parametrize('test', ['pw', 'galerkin'])
def test_test_values_at_the_ends(test):
    ax = systems.Axis(6, 3, 4, test, 'none')
    e0 = np.zeros(ax.n)
    e0[0] = 1.0
    e1 = np.zeros(ax.n)
    e1[-1] = 1.0
    assert np.array_equal(LM.test_at(ax, 0.0), e0)
    assert np.array_equal(LM.test_at(ax, 1.0), e1)


def test_face_term_of_unit_flux_closed_forms():
    """G = 1 on the face y = 1: int T_i(x) dx is the cell length (PW) or
    (t_{i+p+1} - t_i) / (p + 1) (B-splines), placed in the last y row."""
    for test in ('pw', 'galerkin'):
        p = 2
        axes = [systems.Axis(8, p, p + 1, test, 'dirichlet0'), systems.Axis(5, p, p + 1, test, 'none')]
        g = np.ones(len(axes[0].points()[0]))
        r = LM.face_rhs(axes, 1, 1, g)
        assert np.all(r[:-1] == 0.0)
        t = axes[0].knots
        if test == 'pw':
            c = quadrature.pw_cells(t, p, 'dirichlet0')
            want = np.zeros(axes[0].n)
            want[axes[0].rows()] = np.diff(c)
        else:
            want = np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(axes[0].n)])
            want[[0, -1]] = 0.0          # Dirichlet rows test nothing
        assert np.max(np.abs(r[-1] - want)) < 1e-14


def _manufactured(test, p, ne):
    axes = [systems.Axis(ne, p, p + 1, test, 'dirichlet0'), systems.Axis(ne, p, p + 1, test, 'none')]
    px, py = axes[0].points()[0], axes[1].points()[0]
    f = (np.pi ** 2 - 1) * np.outer(np.exp(py), np.sin(np.pi * px))
    faces = {(1, 0): -np.sin(np.pi * px), (1, 1): np.e * np.sin(np.pi * px)}
    b = LM.rhs(axes, [False, True], f, faces)
    u = LM.solve(axes, [False, True], b)
    return poisson_nd.l2_error(axes, u, lambda c: np.sin(np.pi * c[0]) * np.exp(c[1]))


@pytest.mark.parametrize('test,p,lo', [('pw', 2, 1.9), ('pw', 3, 3.8), ('galerkin', 2, 2.9), ('galerkin', 3, 3.8)])
def test_manufactured_neumann_convergence(test, p, lo):
    """u = sin(pi x) e^y: zero on x = 0, 1; flux du/dn = e sin(pi x) on y = 1 and
    -sin(pi x) on y = 0; -Lap u = (pi^2 - 1) u."""
    errs = [_manufactured(test, p, ne) for ne in (4, 8, 16)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > lo), rates


def test_all_dirichlet_reduces_to_poisson_nd():
    axes = [systems.Axis(5, 2, 3, 'pw', 'dirichlet0'), systems.Axis(4, 2, 3, 'pw', 'dirichlet0')]
    assert np.array_equal(LM.assemble(axes, [False, False]), poisson_nd.assemble(axes))


def test_neumann_pencil_spectrum_real_nonnegative():
    """The Neumann 1D pencil has a real spectrum with one zero eigenvalue (the
    constants) and well-conditioned eigenvectors: fast diagonalisation applies
    when another axis is Dirichlet."""
    for test in ('pw', 'galerkin'):
        ax = systems.Axis(32, 3, 4, test, 'none')
        A, C = poisson_nd.raw_mats(ax)
        lam, V = np.linalg.eig(np.linalg.solve(A, -C + LM.boundary_matrix(ax)))
        assert np.max(np.abs(lam.imag)) < 1e-8 * np.max(np.abs(lam.real))
        assert np.sort(lam.real)[0] > -1e-8 * np.max(lam.real)
        assert np.sort(lam.real)[1] > 1.0
        assert np.linalg.cond(V) < 10


def test_sparse_assembly_and_solve_match_dense():
    axes = [systems.Axis(5, 3, 4, 'pw', 'dirichlet0'), systems.Axis(6, 3, 4, 'pw', 'none')]
    nm = [False, True]
    K = LM.assemble(axes, nm)
    assert np.max(np.abs(LM.assemble_sparse(axes, nm).toarray() - K)) == 0.0
    b = np.random.default_rng(3).standard_normal((9, 8))
    assert np.max(np.abs(LM.solve(axes, nm, b, sparse=True) - LM.solve(axes, nm, b))) < 1e-10
