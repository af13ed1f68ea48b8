"""Seeded synthetic inputs shaped like the paper's experiments.

This module holds input recipes only (no arithmetic of the method): it is the
one piece shared by the CUDA path's callers and the oracle's tests.  Random
numbers come from numpy's PCG64 with explicit seeds.

Workloads
  poisson1d   1D Poisson -u'' = f on [0,1], zero Dirichlet, p=2, 64 elements,
              3 Gauss points, f = pi^2 sin(pi x) (exact u = sin(pi x)).
  heat2d      2D explicit heat u_t = Lap u, p=2, 256x256 elements, 3x3 Gauss
              points, dt = 0.1 h^2, 200 steps; initial coefficients: a Gaussian
              bump (centre (0.5,0.5), sigma 0.1) sampled at the knot averages
              (Greville abscissae) plus uniform noise of amplitude 1e-3.
  heat3d      3D explicit heat, p=3 (cubic C2), 128^3 elements (131^3 =
              2,248,091 coefficients), 4x4x4 Gauss points, dt = 0.05 h^2,
              50 steps; coefficients 1e-2 * N(0,1).
  The paper's own experiments (Tables 1, 1a, 2) use no public dataset; these
  seeded inputs have their shapes.
"""
import numpy as np

WORKLOADS = {
    'poisson1d': dict(dim=1, n_elem=64, degree=2, nq=3, bc='dirichlet0', op='poisson'),
    'heat2d': dict(dim=2, n_elem=256, degree=2, nq=3, bc='none', op='heat', dt_h2=0.1, steps=200),
    'heat3d': dict(dim=3, n_elem=128, degree=3, nq=4, bc='none', op='heat', dt_h2=0.05, steps=50),
}


def knot_averages(n_elem, p):
    """Sampling abscissae for initial coefficients: averages of p consecutive
    knots of the open uniform knot vector on [0, 1] (an input recipe)."""
    t = [0.0] * (p + 1) + [k / n_elem for k in range(1, n_elem)] + [1.0] * (p + 1)
    n = n_elem + p
    return np.array([sum(t[j + 1:j + p + 1]) / p for j in range(n)])


def gaussian_bump_2d(n_elem, p, seed=0, sigma=0.1, noise=1e-3):
    """(n, n) coefficients, y slowest: exp(-|x - c|^2 / (2 sigma^2)) + U(-noise, noise)."""
    xi = knot_averages(n_elem, p)
    X, Y = np.meshgrid(xi, xi, indexing='xy')
    g = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * sigma ** 2))
    rng = np.random.Generator(np.random.PCG64(seed))
    return g + rng.uniform(-noise, noise, size=g.shape)


def normal_coeffs(shape, seed=0, scale=1e-2):
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal(shape)


def uniform_coeffs(shape, seed=0, lo=-1.0, hi=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)


def sine_source(x):
    """f = pi^2 sin(pi x), the source of u = sin(pi x) for -u'' = f."""
    return np.pi ** 2 * np.sin(np.pi * x)


def sine_exact(x):
    return np.sin(np.pi * x)


def tensor_samples(points, fn_list):
    """Sum over terms of products fn[a](x_a) on the tensor grid of 1D point
    sets, x fastest: shape (len(z), len(y), len(x))[-d:]."""
    d = len(points)
    out = 0.0
    for fns in fn_list:
        term = np.ones(1)
        for a in reversed(range(d)):
            term = np.multiply.outer(term, fns[a](points[a])) if term.ndim else term
        out = out + term.reshape([len(points[a]) for a in reversed(range(d))])
    return out


def sine_product_source(points, k):
    """f = pi^2 (sum_a k_a^2) prod_a sin(k_a pi x_a) on the tensor grid of the
    1D point sets: the source of u = prod_a sin(k_a pi x_a) for -Lap u = f."""
    fns = tuple((lambda x, kk=kk: np.sin(kk * np.pi * x)) for kk in k)
    return np.pi ** 2 * sum(kk * kk for kk in k) * tensor_samples(points, [fns])


def sine_product_exact(k):
    """u = prod_a sin(k_a pi x_a) on coordinate arrays (x first)."""
    def u(coords):
        r = 1.0
        for a, x in enumerate(coords):
            r = r * np.sin(k[a] * np.pi * x)
        return r
    return u


def batch_shapes(count, seed=0, lo=32, hi=512, rungs=16):
    """Shapes (n_elem_x, n_elem_y, degree) of a batch of square 2D instances:
    N log-uniform on `rungs` geometric rungs from lo to hi, degree uniform in
    {2, 3}."""
    ladder = np.unique(np.round(np.geomspace(lo, hi, rungs)).astype(int))
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        n = int(ladder[int(rng.integers(0, len(ladder)))])
        out.append((n, n, int(rng.integers(2, 4))))
    return out


def initial_state(name, seed=0):
    w = WORKLOADS[name]
    n = w['n_elem'] + w['degree']
    if name == 'heat2d':
        return gaussian_bump_2d(w['n_elem'], w['degree'], seed)
    if name == 'heat3d':
        return normal_coeffs((n, n, n), seed)
    raise KeyError(name)


def dt_of(name):
    w = WORKLOADS[name]
    return w['dt_h2'] / w['n_elem'] ** 2
