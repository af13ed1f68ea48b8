"""Precision study of the split explicit step (Sec. 4.2, Eq. (6)) in numpy:
which parts of the double-float step can run in plain FP32 and still meet
the FP32-path tolerance (rel-L2 <= 1e-5, and max-abs <= 1e-5 max|ref|)
against the FP64 oracle on the heat workloads.  Not a test (pytest does not
collect it); run

  python tests/study_step_precision.py 128 50 pw 3 3      # heat3d, PW
  python tests/study_step_precision.py 128 50 galerkin 3 3
  python tests/study_step_precision.py 256 200 pw 2 2     # heat2d

arguments: elements per axis, steps, test, degree, dimension.  Each variant
runs the split step u' = u + dt sum_a A_a^{-1} C_a u with the contraction
g = C u and the banded LU solve in the precision named:

  fp64        everything FP64 (the split form's own rounding; control)
  g64_s32     g exact, FP32 substitution (no refinement)
  f32         g in FP32 (FP32 tables and state), FP32 substitution
  mixed       g in FP32 except the first/last 3 rows of every line, FP32
              substitution, FP32 accumulation across axes
  g64_ref32   g exact, FP32 solve + one refinement with an FP32 residual
  g64_ref64   g exact, FP32 solve + one refinement with an exact residual
              (what the library's FP32-pair step does, in double-float)
  gdiff_ref64 g in the difference form sum_w c_w (u_w - u_i) (every row of C
              sums to zero, so the FP32 rounding of C's row sum drops out)
              with FP32 differences, products and sums, then as g64_ref64
"""
import sys
import time

import numpy as np

sys.path.insert(0, __file__.rsplit('/tests/', 1)[0])
from oracle import heat, systems  # noqa: E402
from paper_1910_08535_gb300 import workloads  # noqa: E402

B = 3   # boundary rows per line end kept exact in the 'mixed' variant


def main(ne, steps, test, p, dim):
    ax = systems.Axis(ne, p, p + 1, test, 'none')
    A, C = systems.mass(ax), systems.laplace(ax)
    n = A.shape[0]
    h = 1.0 / ne
    if dim == 3:
        dt, u0 = 0.05 * h * h, workloads.normal_coeffs((n,) * 3, seed=0)
    else:
        dt, u0 = 0.1 * h * h, workloads.gaussian_bump_2d(ne, p, seed=0)
    # banded LU without pivoting
    M = A.copy()
    Lf = np.eye(n)
    for k in range(n):
        for i in range(k + 1, min(n, k + p + 1)):
            Lf[i, k] = M[i, k] / M[k, k]
            M[i, k:] -= Lf[i, k] * M[k, k:]
    Uf = np.triu(M)

    def along(mat, arr, a):
        d = arr.ndim - 1 - a
        return np.moveaxis(np.tensordot(mat, arr, axes=([1], [d])), 0, d)

    def subst(g, a, dt_):
        d = g.ndim - 1 - a
        x = np.moveaxis(g, d, 0).astype(dt_).copy()
        L_, U_, di = Lf.astype(dt_), Uf.astype(dt_), (1.0 / np.diag(Uf)).astype(dt_)
        for i in range(n):
            for m in range(1, p + 1):
                if i - m >= 0:
                    x[i] = x[i] - L_[i, i - m] * x[i - m]
        for i in range(n - 1, -1, -1):
            for m in range(1, p + 1):
                if i + m < n:
                    x[i] = x[i] - U_[i, i + m] * x[i + m]
            x[i] = x[i] * di[i]
        return np.moveaxis(x, 0, d).astype(np.float64)

    C32, A32 = C.astype(np.float32), A.astype(np.float32)

    def g_exact(u, a):
        return along(C, u, a)

    def g_f32(u, a):
        return along(C32, u.astype(np.float32), a).astype(np.float64)

    def g_mixed(u, a):
        g, gx = g_f32(u, a), g_exact(u, a)
        for s in (slice(0, B), slice(n - B, n)):
            sl = [slice(None)] * u.ndim
            sl[u.ndim - 1 - a] = s
            g[tuple(sl)] = gx[tuple(sl)]
        return g

    def inc(gf, solve, acc32=False):
        def f(u):
            acc = None
            for a in range(u.ndim):
                w = solve(gf(u, a), a)
                if acc32:
                    w = w.astype(np.float32).astype(np.float64)
                    acc = w if acc is None else (acc + w).astype(np.float32).astype(np.float64)
                else:
                    acc = w if acc is None else acc + w
            return acc
        return f

    offs = sorted({j - i for i in range(n) for j in range(n) if C[i, j] != 0})

    def g_diff(u, a):
        d = u.ndim - 1 - a
        x = np.moveaxis(u, d, 0)
        g = np.zeros(x.shape, dtype=np.float32)
        for o in offs:
            rows = np.arange(max(0, -o), min(n, n - o))
            c = C32[rows, rows + o].reshape((-1,) + (1,) * (x.ndim - 1))
            dif = (x[rows + o] - x[rows]).astype(np.float32)
            g[rows] = g[rows] + (c * dif).astype(np.float32)
        return np.moveaxis(g.astype(np.float64), 0, d)

    def refine(resid):
        def s(g, a):
            w0 = subst(g.astype(np.float32), a, np.float32)
            if resid == 'f32':
                rho = (g.astype(np.float32) - along(A32, w0.astype(np.float32), a)).astype(np.float64)
            else:
                rho = g - along(A, w0, a)
            return w0 + subst(rho.astype(np.float32), a, np.float32)
        return s

    variants = {
        'fp64': inc(g_exact, lambda g, a: subst(g, a, np.float64)),
        'g64_s32': inc(g_exact, lambda g, a: subst(g, a, np.float32)),
        'f32': inc(g_f32, lambda g, a: subst(g, a, np.float32)),
        'mixed': inc(g_mixed, lambda g, a: subst(g, a, np.float32), acc32=True),
        'g64_ref32': inc(g_exact, refine('f32')),
        'g64_ref64': inc(g_exact, refine('exact')),
        'gdiff_ref64': inc(g_diff, refine('exact')),
    }
    t = time.time()
    ref = heat.run([ax] * dim, u0, dt, steps)
    print(f'{test} p={p} d={dim} N={ne} steps={steps}: oracle {time.time() - t:.1f}s, '
          f'norm growth {np.linalg.norm(ref) / np.linalg.norm(u0):.3g}', flush=True)
    for name, f in variants.items():
        u = u0.copy()
        for _ in range(steps):
            u = u + dt * f(u)
        e = u - ref
        print(f'  {name:10s} rel-L2 {np.linalg.norm(e) / np.linalg.norm(ref):.3e}  '
              f'max-abs/max|ref| {np.abs(e).max() / np.abs(ref).max():.3e}', flush=True)


if __name__ == '__main__':
    a = sys.argv[1:]
    main(int(a[0]), int(a[1]), a[2], int(a[3]), int(a[4]))
