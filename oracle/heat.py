"""Explicit Euler heat steps, u_t = Lap u (oracle; test infrastructure only).

Sec. 4.2, Eqs. (5)-(6): (v, u_{t+1}) = (v, u_t + Dt F u_t + Dt RHS).  With
F = Laplacian and RHS = 0 every step is an L2 projection: generate the
right-hand side T(u_t + Dt Lap u_t) with the chosen tests T (PW indicators or
B-splines), then solve with the mass matrix, factorized once and reused
(ADS, Sec. 4.1).  No boundary condition enters the non-integrated form.
"""
import numpy as np

from . import tensor


def step_quadrature(axes, u, dt, masses=None):
    """One step with the RHS generated point by point (tensor quadrature grid)."""
    masses = tensor.mass_mats(axes) if masses is None else masses
    r = tensor.rhs_heat_quadrature(axes, u, dt)
    return tensor.ads_solve(masses, r)


def run(axes, u0, dt, nsteps, route='system'):
    """``nsteps`` explicit steps from u0.

    route='system'     RHS from the assembled 1D systems (Kronecker form);
    route='quadrature' RHS from the quadrature grid (small meshes only).
    Both solve with the pivoted-LU ADS solve.
    """
    masses = tensor.mass_mats(axes)
    laps = tensor.lap_mats(axes)
    u = np.asarray(u0, dtype=np.float64).copy()
    for _ in range(nsteps):
        if route == 'quadrature':
            r = tensor.rhs_heat_quadrature(axes, u, dt)
        else:
            r = tensor.apply_heat_system(axes, u, dt, masses, laps)
        u = tensor.ads_solve(masses, r)
    return u
