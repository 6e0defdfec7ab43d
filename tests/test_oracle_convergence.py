"""Observed order of convergence of the oracle's scheme on a smooth exact
solution (CPU; pins the whole semi-discrete scheme of Sect. 2-3 with its
order separation and the SSP-RK3 time stepping).

The smooth solution is a steady vortex in cyclostrophic balance over a flat
bottom, an exact solution of the unforced shallow water equations (Eq. 1-5
with h_b = const, no friction, no Coriolis): with r the distance from the
centre, azimuthal velocity u_theta = A r exp(-r^2 / (2 sigma^2)) and
g d(xi)/dr = u_theta^2 / r, i.e. xi = -(A^2 sigma^2 / (2 g)) exp(-r^2 / sigma^2);
the flow is divergence free and the pressure gradient balances the
centripetal acceleration, so the exact state does not change in time.  The
vortex decays to 4e-6 of its peak speed at the walls of the unit square.

The error is || c(T) - c(0) || (the coefficient vectors are orthonormal
coordinates, so this is the L2 distance of the discrete solution at T from the
L2 projection of the exact one), on split-square grids with fixed dt = T / N
at CFL 0.1.  The observed order between the two finest grids must be at least
p + 1 - 0.35 (measured: p = 0: 0.95 on 64 -> 128, p = 1: 2.29 on 16 -> 32,
p = 2: 2.79 on 32 -> 64, still rising towards 3, p = 3: 3.94 on 16 -> 32);
a dropped or mis-signed term of the flux, the pressure or the velocity solve
collapses it.
"""
import numpy as np
import pytest

import oracle as O
from paper_2311_11348_gb300 import inputs

G, A, SIGMA = 1.0, 1.0, 0.1


def vortex(x, y):
    dx, dy = x - 0.5, y - 0.5
    r2 = dx * dx + dy * dy
    w = A * np.exp(-r2 / (2 * SIGMA * SIGMA))  # u_theta / r
    xi = -(A * A * SIGMA * SIGMA / (2 * G)) * np.exp(-r2 / (SIGMA * SIGMA))
    H = 1.0 + xi
    return xi, -H * w * dy, H * w * dx


def error_after(p, n, T):
    xy, tri = inputs.split_square_mesh(n, 1.0)
    m = O.Mesh(xy, tri, np.ones(len(xy)), np.full(len(tri), p, np.int8))
    P = O.Params(g=G, cfl=0.1, rk_order=3)
    c0 = m.project_state(vortex, n=10)
    steps = int(np.ceil(T / m.dt(P, c0)))
    c, _ = m.run(P, c0, 0.0, steps, T / steps)
    return float(np.sqrt(np.sum((c - c0) ** 2)))


def test_the_vortex_is_a_steady_solution():
    """the exact fields satisfy the steady equations pointwise (finite differences)"""
    x = np.linspace(0.2, 0.8, 61)
    X, Y = np.meshgrid(x, x, indexing="ij")
    h = 1e-5
    xi, U, V = vortex(X, Y)
    H = 1.0 + xi
    u, v = U / H, V / H

    def d(f, axis):
        if axis == 0:
            return (f(X + h, Y) - f(X - h, Y)) / (2 * h)
        return (f(X, Y + h) - f(X, Y - h)) / (2 * h)

    def flux(i):
        def f(a, b):
            xi_, U_, V_ = vortex(a, b)
            H_ = 1.0 + xi_
            return [U_, V_, U_ * U_ / H_ + 0.5 * G * H_ * H_, U_ * V_ / H_, V_ * V_ / H_ + 0.5 * G * H_ * H_][i]
        return f

    mass = d(flux(0), 0) + d(flux(1), 1)
    momx = d(flux(2), 0) + d(flux(3), 1)
    momy = d(flux(3), 0) + d(flux(4), 1)
    scale = np.abs(U).max()
    assert np.abs(mass).max() < 1e-6 * scale
    assert np.abs(momx).max() < 1e-6 * scale and np.abs(momy).max() < 1e-6 * scale
    assert np.abs(u).max() > 0.05 and np.abs(xi).max() > 1e-3  # not a trivial state


@pytest.mark.parametrize("p, grids, T", [(0, (32, 64, 128), 0.05), (1, (8, 16, 32), 0.1), (2, (16, 32, 64), 0.02),
                                         pytest.param(3, (8, 16, 32), 0.02, marks=pytest.mark.slow)])
def test_observed_order_is_p_plus_one(p, grids, T):
    e = [error_after(p, n, T) for n in grids]
    rates = [np.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
    assert e[0] > e[1] > e[2]
    assert rates[-1] >= p + 1 - 0.35, (p, e, rates)
