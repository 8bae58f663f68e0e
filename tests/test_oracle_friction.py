"""Pins of the oracle's Manning friction (Sec. 3.1, Eq. manning, read with the
factor h the printed form lacks: the momentum sink is g n^2 (hu) |u| h^{-4/3},
applied after the hyperbolic update, semi-implicitly, on wet cells).

Each test checks the oracle against something the mathematics fixes, not a
retyped update:
  * on a uniform, flat, wet sheet the hyperbolic update is the identity and
    the momentum obeys the ODE d|u|/dt = -k |u|^2, k = g n^2 h^{-4/3}, whose
    solution is |u|(t) = |u0| / (1 + k |u0| t): 1/|u| grows linearly in t.
    The semi-implicit step s -> s / (1 + dt k s) adds exactly k dt to 1/s,
    so it reproduces the solution for any dt, to round-off, with the
    direction of the velocity kept;
  * on an inclined plane the bed slope S drives the flow, and the steady
    uniform flow is Manning's normal flow, S = n^2 q^2 / h^{10/3}, i.e.
    h = (n q / sqrt(S))^{3/5}, which the oracle's steady state reaches as
    dt -> 0.
An exponent h^{-1/3} in place of h^{-4/3}, n in place of n^2, a dropped
factor h, or u replaced by hu each moves these limits far outside the
tolerances below.
"""
import math

import numpy as np
import pytest

import oracle

G = 9.81


def sheet(nx, ny, h, hu, hv, b=None):
    shape = (ny + 4, nx + 4)
    arrs = [np.full(shape, v, dtype=np.float64) for v in (h, hu, hv)]
    arrs.append(np.zeros(shape) if b is None else b)
    return arrs


def test_uniform_sheet_decays_as_the_manning_ode():
    """|u|(T) from the oracle equals |u0| / (1 + k |u0| T) to round-off for
    every step size; h untouched, direction kept."""
    h0, u0, v0, n, T = 2.5, 1.2, -0.7, 0.05, 60.0
    s0 = math.hypot(u0, v0)
    k = G * n * n / h0 ** (4.0 / 3.0)
    exact = s0 / (1.0 + k * s0 * T)
    for nsteps in (1, 7, 60, 240):
        dt = T / nsteps
        h, hu, hv, b = sheet(8, 8, h0, h0 * u0, h0 * v0)
        for _ in range(nsteps):
            h, hu, hv, _, _ = oracle.step_grid(h, hu, hv, b, 5.0, 5.0, dt, g=G,
                                               drytol=1e-3, manning_n=n)
            # the sheet is uniform: every cell, ghosts included, takes the
            # interior value
            h, hu, hv = (np.full_like(a, a[4, 4]) for a in (h, hu, hv))
        assert h[4, 4] == h0, "the hyperbolic update of a uniform sheet is the identity"
        u, v = hu[4, 4] / h0, hv[4, 4] / h0
        assert abs(u * v0 - v * u0) <= 1e-14 * s0 * s0, "friction keeps the direction"
        err = abs(math.hypot(u, v) - exact) / exact
        assert err <= 1e-13 * nsteps, (nsteps, err)


def test_friction_acts_only_on_wet_cells_and_not_at_n_zero():
    """n = 0 leaves momentum untouched bit for bit; a cell at most drytol
    deep loses its momentum."""
    h, hu, hv, b = sheet(8, 8, 2.5, 3.0, -1.75)
    out = oracle.step_grid(h, hu, hv, b, 5.0, 5.0, 0.5, g=G, drytol=1e-3, manning_n=0.0)
    assert np.array_equal(out[1], hu) and np.array_equal(out[2], hv)
    h, hu, hv, b = sheet(8, 8, 1e-3, 1e-4, 1e-4)
    out = oracle.step_grid(h, hu, hv, b, 5.0, 5.0, 0.5, g=G, drytol=1e-3, manning_n=0.03)
    assert np.all(out[1][2:-2, 2:-2] == 0.0) and np.all(out[2][2:-2, 2:-2] == 0.0)


def plane_speed(S, n, h0, dt, direction, t_end=1200.0, dx=5.0):
    """Steady speed of uniform flow of depth h0 on the plane b = -S (d . x)
    (d a unit vector) with every ghost holding the same uniform flow (an
    infinite plane), stepped with a fixed dt from a slow start."""
    nx = ny = 8
    c = (np.arange(nx + 4) - 2 + 0.5) * dx
    X, Y = np.meshgrid(c, c)
    b = -S * (direction[0] * X + direction[1] * Y)
    h, hu, hv, _ = sheet(nx, ny, h0, 0.1 * h0 * direction[0], 0.1 * h0 * direction[1])
    t = 0.0
    while t < t_end:
        h, hu, hv, _, _ = oracle.step_grid(h, hu, hv, b, dx, dx, dt, g=G,
                                           drytol=1e-3, manning_n=n)
        t += dt
        assert np.allclose(hu[2:-2, 2:-2], hu[4, 4], rtol=1e-11, atol=1e-14)
        assert np.allclose(h[2:-2, 2:-2], h0, rtol=1e-13, atol=0.0)
        h, hu, hv = (np.full_like(a, a[4, 4]) for a in (h, hu, hv))
    u, v = hu[4, 4] / h0, hv[4, 4] / h0
    # the flow runs down the slope
    assert abs(u * direction[1] - v * direction[0]) <= 1e-12 * math.hypot(u, v)
    return math.hypot(u, v)


@pytest.mark.parametrize("h0,direction", [(0.8, (1.0, 0.0)), (1.6, (0.6, 0.8))])
def test_inclined_plane_tends_to_manning_normal_flow(h0, direction):
    """On the plane b = -S x' (x' along `direction`, so the diagonal case needs
    the speed sqrt(u^2 + v^2), not each component) the gravity source and
    the friction balance.  Friction acts after the source (splitting, Sec.
    3.2), so the steady speed of a step dt lies O(dt) below the exact one;
    as dt -> 0 it tends, at first order, to Manning's normal velocity
    sqrt(S) h^{2/3} / n, i.e. h = (n q / sqrt(S))^{3/5} for the unit
    discharge q = h u."""
    S, n = 0.002, 0.03
    u_normal = math.sqrt(S) * h0 ** (2.0 / 3.0) / n
    u1 = plane_speed(S, n, h0, 0.2, direction)
    u2 = plane_speed(S, n, h0, 0.1, direction)
    ratio = (u_normal - u1) / (u_normal - u2)
    assert 1.95 <= ratio <= 2.05, ratio
    u_limit = 2.0 * u2 - u1  # Richardson extrapolation of a first-order limit
    assert u_limit == pytest.approx(u_normal, rel=2e-6)
    h_normal = (n * h0 * u_limit / math.sqrt(S)) ** 0.6
    assert h_normal == pytest.approx(h0, rel=2e-6)
