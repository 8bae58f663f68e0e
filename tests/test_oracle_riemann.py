"""Pins of the oracle's augmented Riemann solver (Sec. 3.3) against facts the
method and the mathematics fix: flux-difference splitting with the bathymetry
source, well balancing, mirror symmetry, dam-break front speeds, positivity of
the middle depths and the reflecting-wall test.  None of these re-types the
solver's formulas; each compares with a closed form or an invariant."""
import numpy as np
import pytest

import oracle

G = 9.81
TOL = 1e-3


def flux(h, n, t):
    """Physical flux of the 1D system in the normal frame (Sec. 3.2)."""
    if h <= 0:
        return np.zeros(3)
    return np.array([n, n * n / h + 0.5 * G * h * h, n * t / h])


def fluctuations(Z, s):
    am = np.zeros(3)
    ap = np.zeros(3)
    for p in range(3):
        if s[p] < 0:
            am += Z[p]
        elif s[p] > 0:
            ap += Z[p]
        else:
            am += 0.5 * Z[p]
            ap += 0.5 * Z[p]
    return am, ap


def test_dry_dry_gives_no_waves():
    Z, s = oracle.riemann(5e-4, 1e-4, 0.0, 1.0, 0.0, 0.0, 0.0, 0.3, G, TOL)
    assert np.all(Z == 0) and np.all(s == 0)


def test_flux_difference_splitting_with_source():
    """Wet-wet: the f-waves sum to f(QR) - f(QL) - psi, psi = (0, -g hbar db, 0)
    (Sec. 3.2: the source is folded into the Riemann solution)."""
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(2000):
        hL, hR = rng.uniform(0.05, 5.0, 2)
        uL, uR, vL, vR = rng.uniform(-3.0, 3.0, 4)
        bL, bR = rng.uniform(-0.3, 0.3, 2) * min(hL, hR)
        Z, s = oracle.riemann(hL, hL * uL, hL * vL, bL, hR, hR * uR, hR * vR, bR, G, TOL)
        expect = flux(hR, hR * uR, hR * vR) - flux(hL, hL * uL, hL * vL)
        expect[1] += G * 0.5 * (hL + hR) * (bR - bL)
        got = Z.sum(axis=0)
        scale = np.abs(flux(hR, hR * uR, hR * vR)).max() + np.abs(flux(hL, hL * uL, hL * vL)).max()
        worst = max(worst, np.abs(got - expect).max() / scale)
    assert worst < 1e-13


@pytest.mark.parametrize("h,u", [(1.0, 0.7), (2.5, -1.2), (0.2, 3.0)])
def test_mirror_states_have_zero_mass_flux(h, u):
    """(h, u | h, -u) on a flat bed is a reflecting wall: the interface mass
    flux f(QL) + A^-dQ vanishes."""
    Z, s = oracle.riemann(h, h * u, 0.3, 0.0, h, -h * u, 0.3, 0.0, G, TOL)
    am, ap = fluctuations(Z, s)
    assert abs(h * u + am[0]) <= 1e-14 * (1 + abs(h * u))


def test_lake_at_rest_edge_is_exactly_zero():
    """Still water over a bed step: all f-waves are exactly zero (dyadic data
    so that h + b is exact)."""
    for bL, bR in [(0.25, 0.5), (0.5, 0.125), (-0.75, 0.375)]:
        eta = 1.0
        Z, s = oracle.riemann(eta - bL, 0.0, 0.0, bL, eta - bR, 0.0, 0.0, bR, G, TOL)
        assert np.all(Z == 0.0)


def test_mirror_symmetry():
    """Solving the mirrored problem (x -> -x) gives the mirrored waves:
    wave p <-> 2-p, speeds negated, normal-momentum component negated."""
    rng = np.random.default_rng(2)
    for _ in range(500):
        hL, hR = rng.uniform(0.0, 4.0, 2)
        hL = 0.0 if hL < 0.3 else hL
        hR = 0.0 if hR < 0.3 else hR
        uL, uR, vL, vR = rng.uniform(-2.0, 2.0, 4)
        bL, bR = rng.uniform(-1.0, 1.0, 2)
        qL = (hL, hL * uL, hL * vL, bL)
        qR = (hR, hR * uR, hR * vR, bR)
        Z, s = oracle.riemann(*qL, *qR, G, TOL)
        M = lambda q: (q[0], -q[1], q[2], q[3])
        Zm, sm = oracle.riemann(*M(qR), *M(qL), G, TOL)
        for p in range(3):
            q = 2 - p
            np.testing.assert_allclose(sm[q], -s[p], rtol=1e-13, atol=1e-13)
            np.testing.assert_allclose(Zm[q], Z[p] * np.array([1.0, -1.0, 1.0]),
                                       rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("h0", [0.5, 2.0, 5.0])
def test_dry_bed_front_speeds(h0):
    """Wet | dry on a flat bed: the fastest wave is the dam-break (Ritter)
    front u + 2 sqrt(g h) and the slowest the rarefaction head u - sqrt(g h)."""
    Z, s = oracle.riemann(h0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, G, TOL)
    c = np.sqrt(G * h0)
    assert s[2] == pytest.approx(2 * c, rel=1e-15)
    assert s[0] == pytest.approx(-c, rel=1e-15)
    Zm, sm = oracle.riemann(0.0, 0.0, 0.0, 0.0, h0, 0.0, 0.0, 0.0, G, TOL)
    assert sm[0] == pytest.approx(-2 * c, rel=1e-15)


def test_einfeldt_bounds_and_positivity():
    """Wet-wet speeds bound the characteristic speeds of both states; the
    middle depths of the wave fan stay non-negative."""
    rng = np.random.default_rng(3)
    for _ in range(2000):
        hL, hR = rng.uniform(1e-2, 5.0, 2)
        uL, uR = rng.uniform(-8.0, 8.0, 2)
        bL, bR = rng.uniform(-2.0, 2.0, 2)
        Z, s = oracle.riemann(hL, hL * uL, 0.0, bL, hR, hR * uR, 0.0, bR, G, TOL)
        if Z[0, 0] == 0 and Z[2, 0] == 0 and Z[1, 1] == 0:
            continue  # a wall / degenerate edge
        assert s[0] <= uL - np.sqrt(G * hL) + 1e-12
        assert s[2] >= uR + np.sqrt(G * hR) - 1e-12
        assert s[0] < s[2]
        beta1 = Z[0, 0] / s[0] if s[0] != 0 else 0.0
        beta3 = Z[2, 0] / s[2] if s[2] != 0 else 0.0
        if s[0] < 0 < s[2]:
            assert hL + beta1 >= -1e-12 * (1 + hL)
            assert hR - beta3 >= -1e-12 * (1 + hR)


def test_wall_test_blocks_flow_into_high_dry_bed():
    """Slow water against a dry cell whose bed is far above the surface: the
    edge acts as a reflecting wall, so no mass enters the dry cell and the
    interface mass flux vanishes (Sec. 3.3, artificial Riemann problems)."""
    h, u = 1.0, 0.5
    Z, s = oracle.riemann(h, h * u, 0.0, 0.0, 0.0, 0.0, 0.0, 5.0, G, TOL)
    am, ap = fluctuations(Z, s)
    assert np.all(ap == 0.0)
    assert abs(h * u + am[0]) < 1e-14
    # a bed just above the surface but below the wall run-up is overtopped
    Z2, s2 = oracle.riemann(h, h * 3.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.05, G, TOL)
    am2, ap2 = fluctuations(Z2, s2)
    assert ap2[0] < 0.0  # mass flux enters the dry cell (dq = -nu * A^+dQ)
