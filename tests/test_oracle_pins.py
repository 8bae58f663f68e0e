"""Integration pins of the oracle's wave-propagation step (Sec. 3.2, 3.3) and
forest geometry (Sec. 4) against closed forms and invariants: Stoker and
Ritter dam breaks, lake at rest over a bump (submerged and emerged), exact
mass conservation with walls, four-fold symmetry of a radial dam break,
stability of the transverse terms at CFL 0.9, the effective-resolution values
the paper prints, and the bilinear DEM cell average."""
import math
import os

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_2403_15435_gb300 import inputs

G = 9.81
HERE = os.path.dirname(os.path.abspath(__file__))


def run(prob, t_end=None, max_steps=1 << 30):
    f = oracle.OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    f.step(prob.t_end if t_end is None else t_end, max_steps)
    return f


def assemble(f, field=0):
    """Uniform-level forest -> global [NY][NX] array."""
    cfg = f.cfg
    L, X, Y = f.patch_info()
    arr = f.read()[field]
    m = cfg.mx
    lev = int(L[0])
    assert np.all(L == lev)
    out = np.zeros((cfg.mj * m << lev, cfg.mi * m << lev))
    for k in range(len(L)):
        out[Y[k] * m:(Y[k] + 1) * m, X[k] * m:(X[k] + 1) * m] = arr[k]
    return out


# ---------------------------------------------------------------- Stoker --

def stoker_exact(x, t, hl=2.0, hr=0.5, x0=320.0):
    """Dam break on a wet bed: left rarefaction, right shock (closed form)."""
    cl = math.sqrt(G * hl)
    f = lambda hm: 2 * (cl - math.sqrt(G * hm)) - (hm - hr) * math.sqrt(0.5 * G * (1 / hm + 1 / hr))
    hm = brentq(f, hr, hl, xtol=1e-15)
    um = 2 * (cl - math.sqrt(G * hm))
    s = hm * um / (hm - hr)
    xi = (x - x0) / t
    cm = math.sqrt(G * hm)
    h = np.full_like(x, hl)
    rare = (xi > -cl) & (xi < um - cm)
    h[rare] = ((2 * cl - xi[rare]) / 3) ** 2 / G
    h[(xi >= um - cm) & (xi < s)] = hm
    h[xi >= s] = hr
    return h, hm, um, s


def test_stoker_closed_form_values():
    _, hm, um, s = stoker_exact(np.zeros(1), 1.0)
    assert hm == pytest.approx(1.10349, abs=1e-5)
    assert um == pytest.approx(2.27854, abs=1e-5)
    assert s == pytest.approx(4.16632, abs=1e-5)


def test_stoker_dam_break_converges():
    errs = []
    for n in (128, 256):
        f = run(inputs.stoker(n))
        h = assemble(f, 0)
        hv = assemble(f, 2)
        x = (np.arange(n) + 0.5) * 640.0 / n
        he, *_ = stoker_exact(x, 20.0)
        errs.append(np.abs(h.mean(axis=0) - he).sum() / np.abs(he).sum())
        assert np.all(h == h[0:1, :]), "1D-in-2D rows must be identical"
        assert np.all(hv == 0.0)
    assert errs[0] <= 0.02
    assert errs[1] < errs[0]
    assert math.log2(errs[0] / errs[1]) >= 0.6


def test_ritter_dry_dam_break_front():
    """Dam break onto a dry flat bed (Ritter): the depth profile
    h = (2 c0 - x/t)^2 / (9 g) is approached at first order in L1, and the
    wet front (h > 1e-4 m) approaches x0 + 2 sqrt(g h0) t from behind as the
    grid is refined (the thin film at the tip is smeared over a few cells)."""
    h0, x0, t = 1.0, 160.0, 10.0
    c0 = math.sqrt(G * h0)
    front_exact = x0 + 2 * c0 * t
    errs, lags = [], []
    for n in (256, 512):
        prob = inputs.stoker(n)
        prob.cfg.drytol = 1e-4
        prob.ic = lambda x, y, b: (np.where(x < x0, h0, 0.0), np.zeros_like(x), np.zeros_like(x))
        f = run(prob, t_end=t)
        h = assemble(f, 0)[0]
        dx = 640.0 / n
        x = (np.arange(n) + 0.5) * dx
        xi = (x - x0) / t
        he = np.where(xi <= -c0, h0, np.where(xi < 2 * c0, (2 * c0 - xi) ** 2 / (9 * G), 0.0))
        errs.append(np.abs(h - he).sum() / np.abs(he).sum())
        front = x[np.nonzero(h > 1e-4)[0][-1]] + 0.5 * dx
        lags.append(front_exact - front)
        assert np.all(h[x > front_exact + dx] == 0.0), "no water ahead of the front"
    assert errs[0] <= 0.02 and errs[1] <= 0.6 * errs[0]
    assert 0.0 <= lags[1] < lags[0] <= 0.25 * (front_exact - x0)


# ----------------------------------------------------------- lake at rest --

@pytest.mark.parametrize("n,eta", [(64, 1.0), (64, 0.3), (128, 0.3)])
def test_lake_at_rest_is_preserved(n, eta):
    """Still water over a Gaussian bump stays at rest to round-off for 1000
    steps, submerged (eta = 1) and emerged (eta = 0.3); at 128 cells the
    shoreline has cells with 0 < h <= drytol (Sec. 3.3)."""
    prob = inputs.lake_at_rest(n, patch=32, eta=eta)
    prob.cfg.dt_initial = 0.5
    f = oracle.OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    h0 = f.read()[0]
    f.step(1e9, 1000)
    h, hu, hv, b = f.read()
    wet = h > prob.cfg.drytol
    assert np.abs((h + b)[wet] - eta).max() <= 1e-13
    assert np.abs(h - h0).max() <= 1e-13  # dry cells keep their film too
    assert np.abs(hu).max() <= 1e-13 and np.abs(hv).max() <= 1e-13
    assert f.time()["steps"] == 1000


# ------------------------------------------------------------------ mass --

def test_mass_conserved_with_walls_wet():
    prob = inputs.stoker(128, patch=32)
    f = oracle.OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    m0 = f.mass()
    f.step(20.0)
    assert abs(f.mass() - m0) / m0 <= 1e-13


def test_mass_conserved_with_walls_dry_front_and_friction():
    """Dry bed, terrain and Manning friction: the flux form conserves volume
    exactly; the only change is the volume added where a negative depth is
    reset to zero, which the step reports."""
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0)
    f = oracle.OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    m0 = f.mass()
    f.step(20.0)
    info = f.time()
    assert abs(f.mass() - m0 - info["clipvol"]) / m0 <= 1e-13
    assert info["clipvol"] / m0 < 1e-5


def test_mass_exact_on_flat_dry_bed():
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0, flat=True)
    f = oracle.OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    m0 = f.mass()
    f.step(20.0)
    assert f.time()["nclip"] == 0
    assert abs(f.mass() - m0) / m0 <= 1e-13


# -------------------------------------------------------------- symmetry --

def test_radial_dam_break_fourfold_symmetry():
    """Radial dam break on a flat bed keeps the symmetries of its square grid:
    h(i,j) = h(N-1-i,j) = h(i,N-1-j) = h(j,i) (Sec. 5.1 motivates this)."""
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0, flat=True)
    f = run(prob, t_end=15.0)
    h = assemble(f, 0)
    scale = np.abs(h).max()
    for other in (h[:, ::-1], h[::-1, :], h.T):
        assert np.abs(h - other).max() <= 1e-12 * scale
    hu = assemble(f, 1)
    hv = assemble(f, 2)
    assert np.abs(hu - hv.T).max() <= 1e-12 * np.abs(hu).max()
    assert np.abs(hu + hu[:, ::-1]).max() <= 1e-12 * np.abs(hu).max()


def test_transverse_terms_keep_diagonal_flow_stable():
    """Uniform diagonal flow with a small hump at CFL 0.9: the unsplit scheme
    is stable only with correct transverse propagation (without it the bound
    is CFL 0.5 in 2D), so the solution must stay bounded and smooth."""
    n = 64
    prob = inputs.stoker(n, patch=32)
    prob.cfg.bc = (inputs.BC_EXTRAP,) * 4
    u0 = 2.0

    def ic(x, y, b):
        h = 1.0 + 0.01 * np.exp(-((x - 320) ** 2 + (y - 320) ** 2) / (2 * 40.0 ** 2))
        return h, u0 * h, u0 * h

    prob.ic = ic
    f = run(prob, t_end=30.0)
    h = assemble(f, 0)
    assert np.isfinite(h).all()
    assert h.max() < 1.011 and h.min() > 0.99


# -------------------------------------------------- equivalence (ghost copy) --

def test_patches_equal_single_grid_bitwise():
    """A uniform forest of 4x4 patches advances exactly like one 128x128 grid:
    same-level ghost copy and the wall boundary are exact."""
    big = inputs.radial_dambreak(128, 128, dx=4.0, radius=120.0)
    small = inputs.radial_dambreak(128, 32, dx=4.0, radius=120.0)
    fa = run(big, t_end=6.0)
    fb = run(small, t_end=6.0)
    assert fa.time()["steps"] == fb.time()["steps"]
    for k in range(3):
        assert np.array_equal(assemble(fa, k), assemble(fb, k))


# ------------------------------------------------------ forest geometry --

def test_effective_resolution_golden():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "effective_resolution.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        mi, mj, mx, Lx, Ly, lev, nx, ny = map(int, r[:8])
        dxp = float(r[8])
        cfg = inputs.Config(mi=mi, mj=mj, mx=mx, minlevel=lev, maxlevel=lev,
                            xupper=Lx, yupper=Ly)
        f = oracle.OracleForest(cfg)
        L, X, Y = f.patch_info()
        assert (X.max() + 1) * mx == nx and (Y.max() + 1) * mx == ny
        dx = Lx / nx
        assert round(dx, 1 if dxp < 1 else 1) == pytest.approx(dxp, abs=0.05)


# ------------------------------------------------------------- topography --

def test_dem_average_exact_for_bilinear_surface():
    """The cell average of the DEM interpolant is exact when the DEM samples a
    bilinear function: the mean of a + bx + cy + dxy over a rectangle is its
    value at the centre.  Rectangles straddle many DEM cells."""
    a, bb, c, d = 1.5, 0.02, -0.03, 1e-4
    x = np.linspace(0, 100, 51)
    y = np.linspace(0, 60, 31)
    X, Y = np.meshgrid(x, y)
    dem = inputs.Dem(a + bb * X + c * Y + d * X * Y, 0.0, 0.0, 2.0, 2.0)
    rng = np.random.default_rng(4)
    for _ in range(200):
        xa, xb = np.sort(rng.uniform(0, 100, 2))
        ya, yb = np.sort(rng.uniform(0, 60, 2))
        if xb - xa < 1e-3 or yb - ya < 1e-3:
            continue
        xm, ym = 0.5 * (xa + xb), 0.5 * (ya + yb)
        assert oracle.dem_average(dem, xa, xb, ya, yb) == pytest.approx(
            a + bb * xm + c * ym + d * xm * ym, rel=1e-12)


def test_dem_average_outside_extent_is_constant_extension():
    rng = np.random.default_rng(5)
    z = rng.uniform(0, 1, (5, 6))
    dem = inputs.Dem(z, 10.0, 20.0, 1.0, 1.0)
    # rectangle half outside on the left: brute-force midpoint sum
    xa, xb, ya, yb = 8.0, 12.0, 20.5, 22.5
    n = 400
    xs = xa + (np.arange(n) + 0.5) * (xb - xa) / n
    ys = ya + (np.arange(n) + 0.5) * (yb - ya) / n
    XX, YY = np.meshgrid(np.clip(xs, 10, 15), np.clip(ys, 20, 24))
    from scipy.interpolate import RegularGridInterpolator
    f = RegularGridInterpolator((20 + np.arange(5), 10 + np.arange(6)), z)
    ref = f(np.stack([YY.ravel(), XX.ravel()], 1)).mean()
    assert oracle.dem_average(dem, xa, xb, ya, yb) == pytest.approx(ref, rel=1e-5)


def test_coarse_bed_is_mean_of_fine_beds():
    """Cell averages are conservative across levels: a coarse cell's bed is the
    mean of its four children's beds up to round-off (Sec. 6.2)."""
    prob = inputs.radial_dambreak(64, 32, dx=8.0)
    coarse = oracle.OracleForest(prob.cfg, prob.dem)
    cfg2 = inputs.Config(**{**prob.cfg.__dict__, "minlevel": 1, "maxlevel": 1})
    fine = oracle.OracleForest(cfg2, prob.dem)
    bc = assemble(coarse, 3)
    bf = assemble(fine, 3)
    mean = 0.25 * (bf[0::2, 0::2] + bf[1::2, 0::2] + bf[0::2, 1::2] + bf[1::2, 1::2])
    assert np.abs(bc - mean).max() <= 1e-12 * (1 + np.abs(bc).max())
