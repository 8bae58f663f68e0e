"""Seeded synthetic workloads (problem set-up only, no solver arithmetic).

Shared by the tests, the benchmark and the oracle harness: every function here
builds a problem description -- a configuration, a DEM grid, an initial
condition and gauge points -- from a 64-bit seed.  Nothing here evaluates the
wave-propagation method; both the CUDA library and the CPU oracle receive the
same arrays.

The workloads stand in for the paper's test cases (Sec. 5, Sec. 6), whose
datasets (UK Environment Agency benchmarks, the CADAM Malpasset DEM) are not
available: the shapes, sizes, depths, Manning coefficients and CFL numbers
follow the paper and the benchmark configuration list; the terrain is synthetic.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

BC_WALL = 0
BC_EXTRAP = 1

SEED_BASE = 20240322


@dataclasses.dataclass
class Config:
    """Forest, physics and control parameters (Sec. 4, Sec. 5.1, Sec. 6.6)."""

    mi: int = 1
    mj: int = 1
    mx: int = 32
    minlevel: int = 0
    maxlevel: int = 0
    bc: Tuple[int, int, int, int] = (BC_WALL, BC_WALL, BC_WALL, BC_WALL)
    xlower: float = 0.0
    xupper: float = 1.0
    ylower: float = 0.0
    yupper: float = 1.0
    g: float = 9.81
    drytol: float = 1e-3
    manning_n: float = 0.0
    cfl_desired: float = 0.9
    cfl_max: float = 1.0
    dt_initial: float = 1e-2
    dt_max: float = math.inf
    tag_depth: float = 1e-3
    tag_speed: float = 0.01
    tag_deta: float = 0.05
    eta0: float = 0.0
    src_box: Tuple[float, float, float, float] = (0.0, -1.0, 0.0, -1.0)
    src_level: int = 0
    regrid_interval: int = 0
    precision: int = 0  # 0 = FP64, 1 = FP32 surface-deviation form
    # criterion 2 (velocity-depth product) threshold on |hu| in m^2/s
    tag_flux: float = math.inf
    # criterion 5 (flow grades): up to 4 (kind, value, level), kind 0 = depth,
    # 1 = speed; a wet cell above value asks for at least that level
    grades: Tuple[Tuple[int, float, int], ...] = ()
    # scheme variants of Sec. 3.2 (all 0: second order, unsplit, with
    # transverse propagation)
    first_order: int = 0
    no_transverse: int = 0
    dim_split: int = 0
    # inflow hydrograph (Sec. 5.1): up to 16 (t, Q) points, Q the discharge
    # in m^3/s through the segment [inflow_lo, inflow_hi] of side
    # inflow_side (0 left, 1 right, 2 bottom, 3 top); () = no inflow;
    # inflow_tau is the minimum interior depth of the boundary rule
    # level subcycling: level L takes 2^(L - minlevel) steps per macro step
    subcycle: int = 0
    hydrograph: Tuple[Tuple[float, float], ...] = ()
    inflow_side: int = 0
    inflow_lo: float = 0.0
    inflow_hi: float = 0.0
    inflow_tau: float = 1e-4
    # refinement regions (Sec. 4.1 criterion 4, Sec. 6.4): up to 8
    # (x0, x1, y0, y1, t0, t1, minlevel, maxlevel); while t0 <= t <= t1 a
    # cell whose centre lies in the box asks for a level in
    # [minlevel, maxlevel] (overlaps: the largest of each)
    regions: Tuple[Tuple[float, float, float, float, float, float, int, int], ...] = ()


@dataclasses.dataclass
class Dem:
    z: np.ndarray  # [ny][nx] nodal elevations
    x0: float
    y0: float
    dx: float
    dy: float


# An initial condition maps cell centres and cell-averaged beds to h, hu, hv.
InitialCondition = Callable[[np.ndarray, np.ndarray, np.ndarray],
                            Tuple[np.ndarray, np.ndarray, np.ndarray]]


@dataclasses.dataclass
class Problem:
    name: str
    cfg: Config
    dem: Optional[Dem]
    ic: InitialCondition
    t_end: float
    gauges: Optional[np.ndarray] = None  # [n][2]


# --------------------------------------------------------------------------
# terrain generators
# --------------------------------------------------------------------------

def flat_dem(cfg: Config, value: float = 0.0) -> Dem:
    z = np.full((2, 2), value, dtype=np.float64)
    return Dem(z, cfg.xlower, cfg.ylower, cfg.xupper - cfg.xlower,
               cfg.yupper - cfg.ylower)


def node_grid(cfg: Config, spacing: float):
    nx = int(round((cfg.xupper - cfg.xlower) / spacing)) + 1
    ny = int(round((cfg.yupper - cfg.ylower) / spacing)) + 1
    x = cfg.xlower + spacing * np.arange(nx)
    y = cfg.ylower + spacing * np.arange(ny)
    return np.meshgrid(x, y)


def gaussian_sum_dem(cfg: Config, n: int, seed: int, spacing: float,
                     amp=(0.0, 3.0), width=(20.0, 200.0)) -> Dem:
    """Sum of n Gaussian mounds, amplitudes U[amp], widths U[width], centres
    uniform over the domain."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(amp[0], amp[1], n)
    W = rng.uniform(width[0], width[1], n)
    cx = rng.uniform(cfg.xlower, cfg.xupper, n)
    cy = rng.uniform(cfg.ylower, cfg.yupper, n)
    X, Y = node_grid(cfg, spacing)
    z = np.zeros_like(X)
    for k in range(n):
        z += A[k] * np.exp(-((X - cx[k]) ** 2 + (Y - cy[k]) ** 2) / (2 * W[k] ** 2))
    return Dem(z, cfg.xlower, cfg.ylower, spacing, spacing)


def value_noise(X: np.ndarray, Y: np.ndarray, seed: int, octaves: int,
                base_wavelength: float) -> np.ndarray:
    """Fractal value noise: octaves of bilinearly interpolated seeded lattice
    values, halving the wavelength and the amplitude each octave; normalised to
    unit peak amplitude."""
    rng = np.random.default_rng(seed)
    out = np.zeros_like(X)
    amp = 1.0
    wl = base_wavelength
    x0, y0 = X.min(), Y.min()
    for _ in range(octaves):
        gx = int(math.ceil((X.max() - x0) / wl)) + 2
        gy = int(math.ceil((Y.max() - y0) / wl)) + 2
        lat = rng.uniform(-1.0, 1.0, (gy, gx))
        fx = (X - x0) / wl
        fy = (Y - y0) / wl
        i = np.floor(fx).astype(int)
        j = np.floor(fy).astype(int)
        ax = fx - i
        ay = fy - j
        v = ((1 - ay) * ((1 - ax) * lat[j, i] + ax * lat[j, i + 1]) +
             ay * ((1 - ax) * lat[j + 1, i] + ax * lat[j + 1, i + 1]))
        out += amp * v
        amp *= 0.5
        wl *= 0.5
    peak = np.abs(out).max()
    return out / peak if peak > 0 else out


def nested_dems(cfg: Config, seed: int, boxes, spacings,
                relief: float = 3.0) -> List[Dem]:
    """Overlapping DEMs of one seeded terrain at several resolutions (Sec.
    6.2: 2, 5 and 20 m DEMs over parts of the Malpasset domain): DEM k
    samples, at spacing spacings[k] over boxes[k] (x0, x1, y0, y1; None =
    the whole domain; widened outward to whole spacings), a valley across y
    with a slope along x plus octaves of value noise anchored to the domain
    (wavelengths 256 m, 128 m, ...) down to four node spacings of that DEM.
    Finer DEMs therefore carry detail the coarser ones leave out."""
    W = cfg.yupper - cfg.ylower
    lat = []

    def noise(X, Y, octaves):
        out = np.zeros_like(X)
        for o in range(octaves):
            wl = 256.0 / 2 ** o
            gx = int(math.ceil((cfg.xupper - cfg.xlower) / wl)) + 3
            gy = int(math.ceil((cfg.yupper - cfg.ylower) / wl)) + 3
            while len(lat) <= o:
                lat.append(np.random.default_rng([seed, len(lat)]).uniform(-1.0, 1.0, (gy, gx)))
            fx = (X - cfg.xlower) / wl + 1.0
            fy = (Y - cfg.ylower) / wl + 1.0
            i = np.clip(np.floor(fx).astype(int), 0, gx - 2)
            j = np.clip(np.floor(fy).astype(int), 0, gy - 2)
            ax, ay = fx - i, fy - j
            L = lat[o]
            out += 0.5 ** o * ((1 - ay) * ((1 - ax) * L[j, i] + ax * L[j, i + 1]) +
                               ay * ((1 - ax) * L[j + 1, i] + ax * L[j + 1, i + 1]))
        return out

    dems = []
    for box, sp in zip(boxes, spacings):
        if box is None:
            box = (cfg.xlower, cfg.xupper, cfg.ylower, cfg.yupper)
        x0 = math.floor(box[0] / sp) * sp
        y0 = math.floor(box[2] / sp) * sp
        nx = int(math.ceil((box[1] - x0) / sp)) + 1
        ny = int(math.ceil((box[3] - y0) / sp)) + 1
        X, Y = np.meshgrid(x0 + sp * np.arange(nx), y0 + sp * np.arange(ny))
        base = 0.02 * (X - cfg.xlower) + relief * ((Y - cfg.ylower - 0.5 * W) / (0.5 * W)) ** 2
        octaves = max(1, int(math.floor(math.log2(256.0 / (4.0 * sp)))) + 1)
        dems.append(Dem(base + 0.5 * noise(X, Y, octaves), x0, y0, sp, sp))
    return dems


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def stoker(nx: int = 128, patch: Optional[int] = None) -> Problem:
    """1D-in-2D wet-wet dam break on a flat bed (Stoker closed form):
    128x128 at dx = 5 m, h = 2 m for x < 320 m and 0.5 m elsewhere, walls,
    CFL 0.9, t = 20 s, n = 0.  With patch=None one patch spans the grid."""
    dx = 640.0 / nx
    m = patch or nx
    cfg = Config(mi=nx // m, mj=nx // m, mx=m, xupper=640.0, yupper=640.0,
                 drytol=1e-3, manning_n=0.0, dt_initial=0.5 * dx / 5.0)

    def ic(x, y, b):
        h = np.where(x < 320.0, 2.0, 0.5)
        return h, np.zeros_like(h), np.zeros_like(h)

    return Problem("stoker", cfg, flat_dem(cfg), ic, 20.0)


def lake_at_rest(nx: int = 128, patch: Optional[int] = None, eta: float = 1.0,
                 amp: float = 0.5, sigma: float = 50.0) -> Problem:
    """Still water at surface eta over a Gaussian bump of amplitude amp and
    width sigma centred in the 640 m square; eta = 0.3 emerges the bump."""
    m = patch or nx
    cfg = Config(mi=nx // m, mj=nx // m, mx=m, xupper=640.0, yupper=640.0,
                 drytol=1e-3, manning_n=0.0, dt_initial=0.5)
    X, Y = node_grid(cfg, 640.0 / nx / 2)
    z = amp * np.exp(-((X - 320.0) ** 2 + (Y - 320.0) ** 2) / (2 * sigma ** 2))
    dem = Dem(z, 0.0, 0.0, 640.0 / nx / 2, 640.0 / nx / 2)

    def ic(x, y, b):
        h = np.maximum(eta - b, 0.0)
        return h, np.zeros_like(h), np.zeros_like(h)

    return Problem("lake_at_rest", cfg, dem, ic, 0.0)


def radial_dambreak(n: int = 1024, patch: int = 32, dx: float = 2.0,
                    radius: float = 200.0, depth: float = 5.0,
                    flat: bool = False, seed: int = SEED_BASE + 1,
                    manning_n: float = 0.033, drytol: float = 1e-3) -> Problem:
    """Radial dam break onto a dry bed over seeded smooth terrain: n x n cells
    of dx metres in patch x patch patches, 40 Gaussians (amplitudes U[0,3] m,
    widths U[20,200] m), cylinder of the given radius at the given depth,
    drytol 1e-3 m, Manning 0.033, t = 60 s."""
    L = n * dx
    cfg = Config(mi=n // patch, mj=n // patch, mx=patch, xupper=L, yupper=L,
                 drytol=drytol, manning_n=manning_n, dt_initial=0.1,
                 tag_depth=drytol)
    dem = flat_dem(cfg) if flat else gaussian_sum_dem(cfg, 40, seed, dx)
    c = 0.5 * L

    def ic(x, y, b):
        r2 = (x - c) ** 2 + (y - c) ** 2
        h = np.where(r2 < radius * radius, depth, 0.0)
        return h, np.zeros_like(h), np.zeros_like(h)

    return Problem("radial_dambreak", cfg, dem, ic, 60.0)


def v_valley(mi: int = 16, mj: int = 8, patch: int = 32, minlevel: int = 2,
             maxlevel: int = 4, seed: int = SEED_BASE + 2,
             dem_spacing: float = 2.0, depth: float = 20.0,
             breach_x: float = 500.0, manning_n: float = 0.033,
             n_gauges: int = 16, Lx: float = 4000.0, Ly: float = 2000.0,
             breach_width: Optional[float] = None) -> Problem:
    """Synthetic V-valley (4 km x 2 km): side slope 0.05, down-valley slope
    0.005, seeded fractal noise of 0.5 m amplitude; reservoir upstream of
    x = breach_x filled to `depth` above the thalweg at the breach, dry
    downstream, instantaneous full breach (or, with breach_width, a dam 5 m
    above the reservoir surface along x = breach_x with a breach of that
    width centred on the thalweg); n = 0.033; 16 seeded gauges along the
    thalweg and banks; regrid every 4 steps."""
    cfg = Config(mi=mi, mj=mj, mx=patch, minlevel=minlevel, maxlevel=maxlevel,
                 xupper=Lx, yupper=Ly, drytol=1e-4, manning_n=manning_n,
                 dt_initial=0.05, tag_depth=1e-4, tag_speed=0.01,
                 tag_deta=0.05, regrid_interval=4,
                 src_box=(0.0, breach_x, 0.0, Ly), src_level=maxlevel)
    X, Y = node_grid(cfg, dem_spacing)
    noise = value_noise(X, Y, seed, 6, 800.0)
    z = 0.05 * np.abs(Y - 0.5 * Ly) + 0.005 * (Lx - X) + 0.5 * noise
    surface = 0.005 * (Lx - breach_x) + depth
    if breach_width is not None:
        dam = (X >= breach_x) & (X < breach_x + 4 * dem_spacing) & \
            (np.abs(Y - 0.5 * Ly) >= 0.5 * breach_width)
        z = np.where(dam, np.maximum(z, surface + 5.0), z)
    dem = Dem(z, 0.0, 0.0, dem_spacing, dem_spacing)
    cfg.eta0 = surface

    def ic(x, y, b):
        h = np.where(x < breach_x, np.maximum(surface - b, 0.0), 0.0)
        return h, np.zeros_like(h), np.zeros_like(h)

    rng = np.random.default_rng(seed + 1000)
    gx = rng.uniform(breach_x + 100.0, Lx - 100.0, n_gauges)
    off = rng.choice([-1.0, 0.0, 1.0], n_gauges) * rng.uniform(0.0, 150.0, n_gauges)
    gauges = np.stack([gx, 0.5 * Ly + off], axis=1)
    return Problem("v_valley", cfg, dem, ic, 600.0, gauges)


def valley_2km(seed: int = SEED_BASE + 41, depth: float = 12.0,
               breach_x: float = 350.0, patch: int = 32,
               precision: int = 0) -> Problem:
    """A 2 km x 1 km V-valley (the 4 km x 2 km valley at half the size):
    4 x 2 blocks of 32 x 32 patches (8 x 4 of 16 x 16) on levels 0..3, so the
    finest cells are 1.95 m; reservoir at `depth` above the thalweg upstream
    of `breach_x`, refined to level 1 there; 8 gauges."""
    scale = 32 // patch
    prob = v_valley(mi=4 * scale, mj=2 * scale, patch=patch, minlevel=0, maxlevel=3,
                    seed=seed, dem_spacing=8.0, depth=depth, breach_x=breach_x,
                    n_gauges=8, Lx=2000.0, Ly=1000.0)
    prob.cfg.src_level = 1
    prob.cfg.precision = precision
    return prob


def inflow_channel(nx: int = 128, patch: int = 32, q: float = 2.0, h0: float = 1.0,
                   t_end: float = 30.0) -> Problem:
    """1D-in-2D bore from the inflow boundary (Sec. 5.1): a 640 m x 40 m
    channel at rest at depth h0 over a flat bed, the whole left side an
    inflow of unit discharge q (m^2/s), walls elsewhere, n = 0.  The exact
    solution is a bore of the Eq. 2-shock state moving right."""
    dx = 640.0 / nx
    m = patch
    rows = max(m, int(round(40.0 / dx)) // m * m)
    cfg = Config(mi=nx // m, mj=rows // m, mx=m, xupper=640.0, yupper=rows * dx,
                 drytol=1e-4, manning_n=0.0, dt_initial=0.2 * dx / 5.0,
                 hydrograph=((0.0, q * rows * dx),), inflow_side=0,
                 inflow_lo=0.0, inflow_hi=rows * dx, inflow_tau=1e-4)

    def ic(x, y, b):
        h = np.full_like(x, h0)
        return h, np.zeros_like(h), np.zeros_like(h)

    return Problem("inflow_channel", cfg, flat_dem(cfg), ic, t_end)


def flood_speed(patch: int = 32, minlevel: int = 0, maxlevel: int = 3,
                precision: int = 0, peak: float = 20.0, t_end: float = 21600.0) -> Problem:
    """Synthetic stand-in for Test Case 1 (Sec. 5.1, flood propagation over
    an extended floodplain): a flat, dry 1000 m x 2000 m plain, an inflow of
    Q(t) through 20 m of the left side at its midline (990 <= y <= 1010):
    Q rises linearly to `peak` m^3/s in 60 min, holds for 180 min and falls
    to zero in the next 60 min; walls elsewhere, tau = drytol = 1e-4 m,
    CFL 0.9, Manning n = 0.03, 6 h.  Blocks of 1000 m (1 x 2) with patches
    of `patch` cells on levels minlevel..maxlevel (level 3 with 32-cell
    patches: 3.9 m cells, the paper's 5 m being no power-of-two division of
    the domain); refinement follows the wet region (tag_depth = tau) and the
    inflow segment (source box, refined to maxlevel)."""
    cfg = Config(mi=1, mj=2, mx=patch, minlevel=minlevel, maxlevel=maxlevel,
                 xupper=1000.0, yupper=2000.0, drytol=1e-4, manning_n=0.03,
                 dt_initial=1.0, tag_depth=1e-4, tag_speed=1e9, tag_deta=1e9,
                 src_box=(0.0, 100.0, 900.0, 1100.0), src_level=maxlevel,
                 precision=precision,
                 hydrograph=((0.0, 0.0), (3600.0, peak), (14400.0, peak), (18000.0, 0.0)),
                 inflow_side=0, inflow_lo=990.0, inflow_hi=1010.0, inflow_tau=1e-4)

    def ic(x, y, b):
        z = np.zeros_like(x)
        return z, z.copy(), z.copy()

    return Problem("flood_speed", cfg, flat_dem(cfg), ic, t_end)


def canyon_plain(patch: int = 32, minlevel: int = 0, maxlevel: int = 4,
                 seed: int = SEED_BASE + 7, dem_spacing: float = 10.0,
                 depth: float = 55.0, precision: int = 1, near_gauges: int = 0) -> Problem:
    """Large AMR workload (the Malpasset set-up's shape, Sec. 6.2-6.4): a
    17 km x 9 km domain of 1 km blocks; for x < 10 km a canyon -- fractal
    terrain 60-120 m high cut 50 m deep by a meandering channel (centre line
    a seeded sinusoid of 800 m amplitude and 3 km wavelength, width varying
    between 100 and 300 m) falling 0.004 per metre seawards -- then a
    coastal plain at slope 0.002 down to the sea at x = 17 km; a reservoir
    in the channel upstream of x = 2 km filled `depth` m above its bed,
    instantaneous dam break, dry downstream, n = 0.033.  Levels
    minlevel..maxlevel (5 levels: 31.25 m to 1.95 m cells with 32-cell
    patches); refinement to maxlevel where water flows and over the
    reservoir (source box).  Gauges: 16 on the channel's centre line from
    x = 2.5 km to 16 km, then near_gauges more on it from x = 2050 m to
    2800 m (reached in the flood's first seconds)."""
    Lx, Ly = 17000.0, 9000.0
    cfg = Config(mi=17, mj=9, mx=patch, minlevel=minlevel, maxlevel=maxlevel,
                 xupper=Lx, yupper=Ly, drytol=1e-3, manning_n=0.033, dt_initial=0.05,
                 tag_depth=1e-3, tag_speed=0.1, tag_deta=1e9, precision=precision,
                 src_box=(0.0, 2000.0, 0.0, Ly), src_level=maxlevel)
    rng = np.random.default_rng(seed)
    phase = rng.uniform(0.0, 2 * np.pi)
    wphase = rng.uniform(0.0, 2 * np.pi)
    X, Y = node_grid(cfg, dem_spacing)
    centre = 0.5 * Ly + 800.0 * np.sin(2 * np.pi * X / 3000.0 + phase)
    width = 200.0 + 100.0 * np.sin(2 * np.pi * X / 4100.0 + wphase)
    noise = value_noise(X, Y, seed, 6, 2000.0)
    canyon = 90.0 + 30.0 * noise + 0.004 * (10000.0 - X)
    d = np.abs(Y - centre)
    cut = np.clip(1.0 - (d - 0.5 * width) / 150.0, 0.0, 1.0)  # channel banks
    canyon = canyon - 50.0 * cut
    plain = 0.002 * (Lx - X) + 0.5 * noise
    blend = np.clip((X - 9500.0) / 1000.0, 0.0, 1.0)  # canyon mouth
    z = (1.0 - blend) * canyon + blend * plain
    dem = Dem(z, 0.0, 0.0, dem_spacing, dem_spacing)
    i_dam = int(round(2000.0 / dem_spacing))
    j_c = np.argmin(np.abs(Y[:, i_dam] - centre[:, i_dam]))
    surface = float(z[j_c, i_dam]) + depth
    cfg.eta0 = 0.0

    def ic(x, y, b):
        h = np.where(x < 2000.0, np.maximum(surface - b, 0.0), 0.0)
        return h, np.zeros_like(h), np.zeros_like(h)

    gx = np.linspace(2500.0, 16000.0, 16)
    if near_gauges:
        gx = np.concatenate([gx, np.linspace(2050.0, 2800.0, near_gauges)])
    gy = 0.5 * Ly + 800.0 * np.sin(2 * np.pi * gx / 3000.0 + phase)
    return Problem("canyon_plain", cfg, dem, ic, 4000.0, np.stack([gx, gy], 1))


def valley_ensemble(n: int, seed: int = SEED_BASE + 4, precision: int = 1):
    """n scenarios of the 2 km x 1 km valley for one batched context:
    breach width U[50, 400] m, reservoir depth U[10, 30] m, Manning n
    U[0.02, 0.05], terrain noise seeded per scenario; one forest
    configuration (from the first scenario).  Returns the problems."""
    rng = np.random.default_rng(seed)
    probs = []
    for k in range(n):
        prob = v_valley(mi=4, mj=2, patch=32, minlevel=0, maxlevel=3,
                        seed=seed + 100 + k, dem_spacing=8.0,
                        depth=float(rng.uniform(10.0, 30.0)), breach_x=350.0,
                        manning_n=float(rng.uniform(0.02, 0.05)), n_gauges=8,
                        Lx=2000.0, Ly=1000.0,
                        breach_width=float(rng.uniform(50.0, 400.0)))
        prob.cfg.src_level = 1
        prob.cfg.precision = precision
        probs.append(prob)
    return probs


def valley_ensemble_full(n: int, seed: int = SEED_BASE + 5, precision: int = 1):
    """n scenarios of the full 4 km x 2 km valley (16 x 8 blocks of 32 x 32
    patches, levels 2-4, 2048 patches before any refinement): breach width
    U[50, 400] m, reservoir depth U[10, 30] m, Manning n U[0.02, 0.05],
    terrain noise seeded per scenario (DEM nodes every 8 m)."""
    rng = np.random.default_rng(seed)
    probs = []
    for k in range(n):
        prob = v_valley(seed=seed + 100 + k, dem_spacing=8.0,
                        depth=float(rng.uniform(10.0, 30.0)),
                        manning_n=float(rng.uniform(0.02, 0.05)), n_gauges=16,
                        breach_width=float(rng.uniform(50.0, 400.0)))
        prob.cfg.precision = precision
        probs.append(prob)
    return probs


def cnn_init(seed: int, nch: int = 16, taps: int = 9) -> np.ndarray:
    """Seeded initial parameters of the refinement predictor in its layout
    (three layers of W[nch][taps * nch] then b[nch], then wh[nch], bh):
    He-normal weights, zero biases, a small normal head."""
    rng = np.random.default_rng(seed)
    k = taps * nch
    parts = []
    for _ in range(3):
        parts += [rng.normal(0.0, math.sqrt(2.0 / k), nch * k), rng.normal(0.0, 0.05, nch)]
    parts += [rng.normal(0.0, 0.25, nch), np.array([-0.5])]
    return np.concatenate(parts).astype(np.float32)


def cell_centres(cfg: Config, levels: Sequence[int], pxs: Sequence[int],
                 pys: Sequence[int]):
    """Cell centres [npatch][mx][mx] of a patch list (row index j, column i)."""
    m = cfg.mx
    xs = np.empty((len(levels), m, m))
    ys = np.empty((len(levels), m, m))
    idx = np.arange(m)
    for k, (L, px, py) in enumerate(zip(levels, pxs, pys)):
        dx = (cfg.xupper - cfg.xlower) / (cfg.mi * m * (1 << L))
        dy = (cfg.yupper - cfg.ylower) / (cfg.mj * m * (1 << L))
        xc = cfg.xlower + (px * m + idx + 0.5) * dx
        yc = cfg.ylower + (py * m + idx + 0.5) * dy
        xs[k] = xc[None, :]
        ys[k] = yc[:, None]
    return xs, ys
