"""FP64 CPU oracle for the GeoFlood wave-propagation step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  It wraps ``liboracle.so``, built from
``geoflood_oracle.c`` with gcc (``-ffp-contract=off``), and shares no code with
the CUDA library.  The Python surface mirrors the product binding's
``Forest`` so one test harness drives both.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geoflood_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KEEP, REFINE, COARSEN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (plain gcc, no FMA)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd, cwd=_HERE)
    os.replace(tmp, _LIB)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [
        ("mi", C.c_int), ("mj", C.c_int), ("mx", C.c_int),
        ("minlevel", C.c_int), ("maxlevel", C.c_int), ("bc", C.c_int * 4),
        ("xlower", C.c_double), ("xupper", C.c_double),
        ("ylower", C.c_double), ("yupper", C.c_double),
        ("g", C.c_double), ("drytol", C.c_double), ("manning_n", C.c_double),
        ("cfl_desired", C.c_double), ("cfl_max", C.c_double),
        ("dt_initial", C.c_double), ("dt_max", C.c_double),
        ("tag_depth", C.c_double), ("tag_speed", C.c_double),
        ("tag_deta", C.c_double), ("eta0", C.c_double),
        ("src_box", C.c_double * 4), ("src_level", C.c_int),
        ("tag_flux", C.c_double), ("ngrades", C.c_int),
        ("grade_kind", C.c_int * 4), ("grade_value", C.c_double * 4),
        ("grade_level", C.c_int * 4),
        ("first_order", C.c_int), ("no_transverse", C.c_int), ("dim_split", C.c_int),
        ("subcycle", C.c_int), ("n_hydro", C.c_int), ("inflow_side", C.c_int),
        ("inflow_lo", C.c_double), ("inflow_hi", C.c_double), ("inflow_tau", C.c_double),
        ("hydro_t", C.c_double * 16), ("hydro_q", C.c_double * 16),
        ("nregions", C.c_int), ("region_minlevel", C.c_int * 8),
        ("region_maxlevel", C.c_int * 8),
        ("region_x0", C.c_double * 8), ("region_x1", C.c_double * 8),
        ("region_y0", C.c_double * 8), ("region_y1", C.c_double * 8),
        ("region_t0", C.c_double * 8), ("region_t1", C.c_double * 8),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            vp = C.c_void_p
            L.oracle_riemann.argtypes = [C.c_double] * 10 + [dp, dp]
            L.oracle_step_grid.argtypes = ([C.c_int, C.c_int] + [dp] * 4 +
                                           [C.c_double] * 6 + [dp] * 4 +
                                           [C.POINTER(C.c_long), dp])
            L.oracle_step_grid_ex.argtypes = ([C.c_int, C.c_int] + [dp] * 4 +
                                              [C.c_double] * 6 + [C.c_int] * 3 +
                                              [dp] * 4 + [C.POINTER(C.c_long), dp])
            L.oracle_hydrograph.restype = C.c_double
            L.oracle_hydrograph.argtypes = [C.POINTER(_Cfg), C.c_double]
            L.oracle_inflow_depth.restype = C.c_double
            L.oracle_inflow_depth.argtypes = [C.c_double] * 5 + [dp, dp]
            L.oracle_dems_average.restype = C.c_double
            L.oracle_dems_average.argtypes = ([C.c_int, C.POINTER(dp), ip, ip] + [dp] * 4 +
                                              [C.c_double] * 4)
            L.oracle_forest_set_topos.argtypes = [vp, C.c_int, C.POINTER(dp), ip, ip] + [dp] * 4
            L.oracle_dem_average.restype = C.c_double
            L.oracle_dem_average.argtypes = [dp, C.c_int, C.c_int] + [C.c_double] * 8
            L.oracle_forest_new.restype = vp
            L.oracle_forest_new.argtypes = [C.POINTER(_Cfg)]
            L.oracle_forest_free.argtypes = [vp]
            L.oracle_forest_set_topo.argtypes = [vp, dp, C.c_int, C.c_int] + [C.c_double] * 4
            L.oracle_forest_npatch.argtypes = [vp]
            L.oracle_forest_patch_info.argtypes = [vp, ip, ip, ip]
            L.oracle_forest_write.argtypes = [vp, dp, dp, dp]
            L.oracle_forest_read.argtypes = [vp, dp, dp, dp, dp]
            L.oracle_forest_read_tiles.argtypes = [vp, dp]
            L.oracle_forest_set_time.argtypes = [vp, C.c_double, C.c_double]
            lp = C.POINTER(C.c_long)
            L.oracle_forest_get_time.argtypes = [vp, dp, dp, lp, lp, lp, dp]
            L.oracle_forest_step.argtypes = [vp, C.c_double, C.c_int, dp, ip]
            L.oracle_forest_tags.argtypes = [vp, C.POINTER(C.c_uint8)]
            L.oracle_forest_regrid.argtypes = [vp]
            L.oracle_forest_regrid_flags.argtypes = [vp, C.POINTER(C.c_uint8)]
            L.oracle_forest_mass.restype = C.c_double
            L.oracle_forest_mass.argtypes = [vp]
            L.oracle_forest_set_gauges.argtypes = [vp, dp, C.c_int]
            L.oracle_forest_gauges.argtypes = [vp, dp, dp]
            L.oracle_forest_ghost_fill.argtypes = [vp]
            _lib = L
    return _lib


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def riemann(hL, nL, tL, bL, hR, nR, tR, bR, g=9.81, drytol=1e-3):
    """Augmented Riemann solve at one edge: returns (Z[3][3], s[3])."""
    Z = np.zeros(9)
    s = np.zeros(3)
    lib().oracle_riemann(hL, nL, tL, bL, hR, nR, tR, bR, g, drytol, _p(Z), _p(s))
    return Z.reshape(3, 3), s


def hydrograph(cfg, t):
    """Discharge Q(t) of the configuration's inflow hydrograph (m^3/s)."""
    c = _cfg_struct(cfg)
    return lib().oracle_hydrograph(C.byref(c), float(t))


def inflow_depth(q, h_int, qn_int, g=9.81, tau=1e-4):
    """Ghost depth of the inflow boundary (Sec. 5.1, Eq. riemann / Eq.
    2-shock) and the interior depth and speed the equations used."""
    hu = C.c_double()
    uu = C.c_double()
    h = lib().oracle_inflow_depth(q, h_int, qn_int, g, tau, C.byref(hu), C.byref(uu))
    return h, hu.value, uu.value


def _dem_arrays(dems):
    zs = [np.ascontiguousarray(d.z, dtype=np.float64) for d in dems]
    n = len(zs)
    zp = (C.POINTER(C.c_double) * n)(*[_p(z) for z in zs])
    ints = lambda v: (C.c_int * n)(*v)
    dbl = lambda v: (C.c_double * n)(*v)
    return (zs, n, zp, ints([z.shape[1] for z in zs]), ints([z.shape[0] for z in zs]),
            dbl([d.x0 for d in dems]), dbl([d.y0 for d in dems]),
            dbl([d.dx for d in dems]), dbl([d.dy for d in dems]))


def dems_average(dems, xa, xb, ya, yb):
    """Cell average of the composite interpolant of several DEMs (Sec. 6.2)."""
    zs, n, zp, nx, ny, x0, y0, dx, dy = _dem_arrays(dems)
    return lib().oracle_dems_average(n, zp, nx, ny, x0, y0, dx, dy, xa, xb, ya, yb)


def dem_average(dem, xa, xb, ya, yb):
    z = np.ascontiguousarray(dem.z, dtype=np.float64)
    ny, nx = z.shape
    return lib().oracle_dem_average(_p(z), nx, ny, dem.x0, dem.y0, dem.dx,
                                    dem.dy, xa, xb, ya, yb)


def step_grid(h, hu, hv, b, dx, dy, dt, g=9.81, drytol=1e-3, manning_n=0.0,
              order=2, transverse=True, dim_split=False):
    """One step on a single [ny+4][nx+4] grid with filled ghosts (Sec. 3.2;
    order 1 drops the limited corrections, transverse=False the transverse
    terms, dim_split=True takes an x sweep, then a y sweep on its result).
    Cells outside the interior are returned as given."""
    H, W = h.shape
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (h, hu, hv, b)]
    out = [np.empty_like(arrs[0]) for _ in range(3)]
    cm = C.c_double()
    nc = C.c_long()
    cd = C.c_double()
    lib().oracle_step_grid_ex(W - 4, H - 4, *[_p(a) for a in arrs], dx, dy, dt, g,
                              drytol, manning_n, int(order), int(bool(transverse)),
                              int(bool(dim_split)), *[_p(a) for a in out],
                              C.byref(cm), C.byref(nc), C.byref(cd))
    return out[0], out[1], out[2], cm.value, nc.value


def _cfg_struct(cfg) -> _Cfg:
    c = _Cfg()
    for name in ("mi", "mj", "mx", "minlevel", "maxlevel", "src_level"):
        setattr(c, name, int(getattr(cfg, name)))
    for name in ("xlower", "xupper", "ylower", "yupper", "g", "drytol",
                 "manning_n", "cfl_desired", "cfl_max", "dt_initial", "dt_max",
                 "tag_depth", "tag_speed", "tag_deta", "eta0"):
        setattr(c, name, float(getattr(cfg, name)))
    for k in range(4):
        c.bc[k] = int(cfg.bc[k])
        c.src_box[k] = float(cfg.src_box[k])
    c.tag_flux = float(getattr(cfg, "tag_flux", float("inf")))
    grades = list(getattr(cfg, "grades", ()))
    assert len(grades) <= 4
    c.ngrades = len(grades)
    for k, (kind, value, level) in enumerate(grades):
        c.grade_kind[k] = int(kind)
        c.grade_value[k] = float(value)
        c.grade_level[k] = int(level)
    c.first_order = int(cfg.first_order)
    c.no_transverse = int(cfg.no_transverse)
    c.dim_split = int(cfg.dim_split)
    c.subcycle = int(cfg.subcycle)
    hyd = list(cfg.hydrograph)
    assert len(hyd) <= 16
    c.n_hydro = len(hyd)
    for k, (t, q) in enumerate(hyd):
        c.hydro_t[k] = float(t)
        c.hydro_q[k] = float(q)
    c.inflow_side = int(cfg.inflow_side)
    c.inflow_lo = float(cfg.inflow_lo)
    c.inflow_hi = float(cfg.inflow_hi)
    c.inflow_tau = float(cfg.inflow_tau)
    regions = list(getattr(cfg, "regions", ()))
    assert len(regions) <= 8
    c.nregions = len(regions)
    for k, (x0, x1, y0, y1, t0, t1, lmin, lmax) in enumerate(regions):
        c.region_x0[k], c.region_x1[k] = float(x0), float(x1)
        c.region_y0[k], c.region_y1[k] = float(y0), float(y1)
        c.region_t0[k], c.region_t1[k] = float(t0), float(t1)
        c.region_minlevel[k], c.region_maxlevel[k] = int(lmin), int(lmax)
    return c


class OracleForest:
    """Quadtree forest of patches advanced by the oracle."""

    def __init__(self, cfg, dem=None):
        self._h = None
        self.cfg = cfg
        self._c = _cfg_struct(cfg)
        self._h = lib().oracle_forest_new(C.byref(self._c))
        if not self._h:
            raise ValueError("oracle: bad configuration")
        if dem is not None:
            self.set_topo(dem)

    def close(self):
        if self._h:
            lib().oracle_forest_free(self._h)
            self._h = None

    __del__ = close

    def set_topo(self, dem):
        if isinstance(dem, (list, tuple)):
            zs, n, zp, nx, ny, x0, y0, dx, dy = _dem_arrays(dem)
            rc = lib().oracle_forest_set_topos(self._h, n, zp, nx, ny, x0, y0, dx, dy)
            assert rc == 0
            return
        z = np.ascontiguousarray(dem.z, dtype=np.float64)
        ny, nx = z.shape
        rc = lib().oracle_forest_set_topo(self._h, _p(z), nx, ny, dem.x0,
                                          dem.y0, dem.dx, dem.dy)
        if rc:
            raise ValueError("oracle: bad DEM")

    @property
    def npatch(self):
        return lib().oracle_forest_npatch(self._h)

    def patch_info(self):
        n = self.npatch
        L = np.empty(n, np.int32)
        X = np.empty(n, np.int32)
        Y = np.empty(n, np.int32)
        lib().oracle_forest_patch_info(self._h, _p(L, C.c_int), _p(X, C.c_int),
                                       _p(Y, C.c_int))
        return L, X, Y

    def write(self, h, hu, hv):
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (h, hu, hv)]
        lib().oracle_forest_write(self._h, *[_p(x) for x in a])

    def read(self):
        n, m = self.npatch, self.cfg.mx
        out = [np.empty((n, m, m)) for _ in range(4)]
        lib().oracle_forest_read(self._h, *[_p(x) for x in out])
        return tuple(out)

    def read_tiles(self):
        n, T = self.npatch, self.cfg.mx + 4
        out = np.empty((n, 4, T, T))
        lib().oracle_forest_read_tiles(self._h, _p(out))
        return out

    def set_state(self, ic):
        from paper_2403_15435_gb300.inputs import cell_centres
        L, X, Y = self.patch_info()
        xs, ys = cell_centres(self.cfg, L, X, Y)
        b = self.read()[3]
        h, hu, hv = ic(xs, ys, b)
        self.write(h, hu, hv)

    def set_time(self, t, dt_next):
        lib().oracle_forest_set_time(self._h, float(t), float(dt_next))

    def time(self):
        t, dt = C.c_double(), C.c_double()
        s, r, c = C.c_long(), C.c_long(), C.c_long()
        cv = C.c_double()
        lib().oracle_forest_get_time(self._h, C.byref(t), C.byref(dt),
                                     C.byref(s), C.byref(r), C.byref(c),
                                     C.byref(cv))
        return dict(t=t.value, dt_next=dt.value, steps=s.value,
                    rejects=r.value, nclip=c.value, clipvol=cv.value)

    def step(self, t_target, max_steps=1 << 30):
        t = C.c_double()
        n = C.c_int()
        rc = lib().oracle_forest_step(self._h, float(t_target), int(max_steps),
                                      C.byref(t), C.byref(n))
        if rc:
            raise RuntimeError("oracle: step failed (%d)" % rc)
        return t.value, n.value

    def tags(self):
        f = np.empty(self.npatch, np.uint8)
        lib().oracle_forest_tags(self._h, _p(f, C.c_uint8))
        return f

    def regrid(self):
        return lib().oracle_forest_regrid(self._h)

    def regrid_flags(self, flags):
        """Regrid from given per-leaf flags (0 keep, 1 refine, 2 coarsen)."""
        f = np.ascontiguousarray(flags, dtype=np.uint8)
        assert f.shape == (self.npatch,)
        return lib().oracle_forest_regrid_flags(self._h, _p(f, C.c_uint8))

    def mass(self):
        return lib().oracle_forest_mass(self._h)

    def set_gauges(self, xy):
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        self._ng = len(xy)
        lib().oracle_forest_set_gauges(self._h, _p(xy), len(xy))

    def gauges(self):
        out = np.empty((self._ng, 5))
        arr = np.empty(self._ng)
        lib().oracle_forest_gauges(self._h, _p(out), _p(arr))
        return out, arr

    def ghost_fill(self):
        lib().oracle_forest_ghost_fill(self._h)


def run_problem(prob, t_end=None, max_steps=1 << 30, regrid_interval=None):
    """Set up a Problem on the oracle and advance it; regrids every
    regrid_interval accepted steps when the forest has several levels."""
    f = OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    t_end = prob.t_end if t_end is None else t_end
    k = prob.cfg.regrid_interval if regrid_interval is None else regrid_interval
    if k and prob.cfg.maxlevel > prob.cfg.minlevel:
        done = 0
        while f.time()["t"] < t_end and done < max_steps:
            f.regrid()
            _, n = f.step(t_end, min(k, max_steps - done))
            done += n
    else:
        f.step(t_end, max_steps)
    return f
