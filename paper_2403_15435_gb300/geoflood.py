"""ctypes binding of libgeoflood.so (argument marshalling only).

Every computation runs in the CUDA library; this module converts numpy arrays
and Python values to the C ABI of ``include/geoflood.h`` and raises
:class:`GeoFloodError` on a non-zero status.  It refuses to work without the
built library: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgeoflood.so")
_lib = None
_lock = threading.Lock()

OK = 0
ERRORS = {
    -1: "ARG", -2: "CUDA", -3: "OOM", -4: "CFL", -5: "NAN",
    -6: "NEGATIVE_DEPTH", -7: "TIMEOUT", -8: "CAPACITY", -9: "STATE",
}
KEEP, REFINE, COARSEN = 0, 1, 2
TAGGER_PLAIN, TAGGER_LEARNED = 0, 1
CNN_IN_PIX, CNN_CH = 324, 16


class GeoFloodError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("geoflood error %d (%s): %s" % (code, ERRORS.get(code, "?"), msg))
        self.code = code


class _Cfg(C.Structure):
    _fields_ = [
        ("mi", C.c_int), ("mj", C.c_int), ("mx", C.c_int),
        ("minlevel", C.c_int), ("maxlevel", C.c_int), ("bc", C.c_int * 4),
        ("precision", C.c_int), ("num_scenarios", C.c_int),
        ("max_patches", C.c_int), ("max_gauges", C.c_int),
        ("xlower", C.c_double), ("xupper", C.c_double),
        ("ylower", C.c_double), ("yupper", C.c_double),
        ("g", C.c_double), ("drytol", C.c_double),
        ("cfl_desired", C.c_double), ("cfl_max", C.c_double),
        ("dt_initial", C.c_double), ("dt_max", C.c_double),
        ("tag_depth", C.c_double), ("tag_speed", C.c_double),
        ("tag_deta", C.c_double), ("src_box", C.c_double * 4),
        ("src_level", C.c_int), ("ngrades", C.c_int),
        ("tag_flux", C.c_double), ("grade_kind", C.c_int * 4),
        ("grade_value", C.c_double * 4), ("grade_level", C.c_int * 4),
        ("first_order", C.c_int), ("no_transverse", C.c_int), ("dim_split", C.c_int),
        ("n_hydro", C.c_int), ("inflow_side", C.c_int),
        ("inflow_lo", C.c_double), ("inflow_hi", C.c_double), ("inflow_tau", C.c_double),
        ("hydro_t", C.c_double * 16), ("hydro_q", C.c_double * 16),
        ("subcycle", C.c_int),
        ("nregions", C.c_int), ("region_minlevel", C.c_int * 8),
        ("region_maxlevel", C.c_int * 8),
        ("region_x0", C.c_double * 8), ("region_x1", C.c_double * 8),
        ("region_y0", C.c_double * 8), ("region_y1", C.c_double * 8),
        ("region_t0", C.c_double * 8), ("region_t1", C.c_double * 8),
    ]


class AdvanceStats(C.Structure):
    _fields_ = [(n, C.c_longlong) for n in ("steps", "patch_steps", "checks", "misses",
                                             "regrids", "miss_regrids", "samples")] + \
        [(n, C.c_double) for n in ("step_s", "check_s", "regrid_s", "regrid_host_s")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


QINIT = C.CFUNCTYPE(None, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                    C.POINTER(C.c_double), C.POINTER(C.c_double),
                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libgeoflood.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(
                    "libgeoflood.so is missing: run __graft_entry__.build() "
                    "(nvcc for sm_103a); there is no CPU fallback")
            L = C.CDLL(_LIB_PATH)
            vp, ip, dp = C.c_void_p, C.c_int, C.POINTER(C.c_double)
            pi = C.POINTER(C.c_int)
            ll = C.POINTER(C.c_longlong)
            fp = C.POINTER(C.c_float)
            u16p = C.POINTER(C.c_uint16)
            sig = {
                "geoflood_init_forest": [C.POINTER(_Cfg), vp, C.POINTER(vp)],
                "geoflood_set_scenario": [vp, ip, C.c_double, C.c_double],
                "geoflood_set_topo": [vp, ip, dp, ip, ip] + [C.c_double] * 4,
                "geoflood_set_topos": [vp, ip, ip, C.POINTER(dp), C.POINTER(ip), C.POINTER(ip)]
                                      + [dp] * 4,
                "geoflood_npatch": [vp, ip, pi],
                "geoflood_save": [vp, vp, C.c_size_t, C.POINTER(C.c_size_t)],
                "geoflood_gauge_count": [vp, ip, pi],
                "geoflood_check_bounded_wait": [vp],
                "geoflood_load": [vp, vp, C.c_size_t],
                "geoflood_patch_info": [vp, ip, pi, pi, pi],
                "geoflood_write_patches": [vp, ip, dp, dp, dp],
                "geoflood_read_patches": [vp, ip, dp, dp, dp, dp],
                "geoflood_read_tiles": [vp, ip, dp],
                "geoflood_set_state": [vp, ip, QINIT, vp],
                "geoflood_set_time": [vp, ip, C.c_double, C.c_double],
                "geoflood_get_time": [vp, ip, dp, dp, ll, ll, ll, dp],
                "geoflood_step": [vp, C.c_double, ip, dp, pi],
                "geoflood_tags": [vp, ip, C.POINTER(C.c_uint8)],
                "geoflood_regrid": [vp],
                "geoflood_mass": [vp, ip, dp],
                "geoflood_set_gauges": [vp, ip, dp, ip],
                "geoflood_gauges": [vp, ip, dp, dp],
                "geoflood_profile": [vp, ip],
                "geoflood_profile_read": [vp, C.c_char_p, dp, ll],
                "geoflood_profile_cells": [vp, C.c_char_p, ll],
                "geoflood_launch_count": [vp, ll],
                "geoflood_counters": [vp, ip, ll, ll],
                "geoflood_autotune": [vp, ip, pi, dp],
                "geoflood_set_variant": [vp, ip],
                "geoflood_cnn_set_params": [vp, fp, ip],
                "geoflood_cnn_get_params": [vp, fp, ip],
                "geoflood_cnn_set_scale": [vp, fp],
                "geoflood_cnn_features": [vp, ip, u16p],
                "geoflood_cnn_predict": [vp, ip, fp],
                "geoflood_cnn_grad": [vp, u16p, fp, ip, C.c_float, fp, fp, fp],
                "geoflood_cnn_dataset": [vp, ip],
                "geoflood_cnn_snapshot": [vp],
                "geoflood_check_tags": [vp, ip, pi],
                "geoflood_cnn_commit": [vp, pi, pi],
                "geoflood_cnn_dataset_read": [vp, ip, ip, u16p, fp],
                "geoflood_cnn_train": [vp, ip, ip, C.c_float, C.c_float, C.c_ulonglong, fp],
                "geoflood_set_tagger": [vp, ip, C.c_float],
                "geoflood_advance": [vp, C.c_double, ip, ip, ip, C.POINTER(AdvanceStats)],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.geoflood_destroy.argtypes = [vp]
            L.geoflood_destroy.restype = None
            L.geoflood_last_error.argtypes = [vp]
            L.geoflood_last_error.restype = C.c_char_p
            L.geoflood_cnn_nparam.argtypes = []
            L.geoflood_cnn_nparam.restype = C.c_int
            _lib = L
    return _lib


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def config_struct(cfg: inputs.Config, num_scenarios=1, max_patches=None,
                  max_gauges=64) -> _Cfg:
    c = _Cfg()
    for name in ("mi", "mj", "mx", "minlevel", "maxlevel", "src_level", "precision",
                 "first_order", "no_transverse", "dim_split"):
        setattr(c, name, int(getattr(cfg, name)))
    for name in ("xlower", "xupper", "ylower", "yupper", "g", "drytol",
                 "cfl_desired", "cfl_max", "dt_initial", "dt_max", "tag_depth",
                 "tag_speed", "tag_deta"):
        v = float(getattr(cfg, name))
        setattr(c, name, v if math.isfinite(v) else 1e300)
    for k in range(4):
        c.bc[k] = int(cfg.bc[k])
        c.src_box[k] = float(cfg.src_box[k])
    flux = float(getattr(cfg, "tag_flux", math.inf))
    c.tag_flux = flux if math.isfinite(flux) else 1e300
    grades = list(getattr(cfg, "grades", ()))
    c.ngrades = len(grades)
    for k, (kind, value, level) in enumerate(grades[:4]):
        c.grade_kind[k] = int(kind)
        c.grade_value[k] = float(value)
        c.grade_level[k] = int(level)
    hyd = list(getattr(cfg, "hydrograph", ()))
    if len(hyd) > 16:
        raise ValueError("at most 16 hydrograph points")
    c.n_hydro = len(hyd)
    for k, (t, q) in enumerate(hyd):
        c.hydro_t[k] = float(t)
        c.hydro_q[k] = float(q)
    c.inflow_side = int(getattr(cfg, "inflow_side", 0))
    c.inflow_lo = float(getattr(cfg, "inflow_lo", 0.0))
    c.inflow_hi = float(getattr(cfg, "inflow_hi", 0.0))
    c.inflow_tau = float(getattr(cfg, "inflow_tau", 1e-4))
    c.subcycle = int(getattr(cfg, "subcycle", 0))
    regions = list(getattr(cfg, "regions", ()))
    if len(regions) > 8:
        raise ValueError("at most 8 refinement regions")
    c.nregions = len(regions)
    for k, (x0, x1, y0, y1, t0, t1, lmin, lmax) in enumerate(regions):
        c.region_x0[k], c.region_x1[k] = float(x0), float(x1)
        c.region_y0[k], c.region_y1[k] = float(y0), float(y1)
        c.region_t0[k], c.region_t1[k] = float(t0), float(t1)
        c.region_minlevel[k], c.region_maxlevel[k] = int(lmin), int(lmax)
    c.num_scenarios = int(num_scenarios)
    if max_patches is None:
        per = cfg.mi * cfg.mj * (4 ** cfg.maxlevel)
        max_patches = num_scenarios * min(per, max(4096, cfg.mi * cfg.mj * 4 ** cfg.minlevel * 4))
    c.max_patches = int(max_patches)
    c.max_gauges = int(max_gauges)
    return c


class Forest:
    """One context: forests of num_scenarios scenarios on the GPU."""

    def __init__(self, cfg: inputs.Config, dem=None, num_scenarios=1,
                 max_patches=None, max_gauges=64, stream=None):
        self.cfg = cfg
        self.nscen = num_scenarios
        self._c = config_struct(cfg, num_scenarios, max_patches, max_gauges)
        h = C.c_void_p()
        rc = lib().geoflood_init_forest(C.byref(self._c), stream, C.byref(h))
        if rc:
            raise GeoFloodError(rc, "init_forest")
        self._h = h
        self._ng = {}
        for s in range(num_scenarios):
            self._check(lib().geoflood_set_scenario(self._h, s, cfg.manning_n, cfg.eta0))
            if dem is not None:
                self.set_topo(dem, s)

    def _check(self, rc):
        if rc:
            raise GeoFloodError(rc, lib().geoflood_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().geoflood_destroy(self._h)
            self._h = None

    __del__ = close

    def set_scenario(self, s, manning_n, eta0):
        self._check(lib().geoflood_set_scenario(self._h, s, manning_n, eta0))

    def save(self):
        """Checkpoint of the whole context (geoflood_save) as bytes."""
        n = C.c_size_t()
        rc = lib().geoflood_save(self._h, None, 0, C.byref(n))
        if rc not in (0, -8):
            self._check(rc)
        buf = (C.c_ubyte * n.value)()
        self._check(lib().geoflood_save(self._h, C.cast(buf, C.c_void_p), n.value, C.byref(n)))
        return bytes(buf)

    def load(self, data):
        """Resume from a checkpoint of save() (same configuration)."""
        buf = (C.c_ubyte * len(data)).from_buffer_copy(data)
        self._check(lib().geoflood_load(self._h, C.cast(buf, C.c_void_p), len(data)))

    def set_topo(self, dem, s=0):
        """One DEM, or a list of up to 4 overlapping DEMs (Sec. 6.2)."""
        if isinstance(dem, (list, tuple)):
            zs = [np.ascontiguousarray(d.z, dtype=np.float64) for d in dem]
            n = len(zs)
            zp = (C.POINTER(C.c_double) * n)(*[_p(z) for z in zs])
            ints = lambda v: (C.c_int * n)(*v)
            dbl = lambda v: (C.c_double * n)(*v)
            self._check(lib().geoflood_set_topos(
                self._h, s, n, zp, ints([z.shape[1] for z in zs]), ints([z.shape[0] for z in zs]),
                dbl([d.x0 for d in dem]), dbl([d.y0 for d in dem]),
                dbl([d.dx for d in dem]), dbl([d.dy for d in dem])))
            return
        z = np.ascontiguousarray(dem.z, dtype=np.float64)
        ny, nx = z.shape
        self._check(lib().geoflood_set_topo(self._h, s, _p(z), nx, ny, dem.x0,
                                            dem.y0, dem.dx, dem.dy))

    def npatch_of(self, s=0):
        n = C.c_int()
        self._check(lib().geoflood_npatch(self._h, s, C.byref(n)))
        return n.value

    @property
    def npatch(self):
        return self.npatch_of(0)

    def patch_info(self, s=0):
        n = self.npatch_of(s)
        L = np.empty(n, np.int32)
        X = np.empty(n, np.int32)
        Y = np.empty(n, np.int32)
        self._check(lib().geoflood_patch_info(self._h, s, _p(L, C.c_int),
                                              _p(X, C.c_int), _p(Y, C.c_int)))
        return L, X, Y

    def write(self, h, hu, hv, s=0):
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (h, hu, hv)]
        self._check(lib().geoflood_write_patches(self._h, s, *[_p(x) for x in a]))

    def read(self, s=0):
        n, m = self.npatch_of(s), self.cfg.mx
        out = [np.empty((n, m, m)) for _ in range(4)]
        self._check(lib().geoflood_read_patches(self._h, s, *[_p(x) for x in out]))
        return tuple(out)

    def read_into(self, h, hu, hv, b=None, s=0):
        """Read the state into caller arrays (e.g. pinned host buffers)."""
        ptr = lambda x: _p(x) if x is not None else None
        self._check(lib().geoflood_read_patches(self._h, s, ptr(h), ptr(hu), ptr(hv), ptr(b)))

    def read_tiles(self, s=0):
        n, T = self.npatch_of(s), self.cfg.mx + 4
        out = np.empty((n, 4, T, T))
        self._check(lib().geoflood_read_tiles(self._h, s, _p(out)))
        return out

    def set_state(self, ic, s=0):
        """Initial state through the library's host callback."""
        def cb(n, x, y, b, h, hu, hv, user):
            X = np.ctypeslib.as_array(x, (n,))
            Y = np.ctypeslib.as_array(y, (n,))
            B = np.ctypeslib.as_array(b, (n,))
            hh, uu, vv = ic(X, Y, B)
            np.ctypeslib.as_array(h, (n,))[:] = np.broadcast_to(hh, (n,))
            np.ctypeslib.as_array(hu, (n,))[:] = np.broadcast_to(uu, (n,))
            np.ctypeslib.as_array(hv, (n,))[:] = np.broadcast_to(vv, (n,))
        fn = QINIT(cb)
        self._check(lib().geoflood_set_state(self._h, s, fn, None))

    def set_time(self, t, dt_next, s=0):
        self._check(lib().geoflood_set_time(self._h, s, float(t), float(dt_next)))

    def time(self, s=0):
        t, dt, cv = C.c_double(), C.c_double(), C.c_double()
        st, rj, nc = C.c_longlong(), C.c_longlong(), C.c_longlong()
        self._check(lib().geoflood_get_time(self._h, s, C.byref(t), C.byref(dt),
                                            C.byref(st), C.byref(rj), C.byref(nc),
                                            C.byref(cv)))
        return dict(t=t.value, dt_next=dt.value, steps=st.value, rejects=rj.value,
                    nclip=nc.value, clipvol=cv.value)

    def step(self, t_target, max_steps=1 << 30):
        """Advance every scenario; returns (t, steps) of scenario 0 and keeps
        the per-scenario arrays in last_t / last_steps."""
        t = np.zeros(self.nscen)
        n = np.zeros(self.nscen, np.int32)
        self._check(lib().geoflood_step(self._h, float(t_target), int(min(max_steps, 2**31 - 1)),
                                        _p(t), _p(n, C.c_int)))
        self.last_t, self.last_steps = t, n
        return float(t[0]), int(n[0])

    def tags(self, s=0):
        f = np.empty(self.npatch_of(s), np.uint8)
        self._check(lib().geoflood_tags(self._h, s, _p(f, C.c_uint8)))
        return f

    def regrid(self):
        self._check(lib().geoflood_regrid(self._h))
        return self.npatch

    def mass(self, s=0):
        m = C.c_double()
        self._check(lib().geoflood_mass(self._h, s, C.byref(m)))
        return m.value

    def set_gauges(self, xy, s=0):
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        self._ng[s] = len(xy)
        self._check(lib().geoflood_set_gauges(self._h, s, _p(xy), len(xy)))

    def gauges(self, s=0):
        c = C.c_int()
        self._check(lib().geoflood_gauge_count(self._h, s, C.byref(c)))
        n = c.value
        out = np.empty((n, 5))
        arr = np.empty(n)
        self._check(lib().geoflood_gauges(self._h, s, _p(out), _p(arr)))
        return out, arr

    def profile(self, enable=True, every=1):
        self._check(lib().geoflood_profile(self._h, int(every) if enable else 0))

    def profile_read(self, kernel):
        ms = C.c_double()
        n = C.c_longlong()
        self._check(lib().geoflood_profile_read(self._h, kernel.encode(), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def profile_cells(self, kernel):
        """Interior cells covered by the recorded launches of a kernel."""
        n = C.c_longlong()
        self._check(lib().geoflood_profile_cells(self._h, kernel.encode(), C.byref(n)))
        return n.value

    def counters(self, s=0):
        a, b = C.c_longlong(), C.c_longlong()
        self._check(lib().geoflood_counters(self._h, s, C.byref(a), C.byref(b)))
        return a.value, b.value

    def autotune(self, reps=5):
        v = C.c_int()
        ms = np.full(16, np.nan)
        self._check(lib().geoflood_autotune(self._h, int(reps), C.byref(v), _p(ms)))
        return v.value, ms

    def set_variant(self, variant):
        self._check(lib().geoflood_set_variant(self._h, int(variant)))

    def launch_count(self):
        n = C.c_longlong()
        self._check(lib().geoflood_launch_count(self._h, C.byref(n)))
        return n.value

    # learned refinement predictor -------------------------------------------

    def cnn_set_params(self, prm):
        prm = np.ascontiguousarray(prm, dtype=np.float32)
        self._check(lib().geoflood_cnn_set_params(self._h, _p(prm, C.c_float), len(prm)))

    def cnn_get_params(self):
        prm = np.empty(cnn_nparam(), np.float32)
        self._check(lib().geoflood_cnn_get_params(self._h, _p(prm, C.c_float), len(prm)))
        return prm

    def cnn_set_scale(self, scale):
        sc = np.ascontiguousarray(scale, dtype=np.float32).reshape(4)
        self._check(lib().geoflood_cnn_set_scale(self._h, _p(sc, C.c_float)))

    def cnn_features(self, s=0):
        """BF16 bit patterns [npatch][324][16] (view with bf16_to_float)."""
        out = np.empty((self.npatch_of(s), CNN_IN_PIX, CNN_CH), np.uint16)
        self._check(lib().geoflood_cnn_features(self._h, s, _p(out, C.c_uint16)))
        return out

    def cnn_predict(self, s=0):
        out = np.empty(self.npatch_of(s), np.float32)
        self._check(lib().geoflood_cnn_predict(self._h, s, _p(out, C.c_float)))
        return out

    def cnn_grad(self, x, label, pos_weight=1.0):
        x = np.ascontiguousarray(x, dtype=np.uint16)
        y = np.ascontiguousarray(label, dtype=np.float32)
        n = len(y)
        logit = np.empty(n, np.float32)
        grad = np.empty(cnn_nparam(), np.float32)
        loss = np.empty(1, np.float32)
        self._check(lib().geoflood_cnn_grad(self._h, _p(x, C.c_uint16), _p(y, C.c_float), n,
                                            float(pos_weight), _p(logit, C.c_float),
                                            _p(grad, C.c_float), _p(loss, C.c_float)))
        return logit, grad, float(loss[0])

    def cnn_dataset(self, capacity):
        self._check(lib().geoflood_cnn_dataset(self._h, int(capacity)))

    def cnn_snapshot(self):
        self._check(lib().geoflood_cnn_snapshot(self._h))

    def check_tags(self, observe=False):
        m = C.c_int()
        self._check(lib().geoflood_check_tags(self._h, 1 if observe else 0, C.byref(m)))
        return m.value

    def cnn_commit(self):
        n, npos = C.c_int(), C.c_int()
        self._check(lib().geoflood_cnn_commit(self._h, C.byref(n), C.byref(npos)))
        return n.value, npos.value

    def cnn_dataset_read(self, first, n):
        x = np.empty((n, CNN_IN_PIX, CNN_CH), np.uint16)
        y = np.empty(n, np.float32)
        self._check(lib().geoflood_cnn_dataset_read(self._h, int(first), int(n),
                                                    _p(x, C.c_uint16), _p(y, C.c_float)))
        return x, y

    def cnn_train(self, epochs, batch, lr=1e-3, pos_weight=1.0, seed=0):
        loss = np.zeros(max(1, epochs), np.float32)
        self._check(lib().geoflood_cnn_train(self._h, int(epochs), int(batch), float(lr),
                                             float(pos_weight), int(seed) & (2**64 - 1),
                                             _p(loss, C.c_float)))
        return loss[:epochs]

    def advance(self, t_target, regrid_interval=4, check_interval=4, collect=False,
                regrid_on_miss=False):
        st = AdvanceStats()
        mode = (1 if collect else 0) | (2 if regrid_on_miss else 0)
        self._check(lib().geoflood_advance(self._h, float(t_target), int(regrid_interval),
                                           int(check_interval), mode, C.byref(st)))
        return st.as_dict()

    def set_tagger(self, tagger, threshold=0.5):
        self._check(lib().geoflood_set_tagger(self._h, int(tagger), float(threshold)))


def cnn_nparam():
    return lib().geoflood_cnn_nparam()


def bf16_to_float(bits):
    """Widen BF16 bit patterns to float32 (exact)."""
    return (np.asarray(bits, np.uint16).astype(np.uint32) << 16).view(np.float32)


def check_bounded_wait(stream=None):
    """geoflood_check_bounded_wait: 0 when a wait on a copy that never
    arrives gives up after its bound and succeeds once the copy is done."""
    return lib().geoflood_check_bounded_wait(stream)


def exported_symbols():
    """Names of the entry points include/geoflood.h declares."""
    import re
    hdr = open(os.path.join(os.path.dirname(_HERE), "include", "geoflood.h")).read()
    return sorted(set(re.findall(r"\b(geoflood_[a-z_]+)\s*\(", hdr)))
