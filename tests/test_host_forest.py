"""The library's host quadtree (the regrid rule of Sec. 4 and Sec. 6.6 in
paper_2403_15435_gb300/csrc/gf_forest.cpp, compiled with g++ behind a small C
shim) against the oracle's own regrid given the same flags: random refine /
coarsen flags over many regrids on forests of several shapes and level
ranges.  The two implementations share no code; their leaf lists (Morton
order) must be identical, and each list must tile the domain with the 2:1
balance across faces and corners."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import inputs
from test_oracle_amr import _check_balanced_cover

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ is not available")
    out = str(tmp_path_factory.mktemp("forest") / "libforest_shim.so")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out,
                           os.path.join(HERE, "forest_shim.cpp"),
                           os.path.join(ROOT, "paper_2403_15435_gb300", "csrc", "gf_forest.cpp")])
    lib = C.CDLL(out)
    ip = C.POINTER(C.c_int)
    lib.forest_regrid.argtypes = [C.c_int] * 5 + [ip, ip, ip, C.POINTER(C.c_uint8), C.c_int,
                                                  ip, ip, ip]
    lib.forest_regrid.restype = C.c_int
    return lib


def host_regrid(lib, cfg, L, X, Y, flags):
    n = len(L)
    cap = 4 * n + 64
    outs = [np.zeros(cap, np.int32) for _ in range(3)]
    ins = [np.ascontiguousarray(a, dtype=np.int32) for a in (L, X, Y)]
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    ptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
    m = lib.forest_regrid(cfg.mi, cfg.mj, cfg.minlevel, cfg.maxlevel, n, *[ptr(a) for a in ins],
                          f.ctypes.data_as(C.POINTER(C.c_uint8)), cap, *[ptr(a) for a in outs])
    assert m >= 0
    return [a[:m] for a in outs]


def random_flags(rng, L, cfg, p_refine, p_coarsen):
    """Flags the tagger could give: refine below the finest level, coarsen
    above the coarsest, keep otherwise."""
    u = rng.random(len(L))
    f = np.zeros(len(L), np.uint8)
    f[(u < p_refine) & (L < cfg.maxlevel)] = 1
    f[(u >= p_refine) & (u < p_refine + p_coarsen) & (L > cfg.minlevel)] = 2
    return f


@pytest.mark.parametrize("mi,mj,minl,maxl", [(2, 2, 0, 3), (3, 2, 0, 4), (4, 2, 1, 4), (1, 1, 0, 5)])
def test_host_forest_regrid_equals_oracle_regrid(shim, mi, mj, minl, maxl):
    cfg = inputs.Config(mi=mi, mj=mj, mx=4, minlevel=minl, maxlevel=maxl,
                        xupper=100.0 * mi, yupper=100.0 * mj, drytol=1e-3)
    f = oracle.OracleForest(cfg)
    rng = np.random.default_rng(1000 * mi + 100 * mj + 10 * minl + maxl)
    levels_seen = set()
    for it in range(30):
        L, X, Y = f.patch_info()
        # phases that mostly refine, then mostly coarsen, then mix
        pr, pc = ((0.3, 0.1), (0.05, 0.8), (0.15, 0.4))[it // 10]
        flags = random_flags(rng, L, cfg, pr, pc)
        want = host_regrid(shim, cfg, L, X, Y, flags)
        f.regrid_flags(flags)
        got = f.patch_info()
        for a, b in zip(got, want):
            assert np.array_equal(a, b), "regrid %d: leaf lists differ" % it
        _check_balanced_cover(f, cfg)
        levels_seen |= set(int(v) for v in got[0])
    # the runs reach the finest level and come back down
    assert max(levels_seen) == maxl and min(levels_seen) == minl


def test_host_forest_keeps_the_forest_when_nothing_is_flagged(shim):
    cfg = inputs.Config(mi=2, mj=2, mx=4, minlevel=0, maxlevel=3, xupper=200.0, yupper=200.0)
    f = oracle.OracleForest(cfg)
    rng = np.random.default_rng(5)
    for _ in range(4):
        L, X, Y = f.patch_info()
        f.regrid_flags(random_flags(rng, L, cfg, 0.4, 0.0))
    L, X, Y = f.patch_info()
    got = host_regrid(shim, cfg, L, X, Y, np.zeros(len(L), np.uint8))
    for a, b in zip(got, (L, X, Y)):
        assert np.array_equal(a, b)
