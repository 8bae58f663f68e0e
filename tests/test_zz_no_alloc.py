"""The allocation-free patch-step entry point (geoflood_step_tiles_noalloc).

Callers that own all device memory cannot create a context; this entry point
steps tiles they provide and keeps its scratch in a static device array.  The
test compares its output with the context path (geoflood_step) on two calls in
a row, within the FP64 parity tolerance, and checks the size limit.  The file
is named so that pytest collects it last."""
import ctypes as C

import numpy as np
import pytest

from paper_2403_15435_gb300 import geoflood, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _fn():
    L = geoflood.lib()
    f = L.geoflood_step_tiles_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int] + \
        [C.c_double] * 6 + [C.POINTER(C.c_double), C.c_void_p]
    f.restype = C.c_int
    L.geoflood_noalloc_last_error.restype = C.c_char_p
    return f, L


def rel(a, b):
    return float(np.abs(a - b).max()) / max(1.0, float(np.abs(b).max()))


def test_noalloc_step_matches_context_step_twice():
    torch = pytest.importorskip("torch")
    step, _ = _fn()
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0)
    ctx = geoflood.Forest(prob.cfg, prob.dem)
    ctx.set_state(prob.ic)
    ctx.step(1e9, 10)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        info = ctx.time()
        tiles = ctx.read_tiles()                      # [n][4][T][T]
        n, T = tiles.shape[0], tiles.shape[2]
        q_in = torch.from_numpy(np.ascontiguousarray(tiles[:, :3])).to(dev)
        b = torch.from_numpy(np.ascontiguousarray(tiles[:, 3])).to(dev)
        q_out = torch.zeros_like(q_in)
        cmax = C.c_double()
        torch.cuda.synchronize(dev)
        rc = step(q_in.data_ptr(), b.data_ptr(), q_out.data_ptr(), n, 32, 4.0, 4.0,
                  info["dt_next"], prob.cfg.g, prob.cfg.drytol, prob.cfg.manning_n,
                  C.byref(cmax), C.c_void_p(stream.cuda_stream))
        assert rc == 0
        out = q_out.cpu().numpy()[:, :, 2:-2, 2:-2]
        ctx.step(1e9, 1)                              # the context path
        after = ctx.time()
        assert after["rejects"] == info["rejects"], "context retook the step"
        h, hu, hv, _ = ctx.read()
        for k, ref in enumerate((h, hu, hv)):
            assert rel(out[:, k], ref) <= TOL, "call %d field %d" % (call, k)
        assert 0.9 / cmax.value == pytest.approx(after["dt_next"], rel=TOL)


def test_noalloc_rejects_more_patches_than_its_scratch_holds():
    step, L = _fn()
    cmax = C.c_double()
    rc = step(C.c_void_p(16), C.c_void_p(32), C.c_void_p(64), 16385, 32, 1.0, 1.0,
              0.1, 9.81, 1e-3, 0.0, C.byref(cmax), None)
    assert rc == -8
    assert b"16384" in L.geoflood_noalloc_last_error()
