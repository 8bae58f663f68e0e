"""The allocation-free patch-step entry point (geoflood_step_tiles_noalloc).

Some callers own all device memory themselves (a host code with its own
device pool, or one where cudaMalloc is not allowed) and so cannot create a
context.  This entry point steps tiles they provide and keeps its scratch in
a static device array.  The tests compare its output with the context path
(geoflood_step) on two calls in a row, on 32 x 32 and 16 x 16 patches,
within the FP64 parity tolerance; check that the ghost layers of q_out hold
the wall mirrors of the new edge cells; and check that it refuses too many
patches, misaligned buffers and an output overlapping its inputs before
issuing any work.  The file is named so that pytest collects it last."""
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


def wall_mirror(tiles, m):
    """Expected ghost ring of stepped tiles [n][3][T][T] (interior filled)
    for a lone patch with walls on every side: ghost cell (i, j) takes the
    interior cell mirrored across each wall it lies beyond, with the normal
    momentum of that wall negated."""
    T = m + 4
    idx = np.arange(T) - 2
    mir = np.where(idx < 0, -1 - idx, np.where(idx >= m, 2 * m - 1 - idx, idx)) + 2
    ghost = (idx < 0) | (idx >= m)
    out = tiles[:, :, mir[:, None], mir[None, :]].copy()   # [n][3][row j][col i]
    out[:, 1] *= np.where(ghost[None, :], -1.0, 1.0)           # hu: x walls
    out[:, 2] *= np.where(ghost[:, None], -1.0, 1.0)           # hv: y walls
    return out, ghost[:, None] | ghost[None, :]


@pytest.mark.parametrize("m,dx", [(32, 4.0), (16, 4.0)])
def test_noalloc_step_matches_context_step_twice(m, dx):
    torch = pytest.importorskip("torch")
    step, L = _fn()
    prob = inputs.radial_dambreak(128, m, dx=dx, radius=100.0)
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
        q_out = torch.full_like(q_in, 12345.0)        # sentinel in every entry
        cmax = C.c_double()
        torch.cuda.synchronize(dev)
        rc = step(q_in.data_ptr(), b.data_ptr(), q_out.data_ptr(), n, m, dx, dx,
                  info["dt_next"], prob.cfg.g, prob.cfg.drytol, prob.cfg.manning_n,
                  C.byref(cmax), C.c_void_p(stream.cuda_stream))
        assert rc == 0, L.geoflood_noalloc_last_error()
        full = q_out.cpu().numpy()
        out = full[:, :, 2:-2, 2:-2]
        ctx.step(1e9, 1)                              # the context path
        after = ctx.time()
        assert after["rejects"] == info["rejects"], "context retook the step"
        h, hu, hv, _ = ctx.read()
        for k, ref in enumerate((h, hu, hv)):
            assert rel(out[:, k], ref) <= TOL, "call %d field %d" % (call, k)
        assert 0.9 / cmax.value == pytest.approx(after["dt_next"], rel=TOL)
        # no sentinel survives, and the ghosts are the walls' mirrors
        assert not np.any(full == 12345.0)
        expect, ghost = wall_mirror(full, m)
        assert np.array_equal(full[:, :, ghost], expect[:, :, ghost]), "call %d ghosts" % call


def test_noalloc_rejects_more_patches_than_its_scratch_holds():
    step, L = _fn()
    cmax = C.c_double()
    rc = step(C.c_void_p(16), C.c_void_p(32), C.c_void_p(64), 16385, 32, 1.0, 1.0,
              0.1, 9.81, 1e-3, 0.0, C.byref(cmax), None)
    assert rc == -8
    assert b"16384" in L.geoflood_noalloc_last_error()


def test_noalloc_refuses_misaligned_and_overlapping_buffers():
    """Refused on the host with ARG before any work is issued: the pointers
    below are never dereferenced."""
    step, L = _fn()
    cmax = C.c_double()
    T = 36
    tile = 3 * T * T * 8
    base = 1 << 20

    def call(q_in, b, q_out, n=4):
        return step(C.c_void_p(q_in), C.c_void_p(b), C.c_void_p(q_out), n, 32, 1.0, 1.0,
                    0.1, 9.81, 1e-3, 0.0, C.byref(cmax), None)

    far = base + 64 * tile
    assert call(base + 8, far, 2 * far) == -1          # q_in 8-byte aligned only
    assert b"aligned" in L.geoflood_noalloc_last_error()
    assert call(base, far + 8, 2 * far) == -1          # bed
    assert call(base, far, 2 * far + 8) == -1          # output
    assert call(base, far, base + tile) == -1          # q_out starts inside q_in
    assert b"overlaps" in L.geoflood_noalloc_last_error()
    assert call(base + tile, far, base) == -1          # q_in starts inside q_out
    assert call(base, far, far + 16) == -1             # q_out overlaps b
