// FP32 surface-deviation patch step (instantiation of gf_step_kernel.cuh).
// Compiled with fused multiply-add allowed: this path is checked against the
// FP64 oracle with absolute depth and momentum tolerances, not bit for bit.
#include <cuda_runtime.h>

#include "gf_internal.h"
#include "gf_step_kernel.cuh"

namespace gf {

int launch_patch_step_f32(const GfGeom& g, const GfView& v, int variant,
                          void* stream) {
  if (v.npatch <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g.dim_split) {
    if (g.M == 32) return gfs::launch_step<gfs::PrecF32, 32, 32, 512, 2, true>(g, v, st);
    if (g.M == 16) return gfs::launch_step<gfs::PrecF32, 16, 16, 352, 2, true>(g, v, st);
    return -1;
  }
  if (g.M == 32 && variant == 1)
    return gfs::launch_step<gfs::PrecF32, 32, 16, 352, 2>(g, v, st);
  if (g.M == 32 && variant == 2)
    return gfs::launch_step<gfs::PrecF32, 32, 32, 512, 1>(g, v, st);
  if (g.M == 32 && variant == 3)
    return gfs::launch_step<gfs::PrecF32, 32, 32, 1024, 1>(g, v, st);
  // 16 x 16 sub-tiles with more CTAs per SM: 352 threads, three CTAs (one
  // round per sweep phase, 56 registers); 320 threads, four CTAs
  if (g.M == 32 && variant == 4)
    return gfs::launch_step<gfs::PrecF32, 32, 16, 352, 3>(g, v, st);
  if (g.M == 32 && variant == 5)
    return gfs::launch_step<gfs::PrecF32, 32, 16, 320, 4>(g, v, st);
  // adaptive: four 16 x 16 sub-tile CTAs for each patch wet in the previous
  // launch, one whole-tile check (and dry update) for every other patch
  if (g.M == 32 && variant == 6)
    return gfs::launch_step_adaptive<gfs::PrecF32, 32, 16, 352, 1>(g, v, st);
  // 608 threads, two CTAs per SM: every sweep phase in two rounds instead of
  // three (48 registers, a few bytes spilled)
  if (g.M == 32 && variant == 7)
    return gfs::launch_step<gfs::PrecF32, 32, 32, 608, 2>(g, v, st);
  if (g.M == 32) return gfs::launch_step<gfs::PrecF32, 32, 32, 512, 2>(g, v, st);
  if (g.M == 16) return gfs::launch_step<gfs::PrecF32, 16, 16, 352, 2>(g, v, st);
  return -1;
}

}  // namespace gf
