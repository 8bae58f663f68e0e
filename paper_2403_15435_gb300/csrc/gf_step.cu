// FP64 patch step (instantiation of gf_step_kernel.cuh), the device-side
// time-step controller and the allocation-free entry point.  Compiled with
// -fmad=false so that FP64 results round exactly as the operations are
// written.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <atomic>
#include <cstring>

#include "gf_internal.h"
#include "gf_step_kernel.cuh"

namespace {

__global__ void k_ctl_begin(GfCtl* ctl, int nscen, double t_target,
                            long long max_steps, const int* mask) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nscen) return;
  GfCtl* C = ctl + s;
  C->t_target = t_target;
  C->max_steps = max_steps;
  C->taken = 0;
  C->inrow = 0;
  C->accepted = 0;
  C->cmax_bits = 0ull;
  C->rmax_bits = 0ull;
  C->sub_k = 0;
  C->sub_rej = 0;
  C->step_nclip = 0ull;
  C->step_clipvol = 0.0;
  C->nonfinite = 0;
  const bool go = (mask == nullptr || mask[s]) && C->t < t_target &&
                  max_steps > 0 && C->status == 0;
  C->active = go ? 1 : 0;
  if (go) {
    const double rem = t_target - C->t;
    if (C->dt_next < rem) { C->dt_use = C->dt_next; C->last = 0; }
    else { C->dt_use = rem; C->last = 1; }
  }
}

// The bounded-wait check: an mbarrier expects 16 bytes that no copy will
// bring; the CTA's bounded wait must give up (flag 1), then, once the
// transaction is completed by hand, the same wait must succeed (flag 2).
__global__ void k_wait_check(int* out, unsigned limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    gfs::mbar_init(&bar, 1);
    gfs::mbar_expect_tx(&bar, 16u);
  }
  __syncthreads();
  const bool first = __syncthreads_and(gfs::mbar_wait(&bar, limit, 0u) ? 1 : 0);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(gfs::smem_addr(&bar)),
                 "r"(16u)
                 : "memory");
  }
  __syncthreads();
  const bool second = __syncthreads_and(gfs::mbar_wait(&bar, limit, 0u) ? 1 : 0);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(gfs::smem_addr(&bar)) : "memory");
    out[0] = first ? 0 : 1;
    out[1] = second ? 2 : 0;
  }
}

}  // namespace

namespace gf {

// Kernel variants (the autotuner picks one per context): for 32 x 32
// patches, 0 = one 512-thread CTA per patch (TMA bulk staging of the whole
// tile), 1 = four CTAs of 16 x 16 sub-tiles per patch, 2 = as 0 (FP32) or 1
// (FP64) with the register limit for one CTA per SM; 16 x 16 patches have the
// single variant 0.  Dimensionally split stepping has one kernel per patch
// size (whole-patch CTAs).
int patch_step_variants(int mx, int prec, int dim_split) {
  return dim_split ? 1 : (mx == 32 ? (prec ? 8 : 4) : 1);
}

int launch_patch_step_f64(const GfGeom& g, const GfView& v, int variant,
                          void* stream) {
  if (v.npatch <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g.dim_split) {
    if (g.M == 32) return gfs::launch_step<gfs::PrecF64, 32, 32, 512, 1, true>(g, v, st);
    if (g.M == 16) return gfs::launch_step<gfs::PrecF64, 16, 16, 256, 1, true>(g, v, st);
    return -1;
  }
  if (g.M == 32 && variant == 1)
    return gfs::launch_step<gfs::PrecF64, 32, 16, 256, 2>(g, v, st);
  if (g.M == 32 && variant == 2)
    return gfs::launch_step<gfs::PrecF64, 32, 16, 256, 1>(g, v, st);
  if (g.M == 32 && variant == 3)
    return gfs::launch_step_adaptive<gfs::PrecF64, 32, 16, 352, 1>(g, v, st);
  if (g.M == 32) return gfs::launch_step<gfs::PrecF64, 32, 32, 512, 1>(g, v, st);
  if (g.M == 16) return gfs::launch_step<gfs::PrecF64, 16, 16, 256, 1>(g, v, st);
  return -1;
}

int launch_ctl_begin(GfCtl* ctl, int nscen, double t_target,
                     long long max_steps, const int* mask, void* stream) {
  k_ctl_begin<<<(nscen + 127) / 128, 128, 0,
                static_cast<cudaStream_t>(stream)>>>(ctl, nscen, t_target,
                                                      max_steps, mask);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gf

// ---------------------------------------------------------------------------
// Entry point for callers that cannot allocate device memory.
//
// Some callers own every byte of device memory themselves: a solver embedded
// in a host code with its own memory pool, or code that runs where
// cudaMalloc is not allowed (a section that must not grow the device pool,
// or an allocator that hands out only pre-registered buffers).
// They cannot create a geoflood context, because a context allocates its
// state.  geoflood_step_tiles_noalloc runs the same FP64 patch-step kernel on
// tiles the caller provides, and keeps the small scratch it needs (patch
// table and the reduction cell of the CFL rate) in the static
// device array below, so the call allocates nothing.
//
// Limits and behaviour:
//   - at most GF_NOALLOC_MAX_PATCHES patches per call (the array holds
//     GF_NOALLOC_MAX_PATCHES * 16 bytes + 512 bytes, about 260 KiB, on every
//     GPU that loads the library, until the process exits);
//   - the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (once per device); make that first call before any
//     stream capture;
//   - every call reuses the same array and overwrites what the previous call
//     left there (the reduction cell is cleared at the start of each call),
//     so calls whose kernels overlap on the GPU race: issue them on one stream
//     or order them.
// ---------------------------------------------------------------------------
#define GF_NOALLOC_MAX_PATCHES 16384

namespace {

struct NoallocScratch {
  GfCtl ctl;
  GfScenario scen;
  GfPatch patch[GF_NOALLOC_MAX_PATCHES];
};

static __device__ __align__(256) unsigned char
    gf_noalloc_scratch[sizeof(NoallocScratch)];

__global__ void k_noalloc_init(NoallocScratch* S, int n, double dt,
                               double manning_n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    GfCtl c{};
    c.active = 1;
    c.cur = 0;
    c.dt_use = dt;
    S->ctl = c;
    GfScenario sc{};
    sc.manning_n = manning_n;
    sc.pcount = n;
    S->scen = sc;
  }
  if (k < n) S->patch[k] = GfPatch{0, 0, 0, 0};
}

// Device address of the scratch array on the current device, looked up once
// per device.  Two host threads may look it up at the same time; both store
// the same address, and the atomics make that well defined.
NoallocScratch* noalloc_scratch(int* rc) {
  static std::atomic<NoallocScratch*> addr[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *rc = -2;
    return nullptr;
  }
  NoallocScratch* a = addr[dev].load(std::memory_order_acquire);
  if (!a) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, gf_noalloc_scratch) != cudaSuccess || !p) {
      *rc = -2;
      return nullptr;
    }
    a = static_cast<NoallocScratch*>(p);
    addr[dev].store(a, std::memory_order_release);
  }
  *rc = 0;
  return a;
}

// Whether the byte ranges [a, a + na) and [b, b + nb) intersect.
bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t pa = reinterpret_cast<uintptr_t>(a);
  const uintptr_t pb = reinterpret_cast<uintptr_t>(b);
  return pa < pb + nb && pb < pa + na;
}

thread_local char noalloc_err[256] = "";

int noalloc_fail(int code, const char* msg) {
  snprintf(noalloc_err, sizeof(noalloc_err), "%s", msg);
  return code;
}

}  // namespace

extern "C" const char* geoflood_noalloc_last_error(void) { return noalloc_err; }

extern "C" int geoflood_step_tiles_noalloc(const double* q_in, const double* b,
                                           double* q_out, int npatch, int mx,
                                           double dx, double dy, double dt,
                                           double g, double drytol,
                                           double manning_n, double* cmax,
                                           void* stream) {
  if (!q_in || !b || !q_out || q_in == q_out || !(mx == 16 || mx == 32) ||
      !(dx > 0) || !(dy > 0) || !(dt > 0) || !(g > 0) || !(drytol > 0) ||
      !(manning_n >= 0))
    return noalloc_fail(-1, "step_tiles_noalloc: bad argument");
  if (npatch < 1 || npatch > GF_NOALLOC_MAX_PATCHES)
    return noalloc_fail(-8, "step_tiles_noalloc: npatch must be in [1, 16384]");
  // the kernel stages whole tiles with bulk copies, which need 16-byte
  // aligned addresses (a tile plane is a multiple of 16 bytes for mx = 16
  // and 32, so every tile of an aligned buffer is aligned)
  if ((reinterpret_cast<uintptr_t>(q_in) | reinterpret_cast<uintptr_t>(b) |
       reinterpret_cast<uintptr_t>(q_out)) & 15u)
    return noalloc_fail(-1, "step_tiles_noalloc: q_in, b and q_out must be 16-byte aligned");
  {
    const size_t T = (size_t)mx + 2 * GF_NG;
    const size_t qbytes = 3 * (size_t)npatch * T * T * sizeof(double);
    const size_t bbytes = (size_t)npatch * T * T * sizeof(double);
    if (ranges_overlap(q_out, qbytes, q_in, qbytes) || ranges_overlap(q_out, qbytes, b, bbytes))
      return noalloc_fail(-1, "step_tiles_noalloc: q_out overlaps q_in or b");
  }
  int rc = 0;
  NoallocScratch* S = noalloc_scratch(&rc);
  if (!S) return noalloc_fail(rc, "step_tiles_noalloc: cudaGetSymbolAddress failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // one level-0 patch per tile; the patch width mx*dx is a power-of-two
  // multiple of dx, so the kernel's dx = width / mx is exact
  GfGeom G{};
  G.mi = 1; G.mj = 1; G.M = mx; G.T = mx + 2 * GF_NG;
  G.xlower = 0.0; G.xupper = dx * mx;
  G.ylower = 0.0; G.yupper = dy * mx;
  G.g = g; G.drytol = drytol;
  G.cfl_desired = 0.9; G.cfl_max = 1.0; G.dt_max = 1e300;
  G.nscen = 1;
  GfView V{};
  V.patch = S->patch;
  V.lut = nullptr;
  V.scen = &S->scen;
  V.ctl = &S->ctl;
  V.q[0] = const_cast<double*>(q_in);
  V.q[1] = q_out;
  V.b = const_cast<double*>(b);
  V.npatch = npatch;
  k_noalloc_init<<<(npatch + 255) / 256, 256, 0, st>>>(S, npatch, dt, manning_n);
  if (cudaGetLastError() != cudaSuccess)
    return noalloc_fail(-2, "step_tiles_noalloc: init launch failed");
  const int lr = mx == 32
                     ? gfs::launch_step<gfs::PrecF64, 32, 32, 512, 1>(G, V, st)
                     : gfs::launch_step<gfs::PrecF64, 16, 16, 256, 1>(G, V, st);
  if (lr) return noalloc_fail(-2, "step_tiles_noalloc: step launch failed");
  if (cmax) {
    // the reduction cell and the kernel's status in one copy: a bounded
    // wait that gave up leaves its tile unwritten, and a non-finite value
    // makes the result unusable; both are reported instead of success
    GfCtl c{};
    if (cudaMemcpyAsync(&c, &S->ctl, sizeof(c), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return noalloc_fail(-2, "step_tiles_noalloc: reading the CFL rate failed");
    double v;
    std::memcpy(&v, &c.cmax_bits, sizeof(v));
    *cmax = v;
    if (c.status == -7)
      return noalloc_fail(-7, "step_tiles_noalloc: a bounded device wait expired; "
                              "some tiles were not written");
    if (c.nonfinite || c.status == -5)
      return noalloc_fail(-5, "step_tiles_noalloc: non-finite value in the result");
  }
  return 0;
}

// Confirms, on the GPU in use, that the library's bounded waits end: a wait
// on a transaction that never arrives gives up after its limit (the patch
// step then reports GEOFLOOD_ERR_TIMEOUT and returns), and succeeds once the
// transaction completes.  Runs one CTA; allocates 8 bytes of device memory.
extern "C" int geoflood_check_bounded_wait(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) return -3;
  k_wait_check<<<1, 128, 0, st>>>(d, 4096u);
  int h[2] = {-1, -1};
  const bool ok = cudaGetLastError() == cudaSuccess &&
                  cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                  cudaStreamSynchronize(st) == cudaSuccess;
  cudaFree(d);
  if (!ok) return -2;
  return h[0] == 1 && h[1] == 2 ? 0 : -9;
}
