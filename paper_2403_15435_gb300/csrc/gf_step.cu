// Patch step (FP64) and the device-side time-step controller.
//
// patch_step: one CTA per patch.  The 36x36 tile (32x32 interior + 2 ghost
// layers) of h, hu, hv and b is staged in shared memory by four 1D TMA bulk
// copies; then, in barrier-separated phases, the CTA computes every x-edge's
// augmented Riemann solve (Sec. 3.3), the MC-limited f-wave corrections
// (Sec. 3.2, Eq. wpa_update_corrections), the per-cell x increments and their
// transverse split along y (2D extension, leveque2002 cited in Sec. 3.2), the
// same for y, the unsplit update, Manning friction (Eq. manning), and the
// per-patch CFL rate (warp-shuffle max) and volume.  Compiled with
// -fmad=false so that FP64 results round exactly as the operations are
// written.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>

#include "gf_internal.h"
#include "gf_solver.cuh"

namespace {

using gfk::Side;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src,
                                         unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bounded wait on phase 0 of the barrier; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], "
        "%2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(0u)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = v > w ? v : w;
  }
  return v;
}

__device__ __forceinline__ double warp_sum_tree(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int M>
struct Layout {
  static constexpr int T = M + 2 * GF_NG;
  static constexpr int TT = T * T;
  static constexpr int NR = M + 2;  // lines swept: one ghost line each side
  static constexpr int NE = M + 3;  // edges per line, a in [-1, M+1]
  static constexpr int NEDGE = NR * NE;
  static constexpr int NLIM = NR * (M + 1);   // edges a in [0, M] per line
  static constexpr int NCELL = M * (M + 2);   // cells of the increments
  // shared memory, in doubles
  static constexpr int OFF_W = 4 * TT;
  static constexpr int OFF_F = OFF_W + 12 * NEDGE;
  static constexpr int OFF_G = OFF_F + 3 * M * (M + 1);
  static constexpr int OFF_RED = OFF_G + 3 * M * (M + 1);
  static constexpr int NDOUBLE = OFF_RED + 64;
  static constexpr size_t BYTES = sizeof(double) * NDOUBLE + 16;
};

template <int M>
__device__ __forceinline__ int tix(int i, int j) {
  return (i + GF_NG) + (j + GF_NG) * (M + 2 * GF_NG);
}

// Increment cell of item k in a sweep: items below M*M are interior cells in
// the fixed order (i = k % M, j = k / M) used by the final update, so each
// thread owns the same cells in both sweeps; then the ghost line before and
// the one after.  a is the position along the sweep, line the one across.
template <int M>
__device__ __forceinline__ void cell_item(int k, int dir, int& a, int& line) {
  if (k < M * M) {
    const int i = k % M, j = k / M;
    a = dir == 0 ? i : j;
    line = dir == 0 ? j : i;
  } else if (k < M * M + M) {
    a = k - M * M;
    line = -1;
  } else {
    a = k - M * M - M;
    line = M;
  }
}

template <int M, int NT>
__global__ void __launch_bounds__(NT, 1)
    k_patch_step(const GfGeom G, const GfView V, double* __restrict__ pmass) {
  using Lo = Layout<M>;
  constexpr int TT = Lo::TT, NE = Lo::NE;
  constexpr int RL = (Lo::NLIM + NT - 1) / NT;    // limiter items per thread
  constexpr int RC = (M * M + NT - 1) / NT;       // interior cells per thread
  constexpr int RX = (Lo::NCELL + NT - 1) / NT;   // increment cells per thread

  const int p = blockIdx.x;
  const GfPatch P = V.patch[p];
  GfCtl* C = V.ctl + P.scen;
  if (!C->active) return;

  extern __shared__ __align__(16) double sm[];
  double* sh = sm;
  double* shu = sm + TT;
  double* shv = sm + 2 * TT;
  double* sb = sm + 3 * TT;
  double* W = sm + Lo::OFF_W;
  double* Ftr = sm + Lo::OFF_F;  // [row j][edge a in 0..M][3]
  double* Gtr = sm + Lo::OFF_G;  // [column i][edge a in 0..M][3]
  double* red = sm + Lo::OFF_RED;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + Lo::NDOUBLE);

  const int tid = threadIdx.x;
  const int cur = C->cur;
  const double* qs = V.q[cur] + (size_t)p * 3 * TT;
  double* qd = V.q[cur ^ 1] + (size_t)p * 3 * TT;
  const double* bs = V.b + (size_t)p * TT;

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, 4u * TT * sizeof(double));
    bulk_g2s(sh, qs, TT * sizeof(double), bar);
    bulk_g2s(shu, qs + TT, TT * sizeof(double), bar);
    bulk_g2s(shv, qs + 2 * TT, TT * sizeof(double), bar);
    bulk_g2s(sb, bs, TT * sizeof(double), bar);
  }
  __syncthreads();
  if (!mbar_wait(bar, GF_SPIN_LIMIT)) {
    if (tid == 0) C->status = -7;  // GEOFLOOD_ERR_TIMEOUT
    mbar_wait(bar, GF_SPIN_LIMIT);
    return;
  }

  const double g = G.g, drytol = G.drytol;
  const double dt = C->dt_use;
  const long long NXL = (long long)G.mi * M << P.level;
  const long long NYL = (long long)G.mj * M << P.level;
  const double dx = (G.xupper - G.xlower) / (double)NXL;
  const double dy = (G.yupper - G.ylower) / (double)NYL;
  const double nux = dt / dx, nuy = dt / dy;
  double smx = 0.0, smy = 0.0;

  double X[RC][3];   // nu_x * dQx of owned interior cells
  double Y[RC][3];   // nu_y * dQy

  // ---------------------------------------------------------- two sweeps
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    const double* sn = dir == 0 ? shu : shv;  // normal momentum
    const double* st = dir == 0 ? shv : shu;  // transverse momentum
    const double nu = dir == 0 ? nux : nuy;
    // phase 1: Riemann solves on lines -1..M, edges -1..M+1
    for (int k = tid; k < Lo::NEDGE; k += NT) {
      const int line = k / NE - 1, a = k % NE - 1;
      const int cl = dir == 0 ? tix<M>(a - 1, line) : tix<M>(line, a - 1);
      const int cr = dir == 0 ? tix<M>(a, line) : tix<M>(line, a);
      double Z[9], S[3];
      gfk::riemann<double>(Side<double>{sh[cl], sn[cl], st[cl], sb[cl]},
                           Side<double>{sh[cr], sn[cr], st[cr], sb[cr]}, g,
                           drytol, Z, S);
      double* w = W + 12 * k;
#pragma unroll
      for (int q = 0; q < 9; ++q) w[q] = Z[q];
      w[9] = S[0];
      w[10] = S[1];
      w[11] = S[2];
    }
    __syncthreads();
    // phase 2: fluctuations and limited corrections on edges 0..M
    double AMr[RL][3], APr[RL][3], FFr[RL][3];
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int k = tid + r * NT;
      if (k < Lo::NLIM) {
        const int line = k / (M + 1) - 1, a = k % (M + 1);
        const int e = (line + 1) * NE + a + 1;
        const double* w = W + 12 * e;
        const int cl = dir == 0 ? tix<M>(a - 1, line) : tix<M>(line, a - 1);
        const int cr = dir == 0 ? tix<M>(a, line) : tix<M>(line, a);
        const bool wet = (sh[cl] > drytol) && (sh[cr] > drytol);
        gfk::edge_fluxes<double>(w, w + 9, w - 12, w + 12, nu, wet, AMr[r],
                                 APr[r], FFr[r]);
        if (line >= 0 && line < M) {
          double m = 0.0;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const double as = w[9 + q] > 0.0 ? w[9 + q] : -w[9 + q];
            m = as > m ? as : m;
          }
          if (dir == 0) smx = m > smx ? m : smx;
          else smy = m > smy ? m : smy;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int k = tid + r * NT;
      if (k < Lo::NLIM) {
        const int line = k / (M + 1) - 1, a = k % (M + 1);
        double* w = W + 12 * ((line + 1) * NE + a + 1);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          w[q] = AMr[r][q];
          w[3 + q] = APr[r][q];
          w[6 + q] = FFr[r][q];
        }
      }
    }
    __syncthreads();
    // phase 3: per-cell increments and their transverse split
    double* Tr = dir == 0 ? Gtr : Ftr;
    double MIr[RX][3];
#pragma unroll
    for (int r = 0; r < RX; ++r) {
      const int k = tid + r * NT;
      if (k < Lo::NCELL) {
        int a, line;  // a: position along the sweep, line: across
        cell_item<M>(k, dir, a, line);
        const double* wl = W + 12 * ((line + 1) * NE + a + 1);  // edge a
        const double* wr = wl + 12;                              // edge a+1
        double d[3];  // frame: mass, normal (sweep) momentum, transverse
#pragma unroll
        for (int q = 0; q < 3; ++q)
          d[q] = (wl[3 + q] + wr[q]) + (wr[6 + q] - wl[6 + q]);
        if (r < RC && k < M * M) {
          // store nu * dQ in (h, hu, hv) order
          if (dir == 0) {
            X[r][0] = nu * d[0]; X[r][1] = nu * d[1]; X[r][2] = nu * d[2];
          } else {
            Y[r][0] = nu * d[0]; Y[r][1] = nu * d[2]; Y[r][2] = nu * d[1];
          }
        }
        // split along the other direction: in that frame the "along"
        // momentum is this sweep's transverse momentum
        const int ci = dir == 0 ? tix<M>(a, line) : tix<M>(line, a);
        const int cm = dir == 0 ? tix<M>(a, line - 1) : tix<M>(line - 1, a);
        const int cp = dir == 0 ? tix<M>(a, line + 1) : tix<M>(line + 1, a);
        const double dd[3] = {d[0], d[2], d[1]};
        double pl[3], mi[3];
        gfk::tsplit<double>(sh[ci], st[ci], sn[ci], sb[ci], sh[cm], sb[cm],
                            sh[cp], sb[cp], dd, g, drytol, pl, mi);
        // back to (h, hu, hv): frame (mass, along = st, other = sn)
        const double plh[3] = {pl[0], dir == 0 ? pl[2] : pl[1],
                               dir == 0 ? pl[1] : pl[2]};
        MIr[r][0] = mi[0];
        MIr[r][1] = dir == 0 ? mi[2] : mi[1];
        MIr[r][2] = dir == 0 ? mi[1] : mi[2];
        if (line + 1 <= M) {
          double* o = Tr + 3 * (a * (M + 1) + line + 1);
          o[0] = plh[0]; o[1] = plh[1]; o[2] = plh[2];
        }
      }
    }
    __syncthreads();
    const double nut = dir == 0 ? nux : nuy;
#pragma unroll
    for (int r = 0; r < RX; ++r) {
      const int k = tid + r * NT;
      if (k < Lo::NCELL) {
        int a, line;
        cell_item<M>(k, dir, a, line);
        if (line >= 0) {
          double* o = Tr + 3 * (a * (M + 1) + line);
#pragma unroll
          for (int q = 0; q < 3; ++q) o[q] = -0.5 * nut * (o[q] + MIr[r][q]);
        }
      }
    }
    __syncthreads();
  }

  // ------------------------------------------------ update, friction, out
  const double mn = V.scen[P.scen].manning_n;
  double vol = 0.0, clipd = 0.0;
  unsigned nclip = 0, nwet = 0;
  bool bad = false;
#pragma unroll
  for (int r = 0; r < RC; ++r) {
    const int k = tid + r * NT;
    if (k < M * M) {
      const int i = k % M, j = k / M;
      const int c = tix<M>(i, j);
      const double q[3] = {sh[c], shu[c], shv[c]};
      nwet += q[0] > drytol ? 1u : 0u;
      double o[3];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const double fl = X[r][f] + Y[r][f];
        const double* fa = Ftr + 3 * (j * (M + 1) + i);
        const double* ga = Gtr + 3 * (i * (M + 1) + j);
        const double tf = nux * (fa[3 + f] - fa[f]) + nuy * (ga[3 + f] - ga[f]);
        o[f] = (q[f] - fl) - tf;
      }
      if (o[0] < 0.0) { clipd -= o[0]; o[0] = 0.0; ++nclip; }
      if (mn > 0.0 && o[0] > drytol) {
        const double u = o[1] / o[0], v = o[2] / o[0];
        const double sp = sqrt(u * u + v * v);
        const double D = g * mn * mn * sp / (o[0] * cbrt(o[0]));
        const double den = 1.0 + dt * D;
        o[1] = o[1] / den;
        o[2] = o[2] / den;
      }
      if (o[0] <= drytol) { o[1] = 0.0; o[2] = 0.0; }
      bad |= !(isfinite(o[0]) && isfinite(o[1]) && isfinite(o[2]));
      qd[c] = o[0];
      qd[TT + c] = o[1];
      qd[2 * TT + c] = o[2];
      vol += o[0];
    }
  }

  // block reductions: CFL rate (max), volume (fixed-order tree)
  const int lane = tid & 31, wid = tid >> 5;
  constexpr int NW = NT / 32;
  smx = warp_max(smx);
  smy = warp_max(smy);
  vol = warp_sum_tree(vol);
  nwet = __reduce_add_sync(0xffffffffu, nwet);
  if (lane == 0 && nwet) atomicAdd(&C->wet_updates, (unsigned long long)nwet);
  if (lane == 0) {
    red[wid] = smx;
    red[NW + wid] = smy;
    red[2 * NW + wid] = vol;
  }
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0, my = 0.0, vs = 0.0;
    for (int w = 0; w < NW; ++w) {
      mx = red[w] > mx ? red[w] : mx;
      my = red[NW + w] > my ? red[NW + w] : my;
      vs += red[2 * NW + w];
    }
    const double cx = mx / dx, cy = my / dy;
    const double cm = cx > cy ? cx : cy;
    atomicMax(&C->cmax_bits, (unsigned long long)__double_as_longlong(cm));
    atomicAdd(&C->cell_updates, (unsigned long long)(M * M));
    pmass[p] = vs * (dx * dy);
  }
  if (nclip) {
    atomicAdd(&C->step_nclip, (unsigned long long)nclip);
    atomicAdd(&C->step_clipvol, clipd * (dx * dy));
  }
  if (bad) C->nonfinite = 1;
}

// Controller: one block per scenario.  Sums the per-patch volumes in a fixed
// order, then thread 0 applies the CFL rule (Sec. 5.1, Sec. 6.6): reject and
// retake when dt*cmax > cfl_max, else accept, advance t and pick the next dt.
__global__ void k_controller(const GfGeom G, GfCtl* ctl, const GfScenario* sc,
                             const double* __restrict__ pmass) {
  const int s = blockIdx.x;
  GfCtl* C = ctl + s;
  __shared__ double red[256];
  __shared__ int act;
  if (threadIdx.x == 0) {
    act = C->active;
    if (!act) C->accepted = 0;
  }
  __syncthreads();
  if (!act) return;
  const int off = sc[s].poff, n = sc[s].pcount;
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += pmass[off + k];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double cmax = __longlong_as_double((long long)C->cmax_bits);
  C->cmax_bits = 0ull;
  const double dt = C->dt_use;
  if (C->nonfinite) {
    C->status = -5;  // GEOFLOOD_ERR_NAN
    C->active = 0;
    C->accepted = 0;
    return;
  }
  if (dt * cmax > G.cfl_max) {
    C->dt_next = G.cfl_desired / cmax;
    C->rejects += 1;
    C->accepted = 0;
    C->step_nclip = 0ull;
    C->step_clipvol = 0.0;
    if (++C->inrow > GF_MAXSTEP_REJECT) {
      C->status = -4;  // GEOFLOOD_ERR_CFL
      C->active = 0;
      return;
    }
  } else {
    C->inrow = 0;
    C->cur ^= 1;
    C->t = C->last ? C->t_target : C->t + dt;
    C->steps += 1;
    C->taken += 1;
    C->nclip += (long long)C->step_nclip;
    C->clipvol += C->step_clipvol;
    C->step_nclip = 0ull;
    C->step_clipvol = 0.0;
    C->mass = red[0];
    C->accepted = 1;
    if (cmax > 0.0) {
      const double dn = G.cfl_desired / cmax;
      C->dt_next = dn < G.dt_max ? dn : G.dt_max;
    }
  }
  if (!(C->t < C->t_target) || C->taken >= C->max_steps) {
    C->active = 0;
    return;
  }
  const double rem = C->t_target - C->t;
  if (C->dt_next < rem) { C->dt_use = C->dt_next; C->last = 0; }
  else { C->dt_use = rem; C->last = 1; }
}

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

template <int M, int NT>
int launch_step_t(const GfGeom& g, const GfView& v, double* pmass,
                  cudaStream_t st) {
  constexpr size_t bytes = Layout<M>::BYTES;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_patch_step<M, NT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess)
      return -2;
    attr = true;
  }
  k_patch_step<M, NT><<<v.npatch, NT, bytes, st>>>(g, v, pmass);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace

namespace gf {

int launch_patch_step_f64(const GfGeom& g, const GfView& v, double* pmass,
                          void* stream) {
  if (v.npatch <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g.M == 32) return launch_step_t<32, 512>(g, v, pmass, st);
  if (g.M == 16) return launch_step_t<16, 256>(g, v, pmass, st);
  return -1;
}

int launch_controller(const GfGeom& g, const GfView& v, const double* pmass,
                      int nscen, void* stream) {
  k_controller<<<nscen, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      g, v.ctl, v.scen, pmass);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
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
// cudaMalloc is not allowed (inside a captured region that must not grow the
// pool, or under an allocator that hands out only pre-registered buffers).
// They cannot create a geoflood context, because a context allocates its
// state.  geoflood_step_tiles_noalloc runs the same FP64 patch-step kernel on
// tiles the caller provides, and keeps the small scratch it needs (patch
// table, per-patch volume, the reduction cell of the CFL rate) in the static
// device array below, so the call allocates nothing.
//
// Limits and behaviour:
//   - at most GF_NOALLOC_MAX_PATCHES patches per call (the array holds
//     GF_NOALLOC_MAX_PATCHES * 24 bytes + 512 bytes, about 384 KiB, on every
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
  double pmass[GF_NOALLOC_MAX_PATCHES];
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

NoallocScratch* noalloc_scratch(int* rc) {
  static NoallocScratch* addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *rc = -2;
    return nullptr;
  }
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, gf_noalloc_scratch) != cudaSuccess || !p) {
      *rc = -2;
      return nullptr;
    }
    addr[dev] = static_cast<NoallocScratch*>(p);
  }
  *rc = 0;
  return addr[dev];
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
  const int lr = mx == 32 ? launch_step_t<32, 512>(G, V, S->pmass, st)
                          : launch_step_t<16, 256>(G, V, S->pmass, st);
  if (lr) return noalloc_fail(-2, "step_tiles_noalloc: step launch failed");
  if (cmax) {
    unsigned long long bits = 0;
    if (cudaMemcpyAsync(&bits, &S->ctl.cmax_bits, sizeof(bits),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return noalloc_fail(-2, "step_tiles_noalloc: reading the CFL rate failed");
    double v;
    std::memcpy(&v, &bits, sizeof(v));
    *cmax = v;
  }
  return 0;
}
