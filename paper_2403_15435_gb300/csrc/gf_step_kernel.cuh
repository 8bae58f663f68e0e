// The patch-step kernel, templated on the precision policy:
//   PrecF64 -- plain FP64 state (h, hu, hv) and bed b;
//   PrecF32 -- FP32 surface-deviation state (w = h + b - eta0, hu, hv) with
//              FP32 compensation terms for the update, bed b - eta0, exact
//              wet tests (FP32 with an FP64 tie-break) and FP64 volume sums.
//
// One CTA per patch.  The (M+4)^2 tile of the state and bed is staged in
// shared memory by 1D TMA bulk copies; then, in barrier-separated phases:
// every x-edge's augmented Riemann solve (Sec. 3.3), the MC-limited f-wave
// corrections (Sec. 3.2, Eq. wpa_update_corrections), the per-cell x
// increments and their transverse split along y (2D extension, leveque2002
// cited in Sec. 3.2), the same for y, the unsplit update, Manning friction
// (Eq. manning), and the per-patch CFL rate (warp-shuffle max) and volume.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "gf_internal.h"
#include "gf_solver.cuh"

namespace gfs {

struct PrecF64 {
  using R = double;
  static constexpr bool DEV = false;
};
struct PrecF32 {
  using R = float;
  static constexpr bool DEV = true;
};

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

// Bounded wait for the completion of the barrier's phase with the given
// parity; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned limit,
                                          unsigned parity = 0u) {
  for (unsigned it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], "
        "%2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Phases of the two staging barriers of a CTA that stages one tile after
// another (persistent variant): the parity each barrier completes next.
struct TmaPhase {
  unsigned b0, b1;
  bool init;
};

template <typename R>
__device__ __forceinline__ R warp_max(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const R w = __shfl_xor_sync(0xffffffffu, v, o);
    v = v > w ? v : w;
  }
  return v;
}

__device__ __forceinline__ double warp_sum_tree(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Writes that follow a new value (v0, v1, v2) of cell (gi, gj) of patch p
// (patch position (px, py); nxp x nyp patches on its level), other than the
// cell itself, into the next buffer: the ghost cells of the same-level
// neighbours (snb, one writer per ghost cell) that copy it, and the
// physical-boundary ghost cells of p or of those neighbours that mirror it
// (wall: reflected across the edge with the normal momentum negated;
// extrapolation: the edge cell copied into both ghost layers).  A boundary
// ghost whose mirror source is a neighbour's cell is written by that
// neighbour, so no ghost depends on another CTA's writes in the same launch.
template <typename R, int MP>
__device__ __forceinline__ void emit_edge(R* qnext, int p, int px, int py,
                                          int nxp, int nyp, const int* snb,
                                          const int* bc, bool push, int gi,
                                          int gj, R v0, R v1, R v2) {
  constexpr int TGW = MP + 2 * GF_NG, TG = TGW * TGW;
  if (gi >= GF_NG && gi < MP - GF_NG && gj >= GF_NG && gj < MP - GF_NG) return;
  auto target = [&](int q, int qx, int qy, int x, int y, bool self) {
    R* base = qnext + (size_t)q * 3 * TG;
    auto put = [&](int a, int b, R su, R sv) {
      R* d = base + (a + GF_NG) + (b + GF_NG) * TGW;
      d[0] = v0;
      d[TG] = su * v1;
      d[2 * TG] = sv * v2;
    };
    int xm[2], ym[2], nx = 0, ny = 0;
    R fx = R(1), fy = R(1);
    if (qx == 0 && (x == 0 || x == 1)) {
      if (bc[0] == 0) { xm[nx++] = -1 - x; fx = R(-1); }
      else if (x == 0) { xm[nx++] = -1; xm[nx++] = -2; }
    } else if (qx == nxp - 1 && (x == MP - 1 || x == MP - 2)) {
      if (bc[1] == 0) { xm[nx++] = 2 * MP - 1 - x; fx = R(-1); }
      else if (x == MP - 1) { xm[nx++] = MP; xm[nx++] = MP + 1; }
    }
    if (qy == 0 && (y == 0 || y == 1)) {
      if (bc[2] == 0) { ym[ny++] = -1 - y; fy = R(-1); }
      else if (y == 0) { ym[ny++] = -1; ym[ny++] = -2; }
    } else if (qy == nyp - 1 && (y == MP - 1 || y == MP - 2)) {
      if (bc[3] == 0) { ym[ny++] = 2 * MP - 1 - y; fy = R(-1); }
      else if (y == MP - 1) { ym[ny++] = MP; ym[ny++] = MP + 1; }
    }
    if (!self) put(x, y, R(1), R(1));
    for (int a = 0; a < nx; ++a) put(xm[a], y, fx, R(1));
    for (int b = 0; b < ny; ++b) put(x, ym[b], R(1), fy);
    for (int a = 0; a < nx; ++a)
      for (int b = 0; b < ny; ++b) put(xm[a], ym[b], fx, fy);
  };
  target(p, px, py, gi, gj, true);
  if (!push) return;
  const int dxs = gi < GF_NG ? -1 : (gi >= MP - GF_NG ? 1 : 0);
  const int dys = gj < GF_NG ? -1 : (gj >= MP - GF_NG ? 1 : 0);
  auto nb = [&](int r, int dx, int dy) {
    const int pn = snb[r];
    if (pn >= 0) target(pn, px + dx, py + dy, gi - dx * MP, gj - dy * MP, false);
  };
  if (dxs != 0) nb(dxs < 0 ? 0 : 1, dxs, 0);
  if (dys != 0) nb(dys < 0 ? 2 : 3, 0, dys);
  if (dxs != 0 && dys != 0) nb(4 + (dxs > 0 ? 1 : 0) + (dys > 0 ? 2 : 0), dxs, dys);
}

// Gauge samples of the state this launch starts from (the previous launch's
// accepted result, at time C->t), taken from the CTA's staged window: the
// window covers patch cells [ox - 2, ox + WM + 1]^2; a gauge whose stencil
// starts in sub-tile (ox, oy) is taken by that window's CTA.  mom = false:
// the momenta were not staged (a dry tile, where they are zero).
template <typename R, bool DEV, int MP, int WM>
__device__ __forceinline__ void sample_gauges(const GfView& V, int scen, const GfCtl* C,
                                              int p, int ox, int oy, const R* s0,
                                              const R* shu, const R* shv, const R* sb,
                                              bool mom) {
  constexpr int TGW = MP + 2 * GF_NG, WW = WM + 2 * GF_NG;
  const GfScenario& S = V.scen[scen];
  for (int g = threadIdx.x; g < S.ngauge; g += blockDim.x) {
    const GfGaugeRef r = S.gref[g];
    if (r.p != p) continue;
    const int i0 = r.c % TGW - GF_NG, j0 = r.c / TGW - GF_NG;
    const int ic = i0 < 0 ? 0 : i0, jc = j0 < 0 ? 0 : j0;
    if ((ic / WM) * WM != ox || (jc / WM) * WM != oy) continue;
    const int c = (i0 - ox + GF_NG) + (j0 - oy + GF_NG) * WW;
    const int cs[4] = {c, c + 1, c + WW, c + WW + 1};
    double a[4][4];  // h, hu, hv, h + b per stencil cell
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double b = (double)sb[cs[k]];
      const double h = DEV ? (double)s0[cs[k]] - b : (double)s0[cs[k]];
      a[k][0] = h;
      a[k][1] = mom ? (double)shu[cs[k]] : 0.0;
      a[k][2] = mom ? (double)shv[cs[k]] : 0.0;
      a[k][3] = h + b;
    }
    double v[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) v[f] = gf_bilinear(a[0][f], a[1][f], a[2][f], a[3][f], r.ax, r.ay);
    double* o = S.gout + 5 * g;
    const double t = C->t;
    o[0] = t;
    o[1] = v[0];
    o[2] = v[1];
    o[3] = v[2];
    o[4] = v[3] + (DEV ? S.eta0 : 0.0);
    if (S.garr[g] < 0.0 && v[0] > 0.01) S.garr[g] = t;
  }
}

// Shared-memory layout of one CTA.  DS = dimensional splitting: the x sweep
// covers every row of the window (two ghost rows each side) and there are no
// transverse-flux arrays.
template <class P, int M, bool DS = false>
struct Layout {
  using R = typename P::R;
  static constexpr int T = M + 2 * GF_NG;
  static constexpr int TT = T * T;
  // most lines in one sweep: one ghost line each side (unsplit) or two
  static constexpr int NR = DS ? M + 4 : M + 2;
  static constexpr int NE = M + 3;  // edges per line, a in [-1, M+1]
  static constexpr int NEDGE = NR * NE;
  static constexpr int NLIM = NR * (M + 1);   // edges a in [0, M] per line
  static constexpr int NCELL = M * NR;        // cells of the increments
  static constexpr int NF = P::DEV ? 5 : 4;   // tile fields (+ depth)
  static constexpr size_t TRB = DS ? 0 : sizeof(R) * 3 * M * (M + 1);
  // byte offsets in dynamic shared memory
  static constexpr size_t OFF_W = sizeof(R) * NF * TT;
  static constexpr size_t OFF_F = OFF_W + sizeof(R) * 12 * NEDGE;
  static constexpr size_t OFF_G = OFF_F + TRB;
  static constexpr size_t OFF_RED = align16(OFF_G + TRB);
  static constexpr size_t OFF_NB = OFF_RED + sizeof(double) * 64;  // 8 ints
  static constexpr size_t OFF_WET = OFF_NB + 32;
  static constexpr size_t OFF_BAR = align16(OFF_WET + (P::DEV ? TT : 0));
  static constexpr size_t BYTES = OFF_BAR + 16;
};

template <int M>
__device__ __forceinline__ int tix(int i, int j) {
  return (i + GF_NG) + (j + GF_NG) * (M + 2 * GF_NG);
}

// Increment cell of item k in a sweep over NRL lines: items below M*M are
// interior cells in the fixed order (i = k % M, j = k / M) used by the final
// update, so each thread owns the same cells in both sweeps; then the ghost
// lines before the interior (from line L0 on) and those after it.  a is the
// position along the sweep, line the one across.
template <int M, int NRL, int L0>
__device__ __forceinline__ void cell_item(int k, int dir, int& a, int& line) {
  if (k < M * M) {
    const int i = k % M, j = k / M;
    a = dir == 0 ? i : j;
    line = dir == 0 ? j : i;
  } else {
    constexpr int HALF = (NRL - M) / 2;
    const int r = k - M * M, gl = r / M;
    a = r % M;
    line = gl < HALF ? L0 + gl : M + (gl - HALF);
  }
}

// M is the side of the sub-tile this CTA updates, MP the side of the patch:
// a patch of MP x MP cells is covered by (MP/M)^2 CTAs, each staging its
// (M+4)^2 window (interior + two ghost layers, taken from the patch tile,
// whose ghosts are filled) and writing its M x M cells.  Every cell's update
// depends only on its two-cell neighbourhood, so the result does not depend
// on M.
//
// Scheme variants (Sec. 3.2): G.first_order drops the limited corrections,
// G.no_transverse the transverse terms; DS (dimensional splitting) takes the
// x sweep on every row of the window, updates the interior columns of all
// rows in shared memory (negative depths reset, dry momenta zeroed), and
// takes the y sweep on that state, without transverse terms.
template <class P, int MP, int M, int NT, bool DS = false>
__device__ __forceinline__ int patch_body(const GfGeom& G, const GfView& V,
                                          unsigned char* smraw, const int p,
                                          const int sub, TmaPhase* tp = nullptr,
                                          bool* wrote = nullptr) {
  using R = typename P::R;
  constexpr bool DEV = P::DEV;
  using Lo = Layout<P, M, DS>;
  constexpr int TT = Lo::TT, NE = Lo::NE, NEDGE = Lo::NEDGE;
  constexpr int TGW = MP + 2 * GF_NG, TG = TGW * TGW;  // patch tile
  constexpr int NS1 = MP / M, NSUB = NS1 * NS1;
  constexpr int RL = (Lo::NLIM + NT - 1) / NT;    // limiter items per thread
  constexpr int RC = (M * M + NT - 1) / NT;       // interior cells per thread
  constexpr int RX = (Lo::NCELL + NT - 1) / NT;   // increment cells per thread

  const int unit = p * NSUB + sub;  // CTA work unit: volume slot, same[] flag
  const bool has_gauge = V.gflag != nullptr && V.gflag[p] != 0;
  const int ox = (sub % NS1) * M, oy = (sub / NS1) * M;
  const GfPatch Pt = V.patch[p];
  GfCtl* C = V.ctl + Pt.scen;
  // global tile index of local cell (i, j), and interior index in the patch
  auto gix = [&](int i, int j) { return (ox + i + GF_NG) + (oy + j + GF_NG) * TGW; };
  auto pix = [&](int i, int j) { return (ox + i) + (oy + j) * MP; };

  R* s0 = reinterpret_cast<R*>(smraw);  // h (FP64) or w (deviation form)
  R* shu = s0 + TT;
  R* shv = s0 + 2 * TT;
  R* sb = s0 + 3 * TT;
  R* sdep = DEV ? s0 + 4 * TT : s0;     // depth
  R* W = reinterpret_cast<R*>(smraw + Lo::OFF_W);
  R* Ftr = reinterpret_cast<R*>(smraw + Lo::OFF_F);  // [row j][edge 0..M][3]
  R* Gtr = reinterpret_cast<R*>(smraw + Lo::OFF_G);  // [column i][edge][3]
  double* red = reinterpret_cast<double*>(smraw + Lo::OFF_RED);
  unsigned char* swet = smraw + Lo::OFF_WET;
  int* snb = reinterpret_cast<int*>(smraw + Lo::OFF_NB);  // same-level neighbours
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + Lo::OFF_BAR);

  const int tid = threadIdx.x;
  // level subcycling: this level's period in fine substeps, its buffer
  // (ceil(sub_k / per) steps taken in the macro step so far) and its time
  // step (the macro step's share for the level)
  const bool subc = G.subcycle != 0;
  const int per = subc ? 1 << (G.maxlevel - Pt.level) : 1;
  const int cur = subc ? C->cur ^ ((C->sub_k / per) & 1) : C->cur;
  const double dtp = subc ? (C->dt_use / (double)G.sub_K) * (double)per : C->dt_use;
  const R* qs;
  R* qd;
  const R* bs;
  if constexpr (DEV) {
    qs = V.qf[cur] + (size_t)p * 3 * TG;
    qd = V.qf[cur ^ 1] + (size_t)p * 3 * TG;
    bs = V.bf + (size_t)p * TG;
  } else {
    qs = V.q[cur] + (size_t)p * 3 * TG;
    qd = V.q[cur ^ 1] + (size_t)p * 3 * TG;
    bs = V.b + (size_t)p * TG;
  }

  // A tile whose interior is the same in both buffers (it was dry and copied)
  // needs only its surface and bed to find out whether it is still dry; its
  // momenta are fetched only if water has arrived.
  const bool same_in = V.same != nullptr && V.same[unit] != 0;
  bool mom_issued = false;
  // staging barrier phases (a CTA that stages several tiles keeps them in tp)
  const bool fresh = tp == nullptr || !tp->init;
  const unsigned ph0 = tp ? tp->b0 : 0u, ph1 = tp ? tp->b1 : 0u;
  if constexpr (M == MP) {
    // whole patch: its four contiguous fields arrive by 1D TMA bulk copies,
    // surface and bed on bar[0], the momenta on bar[1]
    if (tid == 0) {
      if (fresh) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
      }
      mbar_expect_tx(bar, 2u * TT * sizeof(R));
      bulk_g2s(s0, qs, TT * sizeof(R), bar);
      bulk_g2s(sb, bs, TT * sizeof(R), bar);
      if (!same_in) {
        mbar_expect_tx(bar + 1, 2u * TT * sizeof(R));
        bulk_g2s(shu, qs + TT, TT * sizeof(R), bar + 1);
        bulk_g2s(shv, qs + 2 * TT, TT * sizeof(R), bar + 1);
      }
    }
    mom_issued = !same_in;
    if (tp) tp->init = true;
    __syncthreads();
    // every wait is bounded; the decision to give up is taken by the whole CTA
    if (!__syncthreads_and(mbar_wait(bar, GF_SPIN_LIMIT, ph0) ? 1 : 0)) {
      if (tid == 0) C->status = -7;  // GEOFLOOD_ERR_TIMEOUT
      mbar_wait(bar, GF_SPIN_LIMIT, ph0);
      if (mom_issued) mbar_wait(bar + 1, GF_SPIN_LIMIT, ph1);
      __syncthreads();
      return -1;
    }
    if (tp) tp->b0 ^= 1u;
  } else {
    // sub-tile: the (M+4)^2 window of each field, row segments read with
    // consecutive threads on consecutive addresses
    for (int k = tid; k < TT; k += NT) {
      const int li = k % Lo::T, lj = k / Lo::T;
      const int g = (ox + li) + (oy + lj) * TGW;
      s0[k] = qs[g];
      shu[k] = qs[TG + g];
      shv[k] = qs[2 * TG + g];
      sb[k] = bs[g];
    }
  }

  // per-patch scalars: computed once by thread 0 (FP64 divisions are slow
  // on this part, so no thread repeats them) and broadcast through shared
  // memory
  double* scal = red + 48;  // dx, dy, nux, nuy, then the R-typed copies
  R* rscal = reinterpret_cast<R*>(red + 52);  // g, drytol, nux, nuy, n, dt
  float* fscal = reinterpret_cast<float*>(red + 60);  // drytol, margin
  if (tid == 0) {
    if constexpr (DEV) {
      // FP32 from the host's per-level tables: one conversion per patch
      const float dtf32 = (float)dtp;
      rscal[0] = G.gf;
      rscal[1] = G.drytolf;
      rscal[2] = dtf32 * G.inv_dxf[Pt.level];
      rscal[3] = dtf32 * G.inv_dyf[Pt.level];
      rscal[4] = V.scen[Pt.scen].manning_f;
      rscal[5] = dtf32;
      fscal[0] = G.drytolf;
      fscal[1] = G.marginf;
    } else {
      const long long NXL = (long long)G.mi * MP << Pt.level;
      const long long NYL = (long long)G.mj * MP << Pt.level;
      const double dx0 = (G.xupper - G.xlower) / (double)NXL;
      const double dy0 = (G.yupper - G.ylower) / (double)NYL;
      scal[0] = dx0;
      scal[1] = dy0;
      scal[2] = dtp / dx0;
      scal[3] = dtp / dy0;
      rscal[0] = (R)G.g;
      rscal[1] = (R)G.drytol;
      rscal[2] = (R)scal[2];
      rscal[3] = (R)scal[3];
      rscal[4] = (R)V.scen[Pt.scen].manning_n;
      rscal[5] = (R)dtp;
    }
  }
  const bool push = V.push != 0 && V.nbr != nullptr;
  if (push && tid < 8) snb[tid] = V.nbr[(size_t)p * 8 + tid];
  const double drytol = G.drytol;
  R smx = R(0), smy = R(0);

  __syncthreads();
  const R g = rscal[0], rdry = rscal[1], nux = rscal[2], nuy = rscal[3];
  const R dtr = rscal[5];
  const float dtf = fscal[0], margin = fscal[1];

  // Per-cell depth and exact wet flag (deviation form), and whether the
  // tile holds any wet cell at all.  A tile whose interior is unchanged and
  // was dry (same_in) can only have taken water into its ghost cells, so the
  // interior is examined only if they hold some.
  constexpr int NRING = TT - M * M;
  auto ring_cell = [&](int k) {  // k-th ghost cell of the window
    const int band = 2 * Lo::T;
    if (k < band) return k;                                 // two bottom rows
    if (k < 2 * band) return (M + GF_NG) * Lo::T + (k - band);  // two top rows
    const int r = k - 2 * band, j = r / 4, c = r % 4;
    return (j + GF_NG) * Lo::T + (c < 2 ? c : M + c);       // side columns
  };
  auto examine = [&](int k) -> int {
    if constexpr (DEV) {
      const float w = s0[k], b = sb[k];
      sdep[k] = w - b;
      const bool wt = gfk::wet_dev(w, b, drytol, dtf, margin);
      swet[k] = wt ? 1 : 0;
      return wt ? 1 : 0;
    } else {
      return s0[k] > rdry ? 1 : 0;
    }
  };
  int anywet = 0;
  if (same_in) {
    for (int k = tid; k < NRING; k += NT) anywet |= examine(ring_cell(k));
    anywet = __syncthreads_or(anywet);
    if (anywet) {
      for (int k = tid; k < M * M; k += NT)
        examine((k % M + GF_NG) + (k / M + GF_NG) * Lo::T);
      __syncthreads();  // the sweeps read every thread's depths and flags
    }
  } else {
    for (int k = tid; k < TT; k += NT) anywet |= examine(k);
    anywet = __syncthreads_or(anywet);
  }
  if constexpr (M == MP) {
    // the momenta: requested now if water arrived at a copied dry tile, and
    // waited for whenever they were requested
    if (anywet && !mom_issued) {
      if (tid == 0) {
        mbar_expect_tx(bar + 1, 2u * TT * sizeof(R));
        bulk_g2s(shu, qs + TT, TT * sizeof(R), bar + 1);
        bulk_g2s(shv, qs + 2 * TT, TT * sizeof(R), bar + 1);
      }
      mom_issued = true;
    }
    if (mom_issued && !__syncthreads_and(mbar_wait(bar + 1, GF_SPIN_LIMIT, ph1) ? 1 : 0)) {
      if (tid == 0) C->status = -7;  // GEOFLOOD_ERR_TIMEOUT
      mbar_wait(bar + 1, GF_SPIN_LIMIT, ph1);
      __syncthreads();
      return -1;
    }
    if (mom_issued && tp) tp->b1 ^= 1u;
  }
  // a dry tile whose interior is already the same in both buffers writes
  // nothing (its update is the identity on the surface, zero momenta)
  const bool skip_writes = same_in && !anywet;
  if (V.same != nullptr && tid == 0) V.same[unit] = anywet ? 0 : 1;
  if (has_gauge && C->accepted && (!subc || C->sub_k == 0))
    sample_gauges<R, DEV, MP, M>(V, Pt.scen, C, p, ox, oy, s0, shu, shv, sb,
                                 M != MP || mom_issued);
  if (skip_writes) {
    // nothing changes: no writes, no waves
    if (wrote) *wrote = false;
    return 0;
  }
  auto wetc = [&](int c) -> bool {
    if constexpr (DEV) return swet[c] != 0;
    else return s0[c] > rdry;
  };
  auto surf = [&](int c) -> R {
    if constexpr (DEV) return s0[c];
    else return s0[c] + sb[c];
  };

  R X[RC][3];   // nu_x * dQx of owned interior cells
  R Y[RC][3];   // nu_y * dQy
  // dimensional splitting, deviation form: compensation terms of the
  // intermediate state of owned interior cells
  float LO1[DS && DEV ? RC : 1][3];
  const float* los = nullptr;
  float* lod = nullptr;
  if constexpr (DEV) {
    los = V.lof[cur] + (size_t)p * 3 * MP * MP;
    lod = V.lof[cur ^ 1] + (size_t)p * 3 * MP * MP;
  }
  const bool corr = G.first_order == 0;              // limited corrections
  const bool trv = !DS && G.no_transverse == 0;      // transverse terms
  double clipd = 0.0;
  float clipf = 0.0f;  // deviation form: clipped depth, FP32 per thread
  unsigned nclip = 0, nwet = 0;

  // A tile without a wet cell (ghosts included) has only dry-dry edges: every
  // wave, correction and transverse term is zero and the update reduces to
  // zeroing the momenta of the (dry) cells, which the dry branch below does
  // without the sweeps; the results are identical.
  // one sweep; the direction is a compile-time constant so that the index
  // arithmetic of the two sweeps is resolved statically
  auto sweep = [&](auto dirc) {
    constexpr int dir = decltype(dirc)::value;
    // lines swept: -1..M (unsplit), -2..M+1 (split, x), 0..M-1 (split, y)
    constexpr int NRL = DS ? (dir == 0 ? M + 4 : M) : M + 2;
    constexpr int L0 = DS ? (dir == 0 ? -2 : 0) : -1;
    const R* sn = dir == 0 ? shu : shv;  // normal momentum
    const R* st = dir == 0 ? shv : shu;  // transverse momentum
    const R nu = dir == 0 ? nux : nuy;
    // phase 1: Riemann solves on the lines, edges -1..M+1.  Consecutive
    // threads take consecutive cells of a row: along the row in the x sweep,
    // across the lines in the y sweep (a column walk would make every tile
    // load a 4-way shared-memory bank conflict); each edge's wave planes
    // keep their place, so the work is the same whichever thread does it
    for (int k = tid; k < NRL * NE; k += NT) {
      const int line = (dir == 0 ? k / NE : k % NRL) + L0;
      const int a = (dir == 0 ? k % NE : k / NRL) - 1;
      const int cl = dir == 0 ? tix<M>(a - 1, line) : tix<M>(line, a - 1);
      const int cr = dir == 0 ? tix<M>(a, line) : tix<M>(line, a);
      R Z[9], S[3];
      gfk::riemann<R, DEV>(
          gfk::Side<R>{sdep[cl], sn[cl], st[cl], sb[cl], s0[cl], wetc(cl)},
          gfk::Side<R>{sdep[cr], sn[cr], st[cr], sb[cr], s0[cr], wetc(cr)}, g,
          rdry, Z, S);
      // waves in planes: component q of edge e at W[q * NEDGE + e], e the
      // edge's place (line, a) in the sweep
      R* w = W + ((line - L0) * NE + a + 1);
#pragma unroll
      for (int q = 0; q < 9; ++q)
        if (!(DEV && q == 3)) w[q * NEDGE] = Z[q];  // FP32: Z[3] is zero, not read
      w[9 * NEDGE] = S[0];
      w[10 * NEDGE] = S[1];
      w[11 * NEDGE] = S[2];
    }
    __syncthreads();
    // phase 2: fluctuations and limited corrections on edges 0..M
    R AMr[RL][3], APr[RL][3], FFr[RL][3];
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int k = tid + r * NT;
      if (k < NRL * (M + 1)) {
        const int line = k / (M + 1) + L0, a = k % (M + 1);
        const int e = (line - L0) * NE + a + 1;
        const R* w = W + e;
        const int cl = dir == 0 ? tix<M>(a - 1, line) : tix<M>(line, a - 1);
        const int cr = dir == 0 ? tix<M>(a, line) : tix<M>(line, a);
        const bool wet = corr && wetc(cl) && wetc(cr);
        gfk::edge_fluxes<R, NEDGE, DEV>(w, w + 9 * NEDGE, w - 1, w + 1, nu, wet,
                                        AMr[r], APr[r], FFr[r]);
        if (line >= 0 && line < M) {
          R m = R(0);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const R sq = w[(9 + q) * NEDGE];
            const R as = sq > R(0) ? sq : -sq;
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
      if (k < NRL * (M + 1)) {
        const int line = k / (M + 1) + L0, a = k % (M + 1);
        R* w = W + ((line - L0) * NE + a + 1);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          w[q * NEDGE] = AMr[r][q];
          w[(3 + q) * NEDGE] = APr[r][q];
          w[(6 + q) * NEDGE] = FFr[r][q];
        }
      }
    }
    __syncthreads();
    // phase 3: per-cell increments and their transverse split (unsplit),
    // or the intermediate state of the x sweep (split)
    R* Tr = dir == 0 ? Gtr : Ftr;
    R MIr[RX][3];
#pragma unroll
    for (int r = 0; r < RX; ++r) {
      const int k = tid + r * NT;
      if (k < M * NRL) {
        int a, line;  // a: position along the sweep, line: across
        cell_item<M, NRL, L0>(k, dir, a, line);
        const R* wl = W + ((line - L0) * NE + a + 1);  // edge a
        const R* wr = wl + 1;                           // edge a+1
        R d[3];  // frame: mass, normal (sweep) momentum, transverse
#pragma unroll
        for (int q = 0; q < 3; ++q)
          d[q] = (wl[(3 + q) * NEDGE] + wr[q * NEDGE]) +
                 (wr[(6 + q) * NEDGE] - wl[(6 + q) * NEDGE]);
        if (r < RC && k < M * M) {
          // store nu * dQ in (h, hu, hv) order
          if (dir == 0) {
            X[r][0] = nu * d[0]; X[r][1] = nu * d[1]; X[r][2] = nu * d[2];
          } else {
            Y[r][0] = nu * d[0]; Y[r][1] = nu * d[2]; Y[r][2] = nu * d[1];
          }
        }
        if constexpr (DS) {
          if constexpr (dir == 0) {
            // intermediate state of cell (a, line) in place: every read of
            // the window in this sweep is behind the barriers above
            const int c = tix<M>(a, line);
            const bool inner = k < M * M;
            const R xs[3] = {nu * d[0], nu * d[1], nu * d[2]};
            const R q[3] = {s0[c], shu[c], shv[c]};
            R o[3];
            if (inner) nwet += wetc(c) ? 1u : 0u;
            if constexpr (!DEV) {
#pragma unroll
              for (int f = 0; f < 3; ++f) o[f] = q[f] - xs[f];
              if (o[0] < R(0)) {
                if (inner) { clipd -= o[0]; ++nclip; }
                o[0] = R(0);
              }
              if (o[0] <= rdry) { o[1] = R(0); o[2] = R(0); }
            } else {
              const int kp = pix(a, line);
              float lo[3];
#pragma unroll
              for (int f = 0; f < 3; ++f) {
                const float x = (inner ? los[f * MP * MP + kp] : 0.0f) - xs[f];
                const float s = q[f] + x;
                const float bb = s - q[f];
                lo[f] = (q[f] - (s - bb)) + (x - bb);
                o[f] = s;
              }
              const float bc = sb[c];
              if (o[0] < bc) {
                if (inner) { clipf += bc - o[0]; ++nclip; }
                o[0] = bc;
                lo[0] = 0.0f;
              }
              const bool wnew = gfk::wet_dev(o[0], bc, drytol, dtf, margin);
              if (!wnew) { o[1] = 0.0f; o[2] = 0.0f; lo[1] = 0.0f; lo[2] = 0.0f; }
              sdep[c] = o[0] - bc;
              swet[c] = wnew ? 1 : 0;
              if (inner && r < RC) {
                LO1[r][0] = lo[0]; LO1[r][1] = lo[1]; LO1[r][2] = lo[2];
              }
            }
            s0[c] = o[0];
            shu[c] = o[1];
            shv[c] = o[2];
          }
          continue;
        }
        if (!trv) continue;
        // split along the other direction: in that frame the "along"
        // momentum is this sweep's transverse momentum
        const int ci = dir == 0 ? tix<M>(a, line) : tix<M>(line, a);
        const int cm = dir == 0 ? tix<M>(a, line - 1) : tix<M>(line - 1, a);
        const int cp = dir == 0 ? tix<M>(a, line + 1) : tix<M>(line + 1, a);
        const R dd[3] = {d[0], d[2], d[1]};
        R pl[3], mi[3];
        gfk::tsplit<R>(sdep[ci], st[ci], sn[ci], surf(ci), wetc(ci), wetc(cm),
                       sb[cm], wetc(cp), sb[cp], dd, g, pl, mi);
        // back to (h, hu, hv): frame (mass, along = st, other = sn)
        const R plh[3] = {pl[0], dir == 0 ? pl[2] : pl[1],
                          dir == 0 ? pl[1] : pl[2]};
        MIr[r][0] = mi[0];
        MIr[r][1] = dir == 0 ? mi[2] : mi[1];
        MIr[r][2] = dir == 0 ? mi[1] : mi[2];
        if (line + 1 <= M) {
          R* o = Tr + 3 * (a * (M + 1) + line + 1);
          o[0] = plh[0]; o[1] = plh[1]; o[2] = plh[2];
        }
      }
    }
    __syncthreads();
    if (DS || !trv) return;
    const R nut = dir == 0 ? nux : nuy;
#pragma unroll
    for (int r = 0; r < RX; ++r) {
      const int k = tid + r * NT;
      if (k < M * NRL) {
        int a, line;
        cell_item<M, NRL, L0>(k, dir, a, line);
        if (line >= 0) {
          R* o = Tr + 3 * (a * (M + 1) + line);
#pragma unroll
          for (int q = 0; q < 3; ++q) o[q] = R(-0.5) * nut * (o[q] + MIr[r][q]);
        }
      }
    }
    __syncthreads();
  };
  if (anywet) {
    sweep(std::integral_constant<int, 0>{});
    sweep(std::integral_constant<int, 1>{});
  }

  // New values of a cell near the patch edge also go to the ghost cells that
  // copy or mirror it (same-level neighbours, physical boundaries).
  R* qnext;
  if constexpr (DEV) qnext = V.qf[cur ^ 1];
  else qnext = V.q[cur ^ 1];
  const int nxp = G.mi << Pt.level, nyp = G.mj << Pt.level;
  auto push_edge = [&](int gi, int gj, R v0, R v1, R v2) {
    emit_edge<R, MP>(qnext, p, Pt.px, Pt.py, nxp, nyp, snb, G.bc, push, gi, gj, v0, v1, v2);
  };

  // ------------------------------------------------ update, friction, out
  const R mn = rscal[4];
  bool bad = false;
  // the compensation terms of every owned cell requested at once, so that
  // their global loads overlap instead of one wait per cell
  float lpre[DEV && !DS ? RC : 1][3];
  if constexpr (DEV && !DS) {
#pragma unroll
    for (int r = 0; r < RC; ++r) {
      const int k = tid + r * NT;
      const int kp = k < M * M ? pix(k % M, k / M) : 0;
#pragma unroll
      for (int f = 0; f < 3; ++f)
        lpre[r][f] = (anywet && k < M * M) ? los[f * MP * MP + kp] : 0.0f;
    }
  }
#pragma unroll
  for (int r = 0; r < RC; ++r) {
    const int k = tid + r * NT;
    if (k >= M * M) continue;
    const int i = k % M, j = k / M;
    const int c = tix<M>(i, j);
    const int cg = gix(i, j), kp = pix(i, j);
    if (!anywet) {
      if (!skip_writes) {
        qd[cg] = s0[c];
        qd[TG + cg] = R(0);
        qd[2 * TG + cg] = R(0);
        push_edge(ox + i, oy + j, s0[c], R(0), R(0));
        if constexpr (DEV) {
          lod[kp] = los[kp];
          lod[MP * MP + kp] = 0.0f;
          lod[2 * MP * MP + kp] = 0.0f;
        }
      }
      continue;
    }
    const R q[3] = {s0[c], shu[c], shv[c]};  // split: the intermediate state
    if (!DS) nwet += wetc(c) ? 1u : 0u;
    R o[3];
    if constexpr (!DEV) {
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const R fl = DS ? Y[r][f] : X[r][f] + Y[r][f];
        const R* fa = Ftr + 3 * (j * (M + 1) + i);
        const R* ga = Gtr + 3 * (i * (M + 1) + j);
        const R tf = trv ? nux * (fa[3 + f] - fa[f]) + nuy * (ga[3 + f] - ga[f]) : R(0);
        o[f] = (q[f] - fl) - tf;
      }
      if (o[0] < R(0)) { clipd -= o[0]; o[0] = R(0); ++nclip; }
      if (mn > R(0) && o[0] > rdry) {
        const R u = o[1] / o[0], v = o[2] / o[0];
        const R sp = sqrt(u * u + v * v);
        const R D = g * mn * mn * sp / (o[0] * cbrt(o[0]));
        const R den = R(1) + dtr * D;
        o[1] = o[1] / den;
        o[2] = o[2] / den;
      }
      if (o[0] <= rdry) { o[1] = R(0); o[2] = R(0); }
    } else {
      // compensated update: (hi + lo) - fl - tf, hi rounded, lo the error
      float lo[3];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const float fl = DS ? Y[r][f] : X[r][f] + Y[r][f];
        const float* fa = Ftr + 3 * (j * (M + 1) + i);
        const float* ga = Gtr + 3 * (i * (M + 1) + j);
        const float tf =
            trv ? nux * (fa[3 + f] - fa[f]) + nuy * (ga[3 + f] - ga[f]) : 0.0f;
        const float lin = DS ? LO1[DS && DEV ? r : 0][f] : lpre[DS ? 0 : r][f];
        const float x = (lin - fl) - tf;
        const float s = q[f] + x;
        const float bb = s - q[f];
        lo[f] = (q[f] - (s - bb)) + (x - bb);
        o[f] = s;
      }
      const float bc = sb[c];
      if (o[0] < bc) {  // negative depth: reset to a dry bed
        clipf += bc - o[0];
        o[0] = bc;
        lo[0] = 0.0f;
        ++nclip;
      }
      const bool wnew = gfk::wet_dev(o[0], bc, drytol, dtf, margin);
      if (mn > 0.0f && wnew) {
        // approximate reciprocals and h^(-4/3) by the fast power (relative
        // error about 1e-6, far inside the FP32 path's tolerance); products
        // rounded on their own, so every kernel variant rounds them alike
        const float h = o[0] - bc;
        const float rh = __fdividef(1.0f, h);
        const float u = __fmul_rn(o[1], rh), v = __fmul_rn(o[2], rh);
        const float sp = sqrtf(u * u + v * v);
        const float D = g * mn * mn * sp * __powf(h, -4.0f / 3.0f);
        const float rden = __fdividef(1.0f, 1.0f + dtr * D);
        o[1] = __fmul_rn(o[1], rden);
        o[2] = __fmul_rn(o[2], rden);
        lo[1] = __fmul_rn(lo[1], rden);
        lo[2] = __fmul_rn(lo[2], rden);
      }
      if (!wnew) { o[1] = 0.0f; o[2] = 0.0f; lo[1] = 0.0f; lo[2] = 0.0f; }
#pragma unroll
      for (int f = 0; f < 3; ++f) lod[f * MP * MP + kp] = lo[f];
    }
    bad |= !(isfinite(o[0]) && isfinite(o[1]) && isfinite(o[2]));
    qd[cg] = o[0];
    qd[TG + cg] = o[1];
    qd[2 * TG + cg] = o[2];
    push_edge(ox + i, oy + j, o[0], o[1], o[2]);
  }
  // block reductions: CFL rate (max) and wet-cell count, one atomic of each
  // per CTA
  const int lane = tid & 31, wid = tid >> 5;
  constexpr int NW = NT / 32;
  static_assert(NW <= 32, "one warp reduces the per-warp partials");
  // the partials fit below the broadcast scalars at red + 48
  static_assert(DEV ? 3 * NW <= 96 : 3 * NW <= 48, "reduction area");
  smx = warp_max(smx);
  smy = warp_max(smy);
  nwet = __reduce_add_sync(0xffffffffu, nwet);
  if constexpr (DEV) {
    float* redf = reinterpret_cast<float*>(red);
    unsigned* redu = reinterpret_cast<unsigned*>(redf + 2 * NW);
    if (lane == 0) {
      redf[wid] = smx;
      redf[NW + wid] = smy;
      redu[wid] = nwet;
    }
    __syncthreads();
    if (wid == 0) {
      float mx = lane < NW ? redf[lane] : 0.0f;
      float my = lane < NW ? redf[NW + lane] : 0.0f;
      const unsigned nw = __reduce_add_sync(0xffffffffu, lane < NW ? redu[lane] : 0u);
      mx = warp_max(mx);
      my = warp_max(my);
      if (lane == 0) {
        const float cx = mx * G.inv_dxf[Pt.level], cy = my * G.inv_dyf[Pt.level];
        double cm = (double)(cx > cy ? cx : cy);
        if (subc) cm = cm * (double)per / (double)G.sub_K;  // cmax / n_L
        atomicMax(&C->cmax_bits, (unsigned long long)__double_as_longlong(cm));
        if (nw) atomicAdd(&C->wet_updates, (unsigned long long)nw);
      }
    }
    if (nclip) {
      atomicAdd(&C->step_nclip, (unsigned long long)nclip);
      atomicAdd(&C->step_clipvol, (double)clipf * G.areal[Pt.level]);
    }
  } else {
    const double dx = scal[0], dy = scal[1];
    unsigned* redu = reinterpret_cast<unsigned*>(red + 2 * NW);
    if (lane == 0) {
      red[wid] = (double)smx;
      red[NW + wid] = (double)smy;
      redu[wid] = nwet;
    }
    __syncthreads();
    if (tid == 0) {
      double mx = 0.0, my = 0.0;
      unsigned nw = 0u;
      for (int w = 0; w < NW; ++w) {
        mx = red[w] > mx ? red[w] : mx;
        my = red[NW + w] > my ? red[NW + w] : my;
        nw += redu[w];
      }
      const double cx = mx / dx, cy = my / dy;
      double cm = cx > cy ? cx : cy;
      if (subc) cm = cm * (double)per / (double)G.sub_K;  // cmax / n_L
      atomicMax(&C->cmax_bits, (unsigned long long)__double_as_longlong(cm));
      if (nw) atomicAdd(&C->wet_updates, (unsigned long long)nw);
    }
    if (nclip) {
      atomicAdd(&C->step_nclip, (unsigned long long)nclip);
      atomicAdd(&C->step_clipvol, clipd * (dx * dy));
    }
  }
  if (bad) C->nonfinite = 1;
  return anywet;
}

// Whole-patch pass of the adaptive variant for a patch expected to be dry:
// one CTA stages the surface and bed of the MP x MP tile (two TMA bulk
// copies), decides whether any cell of the tile holds water and, if none
// does, applies the dry update (copy the surface, zero the momenta) to the
// whole patch.  Returns 1 if the tile held water (the caller then runs the
// M x M sub-tiles one after the other; the result does not depend on the
// split).
template <class P, int MP, int M, int NT>
__device__ __forceinline__ int whole_tile(const GfGeom& G, const GfView& V,
                                          unsigned char* smraw, const int p) {
  using R = typename P::R;
  constexpr bool DEV = P::DEV;
  using Lo = Layout<P, M>;
  constexpr int TGW = MP + 2 * GF_NG, TG = TGW * TGW;
  constexpr int NS1 = MP / M, NSUB = NS1 * NS1;
  static_assert(2 * TG * sizeof(R) <= Lo::OFF_RED, "tile staging fits the sub-tile layout");
  const int tid = threadIdx.x;
  const GfPatch Pt = V.patch[p];
  GfCtl* C = V.ctl + Pt.scen;
  const int cur = C->cur;
  R* s0 = reinterpret_cast<R*>(smraw);
  R* sb = s0 + TG;
  int* snb = reinterpret_cast<int*>(smraw + Lo::OFF_NB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + Lo::OFF_BAR);
  const R* qs;
  R* qd;
  R* qnext;
  const R* bs;
  if constexpr (DEV) {
    qs = V.qf[cur] + (size_t)p * 3 * TG;
    qnext = V.qf[cur ^ 1];
    bs = V.bf + (size_t)p * TG;
  } else {
    qs = V.q[cur] + (size_t)p * 3 * TG;
    qnext = V.q[cur ^ 1];
    bs = V.b + (size_t)p * TG;
  }
  qd = qnext + (size_t)p * 3 * TG;
  bool same_in = V.same != nullptr;
  if (same_in)
    for (int u = 0; u < NSUB; ++u) same_in = same_in && V.same[p * NSUB + u] != 0;
  const bool push = V.push != 0 && V.nbr != nullptr;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, 2u * TG * sizeof(R));
    bulk_g2s(s0, qs, TG * sizeof(R), bar);
    bulk_g2s(sb, bs, TG * sizeof(R), bar);
  }
  if (push && tid < 8) snb[tid] = V.nbr[(size_t)p * 8 + tid];
  __syncthreads();
  if (!__syncthreads_and(mbar_wait(bar, GF_SPIN_LIMIT) ? 1 : 0)) {
    if (tid == 0) C->status = -7;  // GEOFLOOD_ERR_TIMEOUT
    mbar_wait(bar, GF_SPIN_LIMIT);
    __syncthreads();
    return 0;
  }
  const double drytol = G.drytol;
  int anywet = 0;
  for (int k = tid; k < TG; k += NT) {
    if constexpr (DEV) anywet |= gfk::wet_dev(s0[k], sb[k], drytol, G.drytolf, G.marginf) ? 1 : 0;
    else anywet |= s0[k] > drytol ? 1 : 0;
  }
  anywet = __syncthreads_or(anywet);
  if (anywet) return 1;  // the caller runs the sub-tiles
  if (V.gflag != nullptr && V.gflag[p] != 0 && C->accepted)
    sample_gauges<R, DEV, MP, MP>(V, Pt.scen, C, p, 0, 0, s0, s0, s0, sb, false);
  // dry update of the whole patch (skipped when both buffers already agree)
  const float* los = nullptr;
  float* lod = nullptr;
  if constexpr (DEV) {
    los = V.lof[cur] + (size_t)p * 3 * MP * MP;
    lod = V.lof[cur ^ 1] + (size_t)p * 3 * MP * MP;
  }
  if (!same_in) {
    for (int k = tid; k < MP * MP; k += NT) {
      const int i = k % MP, j = k / MP;
      const int c = (i + GF_NG) + (j + GF_NG) * TGW;
      const R w = s0[c];
      qd[c] = w;
      qd[TG + c] = R(0);
      qd[2 * TG + c] = R(0);
      if constexpr (DEV) {
        lod[k] = los[k];
        lod[MP * MP + k] = 0.0f;
        lod[2 * MP * MP + k] = 0.0f;
      }
      emit_edge<R, MP>(qnext, p, Pt.px, Pt.py, G.mi << Pt.level, G.mj << Pt.level, snb, G.bc,
                       push, i, j, w, R(0), R(0));
    }
  }
  if (tid < NSUB && V.same != nullptr) V.same[p * NSUB + tid] = 1;
  return 0;
}

// Controller of a subcycled macro step (one thread of the last CTA of each
// substep launch per scenario).  The macro step of DT = dt_use runs as
// sub_K substeps; the rates cmax / n_L of the levels that stepped arrived in
// cmax_bits.  Substep 0 (every level steps) is checked against cfl_max: a
// violation rejects the macro step, whose remaining substeps then do
// nothing, and it is retaken with DT = cfl_desired / rate.  Later substeps
// are not checked; their rates bound the next DT.  After the last substep
// the time advances by DT and the next macro step is set up.
static __device__ void subcycle_finish(const GfGeom& G, const GfView& V, GfCtl* Cp,
                                       int s, int cells_per_patch) {
  // every field the rule needs, read from L2 at once
  const int K = G.sub_K;
  const int k = __ldcg(&Cp->sub_k), sub_rej = __ldcg(&Cp->sub_rej);
  const double rate = __longlong_as_double((long long)__ldcg(&Cp->cmax_bits));
  const double DT = __ldcg(&Cp->dt_use);
  const double t = __ldcg(&Cp->t), t_target = __ldcg(&Cp->t_target);
  const double dt_next0 = __ldcg(&Cp->dt_next);
  const double clipvol = __ldcg(&Cp->clipvol), step_clipvol = __ldcg(&Cp->step_clipvol);
  const unsigned long long step_nclip = __ldcg(&Cp->step_nclip);
  const unsigned long long cell_updates = __ldcg(&Cp->cell_updates);
  const unsigned long long rmax_bits = __ldcg(&Cp->rmax_bits);
  const long long steps = __ldcg(&Cp->steps), rejects = __ldcg(&Cp->rejects);
  const long long nclip = __ldcg(&Cp->nclip), taken = __ldcg(&Cp->taken);
  const long long max_steps = __ldcg(&Cp->max_steps);
  const int inrow = __ldcg(&Cp->inrow), lastf = __ldcg(&Cp->last);
  const int nonfinite = __ldcg(&Cp->nonfinite);
  Cp->cmax_bits = 0ull;
  const bool end = k == K - 1;
  double tn = t, dtn = dt_next0;
  long long tk = taken;
  if (nonfinite) {
    Cp->status = -5;  // GEOFLOOD_ERR_NAN
    Cp->active = 0;
    Cp->accepted = 0;
    return;
  }
  if (sub_rej) {
    Cp->accepted = 0;
  } else if (k == 0 && DT * rate > G.cfl_max) {
    dtn = G.cfl_desired / rate;
    Cp->dt_next = dtn;
    Cp->rejects = rejects + 1;
    Cp->accepted = 0;
    Cp->step_nclip = 0ull;
    Cp->step_clipvol = 0.0;
    Cp->rmax_bits = 0ull;
    Cp->inrow = inrow + 1;
    Cp->sub_rej = 1;
    if (inrow + 1 > GF_MAXSTEP_REJECT) {
      Cp->status = -4;  // GEOFLOOD_ERR_CFL
      Cp->active = 0;
      return;
    }
  } else {
    // the substep stands: count the levels that stepped
    unsigned long long cells = 0ull;
    for (int L = G.minlevel; L <= G.maxlevel; ++L)
      if (k % (1 << (G.maxlevel - L)) == 0)
        cells += (unsigned long long)V.scen[s].lcount[L] * (unsigned long long)cells_per_patch;
    Cp->cell_updates = cell_updates + cells;
    unsigned long long rb = rmax_bits;
    if (rate > __longlong_as_double((long long)rmax_bits))
      rb = (unsigned long long)__double_as_longlong(rate);
    Cp->nclip = nclip + (long long)step_nclip;
    Cp->clipvol = clipvol + step_clipvol;
    Cp->step_nclip = 0ull;
    Cp->step_clipvol = 0.0;
    Cp->accepted = 1;
    if (end) {
      tn = lastf ? t_target : t + DT;
      tk = taken + 1;
      Cp->inrow = 0;
      Cp->t = tn;
      Cp->steps = steps + 1;
      Cp->taken = tk;
      const double r = __longlong_as_double((long long)rb);
      rb = 0ull;
      if (r > 0.0) {
        const double dn = G.cfl_desired / r;
        dtn = dn < G.dt_max ? dn : G.dt_max;
        Cp->dt_next = dtn;
      }
    }
    Cp->rmax_bits = rb;
  }
  if (!end) {
    Cp->sub_k = k + 1;
    return;
  }
  Cp->sub_k = 0;
  Cp->sub_rej = 0;
  if (!(tn < t_target) || tk >= max_steps) {
    Cp->active = 0;
  } else {
    const double rem = t_target - tn;
    if (dtn < rem) { Cp->dt_use = dtn; Cp->last = 0; }
    else { Cp->dt_use = rem; Cp->last = 1; }
  }
}

// CFL rule of one scenario at the end of a step (Sec. 5.1 maximum CFL,
// Sec. 6.6), not subcycled: reject the step and set a smaller dt when
// dt*cmax exceeds cfl_max, else accept it (swap the state buffers, advance
// t) and pick the next dt = cfl_desired / cmax, clipped to land on t_target.
// One thread runs it: every field it needs is read from L2 at once
// (independent loads, one round trip instead of one per field), the
// decision is taken on the copies, and only the fields that change are
// written back.
static __device__ void ctl_finish(const GfGeom& G, GfCtl* Cp, unsigned long long cells) {
  const double cmax = __longlong_as_double((long long)__ldcg(&Cp->cmax_bits));
  const double dt = __ldcg(&Cp->dt_use);
  const double t = __ldcg(&Cp->t), t_target = __ldcg(&Cp->t_target);
  const double dt_next0 = __ldcg(&Cp->dt_next);
  const double clipvol = __ldcg(&Cp->clipvol), step_clipvol = __ldcg(&Cp->step_clipvol);
  const unsigned long long step_nclip = __ldcg(&Cp->step_nclip);
  const unsigned long long cell_updates = __ldcg(&Cp->cell_updates);
  const long long steps = __ldcg(&Cp->steps), rejects = __ldcg(&Cp->rejects);
  const long long nclip = __ldcg(&Cp->nclip), taken = __ldcg(&Cp->taken);
  const long long max_steps = __ldcg(&Cp->max_steps);
  const int cur = __ldcg(&Cp->cur), lastf = __ldcg(&Cp->last);
  const int inrow = __ldcg(&Cp->inrow), nonfinite = __ldcg(&Cp->nonfinite);
  Cp->cell_updates = cell_updates + cells;
  Cp->cmax_bits = 0ull;
  if (nonfinite) {
    Cp->status = -5;  // GEOFLOOD_ERR_NAN
    Cp->active = 0;
    Cp->accepted = 0;
    return;
  }
  double tn = t, dtn = dt_next0;
  long long tk = taken;
  if (dt * cmax > G.cfl_max) {
    dtn = G.cfl_desired / cmax;
    Cp->dt_next = dtn;
    Cp->rejects = rejects + 1;
    Cp->accepted = 0;
    Cp->step_nclip = 0ull;
    Cp->step_clipvol = 0.0;
    Cp->inrow = inrow + 1;
    if (inrow + 1 > GF_MAXSTEP_REJECT) {
      Cp->status = -4;  // GEOFLOOD_ERR_CFL
      Cp->active = 0;
      return;
    }
  } else {
    tn = lastf ? t_target : t + dt;
    tk = taken + 1;
    Cp->inrow = 0;
    Cp->cur = cur ^ 1;
    Cp->t = tn;
    Cp->steps = steps + 1;
    Cp->taken = tk;
    Cp->nclip = nclip + (long long)step_nclip;
    Cp->clipvol = clipvol + step_clipvol;
    Cp->step_nclip = 0ull;
    Cp->step_clipvol = 0.0;
    Cp->accepted = 1;
    if (cmax > 0.0) {
      const double dn = G.cfl_desired / cmax;
      dtn = dn < G.dt_max ? dn : G.dt_max;
      Cp->dt_next = dtn;
    }
  }
  if (!(tn < t_target) || tk >= max_steps) {
    Cp->active = 0;
  } else {
    const double rem = t_target - tn;
    if (dtn < rem) { Cp->dt_use = dtn; Cp->last = 0; }
    else { Cp->dt_use = rem; Cp->last = 1; }
  }
}

// End of a step: the last CTA to finish applies the CFL rule to every active
// scenario, one thread per scenario (the scenarios' rules are independent).
// The volume of the state is not part of the step; geoflood_mass computes it
// on demand.
template <int NT>
__device__ void step_finish(const GfGeom& G, const GfView& V, int cells_per_patch,
                            bool wrote = true) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    // a CTA that updated the controller's counters (atomics) orders them
    // before it counts itself done; one that did not needs no fence
    if (wrote) __threadfence();
    const unsigned t = atomicAdd(V.done, 1u);
    last = t == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int s = threadIdx.x; s < G.nscen; s += NT) {
    GfCtl* Cp = V.ctl + s;
    if (!__ldcg(&Cp->active)) {
      Cp->accepted = 0;
      continue;
    }
    if (G.subcycle)
      subcycle_finish(G, V, Cp, s, cells_per_patch);
    else
      ctl_finish(G, Cp, (unsigned long long)V.scen[s].pcount * (unsigned long long)cells_per_patch);
  }
  // the next launch reads the counters and the schedule after this kernel
  // has ended, which orders these writes before it
  if (threadIdx.x == 0 && V.sched) {
    V.sched[0] ^= 1u;
    V.sched[3] = V.sched[1];  // wet patches at the head of the next order
    V.sched[1] = 0u;
    V.sched[2] = 0u;
  }
  if (threadIdx.x == 0) *V.done = 0u;
}

// Adaptive variant: the previous launch's wet patches (the head of its
// launch order, sched[3] of them) get NSUB CTAs each, one per M x M
// sub-tile; every other patch gets one CTA that checks the whole tile and
// takes the dry update, or the sub-tiles in turn if water has arrived.  The
// grid has NSUB CTAs per patch; those beyond the work exit at once.
template <class P, int MP, int M, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_patch_step_adaptive(const __grid_constant__ GfGeom G,
                          const __grid_constant__ GfView V) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NSUB = (MP / M) * (MP / M);
  const bool sched = V.sched != nullptr && V.done != nullptr;
  const unsigned par = sched ? V.sched[0] : 0u;
  const int nw = sched ? (int)V.sched[3] : 0;
  const int* ord = sched ? (par ? V.ord1 : V.ord0) : nullptr;
  const int b = blockIdx.x;
  int p = -1, wet = 0;
  int s_lo = 0, s_hi = 0;  // sub-tiles this CTA computes
  bool whole = false, active = false;
  if (b < nw * NSUB) {
    p = ord[b / NSUB];
    s_lo = b % NSUB;
    s_hi = s_lo + 1;
  } else if (b < nw * NSUB + (V.npatch - nw)) {
    p = sched ? ord[nw + (b - nw * NSUB)] : b;
    whole = true;
  }
  if (p >= 0) active = V.ctl[V.patch[p].scen].active != 0;
  if (whole && active && whole_tile<P, MP, M, NT>(G, V, smraw, p)) {
    wet = 1;
    s_lo = 0;
    s_hi = NSUB;
  }
  if (!active) s_hi = s_lo;
  // one call site of the sub-tile body
  for (int sub = s_lo; sub < s_hi; ++sub) {
    wet |= patch_body<P, MP, M, NT>(G, V, smraw, p, sub);
    __syncthreads();
  }
  bool report = whole && threadIdx.x == 0;
  if (!whole && p >= 0 && threadIdx.x == 0) {
    // the last of the patch's CTAs reports whether any sub-tile held water
    if (wet) V.pwet[p] = 1u;
    __threadfence();
    const unsigned c = atomicAdd(V.pcnt + p, 1u);
    if (c == NSUB - 1) {
      __threadfence();
      wet = *(volatile unsigned*)(V.pwet + p) != 0u;
      V.pwet[p] = 0u;
      V.pcnt[p] = 0u;
      report = true;
    }
  }
  if (sched && report) {
    int* nxt = par ? V.ord0 : V.ord1;
    if (wet) nxt[atomicAdd(V.sched + 1, 1u)] = p;
    else nxt[V.npatch - 1 - (int)atomicAdd(V.sched + 2, 1u)] = p;
  }
  if (V.done)
    step_finish<NT>(G, V, MP * MP);
}

template <class P, int MP, int M, int NT, int MINB, bool DS = false>
__global__ void __launch_bounds__(NT, MINB)
    k_patch_step(const __grid_constant__ GfGeom G,
                 const __grid_constant__ GfView V) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NSUB = (MP / M) * (MP / M);
  const int slot = blockIdx.x / NSUB, sub = blockIdx.x % NSUB;
  // launch order: tiles that held water in the previous launch first, so the
  // long wet CTAs start at once and the short dry ones fill in around them
  const bool sched = V.sched != nullptr && V.done != nullptr;
  const unsigned par = sched ? V.sched[0] : 0u;
  const int p = sched ? (par ? V.ord1 : V.ord0)[slot] : slot;
  // run flags (GfView::runf): read by every thread beside the patch record,
  // so that a running tile waits for nothing more
  constexpr bool FLAGS = NSUB == 1 && !DS;
  const bool use_flags = FLAGS && sched && V.runf != nullptr && !G.subcycle;
  unsigned char* rcur = use_flags ? V.runf + (size_t)(par & 1u) * V.runf_stride : nullptr;
  unsigned char* rnxt = use_flags ? V.runf + (size_t)((par ^ 1u) & 1u) * V.runf_stride : nullptr;
  const bool marked = use_flags && rcur[p] != 0;
  // an unmarked dry, unchanged tile without a gauge takes no step (the full
  // path would find its ghost ring dry and write nothing)
  const bool skip = use_flags && !marked && V.same != nullptr && V.same[p] != 0 &&
                    !(V.gflag != nullptr && V.gflag[p] != 0);
  int wet = 0;
  bool wrote = false;
  if (!skip) {
    const GfPatch Pt = V.patch[p];
    bool run = V.ctl[Pt.scen].active != 0;
    if (run && G.subcycle) {
      // level subcycling: only the levels due at this substep step
      const GfCtl& C = V.ctl[Pt.scen];
      run = !C.sub_rej && C.sub_k % (1 << (G.maxlevel - Pt.level)) == 0;
    }
    wrote = true;
    if (run)
      wet = patch_body<P, MP, M, NT, DS>(G, V, smraw, p, sub, nullptr, &wrote);
    else wrote = false;
    if (use_flags && threadIdx.x == 0) {
      // the mark is consumed; a patch that did not run carries it forward
      rcur[p] = 0;
      if (!run) rnxt[p] = 1;
    }
    if (use_flags && wet && threadIdx.x < 9) {
      // water in this tile: it and its same-level neighbours run next launch
      // (their indices were staged in shared memory by the patch body)
      using Lo = Layout<P, M, DS>;
      const int* snb = reinterpret_cast<const int*>(smraw + Lo::OFF_NB);
      const int q = threadIdx.x == 8 ? p : snb[threadIdx.x];
      if (q >= 0) rnxt[q] = 1;
    }
  }
  if (sched && sub == 0 && threadIdx.x == 0) {
    int* nxt = par ? V.ord0 : V.ord1;
    if (wet) nxt[atomicAdd(V.sched + 1, 1u)] = p;
    else nxt[V.npatch - 1 - (int)atomicAdd(V.sched + 2, 1u)] = p;
  }
  if (V.done)
    step_finish<NT>(G, V, MP * MP, wrote);
}

// Launch the patch step on every patch: MP x MP patches, M x M sub-tiles
// per CTA of NT threads (MINB CTAs per SM), DS = dimensional splitting.
template <class P, int MP, int M, int NT, int MINB, bool DS = false>
int launch_step(const GfGeom& g, const GfView& v, cudaStream_t st) {
  constexpr size_t bytes = Layout<P, M, DS>::BYTES;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_patch_step<P, MP, M, NT, MINB, DS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess)
      return -2;
    attr = true;
  }
  constexpr int NSUB = (MP / M) * (MP / M);
  k_patch_step<P, MP, M, NT, MINB, DS><<<v.npatch * NSUB, NT, bytes, st>>>(g, v);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Launch the adaptive variant (NSUB CTAs per patch, see
// k_patch_step_adaptive).
template <class P, int MP, int M, int NT, int MINB>
int launch_step_adaptive(const GfGeom& g, const GfView& v, cudaStream_t st) {
  constexpr size_t bytes = Layout<P, M>::BYTES;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_patch_step_adaptive<P, MP, M, NT, MINB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess)
      return -2;
    attr = true;
  }
  constexpr int NSUB = (MP / M) * (MP / M);
  k_patch_step_adaptive<P, MP, M, NT, MINB><<<v.npatch * NSUB, NT, bytes, st>>>(g, v);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gfs
