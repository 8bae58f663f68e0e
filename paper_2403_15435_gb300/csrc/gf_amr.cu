// Quadtree kernels (FP64): ghost-cell exchange between patches at equal or
// different levels (copy / 2x2 average / limited interpolation) and the
// physical boundaries, topography cell averages from a DEM, regrid data
// transfer, the plain tagger, gauges, volume sums and host staging.
// Compiled with -fmad=false.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "gf_internal.h"
#include "gf_solver.cuh"

namespace {

template <typename T>
struct Geo {
  static constexpr bool DEV = sizeof(T) == 4;  // FP32 surface-deviation form
  const GfGeom& G;
  const GfView& V;
  __device__ Geo(const GfGeom& g, const GfView& v) : G(g), V(v) {}
  __device__ long long nx(int L) const { return (long long)G.mi * G.M << L; }
  __device__ long long ny(int L) const { return (long long)G.mj * G.M << L; }
  __device__ double dx(int L) const { return (G.xupper - G.xlower) / (double)nx(L); }
  __device__ double dy(int L) const { return (G.yupper - G.ylower) / (double)ny(L); }
  __device__ int tix(int i, int j) const { return (i + GF_NG) + (j + GF_NG) * G.T; }
  // tile index of cell (I, J) of a level inside the leaf that the level's
  // lookup table returned for it: that leaf is the patch at (I / M, J / M)
  // of the level, so the local cell is (I mod M, J mod M) (M = 16 or 32)
  __device__ int local(long long I, long long J) const {
    return tix((int)(I & (G.M - 1)), (int)(J & (G.M - 1)));
  }
  // leaf of level L holding cell (I, J) of that level, or -1
  __device__ int leaf(int s, int L, long long I, long long J) const {
    if (L < 0 || L > G.maxlevel) return -1;
    // patch sizes are 16 or 32, so the patch index of a non-negative cell
    // index is a shift (a 64-bit division would be emulated in software)
    const int sh = G.M == 32 ? 5 : 4;
    const long long P = I >= 0 ? I >> sh : -1, Q = J >= 0 ? J >> sh : -1;
    const long long w = (long long)G.mi << L, h = (long long)G.mj << L;
    if (P < 0 || Q < 0 || P >= w || Q >= h) return -1;
    return V.lut[V.scen[s].lut_off + G.lut_lev_off[L] + P + Q * w];
  }
  __device__ T* qp(int p, int buf) const {
    T* base;
    if constexpr (DEV) base = V.qf[buf];
    else base = V.q[buf];
    return base + (size_t)p * 3 * G.T * G.T;
  }
  __device__ T* bp(int p) const {
    T* base;
    if constexpr (DEV) base = V.bf;
    else base = V.b;
    return base + (size_t)p * G.T * G.T;
  }
  // Buffer holding patch p's latest state.  With level subcycling, during a
  // macro step (sub_k > 0) a level with period P = 2^(maxlevel - L) has
  // taken ceil(sub_k / P) steps, each flipping its buffers.
  __device__ int cur_of(int p) const {
    const GfPatch& P = V.patch[p];
    const GfCtl& C = V.ctl[P.scen];
    if (!G.subcycle || C.sub_k == 0) return C.cur;
    const int per = 1 << (G.maxlevel - P.level);
    const int st = (C.sub_k + per - 1) / per;
    return C.cur ^ (st & 1);
  }
  // (h, hu, hv, b) of cell c of patch p at the time of the substep about to
  // run: its latest state, or for a level between two of its steps the
  // linear interpolation in time of h, hu, hv between the states before and
  // after its latest step
  // load_now for a patch p of scenario s: without subcycling the latest
  // buffer is the scenario's current one, read without the patch record
  __device__ void load_now_s(int p, int s, int c, double (&o)[4]) const {
    if (!G.subcycle) {
      load(p, V.ctl[s].cur, c, o);
      return;
    }
    load_now(p, c, o);
  }
  __device__ void load_now(int p, int c, double (&o)[4]) const {
    const int cb = cur_of(p);
    load(p, cb, c, o);
    if (!G.subcycle) return;
    const GfPatch& P = V.patch[p];
    const int k = V.ctl[P.scen].sub_k;
    const int per = 1 << (G.maxlevel - P.level);
    const int r = k % per;
    if (r == 0) return;
    double old[4];
    load(p, cb ^ 1, c, old);
    const double a = (double)r / (double)per;
    for (int f = 0; f < 3; ++f) o[f] = (1.0 - a) * old[f] + a * o[f];
  }
  // (h, hu, hv, b) of cell c of patch p in buffer buf, in FP64; in the
  // deviation form h = w - b exactly and b is the bed minus eta0
  __device__ void load(int p, int buf, int c, double (&o)[4]) const {
    const int TT = G.T * G.T;
    const T* q = qp(p, buf);
    const double b = (double)bp(p)[c];
    o[0] = DEV ? (double)q[c] - b : (double)q[c];
    o[1] = (double)q[TT + c];
    o[2] = (double)q[2 * TT + c];
    o[3] = b;
  }
  // store (h, hu, hv) into cell c of patch p, buffer buf, whose bed is b
  __device__ void store(T* q, int c, double h, double hu, double hv,
                        double b) const {
    const int TT = G.T * G.T;
    q[c] = DEV ? (T)(h + b) : (T)h;
    q[TT + c] = (T)hu;
    q[2 * TT + c] = (T)hv;
  }
};

// Composite value (h, hu, hv, b) at cell (I, J) of level L: the leaf of that
// level, a coarser leaf's cell, or the mean of the finer cells (down to two
// levels finer, which a 2:1 balanced forest never exceeds).
template <typename T>
__device__ void value_at(const Geo<T>& e, int s, int L, long long I,
                         long long J, double (&out)[4], int* err) {
  for (int l = L; l >= 0; --l) {
    const long long Il = I >> (L - l), Jl = J >> (L - l);
    const int p = e.leaf(s, l, Il, Jl);
    if (p >= 0) {
      const int c = e.local(Il, Jl);
      e.load_now_s(p, s, c, out);
      return;
    }
  }
  double v[4][4];
  for (int ch = 0; ch < 4; ++ch) {
    const long long Ic = 2 * I + (ch & 1), Jc = 2 * J + (ch >> 1);
    const int p = e.leaf(s, L + 1, Ic, Jc);
    if (p >= 0) {
      const int c = e.local(Ic, Jc);
      e.load_now_s(p, s, c, v[ch]);
    } else {
      double w[4][4];
      for (int gc = 0; gc < 4; ++gc) {
        const long long Ig = 2 * Ic + (gc & 1), Jg = 2 * Jc + (gc >> 1);
        const int pg = e.leaf(s, L + 2, Ig, Jg);
        if (pg < 0) {
          *err = 1;
          w[gc][0] = w[gc][1] = w[gc][2] = w[gc][3] = 0.0;
          continue;
        }
        const int c = e.local(Ig, Jg);
        e.load_now_s(pg, s, c, w[gc]);
      }
      for (int f = 0; f < 4; ++f)
        v[ch][f] = 0.25 * ((w[0][f] + w[1][f]) + (w[2][f] + w[3][f]));
    }
  }
  for (int f = 0; f < 4; ++f)
    out[f] = 0.25 * ((v[0][f] + v[1][f]) + (v[2][f] + v[3][f]));
}

__device__ __forceinline__ double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

// Beds of the four tile cells that share a parent with tile cell (i, j):
// bs[b][a] is the child at x offset a and y offset b (patch origins are
// even, so siblings differ from (i, j) in the last bit only, ghosts included).
template <typename T, typename B>
__device__ __forceinline__ void child_beds(const Geo<T>& e, const B* bed, int i, int j,
                                           double (&bs)[2][2]) {
  const int i0 = i & ~1, j0 = j & ~1;
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) bs[b][a] = (double)bed[e.tix(i0 + a, j0 + b)];
}

// The four children (a, b) of cell (ic, jc) of level L - 1, whose beds are
// bs[b][a], interpolated from level L - 1 (the rule fill_cell states):
// out[b][a] = (h, hu, hv) of child (2 ic + a, 2 jc + b) of level L.
template <typename T>
__device__ void interp_children(const Geo<T>& e, int s, int L, long long ic, long long jc,
                                const double (&bs)[2][2], double (&out)[2][2][3], int* err) {
  const long long NXc = e.nx(L - 1), NYc = e.ny(L - 1);
  double nb[3][3][4];
  bool in[3][3];
  for (int dj = -1; dj <= 1; ++dj)
    for (int di = -1; di <= 1; ++di) {
      const long long x = ic + di, y = jc + dj;
      in[dj + 1][di + 1] = x >= 0 && y >= 0 && x < NXc && y < NYc;
      if (in[dj + 1][di + 1]) value_at(e, s, L - 1, x, y, nb[dj + 1][di + 1], err);
    }
  const double drytol = e.G.drytol;
  const double* qc = nb[1][1];
  if (qc[0] <= drytol) {
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        out[b][a][0] = qc[0];
        out[b][a][1] = qc[1];
        out[b][a][2] = qc[2];
      }
    return;
  }
  bool allwet = true;
  for (int dj = 0; dj < 3; ++dj)
    for (int di = 0; di < 3; ++di)
      if (in[dj][di] && !(nb[dj][di][0] > drytol)) allwet = false;
  const double etac = qc[0] + qc[3];
  // limited slopes over the coarse cell: surface, then both momenta
  double g[3][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
  if (allwet) {
    const bool hx = in[1][0] && in[1][2], hy = in[0][1] && in[2][1];
    double et[3][3];
    for (int dj = 0; dj < 3; ++dj)
      for (int di = 0; di < 3; ++di)
        et[dj][di] = in[dj][di] ? nb[dj][di][0] + nb[dj][di][3] : 0.0;
    if (hx) g[0][0] = minmod(et[1][2] - et[1][1], et[1][1] - et[1][0]);
    if (hy) g[0][1] = minmod(et[2][1] - et[1][1], et[1][1] - et[0][1]);
    for (int k = 1; k < 3; ++k) {
      if (hx) g[k][0] = minmod(nb[1][2][k] - qc[k], qc[k] - nb[1][0][k]);
      if (hy) g[k][1] = minmod(nb[2][1][k] - qc[k], qc[k] - nb[0][1][k]);
    }
  }
  // the four children: depth d, linearly interpolated momenta m
  double d[2][2], m[2][2][2];
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) {
      const double sx = a ? 0.25 : -0.25, sy = b ? 0.25 : -0.25;
      const double eta = allwet ? (etac + sx * g[0][0]) + sy * g[0][1] : etac;
      const double h = eta - bs[b][a];
      d[b][a] = h > 0.0 ? h : 0.0;
      for (int k = 0; k < 2; ++k)
        m[b][a][k] = (qc[k + 1] + sx * g[k + 1][0]) + sy * g[k + 1][1];
    }
  const double S = (d[0][0] + d[0][1]) + (d[1][0] + d[1][1]);
  bool split[2];
  for (int k = 0; k < 2; ++k) {
    split[k] = !allwet;
    if (allwet) {
      double lo = INFINITY, hi = -INFINITY;
      for (int dj = 0; dj < 3; ++dj)
        for (int di = 0; di < 3; ++di)
          if (in[dj][di]) {
            const double u = nb[dj][di][k + 1] / nb[dj][di][0];
            lo = fmin(lo, u);
            hi = fmax(hi, u);
          }
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a)
          if (d[b][a] > drytol) {
            const double u = m[b][a][k] / d[b][a];
            if (u < lo || u > hi) split[k] = true;
          }
    }
  }
  for (int b0 = 0; b0 < 2; ++b0)
    for (int a0 = 0; a0 < 2; ++a0) {
      const double hf = d[b0][a0];
      out[b0][a0][0] = hf;
      for (int k = 0; k < 2; ++k)
        out[b0][a0][k + 1] = !split[k] ? m[b0][a0][k]
                                       : (S > 0.0 ? (4.0 * qc[k + 1]) * (hf / S) : 0.0);
      if (hf <= drytol) {
        out[b0][a0][1] = 0.0;
        out[b0][a0][2] = 0.0;
      }
    }
}

// Value (h, hu, hv) of cell (I, J) of level L, whose parent's four children
// have the beds bs (bs[J & 1][I & 1] is this cell's), from the forest of the
// view: copy from a same-level leaf, mean of finer cells, or interpolation
// of the coarser level (Sec. 4 ghost cells, Sec. 6.2 surface-preserving
// interpolation).  The interpolation treats the four children together:
// depth = interpolated surface (limited linear over a wet 3x3
// neighbourhood, the parent's surface otherwise) minus the child's bed,
// clamped at zero; momentum = limited linear interpolation over a wet
// neighbourhood unless a wet child's velocity leaves the range of the
// neighbourhood's velocities, else the parent's momentum split in
// proportion to the children's depths.
template <typename T>
__device__ void fill_cell(const Geo<T>& e, int s, int L, long long I,
                          long long J, const double (&bs)[2][2], double (&out)[3], int* err) {
  const double bt = bs[J & 1][I & 1];
  const int p = e.leaf(s, L, I, J);
  if (p >= 0) {
    const int c = e.local(I, J);
    double o4[4];
    e.load_now_s(p, s, c, o4);
    out[0] = o4[0];
    out[1] = o4[1];
    out[2] = o4[2];
    return;
  }
  bool coarser = false;
  for (int l = L - 1; l >= 0 && !coarser; --l)
    coarser = e.leaf(s, l, I >> (L - l), J >> (L - l)) >= 0;
  if (!coarser) {
    double v[4][4];
    value_at(e, s, L + 1, 2 * I, 2 * J, v[0], err);
    value_at(e, s, L + 1, 2 * I + 1, 2 * J, v[1], err);
    value_at(e, s, L + 1, 2 * I, 2 * J + 1, v[2], err);
    value_at(e, s, L + 1, 2 * I + 1, 2 * J + 1, v[3], err);
    for (int f = 0; f < 3; ++f)
      out[f] = 0.25 * ((v[0][f] + v[1][f]) + (v[2][f] + v[3][f]));
    if constexpr (Geo<T>::DEV) {
      // deviation form: over four wet children the mean stored surface is
      // kept (the FP32 beds of two levels are rounded separately, so the
      // mean depth over the coarse bed would not keep still water still)
      const double dt = e.G.drytol;
      if (v[0][0] > dt && v[1][0] > dt && v[2][0] > dt && v[3][0] > dt) {
        const double eta = 0.25 * (((v[0][0] + v[0][3]) + (v[1][0] + v[1][3])) +
                                   ((v[2][0] + v[2][3]) + (v[3][0] + v[3][3])));
        const double h = eta - bt;
        out[0] = h > 0.0 ? h : 0.0;
      }
    }
    return;
  }
  double quad[2][2][3];
  interp_children(e, s, L, I >> 1, J >> 1, bs, quad, err);
  for (int f = 0; f < 3; ++f) out[f] = quad[J & 1][I & 1][f];
}

// Physical boundaries of one tile held in global memory: bottom/top over the
// columns inside the domain, then left/right over every row (Sec. 5.1 closed
// walls mirror the cells and negate the normal momentum; extrapolation
// copies the edge cell).  fields: 0 = h, hu, hv in q; 1 = the bed in b.
template <typename T, typename G2>
__device__ void tile_bc(const G2& e, const GfPatch& P, T* q, T* bfield,
                        int bed) {
  const int M = e.G.M, T_ = e.G.T, TT = T_ * T_;
  const long long NX = e.nx(P.level), NY = e.ny(P.level);
  const int nf = bed ? 1 : 3;
  for (int side = 2; side <= 3; ++side) {
    const bool at = side == 2 ? (P.py == 0) : ((long long)(P.py + 1) * M == NY);
    if (!at) continue;
    const bool wall = e.G.bc[side] == 0;
    const int n = T_ * GF_NG * nf;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const int i = k % T_ - GF_NG, gl = (k / T_) % GF_NG + 1, f = k / (T_ * GF_NG);
      const long long I = (long long)P.px * M + i;
      if (I < 0 || I >= NX) continue;
      const int jg = side == 2 ? -gl : M - 1 + gl;
      const int js = wall ? (side == 2 ? gl - 1 : M - gl) : (side == 2 ? 0 : M - 1);
      T* a = bed ? bfield : q + f * TT;
      T v = a[e.tix(i, js)];
      if (!bed && wall && f == 2) v = -v;
      a[e.tix(i, jg)] = v;
    }
    __syncthreads();
  }
  for (int side = 0; side <= 1; ++side) {
    const bool at = side == 0 ? (P.px == 0) : ((long long)(P.px + 1) * M == NX);
    if (!at) continue;
    const bool wall = e.G.bc[side] == 0;
    const int n = T_ * GF_NG * nf;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const int j = k % T_ - GF_NG, gl = (k / T_) % GF_NG + 1, f = k / (T_ * GF_NG);
      const int ig = side == 0 ? -gl : M - 1 + gl;
      const int is = wall ? (side == 0 ? gl - 1 : M - gl) : (side == 0 ? 0 : M - 1);
      T* a = bed ? bfield : q + f * TT;
      T v = a[e.tix(is, j)];
      if (!bed && wall && f == 1) v = -v;
      a[e.tix(ig, j)] = v;
    }
    __syncthreads();
  }
}

// FP32 ghost operator (defined with the level-change ghosts below).
__device__ void fill_cell_f32(const Geo<float>& e, int s, int cur, int L, long long I,
                              long long J, const float (&bs)[2][2], float (&out)[3],
                              int* err);

// Ghost fill: one CTA per patch, one thread per ghost cell.  Interior-domain
// ghosts from the leaves (reads only leaf interiors, so patches are
// independent), then the physical boundaries.  A ghost cell in a region
// whose same-level neighbour exists is a plain copy of that neighbour's
// stored values; its position in the neighbour follows from the region's
// offset, so only the neighbour's index is looked up (in shared memory).
// (At most 288 threads: one per ghost cell of a 32 x 32 patch's tile.)
template <typename T>
__global__ void __launch_bounds__(288, 1)
    k_ghost_fill(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V, int only_accepted,
                             int* errflag, const int* list) {
  // with a list: only the listed patches, and only the regions without a
  // same-level neighbour (the patch step pushed those)
  const int p = list ? list[blockIdx.x] : blockIdx.x;
  __shared__ int snb[8];
  if (threadIdx.x < 8)
    snb[threadIdx.x] = V.nbr ? V.nbr[(size_t)p * 8 + threadIdx.x] : GF_NBR_OTHER;
  const GfPatch P = V.patch[p];
  const GfCtl* C = V.ctl + P.scen;
  if (only_accepted && !C->accepted) return;
  Geo<T> e(G, V);
  const int M = G.M, T_ = G.T, TT = T_ * T_;
  const int cur = C->cur;
  T* q = e.qp(p, cur);
  const T* bb = e.bp(p);
  const long long NX = e.nx(P.level), NY = e.ny(P.level);
  const int nghost = TT - M * M;
  __syncthreads();
  int err = 0;
  for (int k = threadIdx.x; k < nghost; k += blockDim.x) {
    // enumerate ghost cells: the two bottom rows, the two top rows, then the
    // left and right column pairs of the interior rows
    int i, j;
    const int band = 2 * T_;
    if (k < band) { i = k % T_ - GF_NG; j = k / T_ - GF_NG; }
    else if (k < 2 * band) { i = (k - band) % T_ - GF_NG; j = M + (k - band) / T_; }
    else {
      const int r = k - 2 * band;  // 4 * M cells
      j = r / 4;
      const int c = r % 4;
      i = c < 2 ? c - GF_NG : M + (c - 2);
    }
    const long long I = (long long)P.px * M + i, J = (long long)P.py * M + j;
    if (I < 0 || J < 0 || I >= NX || J >= NY) continue;
    const int c = e.tix(i, j);
    // regions: left, right, bottom, top, then the corners bottom-left,
    // bottom-right, top-left, top-right
    const int dxr = i < 0 ? -1 : (i >= M ? 1 : 0);
    const int dyr = j < 0 ? -1 : (j >= M ? 1 : 0);
    const int region = dxr == 0 ? (dyr < 0 ? 2 : 3)
                                : (dyr == 0 ? (dxr < 0 ? 0 : 1)
                                            : 4 + (dxr > 0 ? 1 : 0) + (dyr > 0 ? 2 : 0));
    const int pn = V.nbr ? snb[region] : e.leaf(P.scen, P.level, I, J);
    if (pn >= 0 && list) continue;
    if (pn >= 0) {
      const int cn = e.tix(i - dxr * M, j - dyr * M);
      const T* qn = e.qp(pn, cur);
      const T a0 = qn[cn], a1 = qn[TT + cn], a2 = qn[2 * TT + cn];
      q[c] = a0;
      q[TT + c] = a1;
      q[2 * TT + c] = a2;
      continue;
    }
    if constexpr (Geo<T>::DEV) {
      if (!G.subcycle) {
        float bs[2][2], out[3];
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a) bs[b][a] = bb[e.tix((i & ~1) + a, (j & ~1) + b)];
        fill_cell_f32(e, P.scen, cur, P.level, I, J, bs, out, &err);
        q[c] = out[0];
        q[TT + c] = out[1];
        q[2 * TT + c] = out[2];
        continue;
      }
    }
    double bs[2][2];
    child_beds(e, bb, i, j, bs);
    const double bt = bs[j & 1][i & 1];
    double out[3];
    fill_cell(e, P.scen, P.level, I, J, bs, out, &err);
    e.store(q, c, out[0], out[1], out[2], bt);
  }
  if (err && errflag) *errflag = 1;
  // physical boundaries last (they mirror the cells filled above)
  __syncthreads();
  tile_bc<T>(e, P, q, nullptr, 0);
}

// ------------------------------------------------------ inflow boundary

// Discharge Q(t) of the inflow hydrograph: piecewise linear through the
// points, constant before the first and after the last (Sec. 5.1).
__device__ double hydro_discharge(const GfGeom& G, double t) {
  const int n = G.n_hydro;
  if (n <= 0) return 0.0;
  if (t <= G.hydro_t[0]) return G.hydro_q[0];
  if (t >= G.hydro_t[n - 1]) return G.hydro_q[n - 1];
  int k = 0;
  while (k + 1 < n && !(t < G.hydro_t[k + 1])) ++k;
  const double a = (t - G.hydro_t[k]) / (G.hydro_t[k + 1] - G.hydro_t[k]);
  return G.hydro_q[k] + (G.hydro_q[k + 1] - G.hydro_q[k]) * a;
}

// F(h) and F'(h) of the boundary equation: shock = false is Eq. riemann
// (the ghost joined to the interior by a rarefaction entering the domain:
// q/h - 2 sqrt(g h) = u_i - 2 sqrt(g h_i)), shock = true Eq. 2-shock (the
// Hugoniot locus: q/h = u_i + (h - h_i) sqrt(g/2 (1/h + 1/h_i))).  Both
// decrease in h where they are solved.
__device__ double inflow_f(bool shock, double h, double q, double hi, double ui,
                           double g, double* dF) {
  if (!shock) {
    *dF = -q / (h * h) - sqrt(g / h);
    return q / h - 2.0 * sqrt(g * h) - ui + 2.0 * sqrt(g * hi);
  }
  const double S = sqrt(0.5 * g * (1.0 / h + 1.0 / hi));
  *dF = -q / (h * h) - S + (h - hi) * g / (4.0 * h * h * S);
  return q / h - ui - (h - hi) * S;
}

// Newton's method from h0 for the root above lo, safeguarded by the
// bracket that the signs of F establish: a step leaving it is replaced by
// the midpoint, or by a doubling while no upper end is known.  At most 100
// iterations; stops when a step is below 1e-14 relative.
__device__ double inflow_root(bool shock, double h0, double lo, double q, double hi_,
                              double ui, double g) {
  double hi = INFINITY, h = h0 > lo ? h0 : 2.0 * lo;
  for (int it = 0; it < 100; ++it) {
    double dF;
    const double F = inflow_f(shock, h, q, hi_, ui, g, &dF);
    if (F > 0.0) lo = h;
    else if (F < 0.0) hi = h;
    else return h;
    double hn = h - F / dF;
    if (!(hn > lo && hn < hi)) hn = isinf(hi) ? 2.0 * h : 0.5 * (lo + hi);
    if (fabs(hn - h) <= 1e-14 * hn) return hn;
    h = hn;
  }
  return h;
}

// Ghost depth for unit discharge q > 0 entering next to an interior cell of
// depth h_int and momentum qn_int into the domain.  An interior thinner than
// tau is replaced by the inflow's critical depth (at least tau) at rest.
// Eq. riemann first (first guess [F q / sqrt(g)]^(2/3), F = 0.5); a depth
// above the interior's is recomputed by Eq. 2-shock (F = 1).
__device__ double inflow_depth(double q, double h_int, double qn_int, double g,
                               double tau) {
  double hi, ui;
  if (h_int < tau) {
    const double hc = cbrt(q * q / g);
    hi = hc > tau ? hc : tau;
    ui = 0.0;
  } else {
    hi = h_int;
    ui = qn_int / h_int;
  }
  double h = inflow_root(false, cbrt(0.25 * q * q / g), 0.0, q, hi, ui, g);
  if (h > hi) h = inflow_root(true, cbrt(q * q / g), hi, q, hi, ui, g);
  return h;
}

// Inflow ghost cells, one CTA per patch on the inflow side, one thread per
// line of its tile (rows for a left or right side, columns otherwise,
// -2..M+1).  A line inside the domain whose centre lies in the segment
// gets, in both ghost layers, the depth of the boundary equations from the
// tile's first cell of that line, the unit discharge Q(t) / W_L normal to
// the side into the domain (W_L = G.inflow_width[L], the width of the
// segment's lines at the patch's level, so that Q(t) enters at every
// resolution) and no tangential momentum; the tile corners
// beyond those ghost cells, where the tile touches a side across the lines,
// follow that side's rule applied to them.  With Q(t) = 0 the side's own
// rule (written by the step and the other ghost kernels) stays.  Runs after
// every other ghost cell of the tile is final.
template <typename T>
__global__ void k_inflow(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V,
                         const int* list, int only_accepted) {
  const int p = list[blockIdx.x];
  const int M = G.M, TT = G.T * G.T;
  // a patch on the inflow side runs in every launch
  if (threadIdx.x == 0 && V.runf != nullptr && V.sched != nullptr)
    V.runf[(size_t)(V.sched[0] & 1u) * V.runf_stride + p] = 1;
  const int l = (int)threadIdx.x - GF_NG;
  if (l >= M + GF_NG) return;
  const GfPatch P = V.patch[p];
  const GfCtl* C = V.ctl + P.scen;
  if (only_accepted && !C->accepted) return;
  // time of the ghost values: the macro step's start plus the substep about
  // to run (level subcycling), else the state's time
  const double tg = G.subcycle ? C->t + (double)C->sub_k * (C->dt_use / (double)G.sub_K) : C->t;
  const double Q = hydro_discharge(G, tg);
  if (!(Q > 0.0)) return;
  Geo<T> e(G, V);
  const int side = G.inflow_side;
  const bool xs = side <= 1;  // left or right side: the lines are rows
  const long long N = xs ? e.ny(P.level) : e.nx(P.level);
  const double d = xs ? e.dy(P.level) : e.dx(P.level);
  const double o = xs ? G.ylower : G.xlower;
  const long long base = (long long)(xs ? P.py : P.px) * M;
  const long long J = base + l;
  if (J < 0 || J >= N) return;
  const double ctr = o + ((double)J + 0.5) * d;
  if (!(ctr >= G.inflow_lo && ctr <= G.inflow_hi)) return;
  const double wd = G.inflow_width[P.level];
  if (!(wd > 0.0)) return;  // no line centre of this level in the segment
  const double q = Q / wd;
  const bool low = side == 0 || side == 2;
  const double sg = low ? 1.0 : -1.0;
  auto cell = [&](int a, int line) { return xs ? e.tix(a, line) : e.tix(line, a); };
  T* qq = e.qp(p, e.cur_of(p));
  const T* bb = e.bp(p);
  const int nf = xs ? 1 : 2, tf = xs ? 2 : 1;  // normal, tangential field
  const int ci = cell(low ? 0 : M - 1, l);
  const double hin = Geo<T>::DEV ? (double)qq[ci] - (double)bb[ci] : (double)qq[ci];
  const double qn = sg * (double)qq[nf * TT + ci];
  const double hg = inflow_depth(q, hin, qn, G.g, G.inflow_tau);
  const double mom[3] = {0.0, xs ? sg * q : 0.0, xs ? 0.0 : sg * q};
  for (int g = 1; g <= GF_NG; ++g) {
    const int c = cell(low ? -g : M - 1 + g, l);
    e.store(qq, c, hg, mom[1], mom[2], (double)bb[c]);
  }
  for (int end = 0; end < 2; ++end) {
    const int pside = xs ? 2 + end : end;
    const bool at = end == 0 ? base == 0 : base + M == N;
    if (!at) continue;
    const bool wall = G.bc[pside] == 0;
    for (int gl = 1; gl <= GF_NG; ++gl) {
      const int ls = wall ? (end == 0 ? gl - 1 : M - gl) : (end == 0 ? 0 : M - 1);
      if (ls != l) continue;
      const int lt = end == 0 ? -gl : M - 1 + gl;
      for (int g = 1; g <= GF_NG; ++g) {
        const int a = low ? -g : M - 1 + g;
        const int src = cell(a, l), dst = cell(a, lt);
        qq[dst] = qq[src];
        qq[nf * TT + dst] = qq[nf * TT + src];
        qq[tf * TT + dst] = wall ? -qq[tf * TT + src] : qq[tf * TT + src];
      }
    }
  }
}

// End of an accepted subcycled macro step (sub_k back at 0): a patch of
// level minlevel stepped once, from the current buffer into the other; its
// new state (tile and, in the deviation form, compensation terms) is
// copied back into the current buffer, where every finer level already is.
template <typename T>
__global__ void k_subcycle_sync(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V) {
  const int p = blockIdx.x;
  const GfPatch P = V.patch[p];
  const GfCtl* C = V.ctl + P.scen;
  if (P.level != G.minlevel || !C->accepted || C->sub_k != 0) return;
  Geo<T> e(G, V);
  const int cur = C->cur, M = G.M, TT = G.T * G.T;
  const T* s = e.qp(p, cur ^ 1);
  T* d = e.qp(p, cur);
  for (int k = threadIdx.x; k < 3 * TT; k += blockDim.x) d[k] = s[k];
  if constexpr (Geo<T>::DEV) {
    const float* ls = V.lof[cur ^ 1] + (size_t)p * 3 * M * M;
    float* ld = V.lof[cur] + (size_t)p * 3 * M * M;
    for (int k = threadIdx.x; k < 3 * M * M; k += blockDim.x) ld[k] = ls[k];
  }
}

// Ghost cells of one patch region without a same-level neighbour (a finer
// or coarser leaf covers it), one thread per cell: regs[k] = patch * 8 +
// region (left, right, bottom, top: 2 x M cells; corners: 2 x 2), filled
// from the leaves by the ghost operators, then copied to the physical-boundary
// ghost cells that mirror it.  Runs after each accepted step; the same-level
// regions and the other boundary ghosts are written by the patch step.
// Store (h, hu, hv) into ghost cell (i, j) of patch P's tile q (bed bt),
// mark the patch to run in the next launch if the cell holds water, and
// write the physical-boundary ghosts that mirror it (wall: reflected,
// normal momentum negated; extrapolation: the edge cell into both layers).
template <typename T>
__device__ void mark_and_mirror(const Geo<T>& e, const GfView& V, T* q, const GfPatch& P,
                                int p, int i, int j, bool water);

template <typename T>
__device__ void store_ghost(const Geo<T>& e, const GfView& V, T* q, const GfPatch& P, int p,
                            int i, int j, const double (&out)[3], double bt) {
  e.store(q, e.tix(i, j), out[0], out[1], out[2], bt);
  mark_and_mirror(e, V, q, P, p, i, j, out[0] > 0.0);
}

// The second half of store_ghost, once ghost cell (i, j) holds its value.
template <typename T>
__device__ void mark_and_mirror(const Geo<T>& e, const GfView& V, T* q, const GfPatch& P,
                                int p, int i, int j, bool water) {
  const GfGeom& G = e.G;
  const int M = G.M, TT = G.T * G.T;
  const int c = e.tix(i, j);
  // water written into this patch's ghost cells: it runs in the next launch
  // (the patch step has flipped the parity, so sched[0] selects it)
  if (water && V.runf != nullptr && V.sched != nullptr)
    V.runf[(size_t)(V.sched[0] & 1u) * V.runf_stride + p] = 1;
  const int nxp = G.mi << P.level, nyp = G.mj << P.level;
  int xm[2], ym[2], nx = 0, ny = 0;
  T fx = T(1), fy = T(1);
  if (P.px == 0 && (i == 0 || i == 1)) {
    if (G.bc[0] == 0) { xm[nx++] = -1 - i; fx = T(-1); }
    else if (i == 0) { xm[nx++] = -1; xm[nx++] = -2; }
  } else if (P.px == nxp - 1 && (i == M - 1 || i == M - 2)) {
    if (G.bc[1] == 0) { xm[nx++] = 2 * M - 1 - i; fx = T(-1); }
    else if (i == M - 1) { xm[nx++] = M; xm[nx++] = M + 1; }
  }
  if (P.py == 0 && (j == 0 || j == 1)) {
    if (G.bc[2] == 0) { ym[ny++] = -1 - j; fy = T(-1); }
    else if (j == 0) { ym[ny++] = -1; ym[ny++] = -2; }
  } else if (P.py == nyp - 1 && (j == M - 1 || j == M - 2)) {
    if (G.bc[3] == 0) { ym[ny++] = 2 * M - 1 - j; fy = T(-1); }
    else if (j == M - 1) { ym[ny++] = M; ym[ny++] = M + 1; }
  }
  if (nx == 0 && ny == 0) return;
  const T v0 = q[c], v1 = q[TT + c], v2 = q[2 * TT + c];
  auto put = [&](int a, int b, T su, T sv) {
    const int d = e.tix(a, b);
    q[d] = v0;
    q[TT + d] = su * v1;
    q[2 * TT + d] = sv * v2;
  };
  for (int a = 0; a < nx; ++a) put(xm[a], j, fx, T(1));
  for (int b = 0; b < ny; ++b) put(i, ym[b], T(1), fy);
  for (int a = 0; a < nx; ++a)
    for (int b = 0; b < ny; ++b) put(xm[a], ym[b], fx, fy);
}

// ------------------------------------------- level-change ghosts in FP32
//
// The FP32 deviation form's ghost operators, for forests without level
// subcycling: the same rules as value_at / interp_children / fill_cell, in
// FP32 arithmetic (FP64 runs at a small fraction of the FP32 rate on this
// part).  They carry the stored surface w = h + b - eta0 instead of the
// depth, so that the means and limited slopes of still water are exactly
// zero and a wet child's stored surface is the interpolated surface itself;
// the wet tests are the patch step's exact ones (wet_dev), so every wet/dry
// decision is the one the FP64 operators take on the same stored values.

// (w, hu, hv, b) of cell c of patch p in buffer cur
__device__ __forceinline__ void load_surf(const Geo<float>& e, int p, int cur, int c,
                                          float (&o)[4]) {
  const int TT = e.G.T * e.G.T;
  const float* q = e.V.qf[cur] + (size_t)p * 3 * TT;
  o[0] = q[c];
  o[1] = q[TT + c];
  o[2] = q[2 * TT + c];
  o[3] = e.V.bf[(size_t)p * TT + c];
}

// Four values of a cell and a lookup-error flag, returned by value from the
// out-of-line lookups below, so that no caller array has its address taken
// (which would put it in local memory).
struct Cell4 {
  float v[4];
  int err;
};

// value_at's composite in FP64 with the surface in place of the depth: the
// rare lookups (a leaf two levels coarser, cells two levels finer), kept out
// of line so that its FP64 arrays stay out of the callers' registers.
__device__ __noinline__ Cell4 surf_at_f64(const GfGeom* G, const GfView* V, int s, int L,
                                          long long I, long long J) {
  const Geo<float> e(*G, *V);
  double d[4];
  Cell4 r{};
  value_at(e, s, L, I, J, d, &r.err);
  r.v[0] = (float)(d[0] + d[3]);
  r.v[1] = (float)d[1];
  r.v[2] = (float)d[2];
  r.v[3] = (float)d[3];
  return r;
}

// (w, hu, hv, b) of cell (I, J) of level L: the leaf of level L or L - 1,
// the mean of four leaves of level L + 1, else the FP64 composite.
__device__ void surf_near_f32(const Geo<float>& e, int s, int cur, int L, long long I,
                              long long J, float (&o)[4], int* err) {
  for (int l = L; l >= L - 1 && l >= 0; --l) {
    const long long Il = I >> (L - l), Jl = J >> (L - l);
    const int p = e.leaf(s, l, Il, Jl);
    if (p >= 0) {
      load_surf(e, p, cur, e.local(Il, Jl), o);
      return;
    }
  }
  if (L + 1 <= e.G.maxlevel) {
    int pc[4];
    bool all = true;
    for (int ch = 0; ch < 4; ++ch) {
      pc[ch] = e.leaf(s, L + 1, 2 * I + (ch & 1), 2 * J + (ch >> 1));
      all = all && pc[ch] >= 0;
    }
    if (all) {
      float v[4][4];
      for (int ch = 0; ch < 4; ++ch)
        load_surf(e, pc[ch], cur, e.local(2 * I + (ch & 1), 2 * J + (ch >> 1)), v[ch]);
      for (int f = 0; f < 4; ++f)
        o[f] = 0.25f * ((v[0][f] + v[1][f]) + (v[2][f] + v[3][f]));
      return;
    }
  }
  const Cell4 r = surf_at_f64(&e.G, &e.V, s, L, I, J);
  for (int f = 0; f < 4; ++f) o[f] = r.v[f];
  if (r.err) *err = 1;
}

__device__ __forceinline__ float minmodf(float a, float b) {
  if (a * b <= 0.0f) return 0.0f;
  return fabsf(a) < fabsf(b) ? a : b;
}

__device__ __forceinline__ bool wet_f32(const GfGeom& G, float w, float b) {
  return gfk::wet_dev(w, b, G.drytol, G.drytolf, G.marginf);
}

// interp_children in FP32: out[b][a] = (w, hu, hv) of child (2 ic + a,
// 2 jc + b) of level L, whose bed is bs[b][a].
__device__ void interp_children_f32(const Geo<float>& e, int s, int cur, int L, long long ic,
                                    long long jc, const float (&bs)[2][2],
                                    float (&out)[2][2][3], int* err) {
  const GfGeom& G = e.G;
  const long long NXc = e.nx(L - 1), NYc = e.ny(L - 1);
  float nb[3][3][4];
  bool in[3][3], wt[3][3];
  // the neighbourhood in three straight-line passes, so that the loads of
  // the nine cells overlap: the leaves of level L - 1 holding them, the
  // values of those found, then the others (surf_near_f32's rarer cases)
  int pl[3][3];
#pragma unroll
  for (int dj = 0; dj < 3; ++dj)
#pragma unroll
    for (int di = 0; di < 3; ++di) {
      const long long x = ic + di - 1, y = jc + dj - 1;
      in[dj][di] = x >= 0 && y >= 0 && x < NXc && y < NYc;
      pl[dj][di] = in[dj][di] ? e.leaf(s, L - 1, x, y) : -1;
    }
#pragma unroll
  for (int dj = 0; dj < 3; ++dj)
#pragma unroll
    for (int di = 0; di < 3; ++di)
      if (pl[dj][di] >= 0) load_surf(e, pl[dj][di], cur, e.local(ic + di - 1, jc + dj - 1), nb[dj][di]);
#pragma unroll
  for (int dj = 0; dj < 3; ++dj)
#pragma unroll
    for (int di = 0; di < 3; ++di) {
      if (in[dj][di] && pl[dj][di] < 0)
        surf_near_f32(e, s, cur, L - 1, ic + di - 1, jc + dj - 1, nb[dj][di], err);
      wt[dj][di] = in[dj][di] && wet_f32(G, nb[dj][di][0], nb[dj][di][3]);
    }
  const float* qc = nb[1][1];
  if (!wt[1][1]) {
    // a dry coarse cell: its depth and momenta in every child
    const float hc = qc[0] - qc[3];
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        out[b][a][0] = hc + bs[b][a];
        out[b][a][1] = qc[1];
        out[b][a][2] = qc[2];
      }
    return;
  }
  bool allwet = true;
  for (int dj = 0; dj < 3; ++dj)
    for (int di = 0; di < 3; ++di)
      if (in[dj][di] && !wt[dj][di]) allwet = false;
  // limited slopes over the coarse cell: surface, then both momenta
  float g[3][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  if (allwet) {
    const bool hx = in[1][0] && in[1][2], hy = in[0][1] && in[2][1];
    for (int k = 0; k < 3; ++k) {
      if (hx) g[k][0] = minmodf(nb[1][2][k] - qc[k], qc[k] - nb[1][0][k]);
      if (hy) g[k][1] = minmodf(nb[2][1][k] - qc[k], qc[k] - nb[0][1][k]);
    }
  }
  // the four children: surface eta, depth d, linearly interpolated momenta m
  float eta[2][2], d[2][2], m[2][2][2];
  bool cw[2][2];
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) {
      const float sx = a ? 0.25f : -0.25f, sy = b ? 0.25f : -0.25f;
      eta[b][a] = allwet ? (qc[0] + sx * g[0][0]) + sy * g[0][1] : qc[0];
      const float h = eta[b][a] - bs[b][a];
      d[b][a] = h > 0.0f ? h : 0.0f;
      cw[b][a] = wet_f32(G, eta[b][a], bs[b][a]);
      for (int k = 0; k < 2; ++k)
        m[b][a][k] = (qc[k + 1] + sx * g[k + 1][0]) + sy * g[k + 1][1];
    }
  const float S = (d[0][0] + d[0][1]) + (d[1][0] + d[1][1]);
  bool split[2];
  for (int k = 0; k < 2; ++k) {
    split[k] = !allwet;
    if (allwet) {
      float lo = INFINITY, hi = -INFINITY;
      for (int dj = 0; dj < 3; ++dj)
        for (int di = 0; di < 3; ++di)
          if (in[dj][di]) {
            // velocities by the fast division (a few ulp): they only bound
            // the children's velocities
            const float u = __fdividef(nb[dj][di][k + 1], nb[dj][di][0] - nb[dj][di][3]);
            lo = fminf(lo, u);
            hi = fmaxf(hi, u);
          }
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a)
          if (cw[b][a]) {
            const float u = __fdividef(m[b][a][k], d[b][a]);
            if (u < lo || u > hi) split[k] = true;
          }
    }
  }
  const float rS = S > 0.0f ? __fdividef(1.0f, S) : 0.0f;
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) {
      // a child with water stores the interpolated surface itself
      out[b][a][0] = eta[b][a] > bs[b][a] ? eta[b][a] : bs[b][a];
      for (int k = 0; k < 2; ++k)
        out[b][a][k + 1] = !cw[b][a] ? 0.0f
                           : !split[k] ? m[b][a][k]
                                       : (4.0f * qc[k + 1]) * (d[b][a] * rS);
    }
}

// fill_cell in FP32: (w, hu, hv) of cell (I, J) of level L, whose parent's
// four children have the beds bs (bs[J & 1][I & 1] is this cell's).
__device__ void fill_cell_f32(const Geo<float>& e, int s, int cur, int L, long long I,
                              long long J, const float (&bs)[2][2], float (&out)[3],
                              int* err) {
  const float bt = bs[J & 1][I & 1];
  const int p = e.leaf(s, L, I, J);
  if (p >= 0) {
    float o4[4];
    load_surf(e, p, cur, e.local(I, J), o4);
    out[0] = o4[0];
    out[1] = o4[1];
    out[2] = o4[2];
    return;
  }
  bool coarser = false;
  for (int l = L - 1; l >= 0 && !coarser; --l)
    coarser = e.leaf(s, l, I >> (L - l), J >> (L - l)) >= 0;
  if (coarser) {
    float quad[2][2][3];
    interp_children_f32(e, s, cur, L, I >> 1, J >> 1, bs, quad, err);
    for (int f = 0; f < 3; ++f) out[f] = quad[J & 1][I & 1][f];
    return;
  }
  // the four finer cells: their leaves, their values, then the rarer cases
  float v[4][4];
  int pc[4];
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) pc[ch] = e.leaf(s, L + 1, 2 * I + (ch & 1), 2 * J + (ch >> 1));
#pragma unroll
  for (int ch = 0; ch < 4; ++ch)
    if (pc[ch] >= 0) load_surf(e, pc[ch], cur, e.local(2 * I + (ch & 1), 2 * J + (ch >> 1)), v[ch]);
  bool all = true;
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) {
    if (pc[ch] < 0)
      surf_near_f32(e, s, cur, L + 1, 2 * I + (ch & 1), 2 * J + (ch >> 1), v[ch], err);
    all = all && wet_f32(e.G, v[ch][0], v[ch][3]);
  }
  for (int f = 1; f < 3; ++f) out[f] = 0.25f * ((v[0][f] + v[1][f]) + (v[2][f] + v[3][f]));
  if (all) {
    // four wet children: their mean stored surface
    const float w = 0.25f * ((v[0][0] + v[1][0]) + (v[2][0] + v[3][0]));
    out[0] = w > bt ? w : bt;
  } else {
    float h[4];
    for (int ch = 0; ch < 4; ++ch) h[ch] = v[ch][0] - v[ch][3];
    out[0] = 0.25f * ((h[0] + h[1]) + (h[2] + h[3])) + bt;
  }
}

// Store (w, hu, hv) into ghost cell (i, j) of patch P's tile q (bed bt),
// then mark and mirror as store_ghost does.
__device__ void store_ghost_f32(const Geo<float>& e, const GfView& V, float* q,
                                const GfPatch& P, int p, int i, int j,
                                const float (&out)[3], float bt) {
  const int TT = e.G.T * e.G.T, c = e.tix(i, j);
  q[c] = out[0];
  q[TT + c] = out[1];
  q[2 * TT + c] = out[2];
  mark_and_mirror(e, V, q, P, p, i, j, out[0] > bt);
}

// Ghost cells of regions without a same-level neighbour, after each step.
// regs[0, nquad) are regions next to a coarser leaf: one thread per 2 x 2
// block of ghost cells (the children of one coarser cell, interpolated
// together: the same values as cell by cell, a quarter of the work);
// regs[nquad, nreg) are regions next to finer leaves: one thread per ghost
// cell (the mean of its four finer cells).  Region r of patch p: 0 left,
// 1 right, 2 bottom, 3 top (2 x M cells each), 4-7 the corners (2 x 2).
// F32: the FP32 operators above (FP32 forests without subcycling).
template <typename T, bool F32>
__global__ void __launch_bounds__(256, 1) k_ghost_other(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V,
                              const int* regs, int nquad, int nreg, int* errflag) {
  const int M = G.M;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nq_items = (long long)nquad * (M / 2);
  const bool quad = idx < nq_items;
  int code, k;
  if (quad) {
    code = regs[idx / (M / 2)];
    k = (int)(idx % (M / 2));
  } else {
    const long long r2 = idx - nq_items;
    if (r2 >= (long long)(nreg - nquad) * 2 * M) return;
    code = regs[nquad + r2 / (2 * M)];
    k = (int)(r2 % (2 * M));
  }
  const int p = code >> 3, r = code & 7;
  int i, j;
  if (quad) {
    // lower-left cell of the block (even, like the coarser cell's children)
    if (r >= 4 && k > 0) return;
    if (r == 0) { i = -2; j = 2 * k; }
    else if (r == 1) { i = M; j = 2 * k; }
    else if (r == 2) { i = 2 * k; j = -2; }
    else if (r == 3) { i = 2 * k; j = M; }
    else {
      i = (r == 4 || r == 6) ? -2 : M;
      j = (r == 4 || r == 5) ? -2 : M;
    }
  } else if (r < 4) {
    const int a = k % 2, b = k / 2;
    if (r == 0) { i = -2 + a; j = b; }
    else if (r == 1) { i = M + a; j = b; }
    else if (r == 2) { i = b; j = -2 + a; }
    else { i = b; j = M + a; }
  } else {
    if (k >= 4) return;
    const int a = k & 1, b = k >> 1;
    i = (r == 4 || r == 6) ? -2 + a : M + a;
    j = (r == 4 || r == 5) ? -2 + b : M + b;
  }
  const GfPatch P = V.patch[p];
  const GfCtl* C = V.ctl + P.scen;
  if (!C->accepted) return;
  Geo<T> e(G, V);
  T* q = e.qp(p, e.cur_of(p));
  const long long I = (long long)P.px * M + i, J = (long long)P.py * M + j;
  if constexpr (F32) {
    const int cur = C->cur;
    const float* bb = e.bp(p);
    float bs[2][2];
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) bs[b][a] = bb[e.tix((i & ~1) + a, (j & ~1) + b)];
    int err = 0;
    if (quad) {
      float out4[2][2][3];
      interp_children_f32(e, P.scen, cur, P.level, I >> 1, J >> 1, bs, out4, &err);
      if (err && errflag) *errflag = 1;
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a)
          store_ghost_f32(e, V, q, P, p, i + a, j + b, out4[b][a], bs[b][a]);
      return;
    }
    float out[3];
    fill_cell_f32(e, P.scen, cur, P.level, I, J, bs, out, &err);
    if (err && errflag) *errflag = 1;
    store_ghost_f32(e, V, q, P, p, i, j, out, bs[j & 1][i & 1]);
    return;
  }
  double bs[2][2];
  child_beds(e, e.bp(p), i, j, bs);
  int err = 0;
  if (quad) {
    double out4[2][2][3];
    interp_children(e, P.scen, P.level, I >> 1, J >> 1, bs, out4, &err);
    if (err && errflag) *errflag = 1;
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a)
        store_ghost(e, V, q, P, p, i + a, j + b, out4[b][a], bs[b][a]);
    return;
  }
  double out[3];
  fill_cell(e, P.scen, P.level, I, J, bs, out, &err);
  if (err && errflag) *errflag = 1;
  store_ghost(e, V, q, P, p, i, j, out, bs[j & 1][i & 1]);
}

// ------------------------------------------------------------ topography

// Bilinear interpolant of DEM k at (x, y), constant beyond its edges.
__device__ double dem_eval(const GfScenario& S, int k, double x, double y) {
  const int nx = S.dnx[k], ny = S.dny[k];
  double fx = (x - S.dx0[k]) / S.ddx[k], fy = (y - S.dy0[k]) / S.ddy[k];
  if (fx < 0.0) fx = 0.0;
  if (fx > (double)(nx - 1)) fx = (double)(nx - 1);
  if (fy < 0.0) fy = 0.0;
  if (fy > (double)(ny - 1)) fy = (double)(ny - 1);
  int i = (int)floor(fx), j = (int)floor(fy);
  if (i > nx - 2) i = nx - 2;
  if (j > ny - 2) j = ny - 2;
  if (i < 0) i = 0;
  if (j < 0) j = 0;
  const double ax = fx - (double)i, ay = fy - (double)j;
  const double* z = S.dem[k];
  const double z00 = z[i + (size_t)j * nx], z10 = z[i + 1 + (size_t)j * nx];
  const double z01 = z[i + (size_t)(j + 1) * nx];
  const double z11 = z[i + 1 + (size_t)(j + 1) * nx];
  return (1.0 - ay) * ((1.0 - ax) * z00 + ax * z10) +
         ay * ((1.0 - ax) * z01 + ax * z11);
}

// Composite interpolant of the scenario's DEMs (Sec. 6.2): the first DEM in
// priority order whose node-to-node extent holds the point; outside every
// extent the last (coarsest) one's, constant beyond its edges.
__device__ double dems_eval(const GfScenario& S, double x, double y) {
  int k = 0;
  for (; k < S.ndem; ++k) {
    const double xe = S.dx0[k] + (double)(S.dnx[k] - 1) * S.ddx[k];
    const double ye = S.dy0[k] + (double)(S.dny[k] - 1) * S.ddy[k];
    if (x >= S.dx0[k] && x <= xe && y >= S.dy0[k] && y <= ye) break;
  }
  return dem_eval(S, k < S.ndem ? k : S.ndem - 1, x, y);
}

// The smallest break point above v along one axis (xaxis: x), at most b:
// the node lines of every DEM (node indices 0..n-1).  The extents' edges are
// node lines, so between consecutive break points every DEM is either
// bilinear or absent.
__device__ double next_break(const GfScenario& S, bool xaxis, double v, double b) {
  double best = b;
  for (int k = 0; k < S.ndem; ++k) {
    const double o = xaxis ? S.dx0[k] : S.dy0[k];
    const double d = xaxis ? S.ddx[k] : S.ddy[k];
    const int n = xaxis ? S.dnx[k] : S.dny[k];
    double f = floor((v - o) / d) + 1.0;
    if (f < 0.0) f = 0.0;
    if (f > (double)n) f = (double)n;
    int i = (int)f;
    while (i > 0 && o + (double)(i - 1) * d > v) --i;
    while (i <= n - 1 && !(o + (double)i * d > v)) ++i;
    if (i <= n - 1) {
      const double xn = o + (double)i * d;
      if (xn < best) best = xn;
    }
  }
  return best;
}

// Exact average over [xa,xb]x[ya,yb] of the composite interpolant: the node
// lines of all DEMs cut the cell into pieces on which it is bilinear; each
// piece contributes its area times its midpoint value.  Rows of pieces in
// increasing y, pieces of a row in increasing x.
__device__ double dem_average(const GfScenario& S, double xa, double xb,
                              double ya, double yb) {
  double sum = 0.0;
  double y0 = ya;
  while (y0 < yb) {
    const double y1 = next_break(S, false, y0, yb);
    double x0 = xa;
    while (x0 < xb) {
      const double x1 = next_break(S, true, x0, xb);
      const double xm = 0.5 * (x0 + x1), ym = 0.5 * (y0 + y1);
      const double w = (x1 - x0) * (y1 - y0);
      sum += w * dems_eval(S, xm, ym);
      x0 = x1;
    }
    y0 = y1;
  }
  return sum / ((xb - xa) * (yb - ya));
}

template <typename T>
__global__ void k_topo(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V, int first,
                       const int* list) {
  const int p = list ? list[blockIdx.x] : first + blockIdx.x;
  const GfPatch P = V.patch[p];
  Geo<T> e(G, V);
  const int M = G.M, T_ = G.T, TT = T_ * T_;
  T* b = e.bp(p);
  const GfScenario& S = V.scen[P.scen];
  // a tile already computed for this position (the same DEMs and eta0):
  // copied, bit for bit what the computation below gives
  const size_t slot = (size_t)S.lut_off + G.lut_lev_off[P.level] + P.px +
                      (size_t)P.py * ((size_t)G.mi << P.level);
  T* cache = V.bcache ? static_cast<T*>(V.bcache) + slot * TT : nullptr;
  if (cache && V.bvalid[slot]) {
    for (int k = threadIdx.x; k < TT; k += blockDim.x) b[k] = cache[k];
    return;
  }
  const long long NX = e.nx(P.level), NY = e.ny(P.level);
  const double dx = e.dx(P.level), dy = e.dy(P.level);
  for (int k = threadIdx.x; k < TT; k += blockDim.x) {
    const int i = k % T_ - GF_NG, j = k / T_ - GF_NG;
    const long long I = (long long)P.px * M + i, J = (long long)P.py * M + j;
    double v = 0.0;
    if (I >= 0 && J >= 0 && I < NX && J < NY && S.ndem > 0) {
      const double xa = G.xlower + (double)I * dx;
      const double xb = G.xlower + (double)(I + 1) * dx;
      const double ya = G.ylower + (double)J * dy;
      const double yb = G.ylower + (double)(J + 1) * dy;
      v = dem_average(S, xa, xb, ya, yb);
    }
    // the deviation form keeps the bed relative to the reference surface
    b[k] = Geo<T>::DEV ? (T)(v - S.eta0) : (T)v;
  }
  __syncthreads();
  tile_bc<T>(e, P, nullptr, b, 1);
  if (cache) {
    // no other CTA of this launch has this position; later launches see the
    // tile and the flag after this kernel ends
    __syncthreads();
    for (int k = threadIdx.x; k < TT; k += blockDim.x) cache[k] = b[k];
    if (threadIdx.x == 0) V.bvalid[slot] = 1;
  }
}

// Regrid transfer: every interior cell of every new patch from the old
// forest by the ghost-cell operators (copy, average, interpolation).  The
// FP32 compensation terms of new cells start at zero.
template <typename T>
__global__ void k_regrid_fill(const __grid_constant__ GfGeom G, const __grid_constant__ GfView O,
                              const __grid_constant__ GfView N,
                              int* errflag, const int* list) {
  const int p = list ? list[blockIdx.x] : blockIdx.x;
  const GfPatch P = N.patch[p];
  Geo<T> eo(G, O), en(G, N);
  const int M = G.M, T_ = G.T;
  const int dst = 1 - O.ctl[P.scen].cur;
  T* q = en.qp(p, dst);
  const T* bn = en.bp(p);
  int err = 0;
  // by blocks of 2 x 2 cells (the children of one cell of level L - 1, all
  // in this patch): a block that the old forest covers with a coarser leaf
  // is interpolated in one go, any other cell by cell, with the same values
  const int H = M / 2;
  for (int k = threadIdx.x; k < H * H; k += blockDim.x) {
    const int i0 = 2 * (k % H), j0 = 2 * (k / H);
    const long long I0 = (long long)P.px * M + i0, J0 = (long long)P.py * M + j0;
    double bs[2][2];
    child_beds(en, bn, i0, j0, bs);
    double out4[2][2][3];
    bool coarse = P.level > 0 && eo.leaf(P.scen, P.level, I0, J0) < 0;
    if (coarse) {
      coarse = false;
      for (int l = P.level - 1; l >= 0 && !coarse; --l)
        coarse = eo.leaf(P.scen, l, I0 >> (P.level - l), J0 >> (P.level - l)) >= 0;
    }
    if (coarse) {
      interp_children(eo, P.scen, P.level, I0 >> 1, J0 >> 1, bs, out4, &err);
    } else {
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a)
          fill_cell(eo, P.scen, P.level, I0 + a, J0 + b, bs, out4[b][a], &err);
    }
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int i = i0 + a, j = j0 + b;
        const int c = (i + GF_NG) + (j + GF_NG) * T_;
        en.store(q, c, out4[b][a][0], out4[b][a][1], out4[b][a][2], bs[b][a]);
        if constexpr (Geo<T>::DEV) {
          const int kc = i + j * M;
          float* lo = N.lof[dst] + (size_t)p * 3 * M * M;
          lo[kc] = 0.0f;
          lo[M * M + kc] = 0.0f;
          lo[2 * M * M + kc] = 0.0f;
        }
      }
  }
  if (err && errflag) *errflag = 1;
}

// Regrid transfer of a patch that is a leaf of both forests: its bed, state
// (ghosts included) and compensation terms are copied from its old slot;
// pairs[k] = (new index, old index).
template <typename T>
__global__ void k_regrid_keep(const __grid_constant__ GfGeom G, const __grid_constant__ GfView O,
                              const __grid_constant__ GfView N, const int2* pairs) {
  const int2 pr = pairs[blockIdx.x];
  const int pn = pr.x, po = pr.y;
  const GfPatch P = N.patch[pn];
  Geo<T> eo(G, O), en(G, N);
  const int M = G.M, TT = G.T * G.T;
  const int src = O.ctl[P.scen].cur, dst = 1 - src;
  const T* qo = eo.qp(po, src);
  T* qn = en.qp(pn, dst);
  const T* bo = eo.bp(po);
  T* bn = en.bp(pn);
  for (int k = threadIdx.x; k < TT; k += blockDim.x) {
    bn[k] = bo[k];
    qn[k] = qo[k];
    qn[TT + k] = qo[TT + k];
    qn[2 * TT + k] = qo[2 * TT + k];
  }
  if constexpr (Geo<T>::DEV) {
    const float* lo = O.lof[src] + (size_t)po * 3 * M * M;
    float* ln = N.lof[dst] + (size_t)pn * 3 * M * M;
    for (int k = threadIdx.x; k < 3 * M * M; k += blockDim.x) ln[k] = lo[k];
  }
}

// Bring every patch's latest state into buffer `target`: a patch whose
// scenario holds it in the other buffer has its tile (ghosts included) and
// compensation terms copied over.  Patch slots are shared by all scenarios,
// so a regrid, which writes every new slot into the buffer opposite the
// latest one, needs that buffer to be the same for every scenario.
template <typename T>
__global__ void k_align_buffers(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V,
                                int target) {
  const int p = blockIdx.x;
  const GfPatch P = V.patch[p];
  const int src = V.ctl[P.scen].cur;
  if (src == target) return;
  Geo<T> e(G, V);
  const int M = G.M, TT = G.T * G.T;
  const T* qs = e.qp(p, src);
  T* qd = e.qp(p, target);
  for (int k = threadIdx.x; k < 3 * TT; k += blockDim.x) qd[k] = qs[k];
  if constexpr (Geo<T>::DEV) {
    const float* ls = V.lof[src] + (size_t)p * 3 * M * M;
    float* ld = V.lof[target] + (size_t)p * 3 * M * M;
    for (int k = threadIdx.x; k < 3 * M * M; k += blockDim.x) ld[k] = ls[k];
  }
}

// Bound what one cell asks for by the refinement regions holding its centre
// (Sec. 4.1 criterion 4, Sec. 6.4): rmin, rmax the largest minimum and the
// largest maximum (rmax < 0: none holds it).  The level the cell asks for
// (L + 1 for r = 2, L for r = 1, L - 1 otherwise, or the grade's level cgl
// if higher) is moved into [rmin, rmax] and becomes r (cgl then -1); netw
// collects the bounded level of a refinement request at this cell (the
// learned tagger's request), L + 1 where no region holds it.
__device__ __forceinline__ void cov_region_bound(int L, int& r, int& cgl, int& netw,
                                                 int rmin, int rmax) {
  if (rmax < 0) {
    netw = L + 1 > netw ? L + 1 : netw;
    return;
  }
  int want = r == 2 ? L + 1 : (r == 1 ? L : L - 1);
  if (cgl > want) want = cgl;
  if (want < rmin) want = rmin;
  if (want > rmax) want = rmax;
  r = want > L ? 2 : (want == L ? 1 : 0);
  cgl = -1;
  int nw = L + 1;
  if (nw < rmin) nw = rmin;
  if (nw > rmax) nw = rmax;
  netw = nw > netw ? nw : netw;
}

// Plain tagger (Sec. 4.1 criteria 1 to 5; Sec. 6.4), with the refinement
// regions active at the scenario's time bounding what each cell asks for.
template <typename T>
__global__ void k_tags(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V,
                       const GfTagOut O) {
  const int p = blockIdx.x;
  const GfPatch P = V.patch[p];
  Geo<T> e(G, V);
  const int M = G.M;
  const int L = P.level;
  const int cur = V.ctl[P.scen].cur;
  // per-level cell sizes from the host's table (the same division as
  // Geo::dx); surfaces are compared with eta0, relative to which the
  // deviation form stores them
  const double sdx = G.dxl[L], sdy = G.dyl[L];
  const double eref = Geo<T>::DEV ? 0.0 : V.scen[P.scen].eta0;
  auto xcen = [&](int i) { return G.xlower + ((double)((long long)P.px * M + i) + 0.5) * sdx; };
  auto ycen = [&](int j) { return G.ylower + ((double)((long long)P.py * M + j) + 0.5) * sdy; };
  // the source box and the regions against the patch's first and last cell
  // centres (the centres grow with the index, so the per-cell test is needed
  // only where an edge crosses the patch): from the host's per-patch table,
  // or computed once by thread 0 (FP64 is slow on this part) and shared;
  // without the table every region is tested per cell
  unsigned box;  // bits 0-1: 1 the box misses the patch, 2 covers it
  if (V.pbox != nullptr) {
    box = V.pbox[p];
  } else {
    __shared__ unsigned sbox;
    if (threadIdx.x == 0) {
      const double x0 = xcen(0), x1 = xcen(M - 1), y0 = ycen(0), y1 = ycen(M - 1);
      const bool none = x1 < G.src_box[0] || x0 > G.src_box[1] || y1 < G.src_box[2] ||
                        y0 > G.src_box[3];
      const bool all = x0 >= G.src_box[0] && x1 <= G.src_box[1] && y0 >= G.src_box[2] &&
                       y1 <= G.src_box[3];
      sbox = (none ? 1u : 0u) | (all ? 2u : 0u);
    }
    __syncthreads();
    box = sbox;
  }
  const bool box_none = (box & 1u) != 0u, box_all = (box & 2u) != 0u;
  const int rbox = L < G.src_level ? 2 : 1;  // a cell in the box asks this
  // refinement regions active now: those covering the patch bound every
  // cell alike (cov_min, cov_max), those crossing it are tested per cell
  const double tnow = V.ctl[P.scen].t;
  int cov_min = -1, cov_max = -1;
  unsigned cross = 0u;
  for (int r = 0; r < G.nregions; ++r) {
    if (!(tnow >= G.rt0[r] && tnow <= G.rt1[r])) continue;
    const unsigned cl = V.pbox != nullptr ? (box >> (2 + 2 * r)) & 3u : 0u;
    if (cl == 1u) continue;
    if (cl == 2u) {
      cov_min = G.rminl[r] > cov_min ? G.rminl[r] : cov_min;
      cov_max = G.rmaxl[r] > cov_max ? G.rmaxl[r] : cov_max;
    } else {
      cross |= 1u << r;
    }
  }
  const bool regs = cov_max >= 0 || cross != 0u;
  int m = box_all && !regs ? rbox : 0;
  int gl = -1;    // the highest level a flow grade asks for (criterion 5)
  int netw = -1;  // with regions: the highest level the learned tagger may ask for
  // Cell (i, j) asks r (2 refine, 1 keep, 0 nothing) and grade level cgl
  // from the criteria; then the source box, then the regions holding its
  // centre move the level it asks for into their bounds.
  auto finish_cell = [&](int i, int j, int r, int cgl) {
    const bool box_cell = !box_none && !box_all;
    double xc = 0.0, yc = 0.0;
    if (box_cell || cross != 0u) {
      xc = xcen(i);
      yc = ycen(j);
    }
    // (without regions a box covering the patch is already in m)
    const bool in_box = box_cell ? (xc >= G.src_box[0] && xc <= G.src_box[1] &&
                                    yc >= G.src_box[2] && yc <= G.src_box[3])
                                 : box_all && regs;
    if (in_box) {
      if (rbox == 2) r = 2;
      else if (r < 1) r = 1;
    }
    if (regs) {
      int rmin = cov_min, rmax = cov_max;
      for (unsigned bits = cross; bits != 0u; bits &= bits - 1u) {
        const int k = __ffs(bits) - 1;
        if (xc >= G.rx0[k] && xc <= G.rx1[k] && yc >= G.ry0[k] && yc <= G.ry1[k]) {
          rmin = G.rminl[k] > rmin ? G.rminl[k] : rmin;
          rmax = G.rmaxl[k] > rmax ? G.rmaxl[k] : rmax;
        }
      }
      cov_region_bound(L, r, cgl, netw, rmin, rmax);
    }
    m = r > m ? r : m;
    gl = cgl > gl ? cgl : gl;
  };
  if constexpr (Geo<T>::DEV) {
    // FP32 deviation form: up to four cells per thread at once, so that a
    // block waits for two rounds of loads (surfaces and beds, then the
    // momenta of the cells deep enough to be tested) instead of one per
    // cell; stop once any cell asks for refinement
    constexpr int U = 4;
    const float* q = e.qp(p, cur);
    const float* bq = e.bp(p);
    const int TT = G.T * G.T;
    for (int k0 = 0; m < 2 && k0 < M * M; k0 += U * (int)blockDim.x) {
      float w[U], b[U], hu[U], hv[U];
      int c[U];
      bool ok[U], deep[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = k0 + u * (int)blockDim.x + (int)threadIdx.x;
        ok[u] = k < M * M;
        c[u] = ok[u] ? e.tix(k % M, k / M) : 0;
        w[u] = ok[u] ? q[c[u]] : 0.0f;
        b[u] = ok[u] ? bq[c[u]] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        deep[u] = ok[u] && w[u] - b[u] > G.tag_depthf;
        hu[u] = deep[u] ? q[TT + c[u]] : 0.0f;
        hv[u] = deep[u] ? q[2 * TT + c[u]] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!ok[u]) continue;
        const int k = k0 + u * (int)blockDim.x + (int)threadIdx.x;
        int r = 0, cgl = -1;
        if (deep[u]) {
          // depth w - b, speed test without a division, surface deviation
          // |w| (one mismatch with the FP64 criterion is possible at a
          // threshold tie; counted in the tests)
          const float h = w[u] - b[u];
          const float st = G.tag_speedf * h;
          const float f2 = hu[u] * hu[u] + hv[u] * hv[u];
          if (f2 > st * st || fabsf(w[u]) > G.tag_detaf || f2 > G.tag_fluxf * G.tag_fluxf) r = 2;
          for (int g = 0; g < G.ngrades; ++g) {
            const float tv = G.grade_valuef[g];
            const bool over = G.grade_kind[g] == 0 ? h > tv : f2 > (tv * h) * (tv * h);
            if (over && G.grade_level[g] > cgl) cgl = G.grade_level[g];
          }
        }
        finish_cell(k % M, k / M, r, cgl);
      }
      if (__syncthreads_or(m == 2)) m = 2;
    }
  } else if (m < 2) {
    // cells in rounds of blockDim; stop once any cell asks for refinement
    for (int k0 = 0; k0 < M * M; k0 += blockDim.x) {
      const int k = k0 + threadIdx.x;
      if (k < M * M) {
        const int i = k % M, j = k / M;
        const int c = e.tix(i, j);
        int r = 0, cgl = -1;
        double v4[4];
        e.load(p, cur, c, v4);
        const double h = v4[0];
        if (h > G.tag_depth) {
          const double u = v4[1] / h, v = v4[2] / h;
          const double sp = sqrt(u * u + v * v);
          const double eta = h + v4[3];
          const double flux = sqrt(v4[1] * v4[1] + v4[2] * v4[2]);
          if (sp > G.tag_speed || fabs(eta - eref) > G.tag_deta) r = 2;
          if (flux > G.tag_flux) r = 2;
          for (int g = 0; g < G.ngrades; ++g) {
            const double val = G.grade_kind[g] == 0 ? h : sp;
            if (val > G.grade_value[g] && G.grade_level[g] > cgl) cgl = G.grade_level[g];
          }
        }
        finish_cell(i, j, r, cgl);
      }
      if (__syncthreads_or(m == 2)) {
        m = 2;
        break;
      }
    }
  }
  // criterion 5 matters only when no cell asks for full refinement
  gl = __reduce_max_sync(0xffffffffu, gl);
  netw = __reduce_max_sync(0xffffffffu, netw);
  __shared__ int wg[32], wn[32];
  if ((threadIdx.x & 31) == 0) {
    wg[threadIdx.x >> 5] = gl;
    wn[threadIdx.x >> 5] = netw;
  }
  m = __reduce_max_sync(0xffffffffu, m);
  __shared__ int wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int mm = 0, gmax = -1, nmax = -1;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      mm = wm[w] > mm ? wm[w] : mm;
      gmax = wg[w] > gmax ? wg[w] : gmax;
      nmax = wn[w] > nmax ? wn[w] : nmax;
    }
    // a flow grade above the patch's level is a request for refinement
    const bool grade_up = mm < 2 && gmax > L;
    // the plain criterion's own verdict: recorded, turned into training
    // labels, or counted as a miss where the patch could still be refined
    const int raw = grade_up ? 2 : mm;
    if (O.raw) O.raw[p] = (uint8_t)raw;
    if (O.label && raw == 2) O.label[p] = 1.0f;
    if (O.misses && raw == 2 && L < G.maxlevel) atomicAdd(O.misses, 1u);
    // learned tags add refinement (or keep a fine patch) on top of it: a
    // request for level L + 1 at every cell, bounded by the regions like
    // the criterion's own (nmax: the highest bounded level; every cell was
    // visited unless a cell already asked for refinement)
    const bool learned = O.logit && O.logit[p] > O.logit_thr;
    if (learned) {
      if (!regs || nmax > L) mm = 2;
      else if (nmax == L && mm < 1) mm = 1;
    }
    uint8_t f;
    if (mm == 2) f = L < G.maxlevel ? 1 : 0;
    else if (gmax > L) f = 1;
    else if (gmax == L || mm == 1) f = 0;
    else f = L > G.minlevel ? 2 : 0;
    if (O.flags) O.flags[p] = f;
  }
}

// Gauges (Sec. 5.1 control points, Sec. 6.5): bilinear in the finest leaf,
// ghosts included; arrival at the first sample with h > 1 cm.
// Stencil of gauge g of scenario S: the finest leaf holding the point, and
// the lower-left cell (i0, j0 in [-1, M-1], ghosts included) and weights of
// the bilinear interpolation between cell centres.
template <typename T>
__device__ GfGaugeRef gauge_locate(const Geo<T>& e, const GfGeom& G, const GfView& V,
                                   const GfScenario& S, int g) {
  const double x = S.gxy[2 * g], y = S.gxy[2 * g + 1];
  int p = -1, L = 0;
  for (int l = G.maxlevel; l >= 0 && p < 0; --l) {
    const double pw = (G.xupper - G.xlower) / (double)(G.mi << l);
    const double ph = (G.yupper - G.ylower) / (double)(G.mj << l);
    long long Pq = (long long)floor((x - G.xlower) / pw);
    long long Qq = (long long)floor((y - G.ylower) / ph);
    const long long w = (long long)G.mi << l, hgt = (long long)G.mj << l;
    if (Pq < 0) Pq = 0;
    if (Qq < 0) Qq = 0;
    if (Pq >= w) Pq = w - 1;
    if (Qq >= hgt) Qq = hgt - 1;
    const int k = V.lut[S.lut_off + G.lut_lev_off[l] + Pq + Qq * w];
    if (k >= 0) { p = k; L = l; }
  }
  GfGaugeRef r{-1, 0, 0.0, 0.0};
  if (p < 0) return r;
  const GfPatch P = V.patch[p];
  const int M = G.M;
  const double fx = (x - G.xlower) / e.dx(L) - 0.5 - (double)((long long)P.px * M);
  const double fy = (y - G.ylower) / e.dy(L) - 0.5 - (double)((long long)P.py * M);
  int i0 = (int)floor(fx), j0 = (int)floor(fy);
  if (i0 < -1) i0 = -1;
  if (j0 < -1) j0 = -1;
  if (i0 > M - 1) i0 = M - 1;
  if (j0 > M - 1) j0 = M - 1;
  r.p = p;
  r.c = e.tix(i0, j0);
  r.ax = fx - (double)i0;
  r.ay = fy - (double)j0;
  return r;
}

template <typename T>
__global__ void k_gauge_refs(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V) {
  const int s = blockIdx.y;
  const GfScenario S = V.scen[s];
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S.ngauge) return;
  Geo<T> e(G, V);
  const GfGaugeRef r = gauge_locate(e, G, V, S, g);
  S.gref[g] = r;
  if (r.p >= 0 && V.gflag != nullptr) V.gflag[r.p] = 1;
}

// Gauges (Sec. 5.1 control points, Sec. 6.5): bilinear in the finest leaf,
// ghosts included; arrival at the first sample with h > 1 cm.  During a
// run the patch step samples each gauge from its staged tile; this kernel
// takes the samples outside the step (registration, end of a run).
template <typename T>
__global__ void k_gauges(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V, int only_accepted) {
  const int s = blockIdx.y;
  const GfScenario S = V.scen[s];
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S.ngauge) return;
  const GfCtl* C = V.ctl + s;
  if (only_accepted && !C->accepted) return;
  Geo<T> e(G, V);
  const GfGaugeRef r = gauge_locate(e, G, V, S, g);
  double* o = S.gout + 5 * g;
  o[0] = C->t;
  if (r.p < 0) { o[1] = o[2] = o[3] = o[4] = 0.0; return; }
  const int p = r.p, T_ = G.T;
  double c4[4][4];
  e.load(p, C->cur, r.c, c4[0]);
  e.load(p, C->cur, r.c + 1, c4[1]);
  e.load(p, C->cur, r.c + T_, c4[2]);
  e.load(p, C->cur, r.c + T_ + 1, c4[3]);
  const double eoff = Geo<T>::DEV ? S.eta0 : 0.0;
  double v[4];
  for (int f = 0; f < 4; ++f) {
    if (f < 3)
      v[f] = gf_bilinear(c4[0][f], c4[1][f], c4[2][f], c4[3][f], r.ax, r.ay);
    else
      v[f] = gf_bilinear(c4[0][0] + c4[0][3], c4[1][0] + c4[1][3], c4[2][0] + c4[2][3],
                         c4[3][0] + c4[3][3], r.ax, r.ay);
  }
  o[1] = v[0]; o[2] = v[1]; o[3] = v[2]; o[4] = v[3] + eoff;
  if (S.garr[g] < 0.0 && v[0] > 0.01) S.garr[g] = C->t;
}

// Volume per patch (fixed-order block tree), then per scenario.
template <typename T>
__global__ void k_patch_mass(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V, double* pmass) {
  const int p = blockIdx.x;
  const GfPatch P = V.patch[p];
  Geo<T> e(G, V);
  const int M = G.M;
  const int cur = V.ctl[P.scen].cur;
  double v = 0.0;
  for (int k = threadIdx.x; k < M * M; k += blockDim.x) {
    double c4[4];
    e.load(p, cur, e.tix(k % M, k / M), c4);
    v += c4[0];
  }
  __shared__ double red[256];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) pmass[p] = red[0] * (e.dx(P.level) * e.dy(P.level));
}

__global__ void k_scen_mass(const GfScenario* sc, const double* pmass,
                            double* smass) {
  const int s = blockIdx.x;
  const int off = sc[s].poff, n = sc[s].pcount;
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += pmass[off + k];
  __shared__ double red[256];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) smass[s] = red[0];
}

// Staging between tiles and dense field-major interior arrays
// [field][count][M][M] in FP64: fields h, hu, hv, b for packing; h, hu, hv
// for unpacking (the deviation form converts w = h + b - eta0 and clears the
// compensation terms).
template <typename T>
__global__ void k_pack(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V, int first, double* out,
                       int cur) {
  const int p = first + blockIdx.x;
  Geo<T> e(G, V);
  const int M = G.M, MM = M * M;
  const size_t plane = (size_t)gridDim.x * MM;
  const double eoff = Geo<T>::DEV ? V.scen[V.patch[p].scen].eta0 : 0.0;
  for (int k = threadIdx.x; k < MM; k += blockDim.x) {
    const int c = (k % M + GF_NG) + (k / M + GF_NG) * G.T;
    double c4[4];
    e.load(p, cur, c, c4);
    const size_t o = (size_t)blockIdx.x * MM + k;
    out[o] = c4[0];
    out[plane + o] = c4[1];
    out[2 * plane + o] = c4[2];
    out[3 * plane + o] = c4[3] + eoff;
  }
}

template <typename T>
__global__ void k_unpack(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V, int first,
                         const double* in, int cur) {
  const int p = first + blockIdx.x;
  Geo<T> e(G, V);
  const int M = G.M, MM = M * M;
  const size_t plane = (size_t)gridDim.x * MM;
  T* q = e.qp(p, cur);
  const T* b = e.bp(p);
  for (int k = threadIdx.x; k < MM; k += blockDim.x) {
    const int c = (k % M + GF_NG) + (k / M + GF_NG) * G.T;
    const size_t o = (size_t)blockIdx.x * MM + k;
    e.store(q, c, in[o], in[plane + o], in[2 * plane + o], (double)b[c]);
    if constexpr (Geo<T>::DEV) {
      float* lo = V.lof[cur] + (size_t)p * 3 * MM;
      lo[k] = 0.0f;
      lo[MM + k] = 0.0f;
      lo[2 * MM + k] = 0.0f;
    }
  }
}

// Input features of the learned refinement predictor on an 18 x 18 pixel
// grid.  The 16 x 16 inner pixels are means over f x f blocks of the patch
// interior (f = M / 16); each ring pixel is the mean over the band of cells
// of the same level that lies beyond the patch edge next to it, M / 2 cells
// deep (f cells wide along the edge, M / 2 x M / 2 at the corners), read from
// whichever leaves cover it; cells outside the domain are left out.  This
// lets the network see water up to half a patch away.  Channels: h, hu, hv,
// bed minus the mean interior bed, each divided by its scale, then level /
// 4; channels 5..15 are zero.  Output [count][324][16] BF16, pixel = Y * 18
// + X.
struct FeatScale {
  float s[4];
};

// Composite value at cell (I, J) of level L next to a patch of that level.
// In a 2:1 balanced forest the leaf holding such a cell is almost always of
// level L, L - 1 or L + 1, so those are looked up first (one or two lookups
// instead of value_at's walk down to level 0 before it tries finer leaves);
// anything else goes to value_at.  The leaf holding a cell is unique, so the
// result is value_at's, computed with the same operations.
template <typename T>
__device__ void value_near(const Geo<T>& e, int s, int L, long long I, long long J,
                           double (&out)[4], int* err) {
  for (int l = L; l >= L - 1 && l >= 0; --l) {
    const long long Il = I >> (L - l), Jl = J >> (L - l);
    const int p = e.leaf(s, l, Il, Jl);
    if (p >= 0) {
      const int c = e.local(Il, Jl);
      e.load_now_s(p, s, c, out);
      return;
    }
  }
  if (L + 1 <= e.G.maxlevel) {
    int pc[4];
    bool all = true;
    for (int ch = 0; ch < 4; ++ch) {
      pc[ch] = e.leaf(s, L + 1, 2 * I + (ch & 1), 2 * J + (ch >> 1));
      all = all && pc[ch] >= 0;
    }
    if (all) {
      double v[4][4];
      for (int ch = 0; ch < 4; ++ch) {
        const long long Ic = 2 * I + (ch & 1), Jc = 2 * J + (ch >> 1);
        e.load_now_s(pc[ch], s, e.local(Ic, Jc), v[ch]);
      }
      for (int f = 0; f < 4; ++f)
        out[f] = 0.25 * ((v[0][f] + v[1][f]) + (v[2][f] + v[3][f]));
      return;
    }
  }
  value_at(e, s, L, I, J, out, err);
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One pixel of the network input: 16 BF16 channels (the four fields, the
// level channel, zeros), written as two 16-byte stores (the pixel's 32
// bytes are 32-byte aligned); each channel rounded to nearest as one
// conversion would.
__device__ __forceinline__ void store_pixel(__nv_bfloat16* op, const float (&v)[4], float lev) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
  const __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
  const __nv_bfloat162 c = __floats2bfloat162_rn(lev, 0.0f);
  uint4 lo;
  lo.x = *reinterpret_cast<const unsigned*>(&a);
  lo.y = *reinterpret_cast<const unsigned*>(&b);
  lo.z = *reinterpret_cast<const unsigned*>(&c);
  lo.w = 0u;
  uint4* o4 = reinterpret_cast<uint4*>(op);
  o4[0] = lo;
  o4[1] = make_uint4(0u, 0u, 0u, 0u);
}

template <typename T>
__global__ void k_cnn_features(const __grid_constant__ GfGeom G,
                               const __grid_constant__ GfView V, int first,
                               FeatScale sc, __nv_bfloat16* out) {
  const int p = first + blockIdx.x;
  const GfPatch P = V.patch[p];
  Geo<T> e(G, V);
  const int M = G.M, f = M / 16, W = M / 2;
  const int cur = V.ctl[P.scen].cur;
  __shared__ double part[256];
  __shared__ double bmean;
  double bs = 0.0;
  for (int k = threadIdx.x; k < M * M; k += blockDim.x) {
    double c4[4];
    e.load(p, cur, e.tix(k % M, k / M), c4);
    bs += c4[3];
  }
  part[threadIdx.x] = bs;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) bmean = part[0] / (double)(M * M);
  __syncthreads();
  __nv_bfloat16* o = out + (size_t)blockIdx.x * 324 * 16;
  const long long NX = e.nx(P.level), NY = e.ny(P.level);
  const long long I0 = (long long)P.px * M, J0 = (long long)P.py * M;
  int err = 0;
  auto emit = [&](int X, int Y, const double (&acc)[4], int cnt) {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (cnt > 0) {
      const double inv = 1.0 / (double)cnt;
      v[0] = (float)(acc[0] * inv / (double)sc.s[0]);
      v[1] = (float)(acc[1] * inv / (double)sc.s[1]);
      v[2] = (float)(acc[2] * inv / (double)sc.s[2]);
      v[3] = (float)((acc[3] * inv - bmean) / (double)sc.s[3]);
    }
    store_pixel(o + (Y * 18 + X) * 16, v, 0.25f * (float)P.level);
  };
  // inner pixels: one thread each, f x f cells of the patch's own tile
  for (int q = threadIdx.x; q < 256; q += blockDim.x) {
    const int X = q % 16 + 1, Y = q / 16 + 1;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = (Y - 1) * f; j < Y * f; ++j)
      for (int i = (X - 1) * f; i < X * f; ++i) {
        double c4[4];
        e.load(p, cur, e.tix(i, j), c4);
        for (int c = 0; c < 4; ++c) acc[c] += c4[c];
      }
    emit(X, Y, acc, f * f);
  }
  // ring pixels: one warp each; the lanes share the band's cells (f x M/2
  // beside an edge, M/2 x M/2 at a corner), read from whichever leaves
  // cover them, and sum them with a warp reduction
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int r = warp; r < 68; r += nwarp) {
    int X, Y;
    if (r < 18) { X = r; Y = 0; }
    else if (r < 36) { X = r - 18; Y = 17; }
    else if (r < 52) { X = 0; Y = r - 36 + 1; }
    else { X = 17; Y = r - 52 + 1; }
    const int i0 = X == 0 ? -W : X == 17 ? M : (X - 1) * f;
    const int i1 = X == 0 ? 0 : X == 17 ? M + W : X * f;
    const int j0 = Y == 0 ? -W : Y == 17 ? M : (Y - 1) * f;
    const int j1 = Y == 0 ? 0 : Y == 17 ? M + W : Y * f;
    const int wi = i1 - i0, ncell = wi * (j1 - j0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int cnt = 0;
    for (int k = lane; k < ncell; k += 32) {
      const long long I = I0 + i0 + k % wi, J = J0 + j0 + k / wi;
      if (I < 0 || J < 0 || I >= NX || J >= NY) continue;
      double c4[4];
      value_near(e, P.scen, P.level, I, J, c4, &err);
      for (int c = 0; c < 4; ++c) acc[c] += c4[c];
      ++cnt;
    }
    for (int c = 0; c < 4; ++c) acc[c] = warp_sum_f64(acc[c]);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) emit(X, Y, acc, cnt);
  }
}

// The same features for the FP32 deviation form, in single precision: the
// depth of a cell is w - b of its stored FP32 values, the block and band
// means are FP32 sums (the features are rounded to BF16, whose unit is 2^15
// times FP32's, so the precision of the sums changes a feature only when it
// lies within a few FP32 units of a BF16 rounding boundary), and the
// lookups are value_near's.  Register use is capped so that two CTAs
// share an SM; each lane keeps its partial sums of all its ring pixels.
__device__ __forceinline__ void load_f32(const GfGeom& G, const GfView& V, int p, int cur, int c,
                                         float (&o)[4]) {
  const int TT = G.T * G.T;
  const float* q = V.qf[cur] + (size_t)p * 3 * TT;
  const float b = V.bf[(size_t)p * TT + c];
  o[0] = q[c] - b;
  o[1] = q[TT + c];
  o[2] = q[2 * TT + c];
  o[3] = b;
}

// value_at for the FP32 feature kernel, kept out of line: it is the rare
// case, and inlined its FP64 arrays would crowd the kernel's registers.
__device__ __noinline__ Cell4 value_at_f32(const GfGeom* G, const GfView* V, int s, int L,
                                           long long I, long long J) {
  const Geo<float> e(*G, *V);
  double d[4];
  Cell4 r{};
  value_at(e, s, L, I, J, d, &r.err);
  for (int f = 0; f < 4; ++f) r.v[f] = (float)d[f];
  return r;
}

// value_near in FP32 (deviation form, no subcycling): the leaf of level L or
// L - 1, the mean of four leaves of level L + 1, else value_at's composite.
__device__ void value_near_f32(const Geo<float>& e, int s, int cur, int L, long long I,
                               long long J, float (&out)[4], int* err) {
  for (int l = L; l >= L - 1 && l >= 0; --l) {
    const long long Il = I >> (L - l), Jl = J >> (L - l);
    const int p = e.leaf(s, l, Il, Jl);
    if (p >= 0) {
      load_f32(e.G, e.V, p, cur, e.local(Il, Jl), out);
      return;
    }
  }
  if (L + 1 <= e.G.maxlevel) {
    int pc[4];
    bool all = true;
    for (int ch = 0; ch < 4; ++ch) {
      pc[ch] = e.leaf(s, L + 1, 2 * I + (ch & 1), 2 * J + (ch >> 1));
      all = all && pc[ch] >= 0;
    }
    if (all) {
      float v[4][4];
      for (int ch = 0; ch < 4; ++ch)
        load_f32(e.G, e.V, pc[ch], cur, e.local(2 * I + (ch & 1), 2 * J + (ch >> 1)), v[ch]);
      for (int f = 0; f < 4; ++f)
        out[f] = 0.25f * ((v[0][f] + v[1][f]) + (v[2][f] + v[3][f]));
      return;
    }
  }
  const Cell4 r = value_at_f32(&e.G, &e.V, s, L, I, J);
  for (int f = 0; f < 4; ++f) out[f] = r.v[f];
  if (r.err) *err = 1;
}

__global__ void __launch_bounds__(256, 2)
    k_cnn_features_f32(const __grid_constant__ GfGeom G, const __grid_constant__ GfView V,
                       int first, FeatScale sc, __nv_bfloat16* out) {
  const int p = first + blockIdx.x;
  const GfPatch P = V.patch[p];
  Geo<float> e(G, V);
  const int M = G.M, f = M / 16, W = M / 2, TT = G.T * G.T;
  const int cur = V.ctl[P.scen].cur;
  __shared__ float part[8];
  __shared__ float bmean;
  __shared__ int snb8[8];  // same-level neighbours by region (GfView::nbr)
  if (threadIdx.x < 8)
    snb8[threadIdx.x] = V.nbr != nullptr ? V.nbr[(size_t)p * 8 + threadIdx.x] : GF_NBR_OTHER;
  const float* bp = V.bf + (size_t)p * TT;
  float bs = 0.0f;
  for (int k = threadIdx.x; k < M * M; k += blockDim.x) bs += bp[e.tix(k % M, k / M)];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bs += __shfl_xor_sync(0xffffffffu, bs, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = bs;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    bmean = t / (float)(M * M);
  }
  __syncthreads();
  __nv_bfloat16* o = out + (size_t)blockIdx.x * 324 * 16;
  const long long NX = e.nx(P.level), NY = e.ny(P.level);
  const long long I0 = (long long)P.px * M, J0 = (long long)P.py * M;
  int err = 0;
  const float lev = 0.25f * (float)P.level;
  auto emit = [&](int X, int Y, const float (&acc)[4], int cnt) {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (cnt > 0) {
      const float inv = 1.0f / (float)cnt;
      v[0] = acc[0] * inv / sc.s[0];
      v[1] = acc[1] * inv / sc.s[1];
      v[2] = acc[2] * inv / sc.s[2];
      v[3] = (acc[3] * inv - bmean) / sc.s[3];
    }
    store_pixel(o + (Y * 18 + X) * 16, v, lev);
  };
  for (int q = threadIdx.x; q < 256; q += blockDim.x) {
    const int X = q % 16 + 1, Y = q / 16 + 1;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int j = (Y - 1) * f; j < Y * f; ++j)
      for (int i = (X - 1) * f; i < X * f; ++i) {
        float c4[4];
        load_f32(G, V, p, cur, e.tix(i, j), c4);
        for (int c = 0; c < 4; ++c) acc[c] += c4[c];
      }
    emit(X, Y, acc, f * f);
  }
  // ring pixels: one warp each.  A pixel's band lies in one of the eight
  // neighbour regions; a same-level neighbour's cells are read from its
  // tile directly (the leaf value_near would find), anything else through
  // the forest lookups.  Every lane first gathers its cells of all of its
  // warp's pixels (pixels warp, warp + 8, ...; their loads overlap), then
  // the warp sums each pixel.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  constexpr int RP = 9;  // pixels per warp: ceil(68 / 8) with 256 threads
  auto ring = [&](int r, int& X, int& Y) {
    if (r < 18) { X = r; Y = 0; }
    else if (r < 36) { X = r - 18; Y = 17; }
    else if (r < 52) { X = 0; Y = r - 36 + 1; }
    else { X = 17; Y = r - 52 + 1; }
  };
  float racc[RP][4];
  int rcnt[RP];
#pragma unroll
  for (int t = 0; t < RP; ++t) {
    racc[t][0] = racc[t][1] = racc[t][2] = racc[t][3] = 0.f;
    rcnt[t] = 0;
    const int r = warp + t * nwarp;
    if (r >= 68) continue;
    int X, Y;
    ring(r, X, Y);
    const int i0 = X == 0 ? -W : X == 17 ? M : (X - 1) * f;
    const int i1 = X == 0 ? 0 : X == 17 ? M + W : X * f;
    const int j0 = Y == 0 ? -W : Y == 17 ? M : (Y - 1) * f;
    const int j1 = Y == 0 ? 0 : Y == 17 ? M + W : Y * f;
    // neighbour region (0 left, 1 right, 2 bottom, 3 top, 4-7 the corners
    // bottom-left, bottom-right, top-left, top-right) and its offset
    const int ox = X == 0 ? -1 : X == 17 ? 1 : 0, oy = Y == 0 ? -1 : Y == 17 ? 1 : 0;
    const int reg = oy == 0 ? (ox < 0 ? 0 : 1)
                  : ox == 0 ? (oy < 0 ? 2 : 3)
                            : 4 + (ox > 0 ? 1 : 0) + (oy > 0 ? 2 : 0);
    const int nb = snb8[reg];
    const int wi = i1 - i0, ncell = wi * (j1 - j0);
    for (int k = lane; k < ncell; k += 32) {
      const int i = i0 + k % wi, j = j0 + k / wi;
      float c4[4];
      if (nb >= 0) {
        load_f32(G, V, nb, cur, e.tix(i - ox * M, j - oy * M), c4);
      } else {
        const long long I = I0 + i, J = J0 + j;
        if (I < 0 || J < 0 || I >= NX || J >= NY) continue;
        value_near_f32(e, P.scen, cur, P.level, I, J, c4, &err);
      }
      for (int c = 0; c < 4; ++c) racc[t][c] += c4[c];
      ++rcnt[t];
    }
  }
#pragma unroll
  for (int t = 0; t < RP; ++t) {
    const int r = warp + t * nwarp;
    if (r >= 68) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      for (int d = 16; d > 0; d >>= 1) racc[t][c] += __shfl_xor_sync(0xffffffffu, racc[t][c], d);
    const int cnt = __reduce_add_sync(0xffffffffu, rcnt[t]);
    int X, Y;
    ring(r, X, Y);
    if (lane == 0) emit(X, Y, racc[t], cnt);
  }
}

inline int ok() { return cudaGetLastError() == cudaSuccess ? 0 : -2; }

}  // namespace

namespace gf {

static int* g_errflag = nullptr;

int launch_ghost_fill(const GfGeom& g, const GfView& v, int only_accepted,
                      void* stream) {
  if (v.npatch <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nghost = g.T * g.T - g.M * g.M;  // 272 (M = 32) or 144 (M = 16)
  const int nt = (nghost + 31) / 32 * 32;
  if (v.prec) k_ghost_fill<float><<<v.npatch, nt, 0, st>>>(g, v, only_accepted, g_errflag, nullptr);
  else k_ghost_fill<double><<<v.npatch, nt, 0, st>>>(g, v, only_accepted, g_errflag, nullptr);
  return ok();
}

int launch_ghost_rest(const GfGeom& g, const GfView& v, const int* regs, int nquad,
                      int nreg, void* stream) {
  if (nreg <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long total = (long long)nquad * (g.M / 2) + (long long)(nreg - nquad) * 2 * g.M;
  const int blocks = (int)((total + 255) / 256);
  if (v.prec && !g.subcycle)
    k_ghost_other<float, true><<<blocks, 256, 0, st>>>(g, v, regs, nquad, nreg, g_errflag);
  else if (v.prec)
    k_ghost_other<float, false><<<blocks, 256, 0, st>>>(g, v, regs, nquad, nreg, g_errflag);
  else k_ghost_other<double, false><<<blocks, 256, 0, st>>>(g, v, regs, nquad, nreg, g_errflag);
  return ok();
}


int launch_subcycle_sync(const GfGeom& g, const GfView& v, void* stream) {
  if (!g.subcycle || v.npatch <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (v.prec) k_subcycle_sync<float><<<v.npatch, 256, 0, st>>>(g, v);
  else k_subcycle_sync<double><<<v.npatch, 256, 0, st>>>(g, v);
  return ok();
}

int launch_inflow(const GfGeom& g, const GfView& v, const int* list, int n,
                  int only_accepted, void* stream) {
  if (n <= 0 || g.n_hydro <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nt = (g.T + 31) / 32 * 32;
  if (v.prec) k_inflow<float><<<n, nt, 0, st>>>(g, v, list, only_accepted);
  else k_inflow<double><<<n, nt, 0, st>>>(g, v, list, only_accepted);
  return ok();
}

int launch_topo(const GfGeom& g, const GfView& v, int first, int count,
                void* stream, const int* list) {
  if (count <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (v.prec) k_topo<float><<<count, 128, 0, st>>>(g, v, first, list);
  else k_topo<double><<<count, 128, 0, st>>>(g, v, first, list);
  return ok();
}

int launch_regrid_fill(const GfGeom& g, const GfView& oldv, const GfView& newv,
                       void* stream, const int* list, int count) {
  const int n = list ? count : newv.npatch;
  if (n <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (newv.prec) k_regrid_fill<float><<<n, 256, 0, st>>>(g, oldv, newv, g_errflag, list);
  else k_regrid_fill<double><<<n, 256, 0, st>>>(g, oldv, newv, g_errflag, list);
  return ok();
}

int launch_regrid_keep(const GfGeom& g, const GfView& oldv, const GfView& newv,
                       const void* pairs, int count, void* stream) {
  if (count <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int2* pr = static_cast<const int2*>(pairs);
  if (newv.prec) k_regrid_keep<float><<<count, 256, 0, st>>>(g, oldv, newv, pr);
  else k_regrid_keep<double><<<count, 256, 0, st>>>(g, oldv, newv, pr);
  return ok();
}

int launch_align_buffers(const GfGeom& g, const GfView& v, int target, void* stream) {
  if (v.npatch <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (v.prec) k_align_buffers<float><<<v.npatch, 256, 0, st>>>(g, v, target);
  else k_align_buffers<double><<<v.npatch, 256, 0, st>>>(g, v, target);
  return ok();
}

int launch_tags(const GfGeom& g, const GfView& v, uint8_t* flags,
                void* stream) {
  GfTagOut o{};
  o.flags = flags;
  return launch_tags_ex(g, v, o, stream);
}

int launch_tags_ex(const GfGeom& g, const GfView& v, const GfTagOut& o,
                   void* stream) {
  if (v.npatch <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (v.prec) k_tags<float><<<v.npatch, 256, 0, st>>>(g, v, o);
  else k_tags<double><<<v.npatch, 256, 0, st>>>(g, v, o);
  return ok();
}

int launch_cnn_features(const GfGeom& g, const GfView& v, int first, int count,
                        const float* scale, void* out, void* stream) {
  if (count <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FeatScale sc{{scale[0], scale[1], scale[2], scale[3]}};
  if (v.prec && !g.subcycle)
    k_cnn_features_f32<<<count, 256, 0, st>>>(g, v, first, sc, static_cast<__nv_bfloat16*>(out));
  else if (v.prec)
    k_cnn_features<float><<<count, 256, 0, st>>>(g, v, first, sc, static_cast<__nv_bfloat16*>(out));
  else
    k_cnn_features<double><<<count, 256, 0, st>>>(g, v, first, sc, static_cast<__nv_bfloat16*>(out));
  return ok();
}

int launch_gauge_refs(const GfGeom& g, const GfView& v, int max_gauges,
                      void* stream) {
  if (max_gauges <= 0) return 0;
  dim3 grid((max_gauges + 63) / 64, g.nscen);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (v.prec) k_gauge_refs<float><<<grid, 64, 0, st>>>(g, v);
  else k_gauge_refs<double><<<grid, 64, 0, st>>>(g, v);
  return ok();
}

int launch_gauges(const GfGeom& g, const GfView& v, int only_accepted,
                  int max_gauges, void* stream) {
  if (max_gauges <= 0) return 0;
  dim3 grid((max_gauges + 63) / 64, g.nscen);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (v.prec) k_gauges<float><<<grid, 64, 0, st>>>(g, v, only_accepted);
  else k_gauges<double><<<grid, 64, 0, st>>>(g, v, only_accepted);
  return ok();
}

int launch_mass(const GfGeom& g, const GfView& v, double* pmass,
                double* smass, int nscen, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (v.npatch > 0) {
    if (v.prec) k_patch_mass<float><<<v.npatch, 256, 0, st>>>(g, v, pmass);
    else k_patch_mass<double><<<v.npatch, 256, 0, st>>>(g, v, pmass);
  }
  k_scen_mass<<<nscen, 256, 0, st>>>(v.scen, pmass, smass);
  return ok();
}

int launch_pack_interior(const GfGeom& g, const GfView& v, int first,
                         int count, double* out, int field_mask, int cur,
                         void* stream) {
  (void)field_mask;
  if (count <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (v.prec) k_pack<float><<<count, 256, 0, st>>>(g, v, first, out, cur);
  else k_pack<double><<<count, 256, 0, st>>>(g, v, first, out, cur);
  return ok();
}

int launch_unpack_interior(const GfGeom& g, const GfView& v, int first,
                           int count, const double* in, int cur,
                           void* stream) {
  if (count <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (v.prec) k_unpack<float><<<count, 256, 0, st>>>(g, v, first, in, cur);
  else k_unpack<double><<<count, 256, 0, st>>>(g, v, first, in, cur);
  return ok();
}

void set_errflag(int* p) { g_errflag = p; }

}  // namespace gf
