// Device-side building blocks of the wave-propagation step: the augmented
// Riemann solver (Sec. 3.3), the MC limiter (Sec. 3.2) and the transverse
// eigen-split of the 2D extension (Sec. 3.2, leveque2002).  Templates on the
// real type; the FP64 translation units are compiled with -fmad=false so
// that every operation rounds as written.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace gfk {

template <typename R>
struct Side {
  R h, n, t, b;  // depth, normal momentum, transverse momentum, bed
  R w;           // surface-deviation form only: stored surface h + b - eta0
  bool wet;      // surface-deviation form only: exact wet test of the cell
};

// Quotient a / b.  FP64: the correctly rounded division, so that the FP64
// path rounds as written.  FP32: the approximate reciprocal times a (within
// 2 ulp for |b| below 2^126, far above any depth, momentum or speed here);
// the product is rounded on its own (never fused into a neighbouring
// addition), so that every kernel variant that inlines this code rounds it
// alike.  Zero numerators still give exact zeros, so a lake at rest keeps
// exactly zero waves.
template <typename R>
__device__ __forceinline__ R qdiv(R a, R b) { return a / b; }
template <>
__device__ __forceinline__ float qdiv<float>(float a, float b) {
  return __fmul_rn(a, __fdividef(1.0f, b));
}

// Product rounded on its own (FP32: never fused into a neighbouring addition).
template <typename R>
__device__ __forceinline__ R rmul(R a, R b) { return a * b; }
template <>
__device__ __forceinline__ float rmul<float>(float a, float b) { return __fmul_rn(a, b); }

template <typename R>
__device__ __forceinline__ R rmin(R a, R b) { return a < b ? a : b; }
template <typename R>
__device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }

// Augmented Riemann solve (Sec. 3.3).  Returns three f-waves Z[p*3 + k]
// (component k: mass, normal momentum, transverse momentum) and speeds s[p].
// Bed jump: a stationary wave whose momentum-flux part -g*hbar*db is the
// bathymetry source and whose depth jump is -db, bounded so no depth in the
// fan is negative.  Acoustic speeds: Einfeldt (HLLE) with Roe averages, or
// the dam-break front speeds at a wet/dry edge.  A dry cell whose bed is
// above the wet surface is tested with the mirrored (reflecting) problem.
//
// DEV = false: plain form, the state is (h, n, t) and the bed b; the wet test
// is h > drytol and the surface jump is formed from depths and beds.
// DEV = true: surface-deviation form, each side also carries its stored
// surface w = h + b - eta0 (b is then the bed minus eta0) and a wet flag
// decided exactly from the stored values; the surface jump is the difference
// of the stored surfaces, so a lake at rest gives exactly zero waves.
template <typename R, bool DEV = false>
__device__ __forceinline__ void riemann(Side<R> l, Side<R> r, R g, R drytol,
                                        R (&Z)[9], R (&s)[3]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) Z[k] = R(0);
  s[0] = s[1] = s[2] = R(0);
  const bool wetl = DEV ? l.wet : (l.h > drytol);
  const bool wetr = DEV ? r.wet : (r.h > drytol);
  if (!wetl && !wetr) return;
  // surface depths: a dry cell keeps its stored depth in its surface so a
  // still shoreline stays at rest; fluxes and speeds see zero depth
  R el = l.h, er = r.h;
  if (!wetl) { l.h = R(0); l.n = R(0); l.t = R(0); }
  if (!wetr) { r.h = R(0); r.n = R(0); r.t = R(0); }

  int wall = 0;  // +1: right side is a wall, -1: left side is a wall
  if (!wetr && (DEV ? r.b > l.w : r.b > l.h + l.b)) {
    const R u = qdiv(l.n, l.h);
    const R c = sqrt(g * l.h);
    const R sw = rmax(c - u, c);       // fastest wave of the mirrored problem
    const R hm = l.h + qdiv(l.n, sw);  // its HLL middle depth
    if (r.b >= l.b + hm) {
      wall = 1;
      r.h = l.h; r.n = -l.n; r.t = l.t; r.b = l.b; er = l.h; r.w = l.w;
    } else if (DEV) {
      r.w = l.w + er;                  // overtopped: step lowered to surface
      r.b = l.w;
    } else {
      r.b = l.h + l.b;
    }
  } else if (!wetl && (DEV ? l.b > r.w : l.b > r.h + r.b)) {
    const R u = qdiv(r.n, r.h);
    const R c = sqrt(g * r.h);
    const R sw = rmax(u + c, c);
    const R hm = r.h - qdiv(r.n, sw);
    if (l.b >= r.b + hm) {
      wall = -1;
      l.h = r.h; l.n = -r.n; l.t = r.t; l.b = r.b; el = r.h; l.w = r.w;
    } else if (DEV) {
      l.w = r.w + el;
      l.b = r.w;
    } else {
      l.b = r.h + r.b;
    }
  }

  const R ul = l.h > R(0) ? qdiv(l.n, l.h) : R(0);
  const R ur = r.h > R(0) ? qdiv(r.n, r.h) : R(0);
  const R vl = l.h > R(0) ? qdiv(l.t, l.h) : R(0);
  const R vr = r.h > R(0) ? qdiv(r.t, r.h) : R(0);
  // FP32: the celerities from the square roots of the depths, which the
  // Roe average needs anyway (two square roots fewer per edge), each product
  // rounded on its own (not fused, so every inlining rounds it alike); FP64:
  // as written, sqrt(g h)
  constexpr bool F32 = std::is_same<R, float>::value;
  const R ql = F32 ? sqrt(l.h) : R(0), qr = F32 ? sqrt(r.h) : R(0);
  const R cl = F32 ? rmul(sqrt(g), ql) : sqrt(g * l.h);
  const R cr = F32 ? rmul(sqrt(g), qr) : sqrt(g * r.h);
  R s1, s3;
  if (l.h > R(0) && r.h > R(0)) {
    const R qlw = F32 ? ql : sqrt(l.h), qrw = F32 ? qr : sqrt(r.h);
    const R uhat = qdiv(qlw * ul + qrw * ur, qlw + qrw);
    const R chat = sqrt(g * (R(0.5) * (l.h + r.h)));
    s1 = rmin(ul - cl, uhat - chat);
    s3 = rmax(ur + cr, uhat + chat);
  } else if (r.h == R(0)) {
    s1 = ul - cl;
    s3 = ul + R(2) * cl;
  } else {
    s1 = ur - R(2) * cr;
    s3 = ur + cr;
  }
  const R s2 = R(0.5) * (s1 + s3);

  const R hbar = R(0.5) * (l.h + r.h);
  const R db = r.b - l.b;
  const R deta = DEV ? r.w - l.w : (er + r.b) - (el + l.b);
  const R den = s3 - s1;
  const R dn = r.n - l.n;
  const R hhll = qdiv(s3 * r.h - s1 * l.h - dn, den);

  // depth jump of the stationary wave, bounded for non-negative depths
  R dhs = -db;
  bool clamped = false;
  if (s1 < R(0) && s3 > R(0)) {
    const R lo = qdiv(hhll * den, s1);
    const R hi = qdiv(hhll * den, s3);
    if (dhs < lo) { dhs = lo; clamped = true; }
    if (dhs > hi) { dhs = hi; clamped = true; }
  } else if (s1 >= R(0)) {
    const R hi = s1 > R(0) ? qdiv(hhll * den, s1) : dhs;
    if (dhs > hi) { dhs = hi; clamped = true; }
    if (dhs < -l.h) { dhs = -l.h; clamped = true; }
  } else {
    const R lo = s3 < R(0) ? qdiv(hhll * den, s3) : dhs;
    if (dhs < lo) { dhs = lo; clamped = true; }
    if (dhs > r.h) { dhs = r.h; clamped = true; }
  }
  const R d1 = clamped ? (r.h - l.h) - dhs : deta;
  const R d3 = (r.n * ur - l.n * ul) + g * hbar * deta;

  const R b1 = qdiv(s3 * d1 - dn, den);
  const R b3 = qdiv(dn - s1 * d1, den);
  const R b2 = d3 - (s1 * s1 * b1 + s3 * s3 * b3);

  Z[0] = s1 * b1;
  Z[1] = s1 * s1 * b1;
  Z[2] = vl * Z[0];
  Z[6] = s3 * b3;
  Z[7] = s3 * s3 * b3;
  Z[8] = vr * Z[6];
  Z[3] = R(0);
  Z[4] = b2;
  Z[5] = (r.n * vr - l.n * vl) - (Z[2] + Z[8]);
  s[0] = s1;
  s[1] = s2;
  s[2] = s3;
  if (wall == 1) {
#pragma unroll
    for (int k = 3; k < 9; ++k) Z[k] = R(0);
  } else if (wall == -1) {
#pragma unroll
    for (int k = 0; k < 6; ++k) Z[k] = R(0);
  }
}

// MC limiter.
template <typename R>
__device__ __forceinline__ R mc(R th) {
  const R a = R(0.5) * (R(1) + th);
  R m = a < R(2) ? a : R(2);
  const R b = R(2) * th;
  m = m < b ? m : b;
  return m > R(0) ? m : R(0);
}

template <typename R>
__device__ __forceinline__ R dot3(const R* a, const R* b) {
  return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

// Fluctuations A-dQ, A+dQ and the limited correction flux of one edge from
// its waves (Z, S) and the waves of its two neighbouring edges (Zm at the
// edge before, Zp at the edge after).  Component c of a wave array is at
// [c * ST] (ST = 1: packed; larger: one plane per component).  nodry = false
// switches the correction off (an edge touching a dry cell).
// Z3Z = true: the middle wave's mass component (Z[3], zero by construction
// of the solver) is neither read nor added, and A+dQ is formed as the wave
// minus its A-dQ part; both give the same values up to the sign of zeros.
template <typename R, int ST = 1, bool Z3Z = false>
__device__ __forceinline__ void edge_fluxes(const R* Z, const R* S,
                                            const R* Zm, const R* Zp, R nu,
                                            bool nodry, R (&am)[3],
                                            R (&ap)[3], R (&ff)[3]) {
  R cm[3][3], cp[3][3], cf[3][3];
  R z[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) z[c] = (Z3Z && c == 3) ? R(0) : Z[c * ST];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const R sp = S[p * ST];
    const R wm = sp < R(0) ? R(1) : (sp == R(0) ? R(0.5) : R(0));
    const R wp = sp > R(0) ? R(1) : (sp == R(0) ? R(0.5) : R(0));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cm[p][k] = z[3 * p + k] * wm;
      cp[p][k] = Z3Z ? z[3 * p + k] - cm[p][k] : z[3 * p + k] * wp;
      cf[p][k] = R(0);
    }
    if (sp != R(0) && nodry) {
      const bool m0 = Z3Z && p == 1;  // mass component known zero
      const R zz = m0 ? z[4] * z[4] + z[5] * z[5] : dot3(z + 3 * p, z + 3 * p);
      if (zz != R(0)) {
        const R* up = sp > R(0) ? Zm : Zp;
        const R u3[3] = {m0 ? R(0) : up[(3 * p) * ST], up[(3 * p + 1) * ST],
                         up[(3 * p + 2) * ST]};
        const R num = m0 ? u3[1] * z[4] + u3[2] * z[5] : dot3(u3, z + 3 * p);
        const R th = qdiv(num, zz);
        const R phi = mc(th);
        const R sg = sp > R(0) ? R(1) : R(-1);
        const R as = sp > R(0) ? sp : -sp;
        const R coef = R(0.5) * sg * (R(1) - nu * as) * phi;
#pragma unroll
        for (int k = 0; k < 3; ++k) cf[p][k] = coef * z[3 * p + k];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (Z3Z && k == 0) {
      am[0] = cm[0][0] + cm[2][0];
      ap[0] = cp[0][0] + cp[2][0];
      ff[0] = cf[0][0] + cf[2][0];
    } else {
      am[k] = (cm[0][k] + cm[2][k]) + cm[1][k];
      ap[k] = (cp[0][k] + cp[2][k]) + cp[1][k];
      ff[k] = (cf[0][k] + cf[2][k]) + cf[1][k];
    }
  }
}

// Transverse split of an increment d = (mass, momentum along the split
// direction, other momentum) in a cell with depth h, momenta ma (along) and
// mo (other): eigenvectors of the split direction's Jacobian with speeds
// w - c, w, w + c.  plus/minus are returned in the same frame.  A part
// entering a dry neighbour whose bed is above the cell's surface is dropped;
// a dry cell splits nothing.  Wet tests and the surface come from the caller:
// wet, wetm, wetp for the cell and its neighbours at -1 and +1, eta the
// cell's surface, bm, bp the neighbours' beds (same datum as eta).
template <typename R>
__device__ __forceinline__ void tsplit(R h, R ma, R mo, R eta, bool wet,
                                       bool wetm, R bm, bool wetp, R bp,
                                       const R (&d)[3], R g, R (&plus)[3],
                                       R (&minus)[3]) {
  plus[0] = plus[1] = plus[2] = R(0);
  minus[0] = minus[1] = minus[2] = R(0);
  if (!wet) return;
  const R w = qdiv(ma, h);
  const R z = qdiv(mo, h);
  const R c = sqrt(g * h);
  const R a1 = qdiv((w + c) * d[0] - d[1], R(2) * c);
  const R a3 = qdiv(d[1] - (w - c) * d[0], R(2) * c);
  const R a2 = d[2] - z * d[0];
  const R l1 = w - c, l2 = w, l3 = w + c;
  const R c1 = l1 * a1, c3 = l3 * a3, c2 = l2 * a2;
  const R W1[3] = {c1, c1 * l1, c1 * z};
  const R W3[3] = {c3, c3 * l3, c3 * z};
  const R W2[3] = {R(0), R(0), c2};
  const bool openp = !(!wetp && (bp > eta));
  const bool openm = !(!wetm && (bm > eta));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R p1 = l1 > R(0) ? W1[k] : R(0), q1 = l1 < R(0) ? W1[k] : R(0);
    const R p3 = l3 > R(0) ? W3[k] : R(0), q3 = l3 < R(0) ? W3[k] : R(0);
    const R p2 = l2 > R(0) ? W2[k] : R(0), q2 = l2 < R(0) ? W2[k] : R(0);
    if (openp) plus[k] = (p1 + p3) + p2;
    if (openm) minus[k] = (q1 + q3) + q2;
  }
}

// Exact wet test of a stored surface-deviation cell: depth = w - b (both
// FP32) compared with drytol as the FP64 value (w - b is exact in double).
// FP32 decides when the rounded difference is clear of drytol by more than
// its rounding bound; otherwise the test is redone in FP64.
// The FP64 tie-break is a separate, non-inlined function so that the
// compiler cannot evaluate it speculatively on every call (FP64 is slow on
// this part).
static __device__ __noinline__ bool wet_dev_tie(float w, float b, double drytol) {
  return ((double)w - (double)b) > drytol;
}

__device__ __forceinline__ bool wet_dev(float w, float b, double drytol,
                                        float dtf, float margin) {
  const float h = w - b;
  if (h > dtf + margin) return true;
  if (h < dtf - margin) return false;
  return wet_dev_tie(w, b, drytol);
}

}  // namespace gfk
