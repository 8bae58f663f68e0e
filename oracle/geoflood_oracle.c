/*
 * GeoFlood FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain double-precision loops, written from the method as the GeoFlood paper
 * (arXiv 2403.15435) states it and from the published methods it names.
 * Each function cites the passage it follows.  Where the paper only cites a
 * method (the augmented solver of Sec. 3.3, the TVD limiter and the 2D
 * extension of Sec. 3.2, the ghost-cell operators of Sec. 4, the tagging
 * thresholds of Sec. 4.1) the comment beside the code states the reading
 * taken; the same readings bind the CUDA library, which shares no code with
 * this file.
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define NG 2
#define MAXLEV 24

/* ------------------------------------------------------------------------ */
/* Augmented Riemann solver, Sec. 3.3 (george2008).                          */
/* ------------------------------------------------------------------------ */

/* Edge states are given in the normal frame: depth h, normal momentum n,
 * transverse momentum t and bed b.  The solver decomposes the jump of the
 * augmented state (h, n, phi = n^2/h + g h^2 / 2, b) into
 *   - a stationary wave (speed 0) carrying the bed jump; its momentum-flux
 *     part -g*hbar*db is the bathymetry source, so the three propagating
 *     f-waves sum to the flux jump minus that source (well balanced, Sec. 3.2
 *     last paragraph and Sec. 3.3);
 *   - two acoustic waves with the Einfeldt (HLLE) speeds built on Roe
 *     averages, replaced by the dam-break front speed u +- 2 sqrt(gh) of the
 *     wet side at a wet/dry edge (Sec. 3.3);
 *   - a corrector wave at the mean speed that carries only momentum flux and
 *     the shear (transverse momentum) flux.
 * A dry cell whose bed lies above the neighbouring wet surface is tested with
 * an artificial reflecting-wall Riemann problem (Sec. 3.3, "artificial
 * Riemann test problems").  Z[p*3+k] is f-wave p, component k. */
void oracle_riemann(double hL, double nL, double tL, double bL, double hR,
                    double nR, double tR, double bR, double g, double drytol,
                    double* Z, double* s) {
  int p, k;
  for (p = 0; p < 9; ++p) Z[p] = 0.0;
  for (p = 0; p < 3; ++p) s[p] = 0.0;

  int wetL = hL > drytol;
  int wetR = hR > drytol;
  if (!wetL && !wetR) return; /* both dry: no waves */
  /* a dry cell keeps its small stored depth in its surface elevation, so a
   * still shoreline is at rest; its fluxes use zero depth */
  double sL = hL, sR = hR;
  if (!wetL) { hL = 0.0; nL = 0.0; tL = 0.0; }
  if (!wetR) { hR = 0.0; nR = 0.0; tR = 0.0; }

  /* Wall test at a wet/dry edge whose dry bed is above the wet surface. */
  int wallR = 0, wallL = 0;
  if (!wetR && bR > hL + bL) {
    double uL = nL / hL;
    double cL = sqrt(g * hL);
    /* HLL middle depth of the mirrored problem (hL, uL | hL, -uL). */
    double sw = cL - uL;
    if (sw < cL) sw = cL;
    double hm = hL + nL / sw;
    if (bR >= bL + hm) {
      wallR = 1;
      hR = hL; nR = -nL; tR = tL; bR = bL; sR = hL;
    } else {
      bR = hL + bL; /* the flow overtops: lower the dry step to the surface */
    }
  } else if (!wetL && bL > hR + bR) {
    double uR = nR / hR;
    double cR = sqrt(g * hR);
    double sw = uR + cR;
    if (sw < cR) sw = cR;
    double hm = hR - nR / sw;
    if (bL >= bR + hm) {
      wallL = 1;
      hL = hR; nL = -nR; tL = tR; bL = bR; sL = hR;
    } else {
      bL = hR + bR;
    }
  }

  double uL = hL > 0.0 ? nL / hL : 0.0;
  double uR = hR > 0.0 ? nR / hR : 0.0;
  double vL = hL > 0.0 ? tL / hL : 0.0;
  double vR = hR > 0.0 ? tR / hR : 0.0;
  double cL = sqrt(g * hL);
  double cR = sqrt(g * hR);

  double s1, s3;
  if (hL > 0.0 && hR > 0.0) {
    double rL = sqrt(hL), rR = sqrt(hR);
    double uhat = (rL * uL + rR * uR) / (rL + rR);
    double chat = sqrt(g * (0.5 * (hL + hR)));
    double a = uL - cL, b2 = uhat - chat;
    s1 = a < b2 ? a : b2;
    a = uR + cR; b2 = uhat + chat;
    s3 = a > b2 ? a : b2;
  } else if (hR == 0.0) {
    s1 = uL - cL;
    s3 = uL + 2.0 * cL;
  } else {
    s1 = uR - 2.0 * cR;
    s3 = uR + cR;
  }
  double s2 = 0.5 * (s1 + s3);

  double hbar = 0.5 * (hL + hR);
  double db = bR - bL;
  double deta = (sR + bR) - (sL + bL);
  double den = s3 - s1;
  double dn = nR - nL;
  double hhll = (s3 * hR - s1 * hL - dn) / den;

  /* Depth jump across the stationary wave: lake-at-rest relation -db,
   * bounded so that both middle depths stay non-negative. */
  double dhs = -db;
  int clamped = 0;
  if (s1 < 0.0 && s3 > 0.0) {
    double lo = hhll * den / s1; /* = -hhll / w1, w1 = -s1/den */
    double hi = hhll * den / s3; /* =  hhll / w3, w3 =  s3/den */
    if (dhs < lo) { dhs = lo; clamped = 1; }
    if (dhs > hi) { dhs = hi; clamped = 1; }
  } else if (s1 >= 0.0) {
    /* all waves move right: the states hL + dhs and hmR must be >= 0 */
    double hi = s1 > 0.0 ? hhll * den / s1 : dhs;
    if (dhs > hi) { dhs = hi; clamped = 1; }
    if (dhs < -hL) { dhs = -hL; clamped = 1; }
  } else {
    /* all waves move left: the states hR - dhs and hmL must be >= 0 */
    double lo = s3 < 0.0 ? hhll * den / s3 : dhs;
    if (dhs < lo) { dhs = lo; clamped = 1; }
    if (dhs > hR) { dhs = hR; clamped = 1; }
  }
  double d1 = clamped ? (hR - hL) - dhs : deta;
  double d2 = dn;
  double d3 = (nR * uR - nL * uL) + g * hbar * deta;

  double beta1 = (s3 * d1 - d2) / den;
  double beta3 = (d2 - s1 * d1) / den;
  double beta2 = d3 - (s1 * s1 * beta1 + s3 * s3 * beta3);

  Z[0] = s1 * beta1;
  Z[1] = s1 * s1 * beta1;
  Z[2] = vL * Z[0];
  Z[6] = s3 * beta3;
  Z[7] = s3 * s3 * beta3;
  Z[8] = vR * Z[6];
  Z[3] = 0.0;
  Z[4] = beta2;
  Z[5] = (nR * vR - nL * vL) - (Z[2] + Z[8]);
  s[0] = s1;
  s[1] = s2;
  s[2] = s3;

  /* Reflecting wall: nothing enters the dry cell. */
  if (wallR)
    for (k = 3; k < 9; ++k) Z[k] = 0.0;
  if (wallL)
    for (k = 0; k < 6; ++k) Z[k] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Wave-propagation step on one grid, Sec. 3.2, Eqs. (wpa_update) and       */
/* (wpa_update_corrections), 2D unsplit extension with transverse           */
/* propagation (leveque2002, cited in Sec. 3.2), Manning friction           */
/* (Eq. manning).                                                            */
/* ------------------------------------------------------------------------ */

/* MC limiter (a TVD limiter, Sec. 3.2). */
static double mc_limiter(double th) {
  double a = 0.5 * (1.0 + th);
  double m = a < 2.0 ? a : 2.0;
  double b = 2.0 * th;
  m = m < b ? m : b;
  return m > 0.0 ? m : 0.0;
}

static double dot3(const double* a, const double* b) {
  return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

/* Transverse split of an increment d (components h, hu, hv) entering a cell,
 * along direction dir (0 = x, 1 = y), using the eigenvectors of that
 * direction's flux Jacobian in the cell's own state.  The positive-speed part
 * goes to the neighbour at +1, the negative part to the neighbour at -1.  A
 * part is dropped when its neighbour is dry with a bed above the cell's
 * surface (the wall test), and both parts are zero in a dry cell. */
static void transverse_split(int dir, double h, double hu, double hv,
                             double b, double hm, double bm, double hp,
                             double bp, const double* d, double g,
                             double drytol, double* plus, double* minus) {
  int k;
  for (k = 0; k < 3; ++k) { plus[k] = 0.0; minus[k] = 0.0; }
  if (h <= drytol) return;
  /* frame: m = mass, a = momentum along dir, o = the other momentum */
  double dm = d[0];
  double da = dir == 0 ? d[1] : d[2];
  double dq = dir == 0 ? d[2] : d[1];
  double w = (dir == 0 ? hu : hv) / h;
  double z = (dir == 0 ? hv : hu) / h;
  double c = sqrt(g * h);
  double a1 = ((w + c) * dm - da) / (2.0 * c);
  double a3 = (da - (w - c) * dm) / (2.0 * c);
  double a2 = dq - z * dm;
  double l1 = w - c, l2 = w, l3 = w + c;
  /* wave vectors lambda_p * a_p * r_p in the frame (m, a, o) */
  double W1[3], W2[3], W3[3];
  double c1 = l1 * a1, c3 = l3 * a3, c2 = l2 * a2;
  W1[0] = c1; W1[1] = c1 * l1; W1[2] = c1 * z;
  W3[0] = c3; W3[1] = c3 * l3; W3[2] = c3 * z;
  W2[0] = 0.0; W2[1] = 0.0; W2[2] = c2;
  double P[3], M[3];
  for (k = 0; k < 3; ++k) {
    double p1 = l1 > 0.0 ? W1[k] : 0.0, q1 = l1 < 0.0 ? W1[k] : 0.0;
    double p3 = l3 > 0.0 ? W3[k] : 0.0, q3 = l3 < 0.0 ? W3[k] : 0.0;
    double p2 = l2 > 0.0 ? W2[k] : 0.0, q2 = l2 < 0.0 ? W2[k] : 0.0;
    P[k] = (p1 + p3) + p2;
    M[k] = (q1 + q3) + q2;
  }
  double eta = h + b;
  int wallp = (hp <= drytol) && (bp > eta);
  int wallm = (hm <= drytol) && (bm > eta);
  if (!wallp) {
    plus[0] = P[0];
    plus[dir == 0 ? 1 : 2] = P[1];
    plus[dir == 0 ? 2 : 1] = P[2];
  }
  if (!wallm) {
    minus[0] = M[0];
    minus[dir == 0 ? 1 : 2] = M[1];
    minus[dir == 0 ? 2 : 1] = M[2];
  }
}

/* One sweep in direction dir over every line of the grid plus one ghost
 * line on each side.  Fills dq (per-cell increment, components h, hu, hv,
 * [H][W][3]) for cells along the interior range and updates *smax. */
static void sweep(int dir, int nx, int ny, const double* h, const double* hu,
                  const double* hv, const double* b, double nu, double g,
                  double drytol, double* dq, double* smax, int order, int c_lo,
                  int c_hi) {
  int W = nx + 2 * NG;
  int na = dir == 0 ? nx : ny;
  int nc = dir == 0 ? ny : nx;
  int ne = na + 3; /* edges a in [-1, na+1] */
  double* Zs = (double*)malloc(sizeof(double) * 9 * ne);
  double* Ss = (double*)malloc(sizeof(double) * 3 * ne);
  double* AM = (double*)malloc(sizeof(double) * 3 * (na + 1));
  double* AP = (double*)malloc(sizeof(double) * 3 * (na + 1));
  double* FF = (double*)malloc(sizeof(double) * 3 * (na + 1));
  int* wd = (int*)malloc(sizeof(int) * ne); /* edge touches a dry cell */
  const double* qn = dir == 0 ? hu : hv;
  const double* qt = dir == 0 ? hv : hu;
  int a, c, p, k;
  for (c = c_lo; c <= c_hi; ++c) {
    for (a = -1; a <= na + 1; ++a) {
      int iL = dir == 0 ? a - 1 : c, jL = dir == 0 ? c : a - 1;
      int iR = dir == 0 ? a : c, jR = dir == 0 ? c : a;
      int L = (iL + NG) + (jL + NG) * W;
      int R = (iR + NG) + (jR + NG) * W;
      oracle_riemann(h[L], qn[L], qt[L], b[L], h[R], qn[R], qt[R], b[R], g,
                     drytol, Zs + 9 * (a + 1), Ss + 3 * (a + 1));
      wd[a + 1] = !(h[L] > drytol) || !(h[R] > drytol);
    }
    /* fluctuations and limited corrections at edges a in [0, na]; an edge
     * with a dry cell on either side takes no correction (first order at
     * wet/dry fronts, so the correction cannot drain a cell below zero) */
    for (a = 0; a <= na; ++a) {
      const double* Z = Zs + 9 * (a + 1);
      const double* S = Ss + 3 * (a + 1);
      double cm[3][3], cp[3][3], cf[3][3];
      for (p = 0; p < 3; ++p) {
        double wm = S[p] < 0.0 ? 1.0 : (S[p] == 0.0 ? 0.5 : 0.0);
        double wp = S[p] > 0.0 ? 1.0 : (S[p] == 0.0 ? 0.5 : 0.0);
        for (k = 0; k < 3; ++k) {
          cm[p][k] = Z[3 * p + k] * wm;
          cp[p][k] = Z[3 * p + k] * wp;
          cf[p][k] = 0.0;
        }
        if (order >= 2 && S[p] != 0.0 && !wd[a + 1]) {
          double zz = dot3(Z + 3 * p, Z + 3 * p);
          if (zz != 0.0) {
            int up = S[p] > 0.0 ? a - 1 : a + 1;
            double th = dot3(Zs + 9 * (up + 1) + 3 * p, Z + 3 * p) / zz;
            double phi = mc_limiter(th);
            double sg = S[p] > 0.0 ? 1.0 : -1.0;
            double as = S[p] > 0.0 ? S[p] : -S[p];
            double coef = 0.5 * sg * (1.0 - nu * as) * phi;
            for (k = 0; k < 3; ++k) cf[p][k] = coef * Z[3 * p + k];
          }
        }
        if (c >= 0 && c < nc) {
          double as = S[p] > 0.0 ? S[p] : -S[p];
          if (as > *smax) *smax = as;
        }
      }
      for (k = 0; k < 3; ++k) {
        AM[3 * a + k] = (cm[0][k] + cm[2][k]) + cm[1][k];
        AP[3 * a + k] = (cp[0][k] + cp[2][k]) + cp[1][k];
        FF[3 * a + k] = (cf[0][k] + cf[2][k]) + cf[1][k];
      }
    }
    /* per-cell increments (normal frame -> h, hu, hv) */
    for (a = 0; a < na; ++a) {
      double dd[3];
      for (k = 0; k < 3; ++k)
        dd[k] = (AP[3 * a + k] + AM[3 * (a + 1) + k]) +
                (FF[3 * (a + 1) + k] - FF[3 * a + k]);
      int i = dir == 0 ? a : c, j = dir == 0 ? c : a;
      double* o = dq + 3 * ((i + NG) + (j + NG) * W);
      o[0] = dd[0];
      o[dir == 0 ? 1 : 2] = dd[1];
      o[dir == 0 ? 2 : 1] = dd[2];
    }
  }
  free(Zs); free(Ss); free(AM); free(AP); free(FF); free(wd);
}

/* Transverse fluxes from the increments of a sweep in direction dir.  The
 * increments are split along the other direction; the flux at the cross
 * edge between cells k-1 and k (stored at cell k) is
 *   -0.5 * nu * (plus-part of cell k-1 + minus-part of cell k). */
static void transverse(int dir, int nx, int ny, const double* h,
                       const double* hu, const double* hv, const double* b,
                       const double* dq, double nu, double g, double drytol,
                       double* tr) {
  int W = nx + 2 * NG, H = ny + 2 * NG;
  int sd = 1 - dir; /* split direction */
  double* PL = (double*)calloc((size_t)3 * W * H, sizeof(double));
  double* MI = (double*)calloc((size_t)3 * W * H, sizeof(double));
  int na = dir == 0 ? nx : ny;
  int nc = dir == 0 ? ny : nx;
  int a, c, k;
  for (c = -1; c <= nc; ++c)
    for (a = 0; a < na; ++a) {
      int i = dir == 0 ? a : c, j = dir == 0 ? c : a;
      int id = (i + NG) + (j + NG) * W;
      int im = sd == 0 ? id - 1 : id - W;
      int ip = sd == 0 ? id + 1 : id + W;
      transverse_split(sd, h[id], hu[id], hv[id], b[id], h[im], b[im], h[ip],
                       b[ip], dq + 3 * id, g, drytol, PL + 3 * id,
                       MI + 3 * id);
    }
  for (c = 0; c <= nc; ++c)
    for (a = 0; a < na; ++a) {
      int i = dir == 0 ? a : c, j = dir == 0 ? c : a;
      int id = (i + NG) + (j + NG) * W;
      int im = sd == 0 ? id - 1 : id - W;
      for (k = 0; k < 3; ++k)
        tr[3 * id + k] = -0.5 * nu * (PL[3 * im + k] + MI[3 * id + k]);
    }
  free(PL); free(MI);
}

/* The Manning step of Eq. (manning) on one updated cell r = (h, hu, hv):
 * semi-implicit, on wet cells, after the hyperbolic update; momenta zeroed
 * where the cell is dry. */
static void friction(double* r, double dt, double g, double drytol, double manning_n) {
  if (manning_n > 0.0 && r[0] > drytol) {
    double u = r[1] / r[0], v = r[2] / r[0];
    double sp = sqrt(u * u + v * v);
    double D = g * manning_n * manning_n * sp / (r[0] * cbrt(r[0]));
    double den = 1.0 + dt * D;
    r[1] = r[1] / den;
    r[2] = r[2] / den;
  }
  if (r[0] <= drytol) { r[1] = 0.0; r[2] = 0.0; }
}

void oracle_step_grid_ex(int nx, int ny, const double* h, const double* hu,
                         const double* hv, const double* b, double dx, double dy,
                         double dt, double g, double drytol, double manning_n,
                         int order, int transv, int dim_split, double* hn,
                         double* hun, double* hvn, double* cmax, long* nclip,
                         double* clipdepth) {
  int W = nx + 2 * NG, H = ny + 2 * NG;
  size_t N = (size_t)W * H;
  double clipsum = 0.0;
  double* dqx = (double*)calloc(3 * N, sizeof(double));
  double* dqy = (double*)calloc(3 * N, sizeof(double));
  double* gtr = (double*)calloc(3 * N, sizeof(double));
  double* ftr = (double*)calloc(3 * N, sizeof(double));
  double nux = dt / dx, nuy = dt / dy;
  double smx = 0.0, smy = 0.0;
  long clip = 0;
  int i, j, k;

  memcpy(hn, h, sizeof(double) * N);
  memcpy(hun, hu, sizeof(double) * N);
  memcpy(hvn, hv, sizeof(double) * N);
  if (!dim_split) {
    /* unsplit: both sweeps from Q^n, transverse terms optional */
    sweep(0, nx, ny, h, hu, hv, b, nux, g, drytol, dqx, &smx, order, -1, ny);
    if (transv) transverse(0, nx, ny, h, hu, hv, b, dqx, nux, g, drytol, gtr);
    sweep(1, nx, ny, h, hu, hv, b, nuy, g, drytol, dqy, &smy, order, -1, nx);
    if (transv) transverse(1, nx, ny, h, hu, hv, b, dqy, nuy, g, drytol, ftr);
    for (j = 0; j < ny; ++j)
      for (i = 0; i < nx; ++i) {
        int id = (i + NG) + (j + NG) * W;
        double q[3] = {h[id], hu[id], hv[id]};
        double r[3];
        for (k = 0; k < 3; ++k) {
          double fl = nux * dqx[3 * id + k] + nuy * dqy[3 * id + k];
          double tf = nux * (ftr[3 * (id + 1) + k] - ftr[3 * id + k]) +
                      nuy * (gtr[3 * (id + W) + k] - gtr[3 * id + k]);
          r[k] = (q[k] - fl) - tf;
        }
        if (r[0] < 0.0) { clipsum -= r[0]; r[0] = 0.0; ++clip; }
        friction(r, dt, g, drytol, manning_n);
        hn[id] = r[0]; hun[id] = r[1]; hvn[id] = r[2];
      }
  } else {
    /* dimensional splitting: the x-sweep updates every row of the interior
     * columns (ghost rows included), the y-sweep runs on that state */
    double* hs = (double*)malloc(sizeof(double) * N);
    double* hus = (double*)malloc(sizeof(double) * N);
    double* hvs = (double*)malloc(sizeof(double) * N);
    memcpy(hs, h, sizeof(double) * N);
    memcpy(hus, hu, sizeof(double) * N);
    memcpy(hvs, hv, sizeof(double) * N);
    sweep(0, nx, ny, h, hu, hv, b, nux, g, drytol, dqx, &smx, order, -2, ny + 1);
    for (j = -2; j < ny + 2; ++j)
      for (i = 0; i < nx; ++i) {
        int id = (i + NG) + (j + NG) * W;
        double r[3] = {h[id] - nux * dqx[3 * id], hu[id] - nux * dqx[3 * id + 1],
                       hv[id] - nux * dqx[3 * id + 2]};
        if (r[0] < 0.0) {
          if (j >= 0 && j < ny) { clipsum -= r[0]; ++clip; }
          r[0] = 0.0;
        }
        if (r[0] <= drytol) { r[1] = 0.0; r[2] = 0.0; }
        hs[id] = r[0]; hus[id] = r[1]; hvs[id] = r[2];
      }
    sweep(1, nx, ny, hs, hus, hvs, b, nuy, g, drytol, dqy, &smy, order, 0, nx - 1);
    for (j = 0; j < ny; ++j)
      for (i = 0; i < nx; ++i) {
        int id = (i + NG) + (j + NG) * W;
        double r[3] = {hs[id] - nuy * dqy[3 * id], hus[id] - nuy * dqy[3 * id + 1],
                       hvs[id] - nuy * dqy[3 * id + 2]};
        if (r[0] < 0.0) { clipsum -= r[0]; r[0] = 0.0; ++clip; }
        friction(r, dt, g, drytol, manning_n);
        hn[id] = r[0]; hun[id] = r[1]; hvn[id] = r[2];
      }
    free(hs); free(hus); free(hvs);
  }
  double cx = smx / dx, cy = smy / dy;
  *cmax = cx > cy ? cx : cy;
  *nclip = clip;
  *clipdepth = clipsum;
  free(dqx); free(dqy); free(gtr); free(ftr);
}

void oracle_step_grid(int nx, int ny, const double* h, const double* hu,
                      const double* hv, const double* b, double dx, double dy,
                      double dt, double g, double drytol, double manning_n,
                      double* hn, double* hun, double* hvn, double* cmax,
                      long* nclip, double* clipdepth) {
  oracle_step_grid_ex(nx, ny, h, hu, hv, b, dx, dy, dt, g, drytol, manning_n, 2, 1, 0,
                      hn, hun, hvn, cmax, nclip, clipdepth);
}

/* ------------------------------------------------------------------------ */
/* Topography: cell average of the bilinear interpolant of one DEM (Sec. 6.2 */
/* conservative topography integral, one DEM).                               */
/* ------------------------------------------------------------------------ */

static double dem_eval(const double* z, int nx, int ny, double x0, double y0,
                       double dx, double dy, double x, double y) {
  double fx = (x - x0) / dx, fy = (y - y0) / dy;
  if (fx < 0.0) fx = 0.0;
  if (fx > (double)(nx - 1)) fx = (double)(nx - 1);
  if (fy < 0.0) fy = 0.0;
  if (fy > (double)(ny - 1)) fy = (double)(ny - 1);
  int i = (int)floor(fx), j = (int)floor(fy);
  if (i > nx - 2) i = nx - 2;
  if (j > ny - 2) j = ny - 2;
  if (i < 0) i = 0;
  if (j < 0) j = 0;
  double ax = fx - (double)i, ay = fy - (double)j;
  double z00 = z[i + (size_t)j * nx], z10 = z[i + 1 + (size_t)j * nx];
  double z01 = z[i + (size_t)(j + 1) * nx];
  double z11 = z[i + 1 + (size_t)(j + 1) * nx];
  return (1.0 - ay) * ((1.0 - ax) * z00 + ax * z10) +
         ay * ((1.0 - ax) * z01 + ax * z11);
}

/* Break points of [a, b] at the DEM node lines strictly inside it. */
static int dem_breaks(double a, double b, double o, double d, int n,
                      double* out) {
  int m = 0;
  out[m++] = a;
  int lo = (int)floor((a - o) / d) - 1, hi = (int)ceil((b - o) / d) + 1;
  if (lo < 0) lo = 0;
  if (hi > n - 1) hi = n - 1;
  int i;
  for (i = lo; i <= hi; ++i) {
    double xn = o + (double)i * d;
    if (xn > a && xn < b) out[m++] = xn;
  }
  out[m++] = b;
  return m;
}

/* Priority order of n DEMs (Sec. 6.2: several overlapping DEMs of different
 * resolutions): the finer node spacing (smaller dx * dy) first, equal
 * spacings in the given order. */
static void dem_order(int n, const double* dx, const double* dy, int* ord) {
  int i, j;
  for (i = 0; i < n; ++i) ord[i] = i;
  for (i = 1; i < n; ++i) /* insertion sort: stable */
    for (j = i; j > 0 && dx[ord[j]] * dy[ord[j]] < dx[ord[j - 1]] * dy[ord[j - 1]]; --j) {
      int t = ord[j]; ord[j] = ord[j - 1]; ord[j - 1] = t;
    }
}

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Sorted distinct break points of [a, b]: its ends and every DEM's node
 * lines strictly inside it.  Returns the count. */
static int dems_breaks(int n, const int* ord, const double* o, const double* d,
                       const int* nn, double a, double b, double** out) {
  size_t cap = 2;
  int k, m = 0;
  for (k = 0; k < n; ++k) cap += (size_t)((b - a) / d[ord[k]]) + 4;
  double* v = (double*)malloc(sizeof(double) * cap);
  v[m++] = a;
  for (k = 0; k < n; ++k) {
    int q = ord[k];
    int lo = (int)floor((a - o[q]) / d[q]) - 1, hi = (int)ceil((b - o[q]) / d[q]) + 1;
    if (lo < 0) lo = 0;
    if (hi > nn[q] - 1) hi = nn[q] - 1;
    for (int i = lo; i <= hi; ++i) {
      double xn = o[q] + (double)i * d[q];
      if (xn > a && xn < b) v[m++] = xn;
    }
  }
  v[m++] = b;
  qsort(v, (size_t)m, sizeof(double), cmp_double);
  int u = 0;
  for (k = 0; k < m; ++k)
    if (u == 0 || v[k] != v[u - 1]) v[u++] = v[k];
  *out = v;
  return u;
}

/* Composite interpolant at (x, y): the bilinear interpolant of the first
 * DEM in priority order whose extent (closed, node to node) holds the
 * point; outside every extent the last one's, extended as a constant
 * beyond its edges. */
static double dems_eval(int n, const int* ord, const double* const* z,
                        const int* nx, const int* ny, const double* x0,
                        const double* y0, const double* dx, const double* dy,
                        double x, double y) {
  int k;
  for (k = 0; k < n; ++k) {
    int q = ord[k];
    double xe = x0[q] + (double)(nx[q] - 1) * dx[q];
    double ye = y0[q] + (double)(ny[q] - 1) * dy[q];
    if (x >= x0[q] && x <= xe && y >= y0[q] && y <= ye) break;
  }
  int q = ord[k < n ? k : n - 1];
  return dem_eval(z[q], nx[q], ny[q], x0[q], y0[q], dx[q], dy[q], x, y);
}

double oracle_dems_average(int n, const double* const* z, const int* nx,
                           const int* ny, const double* x0, const double* y0,
                           const double* dx, const double* dy, double xa,
                           double xb, double ya, double yb) {
  /* Every DEM's node lines (and hence every extent edge) are break points,
   * so the composite interpolant is bilinear on each piece of the partition
   * and its integral over a piece is the piece area times its midpoint
   * value (the integral that the AMR keeps under refinement, Sec. 6.2). */
  int ord[ORACLE_MAXDEM];
  double *xs, *ys;
  dem_order(n, dx, dy, ord);
  int mx = dems_breaks(n, ord, x0, dx, nx, xa, xb, &xs);
  int my = dems_breaks(n, ord, y0, dy, ny, ya, yb, &ys);
  double sum = 0.0;
  int k, l;
  for (l = 0; l + 1 < my; ++l)
    for (k = 0; k + 1 < mx; ++k) {
      double xm = 0.5 * (xs[k] + xs[k + 1]);
      double ym = 0.5 * (ys[l] + ys[l + 1]);
      double w = (xs[k + 1] - xs[k]) * (ys[l + 1] - ys[l]);
      sum += w * dems_eval(n, ord, z, nx, ny, x0, y0, dx, dy, xm, ym);
    }
  free(xs);
  free(ys);
  return sum / ((xb - xa) * (yb - ya));
}

double oracle_dem_average(const double* z, int nx, int ny, double x0,
                          double y0, double dx, double dy, double xa,
                          double xb, double ya, double yb) {
  const double* zz[1] = {z};
  return oracle_dems_average(1, zz, &nx, &ny, &x0, &y0, &dx, &dy, xa, xb, ya, yb);
}

/* ------------------------------------------------------------------------ */
/* Quadtree forest of fixed-size patches, Sec. 4.                            */
/* ------------------------------------------------------------------------ */

struct oracle_forest {
  oracle_config c;
  int M, T; /* patch cells per side, tile side M + 4 */
  int np;
  int *lev, *px, *py;
  double** tile; /* per patch: h, hu, hv, b, each T*T */
  int* lut[MAXLEV];
  int lutw[MAXLEV], luth[MAXLEV];
  int ndem; /* DEMs (0: flat bed at 0) */
  double* dem[ORACLE_MAXDEM];
  int dnx[ORACLE_MAXDEM], dny[ORACLE_MAXDEM];
  double dx0[ORACLE_MAXDEM], dy0[ORACLE_MAXDEM], ddx[ORACLE_MAXDEM], ddy[ORACLE_MAXDEM];
  double t, dt_next;
  /* level subcycling: during a macro step, prev[p] holds patch p's state
   * before its latest step and sub_k the fine substep; ghost cells are then
   * filled from states interpolated in time (NULL outside a macro step) */
  double** prev;
  long sub_k;
  double tg; /* time of the ghost values being filled */
  long steps, rejects, nclip;
  double clipvol; /* volume added by resetting negative depths to zero */
  int ngauge;
  double *gxy, *gout, *garr;
};

static long NXL(const oracle_forest* f, int L) {
  return (long)f->c.mi * f->M * (1L << L);
}
static long NYL(const oracle_forest* f, int L) {
  return (long)f->c.mj * f->M * (1L << L);
}
static double DXL(const oracle_forest* f, int L) {
  return (f->c.xupper - f->c.xlower) / (double)NXL(f, L);
}
static double DYL(const oracle_forest* f, int L) {
  return (f->c.yupper - f->c.ylower) / (double)NYL(f, L);
}
static size_t TI(const oracle_forest* f, int i, int j) {
  return (size_t)(i + NG) + (size_t)(j + NG) * f->T;
}

/* Morton key of a patch on the finest patch grid. */
static uint64_t morton(const oracle_forest* f, int L, int px, int py) {
  uint64_t X = (uint64_t)px << (f->c.maxlevel - L);
  uint64_t Y = (uint64_t)py << (f->c.maxlevel - L);
  uint64_t key = 0;
  int bit;
  for (bit = 0; bit < 31; ++bit) {
    key |= ((X >> bit) & 1ULL) << (2 * bit);
    key |= ((Y >> bit) & 1ULL) << (2 * bit + 1);
  }
  return key;
}

static void build_lut(oracle_forest* f) {
  int L, k;
  for (L = 0; L <= f->c.maxlevel; ++L) {
    int w = f->c.mi << L, h = f->c.mj << L;
    free(f->lut[L]);
    f->lut[L] = (int*)malloc(sizeof(int) * (size_t)w * h);
    f->lutw[L] = w;
    f->luth[L] = h;
    for (k = 0; k < w * h; ++k) f->lut[L][k] = -1;
  }
  for (k = 0; k < f->np; ++k)
    f->lut[f->lev[k]][f->px[k] + f->py[k] * f->lutw[f->lev[k]]] = k;
}

/* Patch index of the leaf at exactly level L holding cell (I, J), or -1. */
static int leaf_at(const oracle_forest* f, int L, long I, long J) {
  long P = I / f->M, Q = J / f->M;
  if (P < 0 || Q < 0 || P >= f->lutw[L] || Q >= f->luth[L]) return -1;
  return f->lut[L][P + Q * f->lutw[L]];
}

/* Composite value of the leaves at cell (I, J) of level L: the leaf's own
 * cell, a coarser leaf's cell (injection) or the mean of the four finer
 * cells.  out = h, hu, hv, b. */
/* Fields 0..nf-1 of tile cell id of patch p at the time the ghost cells are
 * being filled: the stored state, or during a subcycled macro step, for a
 * level between two of its steps, the linear interpolation in time of h, hu
 * and hv between the states before and after its latest step (the bed does
 * not change in time). */
static void cell_read(const oracle_forest* f, int p, size_t id, int nf, double* out) {
  size_t TT = (size_t)f->T * f->T;
  int k;
  for (k = 0; k < nf; ++k) out[k] = f->tile[p][k * TT + id];
  if (!f->prev) return;
  long P = 1L << (f->c.maxlevel - f->lev[p]);
  long r = f->sub_k % P;
  if (r == 0) return;
  double a = (double)r / (double)P;
  for (k = 0; k < nf && k < 3; ++k)
    out[k] = (1.0 - a) * f->prev[p][k * TT + id] + a * f->tile[p][k * TT + id];
}

static void value_at(const oracle_forest* f, int L, long I, long J,
                     double* out) {
  int l, k;
  for (l = L; l >= 0; --l) {
    long Il = I >> (L - l), Jl = J >> (L - l);
    int p = leaf_at(f, l, Il, Jl);
    if (p >= 0) {
      int i = (int)(Il - (long)f->px[p] * f->M);
      int j = (int)(Jl - (long)f->py[p] * f->M);
      cell_read(f, p, TI(f, i, j), 4, out);
      return;
    }
  }
  if (L >= f->c.maxlevel) { /* not covered: cannot happen in a forest */
    for (k = 0; k < 4; ++k) out[k] = 0.0;
    return;
  }
  double v[4][4];
  value_at(f, L + 1, 2 * I, 2 * J, v[0]);
  value_at(f, L + 1, 2 * I + 1, 2 * J, v[1]);
  value_at(f, L + 1, 2 * I, 2 * J + 1, v[2]);
  value_at(f, L + 1, 2 * I + 1, 2 * J + 1, v[3]);
  for (k = 0; k < 4; ++k) out[k] = 0.25 * ((v[0][k] + v[1][k]) + (v[2][k] + v[3][k]));
}

static double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

/* Beds of the four cells of a tile that share a parent with tile cell
 * (i, j): bs[b][a] is the child at x offset a and y offset b.  Patch
 * origins are even, so siblings have the same tile up to the last bit of
 * the local index, ghost cells included. */
static void child_beds(const oracle_forest* f, const double* bed, int i, int j,
                       double bs[2][2]) {
  int i0 = i & ~1, j0 = j & ~1, a, b;
  for (b = 0; b < 2; ++b)
    for (a = 0; a < 2; ++a) bs[b][a] = bed[TI(f, i0 + a, j0 + b)];
}

/* Value of (h, hu, hv) for cell (I, J) of level L whose parent's four
 * children have the beds bs (bs[J & 1][I & 1] is this cell's): copy from a
 * leaf of the same level, mean of the four cells of finer leaves, or
 * interpolation of the coarser level (ghost-cell exchange, Sec. 4 and the
 * quadtree figure; Sec. 6.2 for the surface-based interpolation that keeps
 * lake at rest).  The interpolation treats the parent's four children
 * together:
 *   depth: the interpolated surface (minmod-limited linear when the parent's
 *     3x3 neighbourhood is wet, the parent's surface otherwise) minus the
 *     child's bed, clamped at zero;
 *   momentum: minmod-limited linear interpolation when the neighbourhood is
 *     wet and no wet child's velocity leaves the range of the
 *     neighbourhood's velocities; otherwise the parent's momentum split in
 *     proportion to the children's depths.  Either way the children hold
 *     the parent's momentum, and a shallow child under a deep parent does
 *     not take a velocity the coarse flow does not have. */
static void fill_cell(const oracle_forest* f, int L, long I, long J,
                      const double bs[2][2], double* out) {
  int p = leaf_at(f, L, I, J);
  int k, l;
  if (p >= 0) {
    int i = (int)(I - (long)f->px[p] * f->M), j = (int)(J - (long)f->py[p] * f->M);
    cell_read(f, p, TI(f, i, j), 3, out);
    return;
  }
  int coarser = 0;
  for (l = L - 1; l >= 0; --l)
    if (leaf_at(f, l, I >> (L - l), J >> (L - l)) >= 0) { coarser = 1; break; }
  if (!coarser) {
    double v[4][4];
    value_at(f, L + 1, 2 * I, 2 * J, v[0]);
    value_at(f, L + 1, 2 * I + 1, 2 * J, v[1]);
    value_at(f, L + 1, 2 * I, 2 * J + 1, v[2]);
    value_at(f, L + 1, 2 * I + 1, 2 * J + 1, v[3]);
    for (k = 0; k < 3; ++k)
      out[k] = 0.25 * ((v[0][k] + v[1][k]) + (v[2][k] + v[3][k]));
    return;
  }
  /* interpolation from level L-1 */
  long ic = I >> 1, jc = J >> 1;
  long NXc = NXL(f, L - 1), NYc = NYL(f, L - 1);
  double nb[3][3][4];
  int in[3][3];
  int di, dj, a, b;
  for (dj = -1; dj <= 1; ++dj)
    for (di = -1; di <= 1; ++di) {
      long x = ic + di, y = jc + dj;
      in[dj + 1][di + 1] = x >= 0 && y >= 0 && x < NXc && y < NYc;
      if (in[dj + 1][di + 1]) value_at(f, L - 1, x, y, nb[dj + 1][di + 1]);
    }
  const double* qc = nb[1][1];
  double drytol = f->c.drytol;
  if (qc[0] <= drytol) {
    out[0] = qc[0]; out[1] = qc[1]; out[2] = qc[2];
    return;
  }
  int allwet = 1;
  for (dj = 0; dj < 3; ++dj)
    for (di = 0; di < 3; ++di)
      if (in[dj][di] && !(nb[dj][di][0] > drytol)) allwet = 0;
  double etac = qc[0] + qc[3];
  /* limited slopes per coarse cell of the surface and both momenta */
  double g[3][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
  if (allwet) {
    int hx = in[1][0] && in[1][2], hy = in[0][1] && in[2][1];
    double e[3][3];
    for (dj = 0; dj < 3; ++dj)
      for (di = 0; di < 3; ++di)
        e[dj][di] = in[dj][di] ? nb[dj][di][0] + nb[dj][di][3] : 0.0;
    if (hx) g[0][0] = minmod(e[1][2] - e[1][1], e[1][1] - e[1][0]);
    if (hy) g[0][1] = minmod(e[2][1] - e[1][1], e[1][1] - e[0][1]);
    for (k = 1; k < 3; ++k) {
      if (hx) g[k][0] = minmod(nb[1][2][k] - qc[k], qc[k] - nb[1][0][k]);
      if (hy) g[k][1] = minmod(nb[2][1][k] - qc[k], qc[k] - nb[0][1][k]);
    }
  }
  /* the four children: depth d and linearly interpolated momenta m */
  double d[2][2], m[2][2][2];
  for (b = 0; b < 2; ++b)
    for (a = 0; a < 2; ++a) {
      double sx = a ? 0.25 : -0.25, sy = b ? 0.25 : -0.25;
      double eta = allwet ? (etac + sx * g[0][0]) + sy * g[0][1] : etac;
      double h = eta - bs[b][a];
      d[b][a] = h > 0.0 ? h : 0.0;
      for (k = 0; k < 2; ++k)
        m[b][a][k] = (qc[k + 1] + sx * g[k + 1][0]) + sy * g[k + 1][1];
    }
  double S = (d[0][0] + d[0][1]) + (d[1][0] + d[1][1]);
  int a0 = (int)(I & 1), b0 = (int)(J & 1);
  double hf = d[b0][a0];
  out[0] = hf;
  for (k = 0; k < 2; ++k) {
    int split = !allwet;
    if (allwet) {
      double lo = INFINITY, hi = -INFINITY;
      for (dj = 0; dj < 3; ++dj)
        for (di = 0; di < 3; ++di)
          if (in[dj][di]) {
            double u = nb[dj][di][k + 1] / nb[dj][di][0];
            if (u < lo) lo = u;
            if (u > hi) hi = u;
          }
      for (b = 0; b < 2; ++b)
        for (a = 0; a < 2; ++a)
          if (d[b][a] > drytol) {
            double u = m[b][a][k] / d[b][a];
            if (u < lo || u > hi) split = 1;
          }
    }
    if (!split) out[k + 1] = m[b0][a0][k];
    else out[k + 1] = S > 0.0 ? (4.0 * qc[k + 1]) * (hf / S) : 0.0;
  }
  if (hf <= drytol) { out[1] = 0.0; out[2] = 0.0; }
}

/* ---------------------------------------------------------------------- */
/* Inflow hydrograph (Sec. 5.1, Test Case 1 set-up)                         */
/* ---------------------------------------------------------------------- */

double oracle_hydrograph(const oracle_config* c, double t) {
  int n = c->n_hydro, k;
  if (n <= 0) return 0.0;
  if (t <= c->hydro_t[0]) return c->hydro_q[0];
  if (t >= c->hydro_t[n - 1]) return c->hydro_q[n - 1];
  for (k = 0; k + 1 < n; ++k)
    if (t < c->hydro_t[k + 1]) break;
  double a = (t - c->hydro_t[k]) / (c->hydro_t[k + 1] - c->hydro_t[k]);
  return c->hydro_q[k] + (c->hydro_q[k + 1] - c->hydro_q[k]) * a;
}

/* Eq. riemann as F(h) = q/h - 2 sqrt(g h) - u_i + 2 sqrt(g h_i), and
 * Eq. 2-shock as F(h) = q/h - u_i - (h - h_i) sqrt(g/2 (1/h + 1/h_i)); both
 * decrease in h on the range searched.  Returns F, *dF its derivative. */
static double inflow_eq(int shock, double h, double q, double hi, double ui,
                        double g, double* dF) {
  if (!shock) {
    *dF = -q / (h * h) - sqrt(g / h);
    return q / h - 2.0 * sqrt(g * h) - ui + 2.0 * sqrt(g * hi);
  }
  double S = sqrt(0.5 * g * (1.0 / h + 1.0 / hi));
  *dF = -q / (h * h) - S + (h - hi) * g / (4.0 * h * h * S);
  return q / h - ui - (h - hi) * S;
}

/* Newton's method from h0 for the root of a decreasing F above lo (F > 0
 * just above lo).  The iterates are kept inside the bracket the signs of F
 * have established so far; a Newton step that leaves it is replaced by the
 * bracket's midpoint (or a doubling while no upper end is known). */
static double inflow_newton(int shock, double h0, double lo, double q,
                            double hi_, double ui, double g) {
  double hi = INFINITY, h = h0 > lo ? h0 : 2.0 * lo;
  int it;
  for (it = 0; it < 100; ++it) {
    double dF, F = inflow_eq(shock, h, q, hi_, ui, g, &dF);
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

double oracle_inflow_depth(double q, double h_int, double qn_int, double g,
                           double tau, double* h_used, double* u_used) {
  double hi, ui;
  if (h_int < tau) {
    /* too thin an interior cell (dry included): critical depth of the
     * inflow, at least tau, at rest */
    double hc = cbrt(q * q / g);
    hi = hc > tau ? hc : tau;
    ui = 0.0;
  } else {
    hi = h_int;
    ui = qn_int / h_int;
  }
  if (h_used) *h_used = hi;
  if (u_used) *u_used = ui;
  /* first guess [F q / sqrt(g)]^(2/3), F = 0.5 for Eq. riemann */
  double h = inflow_newton(0, cbrt(0.25 * q * q / g), 0.0, q, hi, ui, g);
  if (h > hi) h = inflow_newton(1, cbrt(q * q / g), hi, q, hi, ui, g);
  return h;
}

/* Inflow ghosts of side `side` of tile p (a tile on that side) after all its
 * mirrors are set: each
 * row (or column) of the tile whose centre lies in the inflow segment and
 * inside the domain gets, in both ghost layers, the depth of Eq. riemann /
 * Eq. 2-shock from the tile's first cell of that line, the unit discharge
 * normal to the side into the domain and no tangential momentum.  With no
 * discharge the side's own rule stays. */
/* Width of the inflow segment as the grid of level L represents it: the
 * number of lines (rows or columns of the side) whose centre lies in
 * [inflow_lo, inflow_hi], times the cell size. */
static double inflow_width(const oracle_forest* f, int L) {
  const oracle_config* c = &f->c;
  int xs = c->inflow_side <= 1;
  long N = xs ? NYL(f, L) : NXL(f, L), J, n = 0;
  double d = xs ? DYL(f, L) : DXL(f, L);
  double o = xs ? c->ylower : c->xlower;
  long J0 = (long)floor((c->inflow_lo - o) / d) - 1, J1 = (long)ceil((c->inflow_hi - o) / d) + 1;
  if (J0 < 0) J0 = 0;
  if (J1 > N - 1) J1 = N - 1;
  for (J = J0; J <= J1; ++J) {
    double ctr = o + ((double)J + 0.5) * d;
    if (ctr >= c->inflow_lo && ctr <= c->inflow_hi) ++n;
  }
  return (double)n * d;
}

static void fill_inflow(const oracle_forest* f, int p, int side) {
  const oracle_config* c = &f->c;
  double Q = oracle_hydrograph(c, f->prev ? f->tg : f->t);
  if (!(Q > 0.0)) return;
  int L = f->lev[p], M = f->M, l, g;
  double wd = inflow_width(f, L);
  if (!(wd > 0.0)) return; /* the segment holds no line centre at this level */
  double q = Q / wd;
  size_t TT = (size_t)f->T * f->T;
  double* t = f->tile[p];
  int xs = side <= 1; /* the side is a left or right one: lines are rows */
  long N = xs ? NYL(f, L) : NXL(f, L);
  double d = xs ? DYL(f, L) : DXL(f, L);
  double o = xs ? c->ylower : c->xlower;
  long base = xs ? (long)f->py[p] * M : (long)f->px[p] * M;
  double sg = (side == 0 || side == 2) ? 1.0 : -1.0;
  for (l = -NG; l < M + NG; ++l) {
    long J = base + l;
    if (J < 0 || J >= N) continue;
    double ctr = o + ((double)J + 0.5) * d;
    if (!(ctr >= c->inflow_lo && ctr <= c->inflow_hi)) continue;
    int a0 = (side == 0 || side == 2) ? 0 : M - 1; /* first interior cell */
    size_t id = xs ? TI(f, a0, l) : TI(f, l, a0);
    double hin = t[id];
    double qn = sg * t[(xs ? 1 : 2) * TT + id];
    double hg = oracle_inflow_depth(q, hin, qn, c->g, c->inflow_tau, NULL, NULL);
    for (g = 1; g <= NG; ++g) {
      int ag = (side == 0 || side == 2) ? -g : M - 1 + g;
      size_t gid = xs ? TI(f, ag, l) : TI(f, l, ag);
      t[gid] = hg;
      t[(xs ? 1 : 2) * TT + gid] = sg * q;
      t[(xs ? 2 : 1) * TT + gid] = 0.0;
    }
  }
  /* where the tile also touches a side across the segment's lines, the
   * corner ghosts beyond the segment's ghost cells follow that side's rule
   * applied to them (wall: mirrored, its normal momentum negated;
   * extrapolation: the nearest one copied), so a segment spanning a whole
   * side next to walls leaves one-dimensional flow one-dimensional */
  for (int end = 0; end < 2; ++end) {
    int pside = xs ? 2 + end : end; /* the side across the lines */
    int at = end == 0 ? base == 0 : base + M == N;
    if (!at) continue;
    int wall = c->bc[pside] == ORACLE_BC_WALL;
    for (g = 1; g <= NG; ++g) {
      int ag = (side == 0 || side == 2) ? -g : M - 1 + g;
      for (int gl = 1; gl <= NG; ++gl) {
        int lt = end == 0 ? -gl : M - 1 + gl;
        int ls = wall ? (end == 0 ? gl - 1 : M - gl) : (end == 0 ? 0 : M - 1);
        size_t dst = xs ? TI(f, ag, lt) : TI(f, lt, ag);
        size_t src = xs ? TI(f, ag, ls) : TI(f, ls, ag);
        for (int k = 0; k < 3; ++k) {
          double v = t[k * TT + src];
          if (wall && k == (xs ? 2 : 1)) v = -v;
          t[k * TT + dst] = v;
        }
      }
    }
  }
}

/* Physical boundary ghosts of one patch tile (Sec. 5.1 closed walls):
 * bottom/top over columns inside the domain, then left/right over all rows.
 * Walls mirror the cells and negate the normal momentum; extrapolation copies
 * the nearest interior cell.  nf = 3 fills h, hu, hv; nf = 4 fills b only. */
static void fill_bc(const oracle_forest* f, int p, int only_b) {
  int L = f->lev[p], M = f->M;
  size_t TT = (size_t)f->T * f->T;
  double* q = f->tile[p];
  long NX = NXL(f, L), NY = NYL(f, L);
  int f0 = only_b ? 3 : 0, f1 = only_b ? 4 : 3;
  int i, j, g, k;
  /* bottom (side 2) and top (side 3) */
  for (int side = 2; side <= 3; ++side) {
    int atb = side == 2 ? (f->py[p] == 0) : ((long)(f->py[p] + 1) * M == NY);
    if (!atb) continue;
    int wall = f->c.bc[side] == ORACLE_BC_WALL;
    for (i = -NG; i < M + NG; ++i) {
      long I = (long)f->px[p] * M + i;
      if (I < 0 || I >= NX) continue;
      for (g = 1; g <= NG; ++g) {
        int jg = side == 2 ? -g : M - 1 + g;
        int js = wall ? (side == 2 ? g - 1 : M - g) : (side == 2 ? 0 : M - 1);
        for (k = f0; k < f1; ++k) {
          double v = q[k * TT + TI(f, i, js)];
          if (wall && k == 2) v = -v;
          q[k * TT + TI(f, i, jg)] = v;
        }
      }
    }
  }
  for (int side = 0; side <= 1; ++side) {
    int atb = side == 0 ? (f->px[p] == 0) : ((long)(f->px[p] + 1) * M == NX);
    if (!atb) continue;
    int wall = f->c.bc[side] == ORACLE_BC_WALL;
    for (j = -NG; j < M + NG; ++j)
      for (g = 1; g <= NG; ++g) {
        int ig = side == 0 ? -g : M - 1 + g;
        int is = wall ? (side == 0 ? g - 1 : M - g) : (side == 0 ? 0 : M - 1);
        for (k = f0; k < f1; ++k) {
          double v = q[k * TT + TI(f, is, j)];
          if (wall && k == 1) v = -v;
          q[k * TT + TI(f, ig, j)] = v;
        }
      }
  }
  /* the inflow segment's ghost cells last: the cells diagonal to the
   * segment (tile corners) keep the mirrors of the side's own rule */
  if (!only_b && f->c.n_hydro > 0) {
    int side = f->c.inflow_side;
    int at = side == 0   ? f->px[p] == 0
             : side == 1 ? (long)(f->px[p] + 1) * M == NXL(f, L)
             : side == 2 ? f->py[p] == 0
                         : (long)(f->py[p] + 1) * M == NYL(f, L);
    if (at) fill_inflow(f, p, side);
  }
}

/* Bed of every tile cell inside the domain from the DEM at the patch's own
 * level; outside the domain by the boundary rule. */
static void fill_topo(oracle_forest* f, int p) {
  int L = f->lev[p], M = f->M, T = f->T;
  size_t TT = (size_t)T * T;
  double dx = DXL(f, L), dy = DYL(f, L);
  long NX = NXL(f, L), NY = NYL(f, L);
  int i, j;
  for (j = -NG; j < M + NG; ++j)
    for (i = -NG; i < M + NG; ++i) {
      long I = (long)f->px[p] * M + i, J = (long)f->py[p] * M + j;
      double v = 0.0;
      if (I >= 0 && J >= 0 && I < NX && J < NY) {
        if (f->ndem > 0) {
          double xa = f->c.xlower + (double)I * dx;
          double xb = f->c.xlower + (double)(I + 1) * dx;
          double ya = f->c.ylower + (double)J * dy;
          double yb = f->c.ylower + (double)(J + 1) * dy;
          v = oracle_dems_average(f->ndem, (const double* const*)f->dem, f->dnx, f->dny,
                                  f->dx0, f->dy0, f->ddx, f->ddy, xa, xb, ya, yb);
        }
      }
      f->tile[p][3 * TT + TI(f, i, j)] = v;
    }
  fill_bc(f, p, 1);
}

void oracle_forest_ghost_fill(oracle_forest* f) {
  int p, i, j, k;
  size_t TT = (size_t)f->T * f->T;
  int M = f->M;
  /* values from the neighbouring leaves (all reads are leaf interiors) */
  double* buf = (double*)malloc(sizeof(double) * 3 * TT);
  for (p = 0; p < f->np; ++p) {
    int L = f->lev[p];
    long NX = NXL(f, L), NY = NYL(f, L);
    for (j = -NG; j < M + NG; ++j)
      for (i = -NG; i < M + NG; ++i) {
        if (i >= 0 && i < M && j >= 0 && j < M) continue;
        long I = (long)f->px[p] * M + i, J = (long)f->py[p] * M + j;
        if (I < 0 || J < 0 || I >= NX || J >= NY) continue;
        double out[3];
        double bs[2][2];
        child_beds(f, f->tile[p] + 3 * TT, i, j, bs);
        fill_cell(f, L, I, J, bs, out);
        for (k = 0; k < 3; ++k) buf[k * TT + TI(f, i, j)] = out[k];
      }
    /* stage, then write after the patch is done (reads are interiors only,
     * so the order over patches does not matter) */
    for (j = -NG; j < M + NG; ++j)
      for (i = -NG; i < M + NG; ++i) {
        if (i >= 0 && i < M && j >= 0 && j < M) continue;
        long I = (long)f->px[p] * M + i, J = (long)f->py[p] * M + j;
        if (I < 0 || J < 0 || I >= NX || J >= NY) continue;
        for (k = 0; k < 3; ++k)
          f->tile[p][k * TT + TI(f, i, j)] = buf[k * TT + TI(f, i, j)];
      }
    fill_bc(f, p, 0);
  }
  free(buf);
}

static oracle_forest* forest_alloc(const oracle_config* cfg) {
  oracle_forest* f = (oracle_forest*)calloc(1, sizeof(oracle_forest));
  f->c = *cfg;
  f->M = cfg->mx;
  f->T = cfg->mx + 2 * NG;
  f->dt_next = cfg->dt_initial;
  return f;
}

static int cmp_key(const void* a, const void* b) {
  const uint64_t* x = (const uint64_t*)a;
  const uint64_t* y = (const uint64_t*)b;
  return x[0] < y[0] ? -1 : (x[0] > y[0] ? 1 : 0);
}

/* Install a leaf list (level, px, py), Morton-sorted, with fresh tiles. */
static void set_leaves(oracle_forest* f, int n, const int* lev, const int* px,
                       const int* py) {
  uint64_t* kv = (uint64_t*)malloc(sizeof(uint64_t) * 2 * n);
  int k;
  for (k = 0; k < n; ++k) {
    kv[2 * k] = morton(f, lev[k], px[k], py[k]);
    kv[2 * k + 1] = (uint64_t)k;
  }
  qsort(kv, n, 2 * sizeof(uint64_t), cmp_key);
  int* L2 = (int*)malloc(sizeof(int) * n);
  int* X2 = (int*)malloc(sizeof(int) * n);
  int* Y2 = (int*)malloc(sizeof(int) * n);
  for (k = 0; k < n; ++k) {
    int o = (int)kv[2 * k + 1];
    L2[k] = lev[o]; X2[k] = px[o]; Y2[k] = py[o];
  }
  free(kv);
  f->np = n;
  f->lev = L2; f->px = X2; f->py = Y2;
  f->tile = (double**)malloc(sizeof(double*) * n);
  size_t TT = (size_t)f->T * f->T;
  for (k = 0; k < n; ++k) f->tile[k] = (double*)calloc(4 * TT, sizeof(double));
  build_lut(f);
}

oracle_forest* oracle_forest_new(const oracle_config* cfg) {
  if (cfg->mx < 4 || cfg->minlevel < 0 || cfg->maxlevel < cfg->minlevel ||
      cfg->maxlevel >= MAXLEV || cfg->nregions < 0 || cfg->nregions > ORACLE_MAXREGION)
    return NULL;
  oracle_forest* f = forest_alloc(cfg);
  int L = cfg->minlevel;
  int w = cfg->mi << L, h = cfg->mj << L, n = w * h, k;
  int* lev = (int*)malloc(sizeof(int) * n);
  int* px = (int*)malloc(sizeof(int) * n);
  int* py = (int*)malloc(sizeof(int) * n);
  for (k = 0; k < n; ++k) { lev[k] = L; px[k] = k % w; py[k] = k / w; }
  set_leaves(f, n, lev, px, py);
  free(lev); free(px); free(py);
  for (k = 0; k < f->np; ++k) fill_topo(f, k);
  return f;
}

void oracle_forest_free(oracle_forest* f) {
  int k;
  if (!f) return;
  for (k = 0; k < f->np; ++k) free(f->tile[k]);
  free(f->tile); free(f->lev); free(f->px); free(f->py);
  for (k = 0; k < MAXLEV; ++k) free(f->lut[k]);
  for (int k = 0; k < f->ndem; ++k) free(f->dem[k]);
  free(f->gxy); free(f->gout); free(f->garr);
  free(f);
}

int oracle_forest_set_topos(oracle_forest* f, int n, const double* const* z,
                            const int* nx, const int* ny, const double* x0,
                            const double* y0, const double* dx,
                            const double* dy) {
  int k;
  if (n < 1 || n > ORACLE_MAXDEM) return -1;
  for (k = 0; k < n; ++k)
    if (!z[k] || nx[k] < 2 || ny[k] < 2 || !(dx[k] > 0.0) || !(dy[k] > 0.0)) return -1;
  for (k = 0; k < f->ndem; ++k) free(f->dem[k]);
  for (k = 0; k < n; ++k) {
    size_t m = (size_t)nx[k] * ny[k];
    f->dem[k] = (double*)malloc(sizeof(double) * m);
    memcpy(f->dem[k], z[k], sizeof(double) * m);
    f->dnx[k] = nx[k]; f->dny[k] = ny[k];
    f->dx0[k] = x0[k]; f->dy0[k] = y0[k]; f->ddx[k] = dx[k]; f->ddy[k] = dy[k];
  }
  f->ndem = n;
  for (k = 0; k < f->np; ++k) fill_topo(f, k);
  return 0;
}

int oracle_forest_set_topo(oracle_forest* f, const double* z, int nx, int ny,
                           double x0, double y0, double dx, double dy) {
  const double* zz[1] = {z};
  return oracle_forest_set_topos(f, 1, zz, &nx, &ny, &x0, &y0, &dx, &dy);
}

int oracle_forest_npatch(const oracle_forest* f) { return f->np; }

void oracle_forest_patch_info(const oracle_forest* f, int* level, int* px,
                              int* py) {
  int k;
  for (k = 0; k < f->np; ++k) { level[k] = f->lev[k]; px[k] = f->px[k]; py[k] = f->py[k]; }
}

int oracle_forest_write(oracle_forest* f, const double* h, const double* hu,
                        const double* hv) {
  int p, i, j, M = f->M;
  size_t TT = (size_t)f->T * f->T;
  for (p = 0; p < f->np; ++p)
    for (j = 0; j < M; ++j)
      for (i = 0; i < M; ++i) {
        size_t s = (size_t)p * M * M + (size_t)j * M + i;
        f->tile[p][TI(f, i, j)] = h[s];
        f->tile[p][TT + TI(f, i, j)] = hu[s];
        f->tile[p][2 * TT + TI(f, i, j)] = hv[s];
      }
  oracle_forest_ghost_fill(f);
  return 0;
}

void oracle_forest_read(const oracle_forest* f, double* h, double* hu,
                        double* hv, double* b) {
  int p, i, j, M = f->M;
  size_t TT = (size_t)f->T * f->T;
  for (p = 0; p < f->np; ++p)
    for (j = 0; j < M; ++j)
      for (i = 0; i < M; ++i) {
        size_t s = (size_t)p * M * M + (size_t)j * M + i;
        if (h) h[s] = f->tile[p][TI(f, i, j)];
        if (hu) hu[s] = f->tile[p][TT + TI(f, i, j)];
        if (hv) hv[s] = f->tile[p][2 * TT + TI(f, i, j)];
        if (b) b[s] = f->tile[p][3 * TT + TI(f, i, j)];
      }
}

void oracle_forest_read_tiles(const oracle_forest* f, double* out) {
  size_t TT = (size_t)f->T * f->T;
  int p;
  for (p = 0; p < f->np; ++p) memcpy(out + (size_t)p * 4 * TT, f->tile[p], sizeof(double) * 4 * TT);
}

void oracle_forest_set_time(oracle_forest* f, double t, double dt_next) {
  f->t = t;
  f->dt_next = dt_next;
}

void oracle_forest_get_time(const oracle_forest* f, double* t, double* dt_next,
                            long* steps, long* rejects, long* nclip,
                            double* clipvol) {
  if (clipvol) *clipvol = f->clipvol;
  if (t) *t = f->t;
  if (dt_next) *dt_next = f->dt_next;
  if (steps) *steps = f->steps;
  if (rejects) *rejects = f->rejects;
  if (nclip) *nclip = f->nclip;
}

/* Gauges (Sec. 5.1 control points, Sec. 6.5 gauge stations): bilinear in the
 * finest leaf holding the point, ghosts included; arrival is the first step
 * end time with depth above 1 cm. */
static void sample_gauges(oracle_forest* f) {
  int g, l;
  size_t TT = (size_t)f->T * f->T;
  for (g = 0; g < f->ngauge; ++g) {
    double x = f->gxy[2 * g], y = f->gxy[2 * g + 1];
    int p = -1, L = 0;
    for (l = f->c.maxlevel; l >= 0 && p < 0; --l) {
      double pw = (f->c.xupper - f->c.xlower) / (double)(f->c.mi << l);
      double ph = (f->c.yupper - f->c.ylower) / (double)(f->c.mj << l);
      long P = (long)floor((x - f->c.xlower) / pw);
      long Q = (long)floor((y - f->c.ylower) / ph);
      if (P < 0) P = 0;
      if (Q < 0) Q = 0;
      if (P >= f->lutw[l]) P = f->lutw[l] - 1;
      if (Q >= f->luth[l]) Q = f->luth[l] - 1;
      int k = f->lut[l][P + Q * f->lutw[l]];
      if (k >= 0) { p = k; L = l; }
    }
    double* o = f->gout + 5 * g;
    o[0] = f->t;
    if (p < 0) { o[1] = o[2] = o[3] = o[4] = 0.0; continue; }
    double dx = DXL(f, L), dy = DYL(f, L);
    double fx = (x - f->c.xlower) / dx - 0.5 - (double)((long)f->px[p] * f->M);
    double fy = (y - f->c.ylower) / dy - 0.5 - (double)((long)f->py[p] * f->M);
    int i0 = (int)floor(fx), j0 = (int)floor(fy);
    if (i0 < -1) i0 = -1;
    if (j0 < -1) j0 = -1;
    if (i0 > f->M - 1) i0 = f->M - 1;
    if (j0 > f->M - 1) j0 = f->M - 1;
    double ax = fx - (double)i0, ay = fy - (double)j0;
    const double* q = f->tile[p];
    double v[4];
    int k;
    for (k = 0; k < 4; ++k) {
      double a00, a10, a01, a11;
      if (k < 3) {
        a00 = q[k * TT + TI(f, i0, j0)];
        a10 = q[k * TT + TI(f, i0 + 1, j0)];
        a01 = q[k * TT + TI(f, i0, j0 + 1)];
        a11 = q[k * TT + TI(f, i0 + 1, j0 + 1)];
      } else {
        a00 = q[TI(f, i0, j0)] + q[3 * TT + TI(f, i0, j0)];
        a10 = q[TI(f, i0 + 1, j0)] + q[3 * TT + TI(f, i0 + 1, j0)];
        a01 = q[TI(f, i0, j0 + 1)] + q[3 * TT + TI(f, i0, j0 + 1)];
        a11 = q[TI(f, i0 + 1, j0 + 1)] + q[3 * TT + TI(f, i0 + 1, j0 + 1)];
      }
      v[k] = (1.0 - ay) * ((1.0 - ax) * a00 + ax * a10) +
             ay * ((1.0 - ax) * a01 + ax * a11);
    }
    o[1] = v[0]; o[2] = v[1]; o[3] = v[2]; o[4] = v[3];
    if (f->garr[g] < 0.0 && v[0] > 0.01) f->garr[g] = f->t;
  }
}

/* Adaptive time stepping with a global dt over all levels (Sec. 5.1: maximum
 * CFL 0.9; Sec. 6.6: initial dt, CFL 0.75): a step whose CFL number exceeds
 * cfl_max is rejected and retaken; the next dt is cfl_desired / cmax. */
/* Level subcycling (Berger-Oliger local time stepping over the quadtree):
 * one macro step of DT advances level L by n_L = 2^(L - minlevel) steps of
 * DT / n_L.  It runs as K = 2^(maxlevel - minlevel) fine substeps of
 * DT / K; level L steps at the substeps k with k mod 2^(maxlevel - L) = 0,
 * from the states of all levels at time t + k DT / K: its own, those of the
 * levels that step with it, and for coarser levels between two of their
 * steps the linear interpolation in time of their states before and after
 * that step (used by the ghost cells).  Every level steps at k = 0: the
 * macro step is retaken with a smaller DT if a level's Courant number
 * DT / n_L * cmax exceeds cfl_max there; later substeps are not retaken,
 * their rates cmax / n_L bound the next DT = cfl_desired / max(cmax / n_L).
 * Ghost cells at level changes are not corrected for the flux mismatch. */
static int forest_macro_steps(oracle_forest* f, double t_target, int max_steps,
                              int* steps_out) {
  int taken = 0, p, inrow = 0, rc = 0;
  size_t TT = (size_t)f->T * f->T;
  int np = f->np;
  long K = 1L << (f->c.maxlevel - f->c.minlevel), k;
  double** nt = (double**)malloc(sizeof(double*) * np);
  double** pv = (double**)malloc(sizeof(double*) * np);
  long* ncl = (long*)malloc(sizeof(long) * np);
  double* cdp = (double*)malloc(sizeof(double) * np);
  for (p = 0; p < np; ++p) {
    nt[p] = (double*)malloc(sizeof(double) * 4 * TT);
    pv[p] = (double*)malloc(sizeof(double) * 4 * TT);
  }
  while (taken < max_steps && f->t < t_target) {
    double rem = t_target - f->t, DT;
    int last;
    if (f->dt_next < rem) { DT = f->dt_next; last = 0; }
    else { DT = rem; last = 1; }
    double dtf = DT / (double)K, rmax = 0.0;
    int rejected = 0;
    for (k = 0; k < K && !rejected; ++k) {
      if (k > 0) {
        /* ghost cells at t + k dtf, coarser levels interpolated in time */
        f->prev = pv;
        f->sub_k = k;
        f->tg = f->t + (double)k * dtf;
        oracle_forest_ghost_fill(f);
        f->prev = NULL;
      }
      double r0 = 0.0;
      for (p = 0; p < np; ++p) {
        int L = f->lev[p];
        long P = 1L << (f->c.maxlevel - L);
        if (k % P) continue;
        double cm, *q = f->tile[p];
        memcpy(nt[p] + 3 * TT, q + 3 * TT, sizeof(double) * TT);
        oracle_step_grid_ex(f->M, f->M, q, q + TT, q + 2 * TT, q + 3 * TT, DXL(f, L),
                            DYL(f, L), dtf * (double)P, f->c.g, f->c.drytol,
                            f->c.manning_n, f->c.first_order ? 1 : 2,
                            !f->c.no_transverse, f->c.dim_split, nt[p], nt[p] + TT,
                            nt[p] + 2 * TT, &cm, &ncl[p], &cdp[p]);
        double r = cm * (double)P / (double)K; /* cmax / n_L */
        if (r > r0) r0 = r;
      }
      if (k == 0 && DT * r0 > f->c.cfl_max) {
        f->dt_next = f->c.cfl_desired / r0;
        f->rejects++;
        rejected = 1;
        break;
      }
      if (r0 > rmax) rmax = r0;
      for (p = 0; p < np; ++p) {
        long P = 1L << (f->c.maxlevel - f->lev[p]);
        if (k % P) continue;
        double* tmp = pv[p];
        pv[p] = f->tile[p];
        f->tile[p] = nt[p];
        nt[p] = tmp;
        f->nclip += ncl[p];
        f->clipvol += cdp[p] * (DXL(f, f->lev[p]) * DYL(f, f->lev[p]));
      }
    }
    if (rejected) {
      if (++inrow > 50) { rc = -1; break; }
      continue;
    }
    inrow = 0;
    f->t = last ? t_target : f->t + DT;
    f->steps++;
    taken++;
    if (rmax > 0.0) {
      double dn = f->c.cfl_desired / rmax;
      f->dt_next = dn < f->c.dt_max ? dn : f->c.dt_max;
    }
    oracle_forest_ghost_fill(f);
    sample_gauges(f);
  }
  for (p = 0; p < np; ++p) { free(nt[p]); free(pv[p]); }
  free(nt); free(pv); free(ncl); free(cdp);
  if (steps_out) *steps_out = taken;
  return rc;
}

int oracle_forest_step(oracle_forest* f, double t_target, int max_steps,
                       double* t_out, int* steps_out) {
  int taken = 0, p, inrow = 0;
  if (f->c.subcycle && f->c.maxlevel > f->c.minlevel) {
    int rc = forest_macro_steps(f, t_target, max_steps, steps_out);
    if (t_out) *t_out = f->t;
    return rc;
  }
  size_t TT = (size_t)f->T * f->T;
  double** nt = (double**)malloc(sizeof(double*) * f->np);
  long* ncl = (long*)malloc(sizeof(long) * f->np);
  double* cdp = (double*)malloc(sizeof(double) * f->np);
  for (p = 0; p < f->np; ++p) nt[p] = (double*)malloc(sizeof(double) * 4 * TT);
  int rc = 0;
  while (taken < max_steps && f->t < t_target) {
    double rem = t_target - f->t, dt;
    int last;
    if (f->dt_next < rem) { dt = f->dt_next; last = 0; }
    else { dt = rem; last = 1; }
    double cmax = 0.0;
    for (p = 0; p < f->np; ++p) {
      int L = f->lev[p];
      double cm;
      double* q = f->tile[p];
      memcpy(nt[p] + 3 * TT, q + 3 * TT, sizeof(double) * TT);
      oracle_step_grid_ex(f->M, f->M, q, q + TT, q + 2 * TT, q + 3 * TT, DXL(f, L),
                          DYL(f, L), dt, f->c.g, f->c.drytol, f->c.manning_n,
                          f->c.first_order ? 1 : 2, !f->c.no_transverse,
                          f->c.dim_split, nt[p],
                          nt[p] + TT, nt[p] + 2 * TT, &cm, &ncl[p], &cdp[p]);
      if (cm > cmax) cmax = cm;
    }
    if (dt * cmax > f->c.cfl_max) {
      f->dt_next = f->c.cfl_desired / cmax;
      f->rejects++;
      if (++inrow > 50) { rc = -1; break; }
      continue;
    }
    inrow = 0;
    for (p = 0; p < f->np; ++p) {
      double* tmp = f->tile[p];
      f->tile[p] = nt[p];
      nt[p] = tmp;
      f->nclip += ncl[p];
      f->clipvol += cdp[p] * (DXL(f, f->lev[p]) * DYL(f, f->lev[p]));
    }
    f->t = last ? t_target : f->t + dt;
    f->steps++;
    taken++;
    if (cmax > 0.0) {
      double dn = f->c.cfl_desired / cmax;
      f->dt_next = dn < f->c.dt_max ? dn : f->c.dt_max;
    }
    oracle_forest_ghost_fill(f);
    sample_gauges(f);
  }
  for (p = 0; p < f->np; ++p) free(nt[p]);
  free(nt); free(ncl); free(cdp);
  if (t_out) *t_out = f->t;
  if (steps_out) *steps_out = taken;
  return rc;
}

/* What one cell asks of the tagger (Sec. 4.1): *r = 2 refine (criteria 1
 * to 3: wet and flowing fast, deep-and-moving, or a deviating surface; the
 * source region below src_level, criterion 4), 1 keep (the source region at
 * or above src_level), 0 nothing; *gl = the highest level a flow grade asks
 * for (criterion 5), -1 if none.  Then the refinement regions active at the
 * state's time (criterion 4's regions between a minimum and a maximum
 * level): a cell whose centre lies in one or more of them wants the level
 * the rest asks for (L + 1 to refine, L to keep, L - 1 otherwise, or a
 * grade's level if higher) moved into [largest minimum, largest maximum],
 * and that level becomes its request (*gl then -1). */
static void cell_flag(const oracle_forest* f, int p, int i, int j, int* r_out, int* gl_out) {
  size_t TT = (size_t)f->T * f->T, id = TI(f, i, j);
  const double* q = f->tile[p];
  double h = q[id];
  int L = f->lev[p];
  int r = 0, gl = -1, k;
  if (h > f->c.tag_depth) {
    double u = q[TT + id] / h, v = q[2 * TT + id] / h;
    double sp = sqrt(u * u + v * v);
    double eta = h + q[3 * TT + id];
    double flux = sqrt(q[TT + id] * q[TT + id] + q[2 * TT + id] * q[2 * TT + id]);
    if (sp > f->c.tag_speed || fabs(eta - f->c.eta0) > f->c.tag_deta) r = 2;
    if (flux > f->c.tag_flux) r = 2;
    for (k = 0; k < f->c.ngrades; ++k) {
      double val = f->c.grade_kind[k] == 0 ? h : sp;
      if (val > f->c.grade_value[k] && f->c.grade_level[k] > gl) gl = f->c.grade_level[k];
    }
  }
  double xc = f->c.xlower + ((double)((long)f->px[p] * f->M + i) + 0.5) * DXL(f, L);
  double yc = f->c.ylower + ((double)((long)f->py[p] * f->M + j) + 0.5) * DYL(f, L);
  if (xc >= f->c.src_box[0] && xc <= f->c.src_box[1] &&
      yc >= f->c.src_box[2] && yc <= f->c.src_box[3]) {
    if (L < f->c.src_level) r = 2;
    else if (r < 1) r = 1;
  }
  {
    int in = 0, rmin = -1, rmax = -1;
    for (k = 0; k < f->c.nregions; ++k) {
      if (!(f->t >= f->c.region_t0[k] && f->t <= f->c.region_t1[k])) continue;
      if (!(xc >= f->c.region_x0[k] && xc <= f->c.region_x1[k] &&
            yc >= f->c.region_y0[k] && yc <= f->c.region_y1[k]))
        continue;
      in = 1;
      if (f->c.region_minlevel[k] > rmin) rmin = f->c.region_minlevel[k];
      if (f->c.region_maxlevel[k] > rmax) rmax = f->c.region_maxlevel[k];
    }
    if (in) {
      int want = r == 2 ? L + 1 : (r == 1 ? L : L - 1);
      if (gl > want) want = gl;
      if (want < rmin) want = rmin;
      if (want > rmax) want = rmax;
      r = want > L ? 2 : (want == L ? 1 : 0);
      gl = -1;
    }
  }
  *r_out = r;
  *gl_out = gl;
}

/* Patch flag: refine when a cell asks for it (below maxlevel) or a flow
 * grade asks for a finer level; keep at the grade's level, or when a cell
 * asks to be kept; otherwise coarsen (above minlevel). */
void oracle_forest_tags(const oracle_forest* f, uint8_t* flags) {
  int p, i, j;
  for (p = 0; p < f->np; ++p) {
    int m = 0, g = -1;
    for (j = 0; j < f->M; ++j)
      for (i = 0; i < f->M; ++i) {
        int c, gl;
        cell_flag(f, p, i, j, &c, &gl);
        if (c > m) m = c;
        if (gl > g) g = gl;
      }
    int L = f->lev[p];
    if (m == 2) flags[p] = L < f->c.maxlevel ? ORACLE_TAG_REFINE : ORACLE_TAG_KEEP;
    else if (g > L) flags[p] = ORACLE_TAG_REFINE;
    else if (g == L || m == 1) flags[p] = ORACLE_TAG_KEEP;
    else flags[p] = L > f->c.minlevel ? ORACLE_TAG_COARSEN : ORACLE_TAG_KEEP;
  }
}

/* level map on the finest patch grid */
typedef struct {
  int W, H, maxl;
  int* m;
} lvlmap;

static void lm_paint(lvlmap* lm, int L, int px, int py) {
  int s = lm->maxl - L, a, b;
  for (b = py << s; b < (py + 1) << s; ++b)
    for (a = px << s; a < (px + 1) << s; ++a) lm->m[a + b * lm->W] = L;
}

/* Largest level among the finest-grid blocks that touch the region of patch
 * (L, px, py) from outside (faces and corners). */
static int lm_ring_max(const lvlmap* lm, int L, int px, int py) {
  int s = lm->maxl - L;
  int x0 = (px << s) - 1, x1 = (px + 1) << s, y0 = (py << s) - 1, y1 = (py + 1) << s;
  int best = -1, a, b;
  for (b = y0; b <= y1; ++b)
    for (a = x0; a <= x1; ++a) {
      if (a > x0 && a < x1 && b > y0 && b < y1) continue;
      if (a < 0 || b < 0 || a >= lm->W || b >= lm->H) continue;
      int v = lm->m[a + b * lm->W];
      if (v > best) best = v;
    }
  return best;
}

/* Regrid, Sec. 4 and Sec. 6.6: refine tagged patches one level, enforce the
 * 2:1 balance across faces and corners (no level skipping), coarsen sibling
 * quartets that all ask for it when the balance allows, then move the data
 * with the ghost-cell operators (copy, average, interpolate). */
int oracle_forest_regrid_flags(oracle_forest* f, const uint8_t* given) {
  int n0 = f->np, k, c;
  uint8_t* flags = (uint8_t*)malloc(n0 ? n0 : 1);
  if (n0) memcpy(flags, given, (size_t)n0);
  int cap = 4 * n0 + 16;
  int* lev = (int*)malloc(sizeof(int) * cap);
  int* px = (int*)malloc(sizeof(int) * cap);
  int* py = (int*)malloc(sizeof(int) * cap);
  int* orig = (int*)malloc(sizeof(int) * cap); /* original index or -1 */
  int n = 0;
  for (k = 0; k < n0; ++k) {
    if (flags[k] == ORACLE_TAG_REFINE) {
      for (c = 0; c < 4; ++c) {
        lev[n] = f->lev[k] + 1;
        px[n] = 2 * f->px[k] + (c & 1);
        py[n] = 2 * f->py[k] + (c >> 1);
        orig[n] = -1;
        ++n;
      }
    } else {
      lev[n] = f->lev[k]; px[n] = f->px[k]; py[n] = f->py[k]; orig[n] = k; ++n;
    }
  }
  lvlmap lm;
  lm.maxl = f->c.maxlevel;
  lm.W = f->c.mi << lm.maxl;
  lm.H = f->c.mj << lm.maxl;
  lm.m = (int*)malloc(sizeof(int) * (size_t)lm.W * lm.H);
  for (k = 0; k < n; ++k) lm_paint(&lm, lev[k], px[k], py[k]);
  int changed = 1;
  while (changed) {
    changed = 0;
    for (k = 0; k < n; ++k) {
      if (lm_ring_max(&lm, lev[k], px[k], py[k]) > lev[k] + 1) {
        if (n + 3 >= cap) {
          cap *= 2;
          lev = (int*)realloc(lev, sizeof(int) * cap);
          px = (int*)realloc(px, sizeof(int) * cap);
          py = (int*)realloc(py, sizeof(int) * cap);
          orig = (int*)realloc(orig, sizeof(int) * cap);
        }
        int L = lev[k] + 1, X = 2 * px[k], Y = 2 * py[k];
        lev[k] = L; px[k] = X; py[k] = Y; orig[k] = -1;
        for (c = 1; c < 4; ++c) {
          lev[n] = L; px[n] = X + (c & 1); py[n] = Y + (c >> 1); orig[n] = -1; ++n;
        }
        for (c = 0; c < 4; ++c) lm_paint(&lm, L, X + (c & 1), Y + (c >> 1));
        changed = 1;
      }
    }
  }
  /* coarsening of complete sibling quartets that are still original leaves */
  int* keep = (int*)malloc(sizeof(int) * n);
  for (k = 0; k < n; ++k) keep[k] = 1;
  int* pos = (int*)malloc(sizeof(int) * (n0 ? n0 : 1));
  for (k = 0; k < n0; ++k) pos[k] = -1;
  for (k = 0; k < n; ++k) if (orig[k] >= 0) pos[orig[k]] = k;
  int nadd = 0;
  int* addL = (int*)malloc(sizeof(int) * (n / 4 + 1));
  int* addX = (int*)malloc(sizeof(int) * (n / 4 + 1));
  int* addY = (int*)malloc(sizeof(int) * (n / 4 + 1));
  for (k = 0; k < n0; ++k) {
    int L = f->lev[k];
    if (L <= f->c.minlevel || (f->px[k] & 1) || (f->py[k] & 1)) continue;
    int sib[4], ok = 1;
    for (c = 0; c < 4 && ok; ++c) {
      int s = leaf_at(f, L, (long)(f->px[k] + (c & 1)) * f->M,
                      (long)(f->py[k] + (c >> 1)) * f->M);
      if (s < 0 || flags[s] != ORACLE_TAG_COARSEN || pos[s] < 0) ok = 0;
      else sib[c] = s;
    }
    if (!ok) continue;
    if (lm_ring_max(&lm, L - 1, f->px[k] / 2, f->py[k] / 2) > L) continue;
    for (c = 0; c < 4; ++c) keep[pos[sib[c]]] = 0;
    addL[nadd] = L - 1; addX[nadd] = f->px[k] / 2; addY[nadd] = f->py[k] / 2; ++nadd;
  }
  int nn = 0;
  int* NL = (int*)malloc(sizeof(int) * (n + nadd));
  int* NX_ = (int*)malloc(sizeof(int) * (n + nadd));
  int* NY_ = (int*)malloc(sizeof(int) * (n + nadd));
  for (k = 0; k < n; ++k)
    if (keep[k]) { NL[nn] = lev[k]; NX_[nn] = px[k]; NY_[nn] = py[k]; ++nn; }
  for (k = 0; k < nadd; ++k) { NL[nn] = addL[k]; NX_[nn] = addX[k]; NY_[nn] = addY[k]; ++nn; }

  /* new forest; the old one is the data source for every new cell */
  oracle_forest* old = (oracle_forest*)malloc(sizeof(oracle_forest));
  *old = *f;
  memset(f->lut, 0, sizeof(f->lut));
  set_leaves(f, nn, NL, NX_, NY_);
  size_t TT = (size_t)f->T * f->T;
  int p, i, j, q;
  for (p = 0; p < f->np; ++p) {
    fill_topo(f, p);
    int L = f->lev[p];
    for (j = 0; j < f->M; ++j)
      for (i = 0; i < f->M; ++i) {
        double out[3];
        long I = (long)f->px[p] * f->M + i, J = (long)f->py[p] * f->M + j;
        double bs[2][2];
        child_beds(f, f->tile[p] + 3 * TT, i, j, bs);
        fill_cell(old, L, I, J, bs, out);
        for (q = 0; q < 3; ++q) f->tile[p][q * TT + TI(f, i, j)] = out[q];
      }
  }
  for (k = 0; k < old->np; ++k) free(old->tile[k]);
  free(old->tile); free(old->lev); free(old->px); free(old->py);
  for (k = 0; k < MAXLEV; ++k) free(old->lut[k]);
  free(old);
  oracle_forest_ghost_fill(f);
  free(flags); free(lev); free(px); free(py); free(orig); free(lm.m);
  free(keep); free(pos); free(addL); free(addX); free(addY);
  free(NL); free(NX_); free(NY_);
  return f->np;
}

int oracle_forest_regrid(oracle_forest* f) {
  uint8_t* flags = (uint8_t*)malloc(f->np ? f->np : 1);
  oracle_forest_tags(f, flags);
  int n = oracle_forest_regrid_flags(f, flags);
  free(flags);
  return n;
}

/* Volume sum_cells h dx dy with Kahan compensation. */
double oracle_forest_mass(const oracle_forest* f) {
  double s = 0.0, comp = 0.0;
  int p, i, j;
  for (p = 0; p < f->np; ++p) {
    double a = DXL(f, f->lev[p]) * DYL(f, f->lev[p]);
    for (j = 0; j < f->M; ++j)
      for (i = 0; i < f->M; ++i) {
        double y = f->tile[p][TI(f, i, j)] * a - comp;
        double t = s + y;
        comp = (t - s) - y;
        s = t;
      }
  }
  return s;
}

int oracle_forest_set_gauges(oracle_forest* f, const double* xy, int n) {
  int g;
  free(f->gxy); free(f->gout); free(f->garr);
  f->ngauge = n;
  f->gxy = (double*)malloc(sizeof(double) * 2 * (n ? n : 1));
  f->gout = (double*)calloc(5 * (n ? n : 1), sizeof(double));
  f->garr = (double*)malloc(sizeof(double) * (n ? n : 1));
  for (g = 0; g < n; ++g) {
    f->gxy[2 * g] = xy[2 * g];
    f->gxy[2 * g + 1] = xy[2 * g + 1];
    f->garr[g] = -1.0;
  }
  sample_gauges(f);
  return 0;
}

void oracle_forest_gauges(const oracle_forest* f, double* out,
                          double* arrival) {
  int g;
  for (g = 0; g < f->ngauge; ++g) {
    if (out) memcpy(out + 5 * g, f->gout + 5 * g, sizeof(double) * 5);
    if (arrival) arrival[g] = f->garr[g];
  }
}
