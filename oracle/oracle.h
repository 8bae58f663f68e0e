/*
 * GeoFlood FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded double-precision restatement of the
 * per-patch wave-propagation step of GeoFlood (Kyanjo, Calhoun & George,
 * "GeoFlood (v1.0.0): Computational model for overland flooding",
 * arXiv 2403.15435).  It exists to check the CUDA library against the
 * method.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * and reference legs may load it; the product path never links, imports or
 * calls anything here, and nothing here includes a product header.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fused multiply-add, IEEE
 * sqrt and division), so every operation rounds exactly as written.
 */
#ifndef GEOFLOOD_ORACLE_H
#define GEOFLOOD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_MAXDEM 4 /* DEMs per forest */
#define ORACLE_MAXREGION 8 /* refinement regions per forest */
#define ORACLE_BC_WALL 0
#define ORACLE_BC_EXTRAP 1

/* Patch flags produced by the tagger (Sec. 4.1 criteria 1 to 5). */
#define ORACLE_TAG_KEEP 0
#define ORACLE_TAG_REFINE 1
#define ORACLE_TAG_COARSEN 2

typedef struct {
  int mi, mj;        /* blocks (trees) of the level-0 arrangement, Sec. 4 */
  int mx;            /* patch cells per side (square patches mx x mx) */
  int minlevel, maxlevel;
  int bc[4];         /* left, right, bottom, top: ORACLE_BC_* */
  double xlower, xupper, ylower, yupper;
  double g, drytol, manning_n;
  double cfl_desired, cfl_max, dt_initial, dt_max;
  double tag_depth, tag_speed, tag_deta, eta0;
  double src_box[4]; /* x0, x1, y0, y1 of the flood-source region */
  int src_level;     /* refine the source region up to this level */
  /* criterion 2: refine where h > tag_depth and |hu| > tag_flux */
  double tag_flux;
  /* criterion 5: flow grades -- a wet cell whose depth (kind 0) or speed
   * (kind 1) exceeds grade_value asks for at least grade_level */
  int ngrades;
  int grade_kind[4];
  double grade_value[4];
  int grade_level[4];
  /* scheme variants of Sec. 3.2 (all 0: second order, unsplit, with
   * transverse propagation): first_order drops the limited corrections,
   * no_transverse the transverse terms, dim_split replaces the unsplit
   * update by an x sweep followed by a y sweep on its result */
  int first_order, no_transverse, dim_split;
  /* inflow hydrograph (Sec. 5.1 set-up, Eq. riemann, Eq. 2-shock): with
   * n_hydro > 0, the ghost cells of side inflow_side (0 left, 1 right,
   * 2 bottom, 3 top) whose centre lies in [inflow_lo, inflow_hi] (the
   * side's coordinate) carry Q(t) divided by the width of those lines at
   * their level into the domain while Q(t) > 0; Q is piecewise linear
   * through (hydro_t[k], hydro_q[k]), k < n_hydro <= 16, and constant
   * beyond the first and last points; inflow_tau is the minimum interior
   * depth of Sec. 5.1 */
  /* level subcycling (0: one time step for all levels; 1: level L takes
   * 2^(L - minlevel) steps per macro step, ghost cells of coarser levels
   * interpolated in time) */
  int subcycle;
  int n_hydro, inflow_side;
  double inflow_lo, inflow_hi, inflow_tau;
  double hydro_t[16], hydro_q[16];
  /* refinement regions (Sec. 4.1 criterion 4: regions refined to a desired
   * resolution between user-given minimum and maximum levels; Sec. 6.4:
   * places and times of interest): while region_t0[k] <= t <= region_t1[k]
   * (t the time of the state), a cell whose centre lies in
   * [region_x0[k], region_x1[k]] x [region_y0[k], region_y1[k]] asks for a
   * level of at least region_minlevel[k] and at most region_maxlevel[k];
   * where several active regions hold the centre, the largest minimum and
   * the largest maximum apply.  nregions <= ORACLE_MAXREGION. */
  int nregions;
  int region_minlevel[8], region_maxlevel[8];
  double region_x0[8], region_x1[8], region_y0[8], region_y1[8];
  double region_t0[8], region_t1[8];
} oracle_config;

typedef struct oracle_forest oracle_forest;

/* Discharge Q(t) of the inflow hydrograph (m^3/s). */
double oracle_hydrograph(const oracle_config* cfg, double t);

/* Ghost depth for the inflow boundary (Sec. 5.1): q > 0 the unit discharge
 * into the domain, h_int and qn_int the depth and the momentum (into the
 * domain) of the interior cell next to the ghost cell.  Solves Eq. riemann,
 * and Eq. 2-shock if that depth exceeds the interior depth, by Newton's
 * method.  *h_used and *u_used (may be NULL) receive the interior depth and
 * speed the equations used (after the minimum-depth rule). */
double oracle_inflow_depth(double q, double h_int, double qn_int, double g,
                           double tau, double* h_used, double* u_used);

/* One augmented Riemann solve at an edge in the normal frame (Sec. 3.3).
 * Inputs per side: depth h, normal momentum n, transverse momentum t, bed b.
 * Outputs: Z[3][3] f-waves (wave p, component k = mass, normal momentum,
 * transverse momentum) and s[3] wave speeds. */
void oracle_riemann(double hL, double nL, double tL, double bL, double hR,
                    double nR, double tR, double bR, double g, double drytol,
                    double* Z, double* s);

/* One unsplit second-order step on a single grid of nx*ny interior cells
 * with 2 filled ghost layers; arrays are [ny+4][nx+4] row-major.  Writes the
 * interior of hn/hun/hvn (ghost entries are copied from the input), returns
 * in *cmax the largest |s|/dx or |s|/dy over the edges that update interior
 * cells, in *nclip the number of negative depths reset to zero and in
 * *clipdepth the sum of the depths so added. */
/* The same step with the scheme's options (see oracle_config). */
void oracle_step_grid_ex(int nx, int ny, const double* h, const double* hu,
                         const double* hv, const double* b, double dx, double dy,
                         double dt, double g, double drytol, double manning_n,
                         int order, int transverse, int dim_split, double* hn,
                         double* hun, double* hvn, double* cmax, long* nclip,
                         double* clipdepth);
void oracle_step_grid(int nx, int ny, const double* h, const double* hu,
                      const double* hv, const double* b, double dx, double dy,
                      double dt, double g, double drytol, double manning_n,
                      double* hn, double* hun, double* hvn, double* cmax,
                      long* nclip, double* clipdepth);

/* Cell average of the bilinear interpolant of a DEM over a rectangle. */
double oracle_dem_average(const double* z, int nx, int ny, double x0,
                          double y0, double dx, double dy, double xa,
                          double xb, double ya, double yb);

/* Cell average of the composite interpolant of n <= ORACLE_MAXDEM
 * overlapping DEMs (Sec. 6.2): at each point the bilinear interpolant of the
 * finest DEM (smallest dx * dy; equal spacings in the given order) whose
 * node-to-node extent holds it; outside every extent the coarsest one's,
 * constant beyond its edges. */
double oracle_dems_average(int n, const double* const* z, const int* nx,
                           const int* ny, const double* x0, const double* y0,
                           const double* dx, const double* dy, double xa,
                           double xb, double ya, double yb);

oracle_forest* oracle_forest_new(const oracle_config* cfg);
void oracle_forest_free(oracle_forest* f);
int oracle_forest_set_topo(oracle_forest* f, const double* z, int nx, int ny,
                           double x0, double y0, double dx, double dy);
/* Several DEMs (arrays per DEM), composed as in oracle_dems_average. */
int oracle_forest_set_topos(oracle_forest* f, int n, const double* const* z,
                            const int* nx, const int* ny, const double* x0,
                            const double* y0, const double* dx,
                            const double* dy);
int oracle_forest_npatch(const oracle_forest* f);
void oracle_forest_patch_info(const oracle_forest* f, int* level, int* px,
                              int* py);
/* Interior arrays [npatch][mx][mx] (row index j, column index i). */
int oracle_forest_write(oracle_forest* f, const double* h, const double* hu,
                        const double* hv);
void oracle_forest_read(const oracle_forest* f, double* h, double* hu,
                        double* hv, double* b);
/* Whole tiles [npatch][4][mx+4][mx+4] (h, hu, hv, b), ghosts included. */
void oracle_forest_read_tiles(const oracle_forest* f, double* out);
void oracle_forest_set_time(oracle_forest* f, double t, double dt_next);
void oracle_forest_get_time(const oracle_forest* f, double* t,
                            double* dt_next, long* steps, long* rejects,
                            long* nclip, double* clipvol);
int oracle_forest_step(oracle_forest* f, double t_target, int max_steps,
                       double* t_out, int* steps_out);
void oracle_forest_tags(const oracle_forest* f, uint8_t* flags);
int oracle_forest_regrid(oracle_forest* f);
/* The same regrid from given per-leaf flags (ORACLE_TAG_*, one per current
 * leaf, in patch order) instead of the tagger's. */
int oracle_forest_regrid_flags(oracle_forest* f, const uint8_t* flags);
double oracle_forest_mass(const oracle_forest* f);
int oracle_forest_set_gauges(oracle_forest* f, const double* xy, int n);
void oracle_forest_gauges(const oracle_forest* f, double* out,
                          double* arrival);
void oracle_forest_ghost_fill(oracle_forest* f);

#ifdef __cplusplus
}
#endif
#endif
