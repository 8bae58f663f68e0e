/*
 * geoflood.h -- C ABI of the GB300 (sm_103a) GeoFlood wave-propagation
 * library.
 *
 * The library advances the 2D shallow-water equations with bathymetry and
 * Manning friction (Sec. 3.1, Eq. shallow, Eq. manning of Kyanjo, Calhoun &
 * George, "GeoFlood (v1.0.0): Computational model for overland flooding",
 * arXiv 2403.15435) by the second-order wave-propagation method with the
 * augmented Riemann solver (Sec. 3.2 Eqs. wpa_update and
 * wpa_update_corrections, Sec. 3.3) on a quadtree of fixed-size patches
 * (Sec. 4), for one or many independent scenarios at once.
 *
 * Conventions for every call:
 *   - the return value is GEOFLOOD_OK (0) or a negative GEOFLOOD_ERR_* code;
 *     geoflood_last_error() then holds a message owned by the context;
 *   - no C++ exception crosses the ABI;
 *   - host pointers are owned by the caller and only read or written during
 *     the call; device state is owned by the context and freed by
 *     geoflood_destroy();
 *   - calls on one context are not thread safe; all device work is issued on
 *     the stream given to geoflood_init_forest() (NULL = a blocking stream
 *     the context creates for itself, since CUDA graphs cannot be captured
 *     on the legacy default stream); calls that return host data
 *     synchronise that stream;
 *   - arrays of patch data are [npatch][mx][mx] row-major (row index j along
 *     y, column index i along x) in the scenario's patch order, which is the
 *     Morton order of the patches on the finest patch grid;
 *   - all floating-point arguments are double.
 */
#ifndef GEOFLOOD_H
#define GEOFLOOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GEOFLOOD_OK 0
#define GEOFLOOD_ERR_ARG -1            /* invalid argument */
#define GEOFLOOD_ERR_CUDA -2           /* a CUDA call failed */
#define GEOFLOOD_ERR_OOM -3            /* device allocation failed */
#define GEOFLOOD_ERR_CFL -4            /* more than 50 rejected steps in a row */
#define GEOFLOOD_ERR_NAN -5            /* a non-finite value appeared */
#define GEOFLOOD_ERR_NEGATIVE_DEPTH -6 /* reserved: negative depths are reset */
#define GEOFLOOD_ERR_TIMEOUT -7        /* a bounded device wait expired */
#define GEOFLOOD_ERR_CAPACITY -8       /* patch table or buffer capacity */
#define GEOFLOOD_ERR_STATE -9          /* call out of order (e.g. no state) */

#define GEOFLOOD_BC_WALL 0   /* reflecting wall (Sec. 5.1 closed boundaries) */
#define GEOFLOOD_BC_EXTRAP 1 /* zero-order extrapolation (open boundary) */

#define GEOFLOOD_FP64 0 /* plain double precision */
/* FP32 surface-deviation form: state w = h + b - eta0, hu, hv in FP32 with
 * FP32 compensation terms for the update; wet/dry tests exact (FP64 where
 * FP32 cannot decide); volumes and time stepping in FP64. */
#define GEOFLOOD_FP32_DEV 1

#define GEOFLOOD_TAG_KEEP 0
#define GEOFLOOD_TAG_REFINE 1
#define GEOFLOOD_TAG_COARSEN 2

/* taggers (geoflood_set_tagger) */
#define GEOFLOOD_TAGGER_PLAIN 0
#define GEOFLOOD_TAGGER_LEARNED 1

/* Forest, physics and control parameters.  Geometry (Sec. 4): mi x mj
 * level-0 blocks, each a patch of mx x mx cells (mx = 16 or 32), levels
 * minlevel..maxlevel with refinement ratio 2; the domain is
 * [xlower, xupper] x [ylower, yupper].  g and drytol (Sec. 5.1 wet/dry
 * threshold tau); CFL control (Sec. 5.1 maximum CFL, Sec. 6.6 initial time
 * step): the next dt is cfl_desired / cmax, a step whose CFL number exceeds
 * cfl_max is retaken.  Tagging (Sec. 4.1): a wet cell (h > tag_depth) asks
 * for refinement when its speed exceeds tag_speed or its surface deviates
 * from eta0 by more than tag_deta (criteria 1, 3) or |hu| exceeds tag_flux
 * (criterion 2); the flood-source box [x0, x1, y0, y1] is refined to
 * src_level (criterion 4, Sec. 6.4); a wet cell whose depth (grade kind 0)
 * or speed (kind 1) exceeds grade_value[k] asks for at least level
 * grade_level[k] (criterion 5, flow grades).  max_patches bounds the
 * patches of all scenarios together. */
typedef struct {
  int mi, mj, mx;
  int minlevel, maxlevel;
  int bc[4]; /* left, right, bottom, top */
  int precision;
  int num_scenarios;
  int max_patches;
  int max_gauges;
  double xlower, xupper, ylower, yupper;
  double g, drytol;
  double cfl_desired, cfl_max, dt_initial, dt_max;
  double tag_depth, tag_speed, tag_deta;
  double src_box[4];
  int src_level;
  int ngrades;         /* flow grades in use (0..4) */
  double tag_flux;     /* criterion 2 threshold on |hu| (m^2/s); inf: off */
  int grade_kind[4];   /* criterion 5: 0 = depth, 1 = speed */
  double grade_value[4];
  int grade_level[4];
  /* scheme variants of Sec. 3.2, each 0 or 1 (all 0: second order, unsplit,
   * with transverse propagation): first_order drops the limited
   * corrections; no_transverse drops the transverse terms of the unsplit
   * update; dim_split replaces the unsplit update by an x sweep over every
   * row of a patch (ghost rows included), then a y sweep on its result
   * (negative depths reset and dry momenta zeroed in between), without
   * transverse terms.  Without transverse terms the unsplit update is
   * stable only up to a Courant number of 1/2 (set cfl_desired and cfl_max
   * accordingly); the split update is stable up to 1.  With dim_split the
   * patch step has a single kernel variant. */
  int first_order, no_transverse, dim_split;
  /* Inflow hydrograph (Sec. 5.1, Test Case 1 set-up; Eq. riemann, Eq.
   * 2-shock).  n_hydro = 0: none.  Otherwise the discharge Q(t) (m^3/s) is
   * piecewise linear through (hydro_t[k], hydro_q[k]), k < n_hydro <= 16,
   * hydro_t strictly increasing, hydro_q >= 0, constant before the first
   * and after the last point; it enters through the segment
   * [inflow_lo, inflow_hi] of side inflow_side (GEOFLOOD_BC order: 0 left,
   * 1 right, 2 bottom, 3 top; the coordinate along that side).  While
   * Q(t) > 0, each ghost line of a tile whose centre lies in the segment
   * carries, in both ghost layers, the unit discharge Q(t) / W normal to
   * the side into the domain (W: the number of such lines at the tile's
   * level times their cell size, so that Q(t) enters at every resolution;
   * none where no line centre of that level lies in the segment), no
   * tangential momentum,
   * and the depth that joins it to the tile's first cell of the line by a
   * single entering wave: Eq. riemann, or Eq. 2-shock where that depth
   * exceeds the interior's, solved by Newton's method (first guesses
   * [F Q'/sqrt(g)]^(2/3), F = 0.5 and 1) safeguarded by bisection.  An
   * interior cell thinner than inflow_tau (> 0) is replaced by the inflow's
   * critical depth (at least inflow_tau) at rest.  With Q(t) = 0 the side's
   * own rule applies.  The ghost values use the time of the state. */
  int n_hydro, inflow_side;
  double inflow_lo, inflow_hi, inflow_tau;
  double hydro_t[16], hydro_q[16];
  /* Level subcycling (0 or 1; no effect when maxlevel = minlevel): one
   * step of geoflood_step becomes a macro step of DT in which level L takes
   * 2^(L - minlevel) steps of DT / 2^(L - minlevel), run as 2^(maxlevel -
   * minlevel) fine substeps; at each, the levels due step together, and
   * ghost cells next to a coarser level between two of its steps take that
   * level's state interpolated linearly in time.  Every level steps at the
   * first substep, whose Courant numbers are checked (a violation retakes
   * the macro step with a smaller DT); later substeps are not checked, their
   * rates bound the next DT = cfl_desired / max_L(cmax_L / n_L).  Steps and
   * max_steps count macro steps; the patch step has a single variant. */
  int subcycle;
  /* Refinement regions (Sec. 4.1 criterion 4: regions refined to a desired
   * resolution between user-given minimum and maximum levels; Sec. 6.4:
   * places and times of interest).  nregions = 0..8.  While
   * region_t0[k] <= t <= region_t1[k] (t the time of the scenario's state),
   * a cell whose centre lies in [region_x0[k], region_x1[k]] x
   * [region_y0[k], region_y1[k]] asks for a level of at least
   * region_minlevel[k] and at most region_maxlevel[k] (minlevel <= these <=
   * maxlevel): the level the other criteria ask for (L + 1 to refine, L to
   * keep, L - 1 otherwise, or a flow grade's level if higher) is moved into
   * [the largest minimum, the largest maximum] of the active regions that
   * hold the centre, dry cells included.  The learned tagger's requests are
   * bounded the same way.  The 2:1 balance of a regrid may still refine
   * past a region's maximum next to finer patches. */
  int nregions;
  int region_minlevel[8], region_maxlevel[8];
  double region_x0[8], region_x1[8], region_y0[8], region_y1[8];
  double region_t0[8], region_t1[8];
} geoflood_config;

typedef struct geoflood_ctx geoflood_ctx;

/* Initial-condition callback: for n cells with centres (x[k], y[k]) and
 * cell-averaged bed b[k], write the depth h[k] and momenta hu[k], hv[k]. */
typedef void (*geoflood_qinit_fn)(int n, const double* x, const double* y,
                                  const double* b, double* h, double* hu,
                                  double* hv, void* user);

/* Create a context: validates cfg, allocates the device state for
 * max_patches patches and builds every scenario's forest uniformly at
 * minlevel with a flat bed at zero and dry cells.  When the bed tiles of
 * every patch position of every level of every scenario fit 16 GiB, it also
 * allocates a cache of them (a patch that a regrid recreates then copies
 * its bed instead of integrating the DEMs again; the cache is cleared when
 * a scenario's DEMs or eta0 change, so results are the same either way).
 * stream is a cudaStream_t (may be NULL).  On success *out receives the
 * context.  Errors: ARG, CUDA, OOM, CAPACITY. */
int geoflood_init_forest(const geoflood_config* cfg, void* stream,
                         geoflood_ctx** out);

/* Free all device and host state of the context (NULL is allowed). */
void geoflood_destroy(geoflood_ctx* ctx);

/* Message of the last failed call (owned by the context; "" if none). */
const char* geoflood_last_error(const geoflood_ctx* ctx);

/* Per-scenario physics: Manning coefficient n (Eq. manning) and reference
 * surface eta0 used by the tagger (|eta - eta0| > tag_deta). */
int geoflood_set_scenario(geoflood_ctx* ctx, int scenario, double manning_n,
                          double eta0);

/* Topography of one scenario from one DEM (Sec. 6.2): z[ny][nx] nodal
 * elevations at (x0 + i dx, y0 + j dy), nx, ny >= 2.  Every cell's bed, ghost
 * cells included, becomes the exact cell average of the DEM's bilinear
 * interpolant (constant beyond the DEM).  The DEM is copied to the device
 * and kept for regrids.  Errors: ARG, CUDA, OOM. */
int geoflood_set_topo(geoflood_ctx* ctx, int scenario, const double* z, int nx,
                      int ny, double x0, double y0, double dx, double dy);

/* Topography of one scenario from 1..4 overlapping or nested DEMs of
 * different resolutions (Sec. 6.2, the Malpasset set-up's 2, 5 and 20 m
 * DEMs): arrays of ndem entries, DEM k being z[k][ny[k]][nx[k]] at
 * (x0[k] + i dx[k], y0[k] + j dy[k]).  At each point the bed is the bilinear
 * interpolant of the finest DEM (smallest dx * dy; equal spacings in the
 * given order) whose node-to-node extent holds the point; outside every
 * extent the coarsest one's, constant beyond its edges.  Every cell's bed is
 * the exact cell average of that composite interpolant (its pieces are cut
 * by every DEM's node lines), so a coarse cell's bed is the mean of its
 * children's and refinement keeps still water still.  The DEMs are copied to
 * the device and kept for regrids; geoflood_set_topo is the case ndem = 1.
 * In the FP32 form the depths are kept.  Errors: ARG (counts, sizes,
 * spacings), CUDA, OOM. */
int geoflood_set_topos(geoflood_ctx* ctx, int scenario, int ndem,
                       const double* const* z, const int* nx, const int* ny,
                       const double* x0, const double* y0, const double* dx,
                       const double* dy);

/* Number of patches of a scenario. */
int geoflood_npatch(geoflood_ctx* ctx, int scenario, int* npatch);

/* Level and position (px, py on that level's patch grid) of every patch of
 * the scenario, in storage order; each array holds npatch ints. */
int geoflood_patch_info(geoflood_ctx* ctx, int scenario, int* level, int* px,
                        int* py);

/* Copy host interior arrays [npatch][mx][mx] into the scenario's current
 * state and refill all ghost cells.  Errors: ARG, CUDA. */
int geoflood_write_patches(geoflood_ctx* ctx, int scenario, const double* h,
                           const double* hu, const double* hv);

/* Copy the scenario's current interior state to host arrays
 * [npatch][mx][mx]; any pointer may be NULL.  Synchronises the stream. */
int geoflood_read_patches(geoflood_ctx* ctx, int scenario, double* h,
                          double* hu, double* hv, double* b);

/* Copy whole patch tiles, ghosts included, to host: [npatch][4][mx+4][mx+4]
 * with fields h, hu, hv, b. */
int geoflood_read_tiles(geoflood_ctx* ctx, int scenario, double* out);

/* Set the initial state through a callback (evaluated on the host once for
 * all interior cells of the scenario), then fill the ghosts. */
int geoflood_set_state(geoflood_ctx* ctx, int scenario, geoflood_qinit_fn fn,
                       void* user);

/* Simulation time and the dt the next step will try. */
int geoflood_set_time(geoflood_ctx* ctx, int scenario, double t,
                      double dt_next);

/* Time, next dt, accepted steps, rejected steps, number of negative depths
 * reset to zero and the volume so added; any pointer may be NULL. */
int geoflood_get_time(geoflood_ctx* ctx, int scenario, double* t,
                      double* dt_next, long long* steps, long long* rejects,
                      long long* nclip, double* clipvol);

/* Checkpoint (no passage of the paper; the restart facility that GeoClaw
 * and ForestClaw runs rely on for long simulations): writes everything a
 * context needs to continue exactly where it stands into the caller's
 * buffer buf of cap bytes -- per scenario its Manning n and eta0, DEMs,
 * forest, time-stepping state and counters, gauges and the current state
 * (whole tiles; in the FP32 form also the compensation terms), and the
 * network's parameters, Adam state, scales and tagger.  *size receives the
 * bytes needed; with buf = NULL or cap too small nothing is written and the
 * call returns CAPACITY (call once to size the buffer).  The record is
 * plain bytes of this host's byte order.  Errors: ARG, CUDA, CAPACITY. */
int geoflood_save(geoflood_ctx* ctx, void* buf, size_t cap, size_t* size);

/* Resume from a checkpoint of geoflood_save: ctx must have been created
 * with the same configuration (compared byte for byte) and precision.
 * Replaces the context's scenarios, forests, DEMs (beds recomputed), state,
 * time-stepping state, gauges and network; stepping on continues bit for
 * bit as the saved context would have.  Errors: ARG (not a checkpoint,
 * another configuration, corrupt or truncated record), CAPACITY, OOM, CUDA;
 * after an error the context's state is unspecified. */
int geoflood_load(geoflood_ctx* ctx, const void* buf, size_t size);

/* Advance every scenario towards t_target by at most max_steps accepted
 * steps of the adaptive scheme (Sec. 3.2, 3.3, Eq. manning; CFL rule of
 * Sec. 5.1): ghost fill, unsplit second-order step with transverse
 * propagation and Manning friction, CFL check with reject/retake, gauges.
 * Each scenario keeps its own dt.  t_out[s] and steps_out[s] (arrays of
 * num_scenarios entries, may be NULL) receive the reached time and the
 * accepted steps taken by this call.  Errors: CFL (a scenario rejected 50
 * steps in a row), NAN, CUDA, STATE. */
int geoflood_step(geoflood_ctx* ctx, double t_target, int max_steps,
                  double* t_out, int* steps_out);

/* Per-patch refinement flags of the plain tagger (Sec. 4.1 criteria 1, 3,
 * 4): GEOFLOOD_TAG_* for each of the scenario's npatch patches. */
int geoflood_tags(geoflood_ctx* ctx, int scenario, uint8_t* flags);

/* Regrid every scenario (Sec. 4, Sec. 6.6): tag, refine one level, enforce
 * the 2:1 face/corner balance, coarsen complete sibling quartets, move the
 * data with the ghost-cell operators (copy, 2x2 average, limited
 * interpolation), recompute the beds and refill the ghosts.  Errors:
 * CAPACITY (more than max_patches patches), CUDA. */
int geoflood_regrid(geoflood_ctx* ctx);

/* Water volume sum h dx dy of a scenario's current state (FP64). */
int geoflood_mass(geoflood_ctx* ctx, int scenario, double* mass);

/* Register n <= max_gauges gauge points xy[n][2] of a scenario (Sec. 5.1
 * control points, Sec. 6.5 gauges); they are sampled after every accepted
 * step. */
int geoflood_set_gauges(geoflood_ctx* ctx, int scenario, const double* xy,
                        int n);

/* Number of gauges of a scenario (as set by geoflood_set_gauges or
 * restored by geoflood_load): the rows geoflood_gauges writes. */
int geoflood_gauge_count(geoflood_ctx* ctx, int scenario, int* n);

/* Latest gauge samples out[n][5] = (t, h, hu, hv, eta) and arrival times
 * arrival[n] (first sample time with h > 0.01 m, -1 if none); either
 * pointer may be NULL. */
int geoflood_gauges(geoflood_ctx* ctx, int scenario, double* out,
                    double* arrival);

/* Kernel timing with CUDA events around launches of the named kernel
 * family ("patch_step", "ghost_fill"): enable = n > 0 starts recording (and
 * clears earlier records), timing every n-th step of each captured chunk of
 * steps (n = 1: every launch; a larger n keeps the cost of the event nodes
 * off the other steps); 0 stops. */
int geoflood_profile(geoflood_ctx* ctx, int enable);

/* Sum of the recorded durations (ms) and number of recorded launches of one
 * kernel family since geoflood_profile(ctx, 1).  Synchronises. */
int geoflood_profile_read(geoflood_ctx* ctx, const char* kernel,
                          double* total_ms, long long* launches);

/* Interior cells covered by the recorded launches of one kernel family
 * since geoflood_profile(ctx, 1): for "patch_step", the patch count times
 * mx^2 of each recorded launch (all patches of the launch, dry or wet), so
 * that a roofline can use the cells of the launches actually timed while
 * the forest changes.  0 for kernels without a count.  Synchronises. */
int geoflood_profile_cells(geoflood_ctx* ctx, const char* kernel, long long* cells);

/* Work counters of a scenario since the context was created: interior cell
 * updates computed by the patch step (rejected steps included) and how many
 * of them were wet (h > drytol) at the start of the step. */
int geoflood_counters(geoflood_ctx* ctx, int scenario, long long* cell_updates,
                      long long* wet_cell_updates);

/* Autotuner of the patch-step kernel shape (patch size, threads per CTA,
 * halo staging): times every available variant reps times on the current
 * state (without advancing it), selects the fastest for this context and
 * returns its number in *variant and the times (ms per launch) in
 * ms_per_variant (one entry per variant, at most 16: eight for 32 x 32
 * patches in FP32, four in FP64, one for 16 x 16; either pointer may be
 * NULL).  Variants of
 * 32 x 32 patches: 0 = one 512-thread CTA per patch staging the whole tile
 * by TMA bulk copies, 1 = four CTAs per patch, each staging a 16 x 16
 * sub-tile with its two-cell halo, 2 = the FP32 shape of 0 or the FP64 shape
 * of 1 with the register budget of one CTA per SM, 3 = FP32: one 1024-thread
 * CTA per patch; FP64: adaptive (four sub-tile CTAs for each patch that held
 * water in the previous step, one CTA that checks the whole tile for every
 * other patch); FP32 only: 4 = the sub-tiles of 1 with three 352-thread CTAs
 * per SM, 5 = with four 320-thread CTAs per SM, 6 = adaptive as FP64's 3,
 * 7 = one 608-thread CTA per patch, two per SM.  Results do not depend on
 * the variant. */
int geoflood_autotune(geoflood_ctx* ctx, int reps, int* variant,
                      double* ms_per_variant);

/* Select a patch-step variant by number (see geoflood_autotune). */
int geoflood_set_variant(geoflood_ctx* ctx, int variant);

/* Number of kernels this context has launched since it was created. */
int geoflood_launch_count(geoflood_ctx* ctx, long long* launches);

/* Failure detection check (no counterpart in the paper): every wait of the
 * library's kernels on an asynchronous copy is bounded; when the bound runs
 * out the kernel records GEOFLOOD_ERR_TIMEOUT for the host and returns
 * instead of hanging.  This call confirms that on the GPU in use: a wait on
 * a transaction that never arrives must give up, and the same wait must
 * succeed once the transaction is completed.  stream may be NULL.  Returns
 * 0 when both happen, GEOFLOOD_ERR_STATE otherwise, CUDA or OOM on a failed
 * call. */
int geoflood_check_bounded_wait(void* stream);

/* One FP64 patch step on caller-owned device buffers, allocating nothing.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let the library allocate device memory -- for example a host code
 * that owns all device memory through its own pool, or code running where a
 * cudaMalloc is not allowed -- and therefore cannot create a context.  It
 * runs the same patch-step kernel as geoflood_step (augmented Riemann solves,
 * limited corrections, transverse terms, update, Manning friction) on npatch
 * independent tiles of one level with a fixed dt.
 *
 *   q_in   device, [npatch][3][mx+4][mx+4] h, hu, hv with the two ghost
 *          layers already filled (e.g. by geoflood_read_tiles);
 *   b      device, [npatch][mx+4][mx+4] bed, ghosts included;
 *   q_out  device, same shape as q_in, not overlapping q_in or b: the
 *          interior of every tile is written; each tile is stepped as a lone
 *          patch with walls on all four sides, so the two ghost layers of
 *          q_out receive the wall mirrors of the new edge cells (normal
 *          momentum negated), not neighbour data: refill them before using
 *          q_out as the next call's q_in;
 *   q_in, b and q_out must be 16-byte aligned (the tiles are staged with
 *   bulk copies); a misaligned or overlapping buffer returns ARG before any
 *   work is issued;
 *   mx     16 or 32; dx, dy the cell sizes; dt the step; g, drytol,
 *          manning_n as in the context API;
 *   cmax   host, may be NULL: receives max over the patches of
 *          max(|s|/dx, |s|/dy) over the edges that update interior cells
 *          (the CFL number of the step is dt * cmax); when non-NULL the call
 *          synchronises the stream and also reads the kernel's status:
 *          TIMEOUT if a bounded wait gave up (some tiles unwritten), NAN if
 *          a non-finite value appeared.  With cmax NULL nothing is read back
 *          and these two errors are not reported;
 *   stream cudaStream_t or NULL.
 *
 * The scratch it needs (patch table and the CFL reduction cell) lives in
 * one static device array of about 260 KiB that every GPU
 * loading the library keeps until the process exits; hence npatch is limited
 * to 16384 and a larger npatch returns GEOFLOOD_ERR_CAPACITY.  The first call
 * on a device looks up that array's device address (once per device), so
 * make the first call before any stream capture.  All calls share the array
 * and each call overwrites the previous call's contents (the reduction cell
 * is cleared at the start of every call): calls whose work overlaps on the
 * GPU race, so keep them on one stream.  Only the device-address lookup is
 * safe to make from several host threads at once; calls made concurrently
 * share the array and race as above.  Errors: ARG, CAPACITY, CUDA, TIMEOUT,
 * NAN; the message is returned by geoflood_noalloc_last_error(). */
int geoflood_step_tiles_noalloc(const double* q_in, const double* b,
                                double* q_out, int npatch, int mx, double dx,
                                double dy, double dt, double g, double drytol,
                                double manning_n, double* cmax, void* stream);

/* Message of the last failed geoflood_step_tiles_noalloc call on this host
 * thread ("" if none). */
const char* geoflood_noalloc_last_error(void);

/* ------------------------------------------------------------------------
 * Learned refinement predictor.
 *
 * The paper refines where the plain criteria of Sec. 4.1 (depth, speed,
 * surface elevation, flood-source region) fire, re-evaluated at every
 * regrid.  This extension predicts those flags several steps ahead so that
 * regridding can run less often: a 3-layer convolutional network (3 x 3
 * kernels, 16 channels, ReLU, mean pool, linear head, logistic output) over
 * an 18 x 18 pixel view of each patch: the 16 x 16 grid of (M/16)^2 cell
 * means of the interior plus a ring whose pixels average the band of
 * same-level cells (composite over the forest, M/2 deep) beyond the edge
 * beside them, leaving out cells outside the domain.
 * Input channels: h, hu, hv, bed minus the interior mean bed (each divided
 * by its scale), level / 4, and zeros.  BF16 operands on the tensor cores,
 * FP32 accumulation and FP32 master parameters.
 *
 * Parameters (FP32, geoflood_cnn_nparam() of them, in this order): for layers
 * l = 1, 2, 3, W_l[16 co][144] with column tap * 16 + ci, tap = (dy + 1) * 3
 * + (dx + 1) (dy the row offset), then b_l[16]; then the head wh[16], bh[1].
 *
 * The plain criterion always judges: with the learned tagger selected,
 * geoflood_tags and geoflood_regrid refine where either the criterion or the
 * network (probability above the threshold) asks for it, and
 * geoflood_check_tags counts what the criterion wants refined that the mesh
 * does not yet resolve, so that a caller can regrid at once on a miss. */

/* Number of network parameters (6977). */
int geoflood_cnn_nparam(void);

/* Load the parameters (host, n floats); resets the Adam moments.  The
 * random initialisation is the caller's.  Errors: ARG (wrong n), OOM. */
int geoflood_cnn_set_params(geoflood_ctx* ctx, const float* prm, int n);

/* Copy the current parameters to host memory (n floats).  STATE if none. */
int geoflood_cnn_get_params(geoflood_ctx* ctx, float* prm, int n);

/* Scales that divide h, hu, hv and the relative bed (4 floats > 0; default
 * 10 m, 10 m^2/s, 10 m^2/s, 10 m). */
int geoflood_cnn_set_scale(geoflood_ctx* ctx, const float* scale);

/* Input features of scenario s: host [npatch][324][16] BF16 bit patterns,
 * pixel = Y * 18 + X over the 18 x 18 view. */
int geoflood_cnn_features(geoflood_ctx* ctx, int s, uint16_t* out);

/* Logits of the network for the patches of scenario s (host, npatch). */
int geoflood_cnn_predict(geoflood_ctx* ctx, int s, float* logit);

/* Forward and backward pass on n host samples x ([n][324][16] BF16 bits)
 * with labels in {0, 1}: the logits, the gradient of the mean weighted
 * cross-entropy (weight pos_weight on positive samples) with respect to
 * every parameter, and that loss.  Any output may be NULL. */
int geoflood_cnn_grad(geoflood_ctx* ctx, const uint16_t* x, const float* label,
                      int n, float pos_weight, float* logit, float* grad,
                      float* loss);

/* Allocate (or clear) a device dataset of up to capacity samples. */
int geoflood_cnn_dataset(geoflood_ctx* ctx, int capacity);

/* Record the features of every current patch as pending samples with
 * labels 0. */
int geoflood_cnn_snapshot(geoflood_ctx* ctx);

/* Evaluate the plain criterion on every patch: *misses = number of patches
 * it wants refined that are below the finest level.  With observe != 0 the
 * patches it flags for refinement get label 1 in the pending samples, which
 * must come from a snapshot of the same patches (STATE otherwise). */
int geoflood_check_tags(geoflood_ctx* ctx, int observe, int* misses);

/* Append the pending samples to the dataset (up to its capacity); returns
 * the dataset size and, if positives is non-NULL, its number of label-1
 * samples. */
int geoflood_cnn_commit(geoflood_ctx* ctx, int* total, int* positives);

/* Copy samples [first, first + n) of the dataset to the host (x or y may be
 * NULL). */
int geoflood_cnn_dataset_read(geoflood_ctx* ctx, int first, int n, uint16_t* x,
                              float* y);

/* Train on the dataset: epochs passes over seeded shuffles (splitmix64 from
 * seed) in minibatches of batch samples, Adam (beta 0.9 / 0.999, eps 1e-8)
 * at learning rate lr on the weighted cross-entropy.  epoch_loss (host,
 * epochs floats, may be NULL) receives the mean minibatch loss of each
 * epoch. */
int geoflood_cnn_train(geoflood_ctx* ctx, int epochs, int batch, float lr,
                       float pos_weight, unsigned long long seed,
                       float* epoch_loss);

/* Time stepping with periodic regridding (Sec. 3.3 regrids every few
 * steps; Sec. 6.4 every 4).  Advances every scenario to t_target in chunks
 * of check_interval steps; after each chunk the plain criterion is
 * evaluated (geoflood_check_tags's count, taken on the device right after
 * the chunk's steps and read back with them; when a regrid is due, the
 * regrid's own tag pass counts the criterion's misses instead) and the
 * forest regrids when
 * regrid_interval steps have passed since the last regrid or, with
 * GEOFLOOD_ADVANCE_REGRID_ON_MISS, as soon as the criterion reports a
 * miss.  With GEOFLOOD_ADVANCE_COLLECT it records training samples instead
 * (features at each regrid, labels OR'ed over the checks up to the next one;
 * no regrid on misses): call geoflood_cnn_dataset first.  Needs
 * 1 <= check_interval <= regrid_interval. */
#define GEOFLOOD_ADVANCE_COLLECT 1
#define GEOFLOOD_ADVANCE_REGRID_ON_MISS 2
typedef struct {
  long long steps;        /* accepted steps (maximum over scenarios) */
  long long patch_steps;  /* sum over steps of the number of patches */
  long long checks;       /* evaluations of the plain criterion */
  long long misses;       /* sum over checks of the patches it wanted refined */
  long long regrids;      /* regrids done */
  long long miss_regrids; /* of which triggered by a miss */
  long long samples;      /* dataset size after the run (COLLECT) */
  /* host wall-clock seconds, each including the waits for the device work
   * it issued: in the steps (with the checks taken inside their readback),
   * in separate criterion checks (COLLECT mode), in the regrids, and, of the
   * regrids' time, in the host quadtree (new leaf lists) */
  double step_s, check_s, regrid_s, regrid_host_s;
} geoflood_advance_stats;
int geoflood_advance(geoflood_ctx* ctx, double t_target, int regrid_interval,
                     int check_interval, int mode, geoflood_advance_stats* out);

/* Select the tagger used by geoflood_tags and geoflood_regrid; threshold is
 * the probability above which the network's flag counts (0 < threshold < 1).
 * LEARNED needs parameters (STATE otherwise). */
int geoflood_set_tagger(geoflood_ctx* ctx, int tagger, float threshold);

#ifdef __cplusplus
}
#endif
#endif
