// Internal device-side structures shared by the kernels and the host runtime
// of the GeoFlood GB300 library.  Not part of the public ABI.
#pragma once

#include <cstdint>

#define GF_NG 2          // ghost layers
#define GF_MAXLEV 16     // deepest level a forest may use
#define GF_MAXREGION 8   // refinement regions per context
#define GF_MAXSTEP_REJECT 50
#define GF_SPIN_LIMIT (1u << 22)  // bounded waits on TMA mbarriers

// One patch: level, position on that level's patch grid, scenario.
struct GfPatch {
  int level, px, py, scen;
};

// Per-scenario constants read by the kernels.
// Where a gauge samples: the finest leaf p holding the point, the tile
// index c of the lower-left cell of its 2 x 2 bilinear stencil and the
// weights (ax, ay) of the upper/right cells.  Refreshed after every regrid.
#define GF_MAXDEM 4  // overlapping DEMs per scenario (Sec. 6.2)

struct GfGaugeRef {
  int p, c;
  double ax, ay;
};

struct GfScenario {
  double manning_n, eta0;
  float manning_f;    // FP32 copy of manning_n
  int pad0;
  // nodal DEMs [dny][dnx] in priority order (finest node spacing first);
  // ndem = 0: flat bed at 0
  int ndem;
  int dnx[GF_MAXDEM], dny[GF_MAXDEM];
  const double* dem[GF_MAXDEM];
  double dx0[GF_MAXDEM], dy0[GF_MAXDEM], ddx[GF_MAXDEM], ddy[GF_MAXDEM];
  int poff, pcount;   // patch range in the table
  int lcount[GF_MAXLEV + 1];  // patches per level
  long long lut_off;  // offset of this scenario's lookup tables
  int ngauge;
  int pad;
  const double* gxy;  // [ngauge][2]
  GfGaugeRef* gref;   // [ngauge]
  double* gout;       // [ngauge][5] latest sample
  double* garr;       // [ngauge] arrival time or -1
};

// Per-scenario time-stepping state, owned by the device controller.
struct GfCtl {
  double t, dt_next, dt_use, t_target;
  double clipvol, step_clipvol;
  unsigned long long cmax_bits;     // max CFL rate of the step (bits of a
                                    // non-negative double, atomicMax'ed)
  unsigned long long step_nclip;
  unsigned long long cell_updates;  // interior cells stepped (all launches)
  unsigned long long wet_updates;   // of which wet (h > drytol) before the step
  long long steps, rejects, nclip, taken, max_steps;
  int cur;       // which state buffer is current
  int active;    // this scenario still advances in the current call
  int last;      // the step in flight is clipped to t_target
  int accepted;  // the last step was accepted
  int inrow;     // consecutive rejections
  int status;    // GEOFLOOD_* error from the device, 0 if none
  int nonfinite; // a non-finite value was produced
  // level subcycling: the fine substep about to run (0 .. sub_K - 1; 0 at
  // macro-step boundaries), whether the macro step in flight was rejected,
  // and the largest rate cmax / n_L seen in it (bits of a double)
  int sub_k;
  int sub_rej;
  int pad;
  unsigned long long rmax_bits;
};

// Forest geometry and physics shared by every scenario.
struct GfGeom {
  int mi, mj, M, T;  // T = M + 2*GF_NG
  int minlevel, maxlevel;
  int bc[4];
  double xlower, xupper, ylower, yupper;
  double g, drytol;
  double cfl_desired, cfl_max, dt_max;
  double tag_depth, tag_speed, tag_deta;
  double src_box[4];
  int src_level;
  int nscen;
  long long lut_per_scen;
  long long lut_lev_off[GF_MAXLEV + 1];
  // per-level cell sizes and FP32 copies of the constants, computed on the
  // host so that the FP32 kernels need no FP64 arithmetic per patch
  double dxl[GF_MAXLEV + 1], dyl[GF_MAXLEV + 1], areal[GF_MAXLEV + 1];
  float inv_dxf[GF_MAXLEV + 1], inv_dyf[GF_MAXLEV + 1];
  float gf, drytolf, marginf;
  float tag_depthf, tag_speedf, tag_detaf;
  // criterion 2 (|hu| > tag_flux) and criterion 5 (flow grades)
  double tag_flux;
  float tag_fluxf;
  int ngrades;
  int grade_kind[4], grade_level[4];
  double grade_value[4];
  float grade_valuef[4];
  // scheme variants (Sec. 3.2); all 0: second order, unsplit, transverse
  int first_order, no_transverse, dim_split;
  // inflow hydrograph (Sec. 5.1): n_hydro points (0 = none) of the
  // discharge through [inflow_lo, inflow_hi] of side inflow_side
  int n_hydro, inflow_side;
  double inflow_lo, inflow_hi, inflow_tau;
  double hydro_t[16], hydro_q[16];
  // per level: lines (rows or columns of the side) whose centre lies in
  // the segment, times the cell size
  double inflow_width[GF_MAXLEV + 1];
  // level subcycling (maxlevel > minlevel): level L takes 2^(L - minlevel)
  // steps per macro step, run as sub_K = 2^(maxlevel - minlevel) substeps
  int subcycle, sub_K;
  // refinement regions (Sec. 4.1 criterion 4, Sec. 6.4): active while
  // rt0 <= t <= rt1, they bound the level a cell whose centre lies in
  // [rx0, rx1] x [ry0, ry1] asks for to [rminl, rmaxl]
  int nregions;
  int rminl[GF_MAXREGION], rmaxl[GF_MAXREGION];
  double rx0[GF_MAXREGION], rx1[GF_MAXREGION], ry0[GF_MAXREGION], ry1[GF_MAXREGION];
  double rt0[GF_MAXREGION], rt1[GF_MAXREGION];
};

// Everything a kernel needs to find patches and their data.
struct GfView {
  const GfPatch* patch;   // [npatch]
  const int* lut;         // per scenario, per level: patch index or -1
  GfScenario* scen;       // [nscen]
  GfCtl* ctl;             // [nscen]
  double* q[2];           // FP64 state buffers [cap][3][T][T]: h, hu, hv
  double* b;              // FP64 beds [cap][T][T]
  float* qf[2];           // FP32 state [cap][3][T][T]: w = h + b - eta0, hu, hv
  float* bf;              // FP32 beds minus eta0 [cap][T][T]
  float* lof[2];          // FP32 compensation terms [cap][3][M][M]
  const int* nbr;         // [npatch][8] same-level neighbours (see below)
  // [npatch] the refinement source box against the patch's cell centres
  // (the first and last in each direction, in FP64): bits 0-1 = 1 it misses
  // the patch, 2 it covers it, 0 it crosses it; bits 2k + 2, 2k + 3 the same
  // for refinement region k; or null (then every box and region is tested
  // per cell)
  const unsigned* pbox;
  unsigned* done;         // CTA completion counter of the step (or null)
  // Launch order of the patch step (or null: patch order).  sched[0] selects
  // which of ord0/ord1 this launch reads; the launch writes the other one
  // with the patches whose tile held water first (sched[1], sched[2] count
  // the wet and dry entries) and its last CTA flips sched[0].  Only with a
  // controller (done != null).
  unsigned* sched;
  int* ord0;
  int* ord1;
  // Per CTA work unit (patch * sub-tiles + sub-tile): 1 when both state
  // buffers hold the same interior (a dry tile was copied), so a dry tile
  // can skip its writes (or null).
  unsigned char* same;
  // 1: the patch step also writes the two edge rows and columns of its new
  // interior into the ghost cells of its same-level neighbours in the next
  // buffer (so the separate ghost fill skips those regions); needs nbr.
  int push;
  // adaptive variant: per patch, whether a sub-tile held water and how many
  // of its CTAs have finished (both back to 0 after the patch is reported)
  unsigned* pwet;
  unsigned* pcnt;
  // per patch: 1 if a gauge samples in it (or null)
  unsigned char* gflag;
  // Bed tiles by position (or null): slot = the lookup-table index of
  // (scenario, level, px, py); bcache holds [slots][T][T] of the state's
  // type (double in FP64, float minus eta0 in the deviation form) and
  // bvalid[slot] says whether that slot holds the tile for the current
  // DEMs and eta0.
  void* bcache;
  unsigned char* bvalid;
  // Per patch, two arrays selected by the launch-order parity sched[0] (or
  // null: every patch runs): 1 if the patch must run in the launch that
  // reads that parity.  A launch clears the flags it reads and sets, in the
  // other array, those of every patch whose tile held water and of its
  // same-level neighbours; the cross-level ghost fill and the inflow set
  // those of the patches whose ghost cells they write.  An unmarked patch
  // whose tile is dry and unchanged in both buffers and that holds no gauge
  // returns before staging: its ghost ring is dry, so the full path would
  // write nothing either.  Whole-tile CTAs only; not with subcycling.
  unsigned char* runf;
  int runf_stride;
  int npatch;
  int prec;               // 0 = FP64, 1 = FP32 surface deviation
};

// Neighbour table entries, per patch in the order left, right, bottom, top,
// bottom-left, bottom-right, top-left, top-right: the index of the leaf of
// the same level there, GF_NBR_OTHER if that region is covered by leaves of
// another level, GF_NBR_OUTSIDE beyond the domain.
#define GF_NBR_OTHER -1
#define GF_NBR_OUTSIDE -2

// Kernel launchers (defined in the .cu files).
// Outputs of the tagging pass (every pointer may be null).  raw: the plain
// criterion per patch (0 coarsen, 1 keep, 2 refine); label: set to 1 where it
// says refine; misses: count of patches it wants refined below the finest
// level; logit/logit_thr: learned predictions that add refinement before
// flags (0 keep, 1 refine, 2 coarsen) are formed.
struct GfTagOut {
  uint8_t* flags;
  uint8_t* raw;
  float* label;
  unsigned* misses;
  const float* logit;
  float logit_thr;
};

#ifdef __CUDACC__
// Bilinear weights of the gauges, one form shared by every kernel that samples.
__device__ __forceinline__ double gf_bilinear(double a00, double a10, double a01,
                                              double a11, double ax, double ay) {
  return (1.0 - ay) * ((1.0 - ax) * a00 + ax * a10) + ay * ((1.0 - ax) * a01 + ax * a11);
}
#endif

namespace gf {
int patch_step_variants(int mx, int prec, int dim_split);
int launch_patch_step_f64(const GfGeom& g, const GfView& v, int variant, void* stream);
int launch_patch_step_f32(const GfGeom& g, const GfView& v, int variant, void* stream);
int launch_ctl_begin(GfCtl* ctl, int nscen, double t_target,
                     long long max_steps, const int* scen_mask, void* stream);
int launch_ghost_fill(const GfGeom& g, const GfView& v, int only_active,
                      void* stream);
// Ghost cells in regions without a same-level neighbour (which the patch
// step's push leaves out) with their boundary mirrors: regs[k] = patch * 8 +
// region, k < nreg; the first nquad regions border a coarser leaf (filled
// by blocks of 2 x 2 children), the others finer leaves.
int launch_ghost_rest(const GfGeom& g, const GfView& v, const int* regs, int nquad,
                      int nreg, void* stream);
// Inflow ghost cells (Sec. 5.1) of the n patches in list (patches on the
// inflow side), after every other ghost cell is final; only_accepted: skip
// scenarios whose last step was rejected.
int launch_inflow(const GfGeom& g, const GfView& v, const int* list, int n,
                  int only_accepted, void* stream);
// Level subcycling, after the last substep of an accepted macro step: the
// patches of level minlevel (one step, an odd number) copy their new state
// (tile and FP32 compensation terms) into the current buffer, which every
// other level is back in after its even number of steps.
int launch_subcycle_sync(const GfGeom& g, const GfView& v, void* stream);
// Beds of patches [first, first + count), or of list[0..count) if list.
int launch_topo(const GfGeom& g, const GfView& v, int first, int count,
                void* stream, const int* list = nullptr);
// Regrid transfer into the new forest: every patch, or list[0..count).
int launch_regrid_fill(const GfGeom& g, const GfView& oldv, const GfView& newv,
                       void* stream, const int* list = nullptr, int count = 0);
// Copy of the patches present in both forests: pairs (int2: new, old).
int launch_regrid_keep(const GfGeom& g, const GfView& oldv, const GfView& newv,
                       const void* pairs, int count, void* stream);
// Latest state of every patch into buffer target (patches whose scenario
// holds it in the other buffer are copied); the caller then sets every
// scenario's cur to target.
int launch_align_buffers(const GfGeom& g, const GfView& v, int target, void* stream);
int launch_tags(const GfGeom& g, const GfView& v, uint8_t* flags,
                void* stream);
// Recompute every scenario's gauge stencils (after a regrid or new gauges).
int launch_gauge_refs(const GfGeom& g, const GfView& v, int max_gauges,
                      void* stream);
int launch_gauges(const GfGeom& g, const GfView& v, int only_accepted,
                  int max_gauges, void* stream);
int launch_mass(const GfGeom& g, const GfView& v, double* pmass,
                double* smass, int nscen, void* stream);
int launch_pack_interior(const GfGeom& g, const GfView& v, int scen_first,
                         int count, double* out, int field_mask, int cur,
                         void* stream);
int launch_unpack_interior(const GfGeom& g, const GfView& v, int first,
                           int count, const double* in, int cur,
                           void* stream);
void set_errflag(int* device_flag);
int launch_tags_ex(const GfGeom& g, const GfView& v, const GfTagOut& o,
                   void* stream);
int launch_cnn_features(const GfGeom& g, const GfView& v, int first, int count,
                        const float* scale, void* out, void* stream);
// learned refinement predictor (gf_cnn.cu)
int cnn_nparam();
int cnn_forward(const void* x0, const void* wb, const float* prm, void* a1,
                void* a2, void* a3, float* v, float* logit, int npatch,
                void* stream);
int cnn_backward(const void* x0, const void* wf, const float* prm,
                 const void* a1, const void* a2, const void* a3, const float* v,
                 const float* logit, const float* label, float pos_weight,
                 float* grad, float* loss, void* d1, void* d2, void* d3,
                 int npatch, void* stream);
int cnn_adam(float* prm, const float* grad, float* m, float* v, float lr,
             int t, void* stream);
int cnn_cast(const float* prm, void* wb, void* wf, void* stream);
int cnn_to_bf16(const float* x, void* y, size_t n, void* stream);
int cnn_gather(const void* x, const float* y, const int* idx, int n, void* xb,
               float* yb, void* stream);
constexpr int CNN_IN_PIX = 324;  // 18 x 18 input pixels per patch
constexpr int CNN_PIX = 256;     // 16 x 16 activation pixels per patch
constexpr int CNN_CH = 16;
}  // namespace gf
