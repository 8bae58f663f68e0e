// C ABI of the GeoFlood GB300 library: context, forest tables, staging and
// the time-stepping driver.  See include/geoflood.h for the contract of each
// entry point.
#include "../../include/geoflood.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>
#include <unordered_map>
#include <thread>

#include "gf_forest.h"
#include "gf_internal.h"

namespace {

struct ProfRec {
  cudaEvent_t a, b;
  long long cells = 0;  // interior cells of the launch (patch step)
};

// Device state of the learned refinement predictor.
struct CnnState {
  float* prm = nullptr;  // FP32 master parameters
  void* wb = nullptr;    // BF16 conv weights [3][16][144]
  void* wf = nullptr;    // and their flipped transposes
  float* grad = nullptr;
  float* am = nullptr;   // Adam moments
  float* av = nullptr;
  int adam_t = 0;
  bool ready = false;
  float scale[4] = {10.f, 10.f, 10.f, 10.f};
  // inference over the current patches (sized to the patch capacity)
  void* x = nullptr;
  void* a[3] = {nullptr, nullptr, nullptr};
  float* pool = nullptr;
  float* logit = nullptr;
  // pending samples: features at a snapshot, labels OR'ed over checks
  void* px = nullptr;
  float* py = nullptr;
  int pend_n = -1;
  long long pend_gen = -1;
  // dataset
  void* dx = nullptr;
  float* dy = nullptr;
  int ds_cap = 0, ds_n = 0;
  // training minibatch
  void* xb = nullptr;
  float* yb = nullptr;
  int* idx = nullptr;
  void* ta[3] = {nullptr, nullptr, nullptr};
  void* td[3] = {nullptr, nullptr, nullptr};
  float* tv = nullptr;
  float* tlogit = nullptr;
  float* loss = nullptr;
  int bcap = 0, idx_cap = 0;
  int tagger = GEOFLOOD_TAGGER_PLAIN;
  float logit_thr = 0.f;
  unsigned* misses = nullptr;
};

}  // namespace

struct geoflood_ctx {
  geoflood_config cfg{};
  cudaStream_t st = nullptr;
  GfGeom G{};
  int cap = 0, nscen = 0, npatch = 0;
  double* q[2] = {nullptr, nullptr};
  double* b[2] = {nullptr, nullptr};
  float* qf[2] = {nullptr, nullptr};  // FP32 surface-deviation state
  float* bf[2] = {nullptr, nullptr};
  float* lof[2] = {nullptr, nullptr};
  int prec = 0;
  int bsel = 0;
  GfPatch* d_patch[2] = {nullptr, nullptr};
  int* d_lut[2] = {nullptr, nullptr};
  int* d_nbr[2] = {nullptr, nullptr};
  unsigned* d_pbox[2] = {nullptr, nullptr};
  unsigned* d_done = nullptr;
  unsigned* d_sched = nullptr;        // launch-order parity and counters
  int* d_ord[2] = {nullptr, nullptr}; // launch orders of the patch step
  unsigned char* d_same = nullptr;    // per work unit: buffers agree
  unsigned char* d_runf = nullptr;    // [2][cap] run flags (see GfView::runf)
  unsigned char* d_gflag = nullptr;   // per patch: holds a gauge
  unsigned* d_pwet = nullptr;         // adaptive variant: per-patch flags
  unsigned* d_pcnt = nullptr;
  int* d_rlist = nullptr;   // regrid: new slots to compute
  int* d_rpairs = nullptr;  // regrid: (new, old) slots to copy
  int* d_glist[2] = {nullptr, nullptr};  // ghost regions next to a level change
  int nglist[2] = {0, 0};
  int nglist_c[2] = {0, 0};  // of which the first ones border a coarser leaf
  int* d_ilist[2] = {nullptr, nullptr};  // patches on the inflow side
  int nilist[2] = {0, 0};
  bool own_stream = false;
  // CUDA graphs of chunks of steps, keyed by chunk length
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int k = 0, tsel = -1, bsel = -1, npatch = -1, gauges = -1, prof = -1, variant = -1;
    // the forest the graph was captured for: its launches carry the number
    // of ghost regions at level changes and of inflow patches, which change
    // with every regrid even when the patch count does not
    long long generation = -1;
    std::vector<ProfRec> ev;   // sampled patch-step launches
    std::vector<ProfRec> evg;  // sampled ghost fills
  };
  std::vector<Graph> graphs;
  int tsel = 0;
  GfScenario* d_scen = nullptr;
  std::vector<GfScenario> h_scen;
  GfCtl* d_ctl = nullptr;
  GfCtl* h_ctl = nullptr;  // pinned mirror
  int* h_rb = nullptr;     // pinned: [0] device error flag, [1] criterion misses
  double* d_pmass = nullptr;
  double* d_smass = nullptr;
  uint8_t* d_flags = nullptr;
  int* d_err = nullptr;
  double* d_stage = nullptr;
  size_t stage_cap = 0;
  std::vector<gf::HostForest> forests;
  std::vector<double*> d_gxy, d_gout, d_garr;
  std::vector<std::vector<double*>> d_dem;  // per scenario, priority order
  std::vector<GfGaugeRef*> d_gref;
  int max_gauges_used = 0;
  int variant = 0;  // patch-step kernel variant (see geoflood_autotune)
  std::string err;
  bool prof = false;
  int prof_every = 1;  // time every n-th patch step of a graph chunk
  std::map<std::string, std::vector<ProfRec>> prof_recs;
  std::map<std::string, double> prof_ms;
  std::map<std::string, long long> prof_n;
  std::map<std::string, long long> prof_cells;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  long long launches = 0;
  long long generation = 0;  // bumped by every regrid
  double regrid_host_s = 0;  // host wall time of the quadtree regrids so far
  // bed tiles by position (see GfView::bcache), allocated when they fit
  // kBedCacheBudget bytes
  void* d_bcache = nullptr;
  unsigned char* d_bvalid = nullptr;
  // pinned staging of host-built tables: uploads read it asynchronously; the
  // event marks when the last upload from it has been consumed
  unsigned char* h_up = nullptr;
  size_t h_up_cap = 0, h_up_used = 0;
  cudaEvent_t up_ev = nullptr;
  bool up_pending = false;
  uint8_t* h_flags = nullptr;  // pinned copy of the tags for the host quadtree
  size_t h_flags_cap = 0;
  CnnState cnn;
};

namespace {

// Device memory the bed cache may take (all scenarios, all levels).
constexpr size_t kBedCacheBudget = size_t(16) << 30;

int fail(geoflood_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                          \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess)                                                \
      return fail(ctx, GEOFLOOD_ERR_CUDA,                                 \
                  std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

#define CKL(expr, name)                                                   \
  do {                                                                    \
    if ((expr) != 0) {                                                    \
      cudaError_t e_ = cudaGetLastError();                                \
      return fail(ctx, GEOFLOOD_ERR_CUDA,                                 \
                  std::string("launch ") + name + ": " +                  \
                      cudaGetErrorString(e_));                            \
    }                                                                     \
  } while (0)

GfView view(geoflood_ctx* c, int t, int bb) {
  GfView v{};
  v.patch = c->d_patch[t];
  v.lut = c->d_lut[t];
  v.scen = c->d_scen;
  v.ctl = c->d_ctl;
  v.q[0] = c->q[0];
  v.q[1] = c->q[1];
  v.b = c->b[bb];
  v.qf[0] = c->qf[0];
  v.qf[1] = c->qf[1];
  v.bf = c->bf[bb];
  v.lof[0] = c->lof[0];
  v.lof[1] = c->lof[1];
  v.nbr = c->d_nbr[t];
  v.pbox = c->d_pbox[t];
  v.done = c->d_done;
  v.sched = c->d_sched;
  v.ord0 = c->d_ord[0];
  v.ord1 = c->d_ord[1];
  v.same = c->d_same;
  v.push = 1;
  v.pwet = c->d_pwet;
  v.gflag = c->d_gflag;
  v.pcnt = c->d_pcnt;
  v.bcache = c->d_bcache;
  v.bvalid = c->d_bvalid;
  v.runf = c->d_runf;
  v.runf_stride = c->cap;
  v.npatch = c->npatch;
  v.prec = c->prec;
  return v;
}
GfView view(geoflood_ctx* c) { return view(c, c->tsel, c->bsel); }

// Events come from a pool created ahead of time so that recording them adds
// no allocation to the launch loop.
cudaEvent_t pool_event(geoflood_ctx* c) {
  if (c->pool_used == c->pool.size()) {
    const size_t grow = c->pool.empty() ? 4096 : c->pool.size();
    for (size_t k = 0; k < grow; ++k) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c->pool.push_back(e);
    }
  }
  return c->pool[c->pool_used++];
}
void prof_begin(geoflood_ctx* c, const char* name, ProfRec* r) {
  if (!c->prof) return;
  r->a = pool_event(c);
  r->b = pool_event(c);
  cudaEventRecord(r->a, c->st);
  (void)name;
}
void prof_end(geoflood_ctx* c, const char* name, ProfRec* r) {
  if (!c->prof) return;
  cudaEventRecord(r->b, c->st);
  c->prof_recs[name].push_back(*r);
}

bool valid_scen(geoflood_ctx* c, int s) { return c && s >= 0 && s < c->nscen; }

int sync_ctl_down(geoflood_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, sizeof(GfCtl) * ctx->nscen,
                     cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int sync_ctl_up(geoflood_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->d_ctl, ctx->h_ctl, sizeof(GfCtl) * ctx->nscen,
                     cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int ensure_stage(geoflood_ctx* ctx, size_t doubles) {
  if (doubles <= ctx->stage_cap) return 0;
  if (ctx->d_stage) cudaFree(ctx->d_stage);
  ctx->d_stage = nullptr;
  CK(cudaMalloc(&ctx->d_stage, doubles * sizeof(double)));
  ctx->stage_cap = doubles;
  return 0;
}

// Start a batch of uploads of at most `bytes` through the pinned staging
// buffer: waits until the previous batch has been consumed, grows the buffer
// if needed.
int upload_begin(geoflood_ctx* ctx, size_t bytes) {
  if (ctx->up_pending) {
    CK(cudaEventSynchronize(ctx->up_ev));
    ctx->up_pending = false;
  }
  if (!ctx->up_ev) CK(cudaEventCreateWithFlags(&ctx->up_ev, cudaEventDisableTiming));
  if (bytes > ctx->h_up_cap) {
    if (ctx->h_up) cudaFreeHost(ctx->h_up);
    ctx->h_up = nullptr;
    ctx->h_up_cap = 0;
    const size_t cap = bytes + bytes / 2 + 4096;
    if (cudaMallocHost((void**)&ctx->h_up, cap) != cudaSuccess) {
      cudaGetLastError();
      ctx->h_up = nullptr;
      return fail(ctx, GEOFLOOD_ERR_OOM, "pinned staging buffer");
    }
    ctx->h_up_cap = cap;
  }
  ctx->h_up_used = 0;
  return 0;
}

// Copy `bytes` from host memory into the staging buffer and enqueue their
// transfer to the device address dst on the context's stream.
int upload_put(geoflood_ctx* ctx, void* dst, const void* src, size_t bytes) {
  if (!bytes) return 0;
  const size_t at = (ctx->h_up_used + 255) & ~size_t(255);
  if (at + bytes > ctx->h_up_cap) return fail(ctx, GEOFLOOD_ERR_STATE, "staging overflow");
  std::memcpy(ctx->h_up + at, src, bytes);
  CK(cudaMemcpyAsync(dst, ctx->h_up + at, bytes, cudaMemcpyHostToDevice, ctx->st));
  ctx->h_up_used = at + bytes;
  return 0;
}

// Close the batch: the buffer may be reused once the stream has passed here.
int upload_end(geoflood_ctx* ctx) {
  CK(cudaEventRecord(ctx->up_ev, ctx->st));
  ctx->up_pending = true;
  return 0;
}

// Room a batch of uploads needs: the bytes plus the alignment of each piece.
size_t upload_room(std::initializer_list<size_t> sizes) {
  size_t t = 0;
  for (size_t b : sizes) t += b + 256;
  return t;
}

// Staging room that upload_tables needs for `total` patches (an upper bound:
// neighbour table, ghost regions, inflow list, launch order, patch table,
// box and region classes, lookup tables, scenarios).
size_t tables_room(const geoflood_ctx* ctx, size_t total) {
  return upload_room({sizeof(int) * 8 * total, sizeof(int) * 8 * total, sizeof(int) * total,
                      sizeof(int) * total, sizeof(GfPatch) * total, sizeof(unsigned) * total,
                      sizeof(int) * (size_t)ctx->nscen * ctx->G.lut_per_scen,
                      sizeof(GfScenario) * ctx->nscen});
}

// Upload the patch table and lookup tables of the current forests into
// table slot t; updates poff/pcount of every scenario.  The uploads are
// asynchronous (staged in pinned memory).
int upload_tables(geoflood_ctx* ctx, int t,
                  const std::vector<std::vector<gf::Leaf>>& lv, bool batch_open = false) {
  size_t total = 0;
  for (auto& v : lv) total += v.size();
  if ((long long)total > ctx->cap)
    return fail(ctx, GEOFLOOD_ERR_CAPACITY,
                "forest needs " + std::to_string(total) +
                    " patches, capacity is " + std::to_string(ctx->cap));
  std::vector<GfPatch> hp(total);
  std::vector<int> lut((size_t)ctx->nscen * ctx->G.lut_per_scen, -1);
  int off = 0;
  for (int s = 0; s < ctx->nscen; ++s) {
    ctx->h_scen[s].poff = off;
    ctx->h_scen[s].pcount = (int)lv[s].size();
    for (int L = 0; L <= GF_MAXLEV; ++L) ctx->h_scen[s].lcount[L] = 0;
    for (const gf::Leaf& l : lv[s]) ctx->h_scen[s].lcount[l.level]++;
    for (size_t k = 0; k < lv[s].size(); ++k) {
      const gf::Leaf& l = lv[s][k];
      hp[off + k] = GfPatch{l.level, l.px, l.py, s};
      const long long w = (long long)ctx->G.mi << l.level;
      lut[(size_t)ctx->h_scen[s].lut_off + ctx->G.lut_lev_off[l.level] + l.px +
          (long long)l.py * w] = off + (int)k;
    }
    off += (int)lv[s].size();
  }
  // same-level neighbours of every patch (left, right, bottom, top, then the
  // corners bottom-left, bottom-right, top-left, top-right)
  std::vector<int> nb(total * 8);
  static const int DX[8] = {-1, 1, 0, 0, -1, 1, -1, 1};
  static const int DY[8] = {0, 0, -1, 1, -1, -1, 1, 1};
  for (size_t k = 0; k < total; ++k) {
    const GfPatch& P = hp[k];
    const long long w = (long long)ctx->G.mi << P.level, h = (long long)ctx->G.mj << P.level;
    for (int r = 0; r < 8; ++r) {
      const long long X = P.px + DX[r], Y = P.py + DY[r];
      if (X < 0 || Y < 0 || X >= w || Y >= h) { nb[k * 8 + r] = GF_NBR_OUTSIDE; continue; }
      const int q = lut[(size_t)ctx->h_scen[P.scen].lut_off + ctx->G.lut_lev_off[P.level] + X + Y * w];
      nb[k * 8 + r] = q >= 0 ? q : GF_NBR_OTHER;
    }
  }
  // ghost regions that no same-level neighbour pushes into (a finer or
  // coarser neighbour), as patch * 8 + region: filled after each step
  // first those next to a coarser leaf, then those next to finer leaves
  std::vector<int> gl, glf;
  for (size_t k = 0; k < total; ++k) {
    const GfPatch& P = hp[k];
    for (int r = 0; r < 8; ++r) {
      if (nb[k * 8 + r] != GF_NBR_OTHER) continue;
      bool coarser = false;
      if (P.level > 0) {
        const long long X = (P.px + DX[r]) >> 1, Y = (P.py + DY[r]) >> 1;
        const long long w = (long long)ctx->G.mi << (P.level - 1);
        coarser = lut[(size_t)ctx->h_scen[P.scen].lut_off + ctx->G.lut_lev_off[P.level - 1] + X +
                      Y * w] >= 0;
      }
      (coarser ? gl : glf).push_back((int)k * 8 + r);
    }
  }
  ctx->nglist_c[t] = (int)gl.size();
  gl.insert(gl.end(), glf.begin(), glf.end());
  // the source box and the refinement regions against each patch's first
  // and last cell centres, in the tag kernel's FP64 arithmetic (this file is
  // compiled without contraction, like the device code): two bits each,
  // 1 misses the patch, 2 covers it, 0 crosses it
  std::vector<unsigned> pbox(total);
  {
    const GfGeom& G = ctx->G;
    const int M = G.M;
    for (size_t k = 0; k < total; ++k) {
      const GfPatch& P = hp[k];
      const double dx = G.dxl[P.level], dy = G.dyl[P.level];
      const double x0 = G.xlower + ((double)((long long)P.px * M) + 0.5) * dx;
      const double x1 = G.xlower + ((double)((long long)P.px * M + M - 1) + 0.5) * dx;
      const double y0 = G.ylower + ((double)((long long)P.py * M) + 0.5) * dy;
      const double y1 = G.ylower + ((double)((long long)P.py * M + M - 1) + 0.5) * dy;
      auto cls = [&](double bx0, double bx1, double by0, double by1) -> unsigned {
        const bool none = x1 < bx0 || x0 > bx1 || y1 < by0 || y0 > by1;
        const bool all = x0 >= bx0 && x1 <= bx1 && y0 >= by0 && y1 <= by1;
        return (none ? 1u : 0u) | (all ? 2u : 0u);
      };
      unsigned bits = cls(G.src_box[0], G.src_box[1], G.src_box[2], G.src_box[3]);
      for (int r = 0; r < G.nregions; ++r)
        bits |= cls(G.rx0[r], G.rx1[r], G.ry0[r], G.ry1[r]) << (2 + 2 * r);
      pbox[k] = bits;
    }
  }
  ctx->nglist[t] = (int)gl.size();
  // patches on the inflow side whose tile lines (ghost lines included) may
  // reach the inflow segment
  std::vector<int> il;
  const GfGeom& G = ctx->G;
  if (G.n_hydro > 0) {
    const bool xs = G.inflow_side <= 1;
    for (size_t k = 0; k < total; ++k) {
      const GfPatch& P = hp[k];
      const long long w = (long long)G.mi << P.level, h = (long long)G.mj << P.level;
      const bool at = G.inflow_side == 0   ? P.px == 0
                      : G.inflow_side == 1 ? P.px == w - 1
                      : G.inflow_side == 2 ? P.py == 0
                                           : P.py == h - 1;
      if (!at) continue;
      const double lo = xs ? G.ylower : G.xlower, hi = xs ? G.yupper : G.xupper;
      const double d = (hi - lo) / (double)((xs ? h : w) * G.M);
      const double a = lo + ((double)(xs ? P.py : P.px) * G.M - GF_NG) * d;
      const double b = a + (double)(G.M + 2 * GF_NG) * d;
      if (b >= G.inflow_lo && a <= G.inflow_hi) il.push_back((int)k);
    }
  }
  ctx->nilist[t] = (int)il.size();
  // a new patch list: launch order back to patch order, no tile known to
  // agree between the buffers
  std::vector<int> iota(total);
  for (size_t k = 0; k < total; ++k) iota[k] = (int)k;
  int rc = batch_open ? 0
                      : upload_begin(ctx, tables_room(ctx, total));
  if (rc) return rc;
  rc |= upload_put(ctx, ctx->d_nbr[t], nb.data(), sizeof(int) * nb.size());
  rc |= upload_put(ctx, ctx->d_pbox[t], pbox.data(), sizeof(unsigned) * total);
  rc |= upload_put(ctx, ctx->d_glist[t], gl.data(), sizeof(int) * gl.size());
  rc |= upload_put(ctx, ctx->d_ilist[t], il.data(), sizeof(int) * il.size());
  rc |= upload_put(ctx, ctx->d_ord[0], iota.data(), sizeof(int) * total);
  CK(cudaMemcpyAsync(ctx->d_ord[1], ctx->d_ord[0], sizeof(int) * total,
                     cudaMemcpyDeviceToDevice, ctx->st));
  CK(cudaMemsetAsync(ctx->d_sched, 0, 8 * sizeof(unsigned), ctx->st));
  CK(cudaMemsetAsync(ctx->d_same, 0, (size_t)ctx->cap * 4, ctx->st));
  CK(cudaMemsetAsync(ctx->d_runf, 1, (size_t)ctx->cap * 2, ctx->st));
  CK(cudaMemsetAsync(ctx->d_pwet, 0, (size_t)ctx->cap * sizeof(unsigned), ctx->st));
  CK(cudaMemsetAsync(ctx->d_gflag, 0, (size_t)ctx->cap, ctx->st));
  CK(cudaMemsetAsync(ctx->d_pcnt, 0, (size_t)ctx->cap * sizeof(unsigned), ctx->st));
  rc |= upload_put(ctx, ctx->d_patch[t], hp.data(), sizeof(GfPatch) * total);
  rc |= upload_put(ctx, ctx->d_lut[t], lut.data(), sizeof(int) * lut.size());
  rc |= upload_put(ctx, ctx->d_scen, ctx->h_scen.data(), sizeof(GfScenario) * ctx->nscen);
  if (rc) return rc;
  return batch_open ? 0 : upload_end(ctx);
}

int upload_scen(geoflood_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->d_scen, ctx->h_scen.data(),
                     sizeof(GfScenario) * ctx->nscen, cudaMemcpyHostToDevice,
                     ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int check_errflag(geoflood_ctx* ctx) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                     ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (e) {
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->st));
    return fail(ctx, GEOFLOOD_ERR_STATE,
                "forest lookup failed (unbalanced or uncovered forest)");
  }
  return 0;
}

int ghost_fill_all(geoflood_ctx* ctx) {
  gf::set_errflag(ctx->d_err);
  // ghost cells rewritten from scratch: every patch runs next
  CK(cudaMemsetAsync(ctx->d_runf, 1, (size_t)ctx->cap * 2, ctx->st));
  ProfRec r;
  prof_begin(ctx, "ghost_fill", &r);
  CKL(gf::launch_ghost_fill(ctx->G, view(ctx), 0, ctx->st), "ghost_fill");
  ctx->launches++;
  if (ctx->nilist[ctx->tsel] > 0) {
    CKL(gf::launch_inflow(ctx->G, view(ctx), ctx->d_ilist[ctx->tsel],
                          ctx->nilist[ctx->tsel], 0, ctx->st),
        "inflow");
    ctx->launches++;
  }
  prof_end(ctx, "ghost_fill", &r);
  return check_errflag(ctx);
}

// After the host writes state or beds, no tile is known to agree between
// the two state buffers.
int forget_same(geoflood_ctx* ctx) {
  CK(cudaMemsetAsync(ctx->d_same, 0, (size_t)ctx->cap * 4, ctx->st));
  // every patch runs until the marks of two launches have built up again
  CK(cudaMemsetAsync(ctx->d_runf, 1, (size_t)ctx->cap * 2, ctx->st));
  return 0;
}

// The bed tiles cached for a scenario no longer match after its DEMs or its
// reference surface change.
int forget_beds(geoflood_ctx* ctx, int s) {
  if (ctx->d_bvalid)
    CK(cudaMemsetAsync(ctx->d_bvalid + (size_t)s * ctx->G.lut_per_scen, 0,
                       (size_t)ctx->G.lut_per_scen, ctx->st));
  return 0;
}

int topo_scenario(geoflood_ctx* ctx, int s) {
  int rc = forget_same(ctx);
  if (rc) return rc;
  if ((rc = forget_beds(ctx, s))) return rc;
  CKL(gf::launch_topo(ctx->G, view(ctx), ctx->h_scen[s].poff,
                      ctx->h_scen[s].pcount, ctx->st),
      "topo");
  ctx->launches++;
  return 0;
}

int cnn_alloc(geoflood_ctx* ctx, void** p, size_t bytes) {
  if (*p) return 0;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ctx, GEOFLOOD_ERR_OOM, "learned tagger: out of device memory");
  }
  return 0;
}

const size_t CNN_X_BYTES = (size_t)gf::CNN_IN_PIX * gf::CNN_CH * 2;
const size_t CNN_A_BYTES = (size_t)gf::CNN_PIX * gf::CNN_CH * 2;

int cnn_params_alloc(geoflood_ctx* ctx) {
  CnnState& n = ctx->cnn;
  const size_t np = (size_t)gf::cnn_nparam();
  int rc = 0;
  rc |= cnn_alloc(ctx, (void**)&n.prm, np * 4);
  rc |= cnn_alloc(ctx, (void**)&n.grad, np * 4);
  rc |= cnn_alloc(ctx, (void**)&n.am, np * 4);
  rc |= cnn_alloc(ctx, (void**)&n.av, np * 4);
  rc |= cnn_alloc(ctx, &n.wb, 3 * 16 * 144 * 2);
  rc |= cnn_alloc(ctx, &n.wf, 3 * 16 * 144 * 2);
  rc |= cnn_alloc(ctx, (void**)&n.loss, 4 * 1024);
  return rc ? GEOFLOOD_ERR_OOM : 0;
}

int cnn_infer_alloc(geoflood_ctx* ctx) {
  CnnState& n = ctx->cnn;
  const size_t cap = (size_t)ctx->cap;
  int rc = 0;
  rc |= cnn_alloc(ctx, &n.x, cap * CNN_X_BYTES);
  for (int l = 0; l < 3; ++l) rc |= cnn_alloc(ctx, &n.a[l], cap * CNN_A_BYTES);
  rc |= cnn_alloc(ctx, (void**)&n.pool, cap * 16 * 4);
  rc |= cnn_alloc(ctx, (void**)&n.logit, cap * 4);
  return rc ? GEOFLOOD_ERR_OOM : 0;
}

int cnn_batch_alloc(geoflood_ctx* ctx, int b) {
  CnnState& n = ctx->cnn;
  if (b <= n.bcap) return 0;
  for (void* p : {n.xb, (void*)n.yb, n.ta[0], n.ta[1], n.ta[2], n.td[0], n.td[1], n.td[2],
                  (void*)n.tv, (void*)n.tlogit})
    cudaFree(p);
  n.xb = nullptr; n.yb = nullptr; n.tv = nullptr; n.tlogit = nullptr;
  for (int l = 0; l < 3; ++l) n.ta[l] = n.td[l] = nullptr;
  n.bcap = 0;
  int rc = 0;
  rc |= cnn_alloc(ctx, &n.xb, (size_t)b * CNN_X_BYTES);
  rc |= cnn_alloc(ctx, (void**)&n.yb, (size_t)b * 4);
  for (int l = 0; l < 3; ++l) {
    rc |= cnn_alloc(ctx, &n.ta[l], (size_t)b * CNN_A_BYTES);
    rc |= cnn_alloc(ctx, &n.td[l], (size_t)b * CNN_A_BYTES);
  }
  rc |= cnn_alloc(ctx, (void**)&n.tv, (size_t)b * 16 * 4);
  rc |= cnn_alloc(ctx, (void**)&n.tlogit, (size_t)b * 4);
  if (rc) return GEOFLOOD_ERR_OOM;
  n.bcap = b;
  return 0;
}

// Features and logits of the current patches [first, first + count).
int cnn_infer(geoflood_ctx* ctx, int first, int count) {
  CnnState& n = ctx->cnn;
  int rc = cnn_infer_alloc(ctx);
  if (rc) return rc;
  CKL(gf::launch_cnn_features(ctx->G, view(ctx), first, count, n.scale, n.x, ctx->st),
      "cnn_features");
  CKL(gf::cnn_forward(n.x, n.wb, n.prm, n.a[0], n.a[1], n.a[2], n.pool, n.logit, count,
                      ctx->st),
      "cnn_forward");
  ctx->launches += 5;
  return 0;
}

// One tagging pass over every patch into ctx->d_flags; with learned tags the
// network's predictions are added to the plain criterion.  misses (device
// counter) and pending labels are filled when asked for.
int tag_pass(geoflood_ctx* ctx, bool learned, unsigned* misses, float* label = nullptr) {
  GfTagOut o{};
  o.flags = ctx->d_flags;
  o.misses = misses;
  o.label = label;
  if (learned) {
    if (!ctx->cnn.ready)
      return fail(ctx, GEOFLOOD_ERR_STATE, "learned tagging without network parameters");
    int rc = cnn_infer(ctx, 0, ctx->npatch);
    if (rc) return rc;
    o.logit = ctx->cnn.logit;
    o.logit_thr = ctx->cnn.logit_thr;
  }
  CKL(gf::launch_tags_ex(ctx->G, view(ctx), o, ctx->st), "tags");
  ctx->launches++;
  return 0;
}

// splitmix64 (Steele, Lea and Flood 2014): the stream behind the minibatch
// shuffles.
uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int geoflood_init_forest(const geoflood_config* cfg, void* stream,
                         geoflood_ctx** out) {
  if (!cfg || !out) return GEOFLOOD_ERR_ARG;
  *out = nullptr;
  const geoflood_config& c = *cfg;
  if (!(c.mx == 16 || c.mx == 32) || c.mi < 1 || c.mj < 1 || c.minlevel < 0 ||
      c.maxlevel < c.minlevel || c.maxlevel > GF_MAXLEV - 2 ||
      c.num_scenarios < 1 || c.max_patches < 1 || c.max_gauges < 0 ||
      !(c.xupper > c.xlower) || !(c.yupper > c.ylower) || !(c.g > 0) ||
      !(c.drytol > 0) || !(c.cfl_desired > 0) || !(c.cfl_max >= c.cfl_desired) ||
      !(c.dt_initial > 0) || !(c.dt_max > 0) ||
      (c.precision != GEOFLOOD_FP64 && c.precision != GEOFLOOD_FP32_DEV))
    return GEOFLOOD_ERR_ARG;
  for (int k = 0; k < 4; ++k)
    if (c.bc[k] != GEOFLOOD_BC_WALL && c.bc[k] != GEOFLOOD_BC_EXTRAP)
      return GEOFLOOD_ERR_ARG;
  if (c.ngrades < 0 || c.ngrades > 4 || !(c.tag_flux > 0)) return GEOFLOOD_ERR_ARG;
  if ((c.first_order | c.no_transverse | c.dim_split | c.subcycle) & ~1) return GEOFLOOD_ERR_ARG;
  if (c.n_hydro < 0 || c.n_hydro > 16) return GEOFLOOD_ERR_ARG;
  if (c.n_hydro > 0) {
    if (c.inflow_side < 0 || c.inflow_side > 3 || !(c.inflow_hi > c.inflow_lo) ||
        !(c.inflow_tau > 0))
      return GEOFLOOD_ERR_ARG;
    for (int k = 0; k < c.n_hydro; ++k)
      if (!(c.hydro_q[k] >= 0 && c.hydro_q[k] < 1e300) || !(c.hydro_t[k] > -1e300 && c.hydro_t[k] < 1e300) ||
          (k > 0 && !(c.hydro_t[k] > c.hydro_t[k - 1])))
        return GEOFLOOD_ERR_ARG;
  }
  for (int k = 0; k < c.ngrades; ++k)
    if ((c.grade_kind[k] != 0 && c.grade_kind[k] != 1) || c.grade_level[k] < c.minlevel ||
        c.grade_level[k] > c.maxlevel)
      return GEOFLOOD_ERR_ARG;
  if (c.nregions < 0 || c.nregions > GF_MAXREGION) return GEOFLOOD_ERR_ARG;
  for (int k = 0; k < c.nregions; ++k)
    if (c.region_minlevel[k] < c.minlevel || c.region_maxlevel[k] > c.maxlevel ||
        c.region_minlevel[k] > c.region_maxlevel[k] || !(c.region_x1[k] >= c.region_x0[k]) ||
        !(c.region_y1[k] >= c.region_y0[k]) || !(c.region_t1[k] >= c.region_t0[k]))
      return GEOFLOOD_ERR_ARG;
  geoflood_ctx* ctx = new geoflood_ctx();
  ctx->cfg = c;
  ctx->st = static_cast<cudaStream_t>(stream);
  if (!ctx->st) {
    // graphs cannot be captured on the legacy default stream: use a
    // blocking stream of our own, which stays ordered with the legacy one
    if (cudaStreamCreate(&ctx->st) != cudaSuccess) {
      delete ctx;
      return GEOFLOOD_ERR_CUDA;
    }
    ctx->own_stream = true;
  }
  ctx->nscen = c.num_scenarios;
  ctx->cap = c.max_patches;
  GfGeom& G = ctx->G;
  G.mi = c.mi; G.mj = c.mj; G.M = c.mx; G.T = c.mx + 2 * GF_NG;
  G.minlevel = c.minlevel; G.maxlevel = c.maxlevel;
  for (int k = 0; k < 4; ++k) G.bc[k] = c.bc[k];
  G.xlower = c.xlower; G.xupper = c.xupper; G.ylower = c.ylower; G.yupper = c.yupper;
  G.g = c.g; G.drytol = c.drytol;
  G.cfl_desired = c.cfl_desired; G.cfl_max = c.cfl_max; G.dt_max = c.dt_max;
  G.tag_depth = c.tag_depth; G.tag_speed = c.tag_speed; G.tag_deta = c.tag_deta;
  for (int k = 0; k < 4; ++k) G.src_box[k] = c.src_box[k];
  G.src_level = c.src_level;
  G.nscen = c.num_scenarios;
  long long acc = 0;
  for (int L = 0; L <= GF_MAXLEV; ++L) {
    G.lut_lev_off[L] = acc;
    if (L <= c.maxlevel) acc += ((long long)c.mi << L) * ((long long)c.mj << L);
  }
  G.lut_per_scen = acc;
  for (int L = 0; L <= GF_MAXLEV; ++L) {
    const double nx = (double)((long long)c.mi * c.mx << L);
    const double ny = (double)((long long)c.mj * c.mx << L);
    G.dxl[L] = (c.xupper - c.xlower) / nx;
    G.dyl[L] = (c.yupper - c.ylower) / ny;
    G.areal[L] = G.dxl[L] * G.dyl[L];
    G.inv_dxf[L] = (float)(1.0 / G.dxl[L]);
    G.inv_dyf[L] = (float)(1.0 / G.dyl[L]);
  }
  G.gf = (float)c.g;
  G.drytolf = (float)c.drytol;
  G.marginf = (float)(c.drytol * 0x1p-20);
  G.tag_depthf = (float)c.tag_depth;
  G.tag_speedf = (float)c.tag_speed;
  G.tag_detaf = (float)c.tag_deta;
  G.tag_flux = c.tag_flux;
  G.tag_fluxf = (float)c.tag_flux;
  G.ngrades = c.ngrades;
  for (int k = 0; k < 4; ++k) {
    G.grade_kind[k] = c.grade_kind[k];
    G.grade_level[k] = c.grade_level[k];
    G.grade_value[k] = c.grade_value[k];
    G.grade_valuef[k] = (float)c.grade_value[k];
  }
  G.first_order = c.first_order;
  G.no_transverse = c.no_transverse;
  G.dim_split = c.dim_split;
  G.subcycle = c.subcycle && c.maxlevel > c.minlevel ? 1 : 0;
  G.sub_K = G.subcycle ? 1 << (c.maxlevel - c.minlevel) : 1;
  G.nregions = c.nregions;
  for (int k = 0; k < GF_MAXREGION; ++k) {
    const bool on = k < c.nregions;
    G.rminl[k] = on ? c.region_minlevel[k] : 0;
    G.rmaxl[k] = on ? c.region_maxlevel[k] : 0;
    G.rx0[k] = on ? c.region_x0[k] : 0.0;
    G.rx1[k] = on ? c.region_x1[k] : 0.0;
    G.ry0[k] = on ? c.region_y0[k] : 0.0;
    G.ry1[k] = on ? c.region_y1[k] : 0.0;
    G.rt0[k] = on ? c.region_t0[k] : 0.0;
    G.rt1[k] = on ? c.region_t1[k] : 0.0;
  }
  G.n_hydro = c.n_hydro;
  G.inflow_side = c.inflow_side;
  G.inflow_lo = c.inflow_lo;
  G.inflow_hi = c.inflow_hi;
  G.inflow_tau = c.inflow_tau;
  for (int k = 0; k < 16; ++k) {
    G.hydro_t[k] = k < c.n_hydro ? c.hydro_t[k] : 0.0;
    G.hydro_q[k] = k < c.n_hydro ? c.hydro_q[k] : 0.0;
  }
  // the segment's width at each level: its line centres times the cell size
  for (int L = 0; L <= GF_MAXLEV; ++L) {
    G.inflow_width[L] = 0.0;
    if (c.n_hydro <= 0 || L > c.maxlevel) continue;
    const bool xs = c.inflow_side <= 1;
    const long long N = (long long)(xs ? c.mj : c.mi) * c.mx << L;
    const double lo = xs ? c.ylower : c.xlower, hi = xs ? c.yupper : c.xupper;
    const double d = (hi - lo) / (double)N;
    long long J0 = (long long)std::floor((c.inflow_lo - lo) / d) - 1;
    long long J1 = (long long)std::ceil((c.inflow_hi - lo) / d) + 1;
    if (J0 < 0) J0 = 0;
    if (J1 > N - 1) J1 = N - 1;
    long long n = 0;
    for (long long J = J0; J <= J1; ++J) {
      const double ctr = lo + ((double)J + 0.5) * d;
      if (ctr >= c.inflow_lo && ctr <= c.inflow_hi) ++n;
    }
    G.inflow_width[L] = (double)n * d;
  }

  const size_t TT = (size_t)G.T * G.T;
  const size_t cap = (size_t)ctx->cap;
  auto alloc = [&](void** p, size_t bytes) -> bool {
    return cudaMalloc(p, bytes) == cudaSuccess;
  };
  bool okk = true;
  ctx->prec = c.precision == GEOFLOOD_FP32_DEV ? 1 : 0;
  const size_t MM = (size_t)G.M * G.M;
  if (ctx->prec) {
    okk &= alloc((void**)&ctx->qf[0], cap * 3 * TT * sizeof(float));
    okk &= alloc((void**)&ctx->qf[1], cap * 3 * TT * sizeof(float));
    okk &= alloc((void**)&ctx->bf[0], cap * TT * sizeof(float));
    okk &= alloc((void**)&ctx->bf[1], cap * TT * sizeof(float));
    okk &= alloc((void**)&ctx->lof[0], cap * 3 * MM * sizeof(float));
    okk &= alloc((void**)&ctx->lof[1], cap * 3 * MM * sizeof(float));
  } else {
    okk &= alloc((void**)&ctx->q[0], cap * 3 * TT * sizeof(double));
    okk &= alloc((void**)&ctx->q[1], cap * 3 * TT * sizeof(double));
    okk &= alloc((void**)&ctx->b[0], cap * TT * sizeof(double));
    okk &= alloc((void**)&ctx->b[1], cap * TT * sizeof(double));
  }
  okk &= alloc((void**)&ctx->d_patch[0], cap * sizeof(GfPatch));
  okk &= alloc((void**)&ctx->d_patch[1], cap * sizeof(GfPatch));
  okk &= alloc((void**)&ctx->d_nbr[0], cap * 8 * sizeof(int));
  okk &= alloc((void**)&ctx->d_nbr[1], cap * 8 * sizeof(int));
  okk &= alloc((void**)&ctx->d_pbox[0], cap * sizeof(unsigned));
  okk &= alloc((void**)&ctx->d_pbox[1], cap * sizeof(unsigned));
  okk &= alloc((void**)&ctx->d_done, sizeof(unsigned));
  okk &= alloc((void**)&ctx->d_sched, 8 * sizeof(unsigned));
  okk &= alloc((void**)&ctx->d_ord[0], cap * sizeof(int));
  okk &= alloc((void**)&ctx->d_ord[1], cap * sizeof(int));
  okk &= alloc((void**)&ctx->d_same, cap * 4);
  okk &= alloc((void**)&ctx->d_runf, cap * 2);
  okk &= alloc((void**)&ctx->d_pwet, cap * sizeof(unsigned));
  okk &= alloc((void**)&ctx->d_gflag, cap);
  okk &= alloc((void**)&ctx->d_pcnt, cap * sizeof(unsigned));
  okk &= alloc((void**)&ctx->d_rlist, cap * sizeof(int));
  okk &= alloc((void**)&ctx->d_rpairs, cap * 2 * sizeof(int));
  okk &= alloc((void**)&ctx->d_glist[0], cap * 8 * sizeof(int));
  okk &= alloc((void**)&ctx->d_glist[1], cap * 8 * sizeof(int));
  okk &= alloc((void**)&ctx->d_ilist[0], cap * sizeof(int));
  okk &= alloc((void**)&ctx->d_ilist[1], cap * sizeof(int));
  okk &= alloc((void**)&ctx->d_lut[0], (size_t)ctx->nscen * G.lut_per_scen * sizeof(int));
  okk &= alloc((void**)&ctx->d_lut[1], (size_t)ctx->nscen * G.lut_per_scen * sizeof(int));
  okk &= alloc((void**)&ctx->d_scen, ctx->nscen * sizeof(GfScenario));
  okk &= alloc((void**)&ctx->d_ctl, ctx->nscen * sizeof(GfCtl));
  okk &= alloc((void**)&ctx->d_pmass, cap * sizeof(double));  // per patch (geoflood_mass)
  okk &= alloc((void**)&ctx->d_smass, ctx->nscen * sizeof(double));
  okk &= alloc((void**)&ctx->d_flags, cap);
  okk &= alloc((void**)&ctx->d_err, sizeof(int));
  okk &= cudaMallocHost((void**)&ctx->h_ctl, ctx->nscen * sizeof(GfCtl)) == cudaSuccess;
  okk &= cudaMallocHost((void**)&ctx->h_rb, 2 * sizeof(int)) == cudaSuccess;
  {
    // bed tiles by position: every patch position of every level, when that
    // fits the budget (else beds are always recomputed from the DEMs)
    const size_t slots = (size_t)ctx->nscen * G.lut_per_scen;
    const size_t bytes = slots * TT * (ctx->prec ? sizeof(float) : sizeof(double));
    if (okk && bytes <= kBedCacheBudget) {
      if (cudaMalloc(&ctx->d_bcache, bytes) != cudaSuccess ||
          cudaMalloc((void**)&ctx->d_bvalid, slots) != cudaSuccess ||
          cudaMemsetAsync(ctx->d_bvalid, 0, slots, ctx->st) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->d_bcache);
        cudaFree(ctx->d_bvalid);
        ctx->d_bcache = nullptr;
        ctx->d_bvalid = nullptr;
      }
    }
  }
  if (!okk) {
    cudaGetLastError();
    geoflood_destroy(ctx);
    return GEOFLOOD_ERR_OOM;
  }
  ctx->h_scen.assign(ctx->nscen, GfScenario{});
  ctx->d_dem.assign(ctx->nscen, std::vector<double*>());
  ctx->d_gxy.assign(ctx->nscen, nullptr);
  ctx->d_gout.assign(ctx->nscen, nullptr);
  ctx->d_garr.assign(ctx->nscen, nullptr);
  ctx->d_gref.assign(ctx->nscen, nullptr);
  for (int s = 0; s < ctx->nscen; ++s) {
    ctx->h_scen[s].lut_off = (long long)s * G.lut_per_scen;
    ctx->forests.emplace_back(c.mi, c.mj, c.minlevel, c.maxlevel);
    ctx->forests.back().uniform(c.minlevel);
  }
  std::memset(ctx->h_ctl, 0, sizeof(GfCtl) * ctx->nscen);
  for (int s = 0; s < ctx->nscen; ++s) ctx->h_ctl[s].dt_next = c.dt_initial;
  int rc = 0;
  do {
    const size_t qbytes = cap * 3 * TT * (ctx->prec ? sizeof(float) : sizeof(double));
    void* q0 = ctx->prec ? (void*)ctx->qf[0] : (void*)ctx->q[0];
    void* q1 = ctx->prec ? (void*)ctx->qf[1] : (void*)ctx->q[1];
    if (cudaMemsetAsync(q0, 0, qbytes, ctx->st) ||
        cudaMemsetAsync(q1, 0, qbytes, ctx->st) ||
        (ctx->prec && (cudaMemsetAsync(ctx->lof[0], 0, cap * 3 * MM * sizeof(float), ctx->st) ||
                       cudaMemsetAsync(ctx->lof[1], 0, cap * 3 * MM * sizeof(float), ctx->st))) ||
        cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->st) ||
        cudaMemsetAsync(ctx->d_done, 0, sizeof(unsigned), ctx->st)) {
      rc = GEOFLOOD_ERR_CUDA;
      break;
    }
    std::vector<std::vector<gf::Leaf>> lv;
    for (auto& f : ctx->forests) lv.push_back(f.leaves());
    if ((rc = upload_tables(ctx, 0, lv))) break;
    ctx->npatch = 0;
    for (auto& v : lv) ctx->npatch += (int)v.size();
    if ((rc = sync_ctl_up(ctx))) break;
    for (int s = 0; s < ctx->nscen && !rc; ++s) rc = topo_scenario(ctx, s);
    if (rc) break;
    rc = ghost_fill_all(ctx);
  } while (0);
  if (rc) {
    geoflood_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return GEOFLOOD_OK;
}

void geoflood_destroy(geoflood_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->st);
  for (int k = 0; k < 2; ++k) {
    cudaFree(ctx->q[k]);
    cudaFree(ctx->b[k]);
    cudaFree(ctx->qf[k]);
    cudaFree(ctx->bf[k]);
    cudaFree(ctx->lof[k]);
    cudaFree(ctx->d_patch[k]);
    cudaFree(ctx->d_lut[k]);
    cudaFree(ctx->d_nbr[k]);
    cudaFree(ctx->d_pbox[k]);
  }
  for (auto& gr : ctx->graphs)
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
  cudaFree(ctx->d_done);
  cudaFree(ctx->d_sched);
  cudaFree(ctx->d_ord[0]);
  cudaFree(ctx->d_ord[1]);
  cudaFree(ctx->d_same);
  cudaFree(ctx->d_runf);
  cudaFree(ctx->d_pwet);
  cudaFree(ctx->d_gflag);
  cudaFree(ctx->d_pcnt);
  cudaFree(ctx->d_rlist);
  cudaFree(ctx->d_rpairs);
  cudaFree(ctx->d_glist[0]);
  cudaFree(ctx->d_glist[1]);
  cudaFree(ctx->d_ilist[0]);
  cudaFree(ctx->d_ilist[1]);
  cudaFree(ctx->d_scen);
  cudaFree(ctx->d_ctl);
  cudaFree(ctx->d_pmass);
  cudaFree(ctx->d_smass);
  cudaFree(ctx->d_flags);
  cudaFree(ctx->d_err);
  cudaFree(ctx->d_stage);
  cudaFree(ctx->d_bcache);
  cudaFree(ctx->d_bvalid);
  for (auto& v : ctx->d_dem)
    for (auto p : v) cudaFree(p);
  for (auto p : ctx->d_gxy) cudaFree(p);
  for (auto p : ctx->d_gout) cudaFree(p);
  for (auto p : ctx->d_garr) cudaFree(p);
  for (auto p : ctx->d_gref) cudaFree(p);
  if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
  if (ctx->h_rb) cudaFreeHost(ctx->h_rb);
  if (ctx->up_pending) cudaEventSynchronize(ctx->up_ev);
  if (ctx->h_up) cudaFreeHost(ctx->h_up);
  if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
  if (ctx->up_ev) cudaEventDestroy(ctx->up_ev);
  if (ctx->own_stream) cudaStreamDestroy(ctx->st);
  for (auto e : ctx->pool) cudaEventDestroy(e);
  CnnState& n = ctx->cnn;
  for (void* p : {(void*)n.prm, n.wb, n.wf, (void*)n.grad, (void*)n.am, (void*)n.av, n.x,
                  n.a[0], n.a[1], n.a[2], (void*)n.pool, (void*)n.logit, n.px, (void*)n.py,
                  n.dx, (void*)n.dy, n.xb, (void*)n.yb, (void*)n.idx, n.ta[0], n.ta[1],
                  n.ta[2], n.td[0], n.td[1], n.td[2], (void*)n.tv, (void*)n.tlogit,
                  (void*)n.loss, (void*)n.misses})
    cudaFree(p);
  delete ctx;
}

const char* geoflood_last_error(const geoflood_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

// In the deviation form the stored surface w = h + b - eta0 depends on the
// bed and eta0: changing either keeps the depths by reading them out before
// and writing them back after.
static int keep_depths(geoflood_ctx* ctx, int s, std::vector<double>& h,
                       std::vector<double>& hu, std::vector<double>& hv) {
  const size_t plane = (size_t)ctx->h_scen[s].pcount * ctx->G.M * ctx->G.M;
  h.resize(plane);
  hu.resize(plane);
  hv.resize(plane);
  return geoflood_read_patches(ctx, s, h.data(), hu.data(), hv.data(), nullptr);
}

int geoflood_set_scenario(geoflood_ctx* ctx, int s, double manning_n,
                          double eta0) {
  if (!valid_scen(ctx, s) || !(manning_n >= 0))
    return fail(ctx, GEOFLOOD_ERR_ARG, "set_scenario: bad argument");
  std::vector<double> h, hu, hv;
  int rc = 0;
  const bool moved = ctx->prec && eta0 != ctx->h_scen[s].eta0;
  if (moved && (rc = keep_depths(ctx, s, h, hu, hv))) return rc;
  ctx->h_scen[s].manning_n = manning_n;
  ctx->h_scen[s].manning_f = (float)manning_n;
  ctx->h_scen[s].eta0 = eta0;
  if ((rc = upload_scen(ctx))) return rc;
  if (!moved) return 0;
  if ((rc = topo_scenario(ctx, s))) return rc;
  return geoflood_write_patches(ctx, s, h.data(), hu.data(), hv.data());
}

int geoflood_set_topos(geoflood_ctx* ctx, int s, int ndem, const double* const* z,
                       const int* nx, const int* ny, const double* x0,
                       const double* y0, const double* dx, const double* dy) {
  if (!valid_scen(ctx, s) || ndem < 1 || ndem > GF_MAXDEM || !z || !nx || !ny || !x0 ||
      !y0 || !dx || !dy)
    return fail(ctx, GEOFLOOD_ERR_ARG, "set_topo: bad argument");
  for (int k = 0; k < ndem; ++k)
    if (!z[k] || nx[k] < 2 || ny[k] < 2 || !(dx[k] > 0) || !(dy[k] > 0) ||
        !std::isfinite(x0[k]) || !std::isfinite(y0[k]) || !std::isfinite(dx[k]) ||
        !std::isfinite(dy[k]))
      return fail(ctx, GEOFLOOD_ERR_ARG, "set_topo: bad DEM " + std::to_string(k));
  // priority: finer node spacing (dx * dy) first, equal spacings in the
  // given order
  int ord[GF_MAXDEM];
  for (int k = 0; k < ndem; ++k) ord[k] = k;
  for (int i = 1; i < ndem; ++i)
    for (int j = i; j > 0 && dx[ord[j]] * dy[ord[j]] < dx[ord[j - 1]] * dy[ord[j - 1]]; --j)
      std::swap(ord[j], ord[j - 1]);
  std::vector<double> h, hu, hv;
  int rc = 0;
  if (ctx->prec && (rc = keep_depths(ctx, s, h, hu, hv))) return rc;
  for (auto p : ctx->d_dem[s]) cudaFree(p);
  ctx->d_dem[s].clear();
  GfScenario& S = ctx->h_scen[s];
  S.ndem = 0;
  for (int r = 0; r < ndem; ++r) {
    const int k = ord[r];
    const size_t n = (size_t)nx[k] * ny[k];
    double* d = nullptr;
    if (cudaMalloc(&d, n * sizeof(double)) != cudaSuccess) {
      for (auto p : ctx->d_dem[s]) cudaFree(p);
      ctx->d_dem[s].clear();
      upload_scen(ctx);
      return fail(ctx, GEOFLOOD_ERR_OOM, "set_topo: DEM allocation");
    }
    ctx->d_dem[s].push_back(d);
    CK(cudaMemcpyAsync(d, z[k], n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    S.dem[r] = d;
    S.dnx[r] = nx[k]; S.dny[r] = ny[k];
    S.dx0[r] = x0[k]; S.dy0[r] = y0[k]; S.ddx[r] = dx[k]; S.ddy[r] = dy[k];
  }
  S.ndem = ndem;
  rc = upload_scen(ctx);
  if (rc) return rc;
  if ((rc = topo_scenario(ctx, s))) return rc;
  if (ctx->prec) return geoflood_write_patches(ctx, s, h.data(), hu.data(), hv.data());
  return ghost_fill_all(ctx);
}

int geoflood_set_topo(geoflood_ctx* ctx, int s, const double* z, int nx,
                      int ny, double x0, double y0, double dx, double dy) {
  const double* zz[1] = {z};
  return geoflood_set_topos(ctx, s, 1, zz, &nx, &ny, &x0, &y0, &dx, &dy);
}

int geoflood_npatch(geoflood_ctx* ctx, int s, int* np) {
  if (!valid_scen(ctx, s) || !np) return fail(ctx, GEOFLOOD_ERR_ARG, "npatch: bad argument");
  *np = ctx->h_scen[s].pcount;
  return 0;
}

int geoflood_patch_info(geoflood_ctx* ctx, int s, int* level, int* px,
                        int* py) {
  if (!valid_scen(ctx, s)) return fail(ctx, GEOFLOOD_ERR_ARG, "patch_info: bad scenario");
  const auto& lv = ctx->forests[s].leaves();
  for (size_t k = 0; k < lv.size(); ++k) {
    if (level) level[k] = lv[k].level;
    if (px) px[k] = lv[k].px;
    if (py) py[k] = lv[k].py;
  }
  return 0;
}

int geoflood_write_patches(geoflood_ctx* ctx, int s, const double* h,
                           const double* hu, const double* hv) {
  if (!valid_scen(ctx, s) || !h || !hu || !hv)
    return fail(ctx, GEOFLOOD_ERR_ARG, "write_patches: bad argument");
  const int n = ctx->h_scen[s].pcount;
  const size_t plane = (size_t)n * ctx->G.M * ctx->G.M;
  int rc = ensure_stage(ctx, 4 * plane);
  if (rc) return rc;
  if ((rc = sync_ctl_down(ctx))) return rc;
  CK(cudaMemcpyAsync(ctx->d_stage, h, plane * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->d_stage + plane, hu, plane * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->d_stage + 2 * plane, hv, plane * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  if ((rc = forget_same(ctx))) return rc;
  CKL(gf::launch_unpack_interior(ctx->G, view(ctx), ctx->h_scen[s].poff, n,
                                 ctx->d_stage, ctx->h_ctl[s].cur, ctx->st),
      "unpack");
  ctx->launches++;
  ctx->h_ctl[s].status = 0;
  ctx->h_ctl[s].nonfinite = 0;
  ctx->h_ctl[s].accepted = 0;  // the state is not a step result
  if ((rc = sync_ctl_up(ctx))) return rc;
  return ghost_fill_all(ctx);
}

int geoflood_read_patches(geoflood_ctx* ctx, int s, double* h, double* hu,
                          double* hv, double* b) {
  if (!valid_scen(ctx, s)) return fail(ctx, GEOFLOOD_ERR_ARG, "read_patches: bad scenario");
  const int n = ctx->h_scen[s].pcount;
  const size_t plane = (size_t)n * ctx->G.M * ctx->G.M;
  int rc = ensure_stage(ctx, 4 * plane);
  if (rc) return rc;
  if ((rc = sync_ctl_down(ctx))) return rc;
  CKL(gf::launch_pack_interior(ctx->G, view(ctx), ctx->h_scen[s].poff, n,
                               ctx->d_stage, 15, ctx->h_ctl[s].cur, ctx->st),
      "pack");
  ctx->launches++;
  double* dst[4] = {h, hu, hv, b};
  for (int f = 0; f < 4; ++f)
    if (dst[f])
      CK(cudaMemcpyAsync(dst[f], ctx->d_stage + f * plane, plane * sizeof(double),
                         cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int geoflood_read_tiles(geoflood_ctx* ctx, int s, double* out) {
  if (!valid_scen(ctx, s) || !out) return fail(ctx, GEOFLOOD_ERR_ARG, "read_tiles: bad argument");
  int rc = sync_ctl_down(ctx);
  if (rc) return rc;
  const size_t TT = (size_t)ctx->G.T * ctx->G.T;
  const int off = ctx->h_scen[s].poff, n = ctx->h_scen[s].pcount;
  const int cur = ctx->h_ctl[s].cur;
  if (!ctx->prec) {
    for (int k = 0; k < n; ++k) {
      CK(cudaMemcpyAsync(out + (size_t)k * 4 * TT, ctx->q[cur] + (size_t)(off + k) * 3 * TT,
                         3 * TT * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
      CK(cudaMemcpyAsync(out + (size_t)k * 4 * TT + 3 * TT,
                         ctx->b[ctx->bsel] + (size_t)(off + k) * TT,
                         TT * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    }
    CK(cudaStreamSynchronize(ctx->st));
    return 0;
  }
  // deviation form: h = w - b exactly, b = (b - eta0) + eta0
  std::vector<float> qh((size_t)n * 3 * TT), bh((size_t)n * TT);
  CK(cudaMemcpyAsync(qh.data(), ctx->qf[cur] + (size_t)off * 3 * TT,
                     qh.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(bh.data(), ctx->bf[ctx->bsel] + (size_t)off * TT,
                     bh.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  const double e0 = ctx->h_scen[s].eta0;
  for (int k = 0; k < n; ++k)
    for (size_t c = 0; c < TT; ++c) {
      const double b = (double)bh[(size_t)k * TT + c];
      double* o = out + (size_t)k * 4 * TT;
      o[c] = (double)qh[(size_t)k * 3 * TT + c] - b;
      o[TT + c] = (double)qh[(size_t)k * 3 * TT + TT + c];
      o[2 * TT + c] = (double)qh[(size_t)k * 3 * TT + 2 * TT + c];
      o[3 * TT + c] = b + e0;
    }
  return 0;
}

int geoflood_set_state(geoflood_ctx* ctx, int s, geoflood_qinit_fn fn,
                       void* user) {
  if (!valid_scen(ctx, s) || !fn) return fail(ctx, GEOFLOOD_ERR_ARG, "set_state: bad argument");
  const int n = ctx->h_scen[s].pcount, M = ctx->G.M;
  const size_t plane = (size_t)n * M * M;
  std::vector<double> x(plane), y(plane), bb(plane), h(plane), hu(plane), hv(plane);
  int rc = geoflood_read_patches(ctx, s, nullptr, nullptr, nullptr, bb.data());
  if (rc) return rc;
  const auto& lv = ctx->forests[s].leaves();
  for (int k = 0; k < n; ++k) {
    const int L = lv[k].level;
    const double dx = (ctx->G.xupper - ctx->G.xlower) / (double)((long long)ctx->G.mi * M << L);
    const double dy = (ctx->G.yupper - ctx->G.ylower) / (double)((long long)ctx->G.mj * M << L);
    for (int j = 0; j < M; ++j)
      for (int i = 0; i < M; ++i) {
        const size_t o = (size_t)k * M * M + (size_t)j * M + i;
        x[o] = ctx->G.xlower + ((double)((long long)lv[k].px * M + i) + 0.5) * dx;
        y[o] = ctx->G.ylower + ((double)((long long)lv[k].py * M + j) + 0.5) * dy;
      }
  }
  fn((int)plane, x.data(), y.data(), bb.data(), h.data(), hu.data(), hv.data(), user);
  return geoflood_write_patches(ctx, s, h.data(), hu.data(), hv.data());
}

int geoflood_set_time(geoflood_ctx* ctx, int s, double t, double dt_next) {
  if (!valid_scen(ctx, s) || !(dt_next > 0)) return fail(ctx, GEOFLOOD_ERR_ARG, "set_time: bad argument");
  int rc = sync_ctl_down(ctx);
  if (rc) return rc;
  ctx->h_ctl[s].t = t;
  ctx->h_ctl[s].dt_next = dt_next;
  ctx->h_ctl[s].status = 0;
  ctx->h_ctl[s].accepted = 0;  // no step result for the next step to sample
  return sync_ctl_up(ctx);
}

int geoflood_get_time(geoflood_ctx* ctx, int s, double* t, double* dt_next,
                      long long* steps, long long* rejects, long long* nclip,
                      double* clipvol) {
  if (!valid_scen(ctx, s)) return fail(ctx, GEOFLOOD_ERR_ARG, "get_time: bad scenario");
  int rc = sync_ctl_down(ctx);
  if (rc) return rc;
  const GfCtl& C = ctx->h_ctl[s];
  if (t) *t = C.t;
  if (dt_next) *dt_next = C.dt_next;
  if (steps) *steps = C.steps;
  if (rejects) *rejects = C.rejects;
  if (nclip) *nclip = C.nclip;
  if (clipvol) *clipvol = C.clipvol;
  return 0;
}

// The steps of geoflood_step; with misses non-null the plain criterion's
// check (geoflood_check_tags's count) also runs on the final state, inside
// the same readback.  Each graph launch is followed by the gauges' sample of
// its final state and one readback of the controllers, the device error flag
// and the check's count (one host wait per launch).  A sample taken before a
// retake is one the next step takes again at its start.
static int step_core(geoflood_ctx* ctx, double t_target, int max_steps, double* t_out,
                     int* steps_out, int* misses) {
  if (!ctx || max_steps < 0) return fail(ctx, GEOFLOOD_ERR_ARG, "step: bad argument");
  CKL(gf::launch_ctl_begin(ctx->d_ctl, ctx->nscen, t_target, max_steps,
                           nullptr, ctx->st),
      "ctl_begin");
  ctx->launches++;
  gf::set_errflag(ctx->d_err);
  const GfView v = view(ctx);
  // The steps run in chunks of K captured as one CUDA graph (patch step with
  // the fused CFL controller, ghost fill, gauges); the device controller
  // deactivates a scenario when it reaches t_target or max_steps accepted
  // steps, after which its patches return at once.  Rejected steps need
  // extra launches, bounded by the controller's limit on rejections in a row.
  const int K = std::max(1, std::min(16, max_steps));
  geoflood_ctx::Graph* gr = nullptr;
  for (auto& c : ctx->graphs)
    if (c.k == K) gr = &c;
  if (!gr) {
    ctx->graphs.emplace_back();
    gr = &ctx->graphs.back();
    gr->k = K;
  }
  const int prof = ctx->prof ? ctx->prof_every : 0;
  if (!gr->exec || gr->generation != ctx->generation || gr->tsel != ctx->tsel ||
      gr->bsel != ctx->bsel ||
      gr->npatch != ctx->npatch || gr->gauges != ctx->max_gauges_used ||
      gr->prof != prof || gr->variant != ctx->variant) {
    gr->ev.clear();
    gr->evg.clear();
    CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
    int lrc = 0;
    for (int it = 0; it < K && !lrc; ++it) {
      // sampled launches are bracketed by external event-record nodes (the
      // events are recorded at every replay)
      const bool sample = prof && it % prof == 0;
      ProfRec r{}, rg{};
      if (sample) {
        r.a = pool_event(ctx);
        r.b = pool_event(ctx);
        rg.a = pool_event(ctx);
        rg.b = pool_event(ctx);
        cudaEventRecordWithFlags(r.a, ctx->st, cudaEventRecordExternal);
      }
      // one step, or with level subcycling the sub_K substeps of a macro
      // step (the patches of level minlevel synchronised after the last)
      for (int sub = 0; sub < ctx->G.sub_K && !lrc; ++sub) {
        if (sample && sub > 0) {
          r.a = pool_event(ctx);
          r.b = pool_event(ctx);
          rg.a = pool_event(ctx);
          rg.b = pool_event(ctx);
          cudaEventRecordWithFlags(r.a, ctx->st, cudaEventRecordExternal);
        }
        lrc |= ctx->prec ? gf::launch_patch_step_f32(ctx->G, v, ctx->variant, ctx->st)
                         : gf::launch_patch_step_f64(ctx->G, v, ctx->variant, ctx->st);
        if (sample) {
          cudaEventRecordWithFlags(r.b, ctx->st, cudaEventRecordExternal);
          r.cells = (long long)ctx->npatch * ctx->G.M * ctx->G.M;
          gr->ev.push_back(r);
          cudaEventRecordWithFlags(rg.a, ctx->st, cudaEventRecordExternal);
        }
        if (sub == ctx->G.sub_K - 1) lrc |= gf::launch_subcycle_sync(ctx->G, v, ctx->st);
        lrc |= gf::launch_ghost_rest(ctx->G, v, ctx->d_glist[ctx->tsel],
                                     ctx->nglist_c[ctx->tsel], ctx->nglist[ctx->tsel],
                                     ctx->st);
        lrc |= gf::launch_inflow(ctx->G, v, ctx->d_ilist[ctx->tsel], ctx->nilist[ctx->tsel], 1,
                                 ctx->st);
        if (sample) {
          cudaEventRecordWithFlags(rg.b, ctx->st, cudaEventRecordExternal);
          gr->evg.push_back(rg);
        }
      }
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(ctx->st, &graph);
    if (lrc || ce != cudaSuccess)
      return fail(ctx, GEOFLOOD_ERR_CUDA, std::string("step: graph capture failed: ") +
                                              cudaGetErrorString(ce != cudaSuccess ? ce : cudaGetLastError()));
    // after a regrid only the kernels' parameters and grids change: update
    // the executable graph in place when its shape allows, else instantiate
    bool updated = false;
    if (gr->exec) {
      cudaGraphExecUpdateResultInfo info{};
      updated = cudaGraphExecUpdate(gr->exec, graph, &info) == cudaSuccess;
      if (!updated) {
        cudaGetLastError();
        cudaGraphExecDestroy(gr->exec);
        gr->exec = nullptr;
      }
    }
    if (!updated) ce = cudaGraphInstantiate(&gr->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess)
      return fail(ctx, GEOFLOOD_ERR_CUDA, std::string("step: graph instantiation failed: ") +
                                              cudaGetErrorString(ce));
    gr->tsel = ctx->tsel;
    gr->bsel = ctx->bsel;
    gr->npatch = ctx->npatch;
    gr->gauges = ctx->max_gauges_used;
    gr->prof = prof;
    gr->variant = ctx->variant;
    gr->generation = ctx->generation;
  }
  const int per_step = ctx->G.sub_K * (1 + (ctx->nglist[ctx->tsel] > 0 ? 1 : 0) +
                                       (ctx->nilist[ctx->tsel] > 0 ? 1 : 0)) +
                       (ctx->G.subcycle ? 1 : 0);
  long long launched = 0;
  const long long limit = (long long)max_steps * 2 + 64;
  unsigned* d_misses = nullptr;
  if (misses) {
    int rc = cnn_alloc(ctx, (void**)&ctx->cnn.misses, sizeof(unsigned));
    if (rc) return rc;
    d_misses = ctx->cnn.misses;
  }
  // the final-state work after a graph launch, then one host wait
  auto finish = [&]() -> int {
    if (ctx->max_gauges_used > 0) {
      CKL(gf::launch_gauges(ctx->G, v, 0, ctx->max_gauges_used, ctx->st), "gauges");
      ctx->launches++;
    }
    if (d_misses) {
      CK(cudaMemsetAsync(d_misses, 0, sizeof(unsigned), ctx->st));
      int rc = tag_pass(ctx, false, d_misses);
      if (rc) return rc;
      CK(cudaMemcpyAsync(ctx->h_rb + 1, d_misses, sizeof(unsigned), cudaMemcpyDeviceToHost,
                         ctx->st));
    }
    CK(cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, sizeof(GfCtl) * ctx->nscen,
                       cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(ctx->h_rb, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (ctx->h_rb[0]) {
      CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->st));
      return fail(ctx, GEOFLOOD_ERR_STATE,
                  "forest lookup failed (unbalanced or uncovered forest)");
    }
    return 0;
  };
  bool finished = false;
  while (max_steps > 0) {
    CK(cudaGraphLaunch(gr->exec, ctx->st));
    ctx->launches += (long long)K * per_step;
    launched += K;
    int rc = finish();
    if (rc) return rc;
    finished = true;
    if (prof) {
      for (auto& r : gr->ev) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        ctx->prof_ms["patch_step"] += ms;
        ctx->prof_n["patch_step"] += 1;
        ctx->prof_cells["patch_step"] += r.cells;
      }
      for (auto& r : gr->evg) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        ctx->prof_ms["ghost_fill"] += ms;
        ctx->prof_n["ghost_fill"] += 1;
      }
    }
    bool any = false;
    for (int s = 0; s < ctx->nscen; ++s) any |= ctx->h_ctl[s].active != 0;
    if (!any) break;
    if (launched > limit) return fail(ctx, GEOFLOOD_ERR_CFL, "step: too many retakes");
  }
  if (!finished) {
    int rc = finish();
    if (rc) return rc;
  }
  if (misses) *misses = ctx->h_rb[1];
  int status = 0;
  for (int s = 0; s < ctx->nscen; ++s) {
    const GfCtl& C = ctx->h_ctl[s];
    if (t_out) t_out[s] = C.t;
    if (steps_out) steps_out[s] = (int)C.taken;
    if (C.status && !status) status = C.status;
  }
  if (status == GEOFLOOD_ERR_NAN) return fail(ctx, status, "non-finite value in the state");
  if (status == GEOFLOOD_ERR_CFL) return fail(ctx, status, "too many rejected steps in a row");
  if (status == GEOFLOOD_ERR_TIMEOUT) return fail(ctx, status, "bounded device wait expired");
  if (status) return fail(ctx, status, "device error");
  return 0;
}

int geoflood_step(geoflood_ctx* ctx, double t_target, int max_steps,
                  double* t_out, int* steps_out) {
  return step_core(ctx, t_target, max_steps, t_out, steps_out, nullptr);
}

int geoflood_tags(geoflood_ctx* ctx, int s, uint8_t* flags) {
  if (!valid_scen(ctx, s) || !flags) return fail(ctx, GEOFLOOD_ERR_ARG, "tags: bad argument");
  int rc = tag_pass(ctx, ctx->cnn.tagger == GEOFLOOD_TAGGER_LEARNED, nullptr);
  if (rc) return rc;
  CK(cudaMemcpyAsync(flags, ctx->d_flags + ctx->h_scen[s].poff,
                     ctx->h_scen[s].pcount, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

}  // extern "C"

namespace {

// A regrid; with misses non-null its tag pass also counts what the plain
// criterion wants refined below the finest level (geoflood_check_tags's
// count), so that a check due together with a regrid needs no pass of its
// own.
int regrid_impl(geoflood_ctx* ctx, int* misses) {
  if (!ctx) return GEOFLOOD_ERR_ARG;
  int rc = sync_ctl_down(ctx);
  if (rc) return rc;
  if (!ctx->h_flags) {
    // the tags of every patch, then the miss count
    if (cudaMallocHost((void**)&ctx->h_flags, (size_t)ctx->cap + 16) != cudaSuccess) {
      cudaGetLastError();
      ctx->h_flags = nullptr;
      return fail(ctx, GEOFLOOD_ERR_OOM, "pinned tag buffer");
    }
    ctx->h_flags_cap = (size_t)ctx->cap;
  }
  const uint8_t* flags_h = ctx->h_flags;
  unsigned* miss_h = reinterpret_cast<unsigned*>(ctx->h_flags + ((ctx->h_flags_cap + 3) & ~size_t(3)));
  unsigned* miss_d = nullptr;
  if (misses) {
    if ((rc = cnn_alloc(ctx, (void**)&ctx->cnn.misses, sizeof(unsigned)))) return rc;
    miss_d = ctx->cnn.misses;
    CK(cudaMemsetAsync(miss_d, 0, sizeof(unsigned), ctx->st));
  }
  if ((rc = tag_pass(ctx, ctx->cnn.tagger == GEOFLOOD_TAGGER_LEARNED, miss_d))) return rc;
  CK(cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, ctx->npatch, cudaMemcpyDeviceToHost, ctx->st));
  if (misses)
    CK(cudaMemcpyAsync(miss_h, miss_d, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (misses) *misses = (int)*miss_h;
  // New forests, scenario by scenario (on several host threads when there
  // are many scenarios); a leaf present in both forests keeps its data
  // (copied from its old slot), a new one is computed from the old forest.
  std::vector<std::vector<gf::Leaf>> lv(ctx->nscen);
  std::vector<std::vector<int>> fresh_s(ctx->nscen), keep_s(ctx->nscen);
  std::vector<char> changed(ctx->nscen, 0);
  auto regrid_one = [&](int s) {
    const gf::HostForest& F = ctx->forests[s];
    const std::vector<gf::Leaf>& old = F.leaves();
    lv[s] = F.regrid(flags_h + ctx->h_scen[s].poff);
    // Both leaf lists are in Morton order of their lower-left corners, and
    // the leaves of one forest have distinct corners, so one merge pass
    // finds the leaves present in both (same corner and level).
    bool same = lv[s].size() == old.size();
    size_t o = 0;
    uint64_t ko = o < old.size() ? F.morton(old[o]) : ~0ull;
    for (size_t k = 0; k < lv[s].size(); ++k) {
      const gf::Leaf& l = lv[s][k];
      const uint64_t kn = F.morton(l);
      while (ko < kn) {
        ++o;
        ko = o < old.size() ? F.morton(old[o]) : ~0ull;
      }
      if (ko == kn && old[o].level == l.level) {
        keep_s[s].push_back((int)k);
        keep_s[s].push_back(ctx->h_scen[s].poff + (int)o);
        same = same && o == k;
      } else {
        fresh_s[s].push_back((int)k);
        same = false;
      }
    }
    changed[s] = same ? 0 : 1;
  };
  const auto t_host = std::chrono::steady_clock::now();
  const int nthreads = std::min(ctx->nscen, std::max(1, std::min(16, (int)std::thread::hardware_concurrency())));
  if (nthreads <= 1) {
    for (int s = 0; s < ctx->nscen; ++s) regrid_one(s);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t)
      pool.emplace_back([&, t]() {
        for (int s = t; s < ctx->nscen; s += nthreads) regrid_one(s);
      });
    for (auto& th : pool) th.join();
  }
  ctx->regrid_host_s +=
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_host).count();
  // nothing to do when no forest changed (the tables and graphs stay)
  bool any_change = false;
  for (int s = 0; s < ctx->nscen; ++s) any_change |= changed[s] != 0;
  if (!any_change) {
    for (int s = 0; s < ctx->nscen; ++s) ctx->forests[s].set_leaves(lv[s]);
    return 0;
  }
  size_t total = 0;
  std::vector<int> fresh;         // new slots computed from the old forest
  std::vector<int> keep;          // (new, old) slot pairs
  for (int s = 0; s < ctx->nscen; ++s) {
    const int off = (int)total;
    for (int k : fresh_s[s]) fresh.push_back(off + k);
    for (size_t k = 0; k < keep_s[s].size(); k += 2) {
      keep.push_back(off + keep_s[s][k]);
      keep.push_back(keep_s[s][k + 1]);
    }
    total += lv[s].size();
  }
  if ((long long)total > ctx->cap)
    return fail(ctx, GEOFLOOD_ERR_CAPACITY,
                "regrid needs " + std::to_string(total) + " patches, capacity is " +
                    std::to_string(ctx->cap));
  // every scenario's latest state into one buffer, so that the new slots
  // (written into the other buffer) overwrite no scenario's latest state:
  // slots are shared, and scenarios that took different numbers of steps
  // hold their latest state in different buffers
  {
    long long ones = 0, zeros = 0;
    for (int s = 0; s < ctx->nscen; ++s)
      (ctx->h_ctl[s].cur ? ones : zeros) += ctx->h_scen[s].pcount;
    const int target = ones > zeros ? 1 : 0;
    bool mixed = false;
    for (int s = 0; s < ctx->nscen; ++s) mixed |= ctx->h_ctl[s].cur != target;
    if (mixed) {
      CKL(gf::launch_align_buffers(ctx->G, view(ctx), target, ctx->st), "align_buffers");
      ctx->launches++;
      for (int s = 0; s < ctx->nscen; ++s) ctx->h_ctl[s].cur = target;
      if ((rc = sync_ctl_up(ctx))) return rc;
    }
  }
  const GfView oldv = view(ctx);
  std::vector<GfScenario> saved = ctx->h_scen;
  const int nt = ctx->tsel ^ 1, nb = ctx->bsel ^ 1;
  // one staging batch for the tables, the regrid lists and the controllers
  if ((rc = upload_begin(ctx, tables_room(ctx, total) +
                                  upload_room({sizeof(int) * fresh.size(),
                                               sizeof(int) * keep.size(),
                                               sizeof(GfCtl) * ctx->nscen}))))
    return rc;
  if ((rc = upload_tables(ctx, nt, lv, true))) {
    upload_end(ctx);
    ctx->h_scen = saved;
    upload_scen(ctx);
    return rc;
  }
  GfView newv = view(ctx, nt, nb);
  newv.npatch = (int)total;
  const int nfresh = (int)fresh.size(), nkeep = (int)keep.size() / 2;
  rc |= upload_put(ctx, ctx->d_rlist, fresh.data(), sizeof(int) * fresh.size());
  rc |= upload_put(ctx, ctx->d_rpairs, keep.data(), sizeof(int) * keep.size());
  if (rc) return rc;
  CKL(gf::launch_topo(ctx->G, newv, 0, nfresh, ctx->st, ctx->d_rlist), "topo");
  gf::set_errflag(ctx->d_err);
  CKL(gf::launch_regrid_fill(ctx->G, oldv, newv, ctx->st, ctx->d_rlist, nfresh), "regrid_fill");
  CKL(gf::launch_regrid_keep(ctx->G, oldv, newv, ctx->d_rpairs, nkeep, ctx->st), "regrid_keep");
  ctx->launches += 3;
  // the controllers after the regrid (stream-ordered behind the fills,
  // which read the old current buffer)
  for (int s = 0; s < ctx->nscen; ++s) {
    ctx->h_ctl[s].cur ^= 1;
    ctx->h_ctl[s].accepted = 0;  // gauges sample step results only
    ctx->forests[s].set_leaves(lv[s]);
  }
  if ((rc = upload_put(ctx, ctx->d_ctl, ctx->h_ctl, sizeof(GfCtl) * ctx->nscen))) return rc;
  if ((rc = upload_end(ctx))) return rc;
  ctx->tsel = nt;
  ctx->bsel = nb;
  ctx->npatch = (int)total;
  ctx->generation++;
  if (ctx->max_gauges_used > 0) {
    CKL(gf::launch_gauge_refs(ctx->G, view(ctx), ctx->max_gauges_used, ctx->st), "gauge_refs");
    ctx->launches++;
  }
  // one wait for the whole regrid: the ghost fill ends by reading the
  // lookup-error flag, which the fills above also set
  return ghost_fill_all(ctx);
}

}  // namespace

extern "C" {

int geoflood_regrid(geoflood_ctx* ctx) { return regrid_impl(ctx, nullptr); }

int geoflood_mass(geoflood_ctx* ctx, int s, double* mass) {
  if (!valid_scen(ctx, s) || !mass) return fail(ctx, GEOFLOOD_ERR_ARG, "mass: bad argument");
  CKL(gf::launch_mass(ctx->G, view(ctx), ctx->d_pmass, ctx->d_smass, ctx->nscen, ctx->st), "mass");
  ctx->launches += 2;
  CK(cudaMemcpyAsync(mass, ctx->d_smass + s, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int geoflood_set_gauges(geoflood_ctx* ctx, int s, const double* xy, int n) {
  if (!valid_scen(ctx, s) || n < 0 || n > ctx->cfg.max_gauges || (n > 0 && !xy))
    return fail(ctx, GEOFLOOD_ERR_ARG, "set_gauges: bad argument");
  cudaFree(ctx->d_gxy[s]);
  cudaFree(ctx->d_gout[s]);
  cudaFree(ctx->d_garr[s]);
  cudaFree(ctx->d_gref[s]);
  ctx->d_gxy[s] = ctx->d_gout[s] = ctx->d_garr[s] = nullptr;
  ctx->d_gref[s] = nullptr;
  const int m = n > 0 ? n : 1;
  CK(cudaMalloc(&ctx->d_gxy[s], 2 * m * sizeof(double)));
  CK(cudaMalloc(&ctx->d_gout[s], 5 * m * sizeof(double)));
  CK(cudaMalloc(&ctx->d_garr[s], m * sizeof(double)));
  CK(cudaMalloc(&ctx->d_gref[s], m * sizeof(GfGaugeRef)));
  if (n > 0)
    CK(cudaMemcpyAsync(ctx->d_gxy[s], xy, 2 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(ctx->d_gout[s], 0, 5 * m * sizeof(double), ctx->st));
  std::vector<double> neg(m, -1.0);
  CK(cudaMemcpyAsync(ctx->d_garr[s], neg.data(), m * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  GfScenario& S = ctx->h_scen[s];
  S.ngauge = n;
  S.gxy = ctx->d_gxy[s];
  S.gout = ctx->d_gout[s];
  S.garr = ctx->d_garr[s];
  S.gref = ctx->d_gref[s];
  int rc = upload_scen(ctx);
  if (rc) return rc;
  ctx->max_gauges_used = 0;
  for (auto& sc : ctx->h_scen) ctx->max_gauges_used = std::max(ctx->max_gauges_used, sc.ngauge);
  CK(cudaMemsetAsync(ctx->d_gflag, 0, (size_t)ctx->cap, ctx->st));
  CKL(gf::launch_gauge_refs(ctx->G, view(ctx), ctx->max_gauges_used, ctx->st), "gauge_refs");
  CKL(gf::launch_gauges(ctx->G, view(ctx), 0, ctx->max_gauges_used, ctx->st), "gauges");
  ctx->launches++;
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int geoflood_gauge_count(geoflood_ctx* ctx, int s, int* n) {
  if (!valid_scen(ctx, s) || !n) return fail(ctx, GEOFLOOD_ERR_ARG, "gauge_count: bad argument");
  *n = ctx->h_scen[s].ngauge;
  return 0;
}

int geoflood_gauges(geoflood_ctx* ctx, int s, double* out, double* arrival) {
  if (!valid_scen(ctx, s)) return fail(ctx, GEOFLOOD_ERR_ARG, "gauges: bad scenario");
  const int n = ctx->h_scen[s].ngauge;
  if (n > 0 && out)
    CK(cudaMemcpyAsync(out, ctx->d_gout[s], 5 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  if (n > 0 && arrival)
    CK(cudaMemcpyAsync(arrival, ctx->d_garr[s], n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int geoflood_profile(geoflood_ctx* ctx, int enable) {
  if (!ctx) return GEOFLOOD_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->st));
  ctx->prof_recs.clear();
  ctx->prof_ms.clear();
  ctx->prof_n.clear();
  ctx->prof_cells.clear();
  for (auto& gr : ctx->graphs) {  // their events come from the pool
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
    gr.exec = nullptr;
  }
  ctx->pool_used = 0;
  if (enable < 0) return fail(ctx, GEOFLOOD_ERR_ARG, "profile: enable must be >= 0");
  if (enable) pool_event(ctx), ctx->pool_used = 0;  // pre-create the pool
  ctx->prof = enable != 0;
  ctx->prof_every = enable > 0 ? enable : 1;
  return 0;
}

int geoflood_profile_read(geoflood_ctx* ctx, const char* kernel,
                          double* total_ms, long long* launches) {
  if (!ctx || !kernel) return GEOFLOOD_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->st));
  double tot = ctx->prof_ms.count(kernel) ? ctx->prof_ms[kernel] : 0.0;
  long long n = ctx->prof_n.count(kernel) ? ctx->prof_n[kernel] : 0;
  auto it = ctx->prof_recs.find(kernel);
  if (it != ctx->prof_recs.end())
    for (auto& r : it->second) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, r.a, r.b));
      tot += ms;
      ++n;
    }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = n;
  return 0;
}

int geoflood_profile_cells(geoflood_ctx* ctx, const char* kernel, long long* cells) {
  if (!ctx || !kernel || !cells) return GEOFLOOD_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->st));
  *cells = ctx->prof_cells.count(kernel) ? ctx->prof_cells[kernel] : 0;
  return 0;
}

int geoflood_counters(geoflood_ctx* ctx, int s, long long* cell_updates,
                      long long* wet_cell_updates) {
  if (!valid_scen(ctx, s)) return fail(ctx, GEOFLOOD_ERR_ARG, "counters: bad scenario");
  int rc = sync_ctl_down(ctx);
  if (rc) return rc;
  if (cell_updates) *cell_updates = (long long)ctx->h_ctl[s].cell_updates;
  if (wet_cell_updates) *wet_cell_updates = (long long)ctx->h_ctl[s].wet_updates;
  return 0;
}

int geoflood_autotune(geoflood_ctx* ctx, int reps, int* variant,
                      double* ms_per_variant) {
  if (!ctx || reps < 1) return GEOFLOOD_ERR_ARG;
  int rc = sync_ctl_down(ctx);
  if (rc) return rc;
  // time every variant on the current state: the launches write only the
  // next-state buffer and the step counters, which are restored afterwards
  std::vector<GfCtl> saved(ctx->h_ctl, ctx->h_ctl + ctx->nscen);
  for (int s = 0; s < ctx->nscen; ++s) {
    ctx->h_ctl[s].active = 1;
    if (!(ctx->h_ctl[s].dt_use > 0)) ctx->h_ctl[s].dt_use = ctx->h_ctl[s].dt_next;
  }
  if ((rc = sync_ctl_up(ctx))) return rc;
  GfView v = view(ctx);
  v.done = nullptr;  // no controller: the state does not advance
  const int nv = gf::patch_step_variants(ctx->G.M, ctx->prec,
                                        ctx->G.dim_split || ctx->G.subcycle);
  cudaEvent_t a = pool_event(ctx), b = pool_event(ctx);
  int best = 0;
  double best_ms = 1e300;
  for (int k = 0; k < nv; ++k) {
    for (int w = 0; w < 2; ++w)  // warm-up
      CKL(ctx->prec ? gf::launch_patch_step_f32(ctx->G, v, k, ctx->st)
                    : gf::launch_patch_step_f64(ctx->G, v, k, ctx->st),
          "autotune");
    CK(cudaEventRecord(a, ctx->st));
    for (int r = 0; r < reps; ++r)
      CKL(ctx->prec ? gf::launch_patch_step_f32(ctx->G, v, k, ctx->st)
                    : gf::launch_patch_step_f64(ctx->G, v, k, ctx->st),
          "autotune");
    CK(cudaEventRecord(b, ctx->st));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    const double per = ms / reps;
    if (ms_per_variant) ms_per_variant[k] = per;
    if (per < best_ms) { best_ms = per; best = k; }
    ctx->launches += reps + 2;
  }
  std::copy(saved.begin(), saved.end(), ctx->h_ctl);
  if ((rc = sync_ctl_up(ctx))) return rc;
  if ((rc = forget_same(ctx))) return rc;
  ctx->variant = best;
  if (variant) *variant = best;
  return 0;
}

int geoflood_set_variant(geoflood_ctx* ctx, int variant) {
  if (!ctx || variant < 0 ||
      variant >= gf::patch_step_variants(ctx->G.M, ctx->prec,
                                         ctx->G.dim_split || ctx->G.subcycle))
    return fail(ctx, GEOFLOOD_ERR_ARG, "set_variant: no such variant");
  ctx->variant = variant;
  // the per-unit volumes of another variant's layout are not reusable
  return forget_same(ctx);
}

int geoflood_launch_count(geoflood_ctx* ctx, long long* launches) {
  if (!ctx || !launches) return GEOFLOOD_ERR_ARG;
  *launches = ctx->launches;
  return 0;
}

// ---------------------------------------------------------------------------
// Learned refinement predictor

int geoflood_cnn_nparam(void) { return gf::cnn_nparam(); }

int geoflood_cnn_set_params(geoflood_ctx* ctx, const float* prm, int n) {
  if (!ctx || !prm || n != gf::cnn_nparam())
    return fail(ctx, GEOFLOOD_ERR_ARG, "cnn_set_params: expected " +
                                           std::to_string(gf::cnn_nparam()) + " parameters");
  int rc = cnn_params_alloc(ctx);
  if (rc) return rc;
  CnnState& c = ctx->cnn;
  CK(cudaMemcpyAsync(c.prm, prm, (size_t)n * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(c.am, 0, (size_t)n * 4, ctx->st));
  CK(cudaMemsetAsync(c.av, 0, (size_t)n * 4, ctx->st));
  CKL(gf::cnn_cast(c.prm, c.wb, c.wf, ctx->st), "cnn_cast");
  ctx->launches++;
  CK(cudaStreamSynchronize(ctx->st));
  c.adam_t = 0;
  c.ready = true;
  return 0;
}

int geoflood_cnn_get_params(geoflood_ctx* ctx, float* prm, int n) {
  if (!ctx || !prm || n != gf::cnn_nparam() || !ctx->cnn.ready)
    return fail(ctx, GEOFLOOD_ERR_ARG, "cnn_get_params: no parameters or bad size");
  CK(cudaMemcpyAsync(prm, ctx->cnn.prm, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int geoflood_cnn_set_scale(geoflood_ctx* ctx, const float* scale) {
  if (!ctx || !scale) return GEOFLOOD_ERR_ARG;
  for (int k = 0; k < 4; ++k)
    if (!(scale[k] > 0.f)) return fail(ctx, GEOFLOOD_ERR_ARG, "cnn_set_scale: scales must be > 0");
  std::copy(scale, scale + 4, ctx->cnn.scale);
  return 0;
}

int geoflood_cnn_features(geoflood_ctx* ctx, int s, uint16_t* out) {
  if (!valid_scen(ctx, s) || !out) return fail(ctx, GEOFLOOD_ERR_ARG, "cnn_features: bad argument");
  CnnState& n = ctx->cnn;
  int rc = cnn_infer_alloc(ctx);
  if (rc) return rc;
  const int first = ctx->h_scen[s].poff, count = ctx->h_scen[s].pcount;
  CKL(gf::launch_cnn_features(ctx->G, view(ctx), first, count, n.scale, n.x, ctx->st),
      "cnn_features");
  ctx->launches++;
  CK(cudaMemcpyAsync(out, n.x, (size_t)count * CNN_X_BYTES, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int geoflood_cnn_predict(geoflood_ctx* ctx, int s, float* logit) {
  if (!valid_scen(ctx, s) || !logit) return fail(ctx, GEOFLOOD_ERR_ARG, "cnn_predict: bad argument");
  if (!ctx->cnn.ready) return fail(ctx, GEOFLOOD_ERR_STATE, "cnn_predict: no parameters");
  const int first = ctx->h_scen[s].poff, count = ctx->h_scen[s].pcount;
  int rc = cnn_infer(ctx, first, count);
  if (rc) return rc;
  CK(cudaMemcpyAsync(logit, ctx->cnn.logit, (size_t)count * 4, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int geoflood_cnn_grad(geoflood_ctx* ctx, const uint16_t* x, const float* label, int n,
                      float pos_weight, float* logit, float* grad, float* loss) {
  if (!ctx || !x || !label || n < 1 || !(pos_weight > 0.f))
    return fail(ctx, GEOFLOOD_ERR_ARG, "cnn_grad: bad argument");
  CnnState& c = ctx->cnn;
  if (!c.ready) return fail(ctx, GEOFLOOD_ERR_STATE, "cnn_grad: no parameters");
  int rc = cnn_batch_alloc(ctx, n);
  if (rc) return rc;
  const int np = gf::cnn_nparam();
  CK(cudaMemcpyAsync(c.xb, x, (size_t)n * CNN_X_BYTES, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(c.yb, label, (size_t)n * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(c.grad, 0, (size_t)np * 4, ctx->st));
  CK(cudaMemsetAsync(c.loss, 0, 4, ctx->st));
  CKL(gf::cnn_forward(c.xb, c.wb, c.prm, c.ta[0], c.ta[1], c.ta[2], c.tv, c.tlogit, n, ctx->st),
      "cnn_forward");
  CKL(gf::cnn_backward(c.xb, c.wf, c.prm, c.ta[0], c.ta[1], c.ta[2], c.tv, c.tlogit, c.yb,
                       pos_weight, c.grad, c.loss, c.td[0], c.td[1], c.td[2], n, ctx->st),
      "cnn_backward");
  ctx->launches += 11;
  if (logit) CK(cudaMemcpyAsync(logit, c.tlogit, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (grad) CK(cudaMemcpyAsync(grad, c.grad, (size_t)np * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (loss) CK(cudaMemcpyAsync(loss, c.loss, 4, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int geoflood_cnn_dataset(geoflood_ctx* ctx, int capacity) {
  if (!ctx || capacity < 0) return GEOFLOOD_ERR_ARG;
  CnnState& c = ctx->cnn;
  if (capacity != c.ds_cap) {
    cudaFree(c.dx);
    cudaFree(c.dy);
    c.dx = nullptr;
    c.dy = nullptr;
    c.ds_cap = 0;
    if (capacity > 0) {
      int rc = cnn_alloc(ctx, &c.dx, (size_t)capacity * CNN_X_BYTES);
      rc |= cnn_alloc(ctx, (void**)&c.dy, (size_t)capacity * 4);
      if (rc) return GEOFLOOD_ERR_OOM;
    }
    c.ds_cap = capacity;
  }
  c.ds_n = 0;
  c.pend_n = -1;
  return 0;
}

int geoflood_cnn_snapshot(geoflood_ctx* ctx) {
  if (!ctx) return GEOFLOOD_ERR_ARG;
  CnnState& c = ctx->cnn;
  const size_t cap = (size_t)ctx->cap;
  int rc = cnn_alloc(ctx, &c.px, cap * CNN_X_BYTES);
  rc |= cnn_alloc(ctx, (void**)&c.py, cap * 4);
  if (rc) return GEOFLOOD_ERR_OOM;
  CKL(gf::launch_cnn_features(ctx->G, view(ctx), 0, ctx->npatch, c.scale, c.px, ctx->st),
      "cnn_features");
  ctx->launches++;
  CK(cudaMemsetAsync(c.py, 0, (size_t)ctx->npatch * 4, ctx->st));
  c.pend_n = ctx->npatch;
  c.pend_gen = ctx->generation;
  return 0;
}

int geoflood_check_tags(geoflood_ctx* ctx, int observe, int* misses) {
  if (!ctx) return GEOFLOOD_ERR_ARG;
  CnnState& c = ctx->cnn;
  if (observe && (c.pend_n != ctx->npatch || c.pend_gen != ctx->generation))
    return fail(ctx, GEOFLOOD_ERR_STATE, "check_tags: no snapshot of the current patches");
  int rc = cnn_alloc(ctx, (void**)&c.misses, sizeof(unsigned));
  if (rc) return rc;
  CK(cudaMemsetAsync(c.misses, 0, sizeof(unsigned), ctx->st));
  if ((rc = tag_pass(ctx, false, c.misses, observe ? c.py : nullptr))) return rc;
  unsigned m = 0;
  CK(cudaMemcpyAsync(&m, c.misses, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (misses) *misses = (int)m;
  return 0;
}

int geoflood_cnn_commit(geoflood_ctx* ctx, int* total, int* positives) {
  if (!ctx) return GEOFLOOD_ERR_ARG;
  CnnState& c = ctx->cnn;
  if (c.pend_n < 0 || c.pend_gen != ctx->generation)
    return fail(ctx, GEOFLOOD_ERR_STATE, "cnn_commit: no snapshot of the current patches");
  const int add = std::min(c.pend_n, c.ds_cap - c.ds_n);
  if (add > 0) {
    CK(cudaMemcpyAsync((char*)c.dx + (size_t)c.ds_n * CNN_X_BYTES, c.px, (size_t)add * CNN_X_BYTES,
                       cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(c.dy + c.ds_n, c.py, (size_t)add * 4, cudaMemcpyDeviceToDevice, ctx->st));
    c.ds_n += add;
  }
  c.pend_n = -1;
  if (positives) {
    std::vector<float> y(c.ds_n);
    if (c.ds_n)
      CK(cudaMemcpyAsync(y.data(), c.dy, (size_t)c.ds_n * 4, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    int npos = 0;
    for (float v : y) npos += v > 0.5f;
    *positives = npos;
  }
  if (total) *total = c.ds_n;
  return 0;
}

int geoflood_cnn_dataset_read(geoflood_ctx* ctx, int first, int n, uint16_t* x, float* y) {
  if (!ctx || first < 0 || n < 0 || first + n > ctx->cnn.ds_n)
    return fail(ctx, GEOFLOOD_ERR_ARG, "cnn_dataset_read: range outside the dataset");
  CnnState& c = ctx->cnn;
  if (n == 0) return 0;
  if (x) CK(cudaMemcpyAsync(x, (char*)c.dx + (size_t)first * CNN_X_BYTES, (size_t)n * CNN_X_BYTES,
                            cudaMemcpyDeviceToHost, ctx->st));
  if (y) CK(cudaMemcpyAsync(y, c.dy + first, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int geoflood_cnn_train(geoflood_ctx* ctx, int epochs, int batch, float lr, float pos_weight,
                       unsigned long long seed, float* epoch_loss) {
  if (!ctx || epochs < 0 || epochs > 1024 || batch < 1 || !(lr > 0.f) || !(pos_weight > 0.f))
    return fail(ctx, GEOFLOOD_ERR_ARG, "cnn_train: bad argument");
  CnnState& c = ctx->cnn;
  if (!c.ready) return fail(ctx, GEOFLOOD_ERR_STATE, "cnn_train: no parameters");
  const int N = c.ds_n;
  if (N < 1) return fail(ctx, GEOFLOOD_ERR_STATE, "cnn_train: empty dataset");
  batch = std::min(batch, N);
  int rc = cnn_batch_alloc(ctx, batch);
  if (rc) return rc;
  if (N > c.idx_cap) {
    cudaFree(c.idx);
    c.idx = nullptr;
    c.idx_cap = 0;
    if ((rc = cnn_alloc(ctx, (void**)&c.idx, (size_t)N * 4))) return rc;
    c.idx_cap = N;
  }
  const int np = gf::cnn_nparam();
  std::vector<int> perm(N);
  uint64_t st = seed;
  CK(cudaMemsetAsync(c.loss, 0, 4 * 1024, ctx->st));
  const int nb = N / batch;  // full batches only
  for (int e = 0; e < epochs; ++e) {
    for (int k = 0; k < N; ++k) perm[k] = k;
    for (int k = N - 1; k > 0; --k) {  // Fisher-Yates
      const int j = (int)(splitmix64(st) % (uint64_t)(k + 1));
      std::swap(perm[k], perm[j]);
    }
    CK(cudaMemcpyAsync(c.idx, perm.data(), (size_t)N * 4, cudaMemcpyHostToDevice, ctx->st));
    for (int b = 0; b < nb; ++b) {
      CKL(gf::cnn_gather(c.dx, c.dy, c.idx + (size_t)b * batch, batch, c.xb, c.yb, ctx->st),
          "cnn_gather");
      CK(cudaMemsetAsync(c.grad, 0, (size_t)np * 4, ctx->st));
      CKL(gf::cnn_forward(c.xb, c.wb, c.prm, c.ta[0], c.ta[1], c.ta[2], c.tv, c.tlogit, batch,
                          ctx->st),
          "cnn_forward");
      CKL(gf::cnn_backward(c.xb, c.wf, c.prm, c.ta[0], c.ta[1], c.ta[2], c.tv, c.tlogit, c.yb,
                           pos_weight, c.grad, c.loss + e, c.td[0], c.td[1], c.td[2], batch,
                           ctx->st),
          "cnn_backward");
      CKL(gf::cnn_adam(c.prm, c.grad, c.am, c.av, lr, ++c.adam_t, ctx->st), "cnn_adam");
      CKL(gf::cnn_cast(c.prm, c.wb, c.wf, ctx->st), "cnn_cast");
      ctx->launches += 14;
    }
    // the host vector is rewritten next epoch: wait for its copy
    CK(cudaStreamSynchronize(ctx->st));
  }
  if (epoch_loss && epochs > 0) {
    std::vector<float> l(epochs);
    CK(cudaMemcpyAsync(l.data(), c.loss, (size_t)epochs * 4, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int e = 0; e < epochs; ++e) epoch_loss[e] = l[e] / (float)nb;
  }
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

int geoflood_advance(geoflood_ctx* ctx, double t_target, int regrid_interval,
                     int check_interval, int mode, geoflood_advance_stats* out) {
  if (!ctx || regrid_interval < 1 || check_interval < 1 || check_interval > regrid_interval ||
      (mode & ~(GEOFLOOD_ADVANCE_COLLECT | GEOFLOOD_ADVANCE_REGRID_ON_MISS)))
    return fail(ctx, GEOFLOOD_ERR_ARG, "advance: bad argument");
  const bool collect = mode & GEOFLOOD_ADVANCE_COLLECT;
  const bool on_miss = (mode & GEOFLOOD_ADVANCE_REGRID_ON_MISS) && !collect;
  geoflood_advance_stats st{};
  int rc = 0;
  if (collect && (rc = geoflood_cnn_snapshot(ctx))) return rc;
  std::vector<double> t(ctx->nscen);
  std::vector<int> n(ctx->nscen);
  int since = 0;
  using clock = std::chrono::steady_clock;
  auto secs = [](clock::time_point a) {
    return std::chrono::duration<double>(clock::now() - a).count();
  };
  const double host0 = ctx->regrid_host_s;
  for (;;) {
    const int want = std::min(check_interval, regrid_interval - since);
    const int np = ctx->npatch;
    // a chunk that cannot end in a regrid takes its check inside the step's
    // readback (a regrid's own tag pass counts the misses)
    const bool fused = !collect && since + want < regrid_interval;
    int fmisses = 0;
    auto t0 = clock::now();
    rc = step_core(ctx, t_target, want, t.data(), n.data(), fused ? &fmisses : nullptr);
    st.step_s += secs(t0);
    if (rc) return rc;
    int taken = 0;
    bool done = true;
    for (int s = 0; s < ctx->nscen; ++s) {
      taken = std::max(taken, n[s]);
      done &= !(t[s] < t_target);
    }
    st.steps += taken;
    st.patch_steps += (long long)taken * np;
    since += taken;
    if (done) break;
    if (taken == 0) return fail(ctx, GEOFLOOD_ERR_STATE, "advance: no progress");
    // the plain criterion judges at every check; a check that falls on a
    // regrid is counted by the regrid's own tag pass
    int misses = 0;
    const bool due = since >= regrid_interval;
    if (due && !collect) {
      t0 = clock::now();
      rc = regrid_impl(ctx, &misses);
      st.regrid_s += secs(t0);
      if (rc) return rc;
      st.checks++;
      st.misses += misses;
      st.regrids++;
      since = 0;
      continue;
    }
    if (fused) {
      misses = fmisses;
    } else {
      t0 = clock::now();
      rc = geoflood_check_tags(ctx, collect ? 1 : 0, &misses);
      st.check_s += secs(t0);
      if (rc) return rc;
    }
    st.checks++;
    st.misses += misses;
    if (due || (on_miss && misses > 0)) {
      if (collect) {
        int total = 0;
        if ((rc = geoflood_cnn_commit(ctx, &total, nullptr))) return rc;
        st.samples = total;
      }
      t0 = clock::now();
      rc = geoflood_regrid(ctx);
      st.regrid_s += secs(t0);
      if (rc) return rc;
      st.regrids++;
      if (!due) st.miss_regrids++;
      since = 0;
      if (collect && (rc = geoflood_cnn_snapshot(ctx))) return rc;
    }
  }
  if (collect) ctx->cnn.pend_n = -1;
  st.regrid_host_s = ctx->regrid_host_s - host0;
  if (out) *out = st;
  return 0;
}

int geoflood_set_tagger(geoflood_ctx* ctx, int tagger, float threshold) {
  if (!ctx || (tagger != GEOFLOOD_TAGGER_PLAIN && tagger != GEOFLOOD_TAGGER_LEARNED) ||
      !(threshold > 0.f && threshold < 1.f))
    return fail(ctx, GEOFLOOD_ERR_ARG, "set_tagger: bad argument");
  if (tagger == GEOFLOOD_TAGGER_LEARNED && !ctx->cnn.ready)
    return fail(ctx, GEOFLOOD_ERR_STATE, "set_tagger: no network parameters");
  ctx->cnn.tagger = tagger;
  ctx->cnn.logit_thr = std::log(threshold / (1.f - threshold));
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoint and resume.  The checkpoint is a flat byte record:
//   "GFCK", version, sizeof(geoflood_config), the configuration bytes,
//   precision, patch size, scenario count, then per scenario: Manning n and
//   eta0, the DEMs (count, then per DEM nx, ny, x0, y0, dx, dy, the nodes),
//   the leaves (count, then level, px, py), the time-stepping state (t,
//   dt_next, steps, rejects, nclip, clipvol, cell and wet-cell updates),
//   the gauges (count, positions, latest sample, arrival), the current state
//   buffer of its patches (whole tiles, ghosts included; in the FP32 form
//   also the compensation terms); then the network (parameters, Adam
//   moments and step, input scales, tagger, threshold; or none).
// Beds are recomputed from the DEMs on load (the same kernel, so the same
// values).
// ---------------------------------------------------------------------------
namespace {

struct Bytes {
  unsigned char* p;
  size_t cap, n = 0;
  void put(const void* src, size_t k) {
    if (p && n + k <= cap) std::memcpy(p + n, src, k);
    n += k;
  }
  template <typename T> void val(const T& v) { put(&v, sizeof(T)); }
};

struct Reader {
  const unsigned char* p;
  size_t n, at = 0;
  bool ok = true;
  void get(void* dst, size_t k) {
    if (!ok || at + k > n) { ok = false; return; }
    std::memcpy(dst, p + at, k);
    at += k;
  }
  template <typename T> T val() { T v{}; get(&v, sizeof(T)); return v; }
};

const char kMagic[4] = {'G', 'F', 'C', 'K'};
const int kVersion = 1;

}  // namespace

extern "C" {

int geoflood_save(geoflood_ctx* ctx, void* buf, size_t cap, size_t* size) {
  if (!ctx || !size) return fail(ctx, GEOFLOOD_ERR_ARG, "save: bad argument");
  int rc = sync_ctl_down(ctx);
  if (rc) return rc;
  Bytes w{static_cast<unsigned char*>(buf), buf ? cap : 0};
  w.put(kMagic, 4);
  w.val(kVersion);
  w.val((int)sizeof(geoflood_config));
  w.put(&ctx->cfg, sizeof(geoflood_config));
  w.val(ctx->prec);
  w.val(ctx->G.M);
  w.val(ctx->nscen);
  const size_t TT = (size_t)ctx->G.T * ctx->G.T, MM = (size_t)ctx->G.M * ctx->G.M;
  const size_t esz = ctx->prec ? sizeof(float) : sizeof(double);
  std::vector<unsigned char> tmp;
  auto dev = [&](const void* d, size_t bytes) {
    tmp.resize(bytes);
    if (bytes) {
      if (cudaMemcpyAsync(tmp.data(), d, bytes, cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
          cudaStreamSynchronize(ctx->st) != cudaSuccess)
        return false;
    }
    w.put(tmp.data(), bytes);
    return true;
  };
  for (int s = 0; s < ctx->nscen; ++s) {
    const GfScenario& S = ctx->h_scen[s];
    const GfCtl& C = ctx->h_ctl[s];
    w.val(S.manning_n);
    w.val(S.eta0);
    w.val(S.ndem);
    for (int k = 0; k < S.ndem; ++k) {
      w.val(S.dnx[k]); w.val(S.dny[k]);
      w.val(S.dx0[k]); w.val(S.dy0[k]); w.val(S.ddx[k]); w.val(S.ddy[k]);
      if (!dev(S.dem[k], (size_t)S.dnx[k] * S.dny[k] * sizeof(double)))
        return fail(ctx, GEOFLOOD_ERR_CUDA, "save: DEM copy");
    }
    const auto& lv = ctx->forests[s].leaves();
    w.val((int)lv.size());
    for (const gf::Leaf& l : lv) { w.val(l.level); w.val(l.px); w.val(l.py); }
    w.val(C.t); w.val(C.dt_next); w.val(C.steps); w.val(C.rejects); w.val(C.nclip);
    w.val(C.clipvol); w.val(C.cell_updates); w.val(C.wet_updates);
    w.val(S.ngauge);
    if (S.ngauge > 0) {
      if (!dev(ctx->d_gxy[s], 2 * S.ngauge * sizeof(double)) ||
          !dev(ctx->d_gout[s], 5 * S.ngauge * sizeof(double)) ||
          !dev(ctx->d_garr[s], S.ngauge * sizeof(double)))
        return fail(ctx, GEOFLOOD_ERR_CUDA, "save: gauge copy");
    }
    const size_t np = (size_t)S.pcount, off = (size_t)S.poff;
    const void* q = ctx->prec ? (const void*)(ctx->qf[C.cur] + off * 3 * TT)
                              : (const void*)(ctx->q[C.cur] + off * 3 * TT);
    if (!dev(q, np * 3 * TT * esz)) return fail(ctx, GEOFLOOD_ERR_CUDA, "save: state copy");
    if (ctx->prec && !dev(ctx->lof[C.cur] + off * 3 * MM, np * 3 * MM * sizeof(float)))
      return fail(ctx, GEOFLOOD_ERR_CUDA, "save: compensation copy");
  }
  const CnnState& c = ctx->cnn;
  const int nprm = gf::cnn_nparam();
  w.val((int)(c.ready ? 1 : 0));
  if (c.ready) {
    if (!dev(c.prm, (size_t)nprm * 4) || !dev(c.am, (size_t)nprm * 4) ||
        !dev(c.av, (size_t)nprm * 4))
      return fail(ctx, GEOFLOOD_ERR_CUDA, "save: network copy");
    w.val(c.adam_t);
  }
  w.put(c.scale, sizeof(c.scale));
  w.val(c.tagger);
  w.val(c.logit_thr);
  *size = w.n;
  if (!buf || cap < w.n)
    return fail(ctx, GEOFLOOD_ERR_CAPACITY,
                "save: the checkpoint needs " + std::to_string(w.n) + " bytes");
  return 0;
}

int geoflood_load(geoflood_ctx* ctx, const void* buf, size_t size) {
  if (!ctx || !buf) return fail(ctx, GEOFLOOD_ERR_ARG, "load: bad argument");
  Reader r{static_cast<const unsigned char*>(buf), size};
  char magic[4];
  r.get(magic, 4);
  if (!r.ok || std::memcmp(magic, kMagic, 4) || r.val<int>() != kVersion ||
      r.val<int>() != (int)sizeof(geoflood_config))
    return fail(ctx, GEOFLOOD_ERR_ARG, "load: not a checkpoint of this library version");
  geoflood_config cfg{};
  r.get(&cfg, sizeof(cfg));
  if (!r.ok || std::memcmp(&cfg, &ctx->cfg, sizeof(cfg)) || r.val<int>() != ctx->prec ||
      r.val<int>() != ctx->G.M || r.val<int>() != ctx->nscen)
    return fail(ctx, GEOFLOOD_ERR_ARG, "load: the checkpoint was taken with another configuration");
  const size_t TT = (size_t)ctx->G.T * ctx->G.T, MM = (size_t)ctx->G.M * ctx->G.M;
  const size_t esz = ctx->prec ? sizeof(float) : sizeof(double);
  struct Scen {
    double manning, eta0;
    std::vector<std::vector<double>> z;
    std::vector<int> nx, ny;
    std::vector<double> x0, y0, dx, dy;
    std::vector<gf::Leaf> leaves;
    GfCtl ctl{};
    int ngauge = 0;
    std::vector<double> gxy, gout, garr;
    std::vector<unsigned char> q, lo;
  };
  std::vector<Scen> sc(ctx->nscen);
  size_t total = 0;
  for (int s = 0; s < ctx->nscen && r.ok; ++s) {
    Scen& x = sc[s];
    x.manning = r.val<double>();
    x.eta0 = r.val<double>();
    const int ndem = r.val<int>();
    if (!r.ok || ndem < 0 || ndem > GF_MAXDEM) return fail(ctx, GEOFLOOD_ERR_ARG, "load: corrupt DEM list");
    for (int k = 0; k < ndem && r.ok; ++k) {
      x.nx.push_back(r.val<int>()); x.ny.push_back(r.val<int>());
      x.x0.push_back(r.val<double>()); x.y0.push_back(r.val<double>());
      x.dx.push_back(r.val<double>()); x.dy.push_back(r.val<double>());
      if (!r.ok || x.nx.back() < 2 || x.ny.back() < 2 ||
          (size_t)x.nx.back() * x.ny.back() * 8 > size)
        return fail(ctx, GEOFLOOD_ERR_ARG, "load: corrupt DEM");
      x.z.emplace_back((size_t)x.nx.back() * x.ny.back());
      r.get(x.z.back().data(), x.z.back().size() * 8);
    }
    const int nl = r.val<int>();
    if (!r.ok || nl < 1 || nl > ctx->cap) return fail(ctx, GEOFLOOD_ERR_ARG, "load: corrupt leaf list");
    for (int k = 0; k < nl && r.ok; ++k) {
      gf::Leaf l;
      l.level = r.val<int>(); l.px = r.val<int>(); l.py = r.val<int>();
      if (l.level < ctx->G.minlevel || l.level > ctx->G.maxlevel || l.px < 0 || l.py < 0 ||
          l.px >= (ctx->G.mi << l.level) || l.py >= (ctx->G.mj << l.level))
        return fail(ctx, GEOFLOOD_ERR_ARG, "load: corrupt leaf");
      x.leaves.push_back(l);
    }
    x.ctl.t = r.val<double>(); x.ctl.dt_next = r.val<double>();
    x.ctl.steps = r.val<long long>(); x.ctl.rejects = r.val<long long>();
    x.ctl.nclip = r.val<long long>(); x.ctl.clipvol = r.val<double>();
    x.ctl.cell_updates = r.val<unsigned long long>();
    x.ctl.wet_updates = r.val<unsigned long long>();
    x.ngauge = r.val<int>();
    if (!r.ok || x.ngauge < 0 || x.ngauge > ctx->cfg.max_gauges)
      return fail(ctx, GEOFLOOD_ERR_ARG, "load: corrupt gauges");
    x.gxy.resize(2 * x.ngauge); x.gout.resize(5 * x.ngauge); x.garr.resize(x.ngauge);
    r.get(x.gxy.data(), x.gxy.size() * 8);
    r.get(x.gout.data(), x.gout.size() * 8);
    r.get(x.garr.data(), x.garr.size() * 8);
    x.q.resize((size_t)nl * 3 * TT * esz);
    r.get(x.q.data(), x.q.size());
    if (ctx->prec) {
      x.lo.resize((size_t)nl * 3 * MM * sizeof(float));
      r.get(x.lo.data(), x.lo.size());
    }
    total += (size_t)nl;
  }
  const int nprm = gf::cnn_nparam();
  const int has_net = r.val<int>();
  std::vector<float> prm, am, av;
  int adam_t = 0;
  if (has_net) {
    prm.resize(nprm); am.resize(nprm); av.resize(nprm);
    r.get(prm.data(), (size_t)nprm * 4);
    r.get(am.data(), (size_t)nprm * 4);
    r.get(av.data(), (size_t)nprm * 4);
    adam_t = r.val<int>();
  }
  float scale[4];
  r.get(scale, sizeof(scale));
  const int tagger = r.val<int>();
  const float thr = r.val<float>();
  if (!r.ok || r.at != size) return fail(ctx, GEOFLOOD_ERR_ARG, "load: truncated or corrupt checkpoint");
  if ((long long)total > ctx->cap) return fail(ctx, GEOFLOOD_ERR_CAPACITY, "load: too many patches");
  int rc = sync_ctl_down(ctx);
  if (rc) return rc;
  // forests, tables and scenario parameters
  std::vector<std::vector<gf::Leaf>> lv(ctx->nscen);
  for (int s = 0; s < ctx->nscen; ++s) {
    lv[s] = sc[s].leaves;
    GfScenario& S = ctx->h_scen[s];
    S.manning_n = sc[s].manning;
    S.manning_f = (float)sc[s].manning;
    S.eta0 = sc[s].eta0;
  }
  if ((rc = upload_tables(ctx, ctx->tsel, lv))) return rc;
  for (int s = 0; s < ctx->nscen; ++s) ctx->forests[s].set_leaves(lv[s]);
  ctx->npatch = (int)total;
  ctx->generation++;
  // DEMs (stored in priority order already) and beds
  for (int s = 0; s < ctx->nscen; ++s) {
    for (auto p : ctx->d_dem[s]) cudaFree(p);
    ctx->d_dem[s].clear();
    GfScenario& S = ctx->h_scen[s];
    S.ndem = 0;
    for (size_t k = 0; k < sc[s].z.size(); ++k) {
      double* d = nullptr;
      if (cudaMalloc(&d, sc[s].z[k].size() * 8) != cudaSuccess)
        return fail(ctx, GEOFLOOD_ERR_OOM, "load: DEM allocation");
      ctx->d_dem[s].push_back(d);
      CK(cudaMemcpyAsync(d, sc[s].z[k].data(), sc[s].z[k].size() * 8, cudaMemcpyHostToDevice, ctx->st));
      S.dem[k] = d;
      S.dnx[k] = sc[s].nx[k]; S.dny[k] = sc[s].ny[k];
      S.dx0[k] = sc[s].x0[k]; S.dy0[k] = sc[s].y0[k];
      S.ddx[k] = sc[s].dx[k]; S.ddy[k] = sc[s].dy[k];
    }
    S.ndem = (int)sc[s].z.size();
  }
  if ((rc = upload_scen(ctx))) return rc;
  for (int s = 0; s < ctx->nscen; ++s)
    if ((rc = forget_beds(ctx, s))) return rc;
  CKL(gf::launch_topo(ctx->G, view(ctx), 0, ctx->npatch, ctx->st), "topo");
  ctx->launches++;
  // states into buffer 0, time-stepping state, gauges
  for (int s = 0; s < ctx->nscen; ++s) {
    const GfScenario& S = ctx->h_scen[s];
    const size_t off = (size_t)S.poff;
    void* q = ctx->prec ? (void*)(ctx->qf[0] + off * 3 * TT) : (void*)(ctx->q[0] + off * 3 * TT);
    CK(cudaMemcpyAsync(q, sc[s].q.data(), sc[s].q.size(), cudaMemcpyHostToDevice, ctx->st));
    if (ctx->prec)
      CK(cudaMemcpyAsync(ctx->lof[0] + off * 3 * MM, sc[s].lo.data(), sc[s].lo.size(),
                         cudaMemcpyHostToDevice, ctx->st));
    GfCtl& C = ctx->h_ctl[s];
    const GfCtl& X = sc[s].ctl;
    C.t = X.t; C.dt_next = X.dt_next; C.steps = X.steps; C.rejects = X.rejects;
    C.nclip = X.nclip; C.clipvol = X.clipvol;
    C.cell_updates = X.cell_updates; C.wet_updates = X.wet_updates;
    C.cur = 0; C.accepted = 0; C.status = 0; C.inrow = 0; C.nonfinite = 0;
    C.sub_k = 0; C.sub_rej = 0; C.rmax_bits = 0ull;
  }
  if ((rc = sync_ctl_up(ctx))) return rc;
  for (int s = 0; s < ctx->nscen; ++s) {
    if ((rc = geoflood_set_gauges(ctx, s, sc[s].gxy.data(), sc[s].ngauge))) return rc;
    if (sc[s].ngauge > 0) {
      CK(cudaMemcpyAsync(ctx->d_gout[s], sc[s].gout.data(), sc[s].gout.size() * 8,
                         cudaMemcpyHostToDevice, ctx->st));
      CK(cudaMemcpyAsync(ctx->d_garr[s], sc[s].garr.data(), sc[s].garr.size() * 8,
                         cudaMemcpyHostToDevice, ctx->st));
    }
  }
  // the network
  if (has_net) {
    if ((rc = geoflood_cnn_set_params(ctx, prm.data(), nprm))) return rc;
    CK(cudaMemcpyAsync(ctx->cnn.am, am.data(), (size_t)nprm * 4, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->cnn.av, av.data(), (size_t)nprm * 4, cudaMemcpyHostToDevice, ctx->st));
    ctx->cnn.adam_t = adam_t;
  }
  std::copy(scale, scale + 4, ctx->cnn.scale);
  ctx->cnn.tagger = has_net ? tagger : GEOFLOOD_TAGGER_PLAIN;
  ctx->cnn.logit_thr = thr;
  CK(cudaStreamSynchronize(ctx->st));
  return forget_same(ctx);
}

}  // extern "C"
