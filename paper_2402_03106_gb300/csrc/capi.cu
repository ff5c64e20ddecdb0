// capi.cu -- host side of libdarts: contexts, validation, the table cache and
// the C entry points declared in include/darts.h.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "darts.h"
#include "darts_device.cuh"
#include "darts_internal.h"

using namespace darts;

struct darts_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int smem_optin = 0;
  // scratch: [0] path counter, [1] ticket|status, [2 .. 2+kStatCount) stats
  unsigned long long* scratch = nullptr;
  double* partials = nullptr;  // block partials, grown on demand
  size_t partials_bytes = 0;
  double* host_hist = nullptr; // device histogram for darts_render_host
  size_t host_hist_bytes = 0;
  unsigned int* status_host = nullptr;  // pinned copy of the scratch status words
  // darts_render_host_async: two device histograms, a copy stream, and per
  // buffer the events "rendered" (compute stream) and "copied" (copy stream)
  double* async_hist[2] = {nullptr, nullptr};
  size_t async_bytes[2] = {0, 0};
  int async_slot = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_rendered[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
  bool copied_pending[2] = {false, false};
  // direction-table cache
  float* table = nullptr;
  size_t table_bytes = 0;
  bool table_valid = false;
  double table_key[9] = {0};
  // launch shape: requested block size of the path kernel (0 = largest that
  // fits), the cap of a warp's claim on the path counter (0 = kPathChunk),
  // and the batched kernel's block size and work items per CTA share (0 =
  // defaults); set by the caller or the autotuners
  int block = 0;
  int chunk = 0;
  int batch_block = 0;
  int batch_items = 0;
  int last_block = 0;
  unsigned long long last_paths = 0;  // paths of the last render
  bool last_fast = false;              // last launch ran the specialised DARTS kernel
  // temporal response: cumulative weights and per-bin DARTS weights
  double* wcdf = nullptr;
  float* wbin = nullptr;
  size_t w_bins = 0;
  // kernel timing
  bool timing = false;
  bool timed = false;
  cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
  // batched rendering: per-medium tables and parameters, work items, graph
  float* batch_tables = nullptr;
  size_t batch_tables_bytes = 0;
  void* batch_buf = nullptr;   // TableParams[n] | TraceParams[n] | BatchItem[m] | item counter
  size_t batch_buf_bytes = 0;
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  uint64_t graph_key = 0;
  // darts_render_frames: lanes (child contexts, each on a stream of its own),
  // the fork event recorded on this context's stream and one join event per lane
  static constexpr int kMaxLanes = 4;
  darts_ctx* lanes[kMaxLanes] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t lane_stream[kMaxLanes] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kMaxLanes] = {nullptr, nullptr, nullptr, nullptr};
  char err[512] = {0};
};

namespace {

// NVTX range over a library call (host side: it brackets the launches the
// call enqueues; a profiler can select kernels by it).  Costs a pointer test
// when no tool is attached.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

darts_status fail(darts_ctx* c, darts_status s, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

darts_status cuda_fail(darts_ctx* c, cudaError_t e, const char* what) {
  cudaGetLastError();  // reported here: a recoverable error must not resurface at a later launch
  if (e == cudaErrorMemoryAllocation) return fail(c, DARTS_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(c, DARTS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                              \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

// Grow a device buffer to at least `bytes`.
cudaError_t ensure(void** ptr, size_t* cap, size_t bytes) {
  if (*cap >= bytes && *ptr) return cudaSuccess;
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e == cudaSuccess) *cap = bytes;
  else cudaGetLastError();  // a failed allocation must not surface later as a launch error
  return e;
}

// n-point Gauss-Legendre nodes/weights on [-1, 1]: Newton iteration on the
// three-term recurrence of the Legendre polynomials.
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 1.0;
    for (int it = 0; it < 64; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double z1 = z;
      z = z1 - p1 / pp;
      if (std::fabs(z - z1) < 1e-15) break;
    }
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

int row_stride_of(int n_mu) { return ((n_mu + 1) + 3) / 4 * 4; }

// Earliest pulse start: one direction table per medium uses S_max of it.
double earliest_t0(const darts_scene* sc) {
  double t0 = sc->emitters[0].t0;
  for (int k = 1; k < sc->n_emitters; ++k) t0 = std::min(t0, sc->emitters[k].t0);
  return t0;
}

// Sensor elements (pixels of a camera, 1 for the point sensor).
uint64_t elements_of(const darts_scene* sc) {
  return sc->sensor.kind == DARTS_SENSOR_PINHOLE ? (uint64_t)sc->sensor.width * sc->sensor.height : 1;
}

// Scenes beyond one point emitter seen by a point sensor in an open box run
// the general variant of the path kernel.
constexpr uint32_t kRisVariantFlags = DARTS_FLAG_IID_CANDIDATES | DARTS_FLAG_EQUIANGULAR | DARTS_FLAG_RESERVOIR;

bool general_scene(const darts_scene* sc) {
  if (sc->n_emitters != 1 || sc->emitters[0].kind != DARTS_EMITTER_POINT) return true;
  return sc->sensor.kind != DARTS_SENSOR_POINT || sc->geom.walls != 0 || sc->geom.n_spheres > 0;
}

darts_status validate(darts_ctx* ctx, const darts_scene* sc, const darts_sampling* sp) {
  if (!sc || !sp) return fail(ctx, DARTS_ERR_INVALID_ARG, "scene and sampling must not be NULL");
  const darts_medium& m = sc->medium;
  if (!(m.sigma_s >= 0.0) || !(m.sigma_a >= 0.0) || !(m.sigma_s + m.sigma_a > 0.0) ||
      !std::isfinite(m.sigma_s + m.sigma_a))
    return fail(ctx, DARTS_ERR_INVALID_ARG, "need finite sigma_s >= 0, sigma_a >= 0, sigma_t > 0");
  if (!(std::fabs(m.g) < 1.0)) return fail(ctx, DARTS_ERR_INVALID_ARG, "need |g| < 1");
  if (!(m.v > 0.0) || !std::isfinite(m.v)) return fail(ctx, DARTS_ERR_INVALID_ARG, "need v > 0");
  if (sc->gate.n_bins < 1) return fail(ctx, DARTS_ERR_INVALID_ARG, "need n_bins >= 1");
  if (!(sc->gate.t_max > sc->gate.t_min) || !std::isfinite(sc->gate.t_max - sc->gate.t_min))
    return fail(ctx, DARTS_ERR_INVALID_ARG, "need finite t_min < t_max");
  if (sc->gate.weights) {
    double tot = 0.0;
    for (int b = 0; b < sc->gate.n_bins; ++b) {
      const double w = sc->gate.weights[b];
      if (!(w >= 0.0) || !std::isfinite(w))
        return fail(ctx, DARTS_ERR_INVALID_ARG, "gate weight %d must be finite and >= 0", b);
      tot += w;
    }
    if (!(tot > 0.0)) return fail(ctx, DARTS_ERR_INVALID_ARG, "gate weights must have a positive sum");
  }
  for (int i = 0; i < 3; ++i)
    if (!(sc->geom.hi[i] > sc->geom.lo[i]) || !std::isfinite(sc->geom.hi[i] - sc->geom.lo[i]))
      return fail(ctx, DARTS_ERR_INVALID_ARG, "the medium box needs finite lo < hi");
  if (sc->n_emitters < 1 || !sc->emitters) return fail(ctx, DARTS_ERR_INVALID_ARG, "need an emitter");
  if (sc->n_emitters > kMaxEmitters)
    return fail(ctx, DARTS_ERR_UNSUPPORTED, "at most %d emitters", kMaxEmitters);
  double e_tot = 0.0;
  for (int k = 0; k < sc->n_emitters; ++k) {
    const darts_emitter& e = sc->emitters[k];
    if (!(e.energy >= 0.0) || !std::isfinite(e.t0) || !std::isfinite(e.energy))
      return fail(ctx, DARTS_ERR_INVALID_ARG, "bad emitter %d", k);
    if (e.kind != DARTS_EMITTER_POINT && e.kind != DARTS_EMITTER_AREA)
      return fail(ctx, DARTS_ERR_INVALID_ARG, "emitter %d: unknown kind", k);
    for (int i = 0; i < 3; ++i)
      if (!(e.pos[i] >= sc->geom.lo[i] && e.pos[i] <= sc->geom.hi[i]))
        return fail(ctx, DARTS_ERR_INVALID_ARG, "emitter %d outside the medium box", k);
    if (e.kind == DARTS_EMITTER_AREA) {
      for (int i = 0; i < 3; ++i)
        if (!std::isfinite(e.u[i]) || !std::isfinite(e.v[i]))
          return fail(ctx, DARTS_ERR_INVALID_ARG, "emitter %d: edge vectors must be finite", k);
      const double cx = e.u[1] * e.v[2] - e.u[2] * e.v[1], cy = e.u[2] * e.v[0] - e.u[0] * e.v[2],
                   cz = e.u[0] * e.v[1] - e.u[1] * e.v[0];
      if (!(cx * cx + cy * cy + cz * cz > 0.0)) return fail(ctx, DARTS_ERR_INVALID_ARG, "emitter %d: zero area", k);
      for (int i = 0; i < 3; ++i) {
        const double far = e.pos[i] + e.u[i] + e.v[i];
        if (!(far >= sc->geom.lo[i] && far <= sc->geom.hi[i]))
          return fail(ctx, DARTS_ERR_INVALID_ARG, "emitter %d extends outside the medium box", k);
      }
    }
    if (!(sc->gate.t_max > e.t0)) return fail(ctx, DARTS_ERR_INVALID_ARG, "gate ends before emitter %d's pulse", k);
    e_tot += e.energy;
  }
  if (!(e_tot > 0.0)) return fail(ctx, DARTS_ERR_INVALID_ARG, "total emitted energy must be > 0");
  const darts_sensor& sen = sc->sensor;
  if (sen.kind == DARTS_SENSOR_POINT) {
    for (int i = 0; i < 3; ++i)
      if (!(sen.pos[i] >= sc->geom.lo[i] && sen.pos[i] <= sc->geom.hi[i]))
        return fail(ctx, DARTS_ERR_INVALID_ARG, "sensor outside the medium box");
    for (int k = 0; k < sc->n_emitters; ++k) {
      const darts_emitter& e = sc->emitters[k];
      double d2 = 0.0;
      for (int i = 0; i < 3; ++i) d2 += (sen.pos[i] - e.pos[i]) * (sen.pos[i] - e.pos[i]);
      if (e.kind == DARTS_EMITTER_POINT && !(d2 > 0.0))
        return fail(ctx, DARTS_ERR_INVALID_ARG, "sensor coincides with emitter %d", k);
    }
  } else if (sen.kind == DARTS_SENSOR_PINHOLE) {
    if (sen.width < 1 || sen.height < 1 || !(sen.fov_deg > 0.0 && sen.fov_deg < 180.0))
      return fail(ctx, DARTS_ERR_INVALID_ARG, "camera needs width, height >= 1 and 0 < fov < 180");
    if ((uint64_t)sen.width * (uint64_t)sen.height > (1ull << 30))  // pixel indices stay 32-bit
      return fail(ctx, DARTS_ERR_INVALID_ARG, "camera needs at most 2^30 pixels");
    double f[3], f2 = 0.0;
    for (int i = 0; i < 3; ++i) {
      if (!std::isfinite(sen.pos[i]) || !std::isfinite(sen.look_at[i]) || !std::isfinite(sen.up[i]))
        return fail(ctx, DARTS_ERR_INVALID_ARG, "camera position, look_at and up must be finite");
      f[i] = sen.look_at[i] - sen.pos[i];
      f2 += f[i] * f[i];
    }
    if (!(f2 > 0.0)) return fail(ctx, DARTS_ERR_INVALID_ARG, "camera look_at equals its position");
    const double rx = f[1] * sen.up[2] - f[2] * sen.up[1], ry = f[2] * sen.up[0] - f[0] * sen.up[2],
                 rz = f[0] * sen.up[1] - f[1] * sen.up[0];
    if (!(rx * rx + ry * ry + rz * rz > 1e-24 * f2))
      return fail(ctx, DARTS_ERR_INVALID_ARG, "camera up must not be parallel to the view direction");
  } else {
    return fail(ctx, DARTS_ERR_INVALID_ARG, "unknown sensor kind %d", sen.kind);
  }
  if (sc->geom.n_spheres < 0 || sc->geom.n_spheres > kMaxSpheres || (sc->geom.n_spheres && !sc->geom.spheres))
    return fail(ctx, DARTS_ERR_INVALID_ARG, "0..%d spheres with a host array", kMaxSpheres);
  for (int k = 0; k < sc->geom.n_spheres; ++k) {
    const double* q = sc->geom.spheres + 5 * k;
    if (!(q[3] > 0.0) || !(q[4] >= 0.0 && q[4] <= 1.0) || !std::isfinite(q[0] + q[1] + q[2] + q[3]))
      return fail(ctx, DARTS_ERR_INVALID_ARG, "sphere %d needs a finite centre, radius > 0 and albedo in [0, 1]", k);
  }
  if (sc->geom.walls < 0 || sc->geom.walls >= 64 || !(sc->geom.wall_albedo >= 0.0 && sc->geom.wall_albedo <= 1.0))
    return fail(ctx, DARTS_ERR_INVALID_ARG, "walls is a 6-bit face mask and wall_albedo in [0, 1]");
  if (sp->paths_per_element > UINT64_MAX / elements_of(sc))
    return fail(ctx, DARTS_ERR_INVALID_ARG, "paths_per_element x sensor elements exceeds 2^64");
  if (sp->max_bounces < 1 || sp->max_bounces > 1024)
    return fail(ctx, DARTS_ERR_INVALID_ARG, "max_bounces must be in 1..1024");
  if (sp->ris_m < 1 || sp->ris_m > trace_max_m())
    return fail(ctx, DARTS_ERR_INVALID_ARG, "ris_m must be in 1..%d", trace_max_m());
  if (sp->table_n_rho < 1 || sp->table_n_s < 1 || sp->table_n_mu < 2 || sp->table_n_mu > 1024)
    return fail(ctx, DARTS_ERR_INVALID_ARG, "table dims: n_rho >= 1, n_s >= 1, 2 <= n_mu <= 1024");
  if (!(sp->mis_alpha > 0.0) || !std::isfinite(sp->mis_alpha))
    return fail(ctx, DARTS_ERR_INVALID_ARG, "mis_alpha must be > 0");
  if (sp->method < DARTS_METHOD_DARTS || sp->method > DARTS_METHOD_DARTS_FULL_GATE)
    return fail(ctx, DARTS_ERR_INVALID_ARG, "unknown method %d", sp->method);
  // the general kernel runs the cooperative 8-candidate RIS (its shared
  // memory holds the 8-candidate task exchange)
  if ((sp->method == DARTS_METHOD_DARTS || sp->method == DARTS_METHOD_DARTS_FULL_GATE) && general_scene(sc) &&
      sp->ris_m != 8)
    return fail(ctx, DARTS_ERR_UNSUPPORTED, "scenes with surfaces, a camera or area emitters need ris_m = 8");
  if ((sp->flags & kRisVariantFlags) && general_scene(sc))
    return fail(ctx, DARTS_ERR_UNSUPPORTED, "the RIS variants run on medium-only scenes with a point emitter and sensor");
  return DARTS_OK;
}

void make_table_params(const darts_scene* sc, const darts_sampling* sp, TableParams* tp) {
  std::memset(tp, 0, sizeof(*tp));
  const darts_medium& m = sc->medium;
  const double D = 1.0 / (3.0 * (m.sigma_a + m.sigma_s * (1.0 - m.g)));
  tp->sigma_t = (float)(m.sigma_s + m.sigma_a);
  tp->sigma_a = (float)m.sigma_a;
  tp->v = (float)m.v;
  tp->phi_k0 = (float)(std::log(m.v) - 1.5 * std::log(4.0 * M_PI * m.v * D));
  tp->phi_invk = (float)(1.0 / (4.0 * m.v * D));
  tp->sa_v = (float)(m.sigma_a * m.v);
  tp->smax = (float)(m.v * (sc->gate.t_max - earliest_t0(sc)));
  tp->n_rho = sp->table_n_rho;
  tp->n_s = sp->table_n_s;
  tp->n_mu = sp->table_n_mu;
  tp->row_stride = row_stride_of(sp->table_n_mu);
  // the rules depend only on the node counts: computed once per process
  struct Rules {
    float mu_x[kMaxTabMuNodes], mu_w[kMaxTabMuNodes], t_x[kMaxTabTNodes], t_w[kMaxTabTNodes];
    Rules() {
      double x[kMaxTabTNodes], w[kMaxTabTNodes];
      gauss_legendre(kMaxTabMuNodes, x, w);
      for (int i = 0; i < kMaxTabMuNodes; ++i) {
        mu_x[i] = (float)x[i];
        mu_w[i] = (float)w[i];
      }
      gauss_legendre(kMaxTabTNodes, x, w);
      for (int i = 0; i < kMaxTabTNodes; ++i) {
        t_x[i] = (float)x[i];
        t_w[i] = (float)w[i];
      }
    }
  };
  static const Rules rules;
  std::memcpy(tp->mu_x, rules.mu_x, sizeof(rules.mu_x));
  std::memcpy(tp->mu_w, rules.mu_w, sizeof(rules.mu_w));
  std::memcpy(tp->t_x, rules.t_x, sizeof(rules.t_x));
  std::memcpy(tp->t_w, rules.t_w, sizeof(rules.t_w));
}

void table_key(const darts_scene* sc, const darts_sampling* sp, double key[9]) {
  key[0] = sc->medium.sigma_s;
  key[1] = sc->medium.sigma_a;
  key[2] = sc->medium.g;
  key[3] = sc->medium.v;
  key[4] = sc->gate.t_max - earliest_t0(sc);
  key[5] = sp->table_n_rho;
  key[6] = sp->table_n_s;
  key[7] = sp->table_n_mu;
  key[8] = 1.0;
}

// Build (or reuse) the context's cached table for this scene.
// Outputs the table launch may zero for the path launch that follows it.
struct ZeroSpec {
  double* a = nullptr;
  double* b = nullptr;
  unsigned long long n = 0;
  bool zeroed = false;  // set when the table launch did it (and the scratch counters)
};

darts_status ensure_table(darts_ctx* ctx, const darts_scene* sc, const darts_sampling* sp,
                          ZeroSpec* z = nullptr) {
  const Range nvtx_range("darts:table");
  double key[9];
  table_key(sc, sp, key);
  const bool hit = ctx->table_valid && std::memcmp(key, ctx->table_key, sizeof(key)) == 0 &&
                   !(sp->flags & DARTS_FLAG_REBUILD_TABLE);
  if (hit) return DARTS_OK;
  TableParams tp;
  make_table_params(sc, sp, &tp);
  const size_t bytes = (size_t)tp.n_rho * tp.n_s * tp.row_stride * sizeof(float);
  CK(ensure((void**)&ctx->table, &ctx->table_bytes, bytes), "table allocation");
  tp.cdf = ctx->table;
  if (z) {  // the path counter and the statistics (not the ticket/status word), and the outputs
    tp.zero_a = z->a;
    tp.zero_b = z->b;
    tp.zero_n = z->a ? z->n : 0;
    tp.zero_scratch = ctx->scratch;
    tp.zero_scratch_n = 2 + kStatCount;
  }
  CK(launch_table(tp, ctx->stream), "table kernel launch");
  if (z) z->zeroed = true;
  std::memcpy(ctx->table_key, key, sizeof(key));
  ctx->table_valid = true;
  return DARTS_OK;
}

void make_trace_params(darts_ctx* ctx, const darts_scene* sc, const darts_sampling* sp,
                       TraceParams* P) {
  std::memset(P, 0, sizeof(*P));
  P->chunk_cap = (unsigned)ctx->chunk;
  const darts_medium& m = sc->medium;
  const darts_emitter& e = sc->emitters[0];
  const double st = m.sigma_s + m.sigma_a;
  const double D = 1.0 / (3.0 * (m.sigma_a + m.sigma_s * (1.0 - m.g)));
  P->sigma_s = (float)m.sigma_s;
  P->sigma_t = (float)st;
  P->inv_st = (float)(1.0 / st);
  P->albedo = (float)(m.sigma_s / st);
  P->sa_v = (float)(m.sigma_a * m.v);
  P->v = (float)m.v;
  P->inv_v = (float)(1.0 / m.v);
  P->phi_k0_d = std::log(m.v) - 1.5 * std::log(4.0 * M_PI * m.v * D);
  P->phi_invk_d = 1.0 / (4.0 * m.v * D);
  P->sa_v_d = m.sigma_a * m.v;
  P->inv_v_d = 1.0 / m.v;
  P->phi_k0 = (float)P->phi_k0_d;
  P->phi_invk = (float)P->phi_invk_d;
  P->g = (float)m.g;
  P->hg_a = (float)((1.0 - m.g * m.g) / (4.0 * M_PI));
  P->hg_b = (float)(1.0 + m.g * m.g);
  P->hg_c = (float)(2.0 * m.g);
  P->hg_dlog_a = (float)(-2.0 * m.g / (1.0 - m.g * m.g));
  P->inv_sigma_s = m.sigma_s > 0.0 ? (float)(1.0 / m.sigma_s) : 0.0f;
  for (int i = 0; i < 3; ++i) {
    P->lo[i] = (float)sc->geom.lo[i];
    P->hi[i] = (float)sc->geom.hi[i];
    P->xe[i] = (float)e.pos[i];
    P->xs[i] = (float)sc->sensor.pos[i];
  }
  P->Ie = (float)(e.energy / (4.0 * M_PI));
  const darts_gate& G = sc->gate;
  P->n_bins = G.n_bins;
  P->S_gate_lo = (float)(m.v * (G.t_min - e.t0));
  P->S_gate_hi = (float)(m.v * (G.t_max - e.t0));
  P->S_bin = (float)(m.v * (G.t_max - G.t_min) / G.n_bins);
  P->inv_S_bin = (float)(G.n_bins / (m.v * (G.t_max - G.t_min)));
  P->tiny_s = (float)(m.v * (G.t_max - G.t_min) / 64.0);
  P->n_rho = sp->table_n_rho;
  P->n_s = sp->table_n_s;
  P->n_mu = sp->table_n_mu;
  P->row_stride = row_stride_of(sp->table_n_mu);
  P->rows = sp->table_n_rho * sp->table_n_s;
  P->inv_smax = (float)(1.0 / (m.v * (G.t_max - earliest_t0(sc))));
  P->n_s_over_8 = (float)(sp->table_n_s / 8.0);
  P->mu_scale = (float)(sp->table_n_mu / 2.0);
  P->inv_mu_scale = (float)(2.0 / sp->table_n_mu);
  P->mis_alpha = (float)sp->mis_alpha;
  P->uniform_sensor = (sp->flags & DARTS_FLAG_SENSOR_UNIFORM_ONLY) ? 1 : 0;
  P->no_eda = (sp->flags & DARTS_FLAG_NO_EDA) ? 1 : 0;
  P->surface_eda = (sp->flags & DARTS_FLAG_SURFACE_EDA) ? 1 : 0;
  P->no_da = (sp->flags & DARTS_FLAG_NO_DA_DISTANCE) ? 1 : 0;
  P->accumulate = (sp->flags & DARTS_FLAG_ACCUMULATE) ? 1 : 0;
  P->ris_mode = ((sp->flags & DARTS_FLAG_IID_CANDIDATES) ? 1 : 0) | ((sp->flags & DARTS_FLAG_EQUIANGULAR) ? 2 : 0) |
                ((sp->flags & DARTS_FLAG_RESERVOIR) ? 4 : 0);
  P->table = ctx->table;
  P->K = sp->max_bounces;
  P->M = sp->ris_m;
  P->key0 = (uint32_t)sp->seed;
  P->key1 = (uint32_t)(sp->seed >> 32);
  P->stream = sp->stream;
  // bin offset of the (single) sensor element: Philox at the element counter
  const U4 r = philox4x32_10(0u, 0u, sp->stream, (kVertexElement << 8) | 0u, P->key0, P->key1);
  double oe = std::floor((double)(r.x >> 8) * (1.0 / 16777216.0) * G.n_bins);
  if (oe >= G.n_bins) oe = G.n_bins - 1;
  P->o_e = (uint32_t)oe;
  const double ne = (double)std::max<uint64_t>(sp->paths_per_element, 1);
  P->wb = (float)(sp->method == DARTS_METHOD_DARTS ? G.n_bins / ne : 1.0 / ne);
  P->spp = std::max<uint64_t>(sp->paths_per_element, 1);
  // general scenes: emitters, surfaces, camera
  P->general = general_scene(sc) ? 1 : 0;
  double e_tot = 0.0;
  for (int k = 0; k < sc->n_emitters; ++k) e_tot += sc->emitters[k].energy;
  double acc = 0.0;
  P->n_emitters = sc->n_emitters;
  for (int k = 0; k < sc->n_emitters; ++k) {
    const darts_emitter& q = sc->emitters[k];
    EmitterParams& E = P->em[k];
    acc += q.energy;
    E.cdf = (float)(acc / e_tot);
    E.wsel = q.energy > 0.0 ? (float)(e_tot / q.energy) : 0.0f;
    E.kind = q.kind;
    E.ie = (float)(q.kind == DARTS_EMITTER_AREA ? q.energy / M_PI : q.energy / (4.0 * M_PI));
    E.s_lo = (float)(m.v * (G.t_min - q.t0));
    E.s_hi = (float)(m.v * (G.t_max - q.t0));
    double nx = q.u[1] * q.v[2] - q.u[2] * q.v[1], ny = q.u[2] * q.v[0] - q.u[0] * q.v[2],
           nz = q.u[0] * q.v[1] - q.u[1] * q.v[0];
    const double nn = std::sqrt(nx * nx + ny * ny + nz * nz);
    for (int i = 0; i < 3; ++i) {
      E.pos[i] = (float)q.pos[i];
      E.u[i] = (float)(q.kind == DARTS_EMITTER_AREA ? q.u[i] : 0.0);
      E.v[i] = (float)(q.kind == DARTS_EMITTER_AREA ? q.v[i] : 0.0);
    }
    E.n[0] = q.kind == DARTS_EMITTER_AREA ? (float)(nx / nn) : 0.0f;
    E.n[1] = q.kind == DARTS_EMITTER_AREA ? (float)(ny / nn) : 0.0f;
    E.n[2] = q.kind == DARTS_EMITTER_AREA ? (float)(nz / nn) : 0.0f;
  }
  P->em[sc->n_emitters - 1].cdf = 1.0f;
  P->n_spheres = sc->geom.n_spheres;
  for (int k = 0; k < sc->geom.n_spheres; ++k) {
    const double* q = sc->geom.spheres + 5 * k;
    P->sph[k] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
    P->sph_albedo[k] = (float)q[4];
  }
  {  // slab grid of the sphere culling (see cast_ray): the medium box in cull_slabs slabs per axis;
     // 32 for a camera (its kernel keeps no histogram tiles in shared memory), else 16
    P->cull_slabs = sc->sensor.kind == DARTS_SENSOR_PINHOLE ? kMaxCullSlabs : 16;
    double ext = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double w = (sc->geom.hi[i] - sc->geom.lo[i]) / P->cull_slabs;
      P->cull_inv_w[i] = (float)(1.0 / w);
      P->cull_off[i] = (float)(-sc->geom.lo[i] / w);
      ext = std::max(ext, sc->geom.hi[i] - sc->geom.lo[i]);
    }
    // far above the FP32 rounding of a ray point (about 1e-7 of the box), so
    // that no sphere a ray can meet is ever left out of its masks
    P->cull_eps = (float)(1e-4 * ext);
  }
  P->walls = sc->geom.walls;
  P->wall_albedo = (float)sc->geom.wall_albedo;
  const darts_sensor& sen = sc->sensor;
  P->camera = sen.kind == DARTS_SENSOR_PINHOLE ? 1 : 0;
  if (P->camera) {
    double f[3], r[3], u[3];
    for (int i = 0; i < 3; ++i) f[i] = sen.look_at[i] - sen.pos[i];
    double fn = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int i = 0; i < 3; ++i) f[i] /= fn;
    r[0] = f[1] * sen.up[2] - f[2] * sen.up[1];
    r[1] = f[2] * sen.up[0] - f[0] * sen.up[2];
    r[2] = f[0] * sen.up[1] - f[1] * sen.up[0];
    double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int i = 0; i < 3; ++i) r[i] /= rn;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    bool inside = true;
    for (int i = 0; i < 3; ++i) {
      P->cam_pos[i] = (float)sen.pos[i];
      P->cam_f[i] = (float)f[i];
      P->cam_r[i] = (float)r[i];
      P->cam_u[i] = (float)u[i];
      if (!(sen.pos[i] >= sc->geom.lo[i] && sen.pos[i] <= sc->geom.hi[i])) inside = false;
    }
    P->cam_inside = inside ? 1 : 0;
    P->cam_th = (float)std::tan(0.5 * sen.fov_deg * M_PI / 180.0);
    P->cam_aspect = (float)((double)sen.width / (double)sen.height);
    P->width = sen.width;
    P->height = sen.height;
  }
  {  // the lean camera kernel: every branch it drops is one this scene never takes
    bool points = true;
    for (int k = 0; k < sc->n_emitters; ++k) points = points && sc->emitters[k].kind == DARTS_EMITTER_POINT;
    P->lean = (P->general && P->camera && P->cam_inside && points && !sc->gate.weights &&
               !(sp->flags & DARTS_FLAG_SURFACE_EDA)) ? 1 : 0;
  }
  P->stats = ctx->scratch + 2;
  P->counter = ctx->scratch;
  P->ticket = reinterpret_cast<unsigned int*>(ctx->scratch + 1);
  P->status = reinterpret_cast<unsigned int*>(ctx->scratch + 1) + 1;
}

// The methods with DARTS samplers need the direction table.
bool uses_table(int method) {
  return method == DARTS_METHOD_DARTS || method == DARTS_METHOD_DARTS_FULL_GATE;
}

// Temporal response: cumulative weights C_b = (W_0 + ... + W_{b-1}) / sum W
// summed left to right in FP64, the per-bin DARTS path weights
// sum W / (N_e W_b), and the point sensor's systematic-sampling offset and
// phase (element 0's Philox draw).  Uploaded to context buffers.
darts_status set_weights(darts_ctx* ctx, const darts_scene* sc, const darts_sampling* sp, TraceParams& P) {
  P.wcdf = nullptr;
  P.wbin = nullptr;
  if (!sc->gate.weights) return DARTS_OK;
  const int B = sc->gate.n_bins;
  if (ctx->w_bins < (size_t)B) {
    cudaFree(ctx->wcdf);
    cudaFree(ctx->wbin);
    ctx->wcdf = nullptr;
    ctx->wbin = nullptr;
    ctx->w_bins = 0;
    CK(cudaMalloc((void**)&ctx->wcdf, (B + 1) * sizeof(double)), "weight allocation");
    CK(cudaMalloc((void**)&ctx->wbin, B * sizeof(float)), "weight allocation");
    ctx->w_bins = (size_t)B;
  }
  std::vector<double> c(B + 1);
  std::vector<float> wb(B);
  double tot = 0.0;
  for (int b = 0; b < B; ++b) tot += sc->gate.weights[b];
  double cum = 0.0;
  c[0] = 0.0;
  const double ne = (double)std::max<uint64_t>(sp->paths_per_element, 1);
  for (int b = 0; b < B; ++b) {
    cum = cum + sc->gate.weights[b];
    c[b + 1] = cum / tot;
    const double w = sc->gate.weights[b];
    wb[b] = w > 0.0 ? (float)(sp->method == DARTS_METHOD_DARTS ? tot / (ne * w) : 1.0) : 0.0f;
  }
  CK(cudaMemcpyAsync(ctx->wcdf, c.data(), (B + 1) * sizeof(double), cudaMemcpyHostToDevice, ctx->stream),
     "weight upload");
  CK(cudaMemcpyAsync(ctx->wbin, wb.data(), B * sizeof(float), cudaMemcpyHostToDevice, ctx->stream),
     "weight upload");
  // pageable sources: make the copies complete before the vectors go away
  CK(cudaStreamSynchronize(ctx->stream), "weight upload");
  P.wcdf = ctx->wcdf;
  P.wbin = ctx->wbin;
  const U4 r = philox4x32_10(0u, 0u, sp->stream, (kVertexElement << 8) | 0u, P.key0, P.key1);
  const uint64_t n = std::max<uint64_t>(sp->paths_per_element, 1);
  uint64_t oe = (uint64_t)std::floor((double)(r.x >> 8) * (1.0 / 16777216.0) * (double)n);
  P.w_oe = std::min(oe, n - 1);
  P.w_phi = (double)(r.y >> 8) * (1.0 / 16777216.0);
  return DARTS_OK;
}

// Common launch of the path kernel for render and debug.
// Launch shape: the requested (or largest) block size whose shared memory
// fits, falling back to FP64 atomics straight into the outputs when no tile
// fits (and always for a camera, whose output has one row per pixel).
void choose_launch(const darts_ctx* ctx, const darts_sampling* sp, const TraceParams& P, bool debug,
                   int* block, bool* tile, size_t* smem) {
  if (P.camera) {  // one histogram row per pixel: FP64 atomics straight into the output
    *tile = false;
    // default: 640 threads below 2^21 paths (a frame with about as many
    // paths as resident lanes runs as long as its longest paths, and a wider
    // block only adds warps per scheduler), 768 from there (the 512x512
    // sphere frame: 10.0 ms against 10.5 at 640 and 11.7 at 512)
    const int dflt = P.N >= (1ull << 21) ? 768 : 640;
    *block = trace_block_for(ctx->block ? ctx->block : dflt, debug, false, sp->method, sp->ris_m, P.general != 0);
    *smem = trace_smem_bytes(sp->method, P, *block, false);
    while (*smem > (size_t)ctx->smem_optin && *block > 512) {
      *block = *block == 896 ? 768 : (*block == 768 ? 640 : 512);
      *smem = trace_smem_bytes(sp->method, P, *block, false);
    }
    return;
  }
  const int want = ctx->block ? ctx->block : 768;
  *tile = true;
  *block = trace_block_for(want, debug, true, sp->method, sp->ris_m, P.general != 0);
  *smem = trace_smem_bytes(sp->method, P, *block, true);
  while (*smem > (size_t)ctx->smem_optin && *block > 512) {
    *block = *block == 768 ? 640 : 512;
    *smem = trace_smem_bytes(sp->method, P, *block, true);
  }
  if (*smem > (size_t)ctx->smem_optin) {
    *tile = false;
    *block = 512;
    *smem = trace_smem_bytes(sp->method, P, *block, false);
  }
}

darts_status run_trace(darts_ctx* ctx, const darts_scene* sc, const darts_sampling* sp,
                       TraceParams& P, bool debug, bool zeroed = false) {
  const Range nvtx_range("darts:trace");
  {
    const darts_status sw = set_weights(ctx, sc, sp, P);
    if (sw != DARTS_OK) return sw;
  }
  ctx->last_fast = sp->method == DARTS_METHOD_DARTS && !P.general;
  const int grid = ctx->sm_count;
  int block;
  bool tile;
  size_t smem;
  choose_launch(ctx, sp, P, debug, &block, &tile, &smem);
  ctx->last_block = block;
  if (smem > (size_t)ctx->smem_optin)
    return fail(ctx, DARTS_ERR_UNSUPPORTED, "direction table of %zu bytes exceeds shared memory", smem);
  const size_t pbytes = (size_t)grid * 2 * P.n_bins * sizeof(double);
  CK(ensure((void**)&ctx->partials, &ctx->partials_bytes, pbytes), "partials allocation");
  P.partials = ctx->partials;
  if (!zeroed) {  // else the table launch just before did this
    if (!tile && !P.accumulate) {  // contributions go straight into the (zeroed) outputs
      const size_t ob = elements_of(sc) * (size_t)P.n_bins * sizeof(double);
      CK(cudaMemsetAsync(P.hist, 0, ob, ctx->stream), "memset");
      if (P.sumsq) CK(cudaMemsetAsync(P.sumsq, 0, ob, ctx->stream), "memset");
    }
    // zero the path counter and the statistics (ticket and status persist)
    CK(cudaMemsetAsync(ctx->scratch, 0, sizeof(unsigned long long), ctx->stream), "memset");
    CK(cudaMemsetAsync(ctx->scratch + 2, 0, kStatCount * sizeof(unsigned long long), ctx->stream), "memset");
  }
  ctx->last_paths = P.N;
  if (ctx->timing) CK(cudaEventRecord(ctx->ev_start, ctx->stream), "event record");
  CK(launch_trace(sp->method, P, grid, block, debug, tile, smem, ctx->stream), "trace kernel launch");
  if (ctx->timing) {
    CK(cudaEventRecord(ctx->ev_stop, ctx->stream), "event record");
    ctx->timed = true;
  }
  return DARTS_OK;
}

}  // namespace

extern "C" {

const char* darts_status_string(darts_status s) {
  switch (s) {
    case DARTS_OK: return "ok";
    case DARTS_ERR_INVALID_ARG: return "invalid argument";
    case DARTS_ERR_CUDA: return "CUDA error";
    case DARTS_ERR_OOM: return "out of device memory";
    case DARTS_ERR_NUMERIC: return "non-finite value produced on the device";
    case DARTS_ERR_TIMEOUT: return "bounded device wait expired";
    case DARTS_ERR_UNSUPPORTED: return "unsupported by this build";
    case DARTS_ERR_BOUNDS: return "device index out of range (checked build)";
  }
  return "unknown status";
}

darts_status darts_create(darts_ctx** out, int cuda_device, void* cuda_stream) {
  if (!out) return DARTS_ERR_INVALID_ARG;
  *out = nullptr;
  darts_ctx* ctx = new (std::nothrow) darts_ctx();
  if (!ctx) return DARTS_ERR_OOM;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || cuda_device < 0 || cuda_device >= n) {
    delete ctx;
    return e != cudaSuccess ? DARTS_ERR_CUDA : DARTS_ERR_INVALID_ARG;
  }
  ctx->device = cuda_device;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (cudaSetDevice(cuda_device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, cuda_device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, cuda_device) != cudaSuccess) {
    delete ctx;
    return DARTS_ERR_CUDA;
  }
  ctx->smem_optin -= 1024;  // static shared memory of the path kernel
  const size_t sbytes = (2 + kStatCount) * sizeof(unsigned long long);
  e = cudaMalloc((void**)&ctx->scratch, sbytes);
  if (e == cudaSuccess) e = cudaMemset(ctx->scratch, 0, sbytes);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->status_host, 2 * sizeof(unsigned int));
  if (e != cudaSuccess) {
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->status_host) cudaFreeHost(ctx->status_host);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? DARTS_ERR_OOM : DARTS_ERR_CUDA;
  }
  *out = ctx;
  return DARTS_OK;
}

darts_status darts_destroy(darts_ctx* ctx) {
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->scratch);
  cudaFreeHost(ctx->status_host);
  cudaFree(ctx->partials);
  cudaFree(ctx->table);
  cudaFree(ctx->host_hist);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  for (int i = 0; i < 2; ++i) {
    cudaFree(ctx->async_hist[i]);
    if (ctx->ev_rendered[i]) cudaEventDestroy(ctx->ev_rendered[i]);
    if (ctx->ev_copied[i]) cudaEventDestroy(ctx->ev_copied[i]);
  }
  cudaFree(ctx->batch_tables);
  cudaFree(ctx->wcdf);
  cudaFree(ctx->wbin);
  cudaFree(ctx->batch_buf);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
  if (ctx->ev_stop) cudaEventDestroy(ctx->ev_stop);
  for (int j = 0; j < darts_ctx::kMaxLanes; ++j) {
    if (ctx->lanes[j]) darts_destroy(ctx->lanes[j]);  // synchronises the lane's stream
    if (ctx->lane_stream[j]) cudaStreamDestroy(ctx->lane_stream[j]);
    if (ctx->ev_join[j]) cudaEventDestroy(ctx->ev_join[j]);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  delete ctx;
  return DARTS_OK;
}

darts_status darts_set_stream(darts_ctx* ctx, void* cuda_stream) {
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)cuda_stream;
  return DARTS_OK;
}

darts_status darts_last_error(const darts_ctx* ctx, char* buf, size_t n) {
  if (!ctx || !buf || n == 0) return DARTS_ERR_INVALID_ARG;
  std::snprintf(buf, n, "%s", ctx->err);
  return DARTS_OK;
}

darts_status darts_sync(darts_ctx* ctx) {
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  // the lanes of darts_render_frames first: each reports (and clears) its own status
  darts_status lane_status = DARTS_OK;
  for (int j = 0; j < darts_ctx::kMaxLanes; ++j) {
    if (!ctx->lanes[j]) continue;
    const darts_status sj = darts_sync(ctx->lanes[j]);
    if (sj != DARTS_OK && lane_status == DARTS_OK) {
      lane_status = sj;
      std::snprintf(ctx->err, sizeof(ctx->err), "frame lane %d: %s", j, ctx->lanes[j]->err);
    }
  }
  if (ctx->copy_stream) CK(cudaStreamSynchronize(ctx->copy_stream), "copy stream synchronize");
  // the status words travel behind the stream's work into pinned memory: one
  // synchronisation, no separate blocking copy
  CK(cudaMemcpyAsync(ctx->status_host, ctx->scratch + 1, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost,
                     ctx->stream), "status read");
  CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  const unsigned int st[2] = {ctx->status_host[0], ctx->status_host[1]};
  if (st[1]) {
    // cleared on the context's stream, so the next launch on it sees the cleared word
    CK(cudaMemsetAsync(reinterpret_cast<unsigned int*>(ctx->scratch + 1) + 1, 0, sizeof(unsigned int), ctx->stream),
       "status clear");
    if (st[1] & 4u) return fail(ctx, DARTS_ERR_BOUNDS, "a device index left its range (access skipped)");
    if (st[1] & 2u) return fail(ctx, DARTS_ERR_TIMEOUT, "a bounded device wait expired");
    return fail(ctx, DARTS_ERR_NUMERIC, "a kernel produced a non-finite contribution");
  }
  return lane_status;
}

darts_status darts_set_kernel_timing(darts_ctx* ctx, int enable) {
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (enable && !ctx->ev_stop) {
    if (!ctx->ev_start) CK(cudaEventCreate(&ctx->ev_start), "event create");
    CK(cudaEventCreate(&ctx->ev_stop), "event create");
  }
  ctx->timing = enable != 0;
  ctx->timed = false;
  return DARTS_OK;
}

darts_status darts_last_kernel_ms(darts_ctx* ctx, float* ms) {
  if (!ctx || !ms) return DARTS_ERR_INVALID_ARG;
  if (!ctx->timed) return fail(ctx, DARTS_ERR_INVALID_ARG, "no timed kernel: enable timing and render first");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(cudaEventSynchronize(ctx->ev_stop), "event synchronize");
  CK(cudaEventElapsedTime(ms, ctx->ev_start, ctx->ev_stop), "event elapsed time");
  return DARTS_OK;
}

darts_status darts_set_launch(darts_ctx* ctx, int block) {
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  if (block != 0 && block != 512 && block != 640 && block != 768 && block != 896)
    return fail(ctx, DARTS_ERR_INVALID_ARG, "block must be 0, 512, 640, 768 or 896");
  ctx->block = block;
  return DARTS_OK;
}

darts_status darts_set_launch_config(darts_ctx* ctx, const darts_launch* cfg) {
  if (!ctx || !cfg) return DARTS_ERR_INVALID_ARG;
  auto batch_ok = [](int b) { return b == 0 || b == 512 || b == 640 || b == 768; };
  if (!(batch_ok(cfg->block) || cfg->block == 896) || !batch_ok(cfg->batch_block))
    return fail(ctx, DARTS_ERR_INVALID_ARG, "block must be 0, 512, 640, 768 or 896; batch_block 0, 512, 640 or 768");
  if (cfg->chunk < 0 || cfg->chunk > 1024 || cfg->batch_items < 0 || cfg->batch_items > 64)
    return fail(ctx, DARTS_ERR_INVALID_ARG, "chunk must be in [0, 1024] and batch_items in [0, 64]");
  ctx->block = cfg->block;
  ctx->chunk = cfg->chunk;
  ctx->batch_block = cfg->batch_block;
  ctx->batch_items = cfg->batch_items;
  return DARTS_OK;
}

darts_status darts_get_launch_config(darts_ctx* ctx, darts_launch* cfg) {
  if (!ctx || !cfg) return DARTS_ERR_INVALID_ARG;
  cfg->block = ctx->block;
  cfg->chunk = ctx->chunk;
  cfg->batch_block = ctx->batch_block;
  cfg->batch_items = ctx->batch_items;
  return DARTS_OK;
}

}  // extern "C"

namespace {
// Total time of `runs` enqueues after one untimed warm-up (CUDA events on
// the context's stream).  `fn` enqueues one render.
template <class F>
darts_status time_enqueues(darts_ctx* ctx, cudaEvent_t e0, cudaEvent_t e1, int runs, F fn, float* total) {
  *total = 0.0f;
  for (int it = 0; it <= runs; ++it) {
    if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "event record");
    const darts_status s = fn();
    if (s != DARTS_OK) return s;
    if (cudaEventRecord(e1, ctx->stream) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "event record");
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return cuda_fail(ctx, cudaGetLastError(), "event timing");
    if (it > 0) *total += ms;
  }
  return DARTS_OK;
}

struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    return e;
  }
  ~EventPair() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

constexpr int kTuneBlocks[4] = {512, 640, 768, 896};  // 896: the DARTS camera kernels only
constexpr int kTuneChunks[5] = {16, 32, 64, 128, 256};
constexpr int kTuneItems[5] = {2, 4, 8, 16, 32};
}  // namespace

extern "C" {

darts_status darts_autotune(darts_ctx* ctx, const darts_scene* scene, const darts_sampling* sampling,
                            int* block_out) {
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  darts_status s = validate(ctx, scene, sampling);
  if (s != DARTS_OK) return s;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const size_t hb = elements_of(scene) * (size_t)scene->gate.n_bins * sizeof(double);
  CK(ensure((void**)&ctx->host_hist, &ctx->host_hist_bytes, 2 * hb), "histogram allocation");
  EventPair ev;
  CK(ev.create(), "event create");
  const int saved_block = ctx->block, saved_chunk = ctx->chunk;
  int best_block = 0, best_chunk = 0;
  float best_ms = 0.0f;
  // a chunk cap above the launch's paths per resident warp changes nothing:
  // those are searched once (the smallest such cap stands for all)
  const uint64_t paths = sampling->paths_per_element * elements_of(scene);
  const bool camera_darts =
      scene->sensor.kind == DARTS_SENSOR_PINHOLE && sampling->method == DARTS_METHOD_DARTS;
  for (int bi = 0; bi < 4 && s == DARTS_OK; ++bi) {
    if (kTuneBlocks[bi] == 896 && !camera_darts) continue;
    bool saturated = false;
    for (int ci = 0; ci < 5 && s == DARTS_OK && !saturated; ++ci) {
      ctx->block = kTuneBlocks[bi];
      ctx->chunk = kTuneChunks[ci];
      saturated = paths <= (uint64_t)kTuneChunks[ci] * ctx->sm_count * (kTuneBlocks[bi] / 32);
      float tot = 0.0f;
      s = time_enqueues(ctx, ev.e0, ev.e1, 3, [&] {
        return darts_render(ctx, scene, sampling, ctx->host_hist, nullptr, 0, nullptr);
      }, &tot);
      // a block size whose shared memory does not fit, or that this scene's
      // kernel is not built for, falls back to another: not a candidate
      if (s == DARTS_OK && ctx->last_block == kTuneBlocks[bi] && (best_block == 0 || tot < best_ms)) {
        best_block = kTuneBlocks[bi];
        best_chunk = kTuneChunks[ci];
        best_ms = tot;
      }
    }
  }
  ctx->block = (s == DARTS_OK && best_block) ? best_block : saved_block;
  ctx->chunk = (s == DARTS_OK && best_block) ? best_chunk : saved_chunk;
  if (block_out) *block_out = ctx->block;
  return s;
}

darts_status darts_autotune_batch(darts_ctx* ctx, int n, const darts_scene* scenes,
                                  const darts_sampling* samplings, double* const* hist_dev,
                                  darts_launch* out) {
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  EventPair ev;
  CK(ev.create(), "event create");
  const int saved_block = ctx->batch_block, saved_items = ctx->batch_items;
  int best_block = 0, best_items = 0;
  float best_ms = 0.0f;
  darts_status s = DARTS_OK;
  for (int bi = 0; bi < 3 && s == DARTS_OK; ++bi) {
    for (int ii = 0; ii < 5 && s == DARTS_OK; ++ii) {
      ctx->batch_block = kTuneBlocks[bi];
      ctx->batch_items = kTuneItems[ii];
      float tot = 0.0f;
      s = time_enqueues(ctx, ev.e0, ev.e1, 2, [&] {
        return darts_render_batch(ctx, n, scenes, samplings, hist_dev, DARTS_BATCH_NO_GRAPH);
      }, &tot);
      if (s == DARTS_OK && (best_block == 0 || tot < best_ms)) {
        best_block = kTuneBlocks[bi];
        best_items = kTuneItems[ii];
        best_ms = tot;
      }
    }
  }
  ctx->batch_block = (s == DARTS_OK && best_block) ? best_block : saved_block;
  ctx->batch_items = (s == DARTS_OK && best_block) ? best_items : saved_items;
  if (out) darts_get_launch_config(ctx, out);
  return s;
}

int32_t darts_table_row_stride(int32_t table_n_mu) { return row_stride_of(table_n_mu); }

darts_status darts_build_table(darts_ctx* ctx, const darts_scene* scene,
                               const darts_sampling* sampling, float* cdf_dev) {
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  darts_status s = validate(ctx, scene, sampling);
  if (s != DARTS_OK) return s;
  if (!cdf_dev) return fail(ctx, DARTS_ERR_INVALID_ARG, "cdf_dev must not be NULL");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  TableParams tp;
  make_table_params(scene, sampling, &tp);
  tp.cdf = cdf_dev;
  if (ctx->timing) CK(cudaEventRecord(ctx->ev_start, ctx->stream), "event record");
  CK(launch_table(tp, ctx->stream), "table kernel launch");
  if (ctx->timing) {  // darts_last_kernel_ms then reports the table kernel
    CK(cudaEventRecord(ctx->ev_stop, ctx->stream), "event record");
    ctx->timed = true;
  }
  return DARTS_OK;
}

darts_status darts_load_table(darts_ctx* ctx, const darts_scene* scene, const darts_sampling* sampling,
                              const float* cdf_dev) {
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  darts_status s = validate(ctx, scene, sampling);
  if (s != DARTS_OK) return s;
  if (!cdf_dev) return fail(ctx, DARTS_ERR_INVALID_ARG, "cdf_dev must not be NULL");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const size_t bytes = (size_t)sampling->table_n_rho * sampling->table_n_s *
                       row_stride_of(sampling->table_n_mu) * sizeof(float);
  CK(ensure((void**)&ctx->table, &ctx->table_bytes, bytes), "table allocation");
  CK(cudaMemcpyAsync(ctx->table, cdf_dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream), "table copy");
  table_key(scene, sampling, ctx->table_key);
  ctx->table_valid = true;
  return DARTS_OK;
}

darts_status darts_render(darts_ctx* ctx, const darts_scene* scene, const darts_sampling* sampling,
                          double* hist_dev, double* sumsq_dev, uint64_t path_offset,
                          const darts_probe* probe) {
  const Range nvtx_range("darts_render");
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  darts_status s = validate(ctx, scene, sampling);
  if (s != DARTS_OK) return s;
  if (!hist_dev) return fail(ctx, DARTS_ERR_INVALID_ARG, "hist_dev must not be NULL");
  if (probe && (probe->stride == 0 || (probe->count && (!probe->contrib_dev || !probe->bin_dev))))
    return fail(ctx, DARTS_ERR_INVALID_ARG, "probe needs stride >= 1 and output buffers");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const size_t hb = elements_of(scene) * (size_t)scene->gate.n_bins * sizeof(double);
  const bool acc = (sampling->flags & DARTS_FLAG_ACCUMULATE) != 0;
  if (sampling->paths_per_element == 0) {
    if (!acc) CK(cudaMemsetAsync(hist_dev, 0, hb, ctx->stream), "memset");
    if (sumsq_dev && !acc) CK(cudaMemsetAsync(sumsq_dev, 0, hb, ctx->stream), "memset");
    CK(cudaMemsetAsync(ctx->scratch, 0, sizeof(unsigned long long), ctx->stream), "memset");
    CK(cudaMemsetAsync(ctx->scratch + 2, 0, kStatCount * sizeof(unsigned long long), ctx->stream), "memset");
    ctx->last_paths = 0;
    return DARTS_OK;
  }
  ZeroSpec z;  // the outputs are zeroed unless the render adds into them
  z.a = acc ? nullptr : hist_dev;
  z.b = acc ? nullptr : sumsq_dev;
  z.n = elements_of(scene) * (unsigned long long)scene->gate.n_bins;
  if (uses_table(sampling->method)) {
    s = ensure_table(ctx, scene, sampling, &z);
    if (s != DARTS_OK) return s;
  }
  TraceParams P;
  make_trace_params(ctx, scene, sampling, &P);
  P.N = sampling->paths_per_element * elements_of(scene);
  P.path_offset = path_offset;
  P.hist = hist_dev;
  P.sumsq = sumsq_dev;
  if (probe && probe->count) {
    P.probe_first = probe->first;
    P.probe_stride = probe->stride;
    P.probe_count = probe->count;
    P.probe_c = probe->contrib_dev;
    P.probe_b = probe->bin_dev;
  }
  return run_trace(ctx, scene, sampling, P, false, z.zeroed);
}

darts_status darts_render_host(darts_ctx* ctx, const darts_scene* scene,
                               const darts_sampling* sampling, double* hist_host,
                               double* sumsq_host, uint64_t path_offset) {
  const Range nvtx_range("darts_render_host");
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  if (!hist_host) return fail(ctx, DARTS_ERR_INVALID_ARG, "hist_host must not be NULL");
  darts_status s = validate(ctx, scene, sampling);
  if (s != DARTS_OK) return s;
  if (sampling->flags & DARTS_FLAG_ACCUMULATE)
    return fail(ctx, DARTS_ERR_UNSUPPORTED, "DARTS_FLAG_ACCUMULATE applies to darts_render's device outputs");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const size_t nh = elements_of(scene) * (size_t)scene->gate.n_bins;
  const size_t hb = nh * sizeof(double);
  CK(ensure((void**)&ctx->host_hist, &ctx->host_hist_bytes, 2 * hb), "histogram allocation");
  s = darts_render(ctx, scene, sampling, ctx->host_hist, sumsq_host ? ctx->host_hist + nh : nullptr, path_offset,
                   nullptr);
  if (s != DARTS_OK) return s;
  CK(cudaMemcpyAsync(hist_host, ctx->host_hist, hb, cudaMemcpyDeviceToHost, ctx->stream), "histogram copy");
  if (sumsq_host)
    CK(cudaMemcpyAsync(sumsq_host, ctx->host_hist + nh, hb, cudaMemcpyDeviceToHost, ctx->stream), "histogram copy");
  return darts_sync(ctx);
}

darts_status darts_render_host_async(darts_ctx* ctx, const darts_scene* scene,
                                     const darts_sampling* sampling, double* hist_host,
                                     double* sumsq_host, uint64_t path_offset) {
  const Range nvtx_range("darts_render_host_async");
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  if (!hist_host) return fail(ctx, DARTS_ERR_INVALID_ARG, "hist_host must not be NULL");
  darts_status s = validate(ctx, scene, sampling);
  if (s != DARTS_OK) return s;
  if (sampling->flags & DARTS_FLAG_ACCUMULATE)
    return fail(ctx, DARTS_ERR_UNSUPPORTED, "DARTS_FLAG_ACCUMULATE applies to darts_render's device outputs");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  // created on first use; a creation that failed part way is completed by the next call
  if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking), "copy stream");
  for (int i = 0; i < 2; ++i) {
    if (!ctx->ev_rendered[i]) CK(cudaEventCreateWithFlags(&ctx->ev_rendered[i], cudaEventDisableTiming), "event");
    if (!ctx->ev_copied[i]) CK(cudaEventCreateWithFlags(&ctx->ev_copied[i], cudaEventDisableTiming), "event");
  }
  const int k = ctx->async_slot;
  const size_t nh = elements_of(scene) * (size_t)scene->gate.n_bins;
  const size_t hb = nh * sizeof(double);
  if (2 * hb > ctx->async_bytes[k]) {  // growing: nothing may still read the old buffer
    CK(cudaStreamSynchronize(ctx->copy_stream), "copy stream synchronize");
    CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    ctx->copied_pending[k] = false;
    CK(ensure((void**)&ctx->async_hist[k], &ctx->async_bytes[k], 2 * hb), "histogram allocation");
  }
  // the copy that last read this buffer (two calls ago) precedes the render into it
  if (ctx->copied_pending[k]) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_copied[k], 0), "stream wait");
  double* dev = ctx->async_hist[k];
  s = darts_render(ctx, scene, sampling, dev, sumsq_host ? dev + nh : nullptr, path_offset, nullptr);
  if (s != DARTS_OK) return s;
  CK(cudaEventRecord(ctx->ev_rendered[k], ctx->stream), "event record");
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_rendered[k], 0), "stream wait");
  CK(cudaMemcpyAsync(hist_host, dev, hb, cudaMemcpyDeviceToHost, ctx->copy_stream), "histogram copy");
  if (sumsq_host)
    CK(cudaMemcpyAsync(sumsq_host, dev + nh, hb, cudaMemcpyDeviceToHost, ctx->copy_stream), "histogram copy");
  CK(cudaEventRecord(ctx->ev_copied[k], ctx->copy_stream), "event record");
  ctx->copied_pending[k] = true;
  ctx->async_slot = k ^ 1;
  return DARTS_OK;
}

darts_status darts_render_frames(darts_ctx* ctx, const darts_scene* scene, const darts_sampling* sampling,
                                 uint32_t n_frames, double* const* hist_dev, double* const* sumsq_dev,
                                 uint64_t path_offset, int32_t in_flight) {
  const Range nvtx_range("darts_render_frames");
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  darts_status s = validate(ctx, scene, sampling);
  if (s != DARTS_OK) return s;
  if (n_frames == 0 || !hist_dev) return fail(ctx, DARTS_ERR_INVALID_ARG, "need n_frames >= 1 and outputs");
  if (in_flight < 1 || in_flight > darts_ctx::kMaxLanes)
    return fail(ctx, DARTS_ERR_INVALID_ARG, "in_flight must be in 1..%d", darts_ctx::kMaxLanes);
  if (sampling->flags & DARTS_FLAG_ACCUMULATE)
    return fail(ctx, DARTS_ERR_UNSUPPORTED, "darts_render_frames overwrites its outputs");
  for (uint32_t i = 0; i < n_frames; ++i)
    if (!hist_dev[i] || (sumsq_dev && !sumsq_dev[i]))
      return fail(ctx, DARTS_ERR_INVALID_ARG, "frame %u: NULL output", i);
  const uint64_t N = sampling->paths_per_element * elements_of(scene);
  if (N > 0 && (uint64_t)(n_frames - 1) > (UINT64_MAX - path_offset) / N)
    return fail(ctx, DARTS_ERR_INVALID_ARG, "path ids of the last frame exceed 2^64");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const int lanes = (int)std::min<uint32_t>((uint32_t)in_flight, n_frames);
  for (int j = 0; j < lanes; ++j) {  // created on first use and kept
    if (!ctx->lane_stream[j])
      CK(cudaStreamCreateWithFlags(&ctx->lane_stream[j], cudaStreamNonBlocking), "lane stream");
    if (!ctx->ev_join[j]) CK(cudaEventCreateWithFlags(&ctx->ev_join[j], cudaEventDisableTiming), "event");
    if (!ctx->lanes[j]) {
      const darts_status c = darts_create(&ctx->lanes[j], ctx->device, ctx->lane_stream[j]);
      if (c != DARTS_OK) return fail(ctx, c, "frame lane %d: context creation failed", j);
    }
    ctx->lanes[j]->block = ctx->block;
  }
  if (!ctx->ev_fork) CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming), "event");
  CK(cudaEventRecord(ctx->ev_fork, ctx->stream), "event record");
  for (int j = 0; j < lanes; ++j) CK(cudaStreamWaitEvent(ctx->lane_stream[j], ctx->ev_fork, 0), "stream wait");
  darts_status r = DARTS_OK;
  for (uint32_t i = 0; i < n_frames && r == DARTS_OK; ++i) {
    darts_ctx* lane = ctx->lanes[i % (uint32_t)lanes];
    r = darts_render(lane, scene, sampling, hist_dev[i], sumsq_dev ? sumsq_dev[i] : nullptr, path_offset + i * N,
                     nullptr);
    if (r != DARTS_OK) std::snprintf(ctx->err, sizeof(ctx->err), "frame %u: %s", i, lane->err);
  }
  // joined even after a failed enqueue: later work on the context's stream
  // waits for every frame that was enqueued
  for (int j = 0; j < lanes; ++j) {
    CK(cudaEventRecord(ctx->ev_join[j], ctx->lane_stream[j]), "event record");
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join[j], 0), "stream wait");
  }
  return r;
}

darts_status darts_get_stats(darts_ctx* ctx, darts_stats* out) {
  if (!ctx || !out) return DARTS_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  unsigned long long v[2 + kStatCount];
  CK(cudaMemcpy(v, ctx->scratch, sizeof(v), cudaMemcpyDeviceToHost), "stats read");
  const unsigned long long* s = v + 2;
  out->paths = ctx->last_paths;  // every launched path is traced to its end
  out->vertices = s[0];
  out->connections_nonempty = s[1];
  out->distance_steps = s[2];
  out->early_exits = s[3];
  out->all_invalid = s[4];
  out->escapes = s[5];
  out->fp64_ellipse = s[10];
  out->fp64_phi = s[11];
  // the specialised DARTS kernel counts no samples: they are its non-empty
  // connections, and none can fall outside its bin
  out->samples = ctx->last_fast ? s[1] : s[6] + s[7];
  out->rejected = ctx->last_fast ? 0 : s[8] + s[9];
  return DARTS_OK;
}

// FNV-1a over bytes (graph cache key).
static uint64_t fnv1a(const void* data, size_t n, uint64_t h) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}

darts_status darts_render_batch(darts_ctx* ctx, int n, const darts_scene* scenes,
                                const darts_sampling* samplings, double* const* hist_dev,
                                uint32_t flags) {
  const Range nvtx_range("darts_render_batch");
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  if (n < 1 || !scenes || !samplings || !hist_dev)
    return fail(ctx, DARTS_ERR_INVALID_ARG, "need n >= 1 media, scenes, samplings and outputs");
  const darts_sampling& s0 = samplings[0];
  int max_bins = 1;
  for (int i = 0; i < n; ++i) {
    darts_status st = validate(ctx, &scenes[i], &samplings[i]);
    if (st != DARTS_OK) return st;
    if (!hist_dev[i]) return fail(ctx, DARTS_ERR_INVALID_ARG, "hist_dev[%d] is NULL", i);
    if (scenes[i].gate.weights)
      return fail(ctx, DARTS_ERR_UNSUPPORTED, "a batch renders media without a temporal response");
    if (samplings[i].flags & (kRisVariantFlags | DARTS_FLAG_ACCUMULATE))
      return fail(ctx, DARTS_ERR_UNSUPPORTED, "a batch runs the default RIS and overwrites its outputs");
    const darts_sampling& si = samplings[i];
    if (general_scene(&scenes[i]))
      return fail(ctx, DARTS_ERR_UNSUPPORTED, "a batch renders point-emitter, point-sensor media without surfaces");
    if (si.method != DARTS_METHOD_DARTS || si.ris_m != 8 || si.table_n_rho != s0.table_n_rho ||
        si.table_n_s != s0.table_n_s || si.table_n_mu != s0.table_n_mu)
      return fail(ctx, DARTS_ERR_UNSUPPORTED,
                  "a batch needs method DARTS, ris_m 8 and one table shape for all media");
    max_bins = std::max(max_bins, scenes[i].gate.n_bins);
  }
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const int rows = s0.table_n_rho * s0.table_n_s, stride = row_stride_of(s0.table_n_mu);
  const size_t tab_floats = (size_t)rows * stride;
  CK(ensure((void**)&ctx->batch_tables, &ctx->batch_tables_bytes, (size_t)n * tab_floats * sizeof(float)),
     "batch table allocation");

  // Work items.  A CTA traces an item alone, so items are sized by estimated
  // cost: per-path cost ~ 1 + sigma_s x box diagonal (the expected vertices of
  // a path grow with the optical size), and a medium is cut into chunks of
  // about 1/8 of a CTA's share of the total, between 2^11 and 2^16 paths, so
  // that no single item outlasts the rest of the launch.
  std::vector<double> cpp(n);
  double total_cost = 0.0;
  for (int i = 0; i < n; ++i) {
    const darts_geometry& g = scenes[i].geom;
    double diag = 0.0;
    for (int a = 0; a < 3; ++a) diag += (g.hi[a] - g.lo[a]) * (g.hi[a] - g.lo[a]);
    cpp[i] = 1.0 + scenes[i].medium.sigma_s * std::sqrt(diag);
    total_cost += cpp[i] * (double)samplings[i].paths_per_element;
  }
  const double items_per_cta = ctx->batch_items ? (double)ctx->batch_items : 8.0;
  const double item_cost = total_cost / (items_per_cta * std::max(ctx->sm_count, 1));
  std::vector<uint64_t> chunk(n);
  size_t n_items = 0;
  for (int i = 0; i < n; ++i) {
    const double c = std::floor(item_cost / cpp[i]);
    chunk[i] = (uint64_t)std::min(65536.0, std::max(2048.0, c));
    n_items += (samplings[i].paths_per_element + chunk[i] - 1) / chunk[i];
  }
  const size_t off_tp = 0, off_trp = ((size_t)n * sizeof(TableParams) + 255) / 256 * 256;
  const size_t off_items = off_trp + ((size_t)n * sizeof(TraceParams) + 255) / 256 * 256;
  const size_t off_cnt = off_items + (n_items * sizeof(BatchItem) + 255) / 256 * 256;
  const size_t total = off_cnt + 256;
  CK(ensure(&ctx->batch_buf, &ctx->batch_buf_bytes, total), "batch buffer allocation");
  unsigned char* host = static_cast<unsigned char*>(std::malloc(total));
  if (!host) return fail(ctx, DARTS_ERR_OOM, "host staging buffer");
  std::memset(host, 0, total);
  unsigned char* dev = static_cast<unsigned char*>(ctx->batch_buf);
  TableParams* tps = reinterpret_cast<TableParams*>(host + off_tp);
  TraceParams* trps = reinterpret_cast<TraceParams*>(host + off_trp);
  BatchItem* items = reinterpret_cast<BatchItem*>(host + off_items);
  size_t k = 0;
  uint64_t total_paths = 0;
  // Media in order of decreasing total estimated cost (heavy media start
  // early, light ones fill the tail); the items of one medium stay contiguous
  // so that a CTA restages a table only when the medium changes.
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return cpp[a] * (double)samplings[a].paths_per_element > cpp[b] * (double)samplings[b].paths_per_element;
  });
  for (int i = 0; i < n; ++i) {
    make_table_params(&scenes[i], &samplings[i], &tps[i]);
    tps[i].cdf = ctx->batch_tables + (size_t)i * tab_floats;
    make_trace_params(ctx, &scenes[i], &samplings[i], &trps[i]);
    trps[i].table = ctx->batch_tables + (size_t)i * tab_floats;
    trps[i].N = samplings[i].paths_per_element;
    trps[i].path_offset = 0;
    trps[i].bin_base = trps[i].o_e % (unsigned long long)scenes[i].gate.n_bins;
    trps[i].hist = hist_dev[i];
    total_paths += samplings[i].paths_per_element;
  }
  for (int oi = 0; oi < n; ++oi) {
    const int i = order[oi];
    for (uint64_t f = 0; f < samplings[i].paths_per_element; f += chunk[i]) {
      items[k].medium = (unsigned)i;
      items[k].first = f;
      items[k].count = std::min<uint64_t>(chunk[i], samplings[i].paths_per_element - f);
      ++k;
    }
  }
  BatchParams bp;
  bp.params = reinterpret_cast<const TraceParams*>(dev + off_trp);
  bp.items = reinterpret_cast<const BatchItem*>(dev + off_items);
  bp.n_items = (int)n_items;
  bp.n_media = n;
  bp.item_counter = reinterpret_cast<unsigned int*>(dev + off_cnt);
  bp.max_bins = max_bins;
  bp.rows = rows;
  bp.row_stride = stride;
  bp.stats = ctx->scratch + 2;
  int block = ctx->batch_block ? ctx->batch_block : 768;  // 24 warps per SM unless tuned
  size_t smem = batch_smem_bytes(bp, block);
  while (smem > (size_t)ctx->smem_optin && block > 512) {
    block = block == 768 ? 640 : 512;
    smem = batch_smem_bytes(bp, block);
  }
  if (smem > (size_t)ctx->smem_optin) {
    std::free(host);
    return fail(ctx, DARTS_ERR_UNSUPPORTED, "batch shared memory of %zu bytes does not fit", smem);
  }
  uint64_t key = fnv1a(host, total, 1469598103934665603ull);
  key = fnv1a(&bp, sizeof(bp), key);
  key = fnv1a(&block, sizeof(block), key);
  // upload (outside any capture), then run the captured graph
  cudaError_t e = cudaMemcpyAsync(dev, host, off_cnt, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // host buffer is freed next
  std::free(host);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch upload");
  ctx->last_paths = total_paths;
  ctx->last_fast = true;
  const bool use_graph = !(flags & DARTS_BATCH_NO_GRAPH);
  auto enqueue = [&](cudaStream_t st) -> cudaError_t {
    cudaError_t r = cudaMemsetAsync(dev + off_cnt, 0, 256, st);
    if (r == cudaSuccess) r = cudaMemsetAsync(ctx->scratch, 0, (2 + kStatCount) * sizeof(unsigned long long), st);
    if (r == cudaSuccess) r = launch_table_batch(reinterpret_cast<const TableParams*>(dev + off_tp), n, rows, st);
    if (r == cudaSuccess) r = launch_batch(bp, ctx->sm_count, block, smem, st);
    return r;
  };
  if (!use_graph) {
    CK(enqueue(ctx->stream), "batch launch");
    return DARTS_OK;
  }
  if (!ctx->graph_exec || ctx->graph_key != key) {
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->graph_exec = nullptr;
    ctx->graph = nullptr;
    if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking), "stream create");
    CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t r = enqueue(ctx->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t r2 = cudaStreamEndCapture(ctx->capture_stream, &g);
    if (r != cudaSuccess || r2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(ctx, r != cudaSuccess ? r : r2, "batch graph capture");
    }
    ctx->graph = g;
    CK(cudaGraphInstantiate(&ctx->graph_exec, g, 0), "graph instantiate");
    ctx->graph_key = key;
  }
  CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream), "graph launch");
  return DARTS_OK;
}

darts_status darts_adjoint(darts_ctx* ctx, const darts_scene* scene, const darts_sampling* sampling,
                           const double* dLdh_dev, double* grad3_dev, double* grad3_sq_dev,
                           uint64_t path_offset) {
  const Range nvtx_range("darts_adjoint");
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  darts_status s = validate(ctx, scene, sampling);
  if (s != DARTS_OK) return s;
  if (!dLdh_dev || !grad3_dev) return fail(ctx, DARTS_ERR_INVALID_ARG, "dLdh_dev and grad3_dev must not be NULL");
  if (sampling->method != DARTS_METHOD_DARTS)
    return fail(ctx, DARTS_ERR_UNSUPPORTED, "the adjoint is implemented for the DARTS method");
  if (sampling->flags & (kRisVariantFlags | DARTS_FLAG_ACCUMULATE))
    return fail(ctx, DARTS_ERR_UNSUPPORTED, "the adjoint runs the default RIS and overwrites grad3");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (sampling->paths_per_element == 0) {
    CK(cudaMemsetAsync(grad3_dev, 0, 3 * sizeof(double), ctx->stream), "memset");
    if (grad3_sq_dev) CK(cudaMemsetAsync(grad3_sq_dev, 0, 3 * sizeof(double), ctx->stream), "memset");
    return DARTS_OK;
  }
  s = ensure_table(ctx, scene, sampling);
  if (s != DARTS_OK) return s;
  TraceParams P;
  make_trace_params(ctx, scene, sampling, &P);
  P.N = sampling->paths_per_element * elements_of(scene);
  P.path_offset = path_offset;
  P.dLdh = dLdh_dev;
  P.grad3 = grad3_dev;
  P.grad3_sq = grad3_sq_dev;
  const int grid = ctx->sm_count;
  const size_t smem = adjoint_smem_bytes(P);
  if (smem > (size_t)ctx->smem_optin)
    return fail(ctx, DARTS_ERR_UNSUPPORTED, "direction table of %zu bytes exceeds shared memory", smem);
  CK(ensure((void**)&ctx->partials, &ctx->partials_bytes, (size_t)grid * 6 * sizeof(double)), "partials allocation");
  P.partials = ctx->partials;
  CK(cudaMemsetAsync(ctx->scratch, 0, sizeof(unsigned long long), ctx->stream), "memset");
  CK(cudaMemsetAsync(ctx->scratch + 2, 0, kStatCount * sizeof(unsigned long long), ctx->stream), "memset");
  ctx->last_paths = P.N;
  {
    const darts_status sw = set_weights(ctx, scene, sampling, P);
    if (sw != DARTS_OK) return sw;
  }
  ctx->last_fast = !P.general;
  CK(launch_adjoint(P, grid, smem, ctx->stream), "adjoint kernel launch");
  return DARTS_OK;
}

darts_status darts_debug_paths(darts_ctx* ctx, const darts_scene* scene,
                               const darts_sampling* sampling, uint64_t first, uint32_t count,
                               float* contrib_dev, int32_t* bin_dev, int32_t* nvert_dev,
                               uint8_t* decisions_dev) {
  if (!ctx) return DARTS_ERR_INVALID_ARG;
  darts_status s = validate(ctx, scene, sampling);
  if (s != DARTS_OK) return s;
  if (!contrib_dev || !bin_dev || !nvert_dev || !decisions_dev)
    return fail(ctx, DARTS_ERR_INVALID_ARG, "debug outputs must not be NULL");
  if (count == 0) return DARTS_OK;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (uses_table(sampling->method)) {
    s = ensure_table(ctx, scene, sampling);
    if (s != DARTS_OK) return s;
  }
  TraceParams P;
  make_trace_params(ctx, scene, sampling, &P);
  P.N = count;
  P.path_offset = first;
  CK(ensure((void**)&ctx->host_hist, &ctx->host_hist_bytes,
            2 * elements_of(scene) * (size_t)scene->gate.n_bins * sizeof(double)),
     "histogram allocation");
  P.hist = ctx->host_hist;
  P.sumsq = nullptr;
  P.dbg_c = contrib_dev;
  P.dbg_b = bin_dev;
  P.dbg_n = nvert_dev;
  P.dbg_dec = decisions_dev;
  CK(cudaMemsetAsync(decisions_dev, 0xFF, (size_t)count * sampling->max_bounces * 4, ctx->stream), "memset");
  return run_trace(ctx, scene, sampling, P, true);
}

darts_status darts_debug_philox(darts_ctx* ctx, const uint32_t* ctr_dev, uint64_t seed, uint32_t n,
                                uint32_t* out_dev) {
  if (!ctx || (n && (!ctr_dev || !out_dev))) return DARTS_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(launch_philox(ctr_dev, (uint32_t)seed, (uint32_t)(seed >> 32), n, out_dev, ctx->stream), "philox launch");
  return DARTS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free rendering.
//
// Some callers cannot call cudaMalloc: plug-ins hosted by an application that
// reserves all device memory up front in its own pool and forbids libraries
// from allocating behind its back, or pipelines that must not allocate after
// start-up.  darts_create() allocates the context's scratch, so those callers
// cannot use darts_render().  darts_render_static() takes its scratch (path
// counter, statistics, direction table, block partials) from one file-scope
// device array instead; the caller passes only the histogram buffers.
//
// The array lives in every GPU that loads this library until the process
// exits.  In host code its name is only a host-side stand-in for the device
// variable, so the device address is looked up with cudaGetSymbolAddress()
// once per device (with that device current) on the first call there, and
// that address is what the kernels receive.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = 4u << 20;   // 4 MiB per device
constexpr size_t kStaticHeaderBytes = 256;         // counter, ticket, status, statistics
constexpr size_t kStaticTableBytes = 256u << 10;   // direction table, up to 65536 floats
constexpr size_t kStaticPartialBytes = kStaticScratchBytes - kStaticHeaderBytes - kStaticTableBytes;
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct StaticDevice {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_static_scratch
  int sm_count = 0;
  int smem_optin = 0;
};
StaticDevice g_static_dev[kStaticMaxDevices];
std::mutex g_static_mutex;

// A failed CUDA call of the static path: the runtime's last error is taken
// here, as cuda_fail does for context calls, so that it cannot resurface at a
// later, valid launch on this thread.
darts_status static_cuda_fail(cudaError_t e) {
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? DARTS_ERR_OOM : DARTS_ERR_CUDA;
}

// Per-device set-up: device address of the scratch array and launch limits.
cudaError_t static_setup(int dev, StaticDevice** out) {
  std::lock_guard<std::mutex> lock(g_static_mutex);
  StaticDevice& d = g_static_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    d.smem_optin -= 1024;
    d.base = static_cast<unsigned char*>(p);
    d.ready = true;
  }
  *out = &d;
  return cudaSuccess;
}

}  // namespace

extern "C" darts_status darts_render_static(const darts_scene* scene, const darts_sampling* sampling,
                                            double* hist_dev, double* sumsq_dev, uint64_t path_offset,
                                            void* cuda_stream) {
  darts_ctx tmp;  // stack only: carries the launch settings, owns nothing
  darts_ctx* ctx = &tmp;
  darts_status s = validate(ctx, scene, sampling);
  if (s != DARTS_OK) return s;
  if (!hist_dev) return DARTS_ERR_INVALID_ARG;
  if (scene->gate.weights) return DARTS_ERR_UNSUPPORTED;  // no scratch for the weight tables
  if (sampling->flags & DARTS_FLAG_ACCUMULATE) return DARTS_ERR_UNSUPPORTED;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_cuda_fail(e);
  if (dev < 0 || dev >= kStaticMaxDevices) return DARTS_ERR_UNSUPPORTED;
  StaticDevice* sd = nullptr;
  e = static_setup(dev, &sd);
  if (e != cudaSuccess) return static_cuda_fail(e);
  const cudaStream_t stream = (cudaStream_t)cuda_stream;
  const int B = scene->gate.n_bins;
  const size_t hb = elements_of(scene) * (size_t)B * sizeof(double);
  unsigned long long* header = reinterpret_cast<unsigned long long*>(sd->base);
  float* table = reinterpret_cast<float*>(sd->base + kStaticHeaderBytes);
  double* partials = reinterpret_cast<double*>(sd->base + kStaticHeaderBytes + kStaticTableBytes);

  tmp.device = dev;
  tmp.stream = stream;
  tmp.sm_count = sd->sm_count;
  tmp.smem_optin = sd->smem_optin;
  tmp.scratch = header;
  tmp.table = table;

  // Every size check comes before the first enqueued operation: a refused
  // request leaves the stream, the outputs and the scratch untouched.
  const bool with_table = uses_table(sampling->method);
  const size_t table_bytes = (size_t)sampling->table_n_rho * sampling->table_n_s *
                             row_stride_of(sampling->table_n_mu) * sizeof(float);
  if (with_table && table_bytes > kStaticTableBytes) return DARTS_ERR_UNSUPPORTED;
  TraceParams P;
  make_trace_params(ctx, scene, sampling, &P);
  P.N = sampling->paths_per_element * elements_of(scene);
  P.path_offset = path_offset;
  P.hist = hist_dev;
  P.sumsq = sumsq_dev;
  P.partials = partials;
  int block;
  bool tile;
  size_t smem;
  choose_launch(&tmp, sampling, P, false, &block, &tile, &smem);
  if (smem > (size_t)tmp.smem_optin) return DARTS_ERR_UNSUPPORTED;
  // block partials are used only by the shared-memory tiles of a point sensor
  const size_t partial_bytes = (size_t)sd->sm_count * 2 * (size_t)B * sizeof(double);
  if (tile && partial_bytes > kStaticPartialBytes) return DARTS_ERR_UNSUPPORTED;

  // the array keeps the previous call's contents: reset counter, ticket, status, statistics
  e = cudaMemsetAsync(header, 0, kStaticHeaderBytes, stream);
  if (e != cudaSuccess) return static_cuda_fail(e);
  if (sampling->paths_per_element == 0 || !tile) {  // zero outputs: empty render, or FP64 atomics into them
    e = cudaMemsetAsync(hist_dev, 0, hb, stream);
    if (e == cudaSuccess && sumsq_dev) e = cudaMemsetAsync(sumsq_dev, 0, hb, stream);
    if (e != cudaSuccess) return static_cuda_fail(e);
    if (sampling->paths_per_element == 0) return DARTS_OK;
  }
  if (with_table) {
    TableParams tp;
    make_table_params(scene, sampling, &tp);
    tp.cdf = table;
    e = launch_table(tp, stream);
    if (e != cudaSuccess) return static_cuda_fail(e);
  }
  e = launch_trace(sampling->method, P, tmp.sm_count, block, false, tile, smem, stream);
  if (e != cudaSuccess) return static_cuda_fail(e);
  return DARTS_OK;
}
