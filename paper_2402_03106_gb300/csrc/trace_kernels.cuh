// trace_kernels.cuh -- device code of the persistent path-tracing kernels
// (DARTS, its full-gate form, the two baselines, the general-scene variant),
// included by trace.cu and trace_var.cu, which instantiate and launch them.
//
// One CTA per SM.  Every lane of a warp carries one path; a warp executes one
// vertex step for all its live lanes per iteration and refills lanes whose
// path ended from a warp-private pool of path ids (ballot + popc; one global
// atomicAdd per kPathChunk paths), so early-terminating paths (Sec. 5.2 early
// exit, escapes) do not idle their lanes.
//
// DARTS vertex step (Sec. 4-5), vertex k at x_k with elapsed length L:
//   1. C = |x_e - x_k|, S_M = v (T_M - t0) - L, S_m = v (T_m - t0) - L;
//      stop if S_M <= C (no causal continuation, Sec. 5.2).
//   2. direction: one-sample MIS (Eq. 19) of the elliptical DA table row of
//      (C/S_M, S_M) (inverse CDF on the cos bins staged in shared memory) and
//      HG about the previous direction (uniform sphere at the sensor).
//   3. control vertex on the ray: S ~ truncated exponential on
//      [max(S_m, C), min(S_M, S(d_m))) (Eq. 21, medium boundary as the cap),
//      t from Eq. 18 in a cancellation-free form, density p(S) (dt/dS)^-1
//      (Eq. 22); the contribution is accumulated in a register.
//   4. distance: medium event with p_m = 1 - exp(-sigma_t d_m) (Eq. 12), then
//      RIS over M truncated-exponential candidates (Eq. 13-14) from one row of
//      the base-2 radical-inverse table shifted by eps0, weighted by the DA
//      flux Phi(x_j, (S_M - d_j)/v) (Eq. 9-10) in log space, zero when
//      non-causal; throughput albedo * mean(Phi) / Phi_sel (Eq. 15).
// A DARTS path is dedicated to one time bin (Sec. 6.2) and commits once, at
// its end, into a warp-private Kahan tile in shared memory; baseline paths
// commit each contribution to the bin of its time.  Tiles are reduced in FP64
// per block; the last block to finish sums the block partials in fixed order.
#pragma once
#include <algorithm>
#include <atomic>
#include <type_traits>
#include <cfloat>

#include "darts_device.cuh"
#include "darts_internal.h"

namespace darts {
namespace {

constexpr int kMaxM = 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

enum : int { kDarts = 0, kPlain = 1, kVanilla = 2, kDartsFull = 3 };
// DARTS samplers (DA-RIS distances, EDA/MIS directions, truncated-exponential
// control vertices).  kDartsFull targets the whole gate and commits every
// connection to the bin of its own time (weight 1/N_e) instead of dedicating
// the path to one bin.
template <int M>
constexpr bool kIsDartsM = M == kDarts || M == kDartsFull;
enum : int { EV_NONE = 0, EV_EARLY = 1, EV_SCATTER = 2, EV_ESCAPE = 3, EV_INVALID = 4, EV_MAXDEPTH = 5,
             EV_SURFACE = 6 };
// stats slots (after `paths`)
// Event counters.  SAMPLE / REJECT: connection samples with a time, and
// those whose time has zero temporal weight (outside the gate, a zero-weight
// bin, or outside a DARTS path's bin); the second pair counts surface
// connections of a step that also made a control-vertex connection.  The
// specialised DARTS kernel (point sensor, no surfaces) does not count them:
// its samples are its non-empty connections and none is rejected.
enum : int { ST_VERT = 0, ST_CONN = 1, ST_DIST = 2, ST_EARLY = 3, ST_INVALID = 4, ST_ESCAPE = 5,
             ST_SAMPLE = 6, ST_SAMPLE2 = 7, ST_REJECT = 8, ST_REJECT2 = 9,
             ST_FP64E = 10, ST_FP64P = 11 };
static_assert(ST_FP64P + 1 == kStatCount, "statistics layout");

struct Path {
  float x, y, z;     // current vertex
  float wx, wy, wz;  // previous direction (DARTS) / current walk direction (baselines)
  float L, Lc;       // elapsed length, Kahan compensation
  float beta;        // throughput weight
  float c;           // DARTS: summed contribution of the path
  float SM0, Sm0;    // DARTS: v (T_M - t0), v (T_m - t0) of the path's bin
  int k;             // vertex index
  int bin;           // DARTS bin
  unsigned long long j;  // local path index
  // path-replay adjoint: sum over the path's connections of c_v * s_v, and
  // the running sum of d log HG / dg over the walk vertices
  float a0, a1, a2, gsum;
  // general scenes: the path's emitter point and normal (0 for a point
  // emitter), its intensity scale and gate bounds, the sensor element, the
  // medium scattering vertices so far, and whether the direction of the
  // current vertex is already fixed (camera ray, surface bounce)
  float ey0, ey1, ey2, en0, en1, en2, ie, s_hi_e;
  int elem, nmed;
  int surf;          // sphere the current vertex lies on, -1 otherwise
  float salb;        // EDA at surfaces: albedo of the surface the vertex lies on (0: none);
                     // the previous direction (wx, wy, wz) then holds its normal
  bool fixed, miss;
  // full-gate DARTS: the step's control-vertex and surface contributions
  // (flat bin, value; bin -1 when none)
  int cb, cb2;
  float cv, cv2;
};

// Event counting.  Common events set a bit for the current vertex step; the
// warp turns the bits into counts with ballots once per step (no per-lane
// counter registers).  Rare FP64 events go straight to block counters in
// shared memory.
__shared__ unsigned long long s_rare[2];

// Branches a path takes at most once (early exits, the last vertex) or
// almost never (non-finite values, probes, FP64 fallbacks): laid out away
// from the hot loop so that its instructions stay dense in the cache.
#define DARTS_RARE(x) __builtin_expect(!!(x), 0)

// Checked builds (-DDARTS_CHECKS, libdarts_checked.so): every index into an
// output, a tile or the table is tested; one out of range sets status bit 2
// (reported as DARTS_ERR_BOUNDS by darts_sync) and the access is skipped.
// The production build compiles the tests away.
#ifdef DARTS_CHECKS
__device__ __forceinline__ bool index_ok(const TraceParams& P, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  atomicOr(P.status, 4u);
  return false;
}
#define DARTS_INDEX_OK(P, i, n) index_ok((P), (long long)(i), (long long)(n))
#else
#define DARTS_INDEX_OK(P, i, n) true
#endif

struct Counters {
  unsigned bits;
  __device__ __forceinline__ void add(int slot) { bits |= 1u << slot; }
  __device__ __forceinline__ void add_rare(int slot) {
    atomicAdd(&s_rare[slot - ST_FP64E], 1ull);
  }
};

template <int UNROLL = 10>
__device__ __forceinline__ U4 rng(const TraceParams& P, unsigned long long id, uint32_t vertex,
                                  uint32_t group) {
  const unsigned long long gid = P.path_offset + id;
  return philox4x32_10<UNROLL>((uint32_t)gid, (uint32_t)(gid >> 32), P.stream, (vertex << 8) | group,
                       P.key0, P.key1);
}

// The blocks of groups ga and gb at one vertex of a path (see rng).
template <int UNROLL = 10>
__device__ __forceinline__ void rng_pair(const TraceParams& P, unsigned long long id, uint32_t vertex,
                                         uint32_t ga, uint32_t gb, U4* a, U4* b) {
  const unsigned long long gid = P.path_offset + id;
  philox4x32_10_pair<UNROLL>((uint32_t)gid, (uint32_t)(gid >> 32), P.stream, (vertex << 8) | ga,
                             (vertex << 8) | gb, P.key0, P.key1, a, b);
}

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v) {
  const float y = v - comp;
  const float t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// Distance from (x, w) to the medium box boundary.
__device__ __forceinline__ float box_exit(const TraceParams& P, float x, float y, float z, float wx,
                                          float wy, float wz) {
  float d = FLT_MAX;
  if (wx > 0.0f) d = fminf(d, __fdividef(P.hi[0] - x, wx));
  else if (wx < 0.0f) d = fminf(d, __fdividef(P.lo[0] - x, wx));
  if (wy > 0.0f) d = fminf(d, __fdividef(P.hi[1] - y, wy));
  else if (wy < 0.0f) d = fminf(d, __fdividef(P.lo[1] - y, wy));
  if (wz > 0.0f) d = fminf(d, __fdividef(P.hi[2] - z, wz));
  else if (wz < 0.0f) d = fminf(d, __fdividef(P.lo[2] - z, wz));
  return fmaxf(d, 0.0f);
}

// Near-degenerate ellipse (S - C < 2^-12 C): the solve of Eq. 18 in FP64,
// kept out of line so that none of its conversions enter the common path.
__device__ __noinline__ void ellipse_fp64(float delta, float C, float S_lo, float dS, float q,
                                          float* r1, float* den, float* cos_s) {
  const double dd = (double)delta, Cd = (double)C, Sd = (double)S_lo + (double)dS, qd = (double)q;
  const double dend = dd + Cd * qd;                 // S - C mu
  const double nr = dd * dd + 2.0 * Sd * Cd * qd;    // 2 (S - C mu) r1
  *cos_s = (float)((2.0 * Cd * Cd * qd * (1.0 - qd) - dd * dd - 2.0 * Cd * qd * dd) / nr);
  *r1 = (float)(nr / (2.0 * dend));
  *den = (float)dend;
}

// Control vertex on the ray (x, w) with S in [S_lo, S_hi) (Eq. 18, 21, 22).
// uniform_S selects the uniform temporal density of the baseline.  Returns
// the contribution divided by beta and writes S.
__device__ __forceinline__ float connect(const TraceParams& P, float wx, float wy, float wz,
                                         float C, float ax, float ay, float az, float S_lo,
                                         float S_hi, float u, bool uniform_S, float* S_out,
                                         Counters& cnt, float* cos_out = nullptr,
                                         float* t_out = nullptr, float Ie = -1.0f) {
  const float W = S_hi - S_lo;
  float dS, conn_w;  // conn_w = exp(-sigma_t S) / p(S)
  if (!uniform_S) {
    const float em = expm1_neg(-P.sigma_t * W);  // -(1 - e^{-st W})
    dS = -log1m(-em * u) * P.inv_st;
    // e^{-st S} / p_S = e^{-st S_lo} (1 - e^{-st W}) / st
    conn_w = __expf(-P.sigma_t * S_lo) * (-em) * P.inv_st;
  } else {
    dS = u * W;
    conn_w = __expf(-P.sigma_t * (S_lo + dS)) * W;
  }
  const float S = S_lo + dS;
  const float delta = (S_lo - C) + dS;  // S - C without cancellation
  const float qx = wx - ax, qy = wy - ay, qz = wz - az;
  const float q = 0.5f * fmaf(qx, qx, fmaf(qy, qy, qz * qz));  // 1 - mu
  float r1, den, cos_s;
  if (delta < C * (1.0f / 4096.0f)) {
    ellipse_fp64(delta, C, S_lo, dS, q, &r1, &den, &cos_s);
    cnt.add_rare(ST_FP64E);
    if (t_out) *t_out = S - r1;
  } else {
    // with t from Eq. 18: S - C mu = delta + C q, r1 = S - t = (delta^2 + 2 S C q) / (2 (S - C mu)),
    // and the scattering cosine at the control vertex (C mu - t) / r1 written
    // without the cancellation of C mu - t near the emitter
    den = fmaf(C, q, delta);
    const float nr = fmaf(delta, delta, 2.0f * S * C * q);
    r1 = __fdividef(nr, 2.0f * den);
    if (t_out) *t_out = __fdividef(delta * (S + C), 2.0f * den);  // Eq. 18
    const float cq = C * q;
    cos_s = __fdividef(fmaf(2.0f * C * cq, 1.0f - q, -delta * fmaf(2.0f, cq, delta)), nr);
  }
  *S_out = S;
  if (cos_out) *cos_out = cos_s;
  const float f = hg_eval(cos_s, P.hg_a, P.hg_b, P.hg_c);
  // sigma_s e^{-st S} f I_e / r1^2 / p(t),  p(t) = p(S) (S - C mu) / r1
  return __fdividef(P.sigma_s * conn_w * f * (Ie < 0.0f ? P.Ie : Ie), r1 * den);
}

// One distance step of a DARTS vertex, as handed to the RIS evaluation:
// r^2 of a candidate at distance d is (d + b)^2 + h2 with b = <w, x - x_e>
// and h2 the squared distance of x_e from the ray; S_M as a float pair.
struct RisTask {
  float b, h2, SM, SMlo;
  float pm, u3;
  uint32_t e0row;  // eps0 (24 bits) | radical-inverse row << 24
  uint32_t nonempty;  // decision-trace bit of this vertex's control vertex
};
// Task of the kernels built for the RIS variants: the exit distance, and the
// path id and vertex for the uniforms drawn per candidate (global id bits
// 0-31; bits 32-47 | vertex << 16).
struct RisTaskVar : RisTask {
  float dm;
  uint32_t gid_lo, gid_hi_k;
};
template <bool VAR>
using RisTaskT = std::conditional_t<VAR, RisTaskVar, RisTask>;
struct RisResult {
  float factor, dsel;
  int sel, ok;
};

// log Phi (Eq. 9) for a candidate with remaining length s = S_M - d, in FP64
// (small t'), kept out of line.
__device__ __noinline__ float log_phi_fp64(const TraceParams& P, float r2, float SM, float SMlo,
                                           float d) {
  const double s = ((double)SM + (double)SMlo) - (double)d;
  const double tp = s * P.inv_v_d;
  return (float)(P.phi_k0_d - 1.5 * log(tp) - (double)r2 * P.phi_invk_d / tp - P.sa_v_d * tp);
}

// Candidate j of a RIS task: distance (Eq. 13-14, sign fixed) and log target
// weight (Eq. 10, -FLT_MAX when non-causal).
// RIS variants (compiled into the kernels built with VAR only).
// i.i.d. candidate uniform: Philox group 4 + j/4 of the vertex, word j mod 4.
__device__ __forceinline__ float iid_eps(const TraceParams& P, const RisTaskVar& T, int j) {
  const U4 u = philox4x32_10(T.gid_lo, T.gid_hi_k & 0xFFFFu, P.stream,
                             ((T.gid_hi_k >> 16) << 8) | (4u + (uint32_t)j / 4u), P.key0, P.key1);
  return u01((j & 3) == 0 ? u.x : (j & 3) == 1 ? u.y : (j & 3) == 2 ? u.z : u.w);
}

// Equiangular candidate on [0, d_m) about the emitter's closest approach
// t_c = -b at distance h: t = t_c + h tan(theta_a + eps (theta_b - theta_a)).
__device__ __forceinline__ float equi_distance(const RisTaskVar& T, float eps) {
  const float tc = -T.b, hh = sqrtf(fmaxf(T.h2, 1e-30f));
  const float tha = atan2f(-tc, hh), thb = atan2f(T.dm - tc, hh);
  return fminf(fmaxf(fmaf(hh, tanf(fmaf(eps, thb - tha, tha)), tc), 0.0f), T.dm * (1.0f - 1.0f / 8388608.0f));
}

// log(sigma_t e^{-sigma_t d} / (p_m p_eq(d))), p_eq = h / ((theta_b - theta_a)(h^2 + (d - t_c)^2)).
__device__ __forceinline__ float equi_lcorr(const TraceParams& P, const RisTaskVar& T, float d) {
  const float tc = -T.b, hh = sqrtf(fmaxf(T.h2, 1e-30f));
  const float tha = atan2f(-tc, hh), thb = atan2f(T.dm - tc, hh);
  const float dt = d - tc;
  return logf(P.sigma_t) - P.sigma_t * d - logf(T.pm) - logf(hh / ((thb - tha) * fmaf(dt, dt, T.h2)));
}

// Candidate j of a RIS task: distance *d_out and log RIS weight (log Phi of
// Eq. 10, plus the density correction equi_lcorr for equiangular
// candidates), -FLT_MAX when non-causal.  The selected candidate's throughput
// factor carries the same correction.
template <bool VAR>
__device__ __forceinline__ float ris_candidate(const TraceParams& P, const RisTaskT<VAR>& T, int j,
                                               bool act, float* d_out, Counters& cnt) {
  float eps;
  if (VAR && (P.ris_mode & 1)) {
    if constexpr (VAR) eps = iid_eps(P, T, j);
  } else {
    const uint32_t srow = T.e0row >> 24, e0 = T.e0row & 0xFFFFFFu;
    const uint32_t idx = (8u * srow + (uint32_t)j) & 255u;
    const uint32_t ri24 = __brev(idx) >> 8;
    eps = u01(((ri24 + e0) & 0xFFFFFFu) << 8);
  }
  float d, lc = 0.0f;
  if (VAR && (P.ris_mode & 2)) {
    if constexpr (VAR) {
      d = equi_distance(T, eps);
      lc = equi_lcorr(P, T, d);
    }
  } else {
    d = -log1m(T.pm * eps) * P.inv_st;
  }
  const float e = d + T.b;
  const float r2 = fmaf(e, e, T.h2);
  const float s = T.SM - d;  // remaining length budget
  *d_out = d;
  if (P.no_da) return 0.0f;  // ablation: the target equals the candidate density
  if (!(s > 0.0f && r2 < s * s)) return -FLT_MAX;
  if (DARTS_RARE(act && s < P.tiny_s)) {
    cnt.add_rare(ST_FP64P);
    return log_phi_fp64(P, r2, T.SM, T.SMlo, d) + lc;
  }
  const float tp = s * P.inv_v;
  return P.phi_k0 - 1.5f * __logf(tp) - __fdividef(r2 * P.phi_invk, tp) - P.sa_v * tp + lc;
}

// Reservoir uniform of candidate j: Philox group 12 + j/4 of the vertex, word j mod 4.
__device__ __forceinline__ float reservoir_u(const TraceParams& P, const RisTaskVar& T, int j) {
  const U4 u = philox4x32_10(T.gid_lo, T.gid_hi_k & 0xFFFFu, P.stream,
                             ((T.gid_hi_k >> 16) << 8) | (12u + (uint32_t)j / 4u), P.key0, P.key1);
  return u01((j & 3) == 0 ? u.x : (j & 3) == 1 ? u.y : (j & 3) == 2 ? u.z : u.w);
}

// ---- general scenes: surfaces, emitter points, camera -----------------------
constexpr float kGeomEps = 1e-5f;

// Smallest root t > kGeomEps of |x + w t - c| = r, or FLT_MAX.
// The discriminant is r^2 - |o - b w|^2 (the squared distance of the centre
// from the line), not b^2 - (|o|^2 - r^2): for a far sphere the latter
// cancels two large terms and loses most FP32 digits of the hit distance.
// The near root comes from the product of the roots (|o|^2 - r^2) divided
// by the root of larger magnitude, which has no cancellation either.
__device__ __forceinline__ float ray_sphere(const float4 c, float x, float y, float z, float wx,
                                            float wy, float wz) {
  const float ox = x - c.x, oy = y - c.y, oz = z - c.z;
  const float b = fmaf(ox, wx, fmaf(oy, wy, oz * wz));
  const float lx = fmaf(-b, wx, ox), ly = fmaf(-b, wy, oy), lz = fmaf(-b, wz, oz);
  const float disc = fmaf(c.w, c.w, -fmaf(lx, lx, fmaf(ly, ly, lz * lz)));
  if (disc < 0.0f) return FLT_MAX;
  const float q = -b - copysignf(sqrtf(disc), b);
  if (q == 0.0f) return FLT_MAX;
  const float cc = fmaf(ox, ox, fmaf(oy, oy, fmaf(oz, oz, -c.w * c.w)));
  const float ta = q, tb = cc / q;
  const float t0 = fminf(ta, tb), t1 = fmaxf(ta, tb);
  return t0 > kGeomEps ? t0 : (t1 > kGeomEps ? t1 : FLT_MAX);
}

// ---- sphere culling ---------------------------------------------------------
// The general kernels keep, at the start of dynamic shared memory, per axis a
// of the medium box split into G = cull_slabs slabs, the mask M_a[i][j] of the
// spheres whose extent along a, enlarged by cull_eps, meets slabs i..j, and
// the spheres themselves (float4 centre, radius).  A sphere that a segment
// meets overlaps the segment's bounding box on every axis, so it is in
// M_x & M_y & M_z of that box: testing only those spheres, in increasing
// index order, finds the same nearest hit (and the same lowest-index tie) as
// testing every sphere.  Each segment is split into kCullPieces pieces and
// their masks are OR-ed, which tightens the boxes of long diagonal rays (a
// warp tests as many spheres as its lane with the most candidates: on the
// 512x512 sphere frame that maximum is about 10 for a shadow ray cut in two,
// 8 cut in three, 6 cut in four).  The piece loop stays rolled: unrolled, its
// code cost more than the tests it saves; three pieces measured fastest.
__device__ __forceinline__ const unsigned long long* cull_masks() {
  extern __shared__ float4 smem4[];
  return reinterpret_cast<const unsigned long long*>(smem4);
}
__device__ __forceinline__ const float4* cull_spheres(const TraceParams& P) {
  return reinterpret_cast<const float4*>(cull_masks() + 3 * P.cull_slabs * P.cull_slabs);
}
__device__ __forceinline__ int cull_slab(const TraceParams& P, int a, float v) {
  return min(max(__float2int_rd(fmaf(v, P.cull_inv_w[a], P.cull_off[a])), 0), P.cull_slabs - 1);
}
// Masks and spheres, built by the whole block before any path runs.
__device__ __forceinline__ void build_cull(const TraceParams& P, int tid, int nthreads) {
  extern __shared__ float4 smem4[];
  unsigned long long* m = reinterpret_cast<unsigned long long*>(smem4);
  const int G = P.cull_slabs;
  float4* sph = reinterpret_cast<float4*>(m + 3 * G * G);
  for (int k = tid; k < P.n_spheres; k += nthreads) sph[k] = P.sph[k];
  for (int e = tid; e < 3 * G * G; e += nthreads) {
    const int a = e / (G * G), i = (e / G) % G, j = e % G;
    unsigned long long bits = 0;
    for (int k = 0; k < P.n_spheres; ++k) {
      const float4 c = P.sph[k];
      const float ca = a == 0 ? c.x : (a == 1 ? c.y : c.z);
      const float rr = c.w + P.cull_eps;
      if (cull_slab(P, a, ca - rr) <= j && cull_slab(P, a, ca + rr) >= i) bits |= 1ull << k;
    }
    m[e] = bits;
  }
}
constexpr int kCullPieces = 3;
// Spheres that may meet the segment from a along unit w over length len, cut
// into kCullPieces equal pieces: the slab of a point is monotone in its
// coordinate, so a piece's slab range on an axis is the range of its two end
// points' slabs (consecutive pieces share the rounded end point between
// them, and the masks' enlargement covers that rounding).
__device__ __forceinline__ unsigned long long cull_segment(const TraceParams& P, float x, float y, float z,
                                                           float wx, float wy, float wz, float len) {
  const unsigned long long* m = cull_masks();
  const int G = P.cull_slabs, kAxis = G * G;
  int s0 = cull_slab(P, 0, x), s1 = cull_slab(P, 1, y), s2 = cull_slab(P, 2, z);
  unsigned long long bits = 0;
#pragma unroll 1  // one copy of the piece step at each of the three call sites
  for (int k = 1; k <= kCullPieces; ++k) {
    const float t = len * ((float)k * (1.0f / (float)kCullPieces));
    const int e0 = cull_slab(P, 0, fmaf(wx, t, x)), e1 = cull_slab(P, 1, fmaf(wy, t, y)),
              e2 = cull_slab(P, 2, fmaf(wz, t, z));
    bits |= m[min(s0, e0) * G + max(s0, e0)] & m[kAxis + min(s1, e1) * G + max(s1, e1)] &
            m[2 * kAxis + min(s2, e2) * G + max(s2, e2)];
    s0 = e0;
    s1 = e1;
    s2 = e2;
  }
  return bits;
}

// Nearest wall, sphere or open face along (x, w) from inside the box.
// hit: 0 open face, 1 wall, 2 + i sphere i; n: the surface normal facing the
// ray.  Sphere `skip` is the one the ray leaves (outward): being convex it
// cannot be met again, and skipping it keeps FP32 rounding of the start point
// from producing a spurious second hit.  Only the spheres of the segment's
// culling masks are tested (general kernels: they are in shared memory).
__device__ __forceinline__ float cast_ray(const TraceParams& P, float x, float y, float z, float wx,
                                          float wy, float wz, int skip, int* hit, float* nx, float* ny,
                                          float* nz) {
  float d = FLT_MAX;
  int face = -1;
  const float px[3] = {x, y, z}, pw[3] = {wx, wy, wz};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float di = FLT_MAX;
    int fi = -1;
    if (pw[i] > 0.0f) { di = __fdividef(P.hi[i] - px[i], pw[i]); fi = 2 * i + 1; }
    else if (pw[i] < 0.0f) { di = __fdividef(P.lo[i] - px[i], pw[i]); fi = 2 * i; }
    if (di < d) { d = di; face = fi; }
  }
  d = fmaxf(d, 0.0f);
  *hit = (face >= 0 && ((P.walls >> face) & 1)) ? 1 : 0;
  *nx = face / 2 == 0 ? ((face & 1) ? -1.0f : 1.0f) : 0.0f;
  *ny = face / 2 == 1 ? ((face & 1) ? -1.0f : 1.0f) : 0.0f;
  *nz = face / 2 == 2 ? ((face & 1) ? -1.0f : 1.0f) : 0.0f;
  if (P.n_spheres == 0) return d;
  const float4* sph = cull_spheres(P);
  unsigned long long cand = cull_segment(P, x, y, z, wx, wy, wz, d);
  if (skip >= 0) cand &= ~(1ull << skip);
  int hs = -1;
  while (cand) {
    const int k = __ffsll((long long)cand) - 1;
    cand &= cand - 1;
    const float t = ray_sphere(sph[k], x, y, z, wx, wy, wz);
    if (t < d) {
      d = t;
      hs = k;
    }
  }
  if (hs >= 0) {
    const float4 c = sph[hs];
    const float ir = 1.0f / c.w;
    *hit = 2 + hs;
    *nx = (fmaf(wx, d, x) - c.x) * ir;
    *ny = (fmaf(wy, d, y) - c.y) * ir;
    *nz = (fmaf(wz, d, z) - c.z) * ir;
  }
  return d;
}

// No sphere blocks the open segment a -> b (the box is convex: its walls
// never occlude two points inside it).  Sphere `skip` carries a (the segment
// leaves it outward, or the caller's contribution is zero anyway).
__device__ __forceinline__ bool visible(const TraceParams& P, float ax, float ay, float az, float bx,
                                        float by, float bz, int skip) {
  if (P.n_spheres == 0) return true;
  float wx = bx - ax, wy = by - ay, wz = bz - az;
  const float len = sqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
  const float il = 1.0f / len;
  wx *= il;
  wy *= il;
  wz *= il;
  const float4* sph = cull_spheres(P);
  unsigned long long cand = cull_segment(P, ax, ay, az, wx, wy, wz, len);
  if (skip >= 0) cand &= ~(1ull << skip);
  while (cand) {
    const int k = __ffsll((long long)cand) - 1;
    cand &= cand - 1;
    if (ray_sphere(sph[k], ax, ay, az, wx, wy, wz) < len - kGeomEps) return false;
  }
  return true;
}

// Inverse CDF search of a table row (row[0] = 0 <= v < 1 = row[n]): the
// largest lo in [0, n) with row[lo] <= v.  The row's guide (guide_bytes)
// bounds lo to [g[k], g[k + 1]] for k = floor(v kGuide), since
// row[g[k]] <= k / kGuide <= v < (k + 1) / kGuide; a binary search of that
// range follows (about 3.4 steps on the benchmark tables).  The same index
// as a binary search over the whole row, with four dependent shared-memory
// rounds instead of eight.
__device__ __forceinline__ int row_search(const float* row, const uint16_t* g, float v) {
  const int k = min((int)(v * (float)kGuide), kGuide - 1);
  int lo = g[k];
  int n = (int)g[k + 1] - lo + 1;
  while (n > 1) {
    const int half = n >> 1;
    lo = (row[lo + half] > v) ? lo : lo + half;
    n -= half;
  }
  return lo;
}

// Guides of the staged table rows (after them in shared memory): entry
// (r, k) is the largest lo in [0, n_mu) with row r's cdf[lo] <= k / kGuide
// (a binary search; 0 when none is), and n_mu - 1 at k = kGuide.  The
// caller synchronises the block before and after.
__device__ __forceinline__ void build_guides(const float* tab, int rows, int row_stride, int n_mu, int tid,
                                             int nthreads) {
  uint16_t* guide = reinterpret_cast<uint16_t*>(const_cast<float*>(tab) + (size_t)rows * row_stride);
  for (int i = tid; i < rows * (kGuide + 1); i += nthreads) {
    const int r = i / (kGuide + 1), k = i - r * (kGuide + 1);
    int lo = n_mu - 1;
    if (k < kGuide) {
      const float* row = tab + (size_t)r * row_stride;
      const float x = (float)k * (1.0f / (float)kGuide);
      lo = 0;
      int n = n_mu;
      while (n > 1) {
        const int half = n >> 1;
        lo = (row[lo + half] > x) ? lo : lo + half;
        n -= half;
      }
    }
    guide[i] = (uint16_t)lo;
  }
}

// The guide of table row row_i (see build_guides).
__device__ __forceinline__ const uint16_t* row_guide(const TraceParams& P, const float* tab, int row_i) {
  return reinterpret_cast<const uint16_t*>(tab + (size_t)P.rows * P.row_stride) + row_i * (kGuide + 1);
}

// Radiant intensity of the path's emitter point toward x.
__device__ __forceinline__ float emit_intensity(const Path& p, float x, float y, float z) {
  if (p.en0 == 0.0f && p.en1 == 0.0f && p.en2 == 0.0f) return p.ie;
  const float dx = x - p.ey0, dy = y - p.ey1, dz = z - p.ey2;
  const float c = fmaf(dx, p.en0, fmaf(dy, p.en1, dz * p.en2)) * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  return c > 0.0f ? p.ie * c : 0.0f;
}

// d log HG(mu; g) / dg = -2g/(1 - g^2) - 3 (g - mu) / (1 + g^2 - 2 g mu)
__device__ __forceinline__ float hg_dlog_dg(const TraceParams& P, float mu) {
  return fmaf(-3.0f * (P.g - mu), __frcp_rn(fmaf(-P.hg_c, mu, P.hg_b)), P.hg_dlog_a);
}

// Zero temporal weight of time bin b: outside the gate or a zero-weight bin.
__device__ __forceinline__ bool zero_w(const TraceParams& P, int b) {
  return b < 0 || b >= P.n_bins || (P.wbin != nullptr && __ldg(P.wbin + b) == 0.0f);
}

// DARTS bin of sample s of an element under a temporal response W: the
// cumulative weights C (FP64, C[0] = 0, C[B] = 1) are sampled systematically
// at x = ((s + oe) mod N_e + phi) / N_e; the bin is the first b with
// x < C[b + 1].  FP64, as the host builds C, so the integer decision is the
// same on every implementation that follows this arithmetic.
__device__ __forceinline__ int w_bin(const TraceParams& P, unsigned long long s, unsigned long long oe,
                                     double phi) {
  const unsigned long long ne = P.spp;
  const double x = ((double)((s + oe) % ne) + phi) / (double)ne;
  int lo = 0, n = P.n_bins;
  while (n > 0) {
    const int half = n >> 1;
    if (__ldg(P.wcdf + lo + half + 1) <= x) {
      lo += half + 1;
      n -= half + 1;
    } else {
      n = half;
    }
  }
  return min(lo, P.n_bins - 1);
}

// The per-element Philox block (vertex 0xFFFFFE, group 0) and the DARTS bin
// offset o_e = floor(u01(x) B) of a sensor element (R1, R28).
template <int UNROLL = 10>
__device__ __forceinline__ U4 element_block(const TraceParams& P, int elem) {
  return philox4x32_10<UNROLL>((uint32_t)elem, 0u, P.stream, (kVertexElement << 8) | 0u, P.key0, P.key1);
}
template <int UNROLL = 10>
__device__ __forceinline__ unsigned element_offset(const TraceParams& P, int elem) {
  return (unsigned)(((unsigned long long)(element_block<UNROLL>(P, elem).x >> 8) * (unsigned)P.n_bins) >> 24);
}

// LEAN (general kernels only): the scene has point emitters only, a point
// sensor or a camera inside the medium, no temporal response and no EDA at
// surfaces, so those branches are compiled out (the host picks it).
template <int METHOD, int MAXM, bool DEBUG, bool ADJ = false, bool GEN = false, bool VAR = false,
          bool LEAN = false>
struct Stepper {
  // Philox rounds per loop iteration: the lean camera kernel, the one whose
  // code least fits the instruction cache, takes two (1.3 % faster on the
  // 512x512 sphere frame); the others unroll all ten (two cost them 5 %).
  static constexpr int kPU = LEAN ? 2 : 10;
  // the same for the two blocks a lean vertex or refill draws side by side
  static constexpr int kPUP = LEAN ? 2 : 10;
  // Radiant intensity of the path's emitter point toward x, and the zero
  // temporal weight test, without the branches a lean scene never takes.
  __device__ __forceinline__ static float intensity(const Path& p, float x, float y, float z) {
    if constexpr (LEAN) return p.ie;
    else return emit_intensity(p, x, y, z);
  }
  __device__ __forceinline__ static bool zero_weight(const TraceParams& P, int b) {
    if constexpr (LEAN) return b < 0 || b >= P.n_bins;
    else return zero_w(P, b);
  }
  // Initialise a path with local index j.
  __device__ static void init(const TraceParams& P, Path& p, unsigned long long j, int bin) {
    p.x = P.xs[0];
    p.y = P.xs[1];
    p.z = P.xs[2];
    p.L = 0.0f;
    p.Lc = 0.0f;
    p.c = 0.0f;
    p.k = 0;
    p.j = j;
    p.a0 = p.a1 = p.a2 = p.gsum = 0.0f;
    p.wx = 0.0f;
    p.wy = 0.0f;
    p.wz = 1.0f;
    if (METHOD == kDartsFull) {  // the whole gate is the target interval
      p.bin = -1;
      p.Sm0 = P.S_gate_lo;
      p.SM0 = P.S_gate_hi;
      p.beta = 1.0f;
    } else if (METHOD == kDarts) {
      p.bin = P.wcdf ? w_bin(P, P.path_offset + j, P.w_oe, P.w_phi) : bin;
      p.Sm0 = fmaf((float)p.bin, P.S_bin, P.S_gate_lo);
      p.SM0 = fmaf((float)(p.bin + 1), P.S_bin, P.S_gate_lo);
      p.beta = 1.0f;
    } else {
      p.bin = -1;
      const U4 u = rng<kPU>(P, j, 0, 1);
      float s, c;
      sincos_2pi(u01(u.z), &s, &c);
      const float uy = u01(u.y);
      frame_dir(0.0f, 0.0f, 1.0f, fmaf(2.0f, uy, -1.0f), 2.0f * sqrtf(uy * (1.0f - uy)), s, c, &p.wx, &p.wy,
                &p.wz);
      p.beta = 4.0f * kPi;
    }
  }

  // ---- general scenes -------------------------------------------------------
  // Path start: sensor element and (DARTS) bin, the emitter point (chosen by
  // energy, a uniform point on an area emitter), then the point sensor or
  // the camera ray entering the medium (p.miss when it never does).
  // oe_pre: the element's bin offset o_e when the caller has it (else -1),
  // e_pre: gid / spp when the caller has it (cameras).
  __device__ static void init_gen(const TraceParams& P, Path& p, unsigned long long j, int oe_pre = -1,
                                  unsigned long long e_pre = ~0ull) {
    const unsigned long long gid = P.path_offset + j;
    const int B = P.n_bins;
    unsigned long long s = gid;
    p.elem = 0;
    if (P.camera) {  // sample s of pixel elem; ids past the last pixel wrap with s continuing
      const unsigned long long e = e_pre != ~0ull ? e_pre : gid / P.spp;
      const unsigned long long pixels = (unsigned long long)P.width * (unsigned long long)P.height;
      const unsigned long long wrap = e / pixels;
      s = wrap * P.spp + (gid - e * P.spp);
      p.elem = (int)(e - wrap * pixels);
    }
    p.j = j;
    p.L = p.Lc = p.c = 0.0f;
    p.k = 0;
    p.nmed = 0;
    p.a0 = p.a1 = p.a2 = p.gsum = 0.0f;
    p.miss = false;
    p.surf = -1;
    p.salb = 0.0f;
    // emitter point; the camera's jitter block is drawn beside it (two
    // independent Philox chains whose latencies overlap)
    U4 ue, uc = U4{0u, 0u, 0u, 0u};
    if (LEAN) {
      rng_pair<kPUP>(P, j, 0xFFFFFFu, 2, 3, &ue, &uc);
    } else {
      ue = rng<kPU>(P, j, 0xFFFFFFu, 2);
      if (P.camera) uc = rng<kPU>(P, j, 0xFFFFFFu, 3);
    }
    const float target = u01(ue.x);
    int pick = P.n_emitters - 1;
    for (int k = P.n_emitters - 1; k >= 0; --k)
      if (target < P.em[k].cdf) pick = k;
    const EmitterParams& E = P.em[pick];
    const float su = u01(ue.y), sv = u01(ue.z);
    p.ey0 = fmaf(su, E.u[0], fmaf(sv, E.v[0], E.pos[0]));
    p.ey1 = fmaf(su, E.u[1], fmaf(sv, E.v[1], E.pos[1]));
    p.ey2 = fmaf(su, E.u[2], fmaf(sv, E.v[2], E.pos[2]));
    p.en0 = E.n[0];
    p.en1 = E.n[1];
    p.en2 = E.n[2];
    p.ie = E.ie;
    p.s_hi_e = E.s_hi;
    p.beta = E.wsel;
    if (METHOD == kDarts) {
      int b;
      if (oe_pre >= 0) {
        b = (int)((s % (unsigned long long)B + (unsigned)oe_pre) % (unsigned)B);
      } else if (!LEAN && P.wcdf) {
        const U4 uo = element_block<kPU>(P, p.elem);
        const unsigned long long oe = (unsigned long long)floor((double)u01(uo.x) * (double)P.spp);
        b = w_bin(P, s, min(oe, P.spp - 1), (double)u01(uo.y));
      } else {
        const unsigned oe = element_offset<kPU>(P, p.elem);
        b = (int)((s % (unsigned long long)B + oe) % (unsigned)B);
      }
      p.bin = p.elem * B + b;
      p.Sm0 = fmaf((float)b, P.S_bin, E.s_lo);
      p.SM0 = fmaf((float)(b + 1), P.S_bin, E.s_lo);
    } else {  // the baselines bin each contribution by its time (row p.elem)
      p.bin = -1;
      p.Sm0 = E.s_lo;
      p.SM0 = E.s_hi;
    }
    if (P.camera) {
      const int px = p.elem % P.width, py = p.elem / P.width;
      const float sx = (2.0f * ((float)px + u01(uc.x)) / (float)P.width - 1.0f) * P.cam_th * P.cam_aspect;
      const float sy = (1.0f - 2.0f * ((float)py + u01(uc.y)) / (float)P.height) * P.cam_th;
      float wx = P.cam_f[0] + sx * P.cam_r[0] + sy * P.cam_u[0];
      float wy = P.cam_f[1] + sx * P.cam_r[1] + sy * P.cam_u[1];
      float wz = P.cam_f[2] + sx * P.cam_r[2] + sy * P.cam_u[2];
      const float iw = rsqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
      p.wx = wx * iw;
      p.wy = wy * iw;
      p.wz = wz * iw;
      p.fixed = true;
      if (LEAN || P.cam_inside) {
        p.x = P.cam_pos[0];
        p.y = P.cam_pos[1];
        p.z = P.cam_pos[2];
      } else {
        const float o[3] = {P.cam_pos[0], P.cam_pos[1], P.cam_pos[2]}, w[3] = {p.wx, p.wy, p.wz};
        float tin = -FLT_MAX, tout = FLT_MAX;
        int face = -1;
        bool miss = false;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          if (w[i] == 0.0f) {
            if (o[i] < P.lo[i] || o[i] > P.hi[i]) miss = true;
            continue;
          }
          float t1 = (P.lo[i] - o[i]) / w[i], t2 = (P.hi[i] - o[i]) / w[i];
          int f1 = 2 * i, f2 = 2 * i + 1;
          if (t1 > t2) {
            const float tt = t1; t1 = t2; t2 = tt;
            const int ff = f1; f1 = f2; f2 = ff;
          }
          if (t1 > tin) { tin = t1; face = f1; }
          if (t2 < tout) tout = t2;
        }
        if (miss || !(tin <= tout) || tout <= 0.0f || tin < 0.0f) p.miss = true;
        if (face >= 0 && ((P.walls >> face) & 1)) p.miss = true;
        p.x = fmaf(p.wx, tin, o[0]);
        p.y = fmaf(p.wy, tin, o[1]);
        p.z = fmaf(p.wz, tin, o[2]);
        p.L = p.miss ? 0.0f : tin;
      }
    } else {
      p.x = P.xs[0];
      p.y = P.xs[1];
      p.z = P.xs[2];
      p.wx = 0.0f;
      p.wy = 0.0f;
      p.wz = 1.0f;
      p.fixed = false;
      if (!kIsDartsM<METHOD>) {  // the baselines draw the uniform direction here
        const U4 u = rng<kPU>(P, j, 0, 1);
        float sn, cs;
        sincos_2pi(u01(u.z), &sn, &cs);
        const float uy = u01(u.y);
        frame_dir(0.0f, 0.0f, 1.0f, fmaf(2.0f, uy, -1.0f), 2.0f * sqrtf(uy * (1.0f - uy)), sn, cs, &p.wx,
                  &p.wy, &p.wz);
        p.beta *= 4.0f * kPi;
        p.fixed = true;
      }
    }
  }

  // Direct connection from a surface vertex (normal n facing the medium) to
  // the path's emitter point: BRDF albedo / pi, transmittance, intensity,
  // 1 / r^2 and visibility.  Writes r.
  __device__ static float surface_connect(const TraceParams& P, const Path& p, float nx, float ny,
                                          float nz, float albedo, float* r_out) {
    const float dx = p.ey0 - p.x, dy = p.ey1 - p.y, dz = p.ey2 - p.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ir = rsqrtf(r2);
    const float r = r2 * ir;
    *r_out = r;
    const float cs = fmaf(dx, nx, fmaf(dy, ny, dz * nz)) * ir;
    if (!(cs > 0.0f)) return 0.0f;
    if (!visible(P, p.x, p.y, p.z, p.ey0, p.ey1, p.ey2, p.surf)) return 0.0f;
    return albedo * (1.0f / kPi) * cs * __expf(-P.sigma_t * r) * intensity(p, p.x, p.y, p.z) / r2;
  }

  // Surface vertex: move onto the surface, connect, then a cosine-weighted
  // direction (Lambertian: BRDF cos / pdf = albedo) from group 1 of vertex k+1.
  __device__ static float surface_bounce(const TraceParams& P, Path& p, float dm, int hit, float nx,
                                         float ny, float nz, float* r_out) {
    p.x = fmaf(p.wx, dm, p.x);
    p.y = fmaf(p.wy, dm, p.y);
    p.z = fmaf(p.wz, dm, p.z);
    kahan_add(p.L, p.Lc, dm);
    p.surf = hit >= 2 ? hit - 2 : -1;
    const float alb = hit == 1 ? P.wall_albedo : P.sph_albedo[hit - 2];
    const float c = p.beta * surface_connect(P, p, nx, ny, nz, alb, r_out);
    if (!LEAN && P.surface_eda) {  // the next vertex draws its direction (EDA / cosine-lobe MIS)
      p.wx = nx;
      p.wy = ny;
      p.wz = nz;
      p.salb = alb;
      p.fixed = false;
      return c;
    }
    const U4 us = rng<kPU>(P, p.j, (uint32_t)(p.k + 1), 1);
    float sn, cs;
    sincos_2pi(u01(us.z), &sn, &cs);
    const float uc = u01(us.y);
    frame_dir(nx, ny, nz, sqrtf(uc), sqrtf(1.0f - uc), sn, cs, &p.wx, &p.wy, &p.wz);
    p.beta *= alb;
    p.fixed = true;
    return c;
  }

  // DARTS vertex in a general scene.  Returns 1 when the path ended, 0 when
  // the RIS task of the distance step was filled, 2 when the path moved to a
  // surface vertex (no distance step).
  __device__ static int vertex_gen(const TraceParams& P, Path& p, const float* tab, Counters& cnt,
                                   RisTaskT<VAR>& task) {
    if (DARTS_RARE(p.miss)) return 1;  // camera ray that never enters the medium
    cnt.add(ST_VERT);
    const float ex = p.ey0 - p.x, ey = p.ey1 - p.y, ez = p.ey2 - p.z;
    const float C2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    const float C = sqrtf(C2);
    const float invC = __frcp_rn(C);
    const float ax = ex * invC, ay = ey * invC, az = ez * invC;
    const float SM = p.SM0 - p.L, Sm = p.Sm0 - p.L;
    if (DARTS_RARE(!(SM > C))) {
      cnt.add(ST_EARLY);
      record(P, p, 0, EV_EARLY);
      return 1;
    }
    float wx = p.wx, wy = p.wy, wz = p.wz;
    // both draws of the vertex up front: two independent Philox chains
    U4 u1, u0;
    if (LEAN) {
      rng_pair<kPUP>(P, p.j, (uint32_t)p.k, 1, 0, &u1, &u0);
    } else {
      u1 = rng<kPU>(P, p.j, (uint32_t)p.k, 1);
      u0 = rng<kPU>(P, p.j, (uint32_t)p.k, 0);
    }
    if (!p.fixed) {
      // MIS of the EDA table and HG (uniform sphere at the point sensor), Eq. 19
      const float rho = __fdividef(C, SM);
      int i_rho = min(max((int)(rho * (float)P.n_rho), 0), P.n_rho - 1);
      int i_s = (int)floorf((__log2f(SM * P.inv_smax) + 8.0f) * P.n_s_over_8);
      i_s = min(max(i_s, 0), P.n_s - 1);
      const int row_i = i_rho * P.n_s + i_s;
      const int row_c = DARTS_INDEX_OK(P, row_i, P.rows) ? row_i : 0;
      const float* row = tab + row_c * P.row_stride;
      float gamma = __fdividef(rho, rho + P.mis_alpha);
      const bool sensor = p.k == 0;
      if ((sensor && P.uniform_sensor) || P.no_eda) gamma = 0.0f;
      const float gb = sensor ? 0.0f : P.g;
      const float bx = sensor ? 0.0f : p.wx, by = sensor ? 0.0f : p.wy, bz = sensor ? 1.0f : p.wz;
      const float v0 = u01(u1.x), v1 = u01(u1.y);
      float sphi, cphi;
      sincos_2pi(u01(u1.z), &sphi, &cphi);
      const bool eda = v0 < gamma;
      const bool lobe = !LEAN && p.salb > 0.0f;  // base strategy: the cosine lobe about a surface normal
      const int lo = row_search(row, row_guide(P, tab, row_c), v1);
      const float c_lo = row[lo], c_hi = row[lo + 1];
      const float fr = __fdividef(v1 - c_lo, c_hi - c_lo);
      const float mu_eda = fmaf((float)lo + fr, P.inv_mu_scale, -1.0f);
      // 1 -+ mu of the table sample from the bin index: no cancellation near +-1
      const float st_eda = sqrtf(fmaxf(0.0f, ((float)(P.n_mu - lo) - fr) * P.inv_mu_scale *
                                                 (((float)lo + fr) * P.inv_mu_scale)));
      const float mu_hg = lobe ? sqrtf(v1) : hg_sample(gb, v1);
      const float st_hg = lobe ? sqrtf(1.0f - v1) : hg_sin(gb, v1);
      frame_dir(eda ? ax : bx, eda ? ay : by, eda ? az : bz, eda ? mu_eda : mu_hg, eda ? st_eda : st_hg, sphi,
                cphi, &wx, &wy, &wz);
      const float mu_b = eda ? fmaf(wx, bx, fmaf(wy, by, wz * bz)) : mu_hg;
      int bin = lo;
      if (!eda) {
        const float mua = fmaf(wx, ax, fmaf(wy, ay, wz * az));
        bin = min(max((int)floorf((mua + 1.0f) * P.mu_scale), 0), P.n_mu - 1);
      }
      const float pE = (eda ? c_hi - c_lo : row[bin + 1] - row[bin]) * P.mu_scale * (1.0f / kTwoPi);
      const float hg = hg_eval(mu_b, P.hg_a, P.hg_b, P.hg_c);
      const float cl = fmaxf(mu_b, 0.0f) * (1.0f / kPi);  // cosine lobe density; BRDF cos = albedo * cl
      const float pB = sensor ? kInv4Pi : (lobe ? cl : hg);
      const float f = sensor ? 1.0f : (lobe ? p.salb * cl : hg);
      p.beta *= __fdividef(f, fmaf(gamma, pE - pB, pB));
      if (ADJ && !sensor && !lobe) p.gsum += hg_dlog_dg(P, mu_b);
      if (DEBUG) {
        record(P, p, 2, eda ? 1 : 0);
        record(P, p, 3, (uint8_t)(bin & 0xFF));
      }
      if (lobe) {
        p.salb = 0.0f;
        if (!(p.beta > 0.0f)) {  // an EDA direction into the surface: nothing follows
          cnt.add(ST_INVALID);
          record(P, p, 0, EV_INVALID);
          return 1;
        }
      }
    }
    // control vertex, capped at the first surface (case II of Sec. 5.2)
    int hit;
    float nx, ny, nz;
    const float dm = cast_ray(P, p.x, p.y, p.z, wx, wy, wz, p.surf, &hit, &nx, &ny, &nz);
    const float mx = fmaf(wx, dm, -ex), my = fmaf(wy, dm, -ey), mz = fmaf(wz, dm, -ez);
    const float S_dm = dm + sqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz)));
    const float S_hi = fminf(SM, S_dm), S_lo = fmaxf(Sm, C);
    const bool ok = S_hi > S_lo;
    if (ok) {
      float S, cos_s, tctl;
      float cc = connect(P, wx, wy, wz, C, ax, ay, az, S_lo, S_hi, u01(u1.w), false, &S, cnt, &cos_s,
                         &tctl, 1.0f);
      const float qx = fmaf(wx, tctl, p.x), qy = fmaf(wy, tctl, p.y), qz = fmaf(wz, tctl, p.z);
      cc *= intensity(p, qx, qy, qz);
      if (!visible(P, qx, qy, qz, p.ey0, p.ey1, p.ey2, -1)) cc = 0.0f;
      p.c = fmaf(p.beta, cc, p.c);
      cnt.add(ST_CONN);
      cnt.add(ST_SAMPLE);
      if (METHOD == kDartsFull) {  // committed this step to the bin of its time
        const int b = min(max((int)floorf(((p.L + S) - p.Sm0) * P.inv_S_bin), 0), P.n_bins - 1);
        p.cb = p.elem * P.n_bins + b;
        p.cv = p.beta * cc;
        if (zero_weight(P, b)) cnt.add(ST_REJECT);
      }
      if (ADJ) {
        const float cv = p.beta * cc, ell = p.L + S;
        p.a0 = fmaf(cv, fmaf((float)(p.nmed + 1), P.inv_sigma_s, -ell), p.a0);
        p.a1 = fmaf(-cv, ell, p.a1);
        p.a2 = fmaf(cv, p.gsum + hg_dlog_dg(P, cos_s), p.a2);
      }
    }
    const uint8_t nonempty = ok ? 0x10 : 0;
    p.wx = wx;
    p.wy = wy;
    p.wz = wz;
    if (DARTS_RARE(p.k + 1 == P.K)) {
      record(P, p, 0, EV_MAXDEPTH | nonempty);
      return 1;
    }
    const float pm = -expm1_neg(-P.sigma_t * dm);
    if (!(u01(u0.x) < pm)) {
      if (hit == 0) {
        cnt.add(ST_ESCAPE);
        record(P, p, 0, EV_ESCAPE | nonempty);
        return 1;
      }
      record(P, p, 0, EV_SURFACE | nonempty);
      float r;
      const float cs = surface_bounce(P, p, dm, hit, nx, ny, nz, &r);
      const float Lt = p.L + r;
      if (cs > 0.0f) {
        cnt.add(ST_SAMPLE2);
        if (METHOD == kDartsFull) {
          const float y = (Lt - p.Sm0) * P.inv_S_bin;
          const int b = (y >= 0.0f && y < (float)P.n_bins) ? min((int)y, P.n_bins - 1) : -1;
          if (zero_weight(P, b)) cnt.add(ST_REJECT2);
          if (b >= 0) {
            p.cb2 = p.elem * P.n_bins + b;
            p.cv2 = cs;
            p.c += cs;
          }
        } else if (!(Lt >= p.Sm0 && Lt < p.SM0)) {
          cnt.add(ST_REJECT2);
        }
      }
      if (METHOD == kDarts && cs > 0.0f && Lt >= p.Sm0 && Lt < p.SM0) {
        p.c += cs;
        if (ADJ) {
          p.a0 = fmaf(cs, fmaf((float)p.nmed, P.inv_sigma_s, -Lt), p.a0);
          p.a1 = fmaf(-cs, Lt, p.a1);
          p.a2 = fmaf(cs, p.gsum, p.a2);
        }
      }
      p.k += 1;
      return 2;
    }
    cnt.add(ST_DIST);
    task.b = -fmaf(wx, ex, fmaf(wy, ey, wz * ez));
    const float hx = fmaf(wy, ez, -wz * ey), hy = fmaf(wz, ex, -wx * ez), hz = fmaf(wx, ey, -wy * ex);
    task.h2 = fmaf(hx, hx, fmaf(hy, hy, hz * hz));
    task.SM = SM;
    task.SMlo = ((p.SM0 - SM) - p.L) + p.Lc;
    task.pm = pm;
    task.u3 = u01(u0.w);
    task.e0row = (u0.z >> 8) | ((u0.y >> 27) << 24);
    task.nonempty = nonempty;
    if constexpr (VAR) {
      task.dm = dm;
      const unsigned long long gid = P.path_offset + p.j;
      task.gid_lo = (uint32_t)gid;
      task.gid_hi_k = ((uint32_t)(gid >> 32) & 0xFFFFu) | ((uint32_t)p.k << 16);
    }
    return 0;
  }

  // Baseline vertex in a general scene.
  __device__ static bool step_base_gen(const TraceParams& P, Path& p, Counters& cnt, int* out_bin,
                                       float* out_c, int* out_bin2, float* out_c2) {
    *out_bin = -1;
    *out_bin2 = -1;
    if (p.miss) return true;
    cnt.add(ST_VERT);
    const int row = p.elem * P.n_bins;
    int hit;
    float nx, ny, nz;
    const float dm = cast_ray(P, p.x, p.y, p.z, p.wx, p.wy, p.wz, p.surf, &hit, &nx, &ny, &nz);
    if (METHOD == kPlain) {
      const float ex = p.ey0 - p.x, ey = p.ey1 - p.y, ez = p.ey2 - p.z;
      const float C = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
      const float invC = __frcp_rn(C);
      const float SM = p.SM0 - p.L, Sm = p.Sm0 - p.L;
      if (DARTS_RARE(!(SM > C))) {
        cnt.add(ST_EARLY);
        record(P, p, 0, EV_EARLY);
        return true;
      }
      const float mx = fmaf(p.wx, dm, -ex), my = fmaf(p.wy, dm, -ey), mz = fmaf(p.wz, dm, -ez);
      const float S_dm = dm + sqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz)));
      const float S_hi = fminf(SM, S_dm), S_lo = fmaxf(Sm, C);
      const U4 u1 = rng<kPU>(P, p.j, (uint32_t)p.k, 1);
      if (S_hi > S_lo) {
        float S, cos_s, tctl;
        float cc = connect(P, p.wx, p.wy, p.wz, C, ex * invC, ey * invC, ez * invC, S_lo, S_hi,
                           u01(u1.w), true, &S, cnt, &cos_s, &tctl, 1.0f);
        const float qx = fmaf(p.wx, tctl, p.x), qy = fmaf(p.wy, tctl, p.y), qz = fmaf(p.wz, tctl, p.z);
        cc *= intensity(p, qx, qy, qz);
        if (!visible(P, qx, qy, qz, p.ey0, p.ey1, p.ey2, -1)) cc = 0.0f;
        cnt.add(ST_CONN);
        const float y = ((p.L + S) - p.Sm0) * P.inv_S_bin;
        const int b = min(max((int)floorf(y), 0), P.n_bins - 1);
        cnt.add(ST_SAMPLE);
        if (zero_weight(P, b)) cnt.add(ST_REJECT);
        *out_bin = row + b;
        *out_c = p.beta * cc;
        p.c += *out_c;
      }
      if (DARTS_RARE(p.k + 1 == P.K)) {
        record(P, p, 0, EV_MAXDEPTH);
        return true;
      }
      const U4 u0 = rng<kPU>(P, p.j, (uint32_t)p.k, 0);
      const float d = -log1m(u01(u0.x)) * P.inv_st;
      if (!(d < dm)) {
        if (hit == 0) {
          cnt.add(ST_ESCAPE);
          record(P, p, 0, EV_ESCAPE);
          return true;
        }
        record(P, p, 0, EV_SURFACE);
        float r;
        const float cs = surface_bounce(P, p, dm, hit, nx, ny, nz, &r);
        if (cs > 0.0f) {
          const float y = ((p.L + r) - p.Sm0) * P.inv_S_bin;
          cnt.add(ST_SAMPLE2);
          if (zero_weight(P, (y >= 0.0f && y < (float)P.n_bins) ? min((int)y, P.n_bins - 1) : -1)) cnt.add(ST_REJECT2);
          if (y >= 0.0f && y < (float)P.n_bins) {
            *out_bin2 = row + min((int)y, P.n_bins - 1);
            *out_c2 = cs;
            p.c += cs;
          }
        }
        p.k += 1;
        return false;
      }
      p.beta *= P.albedo;
      p.x = fmaf(p.wx, d, p.x);
      p.y = fmaf(p.wy, d, p.y);
      p.z = fmaf(p.wz, d, p.z);
      kahan_add(p.L, p.Lc, d);
      p.surf = -1;
      record(P, p, 0, EV_SCATTER);
    } else {  // vanilla
      const U4 u0 = rng<kPU>(P, p.j, (uint32_t)p.k, 0);
      const float d = -log1m(u01(u0.x)) * P.inv_st;
      if (!(d < dm)) {
        if (hit == 0) {
          cnt.add(ST_ESCAPE);
          record(P, p, 0, EV_ESCAPE);
          return true;
        }
        float r;
        const bool last = p.k + 1 == P.K;
        float cs;
        if (last) {  // connect only: the path ends at this surface vertex
          p.x = fmaf(p.wx, dm, p.x);
          p.y = fmaf(p.wy, dm, p.y);
          p.z = fmaf(p.wz, dm, p.z);
          kahan_add(p.L, p.Lc, dm);
          p.surf = hit >= 2 ? hit - 2 : -1;
          const float alb = hit == 1 ? P.wall_albedo : P.sph_albedo[hit - 2];
          cs = p.beta * surface_connect(P, p, nx, ny, nz, alb, &r);
        } else {
          cs = surface_bounce(P, p, dm, hit, nx, ny, nz, &r);
        }
        if (cs > 0.0f) {
          cnt.add(ST_CONN);
          const float y = ((p.L + r) - p.Sm0) * P.inv_S_bin;
          cnt.add(ST_SAMPLE);
          if (zero_weight(P, (y >= 0.0f && y < (float)P.n_bins) ? min((int)y, P.n_bins - 1) : -1)) cnt.add(ST_REJECT);
          if (y >= 0.0f && y < (float)P.n_bins) {
            *out_bin = row + min((int)y, P.n_bins - 1);
            *out_c = cs;
            p.c += cs;
          }
        }
        if (last) {
          record(P, p, 0, EV_MAXDEPTH);
          return true;
        }
        const float ex = p.x - p.ey0, ey = p.y - p.ey1, ez = p.z - p.ey2;
        const float C = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
        if (!(p.L + C < p.s_hi_e)) {
          cnt.add(ST_EARLY);
          record(P, p, 0, EV_EARLY);
          return true;
        }
        record(P, p, 0, EV_SURFACE);
        p.k += 1;
        return false;
      }
      p.beta *= P.albedo;
      p.x = fmaf(p.wx, d, p.x);
      p.y = fmaf(p.wy, d, p.y);
      p.z = fmaf(p.wz, d, p.z);
      kahan_add(p.L, p.Lc, d);
      p.surf = -1;
      const float ex = p.x - p.ey0, ey = p.y - p.ey1, ez = p.z - p.ey2;
      const float C2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
      const float C = sqrtf(C2);
      const float cos_s = -__fdividef(ex * p.wx + ey * p.wy + ez * p.wz, C);
      const float y = ((p.L + C) - p.Sm0) * P.inv_S_bin;
      cnt.add(ST_SAMPLE);
      if (zero_weight(P, (y >= 0.0f && y < (float)P.n_bins) ? min((int)y, P.n_bins - 1) : -1)) cnt.add(ST_REJECT);
      if (y >= 0.0f && y < (float)P.n_bins) {
        cnt.add(ST_CONN);
        float c = p.beta * hg_eval(cos_s, P.hg_a, P.hg_b, P.hg_c) * __expf(-P.sigma_t * C) *
                  intensity(p, p.x, p.y, p.z) / C2;
        if (!visible(P, p.x, p.y, p.z, p.ey0, p.ey1, p.ey2, -1)) c = 0.0f;
        *out_bin = row + min((int)y, P.n_bins - 1);
        *out_c = c;
        p.c += c;
      }
      if (!(p.L + C < p.s_hi_e)) {
        cnt.add(ST_EARLY);
        record(P, p, 0, EV_EARLY);
        return true;
      }
      if (DARTS_RARE(p.k + 1 == P.K)) {
        record(P, p, 0, EV_MAXDEPTH);
        return true;
      }
      record(P, p, 0, EV_SCATTER);
    }
    const U4 u1 = rng<kPU>(P, p.j, (uint32_t)(p.k + 1), 1);
    float sphi, cphi;
    sincos_2pi(u01(u1.z), &sphi, &cphi);
    float wx, wy, wz;
    const float xh = u01(u1.y);
    frame_dir(p.wx, p.wy, p.wz, hg_sample(P.g, xh), hg_sin(P.g, xh), sphi, cphi, &wx, &wy, &wz);
    p.wx = wx;
    p.wy = wy;
    p.wz = wz;
    p.k += 1;
    return false;
  }

  __device__ static void record(const TraceParams& P, const Path& p, int slot, uint8_t val) {
    if (DEBUG && p.j < P.N && p.k < P.K) P.dbg_dec[(p.j * P.K + p.k) * 4 + slot] = val;
  }

  // Vertex step of a DARTS path up to the distance step: early exit,
  // direction (MIS of the EDA table and the base strategy), control vertex,
  // max-depth test and the Bernoulli medium event.  Returns true when the
  // path ended; otherwise fills the RIS task of its distance step.
  __device__ static bool vertex_darts(const TraceParams& P, Path& p, const float* tab,
                                      Counters& cnt, RisTaskT<VAR>& task) {
    cnt.add(ST_VERT);
    const float ex = P.xe[0] - p.x, ey = P.xe[1] - p.y, ez = P.xe[2] - p.z;
    const float C2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    const float C = sqrtf(C2);
    const float invC = __frcp_rn(C);
    const float ax = ex * invC, ay = ey * invC, az = ez * invC;
    const float SM = p.SM0 - p.L, Sm = p.Sm0 - p.L;
    if (DARTS_RARE(!(SM > C))) {  // Sec. 5.2 early exit
      cnt.add(ST_EARLY);
      record(P, p, 0, EV_EARLY);
      return true;
    }
    // both draws of the vertex up front: two independent Philox chains
    const U4 u1 = rng<kPU>(P, p.j, (uint32_t)p.k, 1);
    const U4 u0 = rng<kPU>(P, p.j, (uint32_t)p.k, 0);
    // ---- direction: MIS of the EDA table and HG / uniform (Eq. 19)
    const float rho = __fdividef(C, SM);
    int i_rho = (int)(rho * (float)P.n_rho);
    i_rho = min(max(i_rho, 0), P.n_rho - 1);
    int i_s = (int)floorf((__log2f(SM * P.inv_smax) + 8.0f) * P.n_s_over_8);
    i_s = min(max(i_s, 0), P.n_s - 1);
    const int row_i = i_rho * P.n_s + i_s;
    const int row_c = DARTS_INDEX_OK(P, row_i, P.rows) ? row_i : 0;
    const float* row = tab + row_c * P.row_stride;
    float gamma = __fdividef(rho, rho + P.mis_alpha);
    const bool sensor = p.k == 0;
    if ((sensor && P.uniform_sensor) || P.no_eda) gamma = 0.0f;
    const float gb = sensor ? 0.0f : P.g;
    const float bx = sensor ? 0.0f : p.wx, by = sensor ? 0.0f : p.wy, bz = sensor ? 1.0f : p.wz;
    const float v0 = u01(u1.x), v1 = u01(u1.y);
    float sphi, cphi;
    sincos_2pi(u01(u1.z), &sphi, &cphi);
    const bool eda = v0 < gamma;
    // inverse CDF of the row: first bin whose upper edge exceeds v1
    const int lo = row_search(row, row_guide(P, tab, row_c), v1);
    const float c_lo = row[lo], c_hi = row[lo + 1];
    const float fr = __fdividef(v1 - c_lo, c_hi - c_lo);
    const float mu_eda = fmaf((float)lo + fr, P.inv_mu_scale, -1.0f);
    // 1 -+ mu of the table sample from the bin index: no cancellation near +-1
    const float st_eda = sqrtf(fmaxf(0.0f, ((float)(P.n_mu - lo) - fr) * P.inv_mu_scale *
                                               (((float)lo + fr) * P.inv_mu_scale)));
    const float mu_hg = hg_sample(gb, v1);
    const float st_hg = hg_sin(gb, v1);
    float wx, wy, wz;
    frame_dir(eda ? ax : bx, eda ? ay : by, eda ? az : bz, eda ? mu_eda : mu_hg, eda ? st_eda : st_hg, sphi,
              cphi, &wx, &wy, &wz);
    const float mu_b = eda ? fmaf(wx, bx, fmaf(wy, by, wz * bz)) : mu_hg;
    int bin = lo;
    if (!eda) {
      const float mua = fmaf(wx, ax, fmaf(wy, ay, wz * az));
      bin = min(max((int)floorf((mua + 1.0f) * P.mu_scale), 0), P.n_mu - 1);
    }
    const float pE = (eda ? c_hi - c_lo : row[bin + 1] - row[bin]) * P.mu_scale * (1.0f / kTwoPi);
    // base density: HG(g) about the previous direction (= the phase function
    // f itself), or the uniform sphere at the sensor where f = 1
    const float hg = hg_eval(mu_b, P.hg_a, P.hg_b, P.hg_c);
    const float pB = sensor ? kInv4Pi : hg;
    const float f = sensor ? 1.0f : hg;
    p.beta *= __fdividef(f, fmaf(gamma, pE - pB, pB));
    if (ADJ && !sensor) p.gsum += hg_dlog_dg(P, mu_b);
    if (DEBUG) {
      record(P, p, 2, eda ? 1 : 0);
      record(P, p, 3, (uint8_t)(bin & 0xFF));
    }
    // ---- control vertex (Eq. 18, 21, 22), medium boundary as the cap
    const float dm = box_exit(P, p.x, p.y, p.z, wx, wy, wz);
    const float mx = fmaf(wx, dm, -ex), my = fmaf(wy, dm, -ey), mz = fmaf(wz, dm, -ez);
    const float S_dm = dm + sqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz)));
    const float S_hi = fminf(SM, S_dm), S_lo = fmaxf(Sm, C);
    const bool ok = S_hi > S_lo;
    if (ok) {
      float S, cos_s;
      const float cc = connect(P, wx, wy, wz, C, ax, ay, az, S_lo, S_hi, u01(u1.w), false, &S, cnt,
                               ADJ ? &cos_s : nullptr);
      p.c = fmaf(p.beta, cc, p.c);
      cnt.add(ST_CONN);
      if (METHOD == kDartsFull) {  // committed this step to the bin of its time
        const int b = min(max((int)floorf(((p.L + S) - p.Sm0) * P.inv_S_bin), 0), P.n_bins - 1);
        p.cb = b;
        p.cv = p.beta * cc;
        cnt.add(ST_SAMPLE);
        if (zero_weight(P, b)) cnt.add(ST_REJECT);
      }
      if (ADJ) {
        // score of log f: k walk vertices + the control vertex scatter (sigma_s),
        // total length L + S attenuates (sigma_t), HG at every scattering vertex (g)
        const float cv = p.beta * cc, ell = p.L + S;
        p.a0 = fmaf(cv, fmaf((float)(p.k + 1), P.inv_sigma_s, -ell), p.a0);
        p.a1 = fmaf(-cv, ell, p.a1);
        p.a2 = fmaf(cv, p.gsum + hg_dlog_dg(P, cos_s), p.a2);
      }
    }
    const uint8_t nonempty = ok ? 0x10 : 0;
    p.wx = wx;  // the walk continues along the connection direction (Eq. 20)
    p.wy = wy;
    p.wz = wz;
    if (DARTS_RARE(p.k + 1 == P.K)) {
      record(P, p, 0, EV_MAXDEPTH | nonempty);
      return true;
    }
    // ---- Bernoulli medium event (Eq. 12)
    const float pm = -expm1_neg(-P.sigma_t * dm);
    if (!(u01(u0.x) < pm)) {
      cnt.add(ST_ESCAPE);
      record(P, p, 0, EV_ESCAPE | nonempty);
      return true;
    }
    cnt.add(ST_DIST);
    // ---- RIS task of the distance step (Eq. 13-15)
    task.b = -fmaf(wx, ex, fmaf(wy, ey, wz * ez));
    const float hx = fmaf(wy, ez, -wz * ey), hy = fmaf(wz, ex, -wx * ez), hz = fmaf(wx, ey, -wy * ex);
    task.h2 = fmaf(hx, hx, fmaf(hy, hy, hz * hz));
    task.SM = SM;
    task.SMlo = ((p.SM0 - SM) - p.L) + p.Lc;  // S_M = SM + SMlo incl. the Kahan term
    task.pm = pm;
    task.u3 = u01(u0.w);
    task.e0row = (u0.z >> 8) | ((u0.y >> 27) << 24);
    task.nonempty = nonempty;
    if constexpr (VAR) {
      task.dm = dm;
      const unsigned long long gid = P.path_offset + p.j;
      task.gid_lo = (uint32_t)gid;
      task.gid_hi_k = ((uint32_t)(gid >> 32) & 0xFFFFu) | ((uint32_t)p.k << 16);
    }
    return false;
  }

  // Apply a RIS selection: throughput (Eq. 15) and vertex advance.
  __device__ static bool finish_ris(const TraceParams& P, Path& p, const RisResult& r,
                                    uint32_t nonempty, Counters& cnt) {
    if (!r.ok) {
      cnt.add(ST_INVALID);
      record(P, p, 0, (uint8_t)(EV_INVALID | nonempty));
      return true;
    }
    record(P, p, 0, (uint8_t)(EV_SCATTER | nonempty));
    record(P, p, 1, (uint8_t)r.sel);
    p.fixed = false;
    p.nmed += 1;
    p.surf = -1;
    p.beta *= r.factor;
    p.x = fmaf(p.wx, r.dsel, p.x);
    p.y = fmaf(p.wy, r.dsel, p.y);
    p.z = fmaf(p.wz, r.dsel, p.z);
    kahan_add(p.L, p.Lc, r.dsel);
    p.k += 1;
    return false;
  }

  // RIS of one lane's task, candidate by candidate (any M <= MAXM).
  __device__ static RisResult ris_lane(const TraceParams& P, const RisTaskT<VAR>& T, Counters& cnt) {
    float dj[MAXM], lw[MAXM];
    float lmax = -FLT_MAX;
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
      if (j < P.M) {
        lw[j] = ris_candidate<VAR>(P, T, j, true, &dj[j], cnt);
        lmax = fmaxf(lmax, lw[j]);
      }
    }
    RisResult r{0.0f, 0.0f, -1, 0};
    if (lmax == -FLT_MAX) return r;
    float wsum = 0.0f;
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
      if (j < P.M) {
        lw[j] = lw[j] == -FLT_MAX ? 0.0f : __expf(lw[j] - lmax);
        wsum += lw[j];
      }
    }
    const float target = T.u3 * wsum;
    float prefix = 0.0f;
    int last_valid = 0;
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
      if (j < P.M) {
        prefix += lw[j];
        if (lw[j] > 0.0f) last_valid = j;
        if (VAR && (P.ris_mode & 4)) {  // reservoir: candidate j replaces the kept one when u_j W_j < w_j
          if constexpr (VAR) {
            if (lw[j] > 0.0f && reservoir_u(P, T, j) * prefix < lw[j]) r.sel = j;
          }
        } else if (r.sel < 0 && prefix > target) {
          r.sel = j;
        }
      }
    }
    if (r.sel < 0) r.sel = last_valid;
    float wsel = 0.0f;
#pragma unroll
    for (int j = 0; j < MAXM; ++j)
      if (j == r.sel) {
        wsel = lw[j];
        r.dsel = dj[j];
      }
    r.factor = P.albedo * __fdividef(wsum, wsel * (float)P.M);
    if constexpr (VAR) {
      if (P.ris_mode & 2) r.factor *= __expf(equi_lcorr(P, T, r.dsel));
    }
    r.ok = 1;
    return r;
  }

  // One vertex of a baseline path.  `out_bin`/`out_c` receive a contribution
  // to commit this step (out_bin < 0: none).  Returns true when the path ended.
  __device__ static bool step_base(const TraceParams& P, Path& p, Counters& cnt, int* out_bin,
                                   float* out_c) {
    cnt.add(ST_VERT);
    *out_bin = -1;
    if (METHOD == kPlain) {
      const float ex = P.xe[0] - p.x, ey = P.xe[1] - p.y, ez = P.xe[2] - p.z;
      const float C = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
      const float invC = 1.0f / C;
      const float SM = P.S_gate_hi - p.L, Sm = P.S_gate_lo - p.L;
      if (DARTS_RARE(!(SM > C))) {
        cnt.add(ST_EARLY);
        record(P, p, 0, EV_EARLY);
        return true;
      }
      const float dm = box_exit(P, p.x, p.y, p.z, p.wx, p.wy, p.wz);
      const float mx = fmaf(p.wx, dm, p.x) - P.xe[0], my = fmaf(p.wy, dm, p.y) - P.xe[1],
                  mz = fmaf(p.wz, dm, p.z) - P.xe[2];
      const float S_dm = dm + sqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz)));
      const float S_hi = fminf(SM, S_dm), S_lo = fmaxf(Sm, C);
      const U4 u1 = rng<kPU>(P, p.j, (uint32_t)p.k, 1);
      if (S_hi > S_lo) {
        float S;
        const float cc = connect(P, p.wx, p.wy, p.wz, C, ex * invC, ey * invC, ez * invC, S_lo,
                                 S_hi, u01(u1.w), true, &S, cnt);
        cnt.add(ST_CONN);
        const float y = ((p.L + S) - P.S_gate_lo) * P.inv_S_bin;
        int b = (int)floorf(y);
        b = min(max(b, 0), P.n_bins - 1);
        cnt.add(ST_SAMPLE);
        if (zero_weight(P, b)) cnt.add(ST_REJECT);
        *out_bin = b;
        *out_c = p.beta * cc;
        p.c += *out_c;
      }
      if (DARTS_RARE(p.k + 1 == P.K)) {
        record(P, p, 0, EV_MAXDEPTH);
        return true;
      }
      const U4 u0 = rng<kPU>(P, p.j, (uint32_t)p.k, 0);
      const float d = -log1m(u01(u0.x)) * P.inv_st;
      if (!(d < dm)) {
        cnt.add(ST_ESCAPE);
        record(P, p, 0, EV_ESCAPE);
        return true;
      }
      p.beta *= P.albedo;
      p.x = fmaf(p.wx, d, p.x);
      p.y = fmaf(p.wy, d, p.y);
      p.z = fmaf(p.wz, d, p.z);
      kahan_add(p.L, p.Lc, d);
      record(P, p, 0, EV_SCATTER);
    } else {  // vanilla: free flight, then a direct connection from the new vertex
      const float dm = box_exit(P, p.x, p.y, p.z, p.wx, p.wy, p.wz);
      const U4 u0 = rng<kPU>(P, p.j, (uint32_t)p.k, 0);
      const float d = -log1m(u01(u0.x)) * P.inv_st;
      if (!(d < dm)) {
        cnt.add(ST_ESCAPE);
        record(P, p, 0, EV_ESCAPE);
        return true;
      }
      p.beta *= P.albedo;
      p.x = fmaf(p.wx, d, p.x);
      p.y = fmaf(p.wy, d, p.y);
      p.z = fmaf(p.wz, d, p.z);
      kahan_add(p.L, p.Lc, d);
      const float ex = p.x - P.xe[0], ey = p.y - P.xe[1], ez = p.z - P.xe[2];
      const float C2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
      const float C = sqrtf(C2);
      const float cos_s = -__fdividef(ex * p.wx + ey * p.wy + ez * p.wz, C);
      const float y = ((p.L + C) - P.S_gate_lo) * P.inv_S_bin;
      cnt.add(ST_SAMPLE);
      if (zero_weight(P, (y >= 0.0f && y < (float)P.n_bins) ? min((int)y, P.n_bins - 1) : -1)) cnt.add(ST_REJECT);
      if (y >= 0.0f && y < (float)P.n_bins) {
        cnt.add(ST_CONN);
        *out_bin = min((int)y, P.n_bins - 1);
        *out_c = p.beta * hg_eval(cos_s, P.hg_a, P.hg_b, P.hg_c) * __expf(-P.sigma_t * C) * P.Ie /
                 C2;
        p.c += *out_c;
      }
      if (!(p.L + C < P.S_gate_hi)) {
        cnt.add(ST_EARLY);
        record(P, p, 0, EV_EARLY);
        return true;
      }
      if (DARTS_RARE(p.k + 1 == P.K)) {
        record(P, p, 0, EV_MAXDEPTH);
        return true;
      }
      record(P, p, 0, EV_SCATTER);
    }
    // next direction by HG sampling (f / p = 1)
    const U4 u1 = rng<kPU>(P, p.j, (uint32_t)(p.k + 1), 1);
    float sphi, cphi;
    sincos_2pi(u01(u1.z), &sphi, &cphi);
    float wx, wy, wz;
    const float xh = u01(u1.y);
    frame_dir(p.wx, p.wy, p.wz, hg_sample(P.g, xh), hg_sin(P.g, xh), sphi, cphi, &wx, &wy, &wz);
    p.wx = wx;
    p.wy = wy;
    p.wz = wz;
    p.k += 1;
    return false;
  }
};

// Commit `val` to bin `bin` of the warp-private Kahan tile; lanes with equal
// bins are serialised (one lane per distinct bin per round).
__device__ __forceinline__ void warp_commit(bool has, int bin, float val, float* wsum, float* wcomp,
                                            float* wsq, bool tile, const TraceParams& P,
                                            bool do_sq, bool merge = true) {
  if (!tile) {  // outputs zeroed before the launch: FP64 atomics into them
    const bool ok = has && DARTS_INDEX_OK(P, bin, (P.camera ? (long long)P.width * P.height : 1ll) * P.n_bins);
    if (!merge) {  // lanes rarely share a bin: each adds its own contribution
      if (ok) {
        atomicAdd(&P.hist[bin], (double)val);
        if (do_sq) atomicAdd(&P.sumsq[bin], (double)val * (double)val);
      }
      return;
    }
    const unsigned act = __ballot_sync(kFull, ok);
    if (!ok) return;
    // lanes adding to the same bin (the baselines and full-gate DARTS bin by
    // time; a one-bin gate sends every path of a pixel to one bin) add once:
    // the group's first lane adds the group's sum and sum of squares, FP64,
    // in lane order
    const unsigned grp = __match_any_sync(act, bin);
    const int lane = threadIdx.x & 31;
    double v = (double)val, q = v * v;
    if (grp != (1u << lane)) {
      double sv = 0.0, sq = 0.0;
      for (unsigned m = grp; m; m &= m - 1) {
        const double x = __shfl_sync(grp, (double)val, __ffs(m) - 1);
        sv += x;
        sq = fma(x, x, sq);
      }
      v = sv;
      q = sq;
    }
    if (lane == __ffs(grp) - 1) {
      atomicAdd(&P.hist[bin], v);
      if (do_sq) atomicAdd(&P.sumsq[bin], q);
    }
    return;
  }
  if (has && !DARTS_INDEX_OK(P, bin, P.n_bins)) has = false;
  unsigned pending = __ballot_sync(kFull, has);
  const int lane = threadIdx.x & 31;
  while (pending) {
    if (has) {
      const unsigned grp = __match_any_sync(pending, bin);
      if (lane == __ffs(grp) - 1) {
        kahan_add(wsum[bin], wcomp[bin], val);
        if (do_sq) wsq[bin] = fmaf(val, val, wsq[bin]);
        has = false;
      }
    }
    __syncwarp();
    pending = __ballot_sync(kFull, has);
  }
}

// Cooperative RIS of a warp (M = 8): every lane that passed the medium event
// publishes its task; each round the 32 lanes evaluate 4 tasks x 8 candidates,
// one candidate per lane, and the 8-lane segments reduce (max), weight
// (exp), scan (prefix sums) and select by ballot.  All lanes must call this.
template <bool VAR>
__device__ __forceinline__ void ris_warp(const TraceParams& P, bool need, const RisTaskT<VAR>& task,
                                         RisTaskT<VAR>* tasks, RisResult* results, RisResult& mine,
                                         Counters& cnt) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(kFull, need);
  if (!m) return;
  const int n = __popc(m);
  const int slot = __popc(m & ((1u << lane) - 1u));
  if (need) tasks[slot] = task;
  __syncwarp();
  const int seg = lane & 24, j = lane & 7;
  for (int base = 0; base < n; base += 4) {
    const int t = base + (lane >> 3);
    const bool act = t < n;
    const RisTaskT<VAR> T = tasks[act ? t : 0];
    float d;
    const float lw = ris_candidate<VAR>(P, T, j, act, &d, cnt);
    const bool valid = act && lw != -FLT_MAX;
    float mx = lw;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o, 8));
    const float w = valid ? __expf(lw - mx) : 0.0f;
    float pre = w;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const float y = __shfl_up_sync(kFull, pre, o, 8);
      if (j >= o) pre += y;
    }
    const float tot = __shfl_sync(kFull, pre, 7, 8);
    const unsigned vb = __ballot_sync(kFull, valid);
    const unsigned vbits = (vb >> seg) & 0xFFu;
    int sel = 0;
    if (VAR && (P.ris_mode & 4)) {  // reservoir: the last candidate j with u_j W_j < w_j is kept
      if constexpr (VAR) {
        const unsigned acc = __ballot_sync(kFull, valid && reservoir_u(P, T, j) * pre < w);
        const unsigned abits = (acc >> seg) & 0xFFu;
        sel = abits ? 31 - __clz(abits) : (vbits ? 31 - __clz(vbits) : 0);
      }
    } else {
      const unsigned gt = __ballot_sync(kFull, act && pre > T.u3 * tot);
      const unsigned gbits = (gt >> seg) & 0xFFu;
      sel = gbits ? __ffs(gbits) - 1 : (vbits ? 31 - __clz(vbits) : 0);
    }
    if (act && j == sel) {  // the selected candidate's lane writes the task's result
      RisResult r;
      r.ok = vbits != 0;
      r.sel = sel;
      r.dsel = d;
      r.factor = P.albedo * __fdividef(tot, w * 8.0f);
      if constexpr (VAR) {
        if (P.ris_mode & 2) r.factor *= __expf(equi_lcorr(P, T, d));
      }
      results[t] = r;
    }
  }
  __syncwarp();
  if (need) mine = results[slot];
  __syncwarp();
}

// Warp sum of the lanes' packed event counts (five 6-bit fields per word,
// each at most 63).  A sum over the warp needs up to 11 bits, so the fields
// are regrouped 12 bits apart before the reductions: fields 0 and 2 of a
// word, fields 1 and 3, and field 4 of both words.  Lane e adds event e to
// the warp's counters.  Warp-uniform.
template <int kEvents>
__device__ __forceinline__ void flush_events(unsigned& ev0, unsigned& ev1, unsigned* wev, int lane) {
  constexpr unsigned kEven = 0x3F03Fu, kOdd = 0xFC0FC0u;  // fields 0, 2 / 1, 3
  const unsigned a0 = __reduce_add_sync(kFull, ev0 & kEven);
  const unsigned b0 = __reduce_add_sync(kFull, (ev0 & kOdd) >> 6);
  unsigned a1 = 0, b1 = 0;
  if constexpr (kEvents > 5) {
    a1 = __reduce_add_sync(kFull, ev1 & kEven);
    b1 = __reduce_add_sync(kFull, (ev1 & kOdd) >> 6);
  }
  const unsigned c = __reduce_add_sync(kFull, (ev0 >> 24) | ((ev1 >> 24) << 12));
  const int w = lane < 5 ? 0 : 1, f = lane - 5 * w;
  const unsigned a = w ? a1 : a0, b = w ? b1 : b0;
  const unsigned v = f == 4 ? c >> (12 * w) : ((f & 1) ? b >> (6 * (f - 1)) : a >> (6 * f));
  if (lane < kEvents) wev[lane] += v & 0xFFFu;
  ev0 = ev1 = 0;
}

// (a + r) mod B for 0 <= a < B and 0 <= r < 64 without a division when B >= 64.
__device__ __forceinline__ int add_mod(int a, int r, int B) {
  const int v = a + r;
  return v < B ? v : (B >= 64 ? v - B : v % B);
}

// The per-warp path loop shared by the single-scene and the batched kernels:
// a warp starts with the ids [first, first_end) and then claims ids
// dyn_base + *counter in chunks of kPathChunk (none once dyn_base >= N, so a
// launch that fits in one wave makes no counter atomics), refills lanes whose
// path ended, runs one vertex step per iteration and commits finished paths
// into the warp tile (or the adjoint sums).
// Weight of a finished DARTS path in its bin: B / N_e, or sum W / (N_e W_b)
// under a temporal response.
template <bool GEN>
__device__ __forceinline__ float path_weight(const TraceParams& P, const Path& p) {
  if (P.wbin == nullptr) return P.wb;
  const int b = GEN ? p.bin - p.elem * P.n_bins : p.bin;
  return __ldg(P.wbin + b);
}

template <int METHOD, int MAXM, bool DEBUG, bool TILE, bool ADJ, bool GEN = false, bool VAR = false,
          bool LEAN = false>
__device__ __forceinline__ void path_loop(const TraceParams& P, const float* tab,
                                          unsigned long long* counter, unsigned long long N,
                                          float* wsum, float* wcomp, float* wsq, RisTaskT<VAR>* wtasks,
                                          RisResult* wresults, unsigned* wev, bool do_sq,
                                          float (&g_s)[3], float (&g_c)[3], float (&g_q)[3],
                                          unsigned long long first = 0, unsigned long long first_end = 0,
                                          unsigned long long dyn_base = 0) {
  const int lane = threadIdx.x & 31;
  const int B = P.n_bins;
  constexpr bool kCoop = kIsDartsM<METHOD> && MAXM == 8;
  const unsigned long long chunk = P.chunk ? P.chunk : (unsigned long long)kPathChunk;
  Counters cnt;
  Path p;
  bool alive = false;
  unsigned long long pool_next = min(first, N), pool_end = min(first_end, N);
  int pool_bin = (int)((P.bin_base + pool_next) % (unsigned long long)B);  // DARTS bin of path pool_next
  bool drained = false;
  constexpr int kEvents = (METHOD == kDarts && !GEN) ? ST_SAMPLE : ST_FP64E;
  constexpr unsigned kSpread = 0x108421u, kFields = 0x1041041u;
  unsigned ev0 = 0, ev1 = 0;  // packed per-lane event counts (6-bit fields)
  int ev_steps = 0;
  // general DARTS kernels: bin offsets o_e of the 32 consecutive sensor
  // elements from cache_e0 on, one per lane (a pixel's paths share o_e, so
  // a refill need not draw the element's Philox block for every path)
  unsigned long long cache_e0 = ~0ull;
  unsigned cache_oe = 0;

  for (;;) {
    // ---- refill lanes whose path ended (ballot + popc, warp-private id pool)
    const unsigned dead = __ballot_sync(kFull, !alive);
    if (dead && !drained) {
      const int rank = __popc(dead & ((1u << lane) - 1u));
      const int n_dead = __popc(dead);
      const unsigned long long avail = pool_end - pool_next;
      long long jn = -1;  // general kernels: the path this lane takes (initialised below)
      if (!alive && (unsigned long long)rank < avail) {
        if constexpr (GEN) {
          jn = (long long)(pool_next + rank);
        } else {
          Stepper<METHOD, MAXM, DEBUG, ADJ, GEN, VAR, LEAN>::init(P, p, pool_next + rank, add_mod(pool_bin, rank, B));
          alive = true;
        }
      }
      if ((unsigned long long)n_dead > avail) {
        unsigned long long base = N;
        if (dyn_base < N) {
          if (lane == 0) base = dyn_base + atomicAdd(counter, chunk);
          base = __shfl_sync(kFull, base, 0);
        }
        if (base >= N) {
          drained = true;
          pool_next = pool_end = 0;
        } else {
          const unsigned long long end = min(base + chunk, N);
          const int base_bin = (int)((P.bin_base + base) % (unsigned long long)B);
          const long long r2 = (long long)rank - (long long)avail;
          if (!alive && jn < 0 && r2 >= 0 && (unsigned long long)r2 < end - base) {
            if constexpr (GEN) {
              jn = (long long)(base + (unsigned long long)r2);
            } else {
              Stepper<METHOD, MAXM, DEBUG, ADJ, GEN, VAR, LEAN>::init(P, p, base + (unsigned long long)r2,
                                                                      add_mod(base_bin, (int)r2, B));
              alive = true;
            }
          }
          const int used = (int)min((unsigned long long)n_dead - avail, end - base);
          pool_next = base + used;
          pool_end = end;
          pool_bin = add_mod(base_bin, used, B);
        }
      } else {
        pool_next += (unsigned long long)n_dead;
        pool_bin = add_mod(pool_bin, n_dead, B);
      }
      if constexpr (GEN) {  // the whole warp is here (dead and drained are warp-uniform)
        int oe_pre = -1;
        unsigned long long e_pre = ~0ull;
        if constexpr (METHOD == kDarts) {
          if (LEAN || !P.wcdf) {
            const bool take = jn >= 0;
            const unsigned long long e =
                (take && P.camera) ? (P.path_offset + (unsigned long long)jn) / P.spp : 0ull;
            const bool miss = take && (e < cache_e0 || e - cache_e0 >= 32ull);
            const unsigned mm = __ballot_sync(kFull, miss);
            if (mm) {  // restart the cache at the first missing lane's element
              cache_e0 = __shfl_sync(kFull, e, __ffs(mm) - 1);
              const unsigned long long pixels = P.camera ? (unsigned long long)P.width * P.height : 1ull;
              cache_oe = element_offset<LEAN ? 2 : 10>(P, (int)((cache_e0 + (unsigned long long)lane) % pixels));
            }
            const bool in = take && e >= cache_e0 && e - cache_e0 < 32ull;
            const unsigned v = __shfl_sync(kFull, cache_oe, in ? (int)(e - cache_e0) : lane);
            if (in) oe_pre = (int)v;
            if (take && P.camera) e_pre = e;
          }
        }
        if (jn >= 0) {
          Stepper<METHOD, MAXM, DEBUG, ADJ, GEN, VAR, LEAN>::init_gen(P, p, (unsigned long long)jn, oe_pre, e_pre);
          alive = true;
        }
      }
    }
    if (!__any_sync(kFull, alive)) break;

    // ---- one vertex step
    cnt.bits = 0;
    if constexpr (METHOD == kDartsFull) {
      p.cb = -1;
      p.cb2 = -1;
    }
    bool fin = false;
    int cbin = -1, cbin2 = -1;
    float cval = 0.0f, cval2 = 0.0f;
    if (kIsDartsM<METHOD>) {
      RisTaskT<VAR> task;
      bool need = false;
      if (alive) {
        if constexpr (GEN) {
          const int st = Stepper<METHOD, MAXM, DEBUG, ADJ, GEN, VAR, LEAN>::vertex_gen(P, p, tab, cnt, task);
          fin = st == 1;
          need = st == 0;
        } else {
          fin = Stepper<METHOD, MAXM, DEBUG, ADJ, GEN, VAR, LEAN>::vertex_darts(P, p, tab, cnt, task);
          need = !fin;
        }
      }
      RisResult r;
      if (kCoop) {
        ris_warp<VAR>(P, need, task, wtasks, wresults, r, cnt);
      } else if (need) {
        r = Stepper<METHOD, MAXM, DEBUG, ADJ, GEN, VAR, LEAN>::ris_lane(P, task, cnt);
      }
      if (need) fin = Stepper<METHOD, MAXM, DEBUG, ADJ, GEN, VAR, LEAN>::finish_ris(P, p, r, task.nonempty, cnt);
      if constexpr (METHOD == kDartsFull) {
        if (alive) {
          cbin = p.cb;
          cval = P.wb * p.cv;
          cbin2 = p.cb2;
          cval2 = P.wb * p.cv2;
        }
      } else if (alive && fin) {
        cbin = p.bin;
        cval = path_weight<GEN>(P, p) * p.c;
      }
    } else if (alive) {
      if constexpr (GEN) {
        fin = Stepper<METHOD, MAXM, DEBUG, ADJ, GEN, VAR, LEAN>::step_base_gen(P, p, cnt, &cbin, &cval, &cbin2, &cval2);
        cval2 *= P.wb;
      } else {
        fin = Stepper<METHOD, MAXM, DEBUG, ADJ, GEN, VAR, LEAN>::step_base(P, p, cnt, &cbin, &cval);
      }
      cval *= P.wb;
    }
    if (DARTS_RARE(cbin >= 0 && !isfinite(cval))) {
      atomicOr(P.status, 1u);
      cval = 0.0f;
    }
    const bool has = alive && cbin >= 0;
    if (alive && fin) {
      if (DARTS_RARE(P.probe_stride && p.j >= P.probe_first && (p.j - P.probe_first) % P.probe_stride == 0)) {
        const unsigned long long slot = (p.j - P.probe_first) / P.probe_stride;
        if (slot < P.probe_count) {
          P.probe_c[slot] = p.c;
          P.probe_b[slot] = p.bin;
        }
      }
      if (DEBUG && p.j < P.N) {
        P.dbg_c[p.j] = p.c;
        P.dbg_b[p.j] = p.bin;
        P.dbg_n[p.j] = (GEN && p.miss) ? 0 : p.k + 1;
      }
    }
    if (ADJ) {
      if (alive && fin) {
        const float wgt = DARTS_INDEX_OK(P, p.bin, (P.camera ? (long long)P.width * P.height : 1ll) * P.n_bins)
                              ? (float)P.dLdh[p.bin] * path_weight<GEN>(P, p) : 0.0f;
        const float gv[3] = {wgt * p.a0, wgt * p.a1, wgt * p.a2};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          kahan_add(g_s[i], g_c[i], gv[i]);
          g_q[i] = fmaf(gv[i], gv[i], g_q[i]);
        }
      }
    } else {
      // DARTS dedicates the paths of one sensor element to distinct bins
      // (sample index + offset mod B): two lanes meet in a bin only with
      // more samples per element than bins, so the general DARTS kernels do
      // not merge lanes (the sums are the same; the baselines and full-gate
      // DARTS bin by time and merge)
      warp_commit(has, cbin, cval, wsum, wcomp, wsq, TILE, P, do_sq, !(GEN && METHOD == kDarts));
      if constexpr ((GEN && METHOD == kPlain) || METHOD == kDartsFull) {
        if (cbin2 >= 0 && !isfinite(cval2)) {
          atomicOr(P.status, 1u);
          cval2 = 0.0f;
        }
        warp_commit(alive && cbin2 >= 0, cbin2, cval2, wsum, wcomp, wsq, TILE, P, do_sq);
      }
    }
    if (fin) alive = false;
    // ---- event counts of this step, kept per lane: multiplying the 5 event
    // bits of a word by 1 + 2^5 + 2^10 + 2^15 + 2^20 puts bit i at position
    // 6i (the shifted copies land on distinct positions, so nothing carries);
    // the 6-bit fields count up to 63 steps before the warp sums them
    ev0 += ((cnt.bits & 31u) * kSpread) & kFields;
    if constexpr (kEvents > 5) ev1 += (((cnt.bits >> 5) & 31u) * kSpread) & kFields;
    if (++ev_steps == 63) {
      flush_events<kEvents>(ev0, ev1, wev, lane);
      ev_steps = 0;
    }
  }
  flush_events<kEvents>(ev0, ev1, wev, lane);
}

template <int METHOD, int MAXM, bool DEBUG, bool TILE, int BLOCK, bool ADJ = false, bool GEN = false,
          bool VAR = false, bool LEAN = false>
__global__ void __launch_bounds__(BLOCK, 1) trace_kernel(const TraceParams P) {
  extern __shared__ float4 smem4[];
  // general kernels: the sphere-culling masks and spheres come first
  float* smem = reinterpret_cast<float*>(smem4) + (GEN ? cull_bytes(P.cull_slabs) / sizeof(float) : 0);
  const int tab_floats = kIsDartsM<METHOD> ? (int)(table_smem_bytes(P.rows, P.row_stride) / sizeof(float)) : 0;
  float* tab = smem;
  constexpr int nwarps = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int B = P.n_bins;
  const bool do_sq = P.sumsq != nullptr;
  const int tile_stride = (do_sq ? 3 : 2) * B;
  constexpr bool kCoop = kIsDartsM<METHOD> && MAXM == 8;
  RisTaskT<VAR>* ris_tasks = reinterpret_cast<RisTaskT<VAR>*>(smem + tab_floats);
  RisResult* ris_results = reinterpret_cast<RisResult*>(ris_tasks + (kCoop ? nwarps * 32 : 0));
  RisTaskT<VAR>* wtasks = ris_tasks + warp * 32;
  RisResult* wresults = ris_results + warp * 32;
  float* tiles = reinterpret_cast<float*>(ris_results + (kCoop ? nwarps * 32 : 0));
  float* wsum = tiles + (size_t)warp * tile_stride;
  float* wcomp = wsum + B;
  float* wsq = wcomp + B;
  __shared__ unsigned long long blk_stats[kStatCount];
  __shared__ unsigned warp_events[nwarps][ST_FP64E];

  // stage the direction table (row stride is a multiple of 4 floats)
  if (kIsDartsM<METHOD>) {
    const float4* src = reinterpret_cast<const float4*>(P.table);
    float4* dst = reinterpret_cast<float4*>(tab);
    for (int i = threadIdx.x; i < P.rows * P.row_stride / 4; i += BLOCK) dst[i] = __ldg(src + i);
  }
  if (GEN) build_cull(P, threadIdx.x, BLOCK);
  if (TILE)
    for (int i = threadIdx.x; i < nwarps * tile_stride; i += BLOCK) tiles[i] = 0.0f;
  if (threadIdx.x < kStatCount) blk_stats[threadIdx.x] = 0;
  if (threadIdx.x < 2) s_rare[threadIdx.x] = 0;
  if (lane < ST_FP64E) warp_events[warp][lane] = 0;
  __syncthreads();
  if (kIsDartsM<METHOD>) {
    build_guides(tab, P.rows, P.row_stride, P.n_mu, threadIdx.x, BLOCK);
    __syncthreads();
  }

  // adjoint: per-lane Kahan sums of the weighted path scores and their squares
  float g_s[3] = {0.0f, 0.0f, 0.0f}, g_c[3] = {0.0f, 0.0f, 0.0f}, g_q[3] = {0.0f, 0.0f, 0.0f};
  // each warp's first chunk is fixed by its index; the counter hands out the rest
  const unsigned long long chunk = P.chunk ? P.chunk : (unsigned long long)kPathChunk;
  const unsigned long long first = ((unsigned long long)blockIdx.x * nwarps + warp) * chunk;
  const unsigned long long dyn_base = (unsigned long long)gridDim.x * nwarps * chunk;
  path_loop<METHOD, MAXM, DEBUG, TILE, ADJ, GEN, VAR, LEAN>(P, tab, P.counter, P.N, wsum, wcomp, wsq, wtasks,
                                                 wresults, warp_events[warp], do_sq, g_s, g_c, g_q, first,
                                                 first + chunk, dyn_base);

  // ---- statistics
  __syncthreads();
  if (threadIdx.x < kStatCount) {
    unsigned long long v = 0;
    if (threadIdx.x < ST_FP64E) {
      for (int w = 0; w < nwarps; ++w) v += warp_events[w][threadIdx.x];
    } else if (threadIdx.x < ST_FP64E + 2) {
      v = s_rare[threadIdx.x - ST_FP64E];
    }
    if (v) atomicAdd(&P.stats[threadIdx.x], v);
  }

  // ---- adjoint: FP64 reduction of the per-lane gradient sums into block partials
  if (ADJ) {
    __shared__ double adj_w[nwarps][6];
    double v[6];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      v[i] = (double)g_s[i] - (double)g_c[i];
      v[3 + i] = (double)g_q[i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(kFull, v[i], o);
      if (lane == 0) adj_w[warp][i] = v[i];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
      double t = 0.0;
      for (int w = 0; w < nwarps; ++w) t += adj_w[w][threadIdx.x];
      P.partials[(size_t)blockIdx.x * 6 + threadIdx.x] = t;
    }
    __threadfence();
    __shared__ unsigned last_adj;
    __syncthreads();
    if (threadIdx.x == 0) last_adj = (atomicAdd(P.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!last_adj) return;
    __threadfence();
    if (threadIdx.x < 6) {
      double t = 0.0;
      for (unsigned g = 0; g < gridDim.x; ++g) t += __ldcg(P.partials + (size_t)g * 6 + threadIdx.x);
      if (threadIdx.x < 3) P.grad3[threadIdx.x] = t;
      else if (P.grad3_sq) P.grad3_sq[threadIdx.x - 3] = t;
    }
    if (threadIdx.x == 0) *P.ticket = 0u;
    return;
  }

  // ---- flush: FP64 reduction of the warp tiles into this block's partials,
  // one 16-byte (sum, sum of squares) store per bin, coalesced over the block
  double2* part = reinterpret_cast<double2*>(P.partials) + (size_t)blockIdx.x * B;
  if (TILE) {
    for (int b = threadIdx.x; b < B; b += BLOCK) {
      double s = 0.0, q = 0.0;
      for (int w = 0; w < nwarps; ++w) {
        const float* t = tiles + (size_t)w * tile_stride;
        s += (double)t[b] - (double)t[B + b];
        if (do_sq) q += (double)t[2 * B + b];
      }
      part[b] = make_double2(s, q);
    }
  }
  // ---- last block: sum the partials in block order (no waiting: atomic ticket)
  __threadfence();
  __shared__ unsigned last;
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(P.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (TILE) {
    const double2* all = reinterpret_cast<const double2*>(P.partials);
    for (int b = threadIdx.x; b < B; b += BLOCK) {
      double s = 0.0, q = 0.0;
      for (unsigned g = 0; g < gridDim.x; ++g) {
        const double2 v = __ldcg(all + (size_t)g * B + b);
        s += v.x;
        q += v.y;
      }
      P.hist[b] = P.accumulate ? P.hist[b] + s : s;
      if (P.sumsq) P.sumsq[b] = P.accumulate ? P.sumsq[b] + q : q;
    }
  }
  if (threadIdx.x == 0) *P.ticket = 0u;
}

// ---------------------------------------------------------------------------
// Batched rendering of many media in one persistent launch.  Each CTA pops
// work items (a path range of one medium) from a global counter; when the
// medium changes it flushes its tiles into the previous medium's histogram
// (FP64 atomics), copies the new medium's parameters into shared memory and
// stages its direction table.
// ---------------------------------------------------------------------------
__global__ void zero_hists_kernel(const TraceParams* Ps) {
  const TraceParams& P = Ps[blockIdx.x];
  for (int b = threadIdx.x; b < P.n_bins; b += blockDim.x) P.hist[b] = 0.0;
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1) trace_batch_kernel(const BatchParams BP) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  __shared__ TraceParams Ps;
  __shared__ int s_item;
  __shared__ unsigned long long s_counter;
  __shared__ unsigned warp_events[BLOCK / 32][ST_FP64E];
  constexpr int nwarps = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tab_floats = (int)(table_smem_bytes(BP.rows, BP.row_stride) / sizeof(float));
  float* tab = smem;
  RisTask* ris_tasks = reinterpret_cast<RisTask*>(smem + tab_floats);
  RisResult* ris_results = reinterpret_cast<RisResult*>(ris_tasks + nwarps * 32);
  float* tiles = reinterpret_cast<float*>(ris_results + nwarps * 32);
  const int tile_stride = 2 * BP.max_bins;
  float* wsum = tiles + (size_t)warp * tile_stride;
  for (int i = threadIdx.x; i < nwarps * tile_stride; i += BLOCK) tiles[i] = 0.0f;
  if (threadIdx.x < 2) s_rare[threadIdx.x] = 0;
  if (lane < ST_FP64E) warp_events[warp][lane] = 0;
  float g_s[3] = {0.0f, 0.0f, 0.0f}, g_c[3] = {0.0f, 0.0f, 0.0f}, g_q[3] = {0.0f, 0.0f, 0.0f};
  int cur = -1;
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(BP.item_counter, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= BP.n_items) break;
    const BatchItem item = BP.items[it];
    if ((int)item.medium != cur) {
      if (cur >= 0) {
        for (int b = threadIdx.x; b < Ps.n_bins; b += BLOCK) {
          double v = 0.0;
          for (int w = 0; w < nwarps; ++w) {
            float* t = tiles + (size_t)w * tile_stride;
            v += (double)t[b] - (double)t[Ps.n_bins + b];
            t[b] = 0.0f;
            t[Ps.n_bins + b] = 0.0f;
          }
          if (v != 0.0) atomicAdd(&Ps.hist[b], v);
        }
      }
      __syncthreads();
      const uint32_t* src = reinterpret_cast<const uint32_t*>(BP.params + item.medium);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&Ps);
      for (int i = threadIdx.x; i < (int)(sizeof(TraceParams) / 4); i += BLOCK) dst[i] = src[i];
      __syncthreads();
      const float4* tsrc = reinterpret_cast<const float4*>(Ps.table);
      for (int i = threadIdx.x; i < BP.rows * BP.row_stride / 4; i += BLOCK) smem4[i] = __ldg(tsrc + i);
      __syncthreads();
      build_guides(tab, BP.rows, BP.row_stride, Ps.n_mu, threadIdx.x, BLOCK);
      cur = (int)item.medium;
    }
    if (threadIdx.x == 0) s_counter = item.first;
    __syncthreads();
    path_loop<kDarts, 8, false, true, false>(Ps, tab, &s_counter, item.first + item.count, wsum,
                                             wsum + Ps.n_bins, nullptr, ris_tasks + warp * 32,
                                             ris_results + warp * 32, warp_events[warp], false, g_s,
                                             g_c, g_q);
    __syncthreads();
  }
  if (cur >= 0) {
    for (int b = threadIdx.x; b < Ps.n_bins; b += BLOCK) {
      double v = 0.0;
      for (int w = 0; w < nwarps; ++w) {
        const float* t = tiles + (size_t)w * tile_stride;
        v += (double)t[b] - (double)t[Ps.n_bins + b];
      }
      if (v != 0.0) atomicAdd(&Ps.hist[b], v);
    }
  }
  __syncthreads();
  if (threadIdx.x < kStatCount) {
    unsigned long long v = 0;
    if (threadIdx.x < ST_FP64E) {
      for (int w = 0; w < nwarps; ++w) v += warp_events[w][threadIdx.x];
    } else if (threadIdx.x < ST_FP64E + 2) {
      v = s_rare[threadIdx.x - ST_FP64E];
    }
    if (v) atomicAdd(&BP.stats[threadIdx.x], v);
  }
}

__global__ void philox_kernel(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t n,
                              uint32_t* out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U4 r = philox4x32_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

// Paths a warp claims at a time: `cap` (kPathChunk when 0; the autotuner
// picks it), or fewer when the launch has fewer than that many paths per
// resident warp, so that a small launch (one camera frame) spreads over
// every warp instead of giving some lanes two paths in a row while other
// warps idle.
unsigned int chunk_for(unsigned long long N, int grid, int block, unsigned int cap) {
  const unsigned long long c = cap ? cap : (unsigned long long)kPathChunk;
  const unsigned long long warps = (unsigned long long)grid * (block / 32);
  const unsigned long long per = warps ? (N + warps - 1) / warps : c;
  return (unsigned int)std::max<unsigned long long>(1, std::min<unsigned long long>(per, c));
}

// Raise a kernel's dynamic shared-memory limit only when a launch needs more
// than was already granted on the current device (the attribute persists;
// setting it on every launch costs a driver call per render).
template <auto KERN>
cudaError_t smem_limit(size_t smem) {
  constexpr int kDevices = 64;
  static std::atomic<int> granted[kDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kDevices && (int)smem <= granted[dev].load(std::memory_order_relaxed)) return cudaSuccess;
  e = cudaFuncSetAttribute(KERN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev >= 0 && dev < kDevices) {
    int cur = granted[dev].load(std::memory_order_relaxed);
    while (cur < (int)smem && !granted[dev].compare_exchange_weak(cur, (int)smem)) {
    }
  }
  return e;
}

template <int METHOD, int MAXM, bool DEBUG, bool TILE, int BLOCK, bool GEN = false, bool VAR = false,
          bool LEAN = false>
cudaError_t launch_one(const TraceParams& p0, int grid, size_t smem, cudaStream_t s) {
  constexpr auto kern = trace_kernel<METHOD, MAXM, DEBUG, TILE, BLOCK, false, GEN, VAR, LEAN>;
  cudaError_t e = smem_limit<kern>(smem);
  if (e != cudaSuccess) return e;
  TraceParams p = p0;
  p.chunk = chunk_for(p.N, grid, BLOCK, p.chunk_cap);
  kern<<<grid, BLOCK, smem, s>>>(p);
  return cudaGetLastError();
}

// Block sizes: the production variant (no debug, shared-memory tile, M = 8)
// is built for 512, 640 and 768 threads; the others for 512.

}  // namespace
}  // namespace darts
