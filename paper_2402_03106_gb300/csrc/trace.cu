// trace.cu -- persistent path-tracing kernels (DARTS and the two baselines).
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
#include <cfloat>

#include "darts_device.cuh"
#include "darts_internal.h"

namespace darts {
namespace {

constexpr int kMaxM = 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

enum : int { kDarts = 0, kPlain = 1, kVanilla = 2 };
enum : int { EV_NONE = 0, EV_EARLY = 1, EV_SCATTER = 2, EV_ESCAPE = 3, EV_INVALID = 4, EV_MAXDEPTH = 5 };
// stats slots (after `paths`)
enum : int { ST_VERT = 0, ST_CONN = 1, ST_DIST = 2, ST_EARLY = 3, ST_INVALID = 4, ST_ESCAPE = 5,
             ST_FP64E = 6, ST_FP64P = 7, ST_SPARE = 8 };

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
};

struct Counters {
  unsigned v[kStatCount];
};

__device__ __forceinline__ U4 rng(const TraceParams& P, unsigned long long id, uint32_t vertex,
                                  uint32_t group) {
  const unsigned long long gid = P.path_offset + id;
  return philox4x32_10((uint32_t)gid, (uint32_t)(gid >> 32), P.stream, (vertex << 8) | group,
                       P.key0, P.key1);
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

// Control vertex on the ray (x, w) with S in [S_lo, S_hi) (Eq. 18, 21, 22).
// uniform_S selects the uniform temporal density of the baseline.  Returns
// the contribution divided by beta (0 when the range is empty) and S.
__device__ __forceinline__ float connect(const TraceParams& P, float x, float y, float z, float wx,
                                         float wy, float wz, float C, float ax, float ay, float az,
                                         float S_lo, float S_hi, float u, bool uniform_S,
                                         float* S_out, Counters& cnt) {
  const float W = S_hi - S_lo;
  float dS, conn_w;  // conn_w = exp(-sigma_t S) / p(S)
  if (!uniform_S) {
    const float em = expm1_neg(-P.sigma_t * W);  // -(1 - e^{-st W})
    dS = -log1m(-em * u) / P.sigma_t;
    // e^{-st S} / p_S = e^{-st S_lo} (1 - e^{-st W}) / st
    conn_w = __expf(-P.sigma_t * S_lo) * (-em) / P.sigma_t;
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
    // near-degenerate ellipse: solve in FP64
    const double dd = (double)delta, Cd = (double)C, Sd = (double)S_lo + (double)dS, qd = (double)q;
    const double dend = dd + Cd * qd;  // S - C mu
    const double r1d = (dd * dd + 2.0 * Sd * Cd * qd) / (2.0 * dend);
    const double td = dd * (Sd + Cd) / (2.0 * dend);
    cos_s = (float)((Cd * (1.0 - qd) - td) / r1d);
    r1 = (float)r1d;
    den = (float)dend;
    cnt.v[ST_FP64E] += 1;
  } else {
    den = fmaf(C, q, delta);                                   // S - C mu
    r1 = __fdividef(fmaf(delta, delta, 2.0f * S * C * q), 2.0f * den);  // S - t
    const float t = __fdividef(delta * (S + C), 2.0f * den);   // Eq. 18
    cos_s = __fdividef(fmaf(C, 1.0f - q, -t), r1);
  }
  *S_out = S;
  const float f = hg_eval(cos_s, P.hg_a, P.hg_b, P.hg_c);
  // sigma_s e^{-st S} f I_e / r1^2 / p(t),  p(t) = p(S) (S - C mu) / r1
  return P.sigma_s * conn_w * f * P.Ie / (r1 * den);
}

// log Phi(r, t') of Eq. 9 with s = v t' (length units), FP32 or FP64 for small s.
__device__ __forceinline__ float log_phi(const TraceParams& P, float r2, float s, double s_d,
                                         bool small, Counters& cnt) {
  if (!small) {
    const float tp = s * P.inv_v;
    return P.phi_k0 - 1.5f * __logf(tp) - __fdividef(r2 * P.phi_invk, tp) - P.sa_v * tp;
  }
  cnt.v[ST_FP64P] += 1;
  const double tp = s_d * P.inv_v_d;
  return (float)(P.phi_k0_d - 1.5 * log(tp) - (double)r2 * P.phi_invk_d / tp - P.sa_v_d * tp);
}

template <int METHOD, int MAXM, bool DEBUG>
struct Stepper {
  // Initialise a path with local index j.
  __device__ static void init(const TraceParams& P, Path& p, unsigned long long j) {
    p.x = P.xs[0];
    p.y = P.xs[1];
    p.z = P.xs[2];
    p.L = 0.0f;
    p.Lc = 0.0f;
    p.c = 0.0f;
    p.k = 0;
    p.j = j;
    p.wx = 0.0f;
    p.wy = 0.0f;
    p.wz = 1.0f;
    if (METHOD == kDarts) {
      const unsigned long long gid = P.path_offset + j;
      p.bin = (int)((gid + P.o_e) % (unsigned long long)P.n_bins);
      p.Sm0 = fmaf((float)p.bin, P.S_bin, P.S_gate_lo);
      p.SM0 = fmaf((float)(p.bin + 1), P.S_bin, P.S_gate_lo);
      p.beta = 1.0f;
    } else {
      p.bin = -1;
      const U4 u = rng(P, j, 0, 1);
      float s, c;
      sincos_2pi(u01(u.z), &s, &c);
      frame_dir(0.0f, 0.0f, 1.0f, fmaf(2.0f, u01(u.y), -1.0f), s, c, &p.wx, &p.wy, &p.wz);
      p.beta = 4.0f * kPi;
    }
  }

  __device__ static void record(const TraceParams& P, const Path& p, int slot, uint8_t val) {
    if (DEBUG && p.j < P.N && p.k < P.K) P.dbg_dec[(p.j * P.K + p.k) * 4 + slot] = val;
  }

  // One vertex of a DARTS path; returns true when the path ended.
  __device__ static bool step_darts(const TraceParams& P, Path& p, const float* tab,
                                    Counters& cnt) {
    cnt.v[ST_VERT] += 1;
    const float ex = P.xe[0] - p.x, ey = P.xe[1] - p.y, ez = P.xe[2] - p.z;
    const float C2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    const float C = sqrtf(C2);
    const float invC = 1.0f / C;
    const float ax = ex * invC, ay = ey * invC, az = ez * invC;
    const float SM = p.SM0 - p.L, Sm = p.Sm0 - p.L;
    if (!(SM > C)) {  // Sec. 5.2 early exit
      cnt.v[ST_EARLY] += 1;
      record(P, p, 0, EV_EARLY);
      return true;
    }
    // ---- direction: MIS of the EDA table and HG / uniform (Eq. 19)
    const float rho = C / SM;
    int i_rho = (int)(rho * (float)P.n_rho);
    i_rho = min(max(i_rho, 0), P.n_rho - 1);
    int i_s = (int)floorf((__log2f(SM * P.inv_smax) + 8.0f) * P.n_s_over_8);
    i_s = min(max(i_s, 0), P.n_s - 1);
    const float* row = tab + (i_rho * P.n_s + i_s) * P.row_stride;
    float gamma = rho / (rho + P.mis_alpha);
    const bool sensor = p.k == 0;
    if (sensor && P.uniform_sensor) gamma = 0.0f;
    const float gb = sensor ? 0.0f : P.g;
    const float bx = sensor ? 0.0f : p.wx, by = sensor ? 0.0f : p.wy, bz = sensor ? 1.0f : p.wz;
    const U4 u1 = rng(P, p.j, (uint32_t)p.k, 1);
    const float v0 = u01(u1.x), v1 = u01(u1.y);
    float sphi, cphi;
    sincos_2pi(u01(u1.z), &sphi, &cphi);
    float wx, wy, wz, pE, mu_b;
    int mu_bin;
    const bool eda = v0 < gamma;
    if (eda) {
      // inverse CDF: first bin whose upper edge exceeds v1
      int lo = 0, n = P.n_mu;
      while (n > 1) {
        const int half = n >> 1;
        const bool right = !(row[lo + half] > v1);
        lo = right ? lo + half : lo;
        n -= half;
      }
      const float c_lo = row[lo], c_hi = row[lo + 1];
      const float frac = __fdividef(v1 - c_lo, c_hi - c_lo);
      const float mu = fmaf((float)lo + frac, 1.0f / P.mu_scale, -1.0f);
      frame_dir(ax, ay, az, mu, sphi, cphi, &wx, &wy, &wz);
      pE = (c_hi - c_lo) * P.mu_scale * (1.0f / kTwoPi);
      mu_b = fmaf(wx, bx, fmaf(wy, by, wz * bz));
      mu_bin = lo;
    } else {
      mu_b = hg_sample(gb, v1);
      frame_dir(bx, by, bz, mu_b, sphi, cphi, &wx, &wy, &wz);
      const float mua = fmaf(wx, ax, fmaf(wy, ay, wz * az));
      int i = (int)floorf((mua + 1.0f) * P.mu_scale);
      i = min(max(i, 0), P.n_mu - 1);
      pE = (row[i + 1] - row[i]) * P.mu_scale * (1.0f / kTwoPi);
      mu_bin = i;
    }
    const float gb2 = gb * gb;
    const float pB = hg_eval(mu_b, (1.0f - gb2) * kInv4Pi, 1.0f + gb2, 2.0f * gb);
    const float f = sensor ? 1.0f : hg_eval(mu_b, P.hg_a, P.hg_b, P.hg_c);
    p.beta *= __fdividef(f, fmaf(gamma, pE - pB, pB));
    if (DEBUG) {
      record(P, p, 2, eda ? 1 : 0);
      record(P, p, 3, (uint8_t)(mu_bin & 0xFF));
    }
    // ---- control vertex (Eq. 18, 21, 22), medium boundary as the cap
    const float dm = box_exit(P, p.x, p.y, p.z, wx, wy, wz);
    const float mx = fmaf(wx, dm, p.x) - P.xe[0], my = fmaf(wy, dm, p.y) - P.xe[1],
                mz = fmaf(wz, dm, p.z) - P.xe[2];
    const float S_dm = dm + sqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz)));
    const float S_hi = fminf(SM, S_dm), S_lo = fmaxf(Sm, C);
    const bool ok = S_hi > S_lo;
    if (ok) {
      float S;
      const float cc = connect(P, p.x, p.y, p.z, wx, wy, wz, C, ax, ay, az, S_lo, S_hi,
                               u01(u1.w), false, &S, cnt);
      p.c = fmaf(p.beta, cc, p.c);
      cnt.v[ST_CONN] += 1;
    }
    const uint8_t nonempty = ok ? 0x10 : 0;
    if (p.k + 1 == P.K) {
      record(P, p, 0, EV_MAXDEPTH | nonempty);
      return true;
    }
    // ---- distance: Bernoulli medium event (Eq. 12) + DA-RIS (Eq. 13-15)
    const U4 u0 = rng(P, p.j, (uint32_t)p.k, 0);
    const float em = expm1_neg(-P.sigma_t * dm);
    const float pm = -em;
    if (!(u01(u0.x) < pm)) {
      cnt.v[ST_ESCAPE] += 1;
      record(P, p, 0, EV_ESCAPE | nonempty);
      return true;
    }
    cnt.v[ST_DIST] += 1;
    const uint32_t srow = u0.y >> 27;  // floor(32 u)
    const uint32_t e0 = u0.z >> 8;     // eps0 as a 24-bit fraction
    const float inv_st = 1.0f / P.sigma_t;
    float dj[MAXM], lw[MAXM];
    float lmax = -FLT_MAX;
    const int M = MAXM == 8 ? 8 : P.M;
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
      if (j < M) {
        const uint32_t idx = (8u * srow + (uint32_t)j) & 255u;
        const uint32_t ri24 = __brev(idx) >> 8;
        const float eps = u01(((ri24 + e0) & 0xFFFFFFu) << 8);
        const float d = -log1m(pm * eps) * inv_st;  // Eq. 14 (sign fixed)
        const float cx = fmaf(wx, d, p.x) - P.xe[0], cy = fmaf(wy, d, p.y) - P.xe[1],
                    cz = fmaf(wz, d, p.z) - P.xe[2];
        const float r2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
        const float s = SM - d;  // remaining length budget
        const bool valid = s > 0.0f && r2 < s * s;
        float l = -FLT_MAX;
        if (valid) {
          const bool small = s < P.tiny_s;
          double s_d = 0.0;
          if (small) s_d = ((double)p.SM0 - (double)p.L + (double)p.Lc) - (double)d;
          l = log_phi(P, r2, s, s_d, small, cnt);
        }
        dj[j] = d;
        lw[j] = l;
        lmax = fmaxf(lmax, l);
      }
    }
    if (lmax == -FLT_MAX) {
      cnt.v[ST_INVALID] += 1;
      record(P, p, 0, EV_INVALID | nonempty);
      return true;
    }
    float wsum = 0.0f;
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
      if (j < M) {
        const float w = lw[j] == -FLT_MAX ? 0.0f : __expf(lw[j] - lmax);
        lw[j] = w;
        wsum += w;
      }
    }
    const float target = u01(u0.w) * wsum;
    float prefix = 0.0f, dsel = 0.0f, wsel = 0.0f;
    int sel = -1, last_valid = 0;
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
      if (j < M) {
        prefix += lw[j];
        if (lw[j] > 0.0f) last_valid = j;
        if (sel < 0 && prefix > target) {
          sel = j;
          dsel = dj[j];
          wsel = lw[j];
        }
      }
    }
    if (sel < 0) {  // rounding at the top end
#pragma unroll
      for (int j = 0; j < MAXM; ++j)
        if (j == last_valid) {
          sel = j;
          dsel = dj[j];
          wsel = lw[j];
        }
    }
    p.beta *= P.albedo * __fdividef(wsum, wsel * (float)M);
    record(P, p, 1, (uint8_t)sel);
    record(P, p, 0, EV_SCATTER | nonempty);
    p.x = fmaf(wx, dsel, p.x);
    p.y = fmaf(wy, dsel, p.y);
    p.z = fmaf(wz, dsel, p.z);
    kahan_add(p.L, p.Lc, dsel);
    p.wx = wx;
    p.wy = wy;
    p.wz = wz;
    p.k += 1;
    return false;
  }

  // One vertex of a baseline path.  `out_bin`/`out_c` receive a contribution
  // to commit this step (out_bin < 0: none).  Returns true when the path ended.
  __device__ static bool step_base(const TraceParams& P, Path& p, Counters& cnt, int* out_bin,
                                   float* out_c) {
    cnt.v[ST_VERT] += 1;
    *out_bin = -1;
    if (METHOD == kPlain) {
      const float ex = P.xe[0] - p.x, ey = P.xe[1] - p.y, ez = P.xe[2] - p.z;
      const float C = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
      const float invC = 1.0f / C;
      const float SM = P.S_gate_hi - p.L, Sm = P.S_gate_lo - p.L;
      if (!(SM > C)) {
        cnt.v[ST_EARLY] += 1;
        record(P, p, 0, EV_EARLY);
        return true;
      }
      const float dm = box_exit(P, p.x, p.y, p.z, p.wx, p.wy, p.wz);
      const float mx = fmaf(p.wx, dm, p.x) - P.xe[0], my = fmaf(p.wy, dm, p.y) - P.xe[1],
                  mz = fmaf(p.wz, dm, p.z) - P.xe[2];
      const float S_dm = dm + sqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz)));
      const float S_hi = fminf(SM, S_dm), S_lo = fmaxf(Sm, C);
      const U4 u1 = rng(P, p.j, (uint32_t)p.k, 1);
      if (S_hi > S_lo) {
        float S;
        const float cc = connect(P, p.x, p.y, p.z, p.wx, p.wy, p.wz, C, ex * invC, ey * invC,
                                 ez * invC, S_lo, S_hi, u01(u1.w), true, &S, cnt);
        cnt.v[ST_CONN] += 1;
        const float y = ((p.L + S) - P.S_gate_lo) * P.inv_S_bin;
        int b = (int)floorf(y);
        b = min(max(b, 0), P.n_bins - 1);
        *out_bin = b;
        *out_c = p.beta * cc;
        p.c += *out_c;
      }
      if (p.k + 1 == P.K) {
        record(P, p, 0, EV_MAXDEPTH);
        return true;
      }
      const U4 u0 = rng(P, p.j, (uint32_t)p.k, 0);
      const float d = -log1m(u01(u0.x)) / P.sigma_t;
      if (!(d < dm)) {
        cnt.v[ST_ESCAPE] += 1;
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
      const U4 u0 = rng(P, p.j, (uint32_t)p.k, 0);
      const float d = -log1m(u01(u0.x)) / P.sigma_t;
      if (!(d < dm)) {
        cnt.v[ST_ESCAPE] += 1;
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
      const float cos_s = -(ex * p.wx + ey * p.wy + ez * p.wz) / C;
      const float y = ((p.L + C) - P.S_gate_lo) * P.inv_S_bin;
      if (y >= 0.0f && y < (float)P.n_bins) {
        cnt.v[ST_CONN] += 1;
        *out_bin = min((int)y, P.n_bins - 1);
        *out_c = p.beta * hg_eval(cos_s, P.hg_a, P.hg_b, P.hg_c) * __expf(-P.sigma_t * C) * P.Ie /
                 C2;
        p.c += *out_c;
      }
      if (!(p.L + C < P.S_gate_hi)) {
        cnt.v[ST_EARLY] += 1;
        record(P, p, 0, EV_EARLY);
        return true;
      }
      if (p.k + 1 == P.K) {
        record(P, p, 0, EV_MAXDEPTH);
        return true;
      }
      record(P, p, 0, EV_SCATTER);
    }
    // next direction by HG sampling (f / p = 1)
    const U4 u1 = rng(P, p.j, (uint32_t)(p.k + 1), 1);
    float sphi, cphi;
    sincos_2pi(u01(u1.z), &sphi, &cphi);
    float wx, wy, wz;
    frame_dir(p.wx, p.wy, p.wz, hg_sample(P.g, u01(u1.y)), sphi, cphi, &wx, &wy, &wz);
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
                                            bool do_sq) {
  if (!tile) {
    if (has) {
      atomicAdd(&P.acc[bin], (double)val);
      if (do_sq) atomicAdd(&P.acc[P.n_bins + bin], (double)val * (double)val);
    }
    return;
  }
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

template <int METHOD, int MAXM, bool DEBUG, bool TILE>
__global__ void __launch_bounds__(512, 1) trace_kernel(const TraceParams P) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int tab_floats = METHOD == kDarts ? P.rows * P.row_stride : 0;
  float* tab = smem;
  const int nwarps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int B = P.n_bins;
  float* tiles = smem + tab_floats;
  float* wsum = tiles + (size_t)warp * 3 * B;
  float* wcomp = wsum + B;
  float* wsq = wcomp + B;
  __shared__ unsigned long long blk_stats[kStatCount];

  // stage the direction table (row stride is a multiple of 4 floats)
  if (METHOD == kDarts) {
    const float4* src = reinterpret_cast<const float4*>(P.table);
    for (int i = threadIdx.x; i < tab_floats / 4; i += blockDim.x) smem4[i] = __ldg(src + i);
  }
  if (TILE)
    for (int i = threadIdx.x; i < nwarps * 3 * B; i += blockDim.x) tiles[i] = 0.0f;
  if (threadIdx.x < kStatCount) blk_stats[threadIdx.x] = 0;
  __syncthreads();

  const bool do_sq = P.sumsq != nullptr;
  Counters cnt;
#pragma unroll
  for (int i = 0; i < kStatCount; ++i) cnt.v[i] = 0;
  Path p;
  bool alive = false;
  unsigned long long pool_next = 0, pool_end = 0;
  bool drained = false;

  for (;;) {
    // ---- refill lanes whose path ended (ballot + popc, warp-private id pool)
    const unsigned dead = __ballot_sync(kFull, !alive);
    if (dead && !drained) {
      const int rank = __popc(dead & ((1u << lane) - 1u));
      const int n_dead = __popc(dead);
      const unsigned long long avail = pool_end - pool_next;
      if (!alive && (unsigned long long)rank < avail) {
        Stepper<METHOD, MAXM, DEBUG>::init(P, p, pool_next + rank);
        alive = true;
      }
      if ((unsigned long long)n_dead > avail) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(P.counter, (unsigned long long)kPathChunk);
        base = __shfl_sync(kFull, base, 0);
        if (base >= P.N) {
          drained = true;
          pool_next = pool_end = 0;
        } else {
          const unsigned long long end = min(base + (unsigned long long)kPathChunk, P.N);
          const long long r2 = (long long)rank - (long long)avail;
          if (!alive && r2 >= 0 && (unsigned long long)r2 < end - base) {
            Stepper<METHOD, MAXM, DEBUG>::init(P, p, base + (unsigned long long)r2);
            alive = true;
          }
          pool_next = base + min((unsigned long long)n_dead - avail, end - base);
          pool_end = end;
        }
      } else {
        pool_next += (unsigned long long)n_dead;
      }
    }
    if (!__any_sync(kFull, alive)) break;

    // ---- one vertex step
    bool fin = false;
    int cbin = -1;
    float cval = 0.0f;
    if (alive) {
      if (METHOD == kDarts) {
        fin = Stepper<METHOD, MAXM, DEBUG>::step_darts(P, p, tab, cnt);
        if (fin) {
          cbin = p.bin;
          cval = P.wb * p.c;
        }
      } else {
        fin = Stepper<METHOD, MAXM, DEBUG>::step_base(P, p, cnt, &cbin, &cval);
        cval *= P.wb;
      }
      if (cbin >= 0 && !isfinite(cval)) {
        atomicOr(P.status, 1u);
        cval = 0.0f;
      }
    }
    const bool has = cbin >= 0;
    if (fin) {
      if (P.probe_stride && p.j >= P.probe_first && (p.j - P.probe_first) % P.probe_stride == 0) {
        const unsigned long long slot = (p.j - P.probe_first) / P.probe_stride;
        if (slot < P.probe_count) {
          P.probe_c[slot] = p.c;
          P.probe_b[slot] = p.bin;
        }
      }
      if (DEBUG && p.j < P.N) {
        P.dbg_c[p.j] = p.c;
        P.dbg_b[p.j] = p.bin;
        P.dbg_n[p.j] = p.k + 1;
      }
    }
    warp_commit(has, cbin, cval, wsum, wcomp, wsq, TILE, P, do_sq);
    if (fin) alive = false;
  }

  // ---- statistics
#pragma unroll
  for (int i = 0; i < kStatCount; ++i) {
    unsigned v = cnt.v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0 && v) atomicAdd(&blk_stats[i], (unsigned long long)v);
  }
  __syncthreads();
  if (threadIdx.x < kStatCount && blk_stats[threadIdx.x])
    atomicAdd(&P.stats[threadIdx.x], blk_stats[threadIdx.x]);

  // ---- flush: FP64 reduction of the warp tiles into this block's partials
  double* part = P.partials + (size_t)blockIdx.x * 2 * B;
  if (TILE) {
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
      double s = 0.0, q = 0.0;
      for (int w = 0; w < nwarps; ++w) {
        const float* t = tiles + (size_t)w * 3 * B;
        s += (double)t[b] - (double)t[B + b];
        q += (double)t[2 * B + b];
      }
      part[b] = s;
      part[B + b] = q;
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
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    double s = 0.0, q = 0.0;
    if (TILE) {
      for (unsigned g = 0; g < gridDim.x; ++g) {
        const double* pg = P.partials + (size_t)g * 2 * B;
        s += __ldcg(pg + b);
        q += __ldcg(pg + B + b);
      }
    } else {
      s = __ldcg(P.acc + b);
      q = __ldcg(P.acc + B + b);
    }
    P.hist[b] = s;
    if (P.sumsq) P.sumsq[b] = q;
  }
  if (threadIdx.x == 0) *P.ticket = 0u;
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

template <int METHOD, int MAXM, bool DEBUG, bool TILE>
cudaError_t launch_one(const TraceParams& p, int grid, int block, size_t smem, cudaStream_t s) {
  auto kern = trace_kernel<METHOD, MAXM, DEBUG, TILE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, s>>>(p);
  return cudaGetLastError();
}

template <int METHOD, bool DEBUG, bool TILE>
cudaError_t launch_m(const TraceParams& p, int grid, int block, size_t smem, cudaStream_t s) {
  if (METHOD == kDarts && p.M != 8) return launch_one<METHOD, kMaxM, DEBUG, TILE>(p, grid, block, smem, s);
  return launch_one<METHOD, 8, DEBUG, TILE>(p, grid, block, smem, s);
}

template <int METHOD>
cudaError_t launch_method(const TraceParams& p, int grid, int block, bool debug, bool tile,
                          size_t smem, cudaStream_t s) {
  if (debug) return tile ? launch_m<METHOD, true, true>(p, grid, block, smem, s)
                         : launch_m<METHOD, true, false>(p, grid, block, smem, s);
  return tile ? launch_m<METHOD, false, true>(p, grid, block, smem, s)
              : launch_m<METHOD, false, false>(p, grid, block, smem, s);
}

}  // namespace

size_t trace_smem_bytes(int method, const TraceParams& p, int block, bool tile) {
  size_t b = method == kDarts ? (size_t)p.rows * p.row_stride * sizeof(float) : 0;
  if (tile) b += (size_t)(block / 32) * 3 * p.n_bins * sizeof(float);
  return b;
}

int trace_max_m() { return kMaxM; }

cudaError_t launch_trace(int method, const TraceParams& p, int grid, int block, bool debug,
                         bool tile, size_t smem, cudaStream_t s) {
  switch (method) {
    case kDarts: return launch_method<kDarts>(p, grid, block, debug, tile, smem, s);
    case kPlain: return launch_method<kPlain>(p, grid, block, debug, tile, smem, s);
    case kVanilla: return launch_method<kVanilla>(p, grid, block, debug, tile, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t n, uint32_t* out,
                          cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  philox_kernel<<<(n + 255) / 256, 256, 0, s>>>(ctr, k0, k1, n, out);
  return cudaGetLastError();
}

}  // namespace darts
