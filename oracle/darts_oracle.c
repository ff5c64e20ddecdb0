/*
 * darts_oracle.c -- plain FP64 CPU oracle for DARTS (He et al. 2024).
 *
 * TEST INFRASTRUCTURE ONLY (see darts_oracle.h).  Slow on purpose: one path
 * at a time, every step written out in the order the paper states it, no
 * blocking, fusion or algebraic shortcuts beyond what an equation states.
 *
 * Section map (paper numbering):
 *   Eq. 1-4   transient path integral and MC estimator      -> render()
 *   Eq. 5-7   residual time, recursive estimator             -> trace_darts()
 *   Eq. 9     transient diffusion Green's function           -> orc_log_phi()
 *   Eq. 10-15 DA distance sampling by RIS                    -> darts_distance()
 *   Eq. 16-18 elliptical DA direction table                  -> orc_build_table()
 *   Eq. 19    one-sample MIS of EDA and phase sampling       -> darts_direction()
 *   Eq. 20-22 elliptical control vertex (case I, box cap)    -> darts_connect()
 *   Sec. 5.2  early exit on the residual upper bound         -> trace_darts()
 *   Sec. 6    "vanilla" direct-connection PT                 -> trace_vanilla()
 *   Eq. 21 with uniform P (Jarabo et al.)                    -> trace_plain()
 */
#include "darts_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Op-count mode (ORC_OPCOUNT: this file compiled as C++ with the counting
 * number type of opcount.hpp) tallies the arithmetic of the forward
 * estimator only.  Checker bookkeeping -- decision margins, conditioning
 * numbers, event statistics, flags -- and the adjoint's score terms still
 * run but are not counted.  Outside that mode these are plain statements. */
#ifdef ORC_OPCOUNT
#define ORC_NOT_COUNTED(stmt) \
  do {                        \
    ++orc_oc::tally.paused;   \
    stmt;                     \
    --orc_oc::tally.paused;   \
  } while (0)
#define ORC_COUNT_PHILOX() orc_oc::bump(orc_oc::PHILOX)
typedef orc_oc_plain orc_tally;
#else
#define ORC_NOT_COUNTED(stmt) \
  do {                        \
    stmt;                     \
  } while (0)
#define ORC_COUNT_PHILOX() ((void)0)
typedef double orc_tally;
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from its published definition (Salmon, Moraes,    */
/* Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten   */
/* rounds of two 32x32->64 multiplies with a Weyl key schedule.             */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  ORC_COUNT_PHILOX();
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double orc_u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* Random-number layout (the paper fixes only "a Sobol row plus a uniform
 * offset", Sec. 4.3).  key = seed; counter = (path lo, path hi, stream,
 * vertex << 8 | group).  group 0 = distance, group 1 = direction and the
 * connection; vertex 0xFFFFFE = per sensor element. */
#define ORC_VERTEX_ELEMENT 0xFFFFFEu

static void orc_rng4(const orc_scene* sc, uint64_t id, uint32_t vertex, uint32_t group,
                     uint32_t out[4]) {
  uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), sc->stream, (vertex << 8) | group};
  uint32_t key[2] = {(uint32_t)sc->seed, (uint32_t)(sc->seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Small vector helpers.                                                     */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static double dist3(const double a[3], const double b[3]) {
  double d[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
  return norm3(d);
}
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }
static double near_int(double y) { return fabs(y - floor(y + 0.5)); }

/* Orthonormal frame around unit n (Duff et al., "Building an Orthonormal
 * Basis, Revisited", JCGT 2017); returns dir = mu*n + s*(cos phi*b1 + sin phi*b2). */
static void frame_dir(const double n[3], double mu, double phi, double out[3]) {
  double sign = n[2] >= 0.0 ? 1.0 : -1.0;
  double a = -1.0 / (sign + n[2]);
  double b = n[0] * n[1] * a;
  double b1[3] = {1.0 + sign * n[0] * n[0] * a, sign * b, -sign * n[0]};
  double b2[3] = {b, sign + n[1] * n[1] * a, -n[1]};
  double s = sqrt(dmax(0.0, 1.0 - mu * mu));
  double cp = cos(phi), sp = sin(phi);
  for (int i = 0; i < 3; ++i) out[i] = mu * n[i] + s * (cp * b1[i] + sp * b2[i]);
}

/* ------------------------------------------------------------------------ */
/* Eq. 9: Phi(x, t') = v / (4 pi v D t')^{3/2} exp(-r^2/(4 v D t') - sigma_a v t'), */
/* D = 1 / (3 (sigma_a + sigma_s (1 - g))); c -> v = c/eta inside the medium. */
/* ------------------------------------------------------------------------ */
double orc_log_phi(double r, double tprime, double sigma_s, double sigma_a, double g,
                   double v) {
  if (!(tprime > 0.0)) return -INFINITY; /* Heaviside step */
  double D = 1.0 / (3.0 * (sigma_a + sigma_s * (1.0 - g)));
  double vdt = v * D * tprime;
  return log(v) - 1.5 * log(4.0 * M_PI * vdt) - r * r / (4.0 * vdt) - sigma_a * v * tprime;
}

/* Henyey-Greenstein phase function (per steradian) and its inversion. */
double orc_hg_pdf(double mu, double g) {
  double den = 1.0 + g * g - 2.0 * g * mu;
  return (1.0 - g * g) / (4.0 * M_PI * den * sqrt(den));
}

double orc_hg_sample(double g, double xi) {
  if (g == 0.0) return 2.0 * xi - 1.0;
  double s = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);
  double mu = (1.0 + g * g - s * s) / (2.0 * g);
  return dmin(1.0, dmax(-1.0, mu));
}

/* d/dg log HG(mu; g) (used by the path-replay score). */
static double hg_dlog_dg(double mu, double g) {
  return -2.0 * g / (1.0 - g * g) - 3.0 * (g - mu) / (1.0 + g * g - 2.0 * g * mu);
}

/* Eq. 18 / Eq. 21: t = (S^2 - C^2) / (2 S - 2 C cos theta); r1 = S - t. */
void orc_ellipse(double S, double C, double mu, double* t, double* r1) {
  *t = (S * S - C * C) / (2.0 * S - 2.0 * C * mu);
  *r1 = S - *t;
}

/* Eq. 22 with the Jacobian written the right way round:
 * p(t) = p(S) (dt/dS)^{-1}, and from Eq. 18 dt/dS = (S - t)/(S - C cos theta). */
double orc_control_pdf(double pS, double S, double C, double mu, double r1) {
  return pS * (S - C * mu) / r1;
}

/* ------------------------------------------------------------------------ */
/* Surfaces, emitters and the camera.                                        */
/* ------------------------------------------------------------------------ */
#define ORC_EPS 1e-5

static void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static void normalize3(double a[3]) {
  double n = norm3(a);
  for (int i = 0; i < 3; ++i) a[i] /= n;
}

/* Smallest root t > ORC_EPS of |x + w t - c| = r, or INFINITY. */
static double ray_sphere(const double c[3], double r, const double x[3], const double w[3]) {
  double oc[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
  double b = dot3(oc, w), cc = dot3(oc, oc) - r * r;
  double disc = b * b - cc;
  if (disc < 0.0) return INFINITY;
  double sq = sqrt(disc);
  double t0 = -b - sq, t1 = -b + sq;
  if (t0 > ORC_EPS) return t0;
  if (t1 > ORC_EPS) return t1;
  return INFINITY;
}

/* Nearest surface or medium-boundary point along (x, w), x inside the box. */
double orc_trace_ray(const orc_scene* sc, const double x[3], const double w[3], int32_t* kind,
                     double normal[3]) {
  double d = INFINITY;
  int face = -1;
  for (int i = 0; i < 3; ++i) {
    double di = INFINITY;
    int fi = -1;
    if (w[i] > 0.0) { di = (sc->hi[i] - x[i]) / w[i]; fi = 2 * i + 1; }
    else if (w[i] < 0.0) { di = (sc->lo[i] - x[i]) / w[i]; fi = 2 * i; }
    if (di < d) { d = di; face = fi; }
  }
  d = dmax(d, 0.0);
  *kind = (face >= 0 && (sc->walls >> face) & 1) ? 1 : 0;
  normal[0] = normal[1] = normal[2] = 0.0;
  if (face >= 0) normal[face / 2] = (face & 1) ? -1.0 : 1.0;  /* walls face inward */
  for (int k = 0; k < sc->n_spheres; ++k) {
    double t = ray_sphere(sc->spheres[k], sc->spheres[k][3], x, w);
    if (t < d) {
      d = t;
      *kind = 2 + k;
      for (int i = 0; i < 3; ++i) normal[i] = (x[i] + w[i] * t - sc->spheres[k][i]) / sc->spheres[k][3];
    }
  }
  return d;
}

/* 1 when no sphere blocks the open segment a -> b (the box is convex, so its
 * walls never occlude two points inside it). */
static int visible(const orc_scene* sc, const double a[3], const double b[3]) {
  double w[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double len = norm3(w);
  for (int i = 0; i < 3; ++i) w[i] /= len;
  for (int k = 0; k < sc->n_spheres; ++k)
    if (ray_sphere(sc->spheres[k], sc->spheres[k][3], a, w) < len - ORC_EPS) return 0;
  return 1;
}

/* The emitter point of a path: chosen among the emitters with probability
 * proportional to energy, a uniform point on an area emitter (an area
 * emitter is treated as point samples, Sec. 7). */
typedef struct {
  double y[3], n[3];
  int kind;
  double energy, t0, wsel;
} emit_pt;

static void pick_emitter(const orc_scene* sc, uint64_t id, emit_pt* e);

/* Radiant intensity toward x of the sampled emitter point: E / 4 pi for an
 * isotropic point; (E / pi) max(0, cos) for a Lambertian area point sampled
 * with density 1 / area (L_e = E / (pi A)). */
static double emit_intensity(const emit_pt* e, const double x[3]) {
  if (e->kind == 0) return e->energy / (4.0 * M_PI);
  double d[3] = {x[0] - e->y[0], x[1] - e->y[1], x[2] - e->y[2]};
  double c = dot3(d, e->n) / norm3(d);
  return c > 0.0 ? e->energy / M_PI * c : 0.0;
}

/* Pinhole camera: ray of pixel `pixel` through the jittered point (jx, jy) of
 * the pixel; the path starts where the ray enters the medium box. */
int orc_camera_ray(const orc_scene* sc, int32_t pixel, double jx, double jy, double x0[3],
                   double w[3], double* leg) {
  double f[3] = {sc->look_at[0] - sc->xs[0], sc->look_at[1] - sc->xs[1], sc->look_at[2] - sc->xs[2]};
  normalize3(f);
  double r[3], u[3];
  cross3(f, sc->up, r);
  normalize3(r);
  cross3(r, f, u);
  double th = tan(0.5 * sc->fov_deg * M_PI / 180.0);
  double aspect = (double)sc->width / (double)sc->height;
  int px = pixel % sc->width, py = pixel / sc->width;
  double sx = (2.0 * (px + jx) / sc->width - 1.0) * th * aspect;
  double sy = (1.0 - 2.0 * (py + jy) / sc->height) * th;
  for (int i = 0; i < 3; ++i) w[i] = f[i] + sx * r[i] + sy * u[i];
  normalize3(w);
  int inside = 1;
  for (int i = 0; i < 3; ++i)
    if (!(sc->xs[i] >= sc->lo[i] && sc->xs[i] <= sc->hi[i])) inside = 0;
  if (inside) {
    for (int i = 0; i < 3; ++i) x0[i] = sc->xs[i];
    *leg = 0.0;
    return 1;
  }
  double tin = -INFINITY, tout = INFINITY;
  int face = -1;
  for (int i = 0; i < 3; ++i) {
    if (w[i] == 0.0) {
      if (sc->xs[i] < sc->lo[i] || sc->xs[i] > sc->hi[i]) return 0;
      continue;
    }
    double t1 = (sc->lo[i] - sc->xs[i]) / w[i], t2 = (sc->hi[i] - sc->xs[i]) / w[i];
    int f1 = 2 * i, f2 = 2 * i + 1;
    if (t1 > t2) { double tt = t1; t1 = t2; t2 = tt; int ff = f1; f1 = f2; f2 = ff; }
    if (t1 > tin) { tin = t1; face = f1; }
    if (t2 < tout) tout = t2;
  }
  if (!(tin <= tout) || tout <= 0.0 || tin < 0.0) return 0;
  if (face >= 0 && (sc->walls >> face) & 1) return 0; /* opaque wall seen from outside */
  for (int i = 0; i < 3; ++i) x0[i] = sc->xs[i] + w[i] * tin;
  *leg = tin;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [-1, 1] by Newton iteration on P_n.               */
/* ------------------------------------------------------------------------ */
void orc_gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

double orc_radical_inverse2(uint32_t i) {
  double f = 0.5, r = 0.0;
  while (i) {
    if (i & 1u) r += f;
    i >>= 1;
    f *= 0.5;
  }
  return r;
}

/* ------------------------------------------------------------------------ */
/* Elliptical DA direction table (Sec. 5.1, Eq. 16-18).                      */
/* Conditioning cells: rho = C/S uniform on [0,1) in n_rho cells; S          */
/* log-spaced over 8 octaves below S_max = v (t_max - t0) in n_s cells.      */
/* Each cell is integrated at its centre; mu in [-1,1] in n_mu equal bins.    */
/* ------------------------------------------------------------------------ */
static double table_smax(const orc_scene* sc) {
  /* one table per medium: S_max of the earliest emitter */
  double t0 = sc->t0;
  for (int i = 0; i < sc->n_emitters; ++i) t0 = dmin(t0, sc->em[i].t0);
  return sc->v * (sc->t_max - t0);
}

static void table_cell_centre(const orc_scene* sc, int row, double* C, double* S) {
  int i_rho = row / sc->n_s, i_s = row % sc->n_s;
  double rho = (i_rho + 0.5) / sc->n_rho;
  *S = table_smax(sc) * pow(2.0, -8.0 + 8.0 * (i_s + 0.5) / sc->n_s);
  *C = rho * *S;
}

int orc_table_row(const orc_scene* sc, double C, double SM, double* margin) {
  double yr = C / SM * sc->n_rho;
  double ys = (log2(SM / table_smax(sc)) + 8.0) * sc->n_s / 8.0;
  int i_rho = (int)floor(yr);
  int i_s = (int)floor(ys);
  if (i_rho < 0) i_rho = 0;
  if (i_rho > sc->n_rho - 1) i_rho = sc->n_rho - 1;
  if (i_s < 0) i_s = 0;
  if (i_s > sc->n_s - 1) i_s = sc->n_s - 1;
  if (margin) {
    double m = 1.0;
    if (yr > 0.5 && yr < sc->n_rho - 0.5) m = dmin(m, near_int(yr) / sc->n_rho);
    if (ys > 0.5 && ys < sc->n_s - 0.5) m = dmin(m, near_int(ys) / sc->n_s);
    *margin = m;
  }
  return i_rho * sc->n_s + i_s;
}

/* Integrand of Eq. 17 at polar distance t along a direction with cosine mu
 * to the major axis: exp(-sigma_t t) Phi(r(t), (S - t)/v), r^2 = C^2 + t^2 - 2Ct mu.
 * Returned as a logarithm. */
static double eda_log_integrand(const orc_scene* sc, double C, double S, double mu, double t) {
  double st = sc->sigma_s + sc->sigma_a;
  double r2 = C * C + t * t - 2.0 * C * t * mu;
  double r = sqrt(dmax(r2, 0.0));
  return -st * t + orc_log_phi(r, (S - t) / sc->v, sc->sigma_s, sc->sigma_a, sc->g, sc->v);
}

/* Fixed rule (the table's definition in this build): per mu-bin, 4
 * Gauss-Legendre nodes in mu; per mu node, the t-range [0, t_M(mu)] of Eq. 18
 * split at the closest approach to the emitter t = C mu when that lies
 * inside (else at t_M / 2), 32 Gauss-Legendre nodes per panel. */
#define ORC_TAB_MU_NODES 4
#define ORC_TAB_T_NODES 32

static double fixed_bin_integral(const orc_scene* sc, double C, double S, int mu_bin) {
  double xm[ORC_TAB_MU_NODES], wm[ORC_TAB_MU_NODES];
  double xt[ORC_TAB_T_NODES], wt[ORC_TAB_T_NODES];
  orc_gauss_legendre(ORC_TAB_MU_NODES, xm, wm);
  orc_gauss_legendre(ORC_TAB_T_NODES, xt, wt);
  double h = 2.0 / sc->n_mu;
  double mu_lo = -1.0 + h * mu_bin;
  double total = 0.0;
  for (int a = 0; a < ORC_TAB_MU_NODES; ++a) {
    double mu = mu_lo + 0.5 * h * (xm[a] + 1.0);
    double tM = (S * S - C * C) / (2.0 * S - 2.0 * C * mu);
    double split = (C * mu > 0.0 && C * mu < tM) ? C * mu : 0.5 * tM;
    double inner = 0.0;
    for (int panel = 0; panel < 2; ++panel) {
      double lo = panel == 0 ? 0.0 : split;
      double hi = panel == 0 ? split : tM;
      for (int b = 0; b < ORC_TAB_T_NODES; ++b) {
        double t = lo + 0.5 * (hi - lo) * (xt[b] + 1.0);
        inner += 0.5 * (hi - lo) * wt[b] * exp(eda_log_integrand(sc, C, S, mu, t));
      }
    }
    total += 0.5 * h * wm[a] * inner;
  }
  return total;
}

/* Adaptive 7/15 Gauss-Kronrod (independent reference for the fixed rule). */
typedef double (*orc_fn)(const void* ctx, double x);

static const double GK_X[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                               0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                               0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                               0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double GK_WK[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                                0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                                0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                                0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double GK_WG[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                                0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

static double gk15(orc_fn f, const void* ctx, double a, double b, double* err) {
  double c = 0.5 * (a + b), hw = 0.5 * (b - a);
  double fc = f(ctx, c);
  double rk = fc * GK_WK[7], rg = fc * GK_WG[3];
  for (int j = 0; j < 7; ++j) {
    double dx = hw * GK_X[j];
    double f1 = f(ctx, c - dx), f2 = f(ctx, c + dx);
    rk += GK_WK[j] * (f1 + f2);
    if (j % 2 == 1) rg += GK_WG[j / 2] * (f1 + f2);
  }
  *err = fabs((rk - rg) * hw);
  return rk * hw;
}

static double adapt(orc_fn f, const void* ctx, double a, double b, double tol, int depth) {
  double err;
  double r = gk15(f, ctx, a, b, &err);
  if (err <= tol || depth > 40) return r;
  double m = 0.5 * (a + b);
  return adapt(f, ctx, a, m, 0.5 * tol, depth + 1) + adapt(f, ctx, m, b, 0.5 * tol, depth + 1);
}

typedef struct {
  const orc_scene* sc;
  double C, S, mu, scale;
} eda_ctx;

static double eda_t_fn(const void* p, double t) {
  const eda_ctx* c = (const eda_ctx*)p;
  return exp(eda_log_integrand(c->sc, c->C, c->S, c->mu, t) - c->scale);
}

static double eda_mu_fn(const void* p, double mu) {
  eda_ctx c = *(const eda_ctx*)p;
  c.mu = mu;
  double tM = (c.S * c.S - c.C * c.C) / (2.0 * c.S - 2.0 * c.C * mu);
  double split = (c.C * mu > 0.0 && c.C * mu < tM) ? c.C * mu : 0.5 * tM;
  return adapt(eda_t_fn, &c, 0.0, split, 1e-13, 0) + adapt(eda_t_fn, &c, split, tM, 1e-13, 0);
}

double orc_table_bin_integral(const orc_scene* sc, int row, int mu_bin, int mode) {
  double C, S;
  table_cell_centre(sc, row, &C, &S);
  if (mode == 0) return fixed_bin_integral(sc, C, S, mu_bin);
  eda_ctx c = {sc, C, S, 0.0, 0.0};
  double h = 2.0 / sc->n_mu;
  double lo = -1.0 + h * mu_bin;
  return adapt(eda_mu_fn, &c, lo, lo + h, 1e-12, 0);
}

/* Each row: integrate every mu-bin, prefix-sum, normalise so cdf[n_mu] = 1. */
int orc_build_table(const orc_scene* sc, double* cdf) {
  int rows = sc->n_rho * sc->n_s, nb = sc->n_mu;
  double* val = (double*)malloc(sizeof(double) * nb);
  if (!val) return -1;
  for (int row = 0; row < rows; ++row) {
    double C, S;
    table_cell_centre(sc, row, &C, &S);
    for (int i = 0; i < nb; ++i) val[i] = fixed_bin_integral(sc, C, S, i);
    double* out = cdf + (size_t)row * (nb + 1);
    out[0] = 0.0;
    for (int i = 0; i < nb; ++i) out[i + 1] = out[i] + val[i];
    double total = out[nb];
    if (total > 0.0 && isfinite(total)) {
      for (int i = 1; i <= nb; ++i) out[i] /= total;
    } else {
      for (int i = 1; i <= nb; ++i) out[i] = (double)i / nb; /* degenerate row: uniform */
    }
    out[nb] = 1.0;
  }
  free(val);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One path.                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  double contrib;
  int32_t bin;
  int32_t flags;
  int32_t nvert;
  /* optional per-vertex records */
  uint8_t* dec;   /* [K][4] */
  double* margin; /* [K]    */
  /* statistics */
  orc_tally n_vert, n_conn, n_conn_nonempty, n_cand, n_early, n_invalid, n_escape;
  /* per-connection output for binned methods (plain / vanilla) */
  int n_out;
  int32_t out_bin[1024];
  double out_c[1024];
  /* adjoint: per-connection scores */
  double score[3];
  int dec_sel;
  /* largest (L + S_hi) / (S_hi - S_lo) over the connections */
  orc_tally cond;
  /* sum over the MIS directions of gamma n_mu / (2 pi p_mix): the relative
   * change of the path's throughput per unit error of the table's CDF values */
  orc_tally tabcond;
  /* weight of a DARTS path in its bin: B / N_e, or sum W / (N_e W_b) */
  double wpath;
  /* connection samples with a time, and those whose time has zero weight
   * (outside the gate, in a zero-weight bin, or outside a DARTS path's bin) */
  orc_tally n_samples, n_rejected;
  /* the path's emitter point and sensor element */
  const emit_pt* E;
  int elem;
} path_rec;

#define ORC_VERTEX_INIT 0xFFFFFFu

static void pick_emitter(const orc_scene* sc, uint64_t id, emit_pt* e) {
  uint32_t u[4];
  orc_rng4(sc, id, ORC_VERTEX_INIT, 2, u);
  double tot = 0.0;
  for (int i = 0; i < sc->n_emitters; ++i) tot += sc->em[i].energy;
  int pick = sc->n_emitters - 1;
  double acc = 0.0, target = orc_u01(u[0]) * tot;
  for (int i = 0; i < sc->n_emitters; ++i) {
    acc += sc->em[i].energy;
    if (target < acc) { pick = i; break; }
  }
  const orc_emitter* m = &sc->em[pick];
  double su = orc_u01(u[1]), sv = orc_u01(u[2]);
  e->kind = m->kind;
  for (int i = 0; i < 3; ++i) e->y[i] = m->pos[i] + (m->kind ? su * m->u[i] + sv * m->v[i] : 0.0);
  cross3(m->u, m->v, e->n);
  if (m->kind) normalize3(e->n);
  e->energy = m->energy;
  e->t0 = m->t0;
  e->wsel = m->energy > 0.0 ? tot / m->energy : 0.0;
}

static void rec_margin_at(path_rec* pr, int k, double m) {
  if (pr->margin && m < pr->margin[k]) pr->margin[k] = m;
}
/* decision margins are checker bookkeeping (argument included) */
#define rec_margin(pr, k, m) ORC_NOT_COUNTED(rec_margin_at(pr, k, m))

/* Direction at vertex k (Sec. 5.1): one-sample MIS (balance heuristic) of the
 * EDA table and the base strategy -- HG about the previous direction for
 * k >= 1, the uniform sphere at the sensor vertex, and, with surf_alb > 0
 * (EDA at a Lambertian surface vertex, the direction sampler of Sec. 5.1
 * applied where the local scattering is the BRDF), the cosine lobe about the
 * surface normal held in wprev, with f = albedo / pi * cos.
 * gamma = (C/S)/(C/S + alpha) (Eq. 19).  Returns the throughput factor f/p
 * and writes the direction. */
static double darts_direction(const orc_scene* sc, const double* cdf, int k, uint64_t id,
                              const double a[3], double C, double SM, const double wprev[3],
                              double w[3], double* mu_base_out, path_rec* pr, double surf_alb) {
  int nb = sc->n_mu;
  double tab_margin;
  int row = orc_table_row(sc, C, SM, &tab_margin);
  rec_margin(pr, k, tab_margin);
  const double* crow = cdf + (size_t)row * (nb + 1);
  double rho = C / SM;
  double gamma = rho / (rho + sc->mis_alpha);
  if ((k == 0 && sc->sensor_uniform_only) || (sc->ablation & 2)) gamma = 0.0;
  double gb = (k == 0) ? 0.0 : sc->g;
  double zaxis[3] = {0.0, 0.0, 1.0};
  const double* axis = (k == 0) ? zaxis : wprev;

  uint32_t u[4];
  orc_rng4(sc, id, (uint32_t)k, 1, u);
  double u0 = orc_u01(u[0]), u1 = orc_u01(u[1]), u2 = orc_u01(u[2]);
  if (gamma > 0.0) rec_margin(pr, k, fabs(u0 - gamma));

  double pE, pB, mu_b;
  int mis_choice, mu_bin;
  if (u0 < gamma) {
    /* EDA: inverse CDF over the cos-theta bins, uniform inside the bin */
    int i = 0;
    while (i < nb - 1 && !(crow[i + 1] > u1)) ++i;
    double lo = crow[i], hi = crow[i + 1];
    rec_margin(pr, k, dmin(u1 - lo, hi - u1));
    double frac = (u1 - lo) / (hi - lo);
    double mu = -1.0 + (i + frac) * (2.0 / nb);
    double phi = 2.0 * M_PI * u2;
    rec_margin(pr, k, fabs(a[2]));
    frame_dir(a, mu, phi, w);
    pE = (hi - lo) * (nb / 2.0) / (2.0 * M_PI);
    mu_b = dot3(w, axis);
    pB = surf_alb > 0.0 ? dmax(mu_b, 0.0) / M_PI : orc_hg_pdf(mu_b, gb);
    mis_choice = 1;
    mu_bin = i;
  } else {
    mu_b = surf_alb > 0.0 ? sqrt(u1) : orc_hg_sample(gb, u1); /* cosine lobe: cos^2 uniform */
    double phi = 2.0 * M_PI * u2;
    rec_margin(pr, k, fabs(axis[2]));
    frame_dir(axis, mu_b, phi, w);
    pB = surf_alb > 0.0 ? mu_b / M_PI : orc_hg_pdf(mu_b, gb);
    double mua = dot3(w, a);
    double y = (mua + 1.0) * (nb / 2.0);
    int i = (int)floor(y);
    if (i < 0) i = 0;
    if (i > nb - 1) i = nb - 1;
    rec_margin(pr, k, near_int(y) / (nb / 2.0)); /* the bin is recorded even when gamma = 0 */
    pE = (crow[i + 1] - crow[i]) * (nb / 2.0) / (2.0 * M_PI);
    mis_choice = 0;
    mu_bin = i;
  }
  double p_mix = gamma * pE + (1.0 - gamma) * pB;
  if (gamma > 0.0) ORC_NOT_COUNTED(pr->tabcond += (orc_tally)(gamma * nb / (2.0 * M_PI) / p_mix));
  double f = (k == 0) ? 1.0 : (surf_alb > 0.0 ? surf_alb / M_PI * dmax(mu_b, 0.0) : orc_hg_pdf(mu_b, sc->g));
  if (pr->dec) {
    pr->dec[k * 4 + 2] = (uint8_t)mis_choice;
    pr->dec[k * 4 + 3] = (uint8_t)(mu_bin & 0xFF);
  }
  *mu_base_out = mu_b;
  return f / p_mix;
}

/* Elliptical control vertex on the ray (x, w), Sec. 5.2 case I with the
 * first surface or the medium boundary as the cap of case II: S ~ truncated
 * exponential on [max(S_m, C), min(S_M, S(d_m))), t from Eq. 18/21, p(t)
 * from Eq. 22; the segment to the emitter point must be unoccluded. */
static double darts_connect(const orc_scene* sc, int k, double beta, const double x[3],
                            const double w[3], double C, double Sm, double SM, double dm,
                            double u3, int uniform_S, double L, path_rec* pr, int* ok,
                            double* S_out) {
  const emit_pt* E = pr->E;
  double st = sc->sigma_s + sc->sigma_a;
  double xm[3] = {x[0] + w[0] * dm, x[1] + w[1] * dm, x[2] + w[2] * dm};
  double S_dm = dm + dist3(xm, E->y);
  double S_hi = dmin(SM, S_dm);
  double S_lo = dmax(Sm, C);
  *ok = 0;
  rec_margin(pr, k, fabs(S_hi - S_lo) / dmax(S_hi, 1e-300));
  if (!(S_hi > S_lo)) return 0.0;
  double Wd = S_hi - S_lo;
  ORC_NOT_COUNTED(if ((L + S_hi) / Wd > pr->cond) pr->cond = (orc_tally)((L + S_hi) / Wd));
  double S, pS;
  if (!uniform_S) {
    double dS = -log1p(-(1.0 - exp(-st * Wd)) * u3) / st;
    S = S_lo + dS;
    pS = st * exp(-st * dS) / (1.0 - exp(-st * Wd));
  } else {
    S = S_lo + u3 * Wd;
    pS = 1.0 / Wd;
  }
  double a[3] = {(E->y[0] - x[0]) / C, (E->y[1] - x[1]) / C, (E->y[2] - x[2]) / C};
  double mu = dot3(w, a);
  double t, r1;
  orc_ellipse(S, C, mu, &t, &r1);
  double pt = orc_control_pdf(pS, S, C, mu, r1);
  double xell[3] = {x[0] + w[0] * t, x[1] + w[1] * t, x[2] + w[2] * t};
  double cos_s = 0.0;
  for (int i = 0; i < 3; ++i) cos_s += (xell[i] - E->y[i]) / r1 * (-w[i]);
  ORC_NOT_COUNTED(if ((S - C) / C < 1.0 / 4096.0) pr->flags |= ORC_FLAG_NEAR_DEGENERATE);
  double Ie = emit_intensity(E, xell);
  double vis = (sc->n_spheres && !visible(sc, xell, E->y)) ? 0.0 : 1.0;
  double c = beta * sc->sigma_s * exp(-st * S) * orc_hg_pdf(cos_s, sc->g) * Ie * vis / (r1 * r1) / pt;
  *ok = 1;
  *S_out = S;
  ORC_NOT_COUNTED(pr->score[2] = hg_dlog_dg(cos_s, sc->g));
  return c;
}

/* Direct connection from a surface vertex xs (normal n facing the medium)
 * to the emitter point: Lambertian BRDF albedo / pi, transmittance, the
 * emitter's intensity toward xs, 1/r^2 and visibility.  Returns 0 when the
 * emitter is behind the surface. */
static double surface_connect(const orc_scene* sc, const emit_pt* E, const double xs[3],
                              const double n[3], double albedo, double* r_out) {
  double d[3] = {E->y[0] - xs[0], E->y[1] - xs[1], E->y[2] - xs[2]};
  double r = norm3(d);
  *r_out = r;
  double cs = dot3(d, n) / r;
  if (!(cs > 0.0)) return 0.0;
  if (sc->n_spheres && !visible(sc, xs, E->y)) return 0.0;
  double st = sc->sigma_s + sc->sigma_a;
  return albedo / M_PI * cs * exp(-st * r) * emit_intensity(E, xs) / (r * r);
}

/* Cosine-weighted direction about n (Malley's method on the frame of n). */
static void cosine_dir(const double n[3], double u1, double u2, double out[3]) {
  double mu = sqrt(u1);
  frame_dir(n, mu, 2.0 * M_PI * u2, out);
}

/* Candidate distances of the RIS step (Sec. 4.3).  eps_j: by default one
 * random row of the 32x8 base-2 radical-inverse table shifted by eps0 modulo
 * 1 on 24-bit integers (exact); with ablation bit 2 (i.i.d. candidates) the
 * uniforms come from Philox groups 4 + j/4, word j mod 4, of the vertex.
 * d_j: truncated exponential on [0, d_m) (Eq. 13-14, sign of Eq. 14 fixed);
 * with ablation bit 3 the equiangular density about the emitter's closest
 * approach on the ray (Kulla and Fajardo 2012, the alternative proposal the
 * paper mentions).  Writes d_j and log p_c(d_j), the candidate density
 * conditioned on d < d_m. */
static void ris_candidates(const orc_scene* sc, uint64_t id, int k, const uint32_t u0[4],
                           const double x[3], const double w[3], const double y[3], double dm,
                           double pm, double* d, double* lpc) {
  int M = sc->ris_m;
  double st = sc->sigma_s + sc->sigma_a;
  uint32_t row = (uint32_t)floor(orc_u01(u0[1]) * 32.0);
  uint32_t e0 = u0[2] >> 8; /* eps0 as a 24-bit fraction */
  /* closest approach of the emitter point to the ray: t_c, h */
  double e[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
  double tc = dot3(w, e);
  double h2 = dot3(e, e) - tc * tc;
  double hh = sqrt(dmax(h2, 1e-30));
  double th_a = atan2(-tc, hh), th_b = atan2(dm - tc, hh);
  for (int j = 0; j < M; ++j) {
    double eps;
    if (sc->ablation & 4) {
      uint32_t uj[4];
      orc_rng4(sc, id, (uint32_t)k, (uint32_t)(4 + j / 4), uj);
      eps = orc_u01(uj[j % 4]);
    } else {
      uint32_t idx = (8u * row + (uint32_t)j) & 255u;
      uint32_t ri24 = (uint32_t)(orc_radical_inverse2(idx) * 16777216.0);
      eps = (double)((ri24 + e0) & 0xFFFFFFu) * (1.0 / 16777216.0);
    }
    if (sc->ablation & 8) {
      double th = th_a + eps * (th_b - th_a);
      double t = tc + hh * tan(th);
      if (t < 0.0) t = 0.0;
      if (t >= dm) t = dm * (1.0 - 1e-12);
      d[j] = t;
      lpc[j] = log(hh / ((th_b - th_a) * (h2 + (t - tc) * (t - tc))));
    } else {
      d[j] = -log1p(-pm * eps) / st;
      lpc[j] = log(st) - st * d[j] - log(pm);
    }
  }
}

/* DA distance sampling by RIS (Sec. 4.3, Eq. 12-15).  Returns 0 = escape,
 * 1 = moved, 2 = every candidate invalid.  On success writes the new vertex
 * and multiplies *beta by sigma_s exp(-sigma_t d) W_RIS / p_m with
 * W_RIS = (1/p_hat(d)) (1/M) sum_i w_i, w_i = p_hat(d_i) / p_c(d_i).
 * Selection: one uniform against the prefix sums of the weights, or with
 * ablation bit 4 weighted reservoir sampling (the streaming form the paper
 * mentions): candidate j replaces the kept one when u_j < w_j / W_j (W_j the
 * sum of w_0..w_j), u_j from Philox groups 12 + j/4, word j mod 4 -- the same
 * selection law. */
static int darts_distance(const orc_scene* sc, int k, uint64_t id, const double x[3],
                          const double w[3], double SM, double dm, double* beta,
                          double xnew[3], double* dsel, path_rec* pr) {
  double st = sc->sigma_s + sc->sigma_a;
  uint32_t u[4];
  orc_rng4(sc, id, (uint32_t)k, 0, u);
  double u0 = orc_u01(u[0]), u3 = orc_u01(u[3]);
  /* Eq. 12: scattering-event Bernoulli */
  double pm = 1.0 - exp(-st * dm);
  rec_margin(pr, k, fabs(u0 - pm));
  if (!(u0 < pm)) return 0;
  int M = sc->ris_m;
  double lw[64], d[64], lphat[64], lpc[64];
  int valid[64];
  double xs[64][3];
  ris_candidates(sc, id, k, u, x, w, pr->E->y, dm, pm, d, lpc);
  int any = 0;
  double lmax = -INFINITY;
  for (int j = 0; j < M; ++j) {
    for (int i = 0; i < 3; ++i) xs[j][i] = x[i] + w[i] * d[j];
    double r = dist3(xs[j], pr->E->y);
    double s = SM - d[j]; /* remaining length budget to the upper gate edge */
    rec_margin(pr, k, fabs(r - s) / dmax(dmax(fabs(r), fabs(s)), 1e-300));
    valid[j] = r < s;
    if (s / sc->v < (sc->t_max - sc->t_min) / 64.0) pr->flags |= ORC_FLAG_SMALL_TPRIME;
    pr->n_cand += 1.0;
    if (sc->ablation & 1) {
      /* ablation: the target equals the candidate density -> every candidate
       * has weight 1 and the selection is a plain draw from p_c */
      lphat[j] = lpc[j];
      lw[j] = 0.0;
      valid[j] = 1;
      if (lw[j] > lmax) lmax = lw[j];
      any = 1;
    } else if (valid[j]) {
      /* Eq. 10 target (unnormalised) over the candidate density */
      double lphi = orc_log_phi(r, s / sc->v, sc->sigma_s, sc->sigma_a, sc->g, sc->v);
      lphat[j] = log(st) - st * d[j] + lphi;
      lw[j] = lphat[j] - lpc[j];
      if (lw[j] > lmax) lmax = lw[j];
      any = 1;
    } else {
      lw[j] = -INFINITY;
    }
  }
  if (!any) return 2;
  double wsum = 0.0;
  for (int j = 0; j < M; ++j) wsum += valid[j] ? exp(lw[j] - lmax) : 0.0;
  int sel = -1;
  double selm = 1.0;
  if (sc->ablation & 16) {
    double W = 0.0;
    for (int j = 0; j < M; ++j) {
      double wj = valid[j] ? exp(lw[j] - lmax) : 0.0;
      W += wj;
      if (!(wj > 0.0)) continue;
      uint32_t uj[4];
      orc_rng4(sc, id, (uint32_t)k, (uint32_t)(12 + j / 4), uj);
      double uu = orc_u01(uj[j % 4]);
      selm = dmin(selm, fabs(uu - wj / W));
      if (uu * W < wj) sel = j;
    }
  } else {
    double target = u3 * wsum, prefix = 0.0;
    for (int j = 0; j < M; ++j) {
      prefix += valid[j] ? exp(lw[j] - lmax) : 0.0;
      if (valid[j]) selm = dmin(selm, fabs(prefix - target) / wsum);
      if (sel < 0 && prefix > target) sel = j;
    }
    if (sel < 0) { /* u3 * wsum rounding at the top end */
      for (int j = M - 1; j >= 0; --j)
        if (valid[j]) { sel = j; break; }
    }
  }
  rec_margin(pr, k, selm);
  /* Eq. 15: W = (1/p_hat(d)) (1/M) sum_i w_i; throughput sigma_s exp(-sigma_t d) W / p_m */
  double log_mean_w = lmax + log(wsum) - log((double)M);
  double Wris = exp(log_mean_w - lphat[sel]);
  *beta *= sc->sigma_s * exp(-st * d[sel]) * Wris / pm;
  for (int i = 0; i < 3; ++i) xnew[i] = xs[sel][i];
  *dsel = d[sel];
  pr->dec_sel = sel;
  if (pr->dec) pr->dec[k * 4 + 1] = (uint8_t)sel;
  return 1;
}

/* Test hook: run the distance step of vertex k of path `id` from an explicit
 * state and report the candidates (distances, validity, log RIS weights),
 * the selected index and the throughput factor. */
int orc_ris_step(const orc_scene* sc, uint64_t id, int k, const double x[3], const double w[3],
                 double SM, double dm, double* d_out, double* lw_out, int32_t* valid_out,
                 int32_t* sel_out, double* factor_out) {
  path_rec pr;
  memset(&pr, 0, sizeof(pr));
  emit_pt E;
  pick_emitter(sc, id, &E);
  pr.E = &E;
  double beta = 1.0, xn[3], dsel;
  int r = darts_distance(sc, k, id, x, w, SM, dm, &beta, xn, &dsel, &pr);
  double st = sc->sigma_s + sc->sigma_a;
  uint32_t u[4];
  orc_rng4(sc, id, (uint32_t)k, 0, u);
  double pm = 1.0 - exp(-st * dm);
  double lpc[64];
  ris_candidates(sc, id, k, u, x, w, E.y, dm, pm, d_out, lpc);
  for (int j = 0; j < sc->ris_m; ++j) {
    double xs_[3] = {x[0] + w[0] * d_out[j], x[1] + w[1] * d_out[j], x[2] + w[2] * d_out[j]};
    double rr = dist3(xs_, E.y), ss = SM - d_out[j];
    valid_out[j] = rr < ss;
    double lphat = log(st) - st * d_out[j] +
                   orc_log_phi(rr, ss / sc->v, sc->sigma_s, sc->sigma_a, sc->g, sc->v);
    lw_out[j] = valid_out[j] ? lphat - lpc[j] : -INFINITY;
  }
  *sel_out = (r == 1) ? (int32_t)pr.dec_sel : -1;
  *factor_out = (r == 1) ? beta : 0.0;
  return r;
}

/* Test hook: the emitter point of path `id`: out = (y[3], n[3], wsel,
 * intensity toward q[3]). */
void orc_sample_emitter(const orc_scene* sc, uint64_t id, const double q[3], double out[8]) {
  emit_pt E;
  pick_emitter(sc, id, &E);
  for (int i = 0; i < 3; ++i) {
    out[i] = E.y[i];
    out[3 + i] = E.n[i];
  }
  out[6] = E.wsel;
  out[7] = emit_intensity(&E, q);
}

/* Sensor elements: the point sensor is element 0 and path id j; the camera's
 * pixel p owns ids p * N_e ... p * N_e + N_e - 1 with sample indices j = 0 ..
 * N_e - 1; ids beyond the last pixel wrap around to pixel 0 with j
 * continuing (N_e, N_e + 1, ...), so the shards of a larger render keep the
 * layout and cover further bins.  A DARTS path is dedicated to bin
 * (j + o_e) mod B with o_e drawn once per element (Sec. 6.2: every frame gets
 * the same number of paths, each path serves one frame). */
static void path_element(const orc_scene* sc, uint64_t id, int* elem, uint64_t* j) {
  if (sc->sensor_kind == 1) {
    uint64_t e = id / sc->paths_per_element;
    uint64_t pixels = (uint64_t)sc->width * (uint64_t)sc->height;
    *elem = (int)(e % pixels);
    *j = (e / pixels) * sc->paths_per_element + id % sc->paths_per_element;
  } else {
    *elem = 0;
    *j = id;
  }
}

static int darts_bin(const orc_scene* sc, int elem, uint64_t j, double* wpath) {
  uint32_t u[4];
  orc_rng4(sc, (uint64_t)elem, ORC_VERTEX_ELEMENT, 0, u);
  int B = sc->n_bins;
  uint64_t ne = sc->paths_per_element;
  if (!sc->weights) {
    uint64_t oe = (uint64_t)floor(orc_u01(u[0]) * B);
    if (oe >= (uint64_t)B) oe = B - 1;
    *wpath = (double)B / (double)ne;
    return (int)((j + oe) % (uint64_t)B);
  }
  /* Interval sampled from W: systematic sampling of the cumulative weights
   * at x = (i + phi) / N_e, i = (j + o_e) mod N_e, phi uniform per element;
   * bin b holds x in [C_b, C_{b+1}), C_b = sum_{i<b} W_i / sum W, so bin b
   * receives N_e P_b paths in expectation, P_b = W_b / sum W. */
  uint64_t oe = (uint64_t)floor(orc_u01(u[0]) * (double)ne);
  if (oe >= ne) oe = ne - 1;
  double x = ((double)((j + oe) % ne) + orc_u01(u[1])) / (double)ne;
  double tot = 0.0;
  for (int i = 0; i < B; ++i) tot += sc->weights[i];
  double cum = 0.0;
  int b = B - 1;
  for (int i = 0; i < B; ++i) {
    double next = cum + sc->weights[i];
    if (x < next / tot) {
      b = i;
      break;
    }
    cum = next;
  }
  *wpath = tot / ((double)ne * sc->weights[b]);
  return b;
}

/* Zero temporal weight: outside the gate or in a zero-weight bin. */
static int zero_weight(const orc_scene* sc, int b) {
  return b < 0 || (sc->weights && !(sc->weights[b] > 0.0));
}

/* Start of a path: the point sensor (direction sampled at vertex 0) or the
 * camera ray, entering the medium after `leg` (direction fixed).  Returns 0
 * when the camera ray misses the medium. */
static int path_start(const orc_scene* sc, uint64_t id, int elem, double x[3], double w[3],
                      double* L, int* fixed) {
  if (sc->sensor_kind == 1) {
    uint32_t u[4];
    orc_rng4(sc, id, ORC_VERTEX_INIT, 3, u);
    *fixed = 1;
    return orc_camera_ray(sc, elem, orc_u01(u[0]), orc_u01(u[1]), x, w, L);
  }
  for (int i = 0; i < 3; ++i) x[i] = sc->xs[i];
  w[0] = 0.0; w[1] = 0.0; w[2] = 1.0;
  *L = 0.0;
  *fixed = 0;
  return 1;
}

static double surface_albedo(const orc_scene* sc, int kind) {
  return kind == 1 ? sc->wall_albedo : sc->spheres[kind - 2][4];
}

static int time_bin(const orc_scene* sc, double T, path_rec* pr, int k);
static void emit(path_rec* pr, int b, double c);

/* A DARTS path (Sec. 4-5).  With full = 0 the path is dedicated to one time
 * bin [T_m, T_M) of its sensor element (Sec. 6.2) and adds its summed
 * contribution there.  With full = 1 ("full-gate" variant) the same samplers
 * target the whole gate [t_min, t_max): every control vertex and surface
 * connection lands in the bin of its own time, like the uniform-temporal
 * tracer, with weight 1/N_e instead of B/N_e. */
static void trace_darts(const orc_scene* sc, const double* cdf, uint64_t id, path_rec* pr,
                        const double* dLdh, double grad[3], int full) {
  int K = sc->max_bounces, B = sc->n_bins;
  double dt = (sc->t_max - sc->t_min) / B;
  int elem;
  uint64_t j;
  path_element(sc, id, &elem, &j);
  int b = full ? 0 : darts_bin(sc, elem, j, &pr->wpath);
  emit_pt E;
  pick_emitter(sc, id, &E);
  pr->E = &E;
  pr->elem = elem;
  pr->bin = full ? -1 : elem * B + b;  /* flat histogram index */
  pr->contrib = 0.0;
  double Tm = full ? sc->t_min : sc->t_min + b * dt;
  double TM = full ? sc->t_max : sc->t_min + (b + 1) * dt;
  double x[3], w[3], L;
  int fixed;
  if (!path_start(sc, id, elem, x, w, &L, &fixed)) return;
  double wprev[3] = {w[0], w[1], w[2]};
  double beta = E.wsel;
  double surf_alb = 0.0; /* albedo of the surface this vertex sits on (EDA at surfaces) */
  double gsum = 0.0;  /* sum of d log HG / dg over medium walk vertices */
  int n_med = 0;      /* medium scattering vertices of the walk */
  double wb = pr->wpath;
  for (int k = 0; k < K; ++k) {
    pr->nvert = k + 1;
    pr->n_vert += 1.0;
    double ev[3] = {E.y[0] - x[0], E.y[1] - x[1], E.y[2] - x[2]};
    double C = norm3(ev);
    double a[3] = {ev[0] / C, ev[1] / C, ev[2] / C};
    /* Eq. 5 residual bounds in length units */
    double SM = sc->v * (TM - E.t0) - L;
    double Sm = sc->v * (Tm - E.t0) - L;
    rec_margin(pr, k, fabs(SM - C) / dmax(SM, 1e-300));
    if (!(SM > C)) { /* Sec. 5.2: no causal continuation remains */
      if (pr->dec) pr->dec[k * 4] = ORC_EV_EARLY;
      pr->n_early += 1.0;
      return;
    }
    if (!fixed) {
      double wn[3], mu_b;
      beta *= darts_direction(sc, cdf, k, id, a, C, SM, wprev, wn, &mu_b, pr, surf_alb);
      if (k >= 1 && surf_alb == 0.0) ORC_NOT_COUNTED(gsum += hg_dlog_dg(mu_b, sc->g));
      for (int i = 0; i < 3; ++i) w[i] = wn[i];
      if (surf_alb > 0.0 && !(beta > 0.0)) { /* an EDA direction into the surface: nothing follows */
        if (pr->dec) pr->dec[k * 4] = ORC_EV_INVALID;
        pr->n_invalid += 1.0;
        return;
      }
      surf_alb = 0.0;
    }
    int32_t hit;
    double nrm[3];
    double dm = orc_trace_ray(sc, x, w, &hit, nrm);
    uint32_t u[4];
    orc_rng4(sc, id, (uint32_t)k, 1, u);
    int ok;
    double S;
    double c = darts_connect(sc, k, beta, x, w, C, Sm, SM, dm, orc_u01(u[3]), 0, L, pr, &ok, &S);
    pr->n_conn += 1.0;
    if (ok) pr->n_samples += 1.0;
    if (ok && full) {
      pr->n_conn_nonempty += 1.0;
      int bt = time_bin(sc, E.t0 + (L + S) / sc->v, pr, k);
      if (zero_weight(sc, bt)) pr->n_rejected += 1.0;
      if (bt >= 0) emit(pr, bt, c);
    } else if (ok) {
      pr->n_conn_nonempty += 1.0;
      pr->contrib += c;
      if (dLdh) {
        double ell = L + S, n = n_med + 1.0;
        double s0 = n / sc->sigma_s - ell, s1 = -ell, s2 = gsum + pr->score[2];
        grad[0] += dLdh[elem * B + b] * wb * c * s0;
        grad[1] += dLdh[elem * B + b] * wb * c * s1;
        grad[2] += dLdh[elem * B + b] * wb * c * s2;
      }
    }
    uint8_t ne = (uint8_t)(ok ? 0x10 : 0);
    if (k + 1 == K) {
      if (pr->dec) pr->dec[k * 4] = ORC_EV_MAXDEPTH | ne;
      return;
    }
    /* medium event (Eq. 12): DA-RIS distance; otherwise the ray reaches the
     * first surface or leaves the medium */
    double st = sc->sigma_s + sc->sigma_a;
    uint32_t u0[4];
    orc_rng4(sc, id, (uint32_t)k, 0, u0);
    double pm = 1.0 - exp(-st * dm);
    if (!(orc_u01(u0[0]) < pm)) {
      rec_margin(pr, k, fabs(orc_u01(u0[0]) - pm));
      if (hit == 0) {
        if (pr->dec) pr->dec[k * 4] = ORC_EV_ESCAPE | ne;
        pr->n_escape += 1.0;
        return;
      }
      /* surface vertex: transmittance / probability = 1 */
      for (int i = 0; i < 3; ++i) x[i] += w[i] * dm;
      L += dm;
      double alb = surface_albedo(sc, hit), r;
      double cs = beta * surface_connect(sc, &E, x, nrm, alb, &r);
      double Ltot = L + r;
      double lo = sc->v * (Tm - E.t0), hi = sc->v * (TM - E.t0);
      if (cs > 0.0) pr->n_samples += 1.0;
      if (full) {
        if (cs > 0.0) {
          int bt = time_bin(sc, E.t0 + Ltot / sc->v, pr, k);
          if (zero_weight(sc, bt)) pr->n_rejected += 1.0;
          if (bt >= 0) emit(pr, bt, cs);
        }
      } else {
        rec_margin(pr, k, dmin(fabs(Ltot - lo), fabs(Ltot - hi)) / hi);
        if (cs > 0.0 && !(Ltot >= lo && Ltot < hi)) pr->n_rejected += 1.0;
      }
      if (!full && cs > 0.0 && Ltot >= lo && Ltot < hi) {
        pr->contrib += cs;
        if (dLdh) {
          double s0 = n_med / sc->sigma_s - Ltot, s1 = -Ltot, s2 = gsum;
          grad[0] += dLdh[elem * B + b] * wb * cs * s0;
          grad[1] += dLdh[elem * B + b] * wb * cs * s1;
          grad[2] += dLdh[elem * B + b] * wb * cs * s2;
        }
      }
      if (pr->dec) pr->dec[k * 4] = ORC_EV_SURFACE | ne;
      if (sc->ablation & 32) { /* EDA at surfaces: the next vertex samples its direction */
        for (int i = 0; i < 3; ++i) wprev[i] = nrm[i];
        surf_alb = alb;
        fixed = 0;
        continue;
      }
      uint32_t us[4];
      orc_rng4(sc, id, (uint32_t)(k + 1), 1, us);
      double wn[3];
      cosine_dir(nrm, orc_u01(us[1]), orc_u01(us[2]), wn);
      for (int i = 0; i < 3; ++i) w[i] = wn[i];
      beta *= alb;
      fixed = 1;
      continue;
    }
    double xn[3], d;
    int r = darts_distance(sc, k, id, x, w, SM, dm, &beta, xn, &d, pr);
    if (r == 0) {
      if (pr->dec) pr->dec[k * 4] = ORC_EV_ESCAPE | ne;
      pr->n_escape += 1.0;
      return;
    }
    if (r == 2) {
      if (pr->dec) pr->dec[k * 4] = ORC_EV_INVALID | ne;
      pr->n_invalid += 1.0;
      return;
    }
    if (pr->dec) pr->dec[k * 4] = ORC_EV_SCATTER | ne;
    for (int i = 0; i < 3; ++i) {
      x[i] = xn[i];
      wprev[i] = w[i];
    }
    L += d;
    n_med += 1;
    fixed = 0;
  }
}

/* Bin of an absolute time for the binned baselines; -1 outside the gate. */
static int time_bin(const orc_scene* sc, double T, path_rec* pr, int k) {
  double y = (T - sc->t_min) / (sc->t_max - sc->t_min) * sc->n_bins;
  if (pr->margin && y > 0.0 && y < sc->n_bins) rec_margin(pr, k, near_int(y) / sc->n_bins);
  if (!(y >= 0.0) || !(y < sc->n_bins)) return -1;
  int b = (int)floor(y);
  return b < sc->n_bins ? b : sc->n_bins - 1;
}

static void emit(path_rec* pr, int b, double c) {
  pr->contrib += c;
  if (pr->n_out < 1024) {
    pr->out_bin[pr->n_out] = b;
    pr->out_c[pr->n_out] = c;
    pr->n_out++;
  }
}

/* Start of a baseline path: the point sensor draws a uniform direction
 * (weight 4 pi, the detector is isotropic); the camera ray has weight 1. */
static int base_start(const orc_scene* sc, uint64_t id, int elem, double x[3], double w[3],
                      double* L, double* beta) {
  int fixed;
  if (!path_start(sc, id, elem, x, w, L, &fixed)) return 0;
  if (!fixed) {
    uint32_t u[4];
    orc_rng4(sc, id, 0, 1, u);
    double mu = 2.0 * orc_u01(u[1]) - 1.0;
    double zaxis[3] = {0.0, 0.0, 1.0};
    frame_dir(zaxis, mu, 2.0 * M_PI * orc_u01(u[2]), w);
    *beta = 4.0 * M_PI;
  } else {
    *beta = 1.0;
  }
  return 1;
}

/* A surface vertex of a baseline path: direct connection binned by time,
 * then a cosine-weighted direction (BRDF cos / pdf = albedo). */
static void base_surface(const orc_scene* sc, uint64_t id, int k, const emit_pt* E, double x[3],
                         double w[3], const double nrm[3], int hit, double L, double* beta,
                         path_rec* pr) {
  double alb = surface_albedo(sc, hit), r;
  double cs = *beta * surface_connect(sc, E, x, nrm, alb, &r);
  pr->n_conn += 1.0;
  if (cs > 0.0) {
    int b = time_bin(sc, E->t0 + (L + r) / sc->v, pr, k);
    pr->n_samples += 1.0;
    if (zero_weight(sc, b)) pr->n_rejected += 1.0;
    if (b >= 0) {
      pr->n_conn_nonempty += 1.0;
      emit(pr, b, cs);
    }
  }
  uint32_t us[4];
  orc_rng4(sc, id, (uint32_t)(k + 1), 1, us);
  cosine_dir(nrm, orc_u01(us[1]), orc_u01(us[2]), w);
  *beta *= alb;
}

/* Baseline "plain transient PT" with Jarabo-style uniform temporal sampling:
 * exponential free flight, HG directions, and at every vertex a control
 * vertex along the walk direction with S uniform over the whole gate
 * (Eq. 21 with uniform P); each contribution is binned by its time. */
static void trace_plain(const orc_scene* sc, uint64_t id, path_rec* pr) {
  int K = sc->max_bounces;
  double st = sc->sigma_s + sc->sigma_a;
  int elem;
  uint64_t j;
  path_element(sc, id, &elem, &j);
  emit_pt E;
  pick_emitter(sc, id, &E);
  pr->E = &E;
  pr->elem = elem;
  pr->bin = -1;
  pr->contrib = 0.0;
  double x[3], w[3], L, beta;
  if (!base_start(sc, id, elem, x, w, &L, &beta)) return;
  beta *= E.wsel;
  double Smin_abs = sc->v * (sc->t_min - E.t0), Smax_abs = sc->v * (sc->t_max - E.t0);
  for (int k = 0; k < K; ++k) {
    pr->nvert = k + 1;
    pr->n_vert += 1.0;
    double C = dist3(E.y, x);
    double SM = Smax_abs - L, Sm = Smin_abs - L;
    if (!(SM > C)) {
      if (pr->dec) pr->dec[k * 4] = ORC_EV_EARLY;
      pr->n_early += 1.0;
      return;
    }
    int32_t hit;
    double nrm[3];
    double dm = orc_trace_ray(sc, x, w, &hit, nrm);
    uint32_t u[4];
    orc_rng4(sc, id, (uint32_t)k, 1, u);
    int ok;
    double S;
    double c = darts_connect(sc, k, beta, x, w, C, Sm, SM, dm, orc_u01(u[3]), 1, L, pr, &ok, &S);
    pr->n_conn += 1.0;
    if (ok) {
      pr->n_conn_nonempty += 1.0;
      int b = time_bin(sc, E.t0 + (L + S) / sc->v, pr, k);
      pr->n_samples += 1.0;
      if (zero_weight(sc, b)) pr->n_rejected += 1.0;
      if (b >= 0) emit(pr, b, c);
    }
    if (k + 1 == K) {
      if (pr->dec) pr->dec[k * 4] = ORC_EV_MAXDEPTH;
      return;
    }
    orc_rng4(sc, id, (uint32_t)k, 0, u);
    double d = -log1p(-orc_u01(u[0])) / st;
    if (!(d < dm)) {
      if (hit == 0) {
        if (pr->dec) pr->dec[k * 4] = ORC_EV_ESCAPE;
        pr->n_escape += 1.0;
        return;
      }
      for (int i = 0; i < 3; ++i) x[i] += w[i] * dm;
      L += dm;
      if (pr->dec) pr->dec[k * 4] = ORC_EV_SURFACE;
      base_surface(sc, id, k, &E, x, w, nrm, hit, L, &beta, pr);
      continue;
    }
    beta *= sc->sigma_s / st; /* sigma_s e^{-st d} / (st e^{-st d}) */
    for (int i = 0; i < 3; ++i) x[i] += w[i] * d;
    L += d;
    if (pr->dec) pr->dec[k * 4] = ORC_EV_SCATTER;
    orc_rng4(sc, id, (uint32_t)(k + 1), 1, u);
    double mu = orc_hg_sample(sc->g, orc_u01(u[1]));
    double wn[3];
    frame_dir(w, mu, 2.0 * M_PI * orc_u01(u[2]), wn);
    for (int i = 0; i < 3; ++i) w[i] = wn[i];
    /* HG sampled exactly: f/p = 1 */
  }
}

/* "Vanilla" transient PT (Sec. 5.2, Fig. 7): exponential free flight, HG
 * directions, a direct shadow connection to the emitter at every scattering
 * vertex, binned by the path's time. */
static void trace_vanilla(const orc_scene* sc, uint64_t id, path_rec* pr) {
  int K = sc->max_bounces;
  double st = sc->sigma_s + sc->sigma_a;
  int elem;
  uint64_t j;
  path_element(sc, id, &elem, &j);
  emit_pt E;
  pick_emitter(sc, id, &E);
  pr->E = &E;
  pr->elem = elem;
  pr->bin = -1;
  pr->contrib = 0.0;
  double x[3], w[3], L, beta;
  if (!base_start(sc, id, elem, x, w, &L, &beta)) return;
  beta *= E.wsel;
  double Smax_abs = sc->v * (sc->t_max - E.t0);
  for (int k = 0; k < K; ++k) {
    pr->nvert = k + 1;
    pr->n_vert += 1.0;
    int32_t hit;
    double nrm[3];
    double dm = orc_trace_ray(sc, x, w, &hit, nrm);
    uint32_t u[4];
    orc_rng4(sc, id, (uint32_t)k, 0, u);
    double d = -log1p(-orc_u01(u[0])) / st;
    double C;
    if (!(d < dm)) {
      if (hit == 0) {
        if (pr->dec) pr->dec[k * 4] = ORC_EV_ESCAPE;
        pr->n_escape += 1.0;
        return;
      }
      for (int i = 0; i < 3; ++i) x[i] += w[i] * dm;
      L += dm;
      C = dist3(E.y, x);
      if (k + 1 == K) {
        /* a surface vertex still closes a path of k + 1 scattering vertices */
        double alb = surface_albedo(sc, hit), r;
        double cs = beta * surface_connect(sc, &E, x, nrm, alb, &r);
        pr->n_conn += 1.0;
        if (cs > 0.0) {
          int b = time_bin(sc, E.t0 + (L + r) / sc->v, pr, k);
          pr->n_samples += 1.0;
          if (zero_weight(sc, b)) pr->n_rejected += 1.0;
          if (b >= 0) {
            pr->n_conn_nonempty += 1.0;
            emit(pr, b, cs);
          }
        }
        if (pr->dec) pr->dec[k * 4] = ORC_EV_MAXDEPTH;
        return;
      }
      base_surface(sc, id, k, &E, x, w, nrm, hit, L, &beta, pr);
      if (!(L + C < Smax_abs)) {
        if (pr->dec) pr->dec[k * 4] = ORC_EV_EARLY;
        pr->n_early += 1.0;
        return;
      }
      if (pr->dec) pr->dec[k * 4] = ORC_EV_SURFACE;
      continue;
    }
    beta *= sc->sigma_s / st;
    for (int i = 0; i < 3; ++i) x[i] += w[i] * d;
    L += d;
    /* direct connection from the new scattering vertex x_{k+1} */
    C = dist3(E.y, x);
    double cos_s = 0.0;
    for (int i = 0; i < 3; ++i) cos_s += (x[i] - E.y[i]) / C * (-w[i]);
    double vis = (sc->n_spheres && !visible(sc, x, E.y)) ? 0.0 : 1.0;
    double c = beta * orc_hg_pdf(cos_s, sc->g) * exp(-st * C) * emit_intensity(&E, x) * vis / (C * C);
    pr->n_conn += 1.0;
    int b = time_bin(sc, E.t0 + (L + C) / sc->v, pr, k);
    pr->n_samples += 1.0;
    if (zero_weight(sc, b)) pr->n_rejected += 1.0;
    if (b >= 0) {
      pr->n_conn_nonempty += 1.0;
      emit(pr, b, c);
    }
    if (!(L + C < Smax_abs)) {
      if (pr->dec) pr->dec[k * 4] = ORC_EV_EARLY;
      pr->n_early += 1.0;
      return;
    }
    if (k + 1 == K) {
      if (pr->dec) pr->dec[k * 4] = ORC_EV_MAXDEPTH;
      return;
    }
    if (pr->dec) pr->dec[k * 4] = ORC_EV_SCATTER;
    orc_rng4(sc, id, (uint32_t)(k + 1), 1, u);
    double mu = orc_hg_sample(sc->g, orc_u01(u[1]));
    double wn[3];
    frame_dir(w, mu, 2.0 * M_PI * orc_u01(u[2]), wn);
    for (int i = 0; i < 3; ++i) w[i] = wn[i];
  }
}

static void trace_one(const orc_scene* sc, int method, const double* cdf, uint64_t id,
                      path_rec* pr, const double* dLdh, double grad[3]) {
  if (method == ORC_DARTS) trace_darts(sc, cdf, id, pr, dLdh, grad, 0);
  else if (method == ORC_DARTS_FULL_GATE) trace_darts(sc, cdf, id, pr, NULL, NULL, 1);
  else if (method == ORC_PLAIN_UNIFORM_T) trace_plain(sc, id, pr);
  else trace_vanilla(sc, id, pr);
}

static int scene_ok(const orc_scene* sc, int method, const double* cdf) {
  if (!(sc->sigma_s >= 0.0) || !(sc->sigma_a >= 0.0) || !(sc->sigma_s + sc->sigma_a > 0.0)) return 0;
  if (!(fabs(sc->g) < 1.0) || !(sc->v > 0.0)) return 0;
  if (sc->n_bins < 1 || !(sc->t_max > sc->t_min) || sc->max_bounces < 1) return 0;
  if (sc->max_bounces > 1024) return 0;
  if (sc->ris_m < 1 || sc->ris_m > 32) return 0;
  if (sc->n_rho < 1 || sc->n_s < 1 || sc->n_mu < 2) return 0;
  if (!(sc->mis_alpha > 0.0)) return 0;
  if ((method == ORC_DARTS || method == ORC_DARTS_FULL_GATE) && !cdf) return 0;
  if (method < ORC_DARTS || method > ORC_DARTS_FULL_GATE) return 0;
  if (sc->paths_per_element < 1) return 0;
  if (sc->n_emitters < 1 || sc->n_emitters > ORC_MAX_EMITTERS) return 0;
  if (sc->n_spheres < 0 || sc->n_spheres > ORC_MAX_SPHERES) return 0;
  if (sc->sensor_kind == 1 && (sc->width < 1 || sc->height < 1 || !(sc->fov_deg > 0.0))) return 0;
  if (sc->weights) {
    double tot = 0.0;
    for (int b = 0; b < sc->n_bins; ++b) {
      if (!(sc->weights[b] >= 0.0) || !isfinite(sc->weights[b])) return 0;
      tot += sc->weights[b];
    }
    if (!(tot > 0.0)) return 0;
  }
  return 1;
}

int orc_trace_paths(const orc_scene* sc, int method, const double* cdf, uint64_t first,
                    uint32_t count, double* contrib, int32_t* bin, uint8_t* decisions,
                    double* margin, int32_t* flags, int32_t* nbounce, double* cond,
                    double* tabcond) {
  if (!scene_ok(sc, method, cdf)) return -1;
  int K = sc->max_bounces;
  path_rec* pr = (path_rec*)malloc(sizeof(path_rec));
  if (!pr) return -2;
  for (uint32_t i = 0; i < count; ++i) {
    memset(pr, 0, sizeof(*pr));
    if (decisions) {
      pr->dec = decisions + (size_t)i * K * 4;
      memset(pr->dec, 0, (size_t)K * 4);
      for (int k = 0; k < K; ++k) {
        pr->dec[k * 4 + 1] = 0xFF;
        pr->dec[k * 4 + 2] = 0xFF;
        pr->dec[k * 4 + 3] = 0xFF;
      }
    }
    if (margin) {
      pr->margin = margin + (size_t)i * K;
      for (int k = 0; k < K; ++k) pr->margin[k] = 1.0;
    }
    trace_one(sc, method, cdf, first + i, pr, NULL, NULL);
    if (contrib) contrib[i] = pr->contrib;
    if (bin) bin[i] = pr->bin;
    if (flags) flags[i] = pr->flags;
    if (nbounce) nbounce[i] = pr->nvert;
    if (cond) cond[i] = pr->cond;
    if (tabcond) tabcond[i] = pr->tabcond;
  }
  free(pr);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Histogram render, Eq. 4, over POSIX threads with per-thread partials      */
/* summed in thread order (deterministic).                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_scene* sc;
  int method;
  const double* cdf;
  uint64_t first, count;
  uint64_t elem_first, n_elem;  /* histogram rows held: elements [elem_first, +n_elem) */
  int outside;                  /* a path of an element outside the rows */
  double* hist;
  double* sumsq;
  double stats[ORC_N_STATS];
  const double* dLdh;
  double grad[3], grad_sq[3];
} work_t;

static void* render_worker(void* p) {
  work_t* wk = (work_t*)p;
  const orc_scene* sc = wk->sc;
  int B = sc->n_bins;
  double inv_n = 1.0 / (double)sc->paths_per_element;
  path_rec* pr = (path_rec*)malloc(sizeof(path_rec));
  double* tmp = (double*)calloc((size_t)B, sizeof(double));
  for (uint64_t i = 0; i < wk->count; ++i) {
    memset(pr, 0, sizeof(*pr));
    double g3[3] = {0.0, 0.0, 0.0};
    trace_one(sc, wk->method, wk->cdf, wk->first + i, pr, wk->dLdh, g3);
    if (wk->dLdh) {
      for (int j = 0; j < 3; ++j) {
        wk->grad[j] += g3[j];
        wk->grad_sq[j] += g3[j] * g3[j];
      }
    }
    if ((uint64_t)pr->elem < wk->elem_first || (uint64_t)pr->elem - wk->elem_first >= wk->n_elem) {
      wk->outside = 1;
      continue;
    }
    size_t row = (size_t)((uint64_t)pr->elem - wk->elem_first) * B;
    if (wk->method == ORC_DARTS) {
      double c = pr->wpath * pr->contrib;
      size_t at = row + (size_t)(pr->bin - pr->elem * B);
      wk->hist[at] += c;
      wk->sumsq[at] += c * c;
    } else {
      for (int j = 0; j < pr->n_out; ++j) tmp[pr->out_bin[j]] += inv_n * pr->out_c[j];
      for (int j = 0; j < pr->n_out; ++j) {
        int b = pr->out_bin[j];
        if (tmp[b] != 0.0) {
          wk->hist[row + b] += tmp[b];
          wk->sumsq[row + b] += tmp[b] * tmp[b];
          tmp[b] = 0.0;
        }
      }
    }
    wk->stats[0] += 1.0;
    wk->stats[1] += pr->n_vert;
    wk->stats[2] += pr->n_conn;
    wk->stats[3] += pr->n_conn_nonempty;
    wk->stats[4] += pr->n_cand;
    wk->stats[5] += pr->n_early;
    wk->stats[6] += pr->n_invalid;
    wk->stats[7] += pr->n_escape;
    wk->stats[8] += pr->n_samples;
    wk->stats[9] += pr->n_rejected;
  }
  free(tmp);
  free(pr);
  return NULL;
}

static int run_threads(const orc_scene* sc, int method, const double* cdf, uint64_t n_paths,
                       uint64_t offset, int n_threads, uint64_t elem_first, uint64_t n_elem,
                       double* hist, double* sumsq,
                       double* stats, const double* dLdh, double* grad3, double* grad3_sq) {
  if (!scene_ok(sc, method, cdf)) return -1;
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > n_paths && n_paths > 0) n_threads = (int)n_paths;
  int B = sc->n_bins;
  uint64_t elements = sc->sensor_kind == 1 ? (uint64_t)sc->width * sc->height : 1;
  if (n_elem == 0) {  /* every element */
    elem_first = 0;
    n_elem = elements;
  }
  if (elem_first >= elements || n_elem > elements - elem_first) return -1;
  size_t HB = (size_t)B * (size_t)n_elem;
  work_t* wk = (work_t*)calloc((size_t)n_threads, sizeof(work_t));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!wk || !th) return -2;
  uint64_t per = n_threads ? n_paths / (uint64_t)n_threads : 0, rem = n_paths - per * n_threads;
  uint64_t start = offset;
  for (int t = 0; t < n_threads; ++t) {
    wk[t].sc = sc;
    wk[t].method = method;
    wk[t].cdf = cdf;
    wk[t].first = start;
    wk[t].count = per + ((uint64_t)t < rem ? 1 : 0);
    start += wk[t].count;
    wk[t].elem_first = elem_first;
    wk[t].n_elem = n_elem;
    wk[t].hist = (double*)calloc(HB, sizeof(double));
    wk[t].sumsq = (double*)calloc(HB, sizeof(double));
    wk[t].dLdh = dLdh;
    pthread_create(&th[t], NULL, render_worker, &wk[t]);
  }
  int outside = 0;
  for (int t = 0; t < n_threads; ++t) {
    pthread_join(th[t], NULL);
    outside |= wk[t].outside;
  }
  if (hist) memset(hist, 0, sizeof(double) * HB);
  if (sumsq) memset(sumsq, 0, sizeof(double) * HB);
  if (stats) memset(stats, 0, sizeof(double) * ORC_N_STATS);
  if (grad3) memset(grad3, 0, sizeof(double) * 3);
  if (grad3_sq) memset(grad3_sq, 0, sizeof(double) * 3);
  for (int t = 0; t < n_threads; ++t) {
    for (size_t b = 0; b < HB; ++b) {
      if (hist) hist[b] += wk[t].hist[b];
      if (sumsq) sumsq[b] += wk[t].sumsq[b];
    }
    for (int j = 0; j < ORC_N_STATS && stats; ++j) stats[j] += wk[t].stats[j];
    for (int j = 0; j < 3; ++j) {
      if (grad3) grad3[j] += wk[t].grad[j];
      if (grad3_sq) grad3_sq[j] += wk[t].grad_sq[j];
    }
    free(wk[t].hist);
    free(wk[t].sumsq);
  }
  free(wk);
  free(th);
  return outside ? -3 : 0;
}

int orc_render(const orc_scene* sc, int method, const double* cdf, uint64_t n_paths,
               uint64_t offset, int n_threads, double* hist, double* sumsq, double* stats) {
  return run_threads(sc, method, cdf, n_paths, offset, n_threads, 0, 0, hist, sumsq, stats,
                     NULL, NULL, NULL);
}

int orc_render_window(const orc_scene* sc, int method, const double* cdf, uint64_t n_paths,
                      uint64_t offset, int n_threads, uint64_t elem_first, uint64_t n_elem,
                      double* hist, double* sumsq, double* stats) {
  if (n_elem == 0) return -1;
  return run_threads(sc, method, cdf, n_paths, offset, n_threads, elem_first, n_elem, hist,
                     sumsq, stats, NULL, NULL, NULL);
}

int orc_adjoint(const orc_scene* sc, const double* cdf, uint64_t n_paths, uint64_t offset,
                int n_threads, const double* dLdh, double* grad3, double* grad3_sq) {
  if (!dLdh || !grad3) return -1;
  return run_threads(sc, ORC_DARTS, cdf, n_paths, offset, n_threads, 0, 0, NULL, NULL, NULL,
                     dLdh, grad3, grad3_sq);
}

#ifdef ORC_OPCOUNT
/* Per-path tallies of the forward estimator's arithmetic (op-count mode
 * only): out[i][ORC_OC_TALLIES] for path first + i, in the order of
 * opcount.hpp (add, mul, div, sqrt, cmp, exp, log, trig, pow, philox), and
 * the path's vertex count in nvert[i].  Single-threaded. */
int orc_opcount_paths(const orc_scene* sc, int method, const double* cdf, uint64_t first,
                      uint32_t count, uint64_t* out, double* nvert) {
  if (!scene_ok(sc, method, cdf)) return -1;
  path_rec* pr = (path_rec*)malloc(sizeof(path_rec));
  if (!pr) return -2;
  for (uint32_t i = 0; i < count; ++i) {
    memset(pr, 0, sizeof(*pr));
    memset(&orc_oc::tally, 0, sizeof(orc_oc::tally));
    trace_one(sc, method, cdf, first + i, pr, NULL, NULL);
    for (int j = 0; j < orc_oc::N; ++j) out[(size_t)i * orc_oc::N + j] = orc_oc::tally.n[j];
    if (nvert) nvert[i] = pr->n_vert;
  }
  free(pr);
  return 0;
}
#endif
