/*
 * darts_oracle.h -- plain FP64 CPU oracle for DARTS transient path tracing.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this code; it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA library against an
 * independent, slow, obviously-correct restatement of the method:
 *   He, Du, Jiang, Jin, "DARTS: Diffusion Approximated Residual Time Sampling
 *   for Time-of-flight Rendering in Homogeneous Scattering Media" (2024).
 *
 * Everything is double precision.  The oracle shares no code, header, table
 * or constant generator with the CUDA path; only the scene description (plain
 * numbers) is common.
 */
#ifndef DARTS_ORACLE_H
#define DARTS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Rendering methods. */
enum { ORC_DARTS = 0, ORC_PLAIN_UNIFORM_T = 1, ORC_VANILLA_DIRECT = 2, ORC_DARTS_FULL_GATE = 3 };

/* Per-path event codes written to decisions[k*4+0] (low nibble). */
enum {
  ORC_EV_NONE = 0,      /* vertex not reached                                */
  ORC_EV_EARLY = 1,     /* residual bound below straight-line distance (Sec.5.2) */
  ORC_EV_SCATTER = 2,   /* connection made (maybe empty), walk continued     */
  ORC_EV_ESCAPE = 3,    /* Bernoulli medium event failed: ray leaves medium  */
  ORC_EV_INVALID = 4,   /* every RIS candidate non-causal: path ends          */
  ORC_EV_MAXDEPTH = 5,  /* k+1 == max_bounces after the connection            */
  ORC_EV_SURFACE = 6    /* the ray reached a surface: the next vertex lies on it */
};

/* Path-level flags (bit mask) reported by the per-path debug routine. */
enum {
  ORC_FLAG_NEAR_DEGENERATE = 1, /* a connection had (S-C)/C < 2^-12            */
  ORC_FLAG_SMALL_TPRIME = 2     /* a RIS candidate had t' < 2^-6 (t_max-t_min) */
};

#define ORC_MAX_EMITTERS 8
#define ORC_MAX_SPHERES 64

/* Pulse emitter: kind 0 = isotropic point; kind 1 = one-sided Lambertian
 * parallelogram pos + s u + t v (s, t in [0,1]) emitting toward u x v. */
typedef struct {
  double pos[3];
  double t0, energy;
  int32_t kind;
  double u[3], v[3];
} orc_emitter;

typedef struct {
  /* medium (Eq. 9, Eq. 12): sigma_s, sigma_a, Henyey-Greenstein g, v = c/eta */
  double sigma_s, sigma_a, g, v;
  /* medium box [lo, hi] (axis aligned, no surfaces) */
  double lo[3], hi[3];
  /* isotropic point pulse emitter: position, start time t0, energy */
  double xe[3];
  double t0, energy;
  /* isotropic point fluence sensor */
  double xs[3];
  /* time gate [t_min, t_max) split into n_bins equal bins */
  double t_min, t_max;
  int32_t n_bins;
  int32_t max_bounces;          /* K: scattering vertices per path, incl. control vertex */
  int32_t ris_m;                /* N_RIS candidates (Eq. 15)                 */
  int32_t n_rho, n_s, n_mu;     /* direction table: C/S cells, S cells, cos bins */
  double mis_alpha;             /* alpha of Eq. 19                           */
  uint64_t seed;                /* Philox key                                */
  uint32_t stream;              /* Philox stream word                        */
  int32_t sensor_uniform_only;  /* 1: no EDA at the sensor vertex            */
  uint64_t paths_per_element;   /* N_e, the per-bin weight is n_bins / N_e   */
  int32_t ablation;             /* bit 0: exponential distance sampling (RIS
                                   weights all 1, no DA target); bit 1: no EDA
                                   direction sampling (gamma = 0); bit 2:
                                   i.i.d. RIS candidates; bit 3: equiangular
                                   candidates; bit 4: reservoir selection;
                                   bit 5: EDA directions at surface vertices
                                   (MIS with the cosine lobe)                 */
  /* emitters (em[0] repeats xe/t0/energy for the single point emitter) */
  int32_t n_emitters;
  orc_emitter em[ORC_MAX_EMITTERS];
  /* sensor: 0 = isotropic point fluence detector at xs; 1 = pinhole camera at
   * xs looking at look_at, vertical field of view fov_deg, width x height
   * pixels, each pixel an element of paths_per_element paths */
  int32_t sensor_kind;
  double look_at[3], up[3];
  double fov_deg;
  int32_t width, height;
  /* opaque Lambertian surfaces: box faces set in `walls` (bit 2*axis + side,
   * side 1 = hi face) with albedo wall_albedo; spheres (cx, cy, cz, r, albedo) */
  int32_t walls;
  double wall_albedo;
  int32_t n_spheres;
  double spheres[ORC_MAX_SPHERES][5];
  /* temporal response W over the gate: weights[n_bins] >= 0, or NULL for 1
   * on every bin.  DARTS samples the target interval of a path from W
   * (Sec. 5.2; Fig. 7), so zero-weight bins receive no paths; the other
   * methods are unaffected except for counting rejected samples. */
  const double* weights;
} orc_scene;

/* Philox4x32-10 block (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Uniform double in [0,1) from a 32-bit word: (x >> 8) * 2^-24. */
double orc_u01(uint32_t x);

/* log of the transient diffusion Green's function, Eq. 9. */
double orc_log_phi(double r, double tprime, double sigma_s, double sigma_a,
                   double g, double v);

/* Henyey-Greenstein density on the sphere and its inversion sampler. */
double orc_hg_pdf(double mu, double g);
double orc_hg_sample(double g, double xi);

/* Polar distance of Eq. 18 / Eq. 21 and the control-vertex density of Eq. 22
 * (Jacobian-corrected): given S, C and mu, return t; r1 = S - t; p(t). */
void orc_ellipse(double S, double C, double mu, double* t, double* r1);
double orc_control_pdf(double pS, double S, double C, double mu, double r1);

/* n-point Gauss-Legendre rule on [-1, 1] by Newton iteration. */
void orc_gauss_legendre(int n, double* x, double* w);

/* Radical inverse in base 2 of i (van der Corput), the first Sobol dimension. */
double orc_radical_inverse2(uint32_t i);

/* Elliptical DA direction table (Eq. 16-18): CDF rows [n_rho*n_s][n_mu+1].
 * Rows are ordered row = i_rho * n_s + i_s. */
int orc_build_table(const orc_scene* sc, double* cdf);
/* Unnormalised integral of one mu-bin of one table cell.  mode 0: the fixed
 * Gauss-Legendre rule of the table; mode 1: adaptive Gauss-Kronrod in both
 * dimensions (used to pin the fixed rule). */
double orc_table_bin_integral(const orc_scene* sc, int row, int mu_bin, int mode);

/* Table cell lookup from (C, S_M). */
int orc_table_row(const orc_scene* sc, double C, double SM, double* margin);

/* Trace `count` paths with ids first .. first+count-1 one by one.
 * contrib[i]: the path's summed contribution (before the per-bin weight);
 * bin[i]: the time bin the path is dedicated to (DARTS) or -1;
 * decisions[i*K*4 + k*4 + j] (optional): per-vertex decision bytes;
 * margin[i*K + k] (optional): smallest relative distance to a decision
 * threshold met at vertex k; flags[i] (optional): ORC_FLAG_* bits;
 * nbounce[i] (optional): vertices visited; cond[i] (optional): the largest
 * (L + S_hi) / (S_hi - S_lo) over the path's control-vertex connections
 * (0 when it has none) -- how strongly an absolute error in the path length
 * L or in the window bounds [S_lo, S_hi) of Eq. 21 is magnified in the
 * contribution, a conditioning number for reduced-precision comparisons.
 * tabcond[i] (optional): the sum over the path's MIS directions of
 * gamma n_mu / (2 pi p_mix), the relative change of its throughput per unit
 * error of the direction table's CDF values (Eq. 19 evaluates p_EDA from
 * two of them).  cdf may be NULL for methods other than DARTS.  Returns 0 on
 * success. */
int orc_trace_paths(const orc_scene* sc, int method, const double* cdf,
                    uint64_t first, uint32_t count, double* contrib,
                    int32_t* bin, uint8_t* decisions, double* margin,
                    int32_t* flags, int32_t* nbounce, double* cond, double* tabcond);

/* Distance step (Eq. 12-15) of vertex k from an explicit state, for tests:
 * candidate distances, validity, log RIS weights, selected index (-1 when
 * the ray escapes or every candidate is invalid) and the throughput factor.
 * Returns 0 = escape, 1 = moved, 2 = all invalid. */
int orc_ris_step(const orc_scene* sc, uint64_t id, int k, const double x[3], const double w[3],
                 double SM, double dm, double* d_out, double* lw_out, int32_t* valid_out,
                 int32_t* sel_out, double* factor_out);

/* Full histogram render of n_paths paths starting at path id `offset`,
 * split over n_threads POSIX threads; hist/sumsq are [elements][n_bins]
 * (elements = 1 for the point sensor, width*height for the camera) and are
 * overwritten.  stats (optional, ORC_N_STATS doubles): paths, vertices,
 * connections, nonempty connections, RIS candidates, early exits,
 * all-invalid stops, escapes, connection samples with a time, and those of
 * them rejected by a zero temporal weight. */
#define ORC_N_STATS 10
int orc_render(const orc_scene* sc, int method, const double* cdf,
               uint64_t n_paths, uint64_t offset, int n_threads,
               double* hist, double* sumsq, double* stats);

/* orc_render restricted to the sensor elements [elem_first, elem_first +
 * n_elem): hist/sumsq are [n_elem][n_bins] (row i = element elem_first + i),
 * so a sample of a large camera frame needs no full-frame buffers.  Every
 * traced path must belong to the window (returns -3 otherwise). */
int orc_render_window(const orc_scene* sc, int method, const double* cdf,
                      uint64_t n_paths, uint64_t offset, int n_threads,
                      uint64_t elem_first, uint64_t n_elem,
                      double* hist, double* sumsq, double* stats);

/* Geometry test hooks: nearest surface along a ray from inside the medium
 * box (returns the distance; *kind = 0 open boundary, 1 wall, 2 sphere;
 * normal[3] the surface normal facing the ray's origin); pinhole ray of a
 * pixel and jitter (returns 0 when the ray misses the medium, else writes
 * the entry point, direction and camera-leg length). */
double orc_trace_ray(const orc_scene* sc, const double x[3], const double w[3], int32_t* kind,
                     double normal[3]);
int orc_camera_ray(const orc_scene* sc, int32_t pixel, double jx, double jy, double x0[3],
                   double w[3], double* leg);
/* The emitter point chosen by path `id`: out = (y[3], n[3], 1/selection
 * probability, radiant intensity toward q). */
void orc_sample_emitter(const orc_scene* sc, uint64_t id, const double q[3], double out[8]);

/* Path-replay score of the DARTS estimator (detached sampling):
 * grad[3] += sum over paths of dLdh[bin] * w_b * sum_v c_v * s_v, with s_v the
 * derivative of log f w.r.t. (sigma_s, sigma_a, g). */
int orc_adjoint(const orc_scene* sc, const double* cdf, uint64_t n_paths,
                uint64_t offset, int n_threads, const double* dLdh,
                double* grad3, double* grad3_sq);

/* Op-count mode only (the library oracle/opcount.py builds with
 * -DORC_OPCOUNT): per-path tallies of the forward estimator's arithmetic,
 * out[count][ORC_OC_TALLIES] = add, mul, div, sqrt, cmp, exp, log, trig, pow,
 * Philox blocks; nvert[count] (optional) the vertices of each path. */
#define ORC_OC_TALLIES 10
int orc_opcount_paths(const orc_scene* sc, int method, const double* cdf, uint64_t first,
                      uint32_t count, uint64_t* out, double* nvert);

#ifdef __cplusplus
}
#endif
#endif
