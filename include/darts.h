/*
 * darts.h -- C ABI of libdarts: GB300 (sm_103a) DARTS transient path tracing.
 *
 * DARTS (He, Du, Jiang, Jin, "Diffusion Approximated Residual Time Sampling
 * for Time-of-flight Rendering in Homogeneous Scattering Media", 2024) traces
 * paths from a sensor through a homogeneous medium.  Each path:
 *   - samples free-path distances by resampled importance sampling with the
 *     transient diffusion approximation as target (Sec. 4, Eq. 9-15);
 *   - samples directions from the tabulated elliptical DA distribution by
 *     inverse CDF, mixed with phase sampling by one-sample MIS (Sec. 5.1,
 *     Eq. 16-19);
 *   - connects every vertex to the emitter through an elliptical control
 *     vertex whose total path length lies in the path's time bin (Sec. 5.2,
 *     Eq. 18-22);
 *   - adds its contribution to a per-pixel time-bin histogram (Eq. 1, Eq. 4).
 *
 * Conventions
 *   - Plain C types only.  Pointers named *_dev are CUDA device pointers
 *     (cudaMalloc / torch CUDA tensors on the context's device); *_host are
 *     host pointers.  The caller owns every buffer it passes.
 *   - Calls are asynchronous and ordered on the context's stream unless
 *     stated otherwise.  Errors found on the device (non-finite values,
 *     bounded waits that expired) are reported by darts_sync().
 *   - Lengths and times share units: a path of length l takes l / v time
 *     (Eq. 3, v = c / eta).  Histogram bins hold time-integrated fluence per
 *     unit emitted energy (not a rate: divide by the bin width for one).
 *   - Functions never throw; they return a darts_status.  The message of the
 *     last failure on a context is available from darts_last_error().
 *   - A context is not thread-safe: calls on one context from several host
 *     threads must be serialised by the caller.  Separate contexts (one per
 *     thread or per device) are independent.
 */
#ifndef DARTS_H
#define DARTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DARTS_OK = 0,
  DARTS_ERR_INVALID_ARG = 1, /* a parameter outside its domain or a NULL required pointer */
  DARTS_ERR_CUDA = 2,        /* a CUDA runtime call failed                               */
  DARTS_ERR_OOM = 3,         /* device memory could not be allocated                     */
  DARTS_ERR_NUMERIC = 4,     /* a kernel produced a non-finite contribution              */
  DARTS_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired                       */
  DARTS_ERR_UNSUPPORTED = 6, /* a feature this build does not implement                  */
  DARTS_ERR_BOUNDS = 7       /* an index left its range on the device (checked build only,
                                libdarts_checked.so; the access was skipped)              */
} darts_status;

typedef enum {
  DARTS_METHOD_DARTS = 0,           /* Sec. 4-5: DA-RIS distance, EDA+MIS direction, ellipse */
  DARTS_METHOD_PLAIN_UNIFORM_T = 1, /* Eq. 21 with uniform P (Jarabo et al.): uniform
                                       temporal control vertex, free flight, HG      */
  DARTS_METHOD_VANILLA_DIRECT = 2,  /* Sec. 5.2 "vanilla": direct shadow connections  */
  DARTS_METHOD_DARTS_FULL_GATE = 3  /* the DARTS samplers targeting the whole gate; each
                                       control-vertex and surface connection lands in
                                       the bin of its own time (weight 1/N_e), like
                                       method 1, instead of one bin per path.  No
                                       adjoint; not in darts_render_batch. */
} darts_method;

/* sampling.flags */
#define DARTS_FLAG_SENSOR_UNIFORM_ONLY (1u << 0) /* no EDA at the sensor vertex        */
#define DARTS_FLAG_REBUILD_TABLE (1u << 1)       /* rebuild the direction table even on a cache hit */
/* Ablations of the two DARTS samplers (the paper's Fig. 13 study): */
#define DARTS_FLAG_NO_DA_DISTANCE (1u << 2) /* distances: plain truncated-exponential draw
                                               (every RIS weight 1, no DA target)       */
#define DARTS_FLAG_NO_EDA (1u << 3)         /* directions: phase function only (gamma = 0) */
/* RIS variants of Sec. 4.3 (ablations): candidates from independent uniforms
 * instead of the shifted Sobol row; candidates from the equiangular density
 * about the emitter's closest approach to the ray instead of the truncated
 * exponential; selection by weighted reservoir sampling.  Path ids must stay
 * below 2^48 with the first or the last. */
#define DARTS_FLAG_IID_CANDIDATES (1u << 4)
#define DARTS_FLAG_EQUIANGULAR (1u << 5)
#define DARTS_FLAG_RESERVOIR (1u << 6)
/* darts_render adds its estimate into hist_dev (and sumsq_dev) instead of
 * overwriting them: k renders of disjoint path ranges leave the sum of k
 * estimates (divide by k for their average).  Device outputs of darts_render
 * only; the host, batched, static and adjoint calls refuse it. */
#define DARTS_FLAG_ACCUMULATE (1u << 7)
/* EDA directions at surface vertices: the direction that leaves a Lambertian
 * wall or sphere is drawn by the one-sample MIS of Eq. 19 from the EDA table
 * and the cosine lobe about the normal (f = albedo cos / pi) instead of the
 * cosine lobe alone (Sec. 5.1's direction sampler at a surface scattering
 * vertex).  DARTS and full-gate DARTS in general scenes; a direction into the
 * surface ends the path (zero throughput). */
#define DARTS_FLAG_SURFACE_EDA (1u << 8)

typedef struct darts_ctx darts_ctx;

/* Homogeneous medium (Eq. 9): scattering and absorption coefficients,
 * Henyey-Greenstein anisotropy g (|g| < 1), speed of light v = c/eta. */
typedef struct {
  double sigma_s, sigma_a, g, v;
} darts_medium;

/* Pulse emitter (Eq. 1: L_e with start time t_e).  kind DARTS_EMITTER_POINT:
 * isotropic point at pos, radiant intensity energy / (4 pi).
 * kind DARTS_EMITTER_AREA: one-sided Lambertian parallelogram pos + s u + t v
 * (s, t in [0, 1]) emitting toward u x v with radiance energy / (pi area);
 * every path draws one uniform point on it and treats it as a point
 * emitter with intensity (energy / pi) cos (Sec. 7 of the paper).  With
 * several emitters every path picks one with probability proportional to
 * its energy; each has its own pulse start time t0 (Fig. 1). */
#define DARTS_EMITTER_POINT 0
#define DARTS_EMITTER_AREA 1
typedef struct {
  double pos[3];
  double t0;     /* start time of the pulse */
  double energy; /* emitted energy */
  int32_t kind;
  double u[3], v[3];
} darts_emitter;

/* Sensor.  kind DARTS_SENSOR_POINT: isotropic point fluence detector at pos
 * (one element; histogram [n_bins]).  kind DARTS_SENSOR_PINHOLE: pinhole
 * camera at pos looking at look_at with the given up vector and vertical
 * field of view, width x height pixels (elements; histogram
 * [height][width][n_bins]); a pixel records radiance averaged over its
 * area, and the camera leg outside the medium counts toward the path time.
 * paths_per_element paths are traced per element. */
#define DARTS_SENSOR_POINT 0
#define DARTS_SENSOR_PINHOLE 1
typedef struct {
  double pos[3];
  int32_t kind;
  double look_at[3], up[3];
  double fov_deg;
  int32_t width, height;
} darts_sensor;

/* Time gate [t_min, t_max) in n_bins equal bins.  weights (optional, host
 * array of n_bins values >= 0 with a positive sum, NULL for none): the
 * sensor's temporal response W per bin (Eq. 1-4; Sec. 5.2 samples the
 * target interval of a path from it, Fig. 7).  DARTS then draws each path's
 * bin from W by systematic sampling of the cumulative weights (FP64), so a
 * bin receives N_e W_b / sum W paths in expectation and zero-weight bins none;
 * the histogram stays the unweighted per-bin estimate (zero where W_b = 0)
 * and the W-weighted pixel value is sum_b W_b h_b.  The other methods use W
 * only to count rejected samples (darts_stats).  Not accepted by
 * darts_render_static or darts_render_batch. */
typedef struct {
  double t_min, t_max;
  int32_t n_bins;
  const double* weights;
} darts_gate;

/* The medium fills the axis-aligned box [lo, hi].  Faces whose bit
 * (2 * axis + 1 for the high face) is set in `walls` are opaque Lambertian
 * walls of albedo wall_albedo; the others are open (paths leave the scene).
 * spheres: host array [n_spheres][5] = centre, radius, albedo of opaque
 * Lambertian spheres inside the box (at most 64).  A path reaching a
 * surface connects from it directly to its emitter point (accepted only when
 * the total length falls in the path's bin) and continues with a
 * cosine-distributed direction; control vertices stay in the medium, capped
 * at the first surface along the ray (case II of Sec. 5.2). */
typedef struct {
  double lo[3], hi[3];
  int32_t walls;
  double wall_albedo;
  int32_t n_spheres;
  const double* spheres;
} darts_geometry;

typedef struct {
  darts_medium medium;
  darts_geometry geom;
  const darts_emitter* emitters; /* host array of 1..8 emitters */
  int32_t n_emitters;
  darts_sensor sensor;
  darts_gate gate;
} darts_scene;

typedef struct {
  uint64_t seed;              /* Philox key                                           */
  uint64_t paths_per_element; /* path budget N_e of this call (>= 0)                  */
  int32_t max_bounces;        /* K: scattering vertices per path incl. the control vertex, 1..1024 */
  int32_t ris_m;              /* RIS candidates N_RIS (Eq. 15), 1..32; 8 in the paper */
  int32_t table_n_rho;        /* direction table: C/S cells (Sec. 5.1), >= 1          */
  int32_t table_n_s;          /* direction table: S cells (octaves below S_max), >= 1 */
  int32_t table_n_mu;         /* direction table: cos-theta bins, 2..1024; 256 in the paper */
  double mis_alpha;           /* alpha of Eq. 19, > 0; 0.5 in the paper               */
  int32_t method;             /* darts_method                                         */
  uint32_t flags;             /* DARTS_FLAG_*                                         */
  uint32_t stream;            /* Philox stream word (independent sub-streams)         */
} darts_sampling;

/* Optional per-path probe of darts_render: for the paths with local index
 * first, first + stride, ... (count of them, local index = path id minus
 * path_offset) the kernel writes the path's unweighted contribution and its
 * bin.  Lets callers check sampled paths of a full-size launch. */
typedef struct {
  uint64_t first;
  uint64_t stride; /* >= 1 */
  uint32_t count;
  float* contrib_dev;  /* [count] */
  int32_t* bin_dev;    /* [count] */
} darts_probe;

/* Counters of the last darts_render on a context. */
typedef struct {
  uint64_t paths;
  uint64_t vertices;             /* path vertices visited                          */
  uint64_t connections_nonempty; /* control vertices sampled                       */
  uint64_t distance_steps;       /* RIS distance steps (each evaluates ris_m candidates) */
  uint64_t early_exits;          /* Sec. 5.2 residual-bound terminations          */
  uint64_t all_invalid;          /* RIS steps whose candidates were all non-causal */
  uint64_t escapes;              /* rays that left the medium                      */
  uint64_t fp64_ellipse;         /* near-degenerate ellipse solves done in FP64     */
  uint64_t fp64_phi;             /* small-t' DA exponents done in FP64              */
  uint64_t samples;              /* connection samples that produced a path time    */
  uint64_t rejected;             /* of them, times of zero temporal weight: outside
                                    the gate, in a zero-weight bin, or (DARTS)
                                    outside the path's bin                          */
} darts_stats;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `cuda_device`; `cuda_stream` is a
 * cudaStream_t (NULL = the legacy default stream).  Allocates the context's
 * scratch (counters, status word, block partials).  *out is NULL on error. */
darts_status darts_create(darts_ctx** out, int cuda_device, void* cuda_stream);

/* Release the context and its device memory (waits for its stream). */
darts_status darts_destroy(darts_ctx* ctx);

/* Change the stream later calls are ordered on. */
darts_status darts_set_stream(darts_ctx* ctx, void* cuda_stream);

/* Static, never-NULL description of a status code. */
const char* darts_status_string(darts_status s);

/* Copy the last error message of ctx (NUL-terminated, truncated to n). */
darts_status darts_last_error(const darts_ctx* ctx, char* buf, size_t n);

/* Wait for the context's stream and report device-side errors recorded by
 * earlier kernels (DARTS_ERR_NUMERIC, DARTS_ERR_TIMEOUT); clears them. */
darts_status darts_sync(darts_ctx* ctx);

/* ---- the hot path ------------------------------------------------------- */

/* Build the elliptical DA direction table (Sec. 5.1, Eq. 16-18) of the
 * scene's medium and gate on the GPU: rows = table_n_rho * table_n_s
 * conditioning cells (C/S uniform on [0,1); S log-spaced over 8 octaves below
 * S_max = v (t_max - t0)), each a normalised CDF over table_n_mu equal
 * cos-theta bins of [-1, 1].  Output cdf_dev: float [rows][row_stride] with
 * row_stride = table_n_mu + 1 rounded up to a multiple of 4; entry j < n_mu+1
 * is the CDF at the j-th bin edge (0 ... 1).  Caller-owned, overwritten. */
darts_status darts_build_table(darts_ctx* ctx, const darts_scene* scene,
                               const darts_sampling* sampling, float* cdf_dev);

/* Install a direction table built elsewhere -- for example tabulated
 * offline, as the paper does (Sec. 5.1, Fig. 6a) -- as the context's cached
 * table for this scene's medium, gate and table dims.  cdf_dev is device
 * memory, [table_n_rho * table_n_s][darts_table_row_stride(table_n_mu)]
 * floats in the layout darts_build_table writes: per row the CDF over the
 * n_mu cos-theta bins, entries 0 .. n_mu non-decreasing from 0 to 1 (the
 * rest of a row is ignored).  It is copied on the context's stream, so the
 * caller may release it after the next darts_sync.  Later renders of a
 * scene with the same medium, gate and dims use it until a render with
 * DARTS_FLAG_REBUILD_TABLE or another medium replaces it.  A table that is
 * not a CDF biases the samples but never makes a kernel read outside it.
 * Returns DARTS_ERR_INVALID_ARG for an invalid scene or a NULL pointer. */
darts_status darts_load_table(darts_ctx* ctx, const darts_scene* scene,
                              const darts_sampling* sampling, const float* cdf_dev);

/* Row stride (floats) of the table written by darts_build_table. */
int32_t darts_table_row_stride(int32_t table_n_mu);

/* Render sampling->paths_per_element paths per sensor element (N paths in
 * all, ids path_offset .. +N-1; the camera's pixel p owns ids
 * p * paths_per_element onwards) and write the histogram estimate
 * hist_dev[elements][n_bins] (double, overwritten; added to with
 * DARTS_FLAG_ACCUMULATE):
 * DARTS dedicates each path to one bin (Sec. 6.2) and weights it by
 * n_bins / N; the baselines bin each contribution by its time and weight it
 * by 1 / N.  sumsq_dev (optional, [n_bins]) receives the sum over paths of
 * the squared weighted per-path bin contribution (for standard errors).
 * Builds the direction table first when the context's cache misses.
 * probe may be NULL. */
darts_status darts_render(darts_ctx* ctx, const darts_scene* scene,
                          const darts_sampling* sampling, double* hist_dev,
                          double* sumsq_dev, uint64_t path_offset,
                          const darts_probe* probe);

/* darts_render into HOST buffers: the histogram (and optional sums of
 * squares) are copied back and the stream is synchronised before return. */
darts_status darts_render_host(darts_ctx* ctx, const darts_scene* scene,
                               const darts_sampling* sampling, double* hist_host,
                               double* sumsq_host, uint64_t path_offset);

/* darts_render into HOST buffers without waiting: the render is queued on
 * the context's stream and the copy back on a second stream of the
 * context, so the copy of one call overlaps the render of the next.  Two
 * device histograms alternate between calls; a render waits (on the
 * device) for the copy that last used its buffer.  hist_host / sumsq_host
 * (page-locked for an asynchronous copy) must stay valid and unread until
 * darts_sync returns, which waits for both streams and reports device
 * errors.  Same arguments and errors as darts_render_host. */
darts_status darts_render_host_async(darts_ctx* ctx, const darts_scene* scene,
                                     const darts_sampling* sampling, double* hist_host,
                                     double* sumsq_host, uint64_t path_offset);

/* A sequence of n_frames frames of one scene (Eq. 4 per frame, as
 * darts_render computes it), with up to `in_flight` frames running at once.
 * Frame i traces the path ids path_offset + i*N .. path_offset + (i+1)*N - 1
 * (N = paths_per_element x sensor elements) into hist_dev[i], and into
 * sumsq_dev[i] when sumsq_dev is not NULL: exactly what darts_render with
 * that path offset writes (up to FP64 summation order).  Frames go round
 * robin to in_flight (1..4) lanes, each a stream, scratch and direction-table
 * cache of its own that the context creates on first use and keeps.  A
 * frame's tail (a few long paths on a few SMs) then overlaps the next
 * frame's start.  Ordering: the frames start after the work enqueued on the
 * context's stream before the call, and work enqueued on it afterwards
 * waits for all of them.  The outputs must be distinct, non-overlapping
 * device buffers of elements x n_bins doubles (overwritten;
 * DARTS_FLAG_ACCUMULATE is refused).  darts_sync also reports the lanes'
 * device status; darts_get_stats and the kernel timing do not cover the
 * frames of this call.  Errors: as darts_render, and DARTS_ERR_INVALID_ARG
 * for n_frames 0, in_flight outside 1..4 or a NULL output. */
darts_status darts_render_frames(darts_ctx* ctx, const darts_scene* scene,
                                 const darts_sampling* sampling, uint32_t n_frames,
                                 double* const* hist_dev, double* const* sumsq_dev,
                                 uint64_t path_offset, int32_t in_flight);

/* Path-replay adjoint of the DARTS estimator (not in the paper; its Sec. 7
 * lists differentiable transient rendering as future work).  Traces the paths
 * path_offset .. +N-1 of `sampling` (use a seed independent of the forward
 * render) and accumulates, per path, dL/dh[b] * (n_bins / N) * sum over its
 * connections v of c_v * s_v, where s_v is the derivative of log f_v w.r.t.
 * (sigma_s, sigma_a, g) with every sampling density held fixed:
 *   d/dsigma_s = n_v / sigma_s - l_v,  d/dsigma_a = -l_v,
 *   d/dg = sum over the scattering vertices of d log HG / dg,
 * n_v the number of scattering vertices and l_v the length of the path.
 * dLdh_dev: double [n_bins] (input); grad3_dev: double [3] (overwritten);
 * grad3_sq_dev: optional double [3], sum over paths of the squared per-path
 * terms (for standard errors).  method must be DARTS
 * (DARTS_ERR_UNSUPPORTED otherwise). */
darts_status darts_adjoint(darts_ctx* ctx, const darts_scene* scene,
                           const darts_sampling* sampling, const double* dLdh_dev,
                           double* grad3_dev, double* grad3_sq_dev, uint64_t path_offset);

/* Render n independent media in one persistent launch (captured once in a
 * CUDA graph and replayed while the arguments stay the same): the direction
 * tables of all media are built by one kernel launch, then every CTA of the
 * path kernel pops work items of at most 2^16 paths of one medium, staging
 * that medium's table in shared memory when it changes.  hist_dev[i]
 * (double [scenes[i].gate.n_bins], overwritten) receives medium i's
 * histogram, exactly as darts_render(scenes[i], samplings[i], path_offset 0)
 * would (up to FP64 summation order).  All media must use method DARTS,
 * ris_m 8 and one table shape.  flags: DARTS_BATCH_NO_GRAPH launches the
 * kernels directly.  Synchronises the stream once to upload the work list. */
#define DARTS_BATCH_NO_GRAPH (1u << 0)
darts_status darts_render_batch(darts_ctx* ctx, int n, const darts_scene* scenes,
                                const darts_sampling* samplings, double* const* hist_dev,
                                uint32_t flags);

/* Counters of the last render on this context (synchronises the stream). */
darts_status darts_get_stats(darts_ctx* ctx, darts_stats* out);

/* Kernel timing: when enabled, every darts_render records a pair of CUDA
 * events on the context's stream immediately around the path kernel launch
 * (the direction-table kernel and the small scratch resets are outside),
 * and every darts_build_table around its table kernel.
 * darts_last_kernel_ms() synchronises on the stop event and returns the
 * elapsed time of the most recent timed kernel in milliseconds. */
darts_status darts_set_kernel_timing(darts_ctx* ctx, int enable);
darts_status darts_last_kernel_ms(darts_ctx* ctx, float* ms);

/* ---- launch shape ---------------------------------------------------------- */

/* Block size of the persistent path kernel (one CTA per SM): 512, 640, 768
 * or 896 threads, or 0 for the default (a point sensor: the largest whose
 * shared memory fits; a camera: 640 below 2^21 paths per render and 768
 * from there, each as far as its shared memory fits; camera kernels other
 * than DARTS's run 512).  The point-sensor DARTS and baseline kernels are
 * built for 512, 640 and 768, the camera kernels of DARTS for all four
 * sizes; the other variants always run 512, and a size a kernel is not
 * built for runs as 512.  Other values return DARTS_ERR_INVALID_ARG. */
darts_status darts_set_launch(darts_ctx* ctx, int block);

/* Launch shape of the context's kernels.  Zero fields take the defaults.
 *   block        path kernel, as darts_set_launch (0, 512, 640, 768, 896);
 *   chunk        paths a warp claims per update of the global path counter,
 *                1..1024 (default 64; a launch with fewer paths per resident
 *                warp claims fewer);
 *   batch_block  threads per CTA of darts_render_batch (0, 512, 640, 768;
 *                default 768);
 *   batch_items  work items per CTA's share of a batch's estimated cost,
 *                1..64 (default 8): more items balance uneven media better,
 *                fewer restage the direction table less often.
 * Out-of-range fields return DARTS_ERR_INVALID_ARG and change nothing. */
typedef struct {
  int32_t block;
  int32_t chunk;
  int32_t batch_block;
  int32_t batch_items;
} darts_launch;
darts_status darts_set_launch_config(darts_ctx* ctx, const darts_launch* cfg);
darts_status darts_get_launch_config(darts_ctx* ctx, darts_launch* cfg);

/* Autotuner of the path kernel's launch shape for one render: times
 * darts_render of (scene, sampling) for every block size (512, 640, 768; 896
 * for a camera render of DARTS) and
 * chunk (16, 32, 64, 128, 256) that the scene's kernel runs (3 timed renders
 * each after one warm-up; CUDA events on the context's stream; chunks above
 * the launch's paths per resident warp are the same launch and are timed
 * once), keeps the fastest pair on the context and returns the block size in
 * *block_out (may be NULL).  Synchronises the stream.  The renders write the
 * context's scratch histogram, not a caller buffer. */
darts_status darts_autotune(darts_ctx* ctx, const darts_scene* scene,
                            const darts_sampling* sampling, int* block_out);

/* Autotuner of darts_render_batch: times the batch (2 timed launches after
 * one warm-up, without graph capture) for every batch block size (512, 640,
 * 768) and work-item granularity (2, 4, 8, 16, 32 items per CTA share),
 * keeps the fastest on the context and returns the context's launch shape
 * in *out (may be NULL).  The renders write the caller's hist_dev outputs,
 * as darts_render_batch does.  Synchronises the stream. */
darts_status darts_autotune_batch(darts_ctx* ctx, int n, const darts_scene* scenes,
                                  const darts_sampling* samplings, double* const* hist_dev,
                                  darts_launch* out);

/* ---- rendering without allocating ----------------------------------------- */

/* darts_render without a context and without any device allocation, for
 * callers that must not call cudaMalloc (for example a plug-in inside a host
 * application that reserves all device memory in its own pool, or a pipeline
 * that may not allocate after start-up; darts_create allocates, so such
 * callers cannot hold a context).  The paper has no counterpart: this is
 * plumbing around the same kernels.
 *
 * Runs on the calling thread's current device, ordered on cuda_stream
 * (cudaStream_t, NULL = legacy default stream).  The caller passes the
 * outputs, exactly as for darts_render: hist_dev (overwritten) and optional
 * sumsq_dev, each [n_bins] for a point sensor and [height][width][n_bins]
 * for a pinhole camera.  No per-path probe, no statistics, no table cache:
 * the direction table is rebuilt on every call.
 *
 * Scratch: one file-scope device array of 4 MiB, present on every GPU that
 * loads the library until the process exits.  It holds the path counter and
 * statistics (256 B), the direction table (at most 256 KiB:
 * table_n_rho * table_n_s * darts_table_row_stride(table_n_mu) <= 65536
 * floats) and, for a point sensor whose histogram tiles fit in shared
 * memory, the block partials (number of SMs * 2 * n_bins doubles, at most
 * 4 MiB - 256 KiB - 256 B).  A camera, and a point sensor with too many bins
 * for the tiles, add straight into the zeroed outputs and need no partials.
 * Requests beyond these limits return DARTS_ERR_UNSUPPORTED before anything
 * is enqueued.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Every call shares the one array and clears the parts that
 * must start at zero; calls whose work overlaps on the GPU (other streams,
 * other threads, concurrent graphs) race on it and must be serialised by the
 * caller.  Device-side non-finite contributions are zeroed as in
 * darts_render but are not reported (there is no context to sync).
 * Returns DARTS_ERR_INVALID_ARG for invalid scenes or a NULL hist_dev,
 * DARTS_ERR_CUDA when a launch or the set-up fails; either way the CUDA
 * runtime's last error is cleared, so a later call is not affected. */
darts_status darts_render_static(const darts_scene* scene, const darts_sampling* sampling,
                                 double* hist_dev, double* sumsq_dev, uint64_t path_offset,
                                 void* cuda_stream);

/* ---- checking ------------------------------------------------------------ */

/* Trace paths first .. first+count-1 one per thread-slot of the render kernel
 * and record, per path: the unweighted contribution, the bin, the number of
 * vertices visited and four decision bytes per vertex
 * [event | nonempty<<4, RIS index, MIS choice, cos bin] in
 * decisions_dev[count][max_bounces][4] (0xFF = not taken).  Any output may be
 * NULL.  Uses the same kernel code as darts_render. */
darts_status darts_debug_paths(darts_ctx* ctx, const darts_scene* scene,
                               const darts_sampling* sampling, uint64_t first,
                               uint32_t count, float* contrib_dev, int32_t* bin_dev,
                               int32_t* nvert_dev, uint8_t* decisions_dev);

/* Philox4x32-10 blocks of the library's generator: out_dev[i*4..i*4+3] for
 * counter ctr_dev[i*4..i*4+3] and key (seed lo, seed hi); n blocks. */
darts_status darts_debug_philox(darts_ctx* ctx, const uint32_t* ctr_dev, uint64_t seed,
                                uint32_t n, uint32_t* out_dev);

#ifdef __cplusplus
}
#endif
#endif /* DARTS_H */
