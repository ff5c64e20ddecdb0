// darts_internal.h -- parameter blocks and launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace darts {

constexpr int kMaxTabMuNodes = 4;   // Gauss-Legendre nodes per cos-theta bin
constexpr int kMaxTabTNodes = 32;   // Gauss-Legendre nodes per t-panel (two panels)
constexpr int kStatCount = 12;      // device event counters (see the ST_ slots of trace.cu)
constexpr int kPathChunk = 64;      // paths a warp claims from the global counter
constexpr int kMaxEmitters = 8;
constexpr int kMaxSpheres = 64;
// Sphere culling of the general kernels: per axis, cull_slabs slabs of the
// medium box (16, or 32 where shared memory allows: camera kernels) and, for
// every slab range [i, j], the mask of the spheres whose (slightly enlarged)
// extent meets it; built in shared memory by each CTA, followed by the
// spheres themselves.
constexpr int kMaxCullSlabs = 32;
__host__ __device__ inline size_t cull_bytes(int slabs) {
  return 3 * (size_t)slabs * slabs * sizeof(unsigned long long) + kMaxSpheres * 4 * sizeof(float);
}

// Guide of each direction-table row in shared memory: for k = 0..kGuide-1
// the largest bin lo with cdf[lo] <= k / kGuide, and n_mu - 1 at k = kGuide
// (uint16 entries, after the rows).  An inverse-CDF search for v then starts
// from the bins [guide[floor(v kGuide)], guide[floor(v kGuide) + 1]].
constexpr int kGuide = 32;
__host__ __device__ inline size_t guide_bytes(int rows) {
  return ((size_t)rows * (kGuide + 1) * sizeof(uint16_t) + 15) / 16 * 16;
}
// Shared memory of a staged direction table: its rows, then their guides.
__host__ __device__ inline size_t table_smem_bytes(int rows, int row_stride) {
  return (size_t)rows * row_stride * sizeof(float) + guide_bytes(rows);
}

// One pulse emitter: an isotropic point (kind 0) or a one-sided Lambertian
// parallelogram pos + s u + t v emitting toward n = u x v / |u x v| (kind 1).
struct EmitterParams {
  float pos[3], u[3], v[3], n[3];
  float ie;          // radiant intensity scale: E / (4 pi) (point), E / pi (area)
  float cdf;         // cumulative energy fraction up to and including this emitter
  float wsel;        // total energy / this emitter's energy (1 / selection probability)
  float s_lo, s_hi;  // v (t_min - t0), v (t_max - t0)
  int kind;
};

// Elliptical DA table build (Sec. 5.1, Eq. 16-18).
struct TableParams {
  float sigma_t, sigma_a, v;
  float phi_k0;    // log v - 1.5 log(4 pi v D)
  float phi_invk;  // 1 / (4 v D)
  float sa_v;      // sigma_a v
  float smax;      // v (t_max - t0)
  int n_rho, n_s, n_mu, row_stride;
  float mu_x[kMaxTabMuNodes], mu_w[kMaxTabMuNodes];
  float t_x[kMaxTabTNodes], t_w[kMaxTabTNodes];
  float* cdf;      // [rows][row_stride]
  // outputs of the path launch that follows, zeroed by this launch (null: none)
  double* zero_a;
  double* zero_b;
  unsigned long long zero_n;       // doubles in each of zero_a, zero_b
  unsigned long long* zero_scratch; // the context's scratch words; word 1 is kept
  int zero_scratch_n;
};

// Path kernels.  Everything the step functions read, in FP32 unless noted.
struct TraceParams {
  // medium
  float sigma_s, sigma_t, inv_st, albedo, sa_v, v, inv_v;
  float phi_k0, phi_invk;          // Eq. 9 in log form, see TableParams
  float hg_a, hg_b, hg_c, g;       // HG constants (hg_eval) and g
  float hg_dlog_a;                 // -2 g / (1 - g^2)
  float inv_sigma_s;               // 1 / sigma_s (0 when sigma_s = 0)
  double phi_k0_d, phi_invk_d, sa_v_d, inv_v_d;  // the same, FP64 (small-t' branch)
  // geometry
  float lo[3], hi[3], xe[3], xs[3];
  float Ie;                        // energy / (4 pi)
  // gate, in length units relative to the pulse start
  float S_gate_lo;                 // v (t_min - t0)
  float S_bin;                     // v (t_max - t_min) / n_bins
  float inv_S_bin;
  float S_gate_hi;                 // v (t_max - t0)
  float tiny_s;                    // 2^-6 v (t_max - t_min): small-t' threshold
  int n_bins;
  // general scenes: several / area emitters, surfaces, a pinhole camera
  int general;                     // run the general variant of the path kernel
  int lean;                        // general scene with point emitters only, a camera inside the
                                   // medium, no temporal response, no EDA at surfaces: the lean
                                   // camera kernel of DARTS
  int n_emitters;
  EmitterParams em[kMaxEmitters];
  int n_spheres;
  float4 sph[kMaxSpheres];         // centre, radius
  float sph_albedo[kMaxSpheres];
  float cull_off[3], cull_inv_w[3]; // slab grid of the box: slab = floor(x inv_w + off), off = -lo inv_w
  float cull_eps;                  // enlargement of a sphere's extent in the masks
  int cull_slabs;                  // slabs per axis of the culling grid
  int walls;                       // box faces with walls: bit 2 * axis + (1: hi face)
  float wall_albedo;
  int camera;                      // 0: point sensor at xs; 1: pinhole camera
  int cam_inside;                  // camera inside the medium box
  float cam_pos[3], cam_f[3], cam_r[3], cam_u[3];
  float cam_th, cam_aspect;
  int width, height;
  unsigned long long spp;          // paths per sensor element
  // direction table
  int n_rho, n_s, n_mu, row_stride, rows;
  float inv_smax, n_s_over_8, mu_scale, inv_mu_scale;  // 1/S_max, n_s / 8, n_mu / 2, 2 / n_mu
  float mis_alpha;
  int uniform_sensor;
  int no_eda;                      // ablation: phase-function directions only
  int surface_eda;                 // EDA/cosine-lobe MIS directions at surface vertices
  int no_da;                       // ablation: truncated-exponential distances (RIS weights 1)
  int ris_mode;                    // bit 0: i.i.d. candidates, 1: equiangular candidates, 2: reservoir
  int accumulate;                  // add the estimate into hist / sumsq instead of overwriting
  const float* table;              // [rows][row_stride]
  // sampling
  int K, M;
  uint32_t key0, key1, stream;
  uint32_t o_e;                    // bin offset of the sensor element
  unsigned long long bin_base;     // (path_offset + o_e) mod n_bins: bin of local path 0
  unsigned long long N;            // paths in this launch (local index 0..N-1)
  unsigned long long path_offset;  // global id = path_offset + local index
  unsigned int chunk;              // paths a warp claims per counter update (set at launch)
  unsigned int chunk_cap;          // largest such claim (0: kPathChunk), the tuned launch shape
  float wb;                        // weight per path contribution (DARTS n_bins/N_e, else 1/N_e)
  // temporal response W (null without): cumulative weights C[0..n_bins]
  // (FP64), per-bin DARTS path weight sum W / (N_e W_b) (0 where W_b = 0),
  // and the point sensor's systematic-sampling offset and phase
  const double* wcdf;
  const float* wbin;
  unsigned long long w_oe;
  double w_phi;
  // outputs and scratch
  double* hist;                    // [elements][n_bins]; zeroed before a launch without tiles
  double* sumsq;                   // [elements][n_bins] or null
  double* partials;                // [grid][n_bins] x (sum, sum of squares): 2 doubles per bin
  unsigned long long* counter;     // path counter
  unsigned int* ticket;            // last-block ticket
  unsigned int* status;            // device status word (bit 0: non-finite)
  unsigned long long* stats;       // [kStatCount]
  // path-replay adjoint
  const double* dLdh;              // [n_bins]
  double* grad3;                   // [3]
  double* grad3_sq;                // [3] or null
  // per-path probe (sampled paths of a full launch)
  unsigned long long probe_first, probe_stride;
  unsigned int probe_count;
  float* probe_c;
  int* probe_b;
  // debug (decision traces), local index < N
  float* dbg_c;
  int* dbg_b;
  int* dbg_n;
  uint8_t* dbg_dec;                // [N][K][4]
};

// Batched rendering: one work item = a range of one medium's paths.
struct BatchItem {
  unsigned int medium;
  unsigned int pad;
  unsigned long long first, count;
};
struct BatchParams {
  const TraceParams* params;   // [n_media], device
  const BatchItem* items;      // [n_items], device, grouped by medium
  int n_items, n_media;
  unsigned int* item_counter;  // zeroed before the launch
  int max_bins;                // tile sizing
  int rows, row_stride;        // direction-table shape (common to the batch)
  unsigned long long* stats;   // [kStatCount]
};

// Launchers (stream-ordered; return the launch's cudaError_t).
cudaError_t launch_table(const TableParams& p, cudaStream_t s);
cudaError_t launch_trace(int method, const TraceParams& p, int grid, int block, bool debug,
                         bool tile, size_t smem, cudaStream_t s);
// The DARTS path kernels built for the RIS variants (ris_mode != 0; point
// sensor, medium only, 512 threads); called by launch_trace.
cudaError_t launch_trace_var(int method, const TraceParams& p, int grid, bool debug, bool tile,
                             size_t smem, cudaStream_t s);
cudaError_t launch_table_batch(const TableParams* ps_dev, int n_media, int rows, cudaStream_t s);
cudaError_t launch_batch(const BatchParams& bp, int grid, int block, size_t smem, cudaStream_t s);
size_t batch_smem_bytes(const BatchParams& bp, int block);
cudaError_t launch_adjoint(const TraceParams& p, int grid, size_t smem, cudaStream_t s);
size_t adjoint_smem_bytes(const TraceParams& p);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t n,
                          uint32_t* out, cudaStream_t s);
size_t trace_smem_bytes(int method, const TraceParams& p, int block, bool tile);
// Block size actually launched for a request (non-production variants use 512).
int trace_block_for(int block, bool debug, bool tile, int method, int M, bool general);
int trace_max_m();

}  // namespace darts
