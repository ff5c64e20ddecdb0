// table.cu -- elliptical DA direction table on the GPU (Sec. 5.1, Eq. 16-18).
//
// For one conditioning cell (C/S = rho, S) the unnormalised density of the
// direction cosine mu to the major axis x_k -> x_e is
//   F(mu) = int_0^{t_M(mu)} exp(-sigma_t t) Phi(r(t, mu), (S - t)/v) dt,
//   r^2 = C^2 + t^2 - 2 C t mu,  t_M = (S^2 - C^2) / (2 (S - C mu))  (Eq. 18),
// with Phi the transient DA Green's function of Eq. 9 (the paper's MC
// integration replaced by a fixed Gauss-Legendre rule: 4 nodes per mu-bin, two
// 32-node panels in t split at the closest approach t = C mu when it lies
// inside the ellipse).  Each CTA integrates one row, turns the bin integrals
// into a normalised CDF by a block scan and writes it.
#include <cfloat>

#include "darts_device.cuh"
#include "darts_internal.h"

namespace darts {
namespace {

constexpr int kTableThreads = 1024;  // 4 lanes per cos bin: one Gauss node each
constexpr int kScanThreads = 256;    // bins per pass of the CDF scan
constexpr int kMaxMu = 1024;

__device__ __forceinline__ float warp_incl_scan(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float n = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Zero the outputs of the path launch that follows (grid-stride over all
// table blocks), so that a render needs no separate memset launches.
__device__ __forceinline__ void zero_outputs(const TableParams& P, int block, int nblocks) {
  if (P.zero_n) {
    const unsigned long long stride = (unsigned long long)nblocks * kTableThreads;
    for (unsigned long long i = (unsigned long long)block * kTableThreads + threadIdx.x; i < P.zero_n; i += stride) {
      P.zero_a[i] = 0.0;
      if (P.zero_b) P.zero_b[i] = 0.0;
    }
  }
  // scratch word 1 (last-block ticket and device status) persists
  if (block == 0 && (int)threadIdx.x < P.zero_scratch_n && threadIdx.x != 1) P.zero_scratch[threadIdx.x] = 0ull;
}

__device__ __forceinline__ void table_row(const TableParams& P, const int row) {
  __shared__ float logF[kMaxMu];
  __shared__ float wsum[kScanThreads / 32];
  __shared__ float wmax[kScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i_rho = row / P.n_s, i_s = row - i_rho * P.n_s;
  const float rho = (i_rho + 0.5f) / P.n_rho;
  const float S = P.smax * exp2f(-8.0f + 8.0f * (i_s + 0.5f) / P.n_s);
  const float C = rho * S;
  const float SmC = S * (1.0f - rho);  // S - C
  const float h = 2.0f / P.n_mu;

  // ---- bin integrals: lane group g = tid / 4 takes bins g, g + 256, ...;
  // lane a = tid % 4 integrates Gauss node a of the bin, the group merges
  // its four partial sums (online log-sum-exp) with shuffles
  const int a = tid & 3;
  const float xa1 = P.mu_x[a] + 1.0f;
  const float wa = 0.5f * h * P.mu_w[a];
  for (int i0 = tid >> 2; i0 < kMaxMu; i0 += kTableThreads / 4) {
    if (i0 - (tid >> 2) >= P.n_mu) break;  // uniform across the block
    const int i = i0;
    float m = -FLT_MAX, s = 0.0f;
    if (i < P.n_mu) {
      const float onem = h * ((float)(P.n_mu - i) - 0.5f * xa1);  // 1 - mu
      const float mu = 1.0f - onem;
      const float tM = SmC * (S + C) / (2.0f * fmaf(C, onem, SmC));
      const float cmu = C * mu;
      const float split = (cmu > 0.0f && cmu < tM) ? cmu : 0.5f * tM;
      // the integrand is exp(lg) tp^(-3/2) with lg = phi_k0 - r^2 / (4 v D tp)
      // - sigma_a v tp - sigma_t t: one reciprocal square root gives both
      // tp^(-3/2) and 1 / tp, and the running log-sum-exp is rescaled once per
      // group of kGroup nodes (two MUFU operations per node)
      constexpr int kGroup = 8;
      const float inv_v = 1.0f / P.v;
#pragma unroll 1
      for (int panel = 0; panel < 2; ++panel) {
        const float lo = panel == 0 ? 0.0f : split;
        const float hw = 0.5f * ((panel == 0 ? split : tM) - lo);
#pragma unroll 1
        for (int b0 = 0; b0 < kMaxTabTNodes; b0 += kGroup) {
          float lg[kGroup], rs[kGroup];
          float gm = -FLT_MAX;
#pragma unroll
          for (int q = 0; q < kGroup; ++q) {
            const float t = fmaf(hw, P.t_x[b0 + q] + 1.0f, lo);
            const float tc = t - C;
            const float r2 = fmaf(tc, tc, 2.0f * C * t * onem);
            const float tp = (S - t) * inv_v;  // t' > 0 inside the ellipse
            rs[q] = rsqrtf(tp);
            lg[q] = P.phi_k0 - r2 * P.phi_invk * (rs[q] * rs[q]) - P.sa_v * tp - P.sigma_t * t;
            gm = fmaxf(gm, lg[q]);
          }
          const float mn = fmaxf(m, gm);
          float acc = 0.0f;
#pragma unroll
          for (int q = 0; q < kGroup; ++q)
            acc = fmaf(P.t_w[b0 + q] * __expf(lg[q] - mn), rs[q] * rs[q] * rs[q], acc);
          s = fmaf(s, __expf(m - mn), wa * hw * acc);
          m = mn;
        }
      }
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      const float mo = __shfl_xor_sync(0xFFFFFFFFu, m, o);
      const float so = __shfl_xor_sync(0xFFFFFFFFu, s, o);
      const float mn = fmaxf(m, mo);
      s = (s > 0.0f ? s * __expf(m - mn) : 0.0f) + (so > 0.0f ? so * __expf(mo - mn) : 0.0f);
      m = mn;
    }
    if (a == 0 && i < P.n_mu) logF[i] = m + __logf(s);
  }
  __syncthreads();
  if (tid >= kScanThreads) return;

  // ---- row maximum of log F, then per-thread runs of consecutive bins and
  // a block-wide exclusive scan (the first kScanThreads threads)
  const int per = (P.n_mu + kScanThreads - 1) / kScanThreads;
  float local_max = -FLT_MAX;
  for (int q = 0; q < per; ++q) {
    const int i = tid * per + q;
    if (i < P.n_mu) local_max = fmaxf(local_max, logF[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xFFFFFFFFu, local_max, o));
  if (lane == 0) wmax[warp] = local_max;
  asm volatile("bar.sync 1, %0;" ::"r"(kScanThreads));
  float M = wmax[0];
  for (int w = 1; w < kScanThreads / 32; ++w) M = fmaxf(M, wmax[w]);

  float run[4];
  float tsum = 0.0f;
  for (int q = 0; q < per; ++q) {
    const int i = tid * per + q;
    const float f = (i < P.n_mu) ? __expf(logF[i] - M) : 0.0f;
    tsum += f;
    run[q] = tsum;
  }
  const float incl = warp_incl_scan(tsum, lane);
  if (lane == 31) wsum[warp] = incl;
  asm volatile("bar.sync 1, %0;" ::"r"(kScanThreads));
  float woff = 0.0f, total = 0.0f;
  for (int w = 0; w < kScanThreads / 32; ++w) {
    if (w < warp) woff += wsum[w];
    total += wsum[w];
  }
  const float excl = woff + incl - tsum;
  float* out = P.cdf + (size_t)row * P.row_stride;
  const bool good = total > 0.0f && isfinite(total);
  const float inv = good ? 1.0f / total : 0.0f;
  for (int q = 0; q < per; ++q) {
    const int i = tid * per + q;
    if (i >= P.n_mu) break;
    const float v = good ? (excl + run[q]) * inv : (float)(i + 1) / P.n_mu;
    out[i + 1] = (i + 1 == P.n_mu) ? 1.0f : fminf(v, 1.0f);
  }
  if (tid == 0) out[0] = 0.0f;
  for (int j = P.n_mu + 1 + tid; j < P.row_stride; j += kScanThreads) out[j] = 1.0f;
}

__global__ void __launch_bounds__(kTableThreads) eda_table_kernel(const TableParams P) {
  zero_outputs(P, blockIdx.x, gridDim.x);
  table_row(P, blockIdx.x);
}

// All media of a batch in one launch: blockIdx.y selects the medium.
__global__ void __launch_bounds__(kTableThreads) eda_table_batch_kernel(const TableParams* Ps) {
  const TableParams& P = Ps[blockIdx.y];
  if ((int)blockIdx.x < P.n_rho * P.n_s) table_row(P, blockIdx.x);
}

}  // namespace

cudaError_t launch_table_batch(const TableParams* ps_dev, int n_media, int rows, cudaStream_t s) {
  if (n_media <= 0) return cudaSuccess;
  eda_table_batch_kernel<<<dim3(rows, n_media), kTableThreads, 0, s>>>(ps_dev);
  return cudaGetLastError();
}

cudaError_t launch_table(const TableParams& p, cudaStream_t s) {
  if (p.n_mu > kMaxMu || p.n_mu > 4 * kScanThreads) return cudaErrorInvalidValue;
  eda_table_kernel<<<p.n_rho * p.n_s, kTableThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace darts
