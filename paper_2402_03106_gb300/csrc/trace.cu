// trace.cu -- launchers of the path kernels (device code in trace_kernels.cuh):
// the DARTS, baseline and general variants, the batched and adjoint launches.
#include "trace_kernels.cuh"

namespace darts {
namespace {

template <int METHOD>
cudaError_t launch_method(const TraceParams& p, int grid, int block, bool debug, bool tile,
                          size_t smem, cudaStream_t s) {
  if (p.general) {  // general scenes: 512 threads, M = 8
    if (kIsDartsM<METHOD> && p.M != 8) return cudaErrorInvalidValue;  // shared memory sized for M = 8
    if (debug) return tile ? launch_one<METHOD, 8, true, true, 512, true>(p, grid, smem, s)
                           : launch_one<METHOD, 8, true, false, 512, true>(p, grid, smem, s);
    if (tile) return launch_one<METHOD, 8, false, true, 512, true>(p, grid, smem, s);
    if constexpr (METHOD == kDarts) {  // camera frames: 640 and 768 threads too, and the lean kernels
      if (p.lean) {
        switch (block) {
          case 640: return launch_one<METHOD, 8, false, false, 640, true, false, true>(p, grid, smem, s);
          case 768: return launch_one<METHOD, 8, false, false, 768, true, false, true>(p, grid, smem, s);
          case 896: return launch_one<METHOD, 8, false, false, 896, true, false, true>(p, grid, smem, s);
          default: return launch_one<METHOD, 8, false, false, 512, true, false, true>(p, grid, smem, s);
        }
      }
      switch (block) {
        case 640: return launch_one<METHOD, 8, false, false, 640, true>(p, grid, smem, s);
        case 768: return launch_one<METHOD, 8, false, false, 768, true>(p, grid, smem, s);
        case 896: return launch_one<METHOD, 8, false, false, 896, true>(p, grid, smem, s);
        default: break;
      }
    }
    return launch_one<METHOD, 8, false, false, 512, true>(p, grid, smem, s);
  }
  const bool m8 = !kIsDartsM<METHOD> || p.M == 8;
  if constexpr (kIsDartsM<METHOD>) {
    if (p.ris_mode) return launch_trace_var(METHOD, p, grid, debug, tile, smem, s);
  }
  if (debug) {
    if (!m8) return tile ? launch_one<METHOD, kMaxM, true, true, 512>(p, grid, smem, s)
                         : launch_one<METHOD, kMaxM, true, false, 512>(p, grid, smem, s);
    return tile ? launch_one<METHOD, 8, true, true, 512>(p, grid, smem, s)
                : launch_one<METHOD, 8, true, false, 512>(p, grid, smem, s);
  }
  if (!m8) return tile ? launch_one<METHOD, kMaxM, false, true, 512>(p, grid, smem, s)
                       : launch_one<METHOD, kMaxM, false, false, 512>(p, grid, smem, s);
  if (!tile) return launch_one<METHOD, 8, false, false, 512>(p, grid, smem, s);
  if constexpr (METHOD == kDartsFull) {  // built for 512 threads only
    return launch_one<METHOD, 8, false, true, 512>(p, grid, smem, s);
  } else {
    switch (block) {
      case 640: return launch_one<METHOD, 8, false, true, 640>(p, grid, smem, s);
      case 768: return launch_one<METHOD, 8, false, true, 768>(p, grid, smem, s);
      default: return launch_one<METHOD, 8, false, true, 512>(p, grid, smem, s);
    }
  }
}

}  // namespace

size_t batch_smem_bytes(const BatchParams& bp, int block) {
  return table_smem_bytes(bp.rows, bp.row_stride) +
         (size_t)(block / 32) * 32 * (sizeof(RisTask) + sizeof(RisResult)) +
         (size_t)(block / 32) * 2 * bp.max_bins * sizeof(float);
}

cudaError_t launch_batch(const BatchParams& bp, int grid, int block, size_t smem, cudaStream_t s) {
  zero_hists_kernel<<<bp.n_media, 128, 0, s>>>(bp.params);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (block) {
    case 768: {
      auto k = trace_batch_kernel<768>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k<<<grid, 768, smem, s>>>(bp);
      break;
    }
    case 640: {
      auto k = trace_batch_kernel<640>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k<<<grid, 640, smem, s>>>(bp);
      break;
    }
    default: {
      auto k = trace_batch_kernel<512>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k<<<grid, 512, smem, s>>>(bp);
    }
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

size_t adjoint_smem_bytes(const TraceParams& p) {
  size_t b = table_smem_bytes(p.rows, p.row_stride) + (p.general ? cull_bytes(p.cull_slabs) : 0);
  if (p.M == 8) b += (size_t)(512 / 32) * 32 * (sizeof(RisTask) + sizeof(RisResult));
  return b;
}

cudaError_t launch_adjoint(const TraceParams& p0, int grid, size_t smem, cudaStream_t s) {
  TraceParams p = p0;
  p.bin_base = (p0.path_offset + p0.o_e) % (unsigned long long)p0.n_bins;
  p.chunk = chunk_for(p.N, grid, 512, p.chunk_cap);
  if (p.general) {
    if (p.M != 8) return cudaErrorInvalidValue;  // shared memory sized for M = 8
    auto kern = trace_kernel<kDarts, 8, false, false, 512, true, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 512, smem, s>>>(p);
  } else if (p.M == 8) {
    auto kern = trace_kernel<kDarts, 8, false, false, 512, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 512, smem, s>>>(p);
  } else {
    auto kern = trace_kernel<kDarts, kMaxM, false, false, 512, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 512, smem, s>>>(p);
  }
  return cudaGetLastError();
}

size_t trace_smem_bytes(int method, const TraceParams& p, int block, bool tile) {
  const bool darts = method == kDarts || method == kDartsFull;
  size_t b = darts ? table_smem_bytes(p.rows, p.row_stride) : 0;
  if (p.general) b += cull_bytes(p.cull_slabs);  // sphere-culling masks and the spheres, first in shared memory
  const size_t task = p.ris_mode ? sizeof(RisTaskVar) : sizeof(RisTask);
  if (darts && p.M == 8) b += (size_t)(block / 32) * 32 * (task + sizeof(RisResult));
  if (tile) b += (size_t)(block / 32) * (p.sumsq ? 3 : 2) * p.n_bins * sizeof(float);
  return b;
}

int trace_max_m() { return kMaxM; }

int trace_block_for(int block, bool debug, bool tile, int method, int M, bool general) {
  const bool wide = block == 640 || block == 768;
  if (debug || method == kDartsFull || (method == kDarts && M != 8)) return 512;
  // camera frames of DARTS: 896 threads too (72 registers a thread)
  if (general) return (!tile && method == kDarts && (wide || block == 896)) ? block : 512;
  return (tile && wide) ? block : 512;
}

cudaError_t launch_trace(int method, const TraceParams& p0, int grid, int block, bool debug,
                         bool tile, size_t smem, cudaStream_t s) {
  TraceParams p = p0;
  p.bin_base = (p0.path_offset + p0.o_e) % (unsigned long long)p0.n_bins;
  switch (method) {
    case kDarts: return launch_method<kDarts>(p, grid, block, debug, tile, smem, s);
    case kPlain: return launch_method<kPlain>(p, grid, block, debug, tile, smem, s);
    case kVanilla: return launch_method<kVanilla>(p, grid, block, debug, tile, smem, s);
    case kDartsFull: return launch_method<kDartsFull>(p, grid, block, debug, tile, smem, s);
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
