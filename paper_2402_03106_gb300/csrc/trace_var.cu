// trace_var.cu -- the DARTS path kernels built for the RIS variants of Sec. 4.3
// (i.i.d. or equiangular candidates, reservoir selection; sampling flags).
// A translation unit of their own, compiled in parallel with trace.cu; the
// production kernels carry none of the variant code.
#include "trace_kernels.cuh"

namespace darts {
namespace {

template <int METHOD>
cudaError_t launch_var_method(const TraceParams& p, int grid, bool debug, bool tile, size_t smem,
                              cudaStream_t s) {
  const bool m8 = p.M == 8;
  if (debug) {
    if (!m8) return tile ? launch_one<METHOD, kMaxM, true, true, 512, false, true>(p, grid, smem, s)
                         : launch_one<METHOD, kMaxM, true, false, 512, false, true>(p, grid, smem, s);
    return tile ? launch_one<METHOD, 8, true, true, 512, false, true>(p, grid, smem, s)
                : launch_one<METHOD, 8, true, false, 512, false, true>(p, grid, smem, s);
  }
  if (!m8) return tile ? launch_one<METHOD, kMaxM, false, true, 512, false, true>(p, grid, smem, s)
                       : launch_one<METHOD, kMaxM, false, false, 512, false, true>(p, grid, smem, s);
  return tile ? launch_one<METHOD, 8, false, true, 512, false, true>(p, grid, smem, s)
              : launch_one<METHOD, 8, false, false, 512, false, true>(p, grid, smem, s);
}

}  // namespace

cudaError_t launch_trace_var(int method, const TraceParams& p, int grid, bool debug, bool tile,
                             size_t smem, cudaStream_t s) {
  if (p.general) return cudaErrorInvalidValue;  // the variants run on medium-only scenes
  switch (method) {
    case kDarts: return launch_var_method<kDarts>(p, grid, debug, tile, smem, s);
    case kDartsFull: return launch_var_method<kDartsFull>(p, grid, debug, tile, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace darts
