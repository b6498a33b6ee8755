// Instances of the bulk-copy (TMA) projected-residual OCD kernel and its
// fault word.
#include "ocd_projected_tma.cuh"

namespace ocd {

KernelFn projected_tma_kernel(int /*umax*/) { return ocd_projected_tma_kernel; }

size_t projected_tma_smem_per_warp(int /*umax*/) { return TmaShape::kWarpBytes; }

cudaError_t projected_tma_fault(unsigned int* bits, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(bits, g_tma_fault, sizeof(unsigned int));
  if (e == cudaSuccess && clear) {
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbol(g_tma_fault, &zero, sizeof(unsigned int));
  }
  return e;
}

}  // namespace ocd
