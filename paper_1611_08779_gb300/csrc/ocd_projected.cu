// Instances of the projected-residual OCD kernel (user bound UMAX = 4 or 8).
#include "ocd_projected.cuh"

namespace ocd {

KernelFn projected_kernel(int umax) {
  return umax <= 4 ? ocd_projected_kernel<4> : ocd_projected_kernel<8>;
}

size_t projected_smem_per_warp(int umax) {
  return (umax <= 4 ? ProjectedShape<4>::kWarpFloats : ProjectedShape<8>::kWarpFloats) *
         sizeof(float);
}

}  // namespace ocd
