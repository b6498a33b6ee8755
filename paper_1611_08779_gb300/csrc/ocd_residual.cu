// Instances of the residual-form OCD kernel: NPP antenna pairs per lane and
// S symbols per item.  NPP = 16 exists only for S = 1 (register budget).
#include "ocd_residual.cuh"

namespace ocd {

KernelFn residual_kernel(int npp, int s) {
  if (s == 2) {
    switch (npp) {
      case 2: return ocd_residual_kernel<2, 2>;
      case 4: return ocd_residual_kernel<4, 2>;
      default: return ocd_residual_kernel<8, 2>;
    }
  }
  switch (npp) {
    case 2: return ocd_residual_kernel<2, 1>;
    case 4: return ocd_residual_kernel<4, 1>;
    case 8: return ocd_residual_kernel<8, 1>;
    default: return ocd_residual_kernel<16, 1>;
  }
}

BatchFn batched_residual_kernel(int npp, int s) {
  if (s == 2) {
    switch (npp) {
      case 2: return ocd_batched_residual_kernel<2, 2>;
      case 4: return ocd_batched_residual_kernel<4, 2>;
      default: return ocd_batched_residual_kernel<8, 2>;
    }
  }
  switch (npp) {
    case 2: return ocd_batched_residual_kernel<2, 1>;
    case 4: return ocd_batched_residual_kernel<4, 1>;
    case 8: return ocd_batched_residual_kernel<8, 1>;
    default: return ocd_batched_residual_kernel<16, 1>;
  }
}

}  // namespace ocd
