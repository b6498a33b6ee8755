// Instances of the residual-form OCD kernel for up to 4 users.
#include "ocd_residual.cuh"

namespace ocd {

KernelFn residual_kernel_u4(int npp) {
  switch (npp) {
    case 2: return ocd_residual_kernel<4, 2>;
    case 4: return ocd_residual_kernel<4, 4>;
    case 8: return ocd_residual_kernel<4, 8>;
    default: return ocd_residual_kernel<4, 16>;
  }
}

}  // namespace ocd
