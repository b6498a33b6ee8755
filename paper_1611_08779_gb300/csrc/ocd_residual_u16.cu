// Instances of the residual-form OCD kernel for up to 16 users.
#include "ocd_residual.cuh"

namespace ocd {

KernelFn residual_kernel_u16(int npp) {
  switch (npp) {
    case 2: return ocd_residual_kernel<16, 2>;
    case 4: return ocd_residual_kernel<16, 4>;
    case 8: return ocd_residual_kernel<16, 8>;
    default: return ocd_residual_kernel<16, 16>;
  }
}

}  // namespace ocd
