// Instances of the residual-form OCD kernel for up to 8 users.
#include "ocd_residual.cuh"

namespace ocd {

KernelFn residual_kernel_u8(int npp) {
  switch (npp) {
    case 2: return ocd_residual_kernel<8, 2>;
    case 4: return ocd_residual_kernel<8, 4>;
    case 8: return ocd_residual_kernel<8, 8>;
    default: return ocd_residual_kernel<8, 16>;
  }
}

}  // namespace ocd
