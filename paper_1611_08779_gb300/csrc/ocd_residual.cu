// Instances of the residual-form OCD kernel (NPP = antenna pairs per lane).
#include "ocd_residual.cuh"

namespace ocd {

KernelFn residual_kernel(int npp) {
  switch (npp) {
    case 2: return ocd_residual_kernel<2>;
    case 4: return ocd_residual_kernel<4>;
    case 8: return ocd_residual_kernel<8>;
    default: return ocd_residual_kernel<16>;
  }
}

}  // namespace ocd
