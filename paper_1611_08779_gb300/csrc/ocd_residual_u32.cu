// Instances of the residual-form OCD kernel for up to 32 users.  The launch
// plan caps the antenna pairs per lane at 8 for this bound (the 64 z registers
// leave no room for 16), so no NPP = 16 instance exists.
#include "ocd_residual.cuh"

namespace ocd {

KernelFn residual_kernel_u32(int npp) {
  switch (npp) {
    case 2: return ocd_residual_kernel<32, 2>;
    case 4: return ocd_residual_kernel<32, 4>;
    default: return ocd_residual_kernel<32, 8>;
  }
}

}  // namespace ocd
