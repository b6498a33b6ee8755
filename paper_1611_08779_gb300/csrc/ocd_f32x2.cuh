// Packed FP32 pairs for the sweeps of the projected kernels: fma.rn.f32x2
// performs two independent IEEE fmas (one per 32-bit half), so a packed
// update gives the same bits as the scalar fmaf sequence it replaces.
#pragma once

namespace ocd {

__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// d <- a * b + d, per half
__device__ __forceinline__ void f2_fma(unsigned long long& d, unsigned long long a,
                                       unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

}  // namespace ocd
