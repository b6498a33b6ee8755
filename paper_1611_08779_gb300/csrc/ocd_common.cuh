// Shared device-side pieces of the OCD detector: launch parameters, the
// projection of Eq. 14 and the per-dimension max-log LLR of Eq. 9.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

namespace ocd {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kUserSlots = 32;  // per-subcarrier slots of the preprocessing tables

// Storage of H and Y: interleaved complex as float32 pairs (8 bytes) or as
// bfloat16 / float16 pairs (4 bytes); outputs are always float32.
enum Storage { kStoreC64 = 0, kStoreBF16 = 1, kStoreF16 = 2 };

struct DetectParams {
  const float2* __restrict__ H;  // [Nsc][B][U]  (16-bit storage: 4-byte elements)
  const float2* __restrict__ Y;  // [Nsc][T][B]
  float2* __restrict__ xhat;     // [Nsc][T][U] or null
  float* __restrict__ llr;       // [Nsc][T][U][Q] or null
  long long items;               // Nsc * ceil(T / S) (one item = S symbols of one subcarrier)
  int Nsc, B, U, T, K;
  int box;        // 1: BOX mode (clip), 0: MMSE mode
  int bpsk;       // 1: BPSK alphabet (real axis only)
  int Q;          // bits per symbol
  int nb;         // bits per real dimension
  int M;          // levels per real dimension
  float alpha;    // regularizer of Algorithm 1: N0/Es (MMSE) or 0 (BOX)
  float box_a;    // clip radius sqrt(Es) * max Re{O}
  float rho_scale;  // Es / N0: rho~ = ||h||^2 * rho_scale
  float sqrt_es;
  float lvl_step;   // 1/sigma: level i sits at (2i + 1 - M) * lvl_step
  // launch geometry (chosen on the host)
  int L, logL;      // lanes per team (power of two) and log2
  int chunk;        // consecutive items per CTA pass (= teams per CTA)
  int scmax;        // largest number of subcarriers a chunk can touch
  int vec_y;        // Y rows may be read with 16-byte loads
  unsigned long long wait_ns;  // limit of any wait for a copy engine (ns)
  int storage;      // Storage of H and Y
  int ymap3d;       // bulk-copy kernel: Y's tensor map is the 3-D view (one copy per 32 antennas)
};

// Converting loads of complex element `idx` of a [.. ] array in `storage`.
__device__ __forceinline__ float2 unpack_c16(uint32_t v, int storage) {
  if (storage == kStoreBF16)  // real part in the low half (lower address)
    return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
  __half2 h;
  memcpy(&h, &v, sizeof(h));
  return __half22float2(h);
}
__device__ __forceinline__ float2 load_c(const float2* base, long long idx, int storage) {
  if (storage == kStoreC64) return __ldg(base + idx);
  return unpack_c16(__ldg(reinterpret_cast<const uint32_t*>(base) + idx), storage);
}
// Two consecutive complex elements idx, idx+1 (idx even, 8/16-byte aligned).
__device__ __forceinline__ float4 load_c2(const float2* base, long long idx, int storage) {
  if (storage == kStoreC64) return __ldg(reinterpret_cast<const float4*>(base + idx));
  const uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint32_t*>(base) + idx));
  const float2 a = unpack_c16(v.x, storage), b = unpack_c16(v.y, storage);
  return make_float4(a.x, a.y, b.x, b.y);
}

using KernelFn = void (*)(DetectParams);

// Residual-form kernels by antenna pairs per lane (2, 4, 8, 16) and symbols
// per item (1, 2).
KernelFn residual_kernel(int npp, int s);
// Projected-residual kernels by user bound (4 or 8) and their per-warp
// shared memory in bytes.
KernelFn projected_kernel(int umax);
size_t projected_smem_per_warp(int umax);
constexpr int kProjectedMaxUsers = 8;
// Bulk-copy (TMA) projected kernel: needs even B and 16-byte aligned H, Y
// (128 threads per CTA).  launch_projected_tma encodes the tensor map of Y
// and launches; cudaErrorNotSupported means the driver offers no tensor-map
// encoder.
constexpr int kTmaMaxUsers = 16;
const void* projected_tma_kernel_ptr(int U);
size_t projected_tma_smem_per_cta(int U);
int projected_tma_threads();
cudaError_t launch_projected_tma(const DetectParams& P, unsigned grid, cudaStream_t stream);
// Reads (and optionally clears) the fault word of the bulk-copy kernels;
// synchronous with respect to the device.
cudaError_t projected_tma_fault(unsigned int* bits, bool clear);
// 16-bit-storage projected kernels (U <= 16): need B % 4 == 0 and 16-byte
// aligned H, Y.
constexpr int kH16MaxUsers = 16;
const void* projected_h16_kernel_ptr(int storage, int U);
size_t projected_h16_smem_per_cta(int U);
cudaError_t launch_projected_h16(const DetectParams& P, unsigned grid, cudaStream_t stream);
cudaError_t projected_h16_fault(unsigned int* bits, bool clear);
// One-symbol projected kernels (T = 1, U <= 8, float32 storage, even B,
// 16-byte aligned H and Y): one lane per subcarrier, one warp per group of
// 32 consecutive subcarriers (128 threads per CTA).
constexpr int kLaneMaxUsers = 8;
const void* projected_lane_kernel_ptr(int U);
size_t projected_lane_smem_per_cta(int U);
int projected_lane_threads();
long long projected_lane_groups(long long Nsc);
cudaError_t launch_projected_lane(const DetectParams& P, unsigned grid, cudaStream_t stream);
// Launches one warp that waits, with the same bounded wait the bulk-copy
// kernels use, on an mbarrier phase nothing completes; the wait expires
// after wait_ns and sets the fault word.  Exercises the timeout path.
cudaError_t projected_tma_wait_selftest(unsigned long long wait_ns, cudaStream_t stream);

// Programmatic dependent launch.  A kernel launched by launch_serialized may
// be scheduled while the kernel ahead of it in the stream drains: pdl_wait()
// returns once that kernel has completed and its writes are visible (a
// no-op after a plain launch), so a kernel calls it before its first access
// to global memory that another kernel may write.  pdl_trigger(), issued
// after a CTA's last global write, lets the launch of the next kernel begin
// once every CTA has issued it or exited, so a grid waiting in pdl_wait
// never holds slots that this grid still needs.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// cudaLaunchKernel with programmatic stream serialization (kernels that call
// pdl_wait as above).
inline cudaError_t launch_serialized(const void* fn, unsigned grid, unsigned block, void** args,
                                     size_t smem, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// Projection onto C_O (Eq. 14): for square QAM clip real and imaginary parts
// independently to [-a, a]; for BPSK clip the real part and zero the
// imaginary part.  MMSE mode has C = C (identity).
__device__ __forceinline__ void project(float& wr, float& wi, const DetectParams& P) {
  if (P.box) {
    wr = fminf(fmaxf(wr, -P.box_a), P.box_a);
    wi = P.bpsk ? 0.0f : fminf(fmaxf(wi, -P.box_a), P.box_a);
  }
}

// Max-log LLRs (Eq. 9) of the bits carried by one real dimension with NB
// bits (M = 2^NB levels), in closed form.  For a separable Gray alphabet the
// minima over O_b^0 and O_b^1 differ only in this dimension, so the other
// dimension's contribution cancels exactly.  u = x / step is the coordinate
// in level units: level i sits at u = 2i + 1 - M and carries the Gray word
// i ^ (i >> 1), first bit most significant.
//
// First bit (1 on the positive levels): between consecutive even integers
// the nearest level of either label is fixed, and
//     d0 - d1 = sign(u) * max_{j = 1 .. M/2} 4 j (|u| - (j - 1))
// in units of step^2 (the j-th line is the difference for nearest levels
// -1 and 2j - 1; consecutive lines meet at the thresholds |u| = 2 (j - 1)),
// which is the exhaustive difference of minima, not an approximation.
// Folding u' = M/2 - |u| maps the positive half of the M-level Gray PAM onto
// an M/2-level one centred at zero whose first bit (1 where u' > 0, the
// inner levels) is the second bit of the original; a level across zero is
// never nearer than its mirror image, so the same form gives every bit.
// out[j] = rs2 * (d0 - d1) with rs2 = rho~ step^2.
template <int NB>
__device__ __forceinline__ void dimension_llr_nb(float u, float rs2, float* out) {
  float v = u;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const int half = 1 << (NB - 1 - j);  // half the levels of this stage
    const float a = fabsf(v);
    if (half == 1) {
      out[j] = rs2 * (4.0f * v);
    } else {
      float m = 4.0f * a;
#pragma unroll
      for (int l = 2; l <= half; ++l) m = fmaxf(m, fmaf(4.0f * l, a, -4.0f * l * (l - 1)));
      out[j] = rs2 * copysignf(m, v);
    }
    v = (float)half - a;
  }
}

__device__ __forceinline__ void dimension_llr(float u, float rs2, const DetectParams& P,
                                              float* out) {
  switch (P.nb) {
    case 1: dimension_llr_nb<1>(u, rs2, out); break;
    case 2: dimension_llr_nb<2>(u, rs2, out); break;
    case 3: dimension_llr_nb<3>(u, rs2, out); break;
    default: dimension_llr_nb<4>(u, rs2, out); break;
  }
}

// Soft-output constants of one user (Section III-C): mu~ = p, rho~ =
// ||h||^2 Es / N0.  u_scale: level units per unit of z, 1 / (mu~ sqrt(Es)
// step) (0 when mu~ = 0); rs2: rho~ step^2.
__device__ __forceinline__ float llr_u_scale(float p, const DetectParams& P) {
  return p > 0.0f ? 1.0f / (p * P.sqrt_es * P.lvl_step) : 0.0f;
}
__device__ __forceinline__ float llr_rs2(float nrm, const DetectParams& P) {
  return nrm * P.rho_scale * (P.lvl_step * P.lvl_step);
}

// Soft output of one user: LLRs of z / (mu~ sqrt(Es)) against the
// unit-energy alphabet; a user with mu~ = 0 gets L = 0.
__device__ __forceinline__ void user_llr(float2 z, float nrm, float p, const DetectParams& P,
                                         float* out) {
  if (!(p > 0.0f)) {
    for (int j = 0; j < P.Q; ++j) out[j] = 0.0f;
    return;
  }
  const float us = llr_u_scale(p, P);
  const float rs2 = llr_rs2(nrm, P);
  dimension_llr(z.x * us, rs2, P, out);
  if (!P.bpsk) dimension_llr(z.y * us, rs2, P, out + P.nb);
}

}  // namespace ocd
