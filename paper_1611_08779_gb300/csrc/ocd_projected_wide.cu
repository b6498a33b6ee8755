// Bulk-copy projected OCD kernels for up to 32 users (warp-level MMA and
// tcgen05 products): launch, the batched kernel pointer and the fault word.
#include "ocd_projected_tc.cuh"
#include "ocd_projected_wide.cuh"

namespace ocd {

const void* projected_wide_kernel_ptr() {
  return reinterpret_cast<const void*>(ocd_projected_wide_kernel);
}

size_t projected_wide_smem_per_cta() { return WideShape::kWarpBytes + 1024; }

int projected_wide_threads() { return WideShape::kThreads; }

cudaError_t launch_projected_wide(const DetectParams& P, unsigned grid, cudaStream_t stream) {
  CUtensorMap map;
  const cudaError_t e = encode_ymap(P, &map);
  if (e != cudaSuccess) return e;
  DetectParams p = P;
  void* args[] = {&p, &map};
  return launch_serialized(projected_wide_kernel_ptr(), grid, WideShape::kThreads, args,
                           projected_wide_smem_per_cta(), stream);
}

const void* projected_tc_kernel_ptr(int T) {
  return T <= 8 ? reinterpret_cast<const void*>(ocd_projected_tc_kernel<8>)
                : reinterpret_cast<const void*>(ocd_projected_tc_kernel<16>);
}

size_t projected_tc_smem_per_cta(int T) {
  return (T <= 8 ? TcShape<8>::kBytes : TcShape<16>::kBytes) + 1024;
}

int projected_tc_threads() { return TcShape<16>::kThreads; }

cudaError_t launch_projected_tc(const DetectParams& P, unsigned grid, cudaStream_t stream) {
  CUtensorMap map;
  const cudaError_t e = encode_ymap_rows(P, &map, P.T <= 8 ? 8 : 16);
  if (e != cudaSuccess) return e;
  DetectParams p = P;
  void* args[] = {&p, &map};
  return launch_serialized(projected_tc_kernel_ptr(P.T), grid, projected_tc_threads(), args,
                           projected_tc_smem_per_cta(P.T), stream);
}

bool wide_fuses(int T) { return OCD_WIDE_FUSE && T <= 8; }

BatchFn batched_wide_kernel(bool fused) {
  return fused ? ocd_batched_wide_kernel<true> : ocd_batched_wide_kernel<false>;
}

cudaError_t projected_wide_fault(unsigned int* bits, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(bits, g_wide_fault, sizeof(unsigned int));
  if (e == cudaSuccess && clear) {
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbol(g_wide_fault, &zero, sizeof(unsigned int));
  }
  return e;
}

}  // namespace ocd
