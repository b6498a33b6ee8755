// 16-bit-storage projected-residual OCD kernels: instances, tensor-map
// encoding, launch, fault word.
#include <cudaTypedefs.h>

#include <mutex>

#include "ocd_projected_h16.cuh"

namespace ocd {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn16() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <int STORE>
const void* pick(int ut) {
  return ut == 1 ? reinterpret_cast<const void*>(ocd_projected_h16_kernel<STORE, 1>)
                 : reinterpret_cast<const void*>(ocd_projected_h16_kernel<STORE, 2>);
}

}  // namespace

const void* projected_h16_kernel_ptr(int storage, int U) {
  const int ut = U <= 8 ? 1 : 2;
  return storage == kStoreBF16 ? pick<kStoreBF16>(ut) : pick<kStoreF16>(ut);
}

size_t projected_h16_smem_per_cta(int U) {
  return 4 * (U <= 8 ? H16Shape<1>::kWarpBytes : H16Shape<2>::kWarpBytes) + 1024;
}

cudaError_t launch_projected_h16(const DetectParams& P, unsigned grid, cudaStream_t stream) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn16();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[2] = {2ull * (cuuint64_t)P.B, (cuuint64_t)P.Nsc * (cuuint64_t)P.T};
  const cuuint64_t strides[1] = {2ull * (cuuint64_t)P.B * 2};
  const cuuint32_t box[2] = {64, 16};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r =
      enc(&map, P.storage == kStoreBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
          2, const_cast<float2*>(P.Y), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  DetectParams p = P;
  void* args[] = {&p, &map};
  return launch_serialized(projected_h16_kernel_ptr(P.storage, P.U), grid, 128, args,
                           projected_h16_smem_per_cta(P.U), stream);
}

cudaError_t projected_h16_fault(unsigned int* bits, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(bits, g_h16_fault, sizeof(unsigned int));
  if (e == cudaSuccess && clear) {
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbol(g_h16_fault, &zero, sizeof(unsigned int));
  }
  return e;
}

}  // namespace ocd
