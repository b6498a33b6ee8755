// Bulk-copy (TMA) projected-residual OCD kernel: tensor-map encoding,
// launch, and the fault word.
#include <cudaTypedefs.h>

#include <mutex>

#include "ocd_projected_tma.cuh"

namespace ocd {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

}  // namespace

const void* projected_tma_kernel_ptr(int U) {
  return U <= 8 ? reinterpret_cast<const void*>(ocd_projected_tma_kernel<1>)
                : reinterpret_cast<const void*>(ocd_projected_tma_kernel<2>);
}

size_t projected_tma_smem_per_cta(int U) {
  return OCD_TMA_WARPS * (U <= 8 ? TmaShape<1>::kWarpBytes : TmaShape<2>::kWarpBytes) + 1024;
}

int projected_tma_threads() { return 32 * OCD_TMA_WARPS; }

cudaError_t encode_ymap(const DetectParams& P, CUtensorMap* map) {
  return encode_ymap_rows(P, map, TmaShape<1>::kPass);
}

cudaError_t encode_ymap_rows(const DetectParams& P, CUtensorMap* map, int rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // Y as a 2-D float tensor: rows = (subcarrier, symbol), 2B floats per row.
  const cuuint64_t dims[2] = {2ull * (cuuint64_t)P.B, (cuuint64_t)P.Nsc * (cuuint64_t)P.T};
  const cuuint64_t strides[1] = {2ull * (cuuint64_t)P.B * sizeof(float)};
  const cuuint32_t box[2] = {2 * TmaShape<1>::kBoxAnt, (cuuint32_t)rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(P.Y), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_ymap_tma(const DetectParams& P, CUtensorMap* map, int* is3d) {
  *is3d = 0;
  if (P.B % TmaShape<1>::kBoxAnt != 0) return encode_ymap(P, map);
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // dims: 32 floats (16 antennas) of a chunk, rows (subcarrier, symbol),
  // chunks; the box fetches a whole 32-antenna block, laid out chunk by
  // chunk exactly as two 2-D boxes would be
  constexpr int kChunk = 2 * TmaShape<1>::kBoxAnt;
  const cuuint64_t dims[3] = {(cuuint64_t)kChunk, (cuuint64_t)P.Nsc * (cuuint64_t)P.T,
                              2ull * (cuuint64_t)P.B / kChunk};
  const cuuint64_t strides[2] = {2ull * (cuuint64_t)P.B * sizeof(float), kChunk * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)kChunk, (cuuint32_t)TmaShape<1>::kPass,
                             (cuuint32_t)TmaShape<1>::kBoxes};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(P.Y), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return encode_ymap(P, map);  // the 2-D view always encodes
  *is3d = 1;
  return cudaSuccess;
}

cudaError_t launch_projected_tma(const DetectParams& P, unsigned grid, cudaStream_t stream) {
  CUtensorMap map;
  DetectParams p = P;
  const cudaError_t e = encode_ymap_tma(P, &map, &p.ymap3d);
  if (e != cudaSuccess) return e;
  void* args[] = {&p, &map};
  return launch_serialized(projected_tma_kernel_ptr(P.U), grid, projected_tma_threads(), args,
                           projected_tma_smem_per_cta(P.U), stream);
}

int tma_steps_per_sc(int B, int T) {
  return ((B + TmaShape<1>::kBB - 1) / TmaShape<1>::kBB) * ((T + TmaShape<1>::kPass - 1) / TmaShape<1>::kPass);
}

BatchFn batched_tma_kernel(int U) {
  return U <= 8 ? ocd_batched_tma_kernel<1> : ocd_batched_tma_kernel<2>;
}

cudaError_t projected_tma_fault(unsigned int* bits, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(bits, g_tma_fault, sizeof(unsigned int));
  if (e == cudaSuccess && clear) {
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbol(g_tma_fault, &zero, sizeof(unsigned int));
  }
  return e;
}

cudaError_t projected_tma_wait_selftest(unsigned long long wait_ns, cudaStream_t stream) {
  ocd_wait_selftest_kernel<<<1, 32, 0, stream>>>(wait_ns);
  return cudaGetLastError();
}

}  // namespace ocd
