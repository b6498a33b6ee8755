// Projected OCD for one symbol per channel, one lane per subcarrier: kernel
// table and launch.
#include "ocd_projected_lane.cuh"

namespace ocd {

namespace {

template <int U>
constexpr const void* lane_fn() {
  return reinterpret_cast<const void*>(ocd_projected_lane_kernel<U>);
}

template <int U>
constexpr size_t lane_smem() {
  return (size_t)LaneShape<U>::kWarps * LaneShape<U>::kWarpBytes;
}

}  // namespace

static_assert(kLaneMaxUsers == 8, "the tables below cover U = 1..8");

const void* projected_lane_kernel_ptr(int U) {
  switch (U) {
    case 1: return lane_fn<1>();
    case 2: return lane_fn<2>();
    case 3: return lane_fn<3>();
    case 4: return lane_fn<4>();
    case 5: return lane_fn<5>();
    case 6: return lane_fn<6>();
    case 7: return lane_fn<7>();
    case 8: return lane_fn<8>();
    default: return nullptr;
  }
}

size_t projected_lane_smem_per_cta(int U) {
  switch (U) {
    case 1: return lane_smem<1>();
    case 2: return lane_smem<2>();
    case 3: return lane_smem<3>();
    case 4: return lane_smem<4>();
    case 5: return lane_smem<5>();
    case 6: return lane_smem<6>();
    case 7: return lane_smem<7>();
    case 8: return lane_smem<8>();
    default: return 0;
  }
}

int projected_lane_threads() { return 32 * LaneShape<1>::kWarps; }

long long projected_lane_groups(long long Nsc) { return (Nsc + 31) / 32; }

cudaError_t launch_projected_lane(const DetectParams& P, unsigned grid, cudaStream_t stream) {
  const void* fn = projected_lane_kernel_ptr(P.U);
  if (!fn) return cudaErrorInvalidValue;
  DetectParams p = P;
  void* args[] = {&p};
  return launch_serialized(fn, grid, projected_lane_threads(), args,
                           projected_lane_smem_per_cta(P.U), stream);
}

}  // namespace ocd
