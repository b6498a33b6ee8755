// Cell table of the batched persistent launches: several independent OCD
// problems ("cells", e.g. the carriers of several base-station sectors with
// their own B, U, Nsc, T, K, mode and alphabet) drained by one persistent
// grid through a ticket counter.
//
// The table travels as a __grid_constant__ kernel parameter (no upload, no
// device allocation, capturable in a CUDA graph), so one launch takes at most
// kBatchCellsPerLaunch cells; the host splits larger families over several
// launches.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; no driver library is linked)

#include "ocd_common.cuh"

namespace ocd {

constexpr int kBatchCellsPerLaunch = 32;

struct BatchCell {  // aligned as CUtensorMap requires
  CUtensorMap ymap;         // Y as [Nsc*T][2B] floats (bulk-copy kernels only)
  DetectParams P;           // the cell's problem and launch geometry
  long long tick_end;       // one past the cell's last ticket (prefix sum)
  int sc_per_tick;          // bulk-copy kernels: subcarriers per ticket
  int pad;
};

struct BatchTable {
  BatchCell cell[kBatchCellsPerLaunch];
  unsigned int total;       // tickets of all cells = cell[ncells-1].tick_end
  int ncells;
};

static_assert(sizeof(BatchTable) < 32000, "kernel parameters are limited to 32 KB");

// Persistent batched kernels: (table, ticket counter).  The counter must be
// zero when the launch starts.
using BatchFn = void (*)(BatchTable, unsigned int*);
// Residual form by antenna pairs per lane and symbols per item (as
// residual_kernel).
BatchFn batched_residual_kernel(int npp, int s);
// Bulk-copy projected form (float32 storage, U <= 16, even B, 16-byte
// aligned H and Y) and its per-CTA shared memory (= projected_tma_smem_per_cta).
BatchFn batched_tma_kernel(int U);
// Tensor map of Y for the bulk-copy kernels; cudaErrorNotSupported when the
// driver offers no tensor-map encoder.
cudaError_t encode_ymap(const DetectParams& P, CUtensorMap* map);
// The same with a box of `rows` received rows (16 antennas wide).
cudaError_t encode_ymap_rows(const DetectParams& P, CUtensorMap* map, int rows);
// Y's tensor map for the 8/16-user bulk-copy kernel: the 3-D view (32
// floats of 16 antennas, rows, 16-antenna chunks; one copy fetches both
// chunks of a 32-antenna block) when B is a multiple of 16, else the 2-D
// view; *is3d tells which (it goes to DetectParams::ymap3d).
cudaError_t encode_ymap_tma(const DetectParams& P, CUtensorMap* map, int* is3d);
// Staged steps (antenna blocks x symbol passes) per subcarrier of the
// bulk-copy kernels.
int tma_steps_per_sc(int B, int T);

// Bulk-copy projected form for 16 < U <= 32 (float32 storage, even B,
// 16-byte aligned H and Y): one warp per CTA.
constexpr int kWideMaxUsers = 32;
const void* projected_wide_kernel_ptr();
size_t projected_wide_smem_per_cta();
int projected_wide_threads();
cudaError_t launch_projected_wide(const DetectParams& P, unsigned grid, cudaStream_t stream);
// T <= 8: the 32-user kernels accumulate q0 in the G phase (the batched
// kernel instance then takes only such cells).
bool wide_fuses(int T);
BatchFn batched_wide_kernel(bool fused);
cudaError_t projected_wide_fault(unsigned int* bits, bool clear);
// The same products on the fifth-generation tensor cores (tcgen05, TMEM
// accumulators) for 16 < U <= 32, T <= 16 (float32 storage, even B, 16-byte
// aligned H and Y): one 320-thread CTA per SM holding the SM's whole TMEM.
constexpr int kTcMaxSymbols = 16;
const void* projected_tc_kernel_ptr(int T);
size_t projected_tc_smem_per_cta(int T);
int projected_tc_threads();
cudaError_t launch_projected_tc(const DetectParams& P, unsigned grid, cudaStream_t stream);

}  // namespace ocd
