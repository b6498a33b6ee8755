// C ABI of the OCD detector: argument validation, launch planning and
// dispatch to the sm_103a kernels.  See include/ocd.h for the contract.
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "ocd.h"
#include "ocd_common.cuh"
#include "ocd_batch.cuh"
#include "ocd_host.h"
#include "ocd_residual.cuh"

namespace ocdh {

constexpr int kVersion = 100;  // 0.1.0

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(OCD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

int pow2_ceil(int v) { return 1 << ilog2(v < 1 ? 1 : v); }

// ---------------------------------------------------------------------------
// Constellation constants (Section II-A, II-D)
// ---------------------------------------------------------------------------
bool alphabet_of(int order, Alphabet& a) {
  switch (order) {
    case 2: a = {1, 1, 2, 1, 1.0, 1.0}; return true;
    case 4: case 16: case 64: case 256: {
      const int Q = order == 4 ? 2 : order == 16 ? 4 : order == 64 ? 6 : 8;
      const int M = 1 << (Q / 2);
      const double sigma = sqrt(2.0 * (M * M - 1) / 3.0);
      a = {Q, Q / 2, M, 0, 1.0 / sigma, (M - 1) / sigma};
      return true;
    }
    default: return false;
  }
}

// ---------------------------------------------------------------------------
// Kernel table: UMAX in {4, 8, 16, 32} x NPP in {2, 4, 8, 16}
// ---------------------------------------------------------------------------
using ocd::KernelFn;
constexpr int kNpps[4] = {2, 4, 8, 16};

DeviceInfo g_dev[kMaxDevices];
std::mutex g_dev_mu;

int device_info(int dev, DeviceInfo& out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(OCD_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (!g_dev[dev].ready) {
    int sms = 0, optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    for (int S = 1; S <= 2; ++S)
      for (int npp : kNpps) {
        e = cudaFuncSetAttribute(ocd::residual_kernel(npp, S),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      }
    for (int umax : {4, 8}) {
      e = cudaFuncSetAttribute(ocd::projected_kernel(umax),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    }
    for (int u : {8, 16}) {
      e = cudaFuncSetAttribute(ocd::projected_tma_kernel_ptr(u),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    }
    for (int st : {(int)ocd::kStoreBF16, (int)ocd::kStoreF16})
      for (int u : {8, 16}) {
        e = cudaFuncSetAttribute(ocd::projected_h16_kernel_ptr(st, u),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      }
    // the batched residual kernels hold a static ticket slot: dynamic
    // shared memory up to the opt-in limit minus kBatchStaticSmem
    for (int S = 1; S <= 2; ++S)
      for (int npp : kNpps) {
        const void* fn = reinterpret_cast<const void*>(ocd::batched_residual_kernel(npp, S));
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, fn);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
        if (fa.sharedSizeBytes > kBatchStaticSmem)
          return fail(OCD_ERR_UNSUPPORTED, "batched kernel holds %zu bytes of static shared memory",
                      fa.sharedSizeBytes);
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)kBatchStaticSmem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      }
    for (int u : {8, 16}) {
      e = cudaFuncSetAttribute(reinterpret_cast<const void*>(ocd::batched_tma_kernel(u)),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    }
    for (int u = 1; u <= ocd::kLaneMaxUsers; ++u) {
      e = cudaFuncSetAttribute(ocd::projected_lane_kernel_ptr(u),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    }
    for (const void* fn : {ocd::projected_wide_kernel_ptr(),
                           reinterpret_cast<const void*>(ocd::batched_wide_kernel(false)),
                           reinterpret_cast<const void*>(ocd::batched_wide_kernel(true)),
                           ocd::projected_tc_kernel_ptr(1), ocd::projected_tc_kernel_ptr(16)}) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    }
    g_dev[dev].sms = sms;
    g_dev[dev].smem_optin = (size_t)optin;
    g_dev[dev].ready = true;
  }
  out = g_dev[dev];
  return OCD_OK;
}

// ---------------------------------------------------------------------------
// Launch plan
// ---------------------------------------------------------------------------

// Two symbols per item when a subcarrier carries several (each staged h
// block then feeds two inner products and two residual updates); the fewest
// lanes per item (fewest shuffles) whose staged channels fit the budget.
// S_req / L_req (0 = default) override the symbols and the lanes per item.
int make_plan(int B, int U, int T, size_t budget, ocd::DetectParams& P, Plan& pl, int S_req,
              int L_req) {
  const int S = S_req ? S_req : (T >= 2 ? 2 : 1);
  const int G = (T + S - 1) / S;
  const int npp_cap = 8;
  const int pairs = (B + 1) / 2;
  int L = 1;
  while (L * npp_cap < pairs) L <<= 1;
  if (L_req > L) L = L_req;
  int nt = 128;
  for (;;) {
    if (L > 32) return fail(OCD_ERR_UNSUPPORTED, "B=%d does not fit the team layout", B);
    int npp = pow2_ceil((pairs + L - 1) / L);
    if (npp < 2) npp = 2;
    const int teams = nt / L;
    const int chunk = teams;
    int scmax = (chunk - 1 + G - 1) / G + 1;
    if (scmax > chunk) scmax = chunk;
    const ocd::ResidualSmem lay = ocd::residual_smem(L, npp, S, U, scmax, teams);
    if (lay.total <= budget) {
      pl.npp = npp; pl.S = S; pl.L = L; pl.nt = nt; pl.smem = lay.total;
      P.L = L; P.logL = ilog2(L); P.chunk = chunk; P.scmax = scmax;
      P.items = (long long)P.Nsc * G;
      return OCD_OK;
    }
    if (L < 32) L <<= 1;
    else if (nt > 32) nt >>= 1;
    else return fail(OCD_ERR_UNSUPPORTED, "B=%d U=%d: one subcarrier exceeds shared memory", B, U);
  }
}

int validate(const void* H, const void* Y, int storage, int Nsc, int B, int U, int T, float N0,
             float Es, int K, int mode, int qam_order, const void* xhat, const void* llr, int algo,
             Alphabet& al) {
  if (algo != OCD_ALGO_AUTO && algo != OCD_ALGO_RESIDUAL && algo != OCD_ALGO_PROJECTED &&
      algo != OCD_ALGO_PROJECTED_WARP && algo != OCD_ALGO_PROJECTED_TC)
    return fail(OCD_ERR_ARG, "unknown algo %d", algo);
  if (storage != OCD_STORE_C64 && storage != OCD_STORE_BF16 && storage != OCD_STORE_F16)
    return fail(OCD_ERR_ARG, "unknown storage %d", storage);
  if (Nsc < 0 || T < 0) return fail(OCD_ERR_ARG, "Nsc=%d and T=%d must be >= 0", Nsc, T);
  if (B < 1 || B > OCD_MAX_ANTENNAS) return fail(OCD_ERR_ARG, "B=%d outside 1..%d", B, OCD_MAX_ANTENNAS);
  if (U < 1 || U > OCD_MAX_USERS) return fail(OCD_ERR_ARG, "U=%d outside 1..%d", U, OCD_MAX_USERS);
  if (K < 0 || K > OCD_MAX_SWEEPS) return fail(OCD_ERR_ARG, "K=%d outside 0..%d", K, OCD_MAX_SWEEPS);
  if (mode != OCD_MMSE && mode != OCD_BOX) return fail(OCD_ERR_ARG, "unknown mode %d", mode);
  if (!alphabet_of(qam_order, al)) return fail(OCD_ERR_ARG, "unsupported qam_order %d", qam_order);
  if (!(Es > 0.0f) || !isfinite(Es)) return fail(OCD_ERR_ARG, "Es must be finite and > 0");
  if (!(N0 >= 0.0f) || !isfinite(N0)) return fail(OCD_ERR_ARG, "N0 must be finite and >= 0");
  if (llr && !(N0 > 0.0f)) return fail(OCD_ERR_ARG, "LLRs need N0 > 0 (rho~ = ||h||^2 Es/N0)");
  // An empty problem may come with NULL pointers (empty tensors have no storage).
  const long long items = (long long)Nsc * T;
  if (items > 0 && !xhat && !llr) return fail(OCD_ERR_ARG, "both outputs are NULL");
  if (items > 0 && (!H || !Y)) return fail(OCD_ERR_ARG, "H and Y must not be NULL");
  if ((((uintptr_t)H | (uintptr_t)Y) & (storage == OCD_STORE_C64 ? 7u : 3u)) || ((uintptr_t)xhat & 7u))
    return fail(OCD_ERR_ARG, "complex arrays must be aligned to their element size");
  if ((uintptr_t)llr & 3u) return fail(OCD_ERR_ARG, "llr must be 4-byte aligned");
  return OCD_OK;
}

bool aligned16(const ocd::DetectParams& P) {
  return ((reinterpret_cast<uintptr_t>(P.H) | reinterpret_cast<uintptr_t>(P.Y)) & 15u) == 0;
}
// Bulk-copy variants: float32 storage needs even B (16-byte rows), 16-bit
// storage B % 4 == 0; both need 16-byte aligned bases.
bool can_tma32(const ocd::DetectParams& P) {
  return P.storage == ocd::kStoreC64 && P.U <= ocd::kTmaMaxUsers && P.B % 2 == 0 &&
         aligned16(P);
}
bool can_h16(const ocd::DetectParams& P) {
  return P.storage != ocd::kStoreC64 && P.U <= ocd::kH16MaxUsers && P.B % 4 == 0 &&
         aligned16(P);
}
bool can_wide(const ocd::DetectParams& P) {
  return P.storage == ocd::kStoreC64 && P.U > ocd::kTmaMaxUsers && P.U <= ocd::kWideMaxUsers &&
         P.B % 2 == 0 && aligned16(P);
}
// tcgen05 products for 16 < U <= 32 with at most 16 symbols per subcarrier
// (float32 storage, even B, 16-byte aligned bases).
bool can_tc(const ocd::DetectParams& P) {
  return can_wide(P) && P.T <= ocd::kTcMaxSymbols;
}
// Where the projected form takes the tcgen05 kernel by default: wherever it
// fits (T <= 16).  Measured faster than the warp-level kernel at every shape
// timed, including the short passes where the warp-level kernel folds q0
// into its G phase (256x32: T = 14 0.181 against 0.239 ms, T = 7 0.170
// against 0.181, T = 1 0.588 against 0.666; 128x32 T = 1 0.638 against
// 0.780; 32x17 T = 5 0.343 against 0.355).
bool prefer_tc(const ocd::DetectParams& P) { return can_tc(P); }
// The same choice for a cell of the batched form, where a tcgen05 launch
// holds whole SMs (all of their shared and tensor memory) while the other
// cells' persistent launches would share them: only for 9..16 symbols.  On
// the 24-cell mix of the benchmark, the tcgen05 kernel for the 256x32 cells
// with 1 and 7 symbols made the batch 6% slower (0.504 -> 0.535 ms) although
// each of those cells alone is faster on it.
bool prefer_tc_batched(const ocd::DetectParams& P) { return can_tc(P) && P.T > 8; }
// One lane per subcarrier: one symbol, float32 storage, U <= 8, even B,
// 16-byte aligned bases.
bool can_lane(const ocd::DetectParams& P) {
  return P.storage == ocd::kStoreC64 && P.T == 1 && P.U <= ocd::kLaneMaxUsers &&
         P.B % 2 == 0 && aligned16(P);
}
bool can_projected(const ocd::DetectParams& P) {
  return can_tma32(P) || can_wide(P) || can_h16(P) || P.U <= ocd::kProjectedMaxUsers;
}

// Algorithm choice for OCD_ALGO_AUTO: the projected form wins whenever its
// two per-subcarrier products are shared by more than one symbol.  For one
// symbol it still wins in its bulk-copy and one-lane-per-subcarrier kernels
// (measured at 32x8, 128x8 and 128x16, T = 1); the load-based projected
// kernel keeps the residual form for T = 1.
int resolve_algo(int algo, const ocd::DetectParams& P) {
  if (algo != OCD_ALGO_AUTO) return algo;
  const bool one_symbol_ok = can_lane(P) || can_tma32(P) || can_wide(P);
  return (can_projected(P) && (P.T >= 2 || one_symbol_ok)) ? OCD_ALGO_PROJECTED
                                                          : OCD_ALGO_RESIDUAL;
}

int lane_grid(const ocd::DetectParams& P, const DeviceInfo& di, unsigned& grid) {
  grid = 0;
  const void* fn = ocd::projected_lane_kernel_ptr(P.U);
  const int lt = ocd::projected_lane_threads();
  int per_sm = 0;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, fn, lt, ocd::projected_lane_smem_per_cta(P.U));
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (per_sm < 1) return OCD_OK;
  // one warp per group of 32 subcarriers, as many as the SMs hold
  // (measured: cutting the warp count to even out the last round of groups
  // loses more than the last round costs)
  const int wpc = lt / 32;
  const long long groups = ocd::projected_lane_groups(P.Nsc);
  const long long wmax = (long long)di.sms * per_sm * wpc;
  const long long warps = groups < wmax ? groups : wmax;
  grid = (unsigned)((warps + wpc - 1) / wpc);
  return OCD_OK;
}

// use_tc: run the tcgen05 kernel (the caller has checked can_tc); false
// keeps the warp-level MMA kernels.
int launch_projected(ocd::DetectParams& P, const DeviceInfo& di, int U, bool use_tc,
                     cudaStream_t stream) {
  const int nt = 128;
  const long long need = (P.Nsc + nt / 32 - 1) / (nt / 32);  // one warp per subcarrier
  int per_sm = 0;
  cudaError_t e;
  if (use_tc) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ocd::projected_tc_kernel_ptr(P.T),
                                                      ocd::projected_tc_threads(),
                                                      ocd::projected_tc_smem_per_cta(P.T));
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm >= 1) {
      // one CTA per SM (it holds the SM's whole tensor memory), persistent
      long long grid = di.sms;
      if (grid > P.Nsc) grid = P.Nsc;
      e = ocd::launch_projected_tc(P, (unsigned)grid, stream);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) return OCD_OK;
      return cuda_fail(e, "projected tcgen05 kernel launch");
    }
    return fail(OCD_ERR_UNSUPPORTED, "tcgen05 kernel cannot be resident");
  }
  if (can_lane(P)) {
    unsigned grid = 0;
    const int st = lane_grid(P, di, grid);
    if (st != OCD_OK) return st;
    if (grid > 0) {
      e = ocd::launch_projected_lane(P, grid, stream);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "projected kernel launch");
      return OCD_OK;
    }
  }
  if (can_wide(P)) {
    const void* fn = ocd::projected_wide_kernel_ptr();
    const int wt = ocd::projected_wide_threads();
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, wt,
                                                      ocd::projected_wide_smem_per_cta());
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm >= 1) {
      long long grid = (long long)di.sms * per_sm;
      if (grid > P.Nsc) grid = P.Nsc;  // one warp (CTA) per subcarrier
      e = ocd::launch_projected_wide(P, (unsigned)grid, stream);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) return OCD_OK;
      if (e != cudaErrorNotSupported) return cuda_fail(e, "projected kernel launch");
    }
  }
  const bool h16 = can_h16(P);
  if (can_tma32(P) || h16) {
    const void* fn =
        h16 ? ocd::projected_h16_kernel_ptr(P.storage, U) : ocd::projected_tma_kernel_ptr(U);
    const size_t smem =
        h16 ? ocd::projected_h16_smem_per_cta(U) : ocd::projected_tma_smem_per_cta(U);
    const int tt = h16 ? nt : ocd::projected_tma_threads();
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, tt, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm >= 1) {
      long long grid = (long long)di.sms * per_sm;
      const long long need_t = (P.Nsc + tt / 32 - 1) / (tt / 32);  // one warp per subcarrier
      if (grid > need_t) grid = need_t;
      e = h16 ? ocd::launch_projected_h16(P, (unsigned)grid, stream)
              : ocd::launch_projected_tma(P, (unsigned)grid, stream);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) return OCD_OK;
      // no tensor-map encoder in this driver: the load-based variant follows
      if (e != cudaErrorNotSupported) return cuda_fail(e, "projected kernel launch");
    }
  }
  if (U > ocd::kProjectedMaxUsers)
    return fail(OCD_ERR_UNSUPPORTED, "projected form for U=%d needs the bulk-copy path "
                "(even B, or B %% 4 == 0 for 16-bit storage; 16-byte aligned H and Y; "
                "float32 storage above 16 users)", U);
  const int umax = U <= 4 ? 4 : 8;
  KernelFn fn = ocd::projected_kernel(umax);
  const size_t smem = (nt / 32) * ocd::projected_smem_per_warp(umax);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (per_sm < 1) return fail(OCD_ERR_UNSUPPORTED, "projected kernel cannot be resident");
  long long grid = (long long)di.sms * per_sm;
  if (grid > need) grid = need;
  void* args[] = {&P};
  e = cudaLaunchKernel((const void*)fn, dim3((unsigned)grid), dim3(nt), args, smem, stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return OCD_OK;
}

void build_params(const void* H, const void* Y, int storage, int Nsc, int B, int U, int T,
                  float N0, float Es, int K, int mode, const Alphabet& al, void* xhat, float* llr,
                  ocd::DetectParams& P) {
  memset(&P, 0, sizeof(P));
  P.H = static_cast<const float2*>(H);
  P.Y = static_cast<const float2*>(Y);
  P.xhat = static_cast<float2*>(xhat);
  P.llr = llr;
  P.items = (long long)Nsc * T;
  P.Nsc = Nsc; P.B = B; P.U = U; P.T = T; P.K = K;
  P.box = mode == OCD_BOX;
  P.bpsk = al.bpsk;
  P.Q = al.Q; P.nb = al.nb; P.M = al.M;
  P.alpha = mode == OCD_MMSE ? (float)((double)N0 / (double)Es) : 0.0f;
  P.sqrt_es = (float)sqrt((double)Es);
  P.box_a = (float)(al.radius * sqrt((double)Es));
  P.rho_scale = N0 > 0.0f ? (float)((double)Es / (double)N0) : 0.0f;
  P.lvl_step = (float)al.step;
  P.storage = storage;
  P.vec_y = (B % 2 == 0) && (((uintptr_t)Y & (storage == ocd::kStoreC64 ? 15u : 7u)) == 0);
  P.wait_ns = kCopyWaitNs;
}

int launch_detect(const void* H, const void* Y, int storage, int Nsc, int B, int U, int T,
                  float N0, float Es, int K, int mode, const Alphabet& al, void* xhat, float* llr,
                  int algo, cudaStream_t stream) {
  const long long items = (long long)Nsc * T;
  if (items == 0) return OCD_OK;
  ocd::DetectParams P;
  build_params(H, Y, storage, Nsc, B, U, T, N0, Es, K, mode, al, xhat, llr, P);

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  DeviceInfo di;
  int st = device_info(dev, di);
  if (st != OCD_OK) return st;

  algo = resolve_algo(algo, P);
  if (algo == OCD_ALGO_PROJECTED_TC) {
    if (!can_tc(P))
      return fail(OCD_ERR_UNSUPPORTED, "the tcgen05 kernel needs 16 < U <= 32, T <= %d, float32 "
                  "storage, even B and 16-byte aligned H and Y", ocd::kTcMaxSymbols);
    return launch_projected(P, di, U, true, stream);
  }
  if (algo == OCD_ALGO_PROJECTED || algo == OCD_ALGO_PROJECTED_WARP) {
    if (!can_projected(P))
      return fail(OCD_ERR_UNSUPPORTED, "projected form does not support U=%d with this storage "
                  "and alignment", U);
    return launch_projected(P, di, U, algo == OCD_ALGO_PROJECTED && prefer_tc(P), stream);
  }

  // Keep several CTAs per SM when the staged channels allow it; otherwise
  // take up to the whole opt-in shared memory of one CTA.
  Plan pl;
  st = make_plan(B, U, T, kSmemBudget, P, pl, 0, 0);
  if (st != OCD_OK) st = make_plan(B, U, T, di.smem_optin, P, pl, 0, 0);
  if (st != OCD_OK) return st;

  KernelFn fn = ocd::residual_kernel(pl.npp, pl.S);
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, pl.nt, pl.smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (per_sm < 1) return fail(OCD_ERR_UNSUPPORTED, "kernel cannot be resident (smem %zu)", pl.smem);
  const long long nchunks = (P.items + P.chunk - 1) / P.chunk;
  long long grid = (long long)di.sms * per_sm;
  if (grid > nchunks) grid = nchunks;
  void* args[] = {&P};
  e = cudaLaunchKernel((const void*)fn, dim3((unsigned)grid), dim3(pl.nt), args, pl.smem, stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return OCD_OK;
}

HostStreams g_hs[kMaxDevices];
std::mutex g_hs_mu;

// Caller holds g_hs_mu.
int host_streams(int dev, HostStreams*& out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(OCD_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
  HostStreams& h = g_hs[dev];
  if (!h.ready) {
    cudaError_t e;
    for (int i = 0; i < kHostStreams; ++i) {
      e = cudaStreamCreateWithFlags(&h.s[i], cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
      e = cudaEventCreateWithFlags(&h.ev_out[i], cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreateWithFlags");
    }
    e = cudaEventCreateWithFlags(&h.ev_in, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreateWithFlags");
    h.ready = true;
  }
  out = &h;
  return OCD_OK;
}

}  // namespace ocdh

using namespace ocdh;

extern "C" {

int ocd_detect_typed(const void* H, const void* Y, int storage, int Nsc, int B, int U, int T,
                     float N0, float Es, int K, int mode, int qam_order, void* xhat, float* llr,
                     int algo, cudaStream_t stream) {
  Alphabet al;
  int st = validate(H, Y, storage, Nsc, B, U, T, N0, Es, K, mode, qam_order, xhat, llr, algo, al);
  if (st != OCD_OK) return st;
  return launch_detect(H, Y, storage, Nsc, B, U, T, N0, Es, K, mode, al, xhat, llr, algo, stream);
}

int ocd_detect_ex(const void* H, const void* Y, int Nsc, int B, int U, int T, float N0, float Es,
                  int K, int mode, int qam_order, void* xhat, float* llr, int algo,
                  cudaStream_t stream) {
  return ocd_detect_typed(H, Y, OCD_STORE_C64, Nsc, B, U, T, N0, Es, K, mode, qam_order, xhat,
                          llr, algo, stream);
}

int ocd_detect(const void* H, const void* Y, int Nsc, int B, int U, int T, float N0, float Es,
               int K, int mode, int qam_order, void* xhat, float* llr, cudaStream_t stream) {
  return ocd_detect_ex(H, Y, Nsc, B, U, T, N0, Es, K, mode, qam_order, xhat, llr, OCD_ALGO_AUTO,
                       stream);
}

int ocd_detect_host(const void* H, const void* Y, int Nsc, int B, int U, int T, float N0, float Es,
                    int K, int mode, int qam_order, void* xhat, float* llr, void* dH, void* dY,
                    void* dX, float* dL, int pieces, cudaStream_t stream) {
  Alphabet al;
  int st = validate(H, Y, OCD_STORE_C64, Nsc, B, U, T, N0, Es, K, mode, qam_order, xhat, llr,
                    OCD_ALGO_AUTO, al);
  if (st != OCD_OK) return st;
  if (pieces < 1 || pieces > 64) return fail(OCD_ERR_ARG, "pieces=%d outside 1..64", pieces);
  const long long items = (long long)Nsc * T;
  if (items == 0) return OCD_OK;
  if (!dH || !dY) return fail(OCD_ERR_ARG, "device staging buffers dH, dY must not be NULL");
  if (xhat && !dX) return fail(OCD_ERR_ARG, "xhat requested but dX is NULL");
  if (llr && !dL) return fail(OCD_ERR_ARG, "llr requested but dL is NULL");
  if (((uintptr_t)dH | (uintptr_t)dY | (uintptr_t)dX) & 7u || ((uintptr_t)dL & 3u))
    return fail(OCD_ERR_ARG, "device staging buffers are misaligned");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  // The internal streams and events are shared by every caller on this
  // device, so the whole enqueue sequence runs under one lock.
  std::lock_guard<std::mutex> lk(g_hs_mu);
  HostStreams* hs = nullptr;
  st = host_streams(dev, hs);
  if (st != OCD_OK) return st;

  e = cudaEventRecord(hs->ev_in, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  for (int i = 0; i < kHostStreams; ++i) {
    e = cudaStreamWaitEvent(hs->s[i], hs->ev_in, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
  }
  if (pieces > Nsc) pieces = Nsc > 0 ? Nsc : 1;
  const size_t hsz = (size_t)B * U * sizeof(float2);
  const size_t ysz = (size_t)T * B * sizeof(float2);
  const size_t xsz = (size_t)T * U * sizeof(float2);
  const size_t lsz = (size_t)T * U * al.Q * sizeof(float);
  for (int p = 0; p < pieces; ++p) {
    const long long a = (long long)Nsc * p / pieces;
    const long long b = (long long)Nsc * (p + 1) / pieces;
    const int n = (int)(b - a);
    if (n == 0) continue;
    cudaStream_t s = hs->s[p % kHostStreams];
    char* dh = static_cast<char*>(dH) + a * hsz;
    char* dy = static_cast<char*>(dY) + a * ysz;
    e = cudaMemcpyAsync(dh, static_cast<const char*>(H) + a * hsz, n * hsz, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H");
    e = cudaMemcpyAsync(dy, static_cast<const char*>(Y) + a * ysz, n * ysz, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync Y");
    char* dx = xhat ? static_cast<char*>(dX) + a * xsz : nullptr;
    float* dl = llr ? reinterpret_cast<float*>(reinterpret_cast<char*>(dL) + a * lsz) : nullptr;
    st = launch_detect(dh, dy, OCD_STORE_C64, n, B, U, T, N0, Es, K, mode, al, dx, dl,
                       OCD_ALGO_AUTO, s);
    if (st != OCD_OK) return st;
    if (xhat) {
      e = cudaMemcpyAsync(static_cast<char*>(xhat) + a * xsz, dx, n * xsz, cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync xhat");
    }
    if (llr) {
      e = cudaMemcpyAsync(reinterpret_cast<char*>(llr) + a * lsz, dl, n * lsz, cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync llr");
    }
  }
  for (int i = 0; i < kHostStreams; ++i) {
    e = cudaEventRecord(hs->ev_out[i], hs->s[i]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    e = cudaStreamWaitEvent(stream, hs->ev_out[i], 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
  }
  return OCD_OK;
}

int ocd_wait_selftest(int limit_us, cudaStream_t stream) {
  if (limit_us < 1 || limit_us > 2000000)
    return fail(OCD_ERR_ARG, "limit_us=%d outside 1..2000000", limit_us);
  cudaError_t e = ocd::projected_tma_wait_selftest(1000ull * (unsigned long long)limit_us, stream);
  if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
  return OCD_OK;
}

int ocd_fault_status(int clear) {
  unsigned int bits = 0, bits16 = 0, bitsw = 0;
  cudaError_t e = ocd::projected_tma_fault(&bits, clear != 0);
  if (e == cudaSuccess) e = ocd::projected_h16_fault(&bits16, clear != 0);
  if (e == cudaSuccess) e = ocd::projected_wide_fault(&bitsw, clear != 0);
  if (e != cudaSuccess) return cuda_fail(e, "reading the fault word");
  return (int)(bits | bits16 | bitsw);
}

const char* ocd_last_error(void) { return g_err; }

int ocd_version(void) { return kVersion; }

}  // extern "C"
