// Host-side helpers shared by the C-ABI translation units (ocd_api.cu,
// ocd_batched.cu): error reporting, argument validation, launch planning and
// per-device state.  Internal; not part of the public header.
#pragma once

#include <cuda_runtime.h>

#include <mutex>

#include "ocd_common.cuh"

namespace ocdh {

constexpr int kMaxDevices = 64;
constexpr size_t kSmemBudget = 72 * 1024;  // preferred per-CTA budget: >= 3 CTAs per SM
constexpr unsigned long long kCopyWaitNs = 1000000000ull;  // 1 s limit on any copy wait
constexpr size_t kBatchStaticSmem = 64;  // static shared memory bound of the batched kernels

// Records a message for ocd_last_error() and returns `code`.
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// Constellation constants (Section II-A, II-D).
struct Alphabet {
  int Q, nb, M, bpsk;
  double step;    // 1/sigma
  double radius;  // max Re{O} at unit energy
};
bool alphabet_of(int order, Alphabet& a);

int validate(const void* H, const void* Y, int storage, int Nsc, int B, int U, int T, float N0,
             float Es, int K, int mode, int qam_order, const void* xhat, const void* llr, int algo,
             Alphabet& al);
void build_params(const void* H, const void* Y, int storage, int Nsc, int B, int U, int T,
                  float N0, float Es, int K, int mode, const Alphabet& al, void* xhat, float* llr,
                  ocd::DetectParams& P);

struct DeviceInfo {
  bool ready = false;
  int sms = 0;
  size_t smem_optin = 0;  // largest dynamic shared memory a CTA may opt into
};
int device_info(int dev, DeviceInfo& out);

// Residual-form launch plan (fills P.L, logL, chunk, scmax, items).
struct Plan {
  int npp, S, L, nt;
  size_t smem;
};
int make_plan(int B, int U, int T, size_t budget, ocd::DetectParams& P, Plan& pl, int S_req,
              int L_req);

bool can_tma32(const ocd::DetectParams& P);  // U <= 16
bool can_lane(const ocd::DetectParams& P);   // T == 1, U <= 8: one lane per subcarrier
bool can_wide(const ocd::DetectParams& P);   // 16 < U <= 32
bool can_tc(const ocd::DetectParams& P);     // the tcgen05 kernel supports the shape
bool prefer_tc(const ocd::DetectParams& P);
bool prefer_tc_batched(const ocd::DetectParams& P);  // ... the default for a batched cell  // ... and is the projected default

// Grid of the one-lane-per-subcarrier kernel for P (0 when it cannot be
// resident on the device).
int lane_grid(const ocd::DetectParams& P, const DeviceInfo& di, unsigned& grid);

// Internal streams (per device, created once) shared by the host-buffer path
// and the batched form; the caller holds g_hs_mu for the whole enqueue.
constexpr int kHostStreams = 4;
struct HostStreams {
  bool ready = false;
  cudaStream_t s[kHostStreams];
  cudaEvent_t ev_in, ev_out[kHostStreams];
};
extern std::mutex g_hs_mu;
int host_streams(int dev, HostStreams*& out);

}  // namespace ocdh
