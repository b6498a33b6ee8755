// Launch parameters of the unfolded (differentiable) OCD kernels; internal.
#pragma once

#include <cuda_runtime.h>

#include "ocd_common.cuh"

namespace ocd {

struct UnfoldParams {
  DetectParams D;                       // alphabet, mode, box radius, sqrt(Es)
  const float2* __restrict__ H;         // [Nsc][B][U] complex64
  const float2* __restrict__ Y;         // [Nsc][T][B] (forward)
  const float* __restrict__ N0;         // [Nsc]
  const float* __restrict__ omega;      // [K]
  const float* __restrict__ alpha;      // [K]
  float2* __restrict__ xhat;            // [Nsc][T][U]: written by the forward, read by the adjoint
  float* __restrict__ llr;              // [Nsc][T][U][Q] or null (forward)
  float2* __restrict__ ckpt;            // [K][Nsc*T][B+U]: r, then z, at the start of each sweep
  const float2* __restrict__ dxhat;     // adjoint inputs (either may be null)
  const float* __restrict__ dllr;
  float* __restrict__ partial;          // [Nsc*T][2K] per-sample parameter adjoints
  float* __restrict__ domega;           // [K] outputs of the adjoint
  float* __restrict__ dalpha;
  const float* __restrict__ bits;       // [Nsc][T][U][Q] labels of the fused loss, or null (forward)
  float* __restrict__ gllr;             // fused loss: d loss / d LLR (forward output)
  float* __restrict__ lpart;            // fused loss: [Nsc*T] per-sample loss sums (forward)
  float* __restrict__ loss;             // fused loss: the mean (forward output, one float)
  const float* __restrict__ gscale;     // factor of the summed parameter gradients, or null (1)
  float inv_n;                          // fused loss: 1 / (Nsc T U Q)
  long long samples;                    // Nsc * T
  int Nsc, B, U, T, K;
  float es;
  int projected;                        // 1: q-space arrangement (checkpoints G and (q, z))
};

// Forward (backward = false) or adjoint + reduction (backward = true).
cudaError_t launch_unfolded(const UnfoldParams& P, bool backward, int sms, cudaStream_t stream);
// Whether the projected arrangement's shared-memory copy fits for (B, U).
bool projected_fits(int B, int U);

}  // namespace ocd
