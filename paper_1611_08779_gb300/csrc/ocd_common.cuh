// Shared device-side pieces of the OCD detector: launch parameters, the
// projection of Eq. 14 and the per-dimension max-log LLR of Eq. 9.
#pragma once

#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

namespace ocd {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kUserSlots = 32;  // per-subcarrier slots of the preprocessing tables

struct DetectParams {
  const float2* __restrict__ H;  // [Nsc][B][U]
  const float2* __restrict__ Y;  // [Nsc][T][B]
  float2* __restrict__ xhat;     // [Nsc][T][U] or null
  float* __restrict__ llr;       // [Nsc][T][U][Q] or null
  long long items;               // Nsc * T (one item = one subcarrier-symbol pair)
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
};

using KernelFn = void (*)(DetectParams);

// Residual-form kernels by antenna pairs per lane (2, 4, 8, 16).
KernelFn residual_kernel(int npp);

// Projection onto C_O (Eq. 14): for square QAM clip real and imaginary parts
// independently to [-a, a]; for BPSK clip the real part and zero the
// imaginary part.  MMSE mode has C = C (identity).
__device__ __forceinline__ void project(float& wr, float& wi, const DetectParams& P) {
  if (P.box) {
    wr = fminf(fmaxf(wr, -P.box_a), P.box_a);
    wi = P.bpsk ? 0.0f : fminf(fmaxf(wi, -P.box_a), P.box_a);
  }
}

// Max-log LLRs (Eq. 9) of the bits carried by one real dimension.  For a
// separable Gray alphabet the minima over O_b^0 and O_b^1 differ only in this
// dimension, so the other dimension's contribution cancels exactly.
__device__ __forceinline__ void dimension_llr(float x, float rho, const DetectParams& P,
                                              float* out) {
  float d0[4], d1[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) { d0[j] = FLT_MAX; d1[j] = FLT_MAX; }
  for (int i = 0; i < P.M; ++i) {
    const float a = (float)(2 * i + 1 - P.M) * P.lvl_step;
    const float e = x - a;
    const float d = e * e;
    const int g = i ^ (i >> 1);  // Gray word of level i
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j < P.nb) {
        if ((g >> (P.nb - 1 - j)) & 1) d1[j] = fminf(d1[j], d);
        else d0[j] = fminf(d0[j], d);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (j < P.nb) out[j] = rho * (d0[j] - d1[j]);
}

// Soft output of one user (Section III-C): mu~ = p, rho~ = ||h||^2 Es / N0,
// LLRs of z / (mu~ sqrt(Es)) against the unit-energy alphabet.
__device__ __forceinline__ void user_llr(float2 z, float nrm, float p, const DetectParams& P,
                                         float* out) {
  if (!(p > 0.0f)) {
    for (int j = 0; j < P.Q; ++j) out[j] = 0.0f;
    return;
  }
  const float inv = 1.0f / (p * P.sqrt_es);
  const float rho = nrm * P.rho_scale;
  dimension_llr(z.x * inv, rho, P, out);
  if (!P.bpsk) dimension_llr(z.y * inv, rho, P, out + P.nb);
}

}  // namespace ocd
