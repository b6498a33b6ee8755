// OCD in the residual form of Algorithm 1, FP32 on the CUDA cores.
//
// Work unit ("item"): one (subcarrier w, OFDM symbol t) pair.  A team of L
// lanes (L a power of two, inside one warp) owns one item: lane l holds the
// residual entries of antenna pairs {l, l+L, l+2L, ...} (NPP pairs, 2*NPP
// antennas) in registers for the whole item, so r never leaves the register
// file between the K sweeps.
//
// A CTA walks over chunks of `chunk` consecutive items (one per team).  The
// channel columns of every subcarrier the chunk touches are staged once into
// shared memory, user-major (h_u contiguous, zero-padded to 2*L*NPP antennas),
// together with the preprocessing of Algorithm 1 (||h_u||^2, d_u^-1, p_u).
// All T symbols of a subcarrier, and all K sweeps, reuse that copy.
//
// Per (sweep k, user u) a team computes the length-B inner product h_u^H r
// (lane-partial FMAs, then an xor-butterfly over the L lanes, which leaves a
// bit-identical sum on every lane), the scalar update with projection
// (Algorithm 1 update line, Eq. 14) redundantly on every lane, and the rank-1
// residual update r <- r - h_u dz (Eq. 15 kept incrementally).
#pragma once

#include "ocd_common.cuh"

namespace ocd {

template <int UMAX, int NPP>
__global__ void __launch_bounds__(128)
ocd_residual_kernel(const DetectParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sH = reinterpret_cast<float2*>(smem_raw);
  float* s_nrm = reinterpret_cast<float*>(sH + (size_t)P.scmax * P.sc_stride);
  float* s_dinv = s_nrm + P.scmax * kUserSlots;
  float* s_p = s_dinv + P.scmax * kUserSlots;

  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nwarps = nt >> 5;
  const int L = P.L;
  const int lt = tid & (L - 1);
  const int team = tid >> P.logL;
  const int BU = P.B * P.U;

  // Antennas B..2*L*NPP-1 of every staged column stay zero for the whole
  // kernel: the staging loop below only ever writes antennas < B.
  for (int i = tid; i < P.scmax * P.sc_stride; i += nt) sH[i] = make_float2(0.0f, 0.0f);

  const long long nchunks = (P.items + P.chunk - 1) / P.chunk;
  for (long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const long long i0 = c * P.chunk;
    const long long i1 = min(i0 + (long long)P.chunk, P.items);
    const long long sc0 = i0 / P.T;
    const int nsc = (int)((i1 - 1) / P.T - sc0 + 1);

    __syncthreads();  // the previous chunk is no longer being read
    // ---- stage H[sc0 .. sc0+nsc) transposed to user-major rows ------------
    {
      const float2* gH = P.H + sc0 * (long long)BU;
      const int tot = nsc * BU;
      for (int e = tid; e < tot; e += nt) {
        const int s = e / BU;
        const int rem = e - s * BU;
        const int b = rem / P.U;
        const int u = rem - b * P.U;
        sH[s * P.sc_stride + u * P.rs + b] = __ldg(gH + e);
      }
    }
    __syncthreads();
    // ---- preprocessing (Algorithm 1): ||h_u||^2, d_u^-1, p_u ---------------
    for (int q = warp; q < nsc * P.U; q += nwarps) {
      const int s = q / P.U;
      const int u = q - s * P.U;
      const float2* row = sH + s * P.sc_stride + u * P.rs;
      float acc = 0.0f;
      for (int b = lane; b < P.B; b += 32) {
        const float2 h = row[b];
        acc = fmaf(h.x, h.x, fmaf(h.y, h.y, acc));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFullMask, acc, o);
      if (lane == 0) {
        const float den = acc + P.alpha;
        const float dinv = den > 0.0f ? 1.0f / den : 0.0f;
        s_nrm[s * kUserSlots + u] = acc;
        s_dinv[s * kUserSlots + u] = dinv;
        s_p[s * kUserSlots + u] = dinv * acc;
      }
    }
    __syncthreads();

    // ---- one item per team ---------------------------------------------------
    const long long it = i0 + team;
    const bool active = it < i1;  // uniform across the team
    const int sl = active ? (int)(it / P.T - sc0) : 0;

    // r = y (Algorithm 1 initialization); Y row of item `it` starts at it*B.
    float4 r[NPP];
    {
      const float2* yrow = P.Y + (active ? it : 0) * (long long)P.B;
#pragma unroll
      for (int j = 0; j < NPP; ++j) {
        const int pidx = lt + j * L;
        const int b0 = 2 * pidx;
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (active) {
          if (P.vec_y) {
            if (b0 < P.B) v = __ldg(reinterpret_cast<const float4*>(yrow) + pidx);
          } else {
            if (b0 < P.B) { const float2 a = __ldg(yrow + b0); v.x = a.x; v.y = a.y; }
            if (b0 + 1 < P.B) { const float2 a = __ldg(yrow + b0 + 1); v.z = a.x; v.w = a.y; }
          }
        }
        r[j] = v;
      }
    }

    float2 z[UMAX];
#pragma unroll
    for (int u = 0; u < UMAX; ++u) z[u] = make_float2(0.0f, 0.0f);

    const float2* hsc = sH + sl * P.sc_stride;
    const float* dinv_s = s_dinv + sl * kUserSlots;
    const float* p_s = s_p + sl * kUserSlots;

    for (int k = 0; k < P.K; ++k) {
#pragma unroll
      for (int u = 0; u < UMAX; ++u) {
        if (u < P.U) {
          const float4* hrow = reinterpret_cast<const float4*>(hsc + u * P.rs);
          float4 h[NPP];
          float ar0 = 0.0f, ai0 = 0.0f, ar1 = 0.0f, ai1 = 0.0f;
#pragma unroll
          for (int j = 0; j < NPP; ++j) {
            h[j] = hrow[lt + j * L];
            // conj(h) * r for the two antennas of the pair
            ar0 = fmaf(h[j].x, r[j].x, ar0);
            ar0 = fmaf(h[j].y, r[j].y, ar0);
            ai0 = fmaf(h[j].x, r[j].y, ai0);
            ai0 = fmaf(-h[j].y, r[j].x, ai0);
            ar1 = fmaf(h[j].z, r[j].z, ar1);
            ar1 = fmaf(h[j].w, r[j].w, ar1);
            ai1 = fmaf(h[j].z, r[j].w, ai1);
            ai1 = fmaf(-h[j].w, r[j].z, ai1);
          }
          float cr = ar0 + ar1;
          float ci = ai0 + ai1;
          for (int o = 1; o < L; o <<= 1) {
            cr += __shfl_xor_sync(kFullMask, cr, o);
            ci += __shfl_xor_sync(kFullMask, ci, o);
          }
          // z_u <- proj(d_u^-1 h_u^H r + p_u z_u); dz = z_new - z_old
          const float dv = dinv_s[u];
          const float pv = p_s[u];
          float wr = fmaf(dv, cr, pv * z[u].x);
          float wi = fmaf(dv, ci, pv * z[u].y);
          project(wr, wi, P);
          const float dr = wr - z[u].x;
          const float di = wi - z[u].y;
          z[u] = make_float2(wr, wi);
          // r <- r - h_u dz
#pragma unroll
          for (int j = 0; j < NPP; ++j) {
            r[j].x = fmaf(-h[j].x, dr, fmaf(h[j].y, di, r[j].x));
            r[j].y = fmaf(-h[j].x, di, fmaf(-h[j].y, dr, r[j].y));
            r[j].z = fmaf(-h[j].z, dr, fmaf(h[j].w, di, r[j].z));
            r[j].w = fmaf(-h[j].z, di, fmaf(-h[j].w, dr, r[j].w));
          }
        }
      }
    }

    // ---- outputs: users are spread over the team's lanes -------------------
    if (active) {
      const float* nrm_s = s_nrm + sl * kUserSlots;
#pragma unroll
      for (int u = 0; u < UMAX; ++u) {
        if (u < P.U && (u & (L - 1)) == lt) {
          if (P.xhat) P.xhat[it * P.U + u] = z[u];
          if (P.llr) user_llr(z[u], nrm_s[u], p_s[u], P, P.llr + (it * P.U + u) * P.Q);
        }
      }
    }
  }
}

}  // namespace ocd
