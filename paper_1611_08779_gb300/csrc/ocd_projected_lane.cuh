// Projected OCD for one symbol per channel (T = 1), one lane per subcarrier.
//
// With T = 1 nothing amortizes the per-subcarrier products over symbols, and
// the work per subcarrier is small: G = H^H H (upper triangle) and
// q0 = H^H y take B (U(U+1)/2 + U) complex multiply-adds, the K sweeps of
// Algorithm 1 in the projected arrangement K U^2 more.  The kernel streams H
// and y once from HBM (the bound) and gives each lane a whole subcarrier, so
// no reduction across lanes is needed anywhere:
//
// * every warp is its own pipeline over groups of 32 consecutive
//   subcarriers (group w, w + W, ... for warp w of W); there is no barrier
//   between the warps of a CTA;
// * a step stages kAPC antennas of the 32 subcarriers of a group (H rows
//   [b0, b0 + kAPC) and the matching entries of y) with 16-byte cp.async
//   copies, the 8 or so lanes that copy one subcarrier's piece reading
//   consecutive global addresses; rows are padded to an odd multiple of 16
//   bytes, so that lane l reading its row l hits distinct banks;
// * lane l accumulates G and q0 of its subcarrier in registers (FP32,
//   antenna by antenna), then runs preprocessing, the K sweeps (Algorithm 1
//   with q = H^H r kept current by q <- q - G[:, u] dz), the projection of
//   Eq. 14 and the LLRs of Eq. 9 with the approximation of Section III-C.
//
// Needs float32 storage, even B, and 16-byte aligned H and Y.  The copies
// complete through cp.async.wait_group (no spin loop of the kernel's own).
#pragma once

#include "ocd_common.cuh"

namespace ocd {

#ifndef OCD_LANE_STAGES
#define OCD_LANE_STAGES 3  // staged steps per warp (two in flight while one is used)
#endif
#ifndef OCD_LANE_MIN_CTAS
#define OCD_LANE_MIN_CTAS 3  // resident CTAs per SM the register budget targets
#endif

template <int U>
struct LaneShape {
  // antennas per step: even (so every piece is a whole number of 16-byte
  // units), at most 16 complex entries of H per subcarrier
  static constexpr int kAPC = (16 / U) & ~1;
  static constexpr int kHBytes = kAPC * U * 8;  // H bytes per subcarrier and step
  static constexpr int kYBytes = kAPC * 8;      // y bytes per subcarrier and step
  static constexpr int odd16(int b) { return (b / 16) % 2 == 1 ? b : b + 16; }
  static constexpr int kHPitch = odd16(kHBytes);  // padded shared-memory rows
  static constexpr int kYPitch = odd16(kYBytes);
  static constexpr int kStageBytes = 32 * (kHPitch + kYPitch);
  static constexpr int kStages = OCD_LANE_STAGES;
  static constexpr int kWarpBytes = kStages * kStageBytes;
  static constexpr int kWarps = 4;
  static constexpr int kHPieces = kHBytes / 16;  // 16-byte pieces per subcarrier and step
  static constexpr int kYPieces = kYBytes / 16;
  static_assert(kAPC >= 2 && kHBytes % 16 == 0 && kYBytes % 16 == 0, "16-byte pieces");
  static_assert(kHPitch % 32 == 16 && kYPitch % 32 == 16, "odd multiples of 16 bytes");
  static_assert(kHBytes >= 16 * U, "a row holds z, ||h||^2 and p of every user");
};

__device__ __forceinline__ void lane_copy16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void lane_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void lane_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ uint32_t lane_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

template <int U>
__global__ void __launch_bounds__(128, OCD_LANE_MIN_CTAS) ocd_projected_lane_kernel(DetectParams P) {
  using S = LaneShape<U>;
  constexpr int APC = S::kAPC;
  extern __shared__ __align__(16) unsigned char lane_smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned char* ws = lane_smem_raw + warp * S::kWarpBytes;

  const int B = P.B;
  const long long Nsc = P.Nsc;
  const long long ngroups = (Nsc + 31) / 32;
  const long long W = (long long)gridDim.x * S::kWarps;
  const long long first = (long long)blockIdx.x * S::kWarps + warp;
  if (first >= ngroups) return;  // whole warp; no CTA-wide barrier follows
  pdl_wait();                      // launched by launch_serialized
  const int nchunk = (B + APC - 1) / APC;
  const long long nsteps = ((ngroups - 1 - first) / W + 1) * nchunk;

  // Copies of step (group g, chunk c) into stage buffer `buf`.  Piece p of
  // the group's H (y) block is piece p % kHPieces of subcarrier p / kHPieces;
  // pieces past the chunk's antennas (last chunk) or past Nsc are skipped.
  // When the pieces of a subcarrier divide 32 a lane copies the same piece j
  // of every (32 / pieces)-th subcarrier, so its offsets advance by constants.
  const int BU = B * U;
  auto issue = [&](long long g, int c, int buf) {
    unsigned char* hb = ws + buf * S::kStageBytes;
    unsigned char* yb = hb + 32 * S::kHPitch;
    const int b0 = c * APC;
    const int bb = min(APC, B - b0);
    const long long sc0 = g * 32;
    const int nsc = (int)min(32LL, Nsc - sc0);
    const int hvalid = bb * U / 2;  // 16-byte pieces of H per subcarrier (bb even)
    const int yvalid = bb / 2;
    const float2* hsrc = P.H + (sc0 * B + b0) * U;
    const float2* ysrc = P.Y + sc0 * B + b0;
    if constexpr (32 % S::kHPieces == 0) {
      constexpr int SPI = 32 / S::kHPieces;
      const int s0 = lane / S::kHPieces, j = lane % S::kHPieces;
      if (j < hvalid) {
#pragma unroll
        for (int i = 0; i < S::kHPieces; ++i) {
          const int sj = s0 + SPI * i;
          if (sj < nsc) lane_copy16(lane_smem(hb + sj * S::kHPitch + 16 * j), hsrc + sj * BU + 2 * j);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < S::kHPieces; ++i) {
        const int p = lane + 32 * i;
        const int sj = p / S::kHPieces, j = p - sj * S::kHPieces;
        if (sj < nsc && j < hvalid)
          lane_copy16(lane_smem(hb + sj * S::kHPitch + 16 * j), hsrc + sj * BU + 2 * j);
      }
    }
    static_assert(32 % S::kYPieces == 0, "y pieces per subcarrier divide 32");
    {
      constexpr int SPI = 32 / S::kYPieces;
      const int s0 = lane / S::kYPieces, j = lane % S::kYPieces;
      if (j < yvalid) {
#pragma unroll
        for (int i = 0; i < S::kYPieces; ++i) {
          const int sj = s0 + SPI * i;
          if (sj < nsc) lane_copy16(lane_smem(yb + sj * S::kYPitch + 16 * j), ysrc + sj * B + 2 * j);
        }
      }
    }
  };

  // G (upper triangle; the diagonal is real) and q0 of this lane's subcarrier
  float gr[U][U], gi[U][U], q0r[U], q0i[U];

  long long ig = first;  // next step to issue: group, chunk
  int ic = 0;
#pragma unroll
  for (int i = 0; i < S::kStages - 1; ++i) {
    if (i < nsteps) {
      issue(ig, ic, i);
      if (++ic == nchunk) { ic = 0; ig += W; }
    }
    lane_commit();
  }
  long long cg = first;  // step being computed
  int cc = 0;
  int buf = 0, ibuf = S::kStages - 1;
  for (long long s = 0; s < nsteps; ++s) {
    lane_wait<S::kStages - 2>();  // this lane's copies of step s have landed
    __syncwarp();                 // ... and every lane's; step s - 1 is consumed
    if (s + S::kStages - 1 < nsteps) {
      issue(ig, ic, ibuf);
      if (++ic == nchunk) { ic = 0; ig += W; }
    }
    lane_commit();
    ibuf = ibuf + 1 == S::kStages ? 0 : ibuf + 1;

    if (cc == 0) {
#pragma unroll
      for (int i = 0; i < U; ++i) {
        q0r[i] = 0.0f;
        q0i[i] = 0.0f;
#pragma unroll
        for (int j = i; j < U; ++j) { gr[i][j] = 0.0f; gi[i][j] = 0.0f; }
      }
    }
    const unsigned char* hrow = ws + buf * S::kStageBytes + lane * S::kHPitch;
    const unsigned char* yrow = ws + buf * S::kStageBytes + 32 * S::kHPitch + lane * S::kYPitch;
    const int b0 = cc * APC;
#pragma unroll
    for (int a = 0; a < APC; ++a) {
      if (b0 + a < B) {  // only the last chunk can be short
        float hr[U], hi[U];
        if constexpr (U % 2 == 0) {
#pragma unroll
          for (int v = 0; v < U / 2; ++v) {
            const float4 h2 = *reinterpret_cast<const float4*>(hrow + (a * U + 2 * v) * 8);
            hr[2 * v] = h2.x; hi[2 * v] = h2.y; hr[2 * v + 1] = h2.z; hi[2 * v + 1] = h2.w;
          }
        } else {
#pragma unroll
          for (int v = 0; v < U; ++v) {
            const float2 h1 = *reinterpret_cast<const float2*>(hrow + (a * U + v) * 8);
            hr[v] = h1.x; hi[v] = h1.y;
          }
        }
        const float2 y = *reinterpret_cast<const float2*>(yrow + a * 8);
#pragma unroll
        for (int i = 0; i < U; ++i) {
          // q0_i += conj(h_i) y
          q0r[i] = fmaf(hr[i], y.x, fmaf(hi[i], y.y, q0r[i]));
          q0i[i] = fmaf(hr[i], y.y, fmaf(-hi[i], y.x, q0i[i]));
          // G_ii += |h_i|^2
          gr[i][i] = fmaf(hr[i], hr[i], fmaf(hi[i], hi[i], gr[i][i]));
          // G_ij += conj(h_i) h_j, j > i
#pragma unroll
          for (int j = i + 1; j < U; ++j) {
            gr[i][j] = fmaf(hr[i], hr[j], fmaf(hi[i], hi[j], gr[i][j]));
            gi[i][j] = fmaf(hr[i], hi[j], fmaf(-hi[i], hr[j], gi[i][j]));
          }
        }
      }
    }

    if (cc == nchunk - 1) {
      const long long sc = cg * 32 + lane;
      if (sc < Nsc) {
        // preprocessing (Algorithm 1): n_u = G_uu, d_u^-1, p_u
        float dv[U], pv[U], qr[U], qi[U], zr[U], zi[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const float den = gr[u][u] + P.alpha;
          dv[u] = den > 0.0f ? 1.0f / den : 0.0f;
          pv[u] = dv[u] * gr[u][u];
          qr[u] = q0r[u];
          qi[u] = q0i[u];
          zr[u] = 0.0f;
          zi[u] = 0.0f;
        }
        for (int k = 0; k < P.K; ++k) {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            // z_u <- proj(d_u^-1 h_u^H r + p_u z_u), with h_u^H r = q_u
            float wr = fmaf(dv[u], qr[u], pv[u] * zr[u]);
            float wi = fmaf(dv[u], qi[u], pv[u] * zi[u]);
            project(wr, wi, P);
            const float dr = wr - zr[u], di = wi - zi[u];
            zr[u] = wr;
            zi[u] = wi;
            // q <- q - G[:, u] dz  (r <- r - h_u dz, Eq. 15, seen through H^H)
#pragma unroll
            for (int j = 0; j < U; ++j) {
              const float cr = j <= u ? gr[j][u] : gr[u][j];
              const float ci = j < u ? gi[j][u] : (j > u ? -gi[u][j] : 0.0f);
              qr[j] = fmaf(-cr, dr, fmaf(ci, di, qr[j]));
              qi[j] = fmaf(-cr, di, fmaf(-ci, dr, qi[j]));
            }
          }
        }
        if (P.xhat) {
#pragma unroll
          for (int u = 0; u < U; ++u) P.xhat[sc * U + u] = make_float2(zr[u], zi[u]);
        }
        if (P.llr) {
          // z, ||h_u||^2 and p_u go to this lane's own row of the consumed
          // stage buffer (rewritten only after the next __syncwarp), so that
          // one rolled loop over the users holds the only copy of the LLR code
          float4* zrow = reinterpret_cast<float4*>(ws + buf * S::kStageBytes + lane * S::kHPitch);
#pragma unroll
          for (int u = 0; u < U; ++u) zrow[u] = make_float4(zr[u], zi[u], gr[u][u], pv[u]);
#pragma unroll 1
          for (int u = 0; u < U; ++u) {
            const float4 v = zrow[u];
            user_llr(make_float2(v.x, v.y), v.z, v.w, P, P.llr + (sc * U + u) * P.Q);
          }
        }
      }
    }
    if (++cc == nchunk) { cc = 0; cg += W; }
    buf = buf + 1 == S::kStages ? 0 : buf + 1;
  }
  lane_wait<0>();
  pdl_trigger();
}

}  // namespace ocd
