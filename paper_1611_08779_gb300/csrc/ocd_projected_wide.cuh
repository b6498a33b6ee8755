// Projected-residual OCD for up to 32 users (four 8-user tiles), channel
// and received vectors staged by the bulk-copy (TMA) engine.  Same algebra
// as ocd_projected_tma.cuh (q = H^H r; q0 = H^H Y^T and G = H^H H once per
// subcarrier on the tensor cores, then the K sweeps on q), with the work of
// one subcarrier split into phases so that one warp's accumulators stay
// within the register file:
//
//   G phase  (one step per staged antenna block): only the channel block
//            is staged; the 10 tiles (m, n), n >= m, of G are accumulated.
//            At the last block G goes to shared memory (Hermitian fill) with
//            the preprocessing of Algorithm 1.
//   q0 pass p (one step per block, per 16 symbols): channel block and the
//            received rows; the 8 tiles of q0 (4 user tiles x 2 symbol
//            tiles) are accumulated in the same registers; at the last block
//            the K sweeps run on q and the outputs are written.
//   T <= 8:  no q0 pass; the G phase stages the received rows too and
//            accumulates the 4 q0 tiles of symbols 0-7 in 32 more registers
//            from the same split channel fragments (wide_walk<true>).
//
// Each accumulator tile keeps two parts, hi*hi and hi*lo + lo*hi of the
// three-term TF32 split, summed once per phase.  One warp per CTA (the
// per-warp staging, G and preprocessing areas take 21 KB of shared memory
// with 16-antenna blocks; q0 reuses the staging buffer of the step being
// finished); with T > 8 the channel block is read once per phase, the
// second time from L2.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; no driver library is linked)

#include <type_traits>

#include "ocd_batch.cuh"
#include "ocd_common.cuh"
#include "ocd_f32x2.cuh"
#include "ocd_mma.cuh"
#include "ocd_tma_util.cuh"

namespace ocd {

#ifndef OCD_WIDE_STAGES
#define OCD_WIDE_STAGES 2     // staging buffers per warp
#endif
#ifndef OCD_WIDE_MIN_CTAS
#define OCD_WIDE_MIN_CTAS 1  // resident CTAs (= warps) per SM the register budget targets
#endif
#ifndef OCD_WIDE_FUSE
#define OCD_WIDE_FUSE 1  // T <= 8: q0 accumulated in the G phase (no q0 pass)
#endif
#ifndef OCD_WIDE_F32X2
#define OCD_WIDE_F32X2 1  // sweeps on packed FP32 pairs of users
#endif
#ifndef OCD_WIDE_BLOCK
#define OCD_WIDE_BLOCK 16     // antennas per staged block (16 or 32)
#endif

struct WideShape {
  static constexpr int kUsers = 32;                         // user slots (4 MMA tiles)
  static constexpr int kPass = 16;                          // symbols per q0 pass
  static constexpr int kBB = OCD_WIDE_BLOCK;                // antennas per staged block
  static constexpr int kBoxAnt = 16;                        // antennas per Y box (128 B rows)
  static constexpr int kBoxBytes = kPass * 128;
  static constexpr int kBoxes = kBB / kBoxAnt;
  static constexpr int kYBytes = kBoxes * kBoxBytes;
  static constexpr int kHBytes = kBB * kUsers * 8;
  static constexpr int kBufBytes = kYBytes + kHBytes;       // multiple of 1024
  static constexpr int kStages = OCD_WIDE_STAGES;
  static constexpr int kUP = kUsers / 2;                    // users per sweep lane
  // q0, later z [pass symbol][u] lives in the staging buffer of the step
  // whose epilogue uses it: that buffer receives its next copy only when the
  // following step starts.  A symbol's row holds the 32 users' (re, im) in
  // kSqRow floats, users 16-31 four floats further on (see wide_sq).
  static constexpr int kSqRow = 2 * kUsers + 8;
  static constexpr int kQBytes = 4 * kPass * kSqRow;
  static_assert(kQBytes <= kBufBytes, "q0 fits in a staging buffer");
  static constexpr int kOffG = kStages * kBufBytes;         // G [i][j]
  // floats per G row: the real run, the imaginary run and 4 floats of pad,
  // so that consecutive rows start 16 bytes apart in bank position
  static constexpr int kGRow = 2 * kUsers + 4;
  static constexpr int kOffPre = kOffG + 4 * kUsers * kGRow;  // (d^-1, p, rho~ step^2, LLR level scale)
  static constexpr int kOffBar = kOffPre + 16 * kUsers;
  static constexpr int kWarpBytes = ((kOffBar + 8 * kStages + 1023) / 1024) * 1024;
  static constexpr int kThreads = 32;                       // one warp per CTA
  static_assert(kBufBytes % 1024 == 0, "swizzled boxes need 1024-byte alignment");
};

// G in shared memory, row i as [Re G_i0 .. Re G_i(NU-1) | Im G_i0 .. Im G_i(NU-1) | pad]:
// a sweep lane reads the real and the imaginary parts of its users as
// separate runs (16-byte aligned for 4 consecutive users).
__device__ __forceinline__ int wide_gre(int i, int j) { return i * WideShape::kGRow + j; }
__device__ __forceinline__ int wide_gim(int i, int j) {
  return i * WideShape::kGRow + WideShape::kUsers + j;
}
// Float index of Re q0 (or z) of symbol t, user u (Im follows): rows of
// kSqRow floats, users 16-31 shifted by four floats, so that the 32
// consecutive floats a sweep lane (2 ts + hf) reads start at bank
// 8 ts + 4 hf (mod 32): the lanes of a quarter warp read distinct banks.
__host__ __device__ constexpr int wide_sq(int t, int u) {
  return t * WideShape::kSqRow + 2 * u + (u >= 16 ? 4 : 0);
}
// Fault word of the wide kernels (bit 0: a wait timed out; bit 1: a batched
// cell's tensor map was misaligned).  Defined here because exactly one
// translation unit (ocd_projected_wide.cu) includes this header.
__device__ unsigned int g_wide_fault = 0;

// Index of G tile (m, n), n >= m, among the 10 upper tiles.
__host__ __device__ constexpr int wide_gtile(int m, int n) { return m * 4 - m * (m - 1) / 2 + (n - m); }

// Two-part split product d[0] += hi*hi, d[1] += hi*lo + lo*hi, issued in two
// rounds over all tiles of a k-step: round 1 (hi*hi, hi*lo) has no
// dependence between consecutive MMAs; round 2 (lo*hi) adds to the d[1] that
// round 1 updated several MMAs earlier, so no MMA waits on the one before.
__device__ __forceinline__ void mma2_round1(float (&d)[2][4], const uint32_t (&ah)[3],
                                            uint32_t bh0, uint32_t bh1, uint32_t bl0,
                                            uint32_t bl1) {
  mma_tf32(d[0], ah[0], ah[1], ah[2], bh0, bh1);
  mma_tf32(d[1], ah[0], ah[1], ah[2], bl0, bl1);
}
__device__ __forceinline__ void mma2_round2(float (&d)[2][4], const uint32_t (&al)[3],
                                            uint32_t bh0, uint32_t bh1) {
  mma_tf32(d[1], al[0], al[1], al[2], bh0, bh1);
}

// Outputs of symbols ts0 .. ts0 + ns - 1 of the pass starting at symbol tb of
// subcarrier sc (z in sq [symbol][user], soft-output constants in spre), one
// item per (symbol, user) and lane: a full set of 32 users splits the item
// index with a shift, and the LLR code is chosen once by the bits per real
// dimension (both dimensions' LLRs stored as float2 pairs when the array is
// 8-byte aligned).
__device__ __forceinline__ void wide_outputs(const DetectParams& P, const float* sq,
                                             const float* spre, long long sc, int tb, int ts0,
                                             int ns) {
  constexpr int NU = WideShape::kUsers;
  const int lane = threadIdx.x & 31;
  const int U = P.U;
  const int T = P.T;
  auto outputs = [&](auto nbc) {
    constexpr int NB = decltype(nbc)::value;
    const bool full = U == NU;
    const bool pairs = !P.bpsk && (reinterpret_cast<uintptr_t>(P.llr) & 7u) == 0;
    for (int f = lane; f < ns * U; f += 32) {
      const int ts = ts0 + (full ? f >> 5 : f / U);
      const int u = f - (ts - ts0) * U;
      const float2 z = *reinterpret_cast<const float2*>(sq + wide_sq(ts, u));
      const long long o = (sc * T + tb + ts) * U + u;
      if (P.xhat) P.xhat[o] = z;
      if (P.llr) {
        float* out = P.llr + o * P.Q;
        const float inv = spre[4 * u + 3];
        if (!(inv > 0.0f)) {
          for (int j = 0; j < P.Q; ++j) out[j] = 0.0f;
        } else {
          const float rs2 = spre[4 * u + 2];
          if (pairs) {
            float L[2 * NB];
            dimension_llr_nb<NB>(z.x * inv, rs2, L);
            dimension_llr_nb<NB>(z.y * inv, rs2, L + NB);
#pragma unroll
            for (int j = 0; j < 2 * NB; j += 2)
              *reinterpret_cast<float2*>(out + j) = make_float2(L[j], L[j + 1]);
          } else {
            dimension_llr_nb<NB>(z.x * inv, rs2, out);
            if (!P.bpsk) dimension_llr_nb<NB>(z.y * inv, rs2, out + NB);
          }
        }
      }
    }
  };
  switch (P.nb) {
    case 1: outputs(std::integral_constant<int, 1>{}); break;
    case 2: outputs(std::integral_constant<int, 2>{}); break;
    case 3: outputs(std::integral_constant<int, 3>{}); break;
    default: outputs(std::integral_constant<int, 4>{}); break;
  }
  __syncwarp();
}

// K sweeps on q (q0 in sq [symbol][user] on entry, z on exit) and the
// outputs of symbols tb .. tb + np - 1 of subcarrier sc, by one warp:
// lane = 2 ts + hf owns users [hf*16, hf*16 + 16) of symbol ts.  G is in sg
// (wide_gre / wide_gim rows), (d^-1, p, rho~ step^2, LLR level scale) per
// user in spre.  Shared by the warp-level and the tcgen05 32-user kernels.
// FULL_TILE: also compile the sweeps of a full user tile without per-user
// guards (faster, more registers: the tcgen05 kernel's 128-register budget
// takes the guarded form only).
template <bool FULL_TILE = true>
__device__ __forceinline__ void wide_sweeps_outputs(const DetectParams& P, float* sq,
                                                    const float* sg, const float* spre,
                                                    long long sc, int tb, int np) {
  constexpr int UP = WideShape::kUP;
  constexpr int NU = WideShape::kUsers;
  const int lane = threadIdx.x & 31;
  const int U = P.U;
  const int T = P.T;
#if OCD_WIDE_F32X2
  {
    // lane = 2 ts + hf holds users [hf*UP, hf*UP + UP) of symbol ts; q as
    // packed pairs of consecutive users, updated with fma.rn.f32x2 (each
    // half one IEEE fma: the same operations, in the same order, as the
    // scalar form)
    const int ts = lane >> 1;
    const int hf = lane & 1;
    const bool act = ts < np;
    unsigned long long QR[UP / 2], QI[UP / 2];
    float zr[UP], zi[UP];
    const float4* q4 = reinterpret_cast<const float4*>(sq + wide_sq(ts & 15, hf * UP));
#pragma unroll
    for (int l2 = 0; l2 < UP / 2; ++l2) {
      // users hf UP + 2 l2 and + 1: (re, im, re, im)
      const float4 v = act ? q4[l2] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      QR[l2] = f2_pack(v.x, v.z);
      QI[l2] = f2_pack(v.y, v.w);
      zr[2 * l2] = zr[2 * l2 + 1] = 0.0f;
      zi[2 * l2] = zi[2 * l2 + 1] = 0.0f;
    }
    const float are = P.box ? P.box_a : __int_as_float(0x7f800000);
    const float aim = P.box ? (P.bpsk ? 0.0f : P.box_a) : __int_as_float(0x7f800000);
    // a full user tile (U equal to the tile) needs no per-user guard: the
    // updates of all users form one block the scheduler can interleave
    auto sweeps = [&](auto fullc) {
      constexpr bool FULL = decltype(fullc)::value;
      for (int k = 0; k < P.K; ++k) {
#pragma unroll 1
        for (int oh = 0; oh < 2; ++oh) {
#pragma unroll
        for (int lu = 0; lu < UP; ++lu) {
          const int u = oh * UP + lu;
          if (FULL || u < U) {
            const float2 dp = *reinterpret_cast<const float2*>(spre + 4 * u);  // (d^-1, p)
            float q0, q1, p0, p1;
            f2_unpack(QR[lu >> 1], q0, q1);
            f2_unpack(QI[lu >> 1], p0, p1);
            const float qr = (lu & 1) ? q1 : q0;
            const float qi = (lu & 1) ? p1 : p0;
            float wr = fmaf(dp.x, qr, dp.y * zr[lu]);
            float wi = fmaf(dp.x, qi, dp.y * zi[lu]);
            wr = fminf(fmaxf(wr, -are), are);
            wi = fminf(fmaxf(wi, -aim), aim);
            const float dr0 = wr - zr[lu];
            const float di0 = wi - zi[lu];
            if (hf == oh) { zr[lu] = wr; zi[lu] = wi; }
            const int owner = (lane & ~1) | oh;
            const float dr = __shfl_sync(kFullMask, dr0, owner);
            const float di = __shfl_sync(kFullMask, di0, owner);
            const unsigned long long DR = f2_pack(dr, dr);
            const unsigned long long NDR = f2_pack(-dr, -dr);
            const unsigned long long NDI = f2_pack(-di, -di);
            const float4* gre = reinterpret_cast<const float4*>(sg + wide_gre(u, hf * UP));
            const float4* gim = reinterpret_cast<const float4*>(sg + wide_gim(u, hf * UP));
            if constexpr (FULL) {
              // a full tile first updates the pair that holds the next user
              // (the next update's input); every q keeps its own operations
              // and their order (the guarded form below measured faster in
              // the slot order of its loads)
              unsigned long long RE[UP / 2], IM[UP / 2];
#pragma unroll
              for (int l4 = 0; l4 < UP / 4; ++l4) {
                const float4 r4 = gre[l4], i4 = gim[l4];
                RE[2 * l4] = f2_pack(r4.x, r4.y);
                RE[2 * l4 + 1] = f2_pack(r4.z, r4.w);
                IM[2 * l4] = f2_pack(i4.x, i4.y);
                IM[2 * l4 + 1] = f2_pack(i4.z, i4.w);
              }
#pragma unroll
              for (int j = 0; j < UP / 2; ++j) {
                const int l2 = (((lu + 1) % UP) / 2 + j) % (UP / 2);
                // qr <- fma(-gx, dr, fma(-gy, di, qr)); qi <- fma(-gx, di, fma(gy, dr, qi))
                f2_fma(QR[l2], IM[l2], NDI);
                f2_fma(QR[l2], RE[l2], NDR);
                f2_fma(QI[l2], IM[l2], DR);
                f2_fma(QI[l2], RE[l2], NDI);
              }
            } else {
#pragma unroll
              for (int l4 = 0; l4 < UP / 4; ++l4) {
                const float4 r4 = gre[l4], i4 = gim[l4];
                const unsigned long long re0 = f2_pack(r4.x, r4.y), re1 = f2_pack(r4.z, r4.w);
                const unsigned long long im0 = f2_pack(i4.x, i4.y), im1 = f2_pack(i4.z, i4.w);
                // qr <- fma(-gx, dr, fma(-gy, di, qr)); qi <- fma(-gx, di, fma(gy, dr, qi))
                f2_fma(QR[2 * l4], im0, NDI);
                f2_fma(QR[2 * l4], re0, NDR);
                f2_fma(QI[2 * l4], im0, DR);
                f2_fma(QI[2 * l4], re0, NDI);
                f2_fma(QR[2 * l4 + 1], im1, NDI);
                f2_fma(QR[2 * l4 + 1], re1, NDR);
                f2_fma(QI[2 * l4 + 1], im1, DR);
                f2_fma(QI[2 * l4 + 1], re1, NDI);
              }
            }
          }
        }
        }
      }
    };
    if (FULL_TILE && U == NU) sweeps(std::integral_constant<bool, FULL_TILE>{});
    else sweeps(std::false_type{});
    __syncwarp();
    if (act) {
      float4* z4 = reinterpret_cast<float4*>(sq + wide_sq(ts, hf * UP));
#pragma unroll
      for (int l2 = 0; l2 < UP / 2; ++l2)
        z4[l2] = make_float4(zr[2 * l2], zi[2 * l2], zr[2 * l2 + 1], zi[2 * l2 + 1]);
    }
    __syncwarp();
  }
#else
  {
    // lane = 2 ts + hf holds users [hf*UP, hf*UP + UP) of symbol ts
    const int ts = lane >> 1;
    const int hf = lane & 1;
    const bool act = ts < np;
    float qr[UP], qi[UP], zr[UP], zi[UP];
#pragma unroll
    for (int l = 0; l < UP; ++l) {
      const int j = hf * UP + l;
      qr[l] = act ? sq[wide_sq(ts, j)] : 0.0f;
      qi[l] = act ? sq[wide_sq(ts, j) + 1] : 0.0f;
      zr[l] = 0.0f;
      zi[l] = 0.0f;
    }
    const float are = P.box ? P.box_a : __int_as_float(0x7f800000);
    const float aim = P.box ? (P.bpsk ? 0.0f : P.box_a) : __int_as_float(0x7f800000);
    for (int k = 0; k < P.K; ++k) {
      // users in two halves of UP (the owner half oh is a loop variable,
      // the slot lu a compile-time index): half the code of a full unroll
#pragma unroll 1
      for (int oh = 0; oh < 2; ++oh) {
#pragma unroll
      for (int lu = 0; lu < UP; ++lu) {
        const int u = oh * UP + lu;
        if (u < U) {
          const float2 dp = *reinterpret_cast<const float2*>(spre + 4 * u);  // (d^-1, p)
          float wr = fmaf(dp.x, qr[lu], dp.y * zr[lu]);
          float wi = fmaf(dp.x, qi[lu], dp.y * zi[lu]);
          wr = fminf(fmaxf(wr, -are), are);
          wi = fminf(fmaxf(wi, -aim), aim);
          const float dr0 = wr - zr[lu];
          const float di0 = wi - zi[lu];
          if (hf == oh) { zr[lu] = wr; zi[lu] = wi; }
          const int owner = (lane & ~1) | oh;
          const float dr = __shfl_sync(kFullMask, dr0, owner);
          const float di = __shfl_sync(kFullMask, di0, owner);
          const float4* gre = reinterpret_cast<const float4*>(sg + wide_gre(u, hf * UP));
          const float4* gim = reinterpret_cast<const float4*>(sg + wide_gim(u, hf * UP));
#pragma unroll
          for (int l4 = 0; l4 < UP / 4; ++l4) {
            const float4 r4 = gre[l4], i4 = gim[l4];
            const float gx[4] = {r4.x, r4.y, r4.z, r4.w}, gy[4] = {i4.x, i4.y, i4.z, i4.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int l = 4 * l4 + c;
              qr[l] = fmaf(-gx[c], dr, fmaf(-gy[c], di, qr[l]));
              qi[l] = fmaf(-gx[c], di, fmaf(gy[c], dr, qi[l]));
            }
          }
        }
      }
      }
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int l = 0; l < UP; ++l) {
        const int j = hf * UP + l;
        sq[wide_sq(ts, j)] = zr[l];
        sq[wide_sq(ts, j) + 1] = zi[l];
      }
    }
    __syncwarp();
  }
#endif
  wide_outputs(P, sq, spre, sc, tb, 0, np);
}

// One warp's walk over subcarriers first, first + stride, ... (< end) of
// problem P (ymap: Y as [Nsc*T][2B] floats, box 32 x 16, 128-byte swizzle).
// Staging area and barriers persist across calls as in tma_walk; returns
// false when a wait timed out.
template <bool FUSED>
__device__ __forceinline__ bool wide_walk(const DetectParams& P, const CUtensorMap* ymap,
                                          unsigned char* ws, uint32_t bar0, uint32_t& parity,
                                          long long first, long long end, long long stride) {
  using S = WideShape;
  constexpr int BB = S::kBB;
  constexpr int NU = S::kUsers;
  const int lane = threadIdx.x & 31;
  float* sg = reinterpret_cast<float*>(ws + S::kOffG);
  float* spre = reinterpret_cast<float*>(ws + S::kOffPre);

  const int U = P.U;
  const int B = P.B;
  const int T = P.T;
  const int gq = lane >> 2;
  const int t = lane & 3;
  // antenna order inside a k-step and swizzled Y offsets as in tma_walk
  const int ta = ((t >> 1) << 3) | (t & 1);
  int yoff[4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
    yoff[kk] = gq * 128 + (((kk | ((t >> 1) << 2)) ^ gq) << 4) + ((t & 1) << 3);
  const int nblk = (B + BB - 1) / BB;
  // FUSED (T <= 8, one n-tile of symbols): q0 is accumulated in the G phase
  // from the same channel fragments, and there is no separate q0 pass
  constexpr bool fused = FUSED;
  const int npasses = fused ? 0 : (T + S::kPass - 1) / S::kPass;
  const long long steps_per_sc = (long long)(npasses + 1) * nblk;
  const long long my_nsc = first < end ? (end - 1 - first) / stride + 1 : 0;
  const long long nsteps = my_nsc * steps_per_sc;
  if (nsteps == 0) return true;

  // Step cursor: (subcarrier, phase, block); phase 0 = G, phase p >= 1 =
  // q0 pass p - 1.
  struct Cursor {
    long long sc;
    int phase, blk;
  };
  auto advance = [&](Cursor& q) {
    if (++q.blk == nblk) {
      q.blk = 0;
      if (++q.phase == npasses + 1) {
        q.phase = 0;
        q.sc += stride;
      }
    }
  };
  auto issue = [&](const Cursor& q, int buf) {
    const int b0 = q.blk * BB;
    const int bb = min(BB, B - b0);
    const uint32_t bar = bar0 + 8 * buf;
    unsigned char* bp = ws + buf * S::kBufBytes;
    const int nbox = (q.phase == 0 && !fused) ? 0 : (bb + S::kBoxAnt - 1) / S::kBoxAnt;
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)(nbox * S::kBoxBytes + bb * U * 8));
    __syncwarp();
    fence_proxy_async();
    if (lane < nbox)
      tma_load_2d(smem_addr(bp + lane * S::kBoxBytes), ymap, 2 * (b0 + S::kBoxAnt * lane),
                  (int)(q.sc * T + (fused ? 0 : (q.phase - 1) * S::kPass)), bar);
    if (lane == 31) {
      const float2* src = P.H + (q.sc * (long long)B + b0) * U;
      bulk_g2s(smem_addr(bp + S::kYBytes), src, (uint32_t)(bb * U * 8), bar);
    }
  };

  // acc[i]: G tile i (G phase) or q0 tile 2m + n (q0 passes); rows 0-7 real
  // and 8-15 imaginary parts of user m*8 + gq.  qf[m]: q0 tile (m, 0) of the
  // fused G phase.
  float acc[10][2][4];
  float qf[4][2][4];

  Cursor cur{first, 0, 0};
  Cursor nxt{first, 0, 0};
  int buf = 0, ibuf = 0;
  for (int i = 0; i < S::kStages - 1 && i < nsteps; ++i) {
    issue(nxt, ibuf);
    advance(nxt);
    ibuf = ibuf + 1 == S::kStages ? 0 : ibuf + 1;
  }
  for (long long s = 0; s < nsteps; ++s) {
    if (s + S::kStages - 1 < nsteps) {
      issue(nxt, ibuf);
      advance(nxt);
      ibuf = ibuf + 1 == S::kStages ? 0 : ibuf + 1;
    }
    if (!mbar_wait(bar0 + 8 * buf, (parity >> buf) & 1, P.wait_ns)) {
      if (lane == 0) atomicOr(&g_wide_fault, 1u);
      for (int i = 1; i < S::kStages; ++i) {
        if (s + i < nsteps) {
          const int bi = (buf + i) % S::kStages;
          mbar_wait(bar0 + 8 * bi, (parity >> bi) & 1, P.wait_ns);
        }
      }
      return false;
    }
    parity ^= 1u << buf;

    const long long sc = cur.sc;
    const int phase = cur.phase;
    const int blk = cur.blk;
    const int bb = min(BB, B - blk * BB);
    const int tb = fused ? 0 : (phase - 1) * S::kPass;
    const int np = fused ? T : phase == 0 ? 0 : min(S::kPass, T - tb);
    const int this_buf = buf;
    advance(cur);
    buf = buf + 1 == S::kStages ? 0 : buf + 1;
    const unsigned char* bp = ws + this_buf * S::kBufBytes;
    const float2* sH = reinterpret_cast<const float2*>(bp + S::kYBytes);

    if (blk == 0) {
#pragma unroll
      for (int i = 0; i < 10; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[i][q][e] = 0.0f;
      if constexpr (FUSED) {
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) qf[m][q][e] = 0.0f;
      }
    }

    // ---------------- products on the tensor cores ------------------------
    // Lane (gq, t) holds h_{a_t, m*8+gq} of the four user tiles; antennas
    // past bb and users past U are masked to zero.
    const float2* hl = sH + ta * U + gq;
    const bool full = bb == BB && U == NU;
    auto split_h = [&](const float2 (&h)[4], uint32_t (&ah)[4][3], uint32_t (&al)[4][3]) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        split_tf32(h[m].x, ah[m][0], al[m][0]);  // a0 = a3 = Re h
        split_tf32(h[m].y, ah[m][2], al[m][2]);  // a2 = Im h
        ah[m][1] = ah[m][2] ^ 0x80000000u;       // a1 = -Im h
        al[m][1] = al[m][2] ^ 0x80000000u;
      }
    };
    auto load_h = [&](int a0, bool ok, float2 (&h)[4]) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const bool okm = full || (ok && m * 8 + gq < U);
        h[m] = okm ? hl[a0 * U + m * 8] : make_float2(0.0f, 0.0f);
      }
    };
    if (phase == 0) {
      for (int box = 0; box * S::kBoxAnt < bb; ++box) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const int a0 = box * S::kBoxAnt + 2 * kk;
          float2 h[4];
          load_h(a0, a0 + ta < bb, h);
          uint32_t ah[4][3], al[4][3];
          split_h(h, ah, al);
#pragma unroll
          for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int n = m; n < 4; ++n)
              mma2_round1(acc[wide_gtile(m, n)], ah[m], ah[n][0], ah[n][2], al[n][0], al[n][2]);
          // lo*hi only off the diagonal: a diagonal tile's lo*hi is the
          // conjugate transpose of its hi*lo (taken in the G epilogue)
#pragma unroll
          for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int n = m + 1; n < 4; ++n)
              mma2_round2(acc[wide_gtile(m, n)], al[m], ah[n][0], ah[n][2]);
          if constexpr (FUSED) {  // q0 of symbols 0-7 from the same fragments
            const float2 ya = *reinterpret_cast<const float2*>(bp + box * S::kBoxBytes + yoff[kk]);
            uint32_t bh0, bl0, bh1, bl1;
            split_tf32(ya.x, bh0, bl0);
            split_tf32(ya.y, bh1, bl1);
#pragma unroll
            for (int m = 0; m < 4; ++m) mma2_round1(qf[m], ah[m], bh0, bh1, bl0, bl1);
#pragma unroll
            for (int m = 0; m < 4; ++m) mma2_round2(qf[m], al[m], bh0, bh1);
          }
        }
      }
    } else {
      for (int box = 0; box * S::kBoxAnt < bb; ++box) {
        const unsigned char* yb = bp + box * S::kBoxBytes;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const int a0 = box * S::kBoxAnt + 2 * kk;
          float2 h[4];
          load_h(a0, a0 + ta < bb, h);
          uint32_t ah[4][3], al[4][3];
          split_h(h, ah, al);
          const float2 ya = *reinterpret_cast<const float2*>(yb + yoff[kk]);
          const float2 yc = *reinterpret_cast<const float2*>(yb + yoff[kk] + 8 * 128);
          uint32_t bh0, bl0, bh1, bl1, ch0, cl0, ch1, cl1;
          split_tf32(ya.x, bh0, bl0);
          split_tf32(ya.y, bh1, bl1);
          split_tf32(yc.x, ch0, cl0);
          split_tf32(yc.y, ch1, cl1);
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            mma2_round1(acc[2 * m], ah[m], bh0, bh1, bl0, bl1);
            mma2_round1(acc[2 * m + 1], ah[m], ch0, ch1, cl0, cl1);
          }
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            mma2_round2(acc[2 * m], al[m], bh0, bh1);
            mma2_round2(acc[2 * m + 1], al[m], ch0, ch1);
          }
        }
      }
    }
    __syncwarp();
    if (blk != nblk - 1) continue;

    if (phase == 0) {
      // ---------------- G epilogue: Hermitian fill and preprocessing ------
      // diagonal tiles: lo*hi[i][j] = conj(hi*lo[j][i]), read back from G's
      // buffer after the hi*lo parts are written there
      float lhr[4][2], lhi[4][2];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float (&a)[2][4] = acc[wide_gtile(m, m)];
          const int i = m * 8 + gq, j = m * 8 + 2 * t + e;
          sg[wide_gre(i, j)] = a[1][e];
          sg[wide_gim(i, j)] = a[1][2 + e];
        }
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int i = m * 8 + gq, j = m * 8 + 2 * t + e;
          lhr[m][e] = sg[wide_gre(j, i)];
          lhi[m][e] = -sg[wide_gim(j, i)];
        }
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int n = m; n < 4; ++n)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float (&a)[2][4] = acc[wide_gtile(m, n)];
            const float re = (n == m ? a[1][e] + lhr[m][e] : a[1][e]) + a[0][e];
            const float im = (n == m ? a[1][2 + e] + lhi[m][e] : a[1][2 + e]) + a[0][2 + e];
            const int i = m * 8 + gq, j = n * 8 + 2 * t + e;
            sg[wide_gre(i, j)] = re;
            sg[wide_gim(i, j)] = im;
            if (n != m) {
              sg[wide_gre(j, i)] = re;
              sg[wide_gim(j, i)] = -im;
            }
          }
      __syncwarp();
      {
        const float nrm = sg[wide_gre(lane, lane)];
        const float den = nrm + P.alpha;
        const float dinv = (lane < U && den > 0.0f) ? 1.0f / den : 0.0f;
        const float p = dinv * nrm;
        spre[4 * lane] = dinv;
        spre[4 * lane + 1] = p;
        spre[4 * lane + 2] = llr_rs2(nrm, P);  // rho~ step^2
        spre[4 * lane + 3] = llr_u_scale(p, P);  // level units per unit of z
        sg[wide_gim(lane, lane)] = 0.0f;  // G_uu is real
      }
      __syncwarp();
      if constexpr (!FUSED) {
        continue;
      } else {
        // the q0 tiles of symbols 0-7 take the slots the epilogue below
        // reads (tiles 2m; tiles 2m + 1 only reach symbols >= T)
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[2 * m][q][e] = qf[m][q][e];
      }
    }

    // ---------------- q0 epilogue, sweeps, outputs ------------------------
    // this step's staging buffer is consumed (the products above are done)
    float* sq = reinterpret_cast<float*>(ws + this_buf * S::kBufBytes);
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int ts = 8 * n + 2 * t + e;
          const int u = m * 8 + gq;
          const float (&a)[2][4] = acc[2 * m + n];
          sq[wide_sq(ts, u)] = a[1][e] + a[0][e];
          sq[wide_sq(ts, u) + 1] = a[1][2 + e] + a[0][2 + e];
        }
    __syncwarp();
    wide_sweeps_outputs(P, sq, sg, spre, sc, tb, np);
  }
  return true;
}

// Single problem: warp (= CTA) b takes subcarriers b, b + gridDim.x, ...
__global__ void __launch_bounds__(32, OCD_WIDE_MIN_CTAS)
ocd_projected_wide_kernel(const __grid_constant__ DetectParams P,
                          const __grid_constant__ CUtensorMap ymap) {
  using S = WideShape;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  unsigned char* ws = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const uint32_t bar0 = smem_addr(ws + S::kOffBar);
  const long long gw = blockIdx.x;
  if (gw >= P.Nsc) return;
  if (lane == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ymap)) : "memory");
    for (int i = 0; i < S::kStages; ++i) mbar_init(bar0 + 8 * i, 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t parity = 0;
  pdl_wait();  // launched by launch_serialized
  if (OCD_WIDE_FUSE && P.T <= 8)
    wide_walk<true>(P, &ymap, ws, bar0, parity, gw, P.Nsc, gridDim.x);
  else
    wide_walk<false>(P, &ymap, ws, bar0, parity, gw, P.Nsc, gridDim.x);
  pdl_trigger();
}

// Several problems: each warp draws tickets (runs of subcarriers of one
// cell) from a device counter, as ocd_batched_tma_kernel.
// FUSED: every cell of the launch has T <= 8 (the planner groups cells by it).
template <bool FUSED>
__global__ void __launch_bounds__(32, OCD_WIDE_MIN_CTAS)
ocd_batched_wide_kernel(const __grid_constant__ BatchTable tab, unsigned int* __restrict__ tickets) {
  using S = WideShape;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  unsigned char* ws = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const uint32_t bar0 = smem_addr(ws + S::kOffBar);
  if (lane == 0) {
    for (int i = 0; i < S::kStages; ++i) mbar_init(bar0 + 8 * i, 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t parity = 0;
  int c = 0, prefetched = -1;
  for (;;) {
    unsigned int tk = 0;
    if (lane == 0) tk = atomicAdd(tickets, 1u);
    tk = __shfl_sync(kFullMask, tk, 0);
    if (tk >= tab.total) return;
    while (tk >= tab.cell[c].tick_end) ++c;
    const BatchCell& C = tab.cell[c];
    if (c != prefetched) {
      if (reinterpret_cast<uintptr_t>(&C.ymap) & 63u) {
        if (lane == 0) atomicOr(&g_wide_fault, 2u);
        return;
      }
      if (lane == 0)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&C.ymap)) : "memory");
      prefetched = c;
    }
    const long long t0 = c ? tab.cell[c - 1].tick_end : 0;
    const long long lo = ((long long)tk - t0) * C.sc_per_tick;
    const long long hi = min(lo + (long long)C.sc_per_tick, (long long)C.P.Nsc);
    if (!wide_walk<FUSED>(C.P, &C.ymap, ws, bar0, parity, lo, hi, 1)) return;
  }
}

}  // namespace ocd
