// Projected-residual OCD (q = H^H r, see ocd_projected.cuh for the algebra)
// with the channel and the received vectors streamed into shared memory by
// the bulk-copy (TMA) engine.
//
// One warp owns one subcarrier at a time and walks a sequence of steps:
// for each subcarrier, for each pass of kPass symbols, for each block of BB
// antennas.  Each step's operands -- the BB channel rows H[b0 .. b0+BB)[:]
// (one contiguous bulk copy) and the pass's received rows restricted to the
// block (one 2-D tensor copy per 16 antennas x 16 symbols, 128-byte
// swizzled) -- land in one of kStages per-warp buffers; the copies of the
// next kStages - 1 steps are in flight while a step is computed.  Completion is
// tracked with one mbarrier per buffer; every wait has an iteration limit,
// after which the warp records a fault in device memory and leaves.
//
//   Products (per step): q0 = H^H Y^T for the pass's 16 symbols and G = H^H H
//     (first pass only) on the tensor cores, as real m16n8k8 TF32 MMAs over
//     the realified K = 2B dimension with the three-term TF32 split, which
//     keeps FP32-level accuracy.  A holds [Re H^H; Im H^H] for the 8 user
//     slots; B is a staged received row (interleaved re/im is exactly the
//     K layout) or, for G, the same channel entries that form A.  A
//     diagonal G tile runs two of the three split products: its lo*hi term
//     is the conjugate transpose of its hi*lo term (products of TF32 values
//     are exact and both sums run over the same k order, so the transposed
//     entry is bit for bit the sum an MMA would give).
//   Epilogue (last block of a pass): the accumulator fragments go to shared
//     memory; the first pass also derives ||h_u||^2 = G_uu, d_u^-1, p_u and
//     the soft-output constants; the K sweeps run with two lanes per symbol;
//     then the LLRs and xhat are written.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; no driver library is linked)

#include <type_traits>

#include "ocd_batch.cuh"
#include "ocd_common.cuh"
#include "ocd_mma.cuh"
#include "ocd_tma_util.cuh"

namespace ocd {

// Per-warp geometry of the bulk-copy kernel (users padded to 8: the MMA tile
// has 16 rows = real and imaginary parts of 8 users).
#ifndef OCD_TMA_BLOCK
#define OCD_TMA_BLOCK 32      // antennas per staged block
#endif
#ifndef OCD_TMA_MIN_CTAS
#define OCD_TMA_MIN_CTAS 3    // resident CTAs per SM the register budget targets
#endif
#ifndef OCD_TMA_STAGES
#define OCD_TMA_STAGES 2      // staging buffers per warp (steps in flight + 1)
#endif
#ifndef OCD_TMA_WARPS
#define OCD_TMA_WARPS 4       // warps per CTA
#endif
#ifndef OCD_TMA_OUT_FAST
#define OCD_TMA_OUT_FAST 1    // output loop without a division, LLR code chosen per pass
#endif
#ifndef OCD_TMA_SKIP_N1
#define OCD_TMA_SKIP_N1 1     // passes of <= 8 symbols skip the second n-tile
#endif
#ifndef OCD_TMA_PARTS
#define OCD_TMA_PARTS 3       // accumulator parts per tile: 3 (hh, hl, lh) or 2 (hh, hl + lh)
#endif

// Users are padded to 8 * UT: an MMA tile has 16 rows = real and imaginary
// parts of 8 users, and UT user tiles (1 or 2) cover up to 16 users.
template <int UT>
struct TmaShape {
  static constexpr int kUsers = 8 * UT;                     // user slots
  static constexpr int kPass = 16;                          // symbols per pass (2 MMA n-tiles)
  static constexpr int kBB = OCD_TMA_BLOCK;                 // antennas per staged block
  static constexpr int kBoxAnt = 16;                        // antennas per Y box (128 B rows)
  static constexpr int kBoxBytes = kPass * 128;             // one swizzled Y box
  static constexpr int kBoxes = kBB / kBoxAnt;              // Y boxes per block
  static constexpr int kYBytes = kBoxes * kBoxBytes;
  static constexpr int kHBytes = kBB * kUsers * 8;          // staged H block (bytes)
  static constexpr int kBufBytes = kYBytes + kHBytes;       // multiple of 1024
  static constexpr int kStages = OCD_TMA_STAGES;
  static constexpr int kHalves = 2;                         // sweep lanes per symbol
  static constexpr int kUP = kUsers / kHalves;              // users per sweep lane
  // per-warp byte offsets (the warp area is 1024-byte aligned for the swizzle)
  static constexpr int kOffQ = kStages * kBufBytes;         // q0, later z [pass symbol][u]
  static constexpr int kOffG = kOffQ + 4 * kPass * SqLayout<kUsers>::kRow;  // full G [i][j]
  static constexpr int kOffPre = kOffG + 8 * kUsers * kUsers;  // (d^-1, p, rho~ step^2, LLR level scale)
  static constexpr int kOffBar = kOffPre + 16 * kUsers;     // one mbarrier per buffer
  static constexpr int kWarpBytes = ((kOffBar + 8 * kStages + 1023) / 1024) * 1024;
  static_assert(kBB % kBoxAnt == 0, "blocks are whole Y boxes");
  static_assert(kBufBytes % 1024 == 0, "swizzled boxes need 1024-byte alignment");
};

// G in shared memory, row i as [Re G_i0 .. Re G_i(NU-1) | Im G_i0 .. Im G_i(NU-1)]:
// a sweep lane reads the real and the imaginary parts of its users as
// separate 16-byte aligned runs.
template <int NU>
__device__ __forceinline__ int tma_gre(int i, int j) { return i * 2 * NU + j; }
template <int NU>
__device__ __forceinline__ int tma_gim(int i, int j) { return i * 2 * NU + NU + j; }

// Fault word of the bulk-copy kernels (bit 0: a wait timed out).  Defined
// here because exactly one translation unit (ocd_projected_tma.cu) includes
// this header; the host reads it through projected_tma_fault().
__device__ unsigned int g_tma_fault = 0;

// One warp's walk over the subcarriers first, first + stride, ... (< end) of
// one problem P whose received rows are described by ymap (Y viewed as a 2-D
// float tensor [Nsc*T rows][2B floats], box 32 x 16 = 16 antennas x 16
// symbols, 128-byte swizzle, out-of-range elements zero).  The warp's
// staging area ws and its barriers (bar0; phase bits in `parity`) outlive the
// call: every copy issued here is also waited for here, so consecutive calls
// may walk different problems.  Returns false when a wait timed out (the
// fault word is set and the warp must leave).
template <int UT>
__device__ __forceinline__ bool tma_walk(const DetectParams& P, const CUtensorMap* ymap,
                                         unsigned char* ws, uint32_t bar0, uint32_t& parity,
                                         long long first, long long end, long long stride) {
  using S = TmaShape<UT>;
  constexpr int BB = S::kBB;
  constexpr int UP = S::kUP;
  constexpr int NU = S::kUsers;
  const int lane = threadIdx.x & 31;
  float* sq = reinterpret_cast<float*>(ws + S::kOffQ);
  float* sg = reinterpret_cast<float*>(ws + S::kOffG);
  float* spre = reinterpret_cast<float*>(ws + S::kOffPre);

  const int U = P.U;
  const int B = P.B;
  const int T = P.T;
  // MMA fragment coordinates: row group gq (user / symbol within a tile), thread t
  const int gq = lane >> 2;
  const int t = lane & 3;
  // Antenna order inside a k-step: {0, 1, 8, 9}[t] + 2 kk (kk = 0..3 within a
  // 16-antenna box).  Byte offset of this lane's entry in the swizzled box,
  // row gq (row gq + 8 is 1024 bytes further and has the same swizzle):
  // chunk (kk | 4 (t >> 1)) lands at chunk ^ gq, half (t & 1).
  const int ta = ((t >> 1) << 3) | (t & 1);
  int yoff[4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
    yoff[kk] = gq * 128 + (((kk | ((t >> 1) << 2)) ^ gq) << 4) + ((t & 1) << 3);
  const int nblk = (B + BB - 1) / BB;
  const int npasses = (T + S::kPass - 1) / S::kPass;
  const long long steps_per_sc = (long long)npasses * nblk;
  const long long my_nsc = first < end ? (end - 1 - first) / stride + 1 : 0;
  const long long nsteps = my_nsc * steps_per_sc;
  if (nsteps == 0) return true;

  // Step cursor: (subcarrier, pass, block) advanced incrementally, so no
  // step needs an integer division.
  struct Cursor {
    long long sc;
    int pass, blk;
  };
  auto advance = [&](Cursor& q) {
    if (++q.blk == nblk) {
      q.blk = 0;
      if (++q.pass == npasses) {
        q.pass = 0;
        q.sc += stride;
      }
    }
  };

  // Issue the copies of the step at cursor q into buffer `buf`.
  auto issue = [&](const Cursor& q, int buf) {
    const int b0 = q.blk * BB;
    const int bb = min(BB, B - b0);
    const int tb = q.pass * S::kPass;
    const uint32_t bar = bar0 + 8 * buf;
    unsigned char* bp = ws + buf * S::kBufBytes;
    const int nbox = (bb + S::kBoxAnt - 1) / S::kBoxAnt;
    // the 3-D view fetches the block's two 16-antenna chunks in one copy (a
    // chunk past B arrives as zeros and still counts)
    const uint32_t ybytes = P.ymap3d ? (uint32_t)S::kYBytes : (uint32_t)(nbox * S::kBoxBytes);
    if (lane == 0) mbar_expect_tx(bar, ybytes + (uint32_t)(bb * U * 8));
    __syncwarp();
    fence_proxy_async();
    if (P.ymap3d) {
      if (lane == 0) tma_load_3d(smem_addr(bp), ymap, 0, (int)(q.sc * T + tb), b0 / S::kBoxAnt, bar);
    } else if (lane < nbox) {
      tma_load_2d(smem_addr(bp + lane * S::kBoxBytes), ymap, 2 * (b0 + S::kBoxAnt * lane),
                  (int)(q.sc * T + tb), bar);
    }
    if (lane == 31) {
      const float2* src = P.H + (q.sc * (long long)B + b0) * U;
      bulk_g2s(smem_addr(bp + S::kYBytes), src, (uint32_t)(bb * U * 8), bar);
    }
  };

  // Accumulator tiles, each with its three split-product parts: q0 for user
  // tile m and symbols 0-7 / 8-15 of the pass; G tiles (m, n), n >= m, in the
  // order (0,0), (0,1), (1,1).  Rows 0-7 hold real parts and rows 8-15
  // imaginary parts of user m*8 + gq.
  constexpr int NG = UT == 1 ? 1 : 3;
  constexpr int NQ = OCD_TMA_PARTS;
  static_assert(NQ == 2 || NQ == 3, "two or three accumulator parts");
  float qacc[UT][2][NQ][4];
  float gacc[NG][NQ][4];

  // prologue: the first kStages - 1 steps in flight
  Cursor cur{first, 0, 0};   // step being computed
  Cursor nxt{first, 0, 0};   // next step to issue
  int buf = 0, ibuf = 0;  // buffer of the current step, of the next issue
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
      if (lane == 0) atomicOr(&g_tma_fault, 1u);
      // let the copies already in flight finish (bounded) before leaving
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
    const int pass = cur.pass;
    const int blk = cur.blk;
    const int b0 = blk * BB;
    const int bb = min(BB, B - b0);
    const int tb = pass * S::kPass;
    const int np = min(S::kPass, T - tb);
    const bool first = pass == 0;
    const int this_buf = buf;
    advance(cur);
    buf = buf + 1 == S::kStages ? 0 : buf + 1;
    const unsigned char* bp = ws + this_buf * S::kBufBytes;
    const float2* sH = reinterpret_cast<const float2*>(bp + S::kYBytes);

    if (blk == 0) {
#pragma unroll
      for (int m = 0; m < UT; ++m)
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
          for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) qacc[m][n][q][e] = 0.0f;
#pragma unroll
      for (int n = 0; n < NG; ++n)
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
          for (int e = 0; e < 4; ++e) gacc[n][q][e] = 0.0f;
    }

    // ---------------- products on the tensor cores ------------------------
    // A k-step covers 4 antennas a_j = base + kb + {0, 1, 8, 9}[j] of a
    // 16-antenna box (kb = 0, 2, 4, 6); realified K index j (0..3) is the
    // real part of antenna a_j and 4 + j its imaginary part.
    // A = [Re H^H; Im H^H] over the 8 user slots:
    //   A[u][j] = Re h_{a_j,u}    A[u][4+j] = Im h_{a_j,u}
    //   A[8+u][j] = -Im h_{a_j,u}   A[8+u][4+j] = Re h_{a_j,u}
    // so A x (x = [Re x_a, Im x_a]) gives Re and Im of h_u^H x.  Lane (gq, t)
    // loads h_{a_t,gq} once: a0 = Re, a2 = Im, a3 = Re, a1 = -Im; its B
    // entries of received row n are Re and Im of y_{n,a_t}, read from the
    // swizzled box (16-byte chunk c of row r sits at chunk c ^ (r & 7)); the
    // antenna order {0, 1, 8, 9} puts the 16 lanes of a half-warp on 16
    // distinct bank slots.  Rows of A beyond U and columns beyond the pass's
    // symbols only reach discarded outputs; antennas beyond B arrive as zeros
    // from the tensor copy, and staged channel rows beyond the block are
    // masked.
    // One k-step: this lane's channel entries h[m] (user m*8 + gq) and the two
    // received values.
    const bool mask_u = U < NU;  // last user tile only partly used
    // two_n: the pass has more than 8 symbols, so the second n-tile of
    // received rows (symbols 8-15) is multiplied too
    auto kstep = [&](const float2 (&h)[UT], const float2 ya, const float2 yc, auto with_g,
                     auto two_n) {
      constexpr bool TWO_N = decltype(two_n)::value;
      uint32_t ah[UT][3], al[UT][3];
#pragma unroll
      for (int m = 0; m < UT; ++m) {
        split_tf32(h[m].x, ah[m][0], al[m][0]);  // a0 = a3 = Re h
        split_tf32(h[m].y, ah[m][2], al[m][2]);  // a2 = Im h
        ah[m][1] = ah[m][2] ^ 0x80000000u;       // a1 = -Im h
        al[m][1] = al[m][2] ^ 0x80000000u;
      }
      uint32_t bh0, bl0, bh1, bl1, ch0 = 0, cl0 = 0, ch1 = 0, cl1 = 0;
      split_tf32(ya.x, bh0, bl0);
      split_tf32(ya.y, bh1, bl1);
      if constexpr (TWO_N) {
        split_tf32(yc.x, ch0, cl0);
        split_tf32(yc.y, ch1, cl1);
      }
      if constexpr (NQ == 3) {
#pragma unroll
        for (int m = 0; m < UT; ++m) {
          mma3_tf32(qacc[m][0], ah[m], al[m], bh0, bh1, bl0, bl1);
          if constexpr (TWO_N) mma3_tf32(qacc[m][1], ah[m], al[m], ch0, ch1, cl0, cl1);
          // G tile (m, n), n >= m: the B column j = n*8 + gq is h_j, i.e. this
          // lane's A entries of user tile n (b0 = Re, b1 = Im).
          if (decltype(with_g)::value) {
#pragma unroll
            for (int n = m; n < UT; ++n) {
              if (n == m) {
                // diagonal tile: hi*hi and hi*lo only; its lo*hi is the
                // conjugate transpose of hi*lo (same exact products, same
                // order: taken in the epilogue, bit for bit the same sums)
                mma_tf32(gacc[m == 0 ? n : 2][0], ah[m][0], ah[m][1], ah[m][2], ah[n][0], ah[n][2]);
                mma_tf32(gacc[m == 0 ? n : 2][1], ah[m][0], ah[m][1], ah[m][2], al[n][0], al[n][2]);
              } else {
                mma3_tf32(gacc[m == 0 ? n : 2], ah[m], al[m], ah[n][0], ah[n][2], al[n][0], al[n][2]);
              }
            }
          }
        }
      } else {
        // two parts: round 1 (hi*hi, hi*lo) over every tile, then round 2
        // (lo*hi into the hi*lo part, updated several MMAs earlier)
#pragma unroll
        for (int m = 0; m < UT; ++m) {
          mma_tf32(qacc[m][0][0], ah[m][0], ah[m][1], ah[m][2], bh0, bh1);
          mma_tf32(qacc[m][0][1], ah[m][0], ah[m][1], ah[m][2], bl0, bl1);
          if constexpr (TWO_N) {
            mma_tf32(qacc[m][1][0], ah[m][0], ah[m][1], ah[m][2], ch0, ch1);
            mma_tf32(qacc[m][1][1], ah[m][0], ah[m][1], ah[m][2], cl0, cl1);
          }
          if (decltype(with_g)::value) {
#pragma unroll
            for (int n = m; n < UT; ++n) {
              mma_tf32(gacc[m == 0 ? n : 2][0], ah[m][0], ah[m][1], ah[m][2], ah[n][0], ah[n][2]);
              mma_tf32(gacc[m == 0 ? n : 2][1], ah[m][0], ah[m][1], ah[m][2], al[n][0], al[n][2]);
            }
          }
        }
#pragma unroll
        for (int m = 0; m < UT; ++m) {
          mma_tf32(qacc[m][0][1], al[m][0], al[m][1], al[m][2], bh0, bh1);
          if constexpr (TWO_N) mma_tf32(qacc[m][1][1], al[m][0], al[m][1], al[m][2], ch0, ch1);
          if (decltype(with_g)::value) {
#pragma unroll
            for (int n = m; n < UT; ++n)
              mma_tf32(gacc[m == 0 ? n : 2][1], al[m][0], al[m][1], al[m][2], ah[n][0], ah[n][2]);
          }
        }
      }
    };
    const float2* hl = sH + ta * U + gq;  // lane's channel entry, antenna offset ta
    auto block = [&](auto with_g, auto two_n) {
      constexpr bool TWO_N = decltype(two_n)::value;
      if (bb == BB && !mask_u) {
        // full block, full user tiles: no masking
        for (int box = 0; box < S::kBoxes; ++box) {
          const unsigned char* yb = bp + box * S::kBoxBytes;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            float2 h[UT];
#pragma unroll
            for (int m = 0; m < UT; ++m) h[m] = hl[(box * S::kBoxAnt + 2 * kk) * U + m * 8];
            const float2 ya = *reinterpret_cast<const float2*>(yb + yoff[kk]);
            const float2 yc = TWO_N ? *reinterpret_cast<const float2*>(yb + yoff[kk] + 8 * 128)
                                    : make_float2(0.f, 0.f);
            kstep(h, ya, yc, with_g, two_n);
          }
        }
        return;
      }
      for (int box = 0; box * S::kBoxAnt < bb; ++box) {
        const unsigned char* yb = bp + box * S::kBoxBytes;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const int a = box * S::kBoxAnt + 2 * kk + ta;
          // channel rows past bb are stale in the staging buffer, and user
          // slots past U hold other rows' entries: both masked
          const bool ok = a < bb;
          float2 h[UT];
#pragma unroll
          for (int m = 0; m < UT; ++m) {
            const bool okm = ok && m * 8 + gq < U;
            h[m] = okm ? hl[(box * S::kBoxAnt + 2 * kk) * U + m * 8] : make_float2(0.f, 0.f);
          }
          const float2 ya = *reinterpret_cast<const float2*>(yb + yoff[kk]);
          const float2 yc = TWO_N ? *reinterpret_cast<const float2*>(yb + yoff[kk] + 8 * 128)
                                  : make_float2(0.f, 0.f);
          kstep(h, ya, yc, with_g, two_n);
        }
      }
    };
    // passes of at most 8 symbols (T <= 8, or a short last pass) skip the
    // second n-tile's MMAs
    if (!OCD_TMA_SKIP_N1 || np > 8) {
      if (first) block(std::true_type{}, std::true_type{});
      else block(std::false_type{}, std::true_type{});
    } else {
      if (first) block(std::true_type{}, std::false_type{});
      else block(std::false_type{}, std::false_type{});
    }
    __syncwarp();
    if (blk != nblk - 1) continue;

    // ---------------- epilogue of a pass ----------------------------------
    // (1) fragments -> shared memory.  Lane (gq, t) holds rows gq (real) and
    // gq + 8 (imaginary) of columns 2t, 2t + 1 of each tile; the split parts
    // are summed smallest first.
#pragma unroll
    for (int m = 0; m < UT; ++m)
#pragma unroll
      for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int ts = 8 * n + 2 * t + e;
          const int u = m * 8 + gq;
          const float (&a)[NQ][4] = qacc[m][n];
          sq[tma_sq<NU>(ts, u)] = (a[NQ - 1][e] + (NQ == 3 ? a[1][e] : 0.0f)) + a[0][e];
          sq[tma_sq<NU>(ts, u) + 1] =
              (a[NQ - 1][2 + e] + (NQ == 3 ? a[1][2 + e] : 0.0f)) + a[0][2 + e];
        }
    if (first) {
      // lo*hi of a diagonal G tile: lo*hi[i][j] = conj(hi*lo[j][i]); the
      // hi*lo parts go to G's buffer first, then each lane reads the entry
      // transposed to its own
      float lhr[UT][2] = {}, lhi[UT][2] = {};
      if constexpr (NQ == 3) {
#pragma unroll
        for (int m = 0; m < UT; ++m)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float (&a)[NQ][4] = gacc[m == 0 ? m : 2];
            const int i = m * 8 + gq, j = m * 8 + 2 * t + e;
            sg[tma_gre<NU>(i, j)] = a[1][e];
            sg[tma_gim<NU>(i, j)] = a[1][2 + e];
          }
        __syncwarp();
#pragma unroll
        for (int m = 0; m < UT; ++m)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int i = m * 8 + gq, j = m * 8 + 2 * t + e;
            lhr[m][e] = sg[tma_gre<NU>(j, i)];
            lhi[m][e] = -sg[tma_gim<NU>(j, i)];
          }
        __syncwarp();
      }
#pragma unroll
      for (int m = 0; m < UT; ++m)
#pragma unroll
        for (int n = m; n < UT; ++n)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float (&a)[NQ][4] = gacc[m == 0 ? n : 2];
            const bool diag3 = NQ == 3 && n == m;
            const float lr = diag3 ? lhr[m][e] : a[NQ - 1][e];
            const float li = diag3 ? lhi[m][e] : a[NQ - 1][2 + e];
            const float re = (lr + (NQ == 3 ? a[1][e] : 0.0f)) + a[0][e];
            const float im = (li + (NQ == 3 ? a[1][2 + e] : 0.0f)) + a[0][2 + e];
            const int i = m * 8 + gq, j = n * 8 + 2 * t + e;
            sg[tma_gre<NU>(i, j)] = re;
            sg[tma_gim<NU>(i, j)] = im;
            if (n != m) {  // lower block from Hermitian symmetry
              sg[tma_gre<NU>(j, i)] = re;
              sg[tma_gim<NU>(j, i)] = -im;
            }
          }
    }
    __syncwarp();
    // (2) preprocessing (Algorithm 1) and soft-output constants
    if (first) {
      if (lane < NU) {
        const float nrm = sg[tma_gre<NU>(lane, lane)];
        const float den = nrm + P.alpha;
        const float dinv = (lane < U && den > 0.0f) ? 1.0f / den : 0.0f;
        const float p = dinv * nrm;
        spre[4 * lane] = dinv;
        spre[4 * lane + 1] = p;
        spre[4 * lane + 2] = llr_rs2(nrm, P);  // rho~ step^2
        spre[4 * lane + 3] = llr_u_scale(p, P);  // level units per unit of z
        sg[tma_gim<NU>(lane, lane)] = 0.0f;  // G_uu is real
      }
      __syncwarp();
    }
    // (3) K sweeps on q: lane = 2 ts + hf holds users [hf*UP, hf*UP + UP)
    {
      const int ts = lane >> 1;
      const int hf = lane & 1;
      const bool act = ts < np;
      float qr[UP], qi[UP], zr[UP], zi[UP];
      {
        // this lane's half of symbol ts: UP users as (re, im) pairs
        const float4* q4 = reinterpret_cast<const float4*>(sq + tma_sq<NU>(ts & 15, hf * UP));
#pragma unroll
        for (int l2 = 0; l2 < UP / 2; ++l2) {
          const float4 v = act ? q4[l2] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          qr[2 * l2] = v.x;
          qi[2 * l2] = v.y;
          qr[2 * l2 + 1] = v.z;
          qi[2 * l2 + 1] = v.w;
          zr[2 * l2] = zr[2 * l2 + 1] = 0.0f;
          zi[2 * l2] = zi[2 * l2 + 1] = 0.0f;
        }
      }
      float dv[NU], pv[NU];
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        dv[u] = spre[4 * u];
        pv[u] = spre[4 * u + 1];
      }
      // Projection of Eq. 14 without branches: clip bounds are +inf in MMSE
      // mode (identity) and 0 on the imaginary axis for BPSK in BOX mode.
      const float are = P.box ? P.box_a : __int_as_float(0x7f800000);
      const float aim = P.box ? (P.bpsk ? 0.0f : P.box_a) : __int_as_float(0x7f800000);
      // a full user tile (U equal to the tile) needs no per-user guard: the
      // updates of all users form one block the scheduler can interleave
      auto sweeps = [&](auto fullc) {
        constexpr bool FULL = decltype(fullc)::value;
        for (int k = 0; k < P.K; ++k) {
#pragma unroll
          for (int u = 0; u < NU; ++u) {
            if (FULL || u < U) {
              const int lu = u % UP;  // compile-time slot of user u
              const int oh = u / UP;  // half that owns user u
              // z_u <- proj(d_u^-1 q_u + p_u z_u), dz = z_new - z_old (owner lane)
              float wr = fmaf(dv[u], qr[lu], pv[u] * zr[lu]);
              float wi = fmaf(dv[u], qi[lu], pv[u] * zi[lu]);
              wr = fminf(fmaxf(wr, -are), are);
              wi = fminf(fmaxf(wi, -aim), aim);
              const float dr0 = wr - zr[lu];
              const float di0 = wi - zi[lu];
              if (hf == oh) { zr[lu] = wr; zi[lu] = wi; }
              const int owner = (lane & ~1) | oh;
              const float dr = __shfl_sync(kFullMask, dr0, owner);
              const float di = __shfl_sync(kFullMask, di0, owner);
              // q <- q - G[:, u] dz for my users, with G[j][u] = conj(G[u][j])
              const float4* gre = reinterpret_cast<const float4*>(sg + tma_gre<NU>(u, hf * UP));
              const float4* gim = reinterpret_cast<const float4*>(sg + tma_gim<NU>(u, hf * UP));
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
      };
      if (U == NU) sweeps(std::true_type{});
      else sweeps(std::false_type{});
      __syncwarp();
      if (act) {
        float4* z4 = reinterpret_cast<float4*>(sq + tma_sq<NU>(ts, hf * UP));  // z overwrites q0
#pragma unroll
        for (int l2 = 0; l2 < UP / 2; ++l2)
          z4[l2] = make_float4(zr[2 * l2], zi[2 * l2], zr[2 * l2 + 1], zi[2 * l2 + 1]);
      }
      __syncwarp();
    }
    // (4) outputs, one item per (symbol ts, user u)
#if OCD_TMA_OUT_FAST
    // A full user tile splits the item index with a shift instead of a
    // division by U, and the LLR code is chosen once per pass by the bits
    // per real dimension instead of once per item.
    auto outputs = [&](auto nbc) {
      constexpr int NB = decltype(nbc)::value;
      const bool full_tile = U == NU;
      // both dimensions' LLRs of an item stored as float2 pairs (Q = 2 NB is
      // even, so every item starts 8-byte aligned when the array does)
      const bool pairs = !P.bpsk && (reinterpret_cast<uintptr_t>(P.llr) & 7u) == 0;
      for (int f = lane; f < np * U; f += 32) {
        const int ts = full_tile ? f / NU : f / U;
        const int u = f - ts * U;
        const float2 z = *reinterpret_cast<const float2*>(sq + tma_sq<NU>(ts, u));
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
#else
    for (int f = lane; f < np * U; f += 32) {
      const int ts = f / U;
      const int u = f - ts * U;
      const float2 z = *reinterpret_cast<const float2*>(sq + tma_sq<NU>(ts, u));
      const long long o = (sc * T + tb + ts) * U + u;
      if (P.xhat) P.xhat[o] = z;
      if (P.llr) {
        float* out = P.llr + o * P.Q;
        const float inv = spre[4 * u + 3];
        if (!(inv > 0.0f)) {
          for (int j = 0; j < P.Q; ++j) out[j] = 0.0f;
        } else {
          const float rs2 = spre[4 * u + 2];
          dimension_llr(z.x * inv, rs2, P, out);
          if (!P.bpsk) dimension_llr(z.y * inv, rs2, P, out + P.nb);
        }
      }
    }
#endif
    __syncwarp();
  }
  return true;
}

// Single problem: warp gw of the persistent grid takes subcarriers gw,
// gw + (warps in the grid), ...
template <int UT>
__global__ void __launch_bounds__(32 * OCD_TMA_WARPS, UT == 1 ? OCD_TMA_MIN_CTAS : 2)
ocd_projected_tma_kernel(const __grid_constant__ DetectParams P,
                         const __grid_constant__ CUtensorMap ymap) {
  using S = TmaShape<UT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // Align within the shared window by pointer arithmetic on the __shared__
  // array itself, so every access below stays a shared-memory access.
  unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  unsigned char* ws = base + warp * S::kWarpBytes;
  const uint32_t bar0 = smem_addr(ws + S::kOffBar);
  const long long nW = (long long)gridDim.x * (blockDim.x >> 5);
  const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  if (gw >= P.Nsc) return;
  if (lane == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ymap)) : "memory");
    for (int i = 0; i < S::kStages; ++i) mbar_init(bar0 + 8 * i, 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t parity = 0;  // bit i: parity of the next phase of buffer i
  // launched by launch_serialized: the set-up above may overlap the drain of
  // the kernel ahead in the stream
  pdl_wait();
  tma_walk<UT>(P, &ymap, ws, bar0, parity, gw, P.Nsc, nW);
  pdl_trigger();
}

// Several problems in one persistent launch: each warp draws tickets from a
// device counter (one atomicAdd per ticket, no waiting on other warps); a
// ticket is a run of consecutive subcarriers of one cell.  Tickets of cell c
// are [tick_end[c-1], tick_end[c]).
template <int UT>
__global__ void __launch_bounds__(32 * OCD_TMA_WARPS, UT == 1 ? OCD_TMA_MIN_CTAS : 2)
ocd_batched_tma_kernel(const __grid_constant__ BatchTable tab, unsigned int* __restrict__ tickets) {
  using S = TmaShape<UT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  unsigned char* ws = base + warp * S::kWarpBytes;
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
    // a warp's tickets increase, so its cell index only moves forward
    while (tk >= tab.cell[c].tick_end) ++c;
    const BatchCell& C = tab.cell[c];
    if (c != prefetched) {
      // a tensor copy needs a 64-byte aligned map: record and leave otherwise
      if (reinterpret_cast<uintptr_t>(&C.ymap) & 63u) {
        if (lane == 0) atomicOr(&g_tma_fault, 2u);
        return;
      }
      if (lane == 0)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&C.ymap)) : "memory");
      prefetched = c;
    }
    const long long t0 = c ? tab.cell[c - 1].tick_end : 0;
    const long long lo = ((long long)tk - t0) * C.sc_per_tick;
    const long long hi = min(lo + (long long)C.sc_per_tick, (long long)C.P.Nsc);
    if (!tma_walk<UT>(C.P, &C.ymap, ws, bar0, parity, lo, hi, 1)) return;
  }
}

// Timeout self-test: waits on a phase that nothing completes (no copy is
// ever issued against this barrier), so the bounded wait must expire.
__global__ void ocd_wait_selftest_kernel(unsigned long long wait_ns) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = smem_addr(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (!mbar_wait(b, 0, wait_ns) && threadIdx.x == 0) atomicOr(&g_tma_fault, 1u);
}

}  // namespace ocd
