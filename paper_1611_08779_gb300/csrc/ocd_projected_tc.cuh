// Projected-residual OCD for 17 to 32 users with the two per-subcarrier
// products on the fifth-generation tensor cores (tcgen05, accumulators in
// tensor memory).  Same algebra as the warp-level 32-user kernel
// (ocd_projected_wide.cuh): q0 = H^H Y^T and G = H^H H per subcarrier, then
// the K sweeps of Algorithm 1 on q = H^H r.
//
// Realified products over K = 2B (antenna a, part c): with the operand rows
//     Re-row u:  (Re h_{a,u}, Im h_{a,u})_a      Im-row u:  (-Im h_{a,u}, Re h_{a,u})_a
//     Y-row t:   (Re y_{t,a}, Im y_{t,a})_a       (the received row as stored)
// the dot product of Re-row u with Y-row t is Re(h_u^H y_t) and of Im-row u
// with it Im(h_u^H y_t); with Re-row j in place of the Y-row they give
// Re G_uj and Im G_uj.  Two subcarriers a, b share every MMA: per K slice of
// 8, A = [Re_a | Re_b | Im_a | Im_b] (M = 128, in tensor memory, row i in
// TMEM lane i) and B = [Y_a | Y_b | Re_a | Re_b] (N = 2 YR + 64, in shared
// memory) accumulate q0 (columns 0 .. 2 YR - 1) and G (the rest) of both;
// the blocks that mix a with b are computed and dropped.
// FP32-level accuracy: A B^T = Ah Bh^T + Ah Bl^T + Al Bh^T with hi = the value
// as stored (the tensor core reads the leading 19 bits of an FP32 operand:
// it truncates, measured) and lo = value - trunc(value); the dropped Al Bl^T
// and the truncation of lo leave about 2^-20 relative error per product.
//
// One CTA (14 warps, all 512 TMEM columns) per SM, persistent over
// subcarriers blockIdx.x + i gridDim.x, blocks of 16 antennas (one 128-byte
// K atom per operand row):
//   warp 0      producer: per pair and block a bulk copy of the 16 channel
//               rows and a 2-D tensor copy of the YR received rows (128-byte
//               swizzle, the operand layout itself) of each subcarrier into
//               a ring of raw stages;
//   warps 2-5   transform, one per TMEM lane quarter: a thread (= user)
//               writes its Re- or Im-row, hi and lo, into the A stage with
//               tcgen05.st; the Re warps also store their rows into B, and
//               all four copy a share of the received rows with their lo rows;
//   warp 1      one thread issues 3 MMAs per K slice (A from TMEM) into the
//               pair's TMEM slot and commits each block (the stage is free
//               again) and each pair (accumulators ready);
//   warps 6-13  epilogue, two per TMEM lane quarter: groups of 8 subcarriers
//               (4 pairs, every accumulator slot) are drained from TMEM, each
//               slot released as soon as it is read; then each warp runs the
//               preprocessing, the K sweeps and the outputs of one of them.
// TMEM: two A stages of 64 columns (hi, lo), then four accumulator slots of
// 96 columns, so the MMAs of one group run under the epilogue of the
// previous one.  Every wait is bounded in wall time; a wait that expires
// sets the fault word and a shared abort flag that ends every role's loop,
// and the async copies and MMAs in flight are waited for (bounded) before
// the TMEM is released.
#pragma once

#include "ocd_projected_wide.cuh"
#include "ocd_tcgen05.cuh"

namespace ocd {

#ifndef OCD_TC_RAW_STAGES
#define OCD_TC_RAW_STAGES 4   // pair blocks whose copies may be in flight (48 KB per SM)
#endif
#ifndef OCD_TC_OP_STAGES
#define OCD_TC_OP_STAGES 2    // operand stages (transform ahead of the MMAs)
#endif

// Two subcarriers a, b share every MMA ("pair").  A = the 128 rows
// [Re_a | Re_b | Im_a | Im_b] (M = 128, TMEM lane i = row i) lives in tensor
// memory; B = the 2 YR + 64 rows [Y_a | Y_b | Re_a | Re_b] (N = 2 YR + 64) in
// shared memory.  The accumulator blocks that mix a with b are computed and
// dropped.
template <int YR>
struct TcShape {
  static_assert(YR == 8 || YR == 16, "received rows per subcarrier: 8 or 16");
  static constexpr int kBA = 16;                          // antennas per staged block
  static constexpr int kN = 2 * YR + 64;                  // MMA N
  static constexpr int kRowRe = 2 * YR;                   // first Re row of B
  static constexpr int kRows = 2 * YR + 64;               // B rows
  static constexpr int kOpBytes = kRows * 128;            // one B buffer (hi or lo)
  static constexpr int kOpStageBytes = 2 * kOpBytes;      // hi and lo
  static constexpr int kOpStages = OCD_TC_OP_STAGES;
  // raw stage: Y_a, Y_b boxes (swizzled, each YR rows), then H_a, H_b
  static constexpr int kRawY = YR * 128;                  // one subcarrier's received rows
  static constexpr int kRawH = kBA * 32 * 8;              // one subcarrier's channel rows
  static constexpr int kRawStageBytes = 2 * kRawY + 2 * kRawH;
  static constexpr int kRawStages = OCD_TC_RAW_STAGES;
  // tensor memory: A stages (hi in columns 0-31, lo in 32-63 of a stage),
  // then the accumulator slots
  static constexpr int kACols = 64;
  static constexpr int kSlots = 4;                        // accumulator slots (pairs)
  static constexpr int kSlotCols = 96;
  static constexpr int kAccCol = kOpStages * kACols;
  static constexpr int kTmemCols = 512;                   // the whole TMEM of an SM
  static constexpr int kEpiG = 32 * WideShape::kGRow * 4;  // G rows (re run | im run | pad)
  static constexpr int kEpiQ = 16 * WideShape::kSqRow * 4;  // q0, then z (wide_sq layout)
  static constexpr int kEpiPre = 32 * 16;                 // (d^-1, p, rho~ step^2, u scale)
  static constexpr int kEpiBytes = kEpiG + kEpiQ + kEpiPre;
  static constexpr int kEpiWarps = 8;                     // one subcarrier each per group
  static constexpr int kOffRaw = kOpStages * kOpStageBytes;
  static constexpr int kOffEpi = kOffRaw + kRawStages * kRawStageBytes;
  static constexpr int kOffBar = kOffEpi + kEpiWarps * kEpiBytes;
  static constexpr int kNumBars = 2 * kRawStages + 2 * kOpStages + 2 * kSlots;
  static constexpr int kOffTmem = kOffBar + 8 * kNumBars;
  static constexpr int kOffAbort = kOffTmem + 4;
  static constexpr int kBytes = kOffAbort + 4;
  static constexpr int kTransformWarps = 4;               // one per TMEM lane quarter of A
  static constexpr int kThreads = 32 * (2 + kTransformWarps + kEpiWarps);  // 448
  static_assert(kEpiWarps == 2 * kSlots, "a group of subcarriers fills the TMEM slots");
  static_assert(kAccCol + kSlots * kSlotCols <= kTmemCols, "A stages and accumulators fit TMEM");
  static_assert(kOpBytes % 1024 == 0 && kRawY % 1024 == 0 && kRawStageBytes % 1024 == 0,
                "1024-byte swizzle phase");
  static_assert(kN <= kSlotCols && kN % 16 == 0, "one pair's accumulators fit a slot");
};

// Cycle counters per role (waits and work), compiled in only with
// OCD_TC_TRACE: four per warp, summed over the CTAs into g_tc_trace.
#ifdef OCD_TC_TRACE
__device__ unsigned long long g_tc_trace[16 * 4];
#define TC_CLOCK(v) const long long v = clock64()
#define TC_ADD(k, v) tr[k] += (unsigned long long)(clock64() - v)
#else
#define TC_CLOCK(v)
#define TC_ADD(k, v)
#endif

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// mbarrier try-wait that lets the thread sleep until the phase completes or
// about `hint_ns` have passed (no issue slots spent while it sleeps).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity,
                                                    uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Bounded wait that also gives up when another role has aborted; an expired
// limit sets the abort flag and bit 0 of the fault word.  Between checks the
// thread sleeps on the barrier (up to 20 us), so waiting roles leave the
// issue slots to the working ones.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns,
                                        volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
    if (*abort_flag) return false;
    if (global_ns() - t0 >= limit_ns) {
      *abort_flag = 1;
      atomicOr(&g_wide_fault, 1u);
      return false;
    }
  }
}
// The same for all 32 lanes of a warp, with one warp-uniform result.
__device__ __forceinline__ bool tc_wait_warp(uint32_t bar, uint32_t parity,
                                             unsigned long long limit_ns, volatile int* abort_flag) {
  const bool ok = tc_wait(bar, parity, limit_ns, abort_flag);
  return __all_sync(kFullMask, ok);
}

// x - trunc_TF32(x) for the four values of a 16-byte chunk.
__device__ __forceinline__ float4 tf32_lo4(float4 v) {
  auto lo = [](float x) { return x - __uint_as_float(__float_as_uint(x) & 0xffffe000u); };
  return make_float4(lo(v.x), lo(v.y), lo(v.z), lo(v.w));
}

template <int YR>
__global__ void __launch_bounds__(TcShape<YR>::kThreads, 1)
ocd_projected_tc_kernel(const __grid_constant__ DetectParams P,
                        const __grid_constant__ CUtensorMap ymap) {
  using S = TcShape<YR>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const uint32_t sbase = smem_addr(base);
  const uint32_t bars = sbase + S::kOffBar;
  constexpr int R = S::kRawStages;
  constexpr int O = S::kOpStages;
  constexpr int NTW = S::kTransformWarps;
  constexpr int EW0 = 2 + NTW;  // first epilogue warp
  auto bar_full = [&](int s) { return bars + 8u * s; };                 // raw stage landed
  auto bar_free = [&](int s) { return bars + 8u * (R + s); };           // raw stage read
  auto bar_ready = [&](int s) { return bars + 8u * (2 * R + s); };      // operands written
  auto bar_empty = [&](int s) { return bars + 8u * (2 * R + O + s); };  // operands consumed
  auto bar_accfull = [&](int j) { return bars + 8u * (2 * R + 2 * O + j); };
  auto bar_accempty = [&](int j) { return bars + 8u * (2 * R + 2 * O + S::kSlots + j); };
  volatile int* abort_flag = reinterpret_cast<volatile int*>(base + S::kOffAbort);

  const int B = P.B;
  const int U = P.U;
  const int T = P.T;
  const int nblk = (B + S::kBA - 1) / S::kBA;
  // this CTA's subcarriers: item i is subcarrier first + i * stride; pair p
  // holds items 2p (half a) and 2p + 1 (half b, absent past the last item)
  const long long first = blockIdx.x;
  const long long stride = gridDim.x;
  const long long nitems = first < P.Nsc ? (P.Nsc - 1 - first) / stride + 1 : 0;
  const long long npairs = (nitems + 1) / 2;

  if (tid == 0) {
    for (int s = 0; s < R; ++s) {
      mbar_init(bar_full(s), 1);
      mbar_init(bar_free(s), NTW);
    }
    for (int s = 0; s < O; ++s) {
      mbar_init(bar_ready(s), NTW);
      mbar_init(bar_empty(s), 1);
    }
    for (int j = 0; j < S::kSlots; ++j) {
      mbar_init(bar_accfull(j), 1);
      mbar_init(bar_accempty(j), 4);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(sbase + S::kOffTmem, S::kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(base + S::kOffTmem);
  pdl_wait();  // launched by launch_serialized
#ifdef OCD_TC_TRACE
  unsigned long long tr[4] = {0, 0, 0, 0};
#endif

  if (warp == 0) {
    // ---------------- producer -------------------------------------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ymap)) : "memory");
      long long g = 0;
      bool ok = true;
      for (long long p = 0; p < npairs && ok; ++p) {
        const bool has_b = 2 * p + 1 < nitems;
        const long long sca = first + 2 * p * stride;
        for (int blk = 0; blk < nblk; ++blk, ++g) {
          const int st = (int)(g % R);
          const long long n = g / R;
          TC_CLOCK(c0);
          if (n > 0 && !tc_wait(bar_free(st), (uint32_t)((n - 1) & 1), P.wait_ns, abort_flag)) {
            ok = false;
            break;
          }
          TC_ADD(0, c0);
          const int b0 = blk * S::kBA;
          const int bb = min(S::kBA, B - b0);
          const uint32_t hbytes = (uint32_t)(bb * U * 8);
          const uint32_t stp = sbase + S::kOffRaw + st * S::kRawStageBytes;
          fence_proxy_async();
          mbar_expect_tx(bar_full(st), (has_b ? 2u : 1u) * (hbytes + (uint32_t)S::kRawY));
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (h == 1 && !has_b) break;
            const long long sc = sca + h * stride;
            tma_load_2d(stp + h * S::kRawY, &ymap, 2 * b0, (int)(sc * T), bar_full(st));
            bulk_g2s(stp + 2 * S::kRawY + h * S::kRawH, P.H + (sc * (long long)B + b0) * U, hbytes,
                     bar_full(st));
          }
        }
      }
      if (!ok) {
        // let the copies in flight land before the CTA can end
        for (long long gg = g - R > 0 ? g - R : 0; gg < g; ++gg)
          mbar_wait(bar_full((int)(gg % R)), (uint32_t)((gg / R) & 1), P.wait_ns);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ------------------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc(128, S::kN);
      long long g = 0;
      bool ok = true;
      for (long long p = 0; p < npairs && ok; ++p) {
        const int slot = (int)(p % S::kSlots);
        const long long m = p / S::kSlots;
        TC_CLOCK(c0);
        if (m > 0 && !tc_wait(bar_accempty(slot), (uint32_t)((m - 1) & 1), P.wait_ns, abort_flag)) {
          ok = false;
          break;
        }
        TC_ADD(0, c0);
        tc_fence_after();
        const uint32_t d = tbase + (uint32_t)(S::kAccCol + slot * S::kSlotCols);
        for (int blk = 0; blk < nblk; ++blk, ++g) {
          const int st = (int)(g % O);
          TC_CLOCK(c1);
          if (!tc_wait(bar_ready(st), (uint32_t)((g / O) & 1), P.wait_ns, abort_flag)) {
            ok = false;
            break;
          }
          TC_ADD(1, c1);
          TC_CLOCK(c2);
          tc_fence_after();
          // A: TMEM columns of the stage (hi, then lo 32 columns on), 8 per
          // K slice; B: descriptors of the stage, K slices 32 bytes (2 units
          // of the start-address field) apart
          const uint32_t ah = tbase + (uint32_t)(st * S::kACols);
          const uint32_t al = ah + 32u;
          const uint32_t hi = sbase + st * S::kOpStageBytes;
          const uint64_t bh = sw128_desc(hi);
          const uint64_t bl = sw128_desc(hi + S::kOpBytes);
          tc_mma_tf32_ts(d, ah, bh, idesc, blk > 0 ? 1u : 0u);
          tc_mma_tf32_ts(d, ah, bl, idesc, 1u);
          tc_mma_tf32_ts(d, al, bh, idesc, 1u);
#pragma unroll
          for (int ks = 1; ks < 4; ++ks) {
            tc_mma_tf32_ts(d, ah + 8 * ks, bh + 2 * ks, idesc, 1u);
            tc_mma_tf32_ts(d, ah + 8 * ks, bl + 2 * ks, idesc, 1u);
            tc_mma_tf32_ts(d, al + 8 * ks, bh + 2 * ks, idesc, 1u);
          }
          tc_commit(bar_empty(st));
          TC_ADD(2, c2);
        }
        if (!ok) break;
        tc_commit(bar_accfull(slot));
      }
      // no MMA may still run when the TMEM is released: wait (bounded) for
      // the commit that covers the last one issued
      if (g > 0) mbar_wait(bar_empty((int)((g - 1) % O)), (uint32_t)(((g - 1) / O) & 1), P.wait_ns);
    }
    __syncwarp();
  } else if (warp < EW0) {
    // ---------------- transform -------------------------------------------
    // Warp with TMEM lane quarter q writes A rows 32q + u (u = lane): the
    // Re-row (q < 2) or the Im-row (q >= 2) of user u of half h = q & 1,
    // hi and lo, with tcgen05.st.  The Re warps also store their rows into
    // B (the G columns); the received rows are copied by all four.
    // An absent half b transforms stale data into rows nobody reads.
    const int q = warp & 3;
    const int h = q & 1;
    const bool imrow = q >= 2;
    const int u = lane;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    long long g = 0;
    bool ok = true;
    for (long long p = 0; p < npairs && ok; ++p) {
      for (int blk = 0; blk < nblk; ++blk, ++g) {
        const int rs = (int)(g % R);
        const int os = (int)(g % O);
        TC_CLOCK(c0);
        if (!tc_wait_warp(bar_full(rs), (uint32_t)((g / R) & 1), P.wait_ns, abort_flag)) {
          ok = false;
          break;
        }
        TC_ADD(0, c0);
        TC_CLOCK(c1);
        if (g >= O && !tc_wait_warp(bar_empty(os), (uint32_t)((g / O - 1) & 1), P.wait_ns,
                                    abort_flag)) {
          ok = false;
          break;
        }
        TC_ADD(1, c1);
        TC_CLOCK(c2);
        tc_fence_after();
        const int bb = min(S::kBA, B - blk * S::kBA);
        unsigned char* hi = base + os * S::kOpStageBytes;
        unsigned char* lo = hi + S::kOpBytes;
        const unsigned char* rawst = base + S::kOffRaw + rs * S::kRawStageBytes;
        const float2* raw = reinterpret_cast<const float2*>(rawst + 2 * S::kRawY + h * S::kRawH);
        const uint32_t ta = tbase + lane_base + (uint32_t)(os * S::kACols);
        const int row = S::kRowRe + 32 * h + u;  // this user's B row (Re warps)
        const bool uok = u < U;
        // K chunk c = antennas 4c .. 4c + 3 (8 columns, two 16-byte chunks)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v[8];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int a = 4 * c + k;
            const float2 x = (uok && a < bb) ? raw[a * U + u] : make_float2(0.0f, 0.0f);
            v[2 * k] = imrow ? -x.y : x.x;
            v[2 * k + 1] = imrow ? x.x : x.y;
          }
          float w[8];
#pragma unroll
          for (int k = 0; k < 8; ++k)
            w[k] = v[k] - __uint_as_float(__float_as_uint(v[k]) & 0xffffe000u);
          tmem_st8(ta + 8 * c, __float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]),
                   __float_as_uint(v[3]), __float_as_uint(v[4]), __float_as_uint(v[5]),
                   __float_as_uint(v[6]), __float_as_uint(v[7]));
          tmem_st8(ta + 32 + 8 * c, __float_as_uint(w[0]), __float_as_uint(w[1]),
                   __float_as_uint(w[2]), __float_as_uint(w[3]), __float_as_uint(w[4]),
                   __float_as_uint(w[5]), __float_as_uint(w[6]), __float_as_uint(w[7]));
          if (!imrow) {
            const int o0 = row * 128 + (((2 * c) ^ (row & 7)) << 4);
            const int o1 = row * 128 + (((2 * c + 1) ^ (row & 7)) << 4);
            *reinterpret_cast<float4*>(hi + o0) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4*>(hi + o1) = make_float4(v[4], v[5], v[6], v[7]);
            *reinterpret_cast<float4*>(lo + o0) = make_float4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<float4*>(lo + o1) = make_float4(w[4], w[5], w[6], w[7]);
          }
        }
        {
          // received rows of both halves, as staged (the same swizzled layout,
          // the same 1024-byte phase) and their lo parts: the 16-byte chunks
          // shared out over the four transform warps
          const int tt = 32 * (q ^ 2) + lane;  // 0 .. 127
#pragma unroll
          for (int c = tt; c < 2 * YR * 8; c += 32 * NTW) {
            const float4 x = *reinterpret_cast<const float4*>(rawst + 16 * c);
            *reinterpret_cast<float4*>(hi + 16 * c) = x;
            *reinterpret_cast<float4*>(lo + 16 * c) = tf32_lo4(x);
          }
        }
        tmem_wait_st();
        fence_proxy_async();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(bar_free(rs));
          mbar_arrive(bar_ready(os));
        }
        TC_ADD(2, c2);
      }
    }
  } else {
    // ---------------- epilogue --------------------------------------------
    // TMEM lane quarter q = rows 32q .. 32q + 31: Re_a, Re_b, Im_a, Im_b;
    // lane = user.  Two warps per quarter: warp ew drains the pairs jp with
    // jp % 2 == ew / 4 of a group of kSlots pairs, and finishes member ew.
    constexpr int NEW = S::kEpiWarps;
    const int q = warp & 3;
    const int ew = warp - EW0;
    const int half = q & 1;
    const int part = q >> 1;                     // 0: real parts, 1: imaginary parts
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const int cq = half * YR;                    // this warp's q0 columns
    const int cg = 2 * YR + 32 * half;           // this warp's G columns
    for (long long p0 = 0; p0 < npairs; p0 += S::kSlots) {
      TC_CLOCK(c0);
      named_bar_sync(1, 32 * NEW);  // every member's buffers are free
      TC_ADD(1, c0);
      for (int jp = ew >> 2; jp < S::kSlots; jp += 2) {
        const long long p = p0 + jp;
        if (p >= npairs) break;
        const int slot = (int)(p % S::kSlots);
        TC_CLOCK(c1);
        if (!tc_wait_warp(bar_accfull(slot), (uint32_t)((p / S::kSlots) & 1), P.wait_ns,
                          abort_flag))
          continue;  // aborted: skip the work, keep the barriers in step
        TC_ADD(0, c1);
        tc_fence_after();
        uint32_t vq[16], vg0[16], vg1[16];
        const uint32_t ta = tbase + lane_base + (uint32_t)(S::kAccCol + slot * S::kSlotCols);
        tmem_ld16(ta + cq, vq);
        tmem_ld16(ta + cg, vg0);
        tmem_ld16(ta + cg + 16, vg1);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_accempty(slot));
        if (2 * p + half >= nitems) continue;  // absent half b
        unsigned char* eb = base + S::kOffEpi + (2 * jp + half) * S::kEpiBytes;
        float* sg = reinterpret_cast<float*>(eb);
        float* sq = reinterpret_cast<float*>(eb + S::kEpiG);
#pragma unroll
        for (int t = 0; t < YR; ++t)
          if (t < T) sq[wide_sq(t, lane) + part] = __uint_as_float(vq[t]);
        // row `lane`'s run of real or imaginary parts as 8 chunks of 4 (the
        // row pad puts the lanes' rows on distinct bank positions)
        float4* row = reinterpret_cast<float4*>(sg + (part ? wide_gim(lane, 0) : wide_gre(lane, 0)));
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          row[c] = make_float4(__uint_as_float(vg0[4 * c]), __uint_as_float(vg0[4 * c + 1]),
                               __uint_as_float(vg0[4 * c + 2]), __uint_as_float(vg0[4 * c + 3]));
          row[4 + c] = make_float4(__uint_as_float(vg1[4 * c]), __uint_as_float(vg1[4 * c + 1]),
                                   __uint_as_float(vg1[4 * c + 2]), __uint_as_float(vg1[4 * c + 3]));
        }
      }
      TC_CLOCK(c2);
      named_bar_sync(1, 32 * NEW);  // every member's G and q0 are in shared memory
      TC_ADD(1, c2);
      TC_CLOCK(c3);
      const long long i = 2 * p0 + ew;  // member ew: pair p0 + ew / 2, half ew % 2
      if (i < nitems && !*abort_flag) {
        unsigned char* eb = base + S::kOffEpi + ew * S::kEpiBytes;
        float* sg = reinterpret_cast<float*>(eb);
        float* sq = reinterpret_cast<float*>(eb + S::kEpiG);
        float* spre = reinterpret_cast<float*>(eb + S::kEpiG + S::kEpiQ);
        {
          // preprocessing of Algorithm 1 and the soft-output constants
          const float nrm = sg[wide_gre(lane, lane)];
          const float den = nrm + P.alpha;
          const float dinv = (lane < U && den > 0.0f) ? 1.0f / den : 0.0f;
          const float pu = dinv * nrm;
          spre[4 * lane] = dinv;
          spre[4 * lane + 1] = pu;
          spre[4 * lane + 2] = llr_rs2(nrm, P);
          spre[4 * lane + 3] = llr_u_scale(pu, P);
          sg[wide_gim(lane, lane)] = 0.0f;  // G_uu is real
        }
        __syncwarp();
        wide_sweeps_outputs<false>(P, sq, sg, spre, first + i * stride, 0, T);
      }
      TC_ADD(2, c3);
    }
  }
#ifdef OCD_TC_TRACE
  if (lane == 0)
    for (int k = 0; k < 4; ++k) atomicAdd(&g_tc_trace[4 * warp + k], tr[k]);
#endif
  pdl_trigger();

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, S::kTmemCols);
  }
}

}  // namespace ocd
