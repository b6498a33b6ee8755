// Projected-residual OCD (q = H^H r; see ocd_projected.cuh for the algebra)
// for H and Y stored as bfloat16 or float16 complex pairs, up to 16 users.
//
// With 16-bit inputs the products need no splitting: a bf16 x bf16 (or
// f16 x f16) product is exact in FP32, and the m16n8k16 MMA accumulates in
// FP32.  A complex entry stored as (re, im) in one 32-bit word is already a
// packed pair along the realified K dimension (k = 2j + {0: re, 1: im} for
// antenna j of an 8-antenna k-step), so B fragments come straight from the
// staged received rows and the A fragment of user rows is the stored channel
// word; the imaginary-part rows of A need (-Im h, Re h), one byte permute and
// one sign flip.  One k-step of 8 antennas issues 2*UT (q0) + UT(UT+1)/2 (G)
// MMAs, against 18 three-term TF32 MMAs per 4 antennas for float32 storage.
//
// Staging per step (32 antennas x 16 symbols): the channel rows by one bulk
// copy, the received rows by one 2-D tensor copy (box 64 x 16 16-bit
// elements = 128-byte rows, 128-byte swizzle), in a kStages ring per warp
// with bounded mbarrier waits.  Epilogue as in the float32 bulk-copy kernel.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "ocd_common.cuh"
#include "ocd_tma_util.cuh"

namespace ocd {

// Fault word of the 16-bit bulk-copy kernels (bit 0: a wait timed out);
// exactly one translation unit (ocd_projected_h16.cu) includes this header.
__device__ unsigned int g_h16_fault = 0;

#ifndef OCD_H16_STAGES
#define OCD_H16_STAGES 3      // staging buffers per warp
#endif
#ifndef OCD_H16_MIN_CTAS
#define OCD_H16_MIN_CTAS 4    // resident CTAs per SM of the one-tile instance (registers <= 128)
#endif

template <int UT>
struct H16Shape {
  static constexpr int kUsers = 8 * UT;                    // user slots
  static constexpr int kPass = 16;                         // symbols per pass (2 n-tiles)
  static constexpr int kBB = 32;                           // antennas per staged block
  static constexpr int kYBytes = kPass * 128;              // one swizzled Y box (64 x 16)
  static constexpr int kHBytes = kBB * kUsers * 4;         // staged H block
  static constexpr int kBufBytes = ((kYBytes + kHBytes + 1023) / 1024) * 1024;
  static constexpr int kStages = OCD_H16_STAGES;
  static constexpr int kUP = kUsers / 2;                   // users per sweep lane
  static constexpr int kOffQ = kStages * kBufBytes;        // q0, later z [pass symbol][u]
  static constexpr int kOffG = kOffQ + 4 * kPass * SqLayout<kUsers>::kRow;
  static constexpr int kOffPre = kOffG + 8 * kUsers * kUsers;
  static constexpr int kOffBar = kOffPre + 16 * kUsers;
  static constexpr int kWarpBytes = ((kOffBar + 8 * kStages + 1023) / 1024) * 1024;
};

// G in shared memory, row i as [Re G_i0 .. Re G_i(NU-1) | Im G_i0 .. Im G_i(NU-1)]:
// a sweep lane reads the real and the imaginary parts of its users as
// separate 16-byte aligned runs.
template <int NU>
__device__ __forceinline__ int h16_gre(int i, int j) { return i * 2 * NU + j; }
template <int NU>
__device__ __forceinline__ int h16_gim(int i, int j) { return i * 2 * NU + NU + j; }

// D += A B for one m16n8k16 tile with 16-bit inputs and FP32 accumulation.
template <int STORE>
__device__ __forceinline__ void mma16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                      uint32_t a3, uint32_t b0, uint32_t b1) {
  if (STORE == kStoreBF16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
}

// (re, im) -> (-im, re) on a packed 16-bit pair (same sign bit for bf16/f16).
__device__ __forceinline__ uint32_t swap_neg(uint32_t v) {
  return __byte_perm(v, 0, 0x1032) ^ 0x00008000u;
}

template <int STORE, int UT>
__global__ void __launch_bounds__(128, UT == 1 ? OCD_H16_MIN_CTAS : 3)
ocd_projected_h16_kernel(const DetectParams P, const __grid_constant__ CUtensorMap ymap) {
  using S = H16Shape<UT>;
  constexpr int BB = S::kBB;
  constexpr int UP = S::kUP;
  constexpr int NU = S::kUsers;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  unsigned char* ws = base + warp * S::kWarpBytes;
  float* sq = reinterpret_cast<float*>(ws + S::kOffQ);
  float* sg = reinterpret_cast<float*>(ws + S::kOffG);
  float* spre = reinterpret_cast<float*>(ws + S::kOffPre);
  const uint32_t bar0 = smem_addr(ws + S::kOffBar);

  const int U = P.U;
  const int B = P.B;
  const int T = P.T;
  const int gq = lane >> 2;
  const int t = lane & 3;
  // swizzled byte offsets of this lane's received entries in a box row gq:
  // antenna kb + t (chunk kb/4) and kb + 4 + t (chunk kb/4 + 1), kb = 0, 8, 16, 24
  int yoff[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) yoff[c] = gq * 128 + ((c ^ gq) << 4) + t * 4;

  const long long nW = (long long)gridDim.x * (blockDim.x >> 5);
  const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  const int nblk = (B + BB - 1) / BB;
  const int npasses = (T + S::kPass - 1) / S::kPass;
  const long long my_nsc = gw < P.Nsc ? (P.Nsc - 1 - gw) / nW + 1 : 0;
  const long long nsteps = my_nsc * npasses * nblk;
  if (nsteps == 0) return;

  if (lane == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ymap)) : "memory");
    for (int i = 0; i < S::kStages; ++i) mbar_init(bar0 + 8 * i, 1);
    fence_mbar_init();
  }
  __syncwarp();
  pdl_wait();  // launched by launch_serialized

  struct Cursor {
    long long sc;
    int pass, blk;
  };
  auto advance = [&](Cursor& q) {
    if (++q.blk == nblk) {
      q.blk = 0;
      if (++q.pass == npasses) {
        q.pass = 0;
        q.sc += nW;
      }
    }
  };
  auto issue = [&](const Cursor& q, int buf) {
    const int b0 = q.blk * BB;
    const int bb = min(BB, B - b0);
    const int tb = q.pass * S::kPass;
    const uint32_t bar = bar0 + 8 * buf;
    unsigned char* bp = ws + buf * S::kBufBytes;
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)(S::kYBytes + bb * U * 4));
    __syncwarp();
    fence_proxy_async();
    if (lane == 0) tma_load_2d(smem_addr(bp), &ymap, 2 * b0, (int)(q.sc * T + tb), bar);
    if (lane == 31) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(P.H) + (q.sc * (long long)B + b0) * U;
      bulk_g2s(smem_addr(bp + S::kYBytes), src, (uint32_t)(bb * U * 4), bar);
    }
  };

  // accumulators: q0 tiles [m][n] (user tile m, symbol tile n) and G tiles
  // for (m, n) in {(0,0), (0,1), (1,1)}; rows gq / gq + 8 = Re / Im of user
  // m*8 + gq.
  constexpr int NG = UT == 1 ? 1 : 3;
  float qacc[UT][2][4];
  float gacc[NG][4];
  uint32_t parity = 0;
  Cursor cur{gw, 0, 0}, nxt{gw, 0, 0};
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
      if (lane == 0) atomicOr(&g_h16_fault, 1u);
      for (int i = 1; i < S::kStages; ++i) {
        if (s + i < nsteps) {
          const int bi = (buf + i) % S::kStages;
          mbar_wait(bar0 + 8 * bi, (parity >> bi) & 1, P.wait_ns);
        }
      }
      return;
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
    const unsigned char* bp = ws + buf * S::kBufBytes;
    advance(cur);
    buf = buf + 1 == S::kStages ? 0 : buf + 1;

    if (blk == 0) {
#pragma unroll
      for (int m = 0; m < UT; ++m)
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
          for (int e = 0; e < 4; ++e) qacc[m][n][e] = 0.0f;
#pragma unroll
      for (int n = 0; n < NG; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) gacc[n][e] = 0.0f;
    }

    // ---------------- products on the tensor cores ------------------------
    // k-step of antennas kb .. kb+7: lane t holds k = 2t, 2t+1 (antenna
    // kb + t) in a0/b0 and k = 2t+8, 2t+9 (antenna kb + 4 + t) in a2/b1.
    // Channel rows past bb are stale in the staging buffer and are masked;
    // received entries past B arrive as zeros from the tensor copy.
    const uint32_t* sH = reinterpret_cast<const uint32_t*>(bp + S::kYBytes);
    auto kstep = [&](int kb, auto with_g) {
      const int ba = kb + t, bc = kb + 4 + t;
      uint32_t a0[UT], a2[UT];
#pragma unroll
      for (int m = 0; m < UT; ++m) {
        const int u = m * 8 + gq;
        a0[m] = (ba < bb && u < U) ? sH[ba * U + u] : 0u;
        a2[m] = (bc < bb && u < U) ? sH[bc * U + u] : 0u;
      }
      uint32_t yb[2][2];
#pragma unroll
      for (int n = 0; n < 2; ++n) {
        const unsigned char* row = bp + n * 8 * 128;
        yb[n][0] = *reinterpret_cast<const uint32_t*>(row + yoff[kb >> 2]);
        yb[n][1] = *reinterpret_cast<const uint32_t*>(row + yoff[(kb >> 2) + 1]);
      }
#pragma unroll
      for (int m = 0; m < UT; ++m) {
        const uint32_t a1 = swap_neg(a0[m]), a3 = swap_neg(a2[m]);
#pragma unroll
        for (int n = 0; n < 2; ++n) mma16<STORE>(qacc[m][n], a0[m], a1, a2[m], a3, yb[n][0], yb[n][1]);
        if (decltype(with_g)::value) {
          // G tile (m, n) for n >= m: B column j = n*8 + gq is h_j, i.e. this
          // lane's A entries of user tile n.
#pragma unroll
          for (int n = m; n < UT; ++n)
            mma16<STORE>(gacc[m == 0 ? n : 2], a0[m], a1, a2[m], a3, a0[n], a2[n]);
        }
      }
    };
    if (bb == BB) {
      // full block: a compile-time k-step loop, so the loads of one k-step
      // can be issued under the MMAs of the one before
      if (first) {
#pragma unroll
        for (int kb = 0; kb < BB; kb += 8) kstep(kb, std::true_type{});
      } else {
#pragma unroll
        for (int kb = 0; kb < BB; kb += 8) kstep(kb, std::false_type{});
      }
    } else if (first) {
      for (int kb = 0; kb < bb; kb += 8) kstep(kb, std::true_type{});
    } else {
      for (int kb = 0; kb < bb; kb += 8) kstep(kb, std::false_type{});
    }
    __syncwarp();
    if (blk != nblk - 1) continue;

    // ---------------- epilogue of a pass ----------------------------------
#pragma unroll
    for (int m = 0; m < UT; ++m)
#pragma unroll
      for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int ts = 8 * n + 2 * t + e;
          const int u = m * 8 + gq;
          sq[tma_sq<NU>(ts, u)] = qacc[m][n][e];
          sq[tma_sq<NU>(ts, u) + 1] = qacc[m][n][2 + e];
        }
    if (first) {
#pragma unroll
      for (int m = 0; m < UT; ++m)
#pragma unroll
        for (int n = m; n < UT; ++n)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float* d = gacc[m == 0 ? n : 2];
            const int i = m * 8 + gq, j = n * 8 + 2 * t + e;
            sg[h16_gre<NU>(i, j)] = d[e];
            sg[h16_gim<NU>(i, j)] = d[2 + e];
            if (n != m) {  // lower block from Hermitian symmetry
              sg[h16_gre<NU>(j, i)] = d[e];
              sg[h16_gim<NU>(j, i)] = -d[2 + e];
            }
          }
    }
    __syncwarp();
    if (first) {
      if (lane < NU) {
        const float nrm = sg[h16_gre<NU>(lane, lane)];
        const float den = nrm + P.alpha;
        const float dinv = (lane < U && den > 0.0f) ? 1.0f / den : 0.0f;
        const float p = dinv * nrm;
        spre[4 * lane] = dinv;
        spre[4 * lane + 1] = p;
        spre[4 * lane + 2] = llr_rs2(nrm, P);  // rho~ step^2
        spre[4 * lane + 3] = llr_u_scale(p, P);  // level units per unit of z
        sg[h16_gim<NU>(lane, lane)] = 0.0f;  // G_uu is real
      }
      __syncwarp();
    }
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
      const float are = P.box ? P.box_a : __int_as_float(0x7f800000);
      const float aim = P.box ? (P.bpsk ? 0.0f : P.box_a) : __int_as_float(0x7f800000);
      for (int k = 0; k < P.K; ++k) {
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          if (u < U) {
            const int lu = u % UP;
            const int oh = u / UP;
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
            const float4* gre = reinterpret_cast<const float4*>(sg + h16_gre<NU>(u, hf * UP));
            const float4* gim = reinterpret_cast<const float4*>(sg + h16_gim<NU>(u, hf * UP));
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
      __syncwarp();
      if (act) {
        float4* z4 = reinterpret_cast<float4*>(sq + tma_sq<NU>(ts, hf * UP));  // z overwrites q0
#pragma unroll
        for (int l2 = 0; l2 < UP / 2; ++l2)
          z4[l2] = make_float4(zr[2 * l2], zi[2 * l2], zr[2 * l2 + 1], zi[2 * l2 + 1]);
      }
      __syncwarp();
    }
    // outputs: a full user tile splits the item index with a shift instead
    // of a division by U; the LLR code is chosen once per pass by the bits
    // per real dimension
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
    __syncwarp();
  }
  pdl_trigger();
}

}  // namespace ocd
