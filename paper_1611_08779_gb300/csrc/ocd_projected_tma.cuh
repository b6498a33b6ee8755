// Projected-residual OCD (q = H^H r, see ocd_projected.cuh for the algebra)
// with the channel and the received vectors streamed into shared memory by
// the bulk-copy (TMA) engine.
//
// One warp owns one subcarrier at a time and walks a sequence of steps:
// for each subcarrier, for each pass of kPass symbols, for each block of BB
// antennas.  Each step's operands -- the BB channel rows H[b0 .. b0+BB)[:]
// (one contiguous copy) and the BB-antenna slices of the pass's received
// rows (one copy per symbol) -- land in one of two per-warp buffers; the
// copy of step s+1 is in flight while step s is computed.  Completion is
// tracked with one mbarrier per buffer; every wait has an iteration limit,
// after which the warp records a fault in device memory and leaves.
//
//   GEMM (per step): lane = c + 4 g; lane (g, c) takes antennas g, g+8, ...
//     of the block and accumulates q0 = H^H y for the pass symbols c, c+4, ...
//     and the columns c, c+4, ... of G = H^H H (first pass only), all from
//     shared memory.  Staged received rows are padded to a stride of 32 mod
//     128 bytes so the four column groups hit distinct banks.
//   Epilogue (last block of a pass): the eight antenna-group partials are
//     summed through shared memory (reusing the drained buffer); the first
//     pass also derives ||h_u||^2 = G_uu, d_u^-1, p_u and the soft-output
//     constants; the K sweeps run with 32/kPass lanes per symbol; then the
//     LLRs and xhat are written.
#pragma once

#include "ocd_common.cuh"

namespace ocd {

constexpr int kTmaWaitLimit = 1 << 22;  // try_wait polls before a wait is declared failed

template <int UMAX>
struct TmaShape {
  static constexpr int kAG = 8;                            // antenna groups
  static constexpr int kCG = 4;                            // column groups
  static constexpr int kTS = 32 / UMAX;                    // pass symbols per lane
  static constexpr int kPass = kCG * kTS;                  // symbols per pass
  static constexpr int kGC = UMAX / kCG;                   // G columns per lane
  static constexpr int kVals = 2 * (kTS * UMAX + UMAX * kGC);  // partial floats per lane
  static constexpr int kRedStride = kVals | 1;             // odd: conflict-free stores
  static constexpr int kBB = UMAX == 8 ? 64 : 32;          // antennas per block
  static constexpr int kYRow = kBB * 8 + 32;               // staged Y row stride (bytes)
  static constexpr int kHBytes = kBB * UMAX * 8;           // staged H block (bytes)
  static constexpr int kBufBytes = kHBytes + kPass * kYRow;
  static constexpr int kRedBytes = 32 * kRedStride * 4;
  static_assert(kRedBytes <= kBufBytes, "reduction area must fit a drained buffer");
  static constexpr int kHalves = 32 / kPass;               // sweep lanes per symbol
  static constexpr int kUP = UMAX / kHalves;               // users per sweep lane
  // per-warp byte offsets
  static constexpr int kOffQ = 2 * kBufBytes;              // q0, later z [pass symbol][u]
  static constexpr int kOffG = kOffQ + 8 * kPass * UMAX;   // full G [i][j]
  static constexpr int kOffPre = kOffG + 8 * UMAX * UMAX;  // (d^-1, p, ||h||^2, 1/(mu sqrtEs))
  static constexpr int kOffBar = kOffPre + 16 * UMAX;      // two mbarriers
  static constexpr int kWarpBytes = kOffBar + 16;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false after the limit.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kTmaWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Fault word of the bulk-copy kernels (bit 0: a wait timed out).  Defined
// here because exactly one translation unit (ocd_projected_tma.cu) includes
// this header; the host reads it through projected_tma_fault().
__device__ unsigned int g_tma_fault = 0;

template <int UMAX>
__global__ void __launch_bounds__(128, 2)
ocd_projected_tma_kernel(const DetectParams P) {
  using S = TmaShape<UMAX>;
  constexpr int TS = S::kTS;
  constexpr int GC = S::kGC;
  constexpr int BB = S::kBB;
  constexpr int UP = S::kUP;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned char* ws = smem_raw + warp * S::kWarpBytes;
  float* sq = reinterpret_cast<float*>(ws + S::kOffQ);
  float* sg = reinterpret_cast<float*>(ws + S::kOffG);
  float* spre = reinterpret_cast<float*>(ws + S::kOffPre);
  const uint32_t bar0 = smem_addr(ws + S::kOffBar);

  const int U = P.U;
  const int B = P.B;
  const int T = P.T;
  const int c = lane & 3;
  const int g = lane >> 2;
  const long long nW = (long long)gridDim.x * (blockDim.x >> 5);
  const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  const int nblk = (B + BB - 1) / BB;
  const int npasses = (T + S::kPass - 1) / S::kPass;
  const long long steps_per_sc = (long long)npasses * nblk;
  const long long my_nsc = gw < P.Nsc ? (P.Nsc - 1 - gw) / nW + 1 : 0;
  const long long nsteps = my_nsc * steps_per_sc;
  if (nsteps == 0) return;

  if (lane == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    fence_mbar_init();
  }
  __syncwarp();

  // Issue the copies of step s into buffer `buf`.
  auto issue = [&](long long s, int buf) {
    const long long scl = s / steps_per_sc;
    const int rem = (int)(s - scl * steps_per_sc);
    const int pass = rem / nblk;
    const int blk = rem - pass * nblk;
    const long long sc = gw + scl * nW;
    const int b0 = blk * BB;
    const int bb = min(BB, B - b0);
    const int tb = pass * S::kPass;
    const int np = min(S::kPass, T - tb);
    const uint32_t bar = bar0 + 8 * buf;
    unsigned char* bp = ws + buf * S::kBufBytes;
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)(bb * U * 8 + np * bb * 8));
    __syncwarp();
    fence_proxy_async();
    if (lane < np) {
      const float2* src = P.Y + ((sc * T + tb + lane) * (long long)B + b0);
      bulk_g2s(smem_addr(bp + S::kHBytes + lane * S::kYRow), src, (uint32_t)(bb * 8), bar);
    }
    if (lane == 31) {
      const float2* src = P.H + (sc * (long long)B + b0) * U;
      bulk_g2s(smem_addr(bp), src, (uint32_t)(bb * U * 8), bar);
    }
  };

  float qa[TS][UMAX][2];
  float ga[UMAX][GC][2];
  uint32_t parity = 0;  // bit i: parity of the next phase of buffer i

  issue(0, 0);
  for (long long s = 0; s < nsteps; ++s) {
    const int buf = (int)(s & 1);
    if (s + 1 < nsteps) issue(s + 1, buf ^ 1);
    if (!mbar_wait(bar0 + 8 * buf, (parity >> buf) & 1)) {
      if (lane == 0) atomicOr(&g_tma_fault, 1u);
      // let the copies already in flight finish (bounded) before leaving
      if (s + 1 < nsteps) mbar_wait(bar0 + 8 * (buf ^ 1), (parity >> (buf ^ 1)) & 1);
      return;
    }
    parity ^= 1u << buf;

    const long long scl = s / steps_per_sc;
    const int rem = (int)(s - scl * steps_per_sc);
    const int pass = rem / nblk;
    const int blk = rem - pass * nblk;
    const long long sc = gw + scl * nW;
    const int b0 = blk * BB;
    const int bb = min(BB, B - b0);
    const int tb = pass * S::kPass;
    const int np = min(S::kPass, T - tb);
    const bool first = pass == 0;
    const unsigned char* bp = ws + buf * S::kBufBytes;
    const float2* sH = reinterpret_cast<const float2*>(bp);

    if (blk == 0) {
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int u = 0; u < UMAX; ++u) { qa[i][u][0] = 0.0f; qa[i][u][1] = 0.0f; }
#pragma unroll
      for (int i = 0; i < UMAX; ++i)
#pragma unroll
        for (int m = 0; m < GC; ++m) { ga[i][m][0] = 0.0f; ga[i][m][1] = 0.0f; }
    }

    // ---------------- GEMM over this block's antennas ----------------------
#pragma unroll 2
    for (int b = g; b < bb; b += S::kAG) {
      float2 h[UMAX];
      const float2* row = sH + b * U;
      if ((U & 1) == 0) {
#pragma unroll
        for (int u = 0; u < UMAX; u += 2) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (u < U) v = *reinterpret_cast<const float4*>(row + u);
          h[u] = make_float2(v.x, v.y);
          h[u + 1] = make_float2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int u = 0; u < UMAX; ++u) h[u] = u < U ? row[u] : make_float2(0.f, 0.f);
      }
      float2 y[TS];
#pragma unroll
      for (int i = 0; i < TS; ++i) {
        const int ts = c + S::kCG * i;
        y[i] = ts < np ? *reinterpret_cast<const float2*>(bp + S::kHBytes + ts * S::kYRow + b * 8)
                       : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int u = 0; u < UMAX; ++u) {
          // q0[t][u] += conj(h[b][u]) y[t][b]
          float re = qa[i][u][0], im = qa[i][u][1];
          re = fmaf(h[u].x, y[i].x, re);
          re = fmaf(h[u].y, y[i].y, re);
          im = fmaf(h[u].x, y[i].y, im);
          im = fmaf(-h[u].y, y[i].x, im);
          qa[i][u][0] = re;
          qa[i][u][1] = im;
        }
      if (first) {
#pragma unroll
        for (int m = 0; m < GC; ++m) {
          const int j = c + S::kCG * m;
          const float2 hj = j < U ? row[j] : make_float2(0.f, 0.f);
#pragma unroll
          for (int i = 0; i < UMAX; ++i) {
            // G[i][j] += conj(h[b][i]) h[b][j]
            float re = ga[i][m][0], im = ga[i][m][1];
            re = fmaf(h[i].x, hj.x, re);
            re = fmaf(h[i].y, hj.y, re);
            im = fmaf(h[i].x, hj.y, im);
            im = fmaf(-h[i].y, hj.x, im);
            ga[i][m][0] = re;
            ga[i][m][1] = im;
          }
        }
      }
    }
    __syncwarp();
    if (blk != nblk - 1) continue;

    // ---------------- epilogue of a pass ----------------------------------
    // (1) partial sums -> drained buffer; sum the eight antenna groups
    float* red = reinterpret_cast<float*>(ws + buf * S::kBufBytes);
    {
      float* mine = red + lane * S::kRedStride;
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int u = 0; u < UMAX; ++u) {
          mine[2 * (i * UMAX + u)] = qa[i][u][0];
          mine[2 * (i * UMAX + u) + 1] = qa[i][u][1];
        }
      if (first) {
#pragma unroll
        for (int i = 0; i < UMAX; ++i)
#pragma unroll
          for (int m = 0; m < GC; ++m) {
            mine[2 * (TS * UMAX + i * GC + m)] = ga[i][m][0];
            mine[2 * (TS * UMAX + i * GC + m) + 1] = ga[i][m][1];
          }
      }
    }
    __syncwarp();
    const int nv = first ? S::kVals : 2 * TS * UMAX;
    for (int f = lane; f < S::kCG * nv; f += 32) {
      const int cc = f / nv;
      const int v = f - cc * nv;
      float acc = 0.0f;
#pragma unroll
      for (int gg = 0; gg < S::kAG; ++gg) acc += red[(cc + S::kCG * gg) * S::kRedStride + v];
      if (v < 2 * TS * UMAX) {
        const int i = (v >> 1) / UMAX;
        const int u = (v >> 1) - i * UMAX;
        sq[2 * ((cc + S::kCG * i) * UMAX + u) + (v & 1)] = acc;
      } else {
        const int e = (v >> 1) - TS * UMAX;
        const int i = e / GC;
        const int j = cc + S::kCG * (e - i * GC);
        sg[2 * (i * UMAX + j) + (v & 1)] = acc;
      }
    }
    __syncwarp();
    // (2) preprocessing (Algorithm 1) and soft-output constants
    if (first) {
      if (lane < UMAX) {
        const float nrm = sg[2 * (lane * UMAX + lane)];
        const float den = nrm + P.alpha;
        const float dinv = (lane < U && den > 0.0f) ? 1.0f / den : 0.0f;
        const float p = dinv * nrm;
        spre[4 * lane] = dinv;
        spre[4 * lane + 1] = p;
        spre[4 * lane + 2] = nrm;
        spre[4 * lane + 3] = p > 0.0f ? 1.0f / (p * P.sqrt_es) : 0.0f;
        sg[2 * (lane * UMAX + lane) + 1] = 0.0f;  // G_uu is real
      }
      __syncwarp();
    }
    // (3) K sweeps on q: lane = kHalves * ts + hf holds users [hf*UP, hf*UP+UP)
    {
      const int ts = lane / S::kHalves;
      const int hf = lane - ts * S::kHalves;
      const bool act = ts < np;
      float qr[UP], qi[UP], zr[UP], zi[UP];
#pragma unroll
      for (int l = 0; l < UP; ++l) {
        const int j = hf * UP + l;
        qr[l] = act ? sq[2 * (ts * UMAX + j)] : 0.0f;
        qi[l] = act ? sq[2 * (ts * UMAX + j) + 1] : 0.0f;
        zr[l] = 0.0f;
        zi[l] = 0.0f;
      }
      for (int k = 0; k < P.K; ++k) {
#pragma unroll
        for (int u = 0; u < UMAX; ++u) {
          if (u < U) {
            const int lu = u % UP;         // compile-time slot of user u
            const int oh = u / UP;         // half that owns user u
            const float dinv = spre[4 * u];
            const float pu = spre[4 * u + 1];
            // z_u <- proj(d_u^-1 q_u + p_u z_u) on the owning lane
            float wr = fmaf(dinv, qr[lu], pu * zr[lu]);
            float wi = fmaf(dinv, qi[lu], pu * zi[lu]);
            project(wr, wi, P);
            float dr = wr - zr[lu];
            float di = wi - zi[lu];
            const bool own = hf == oh;
            if (own) { zr[lu] = wr; zi[lu] = wi; }
            if (S::kHalves == 2) {
              const float pr = __shfl_xor_sync(kFullMask, dr, 1);
              const float pi = __shfl_xor_sync(kFullMask, di, 1);
              if (!own) { dr = pr; di = pi; }
            }
            // q <- q - G[:, u] dz for my users
#pragma unroll
            for (int l = 0; l < UP; ++l) {
              const int j = hf * UP + l;
              const float2 gju = *reinterpret_cast<const float2*>(sg + 2 * (j * UMAX + u));
              qr[l] = fmaf(-gju.x, dr, fmaf(gju.y, di, qr[l]));
              qi[l] = fmaf(-gju.x, di, fmaf(-gju.y, dr, qi[l]));
            }
          }
        }
      }
      __syncwarp();
      if (act) {
#pragma unroll
        for (int l = 0; l < UP; ++l) {
          const int j = hf * UP + l;
          sq[2 * (ts * UMAX + j)] = zr[l];  // z overwrites q0
          sq[2 * (ts * UMAX + j) + 1] = zi[l];
        }
      }
      __syncwarp();
    }
    // (4) outputs
    for (int f = lane; f < np * U; f += 32) {
      const int ts = f / U;
      const int u = f - ts * U;
      const float2 z = make_float2(sq[2 * (ts * UMAX + u)], sq[2 * (ts * UMAX + u) + 1]);
      const long long o = (sc * T + tb + ts) * U + u;
      if (P.xhat) P.xhat[o] = z;
      if (P.llr) {
        float* out = P.llr + o * P.Q;
        const float inv = spre[4 * u + 3];
        if (!(inv > 0.0f)) {
          for (int j = 0; j < P.Q; ++j) out[j] = 0.0f;
        } else {
          const float rho = spre[4 * u + 2] * P.rho_scale;
          dimension_llr(z.x * inv, rho, P, out);
          if (!P.bpsk) dimension_llr(z.y * inv, rho, P, out + P.nb);
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace ocd
