// OCD with the residual carried in projected form, FP32 on the CUDA cores.
//
// Algorithm 1 only ever reads the residual r through the inner products
// h_u^H r.  Carrying q = H^H r (U values) instead of r (B values) gives the
// same iterates in exact arithmetic:
//     initialization  r = y            ->  q = H^H y
//     update          z_u <- proj(d_u^-1 h_u^H r + p_u z_u)
//                                     ->  z_u <- proj(d_u^-1 q_u + p_u z_u)
//     residual        r <- r - h_u dz  ->  q <- q - G[:, u] dz,  G = H^H H
// The length-B work moves into two small dense products per subcarrier,
// q0 = H^H Y^T and G, which all T symbols and all K sweeps share; the sweeps
// themselves cost 4U real FMAs per user update instead of 8B.
//
// One warp owns one subcarrier at a time (persistent over subcarriers).
//   GEMM phase: lane = c + 4 g with antenna group g (0..7) and column group c
//     (0..3).  Lane (g, c) walks the antenna pairs g, g+8, g+16, ... and
//     accumulates q0 for the symbols c, c+4, c+8, ... of the current symbol
//     pass (TS = 32/UMAX of them) and the columns c, c+4, ... of G (both
//     triangles, so every lane runs the same code).  H rows and Y pairs are
//     read with vector loads straight from global memory (this variant
//     serves shapes the bulk-copy variant cannot stage: odd B, unaligned
//     bases).
//   Reduction: the eight antenna-group partials are summed through shared
//     memory (fixed order, g = 0..7).
//   Sweeps: one lane per symbol runs the K round-robin sweeps on q with z in
//     registers and G (full Hermitian) read from shared memory.
//   Soft output: (symbol, user) pairs spread over all lanes (Eq. 9).
#pragma once

#include "ocd_common.cuh"

namespace ocd {

template <int UMAX>
struct ProjectedShape {
  static constexpr int kAG = 8;                       // antenna groups
  static constexpr int kCG = 4;                       // column groups
  static constexpr int kTS = 32 / UMAX;               // symbols per lane per pass
  static constexpr int kPass = kCG * kTS;             // symbols per pass
  static constexpr int kGC = UMAX / kCG;              // G columns per lane (j = c + 4 m)
  static constexpr int kVals = 2 * (kTS * UMAX + UMAX * kGC);  // partial floats per lane
  static constexpr int kRedStride = ((kVals + 3) / 4) * 4 + 4;  // per-lane stride (floats)
  // per-warp shared memory (floats)
  static constexpr int kRed = 32 * kRedStride;        // partials [lane][kRedStride]
  static constexpr int kQ = 2 * kPass * UMAX;         // reduced q0 [pass symbol][u]
  static constexpr int kG = 2 * UMAX * UMAX;          // full G [i][j]
  static constexpr int kZ = 2 * kPass * UMAX;         // z [pass symbol][u]
  static constexpr int kPre = 4 * UMAX;               // (d^-1, p, ||h||^2, -) per user
  static constexpr int kWarpFloats = kRed + kQ + kG + kZ + kPre;
};

template <int UMAX>
__global__ void __launch_bounds__(128, 3)
ocd_projected_kernel(const DetectParams P) {
  using S = ProjectedShape<UMAX>;
  constexpr int TS = S::kTS;
  constexpr int GC = S::kGC;
  extern __shared__ __align__(16) float smem_f[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  float* ws = smem_f + warp * S::kWarpFloats;
  float* red = ws;
  float* sq = red + S::kRed;
  float* sg = sq + S::kQ;
  float* sz = sg + S::kG;
  float* spre = sz + S::kZ;

  const int U = P.U;
  const int B = P.B;
  const int T = P.T;
  const int c = lane & 3;
  const int g = lane >> 2;
  const int pairs = (B + 1) >> 1;
  const long long nwarps_total = (long long)gridDim.x * (blockDim.x >> 5);
  const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  const bool vec_h = (U % 2 == 0) &&
                     ((reinterpret_cast<uintptr_t>(P.H) & (P.storage == kStoreC64 ? 15u : 7u)) == 0);

  for (long long sc = gw; sc < P.Nsc; sc += nwarps_total) {
    const long long hbase = sc * (long long)B * U;
    const long long ybase = sc * (long long)T * B;

    for (int tb = 0; tb < T; tb += S::kPass) {
      const bool first = tb == 0;
      // ---------------- GEMM phase: partial q0 and G over my antennas -------
      float qa[TS][UMAX][2];
      float ga[UMAX][GC][2];
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int u = 0; u < UMAX; ++u) { qa[i][u][0] = 0.0f; qa[i][u][1] = 0.0f; }
#pragma unroll
      for (int i = 0; i < UMAX; ++i)
#pragma unroll
        for (int m = 0; m < GC; ++m) { ga[i][m][0] = 0.0f; ga[i][m][1] = 0.0f; }

      for (int p = g; p < pairs; p += S::kAG) {
        const int b0 = 2 * p;
        const bool ok1 = b0 + 1 < B;
        // two channel rows h[b0][.], h[b0+1][.] (zero beyond U or B)
        float2 h0[UMAX], h1[UMAX];
        {
          const long long r0 = hbase + (long long)b0 * U;
          const long long r1 = r0 + U;
          if (vec_h) {
#pragma unroll
            for (int u = 0; u < UMAX; u += 2) {
              float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
              if (u < U) {
                a = load_c2(P.H, r0 + u, P.storage);
                if (ok1) b = load_c2(P.H, r1 + u, P.storage);
              }
              h0[u] = make_float2(a.x, a.y); h0[u + 1] = make_float2(a.z, a.w);
              h1[u] = make_float2(b.x, b.y); h1[u + 1] = make_float2(b.z, b.w);
            }
          } else {
#pragma unroll
            for (int u = 0; u < UMAX; ++u) {
              h0[u] = u < U ? load_c(P.H, r0 + u, P.storage) : make_float2(0.f, 0.f);
              h1[u] = (u < U && ok1) ? load_c(P.H, r1 + u, P.storage) : make_float2(0.f, 0.f);
            }
          }
        }
        // received pairs y[t][b0], y[t][b0+1] for my symbols of this pass
        float4 yv[TS];
#pragma unroll
        for (int i = 0; i < TS; ++i) {
          const int t = tb + c + S::kCG * i;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (t < T) {
            const long long yr = ybase + (long long)t * B + b0;
            if (P.vec_y) {
              v = load_c2(P.Y, yr, P.storage);
            } else {
              const float2 a = load_c(P.Y, yr, P.storage);
              v.x = a.x; v.y = a.y;
              if (ok1) { const float2 b = load_c(P.Y, yr + 1, P.storage); v.z = b.x; v.w = b.y; }
            }
          }
          yv[i] = v;
        }
        // q0[t][u] += conj(h[b][u]) y[t][b]
#pragma unroll
        for (int i = 0; i < TS; ++i)
#pragma unroll
          for (int u = 0; u < UMAX; ++u) {
            float re = qa[i][u][0], im = qa[i][u][1];
            re = fmaf(h0[u].x, yv[i].x, re); re = fmaf(h0[u].y, yv[i].y, re);
            im = fmaf(h0[u].x, yv[i].y, im); im = fmaf(-h0[u].y, yv[i].x, im);
            re = fmaf(h1[u].x, yv[i].z, re); re = fmaf(h1[u].y, yv[i].w, re);
            im = fmaf(h1[u].x, yv[i].w, im); im = fmaf(-h1[u].y, yv[i].z, im);
            qa[i][u][0] = re; qa[i][u][1] = im;
          }
        // G[i][j] += conj(h[b][i]) h[b][j] for my columns j = c + 4 m
        if (first) {
#pragma unroll
          for (int m = 0; m < GC; ++m) {
            float2 s0 = h0[S::kCG * m], s1 = h1[S::kCG * m];
#pragma unroll
            for (int q = 1; q < S::kCG; ++q) {
              if (c == q) { s0 = h0[q + S::kCG * m]; s1 = h1[q + S::kCG * m]; }
            }
#pragma unroll
            for (int i = 0; i < UMAX; ++i) {
              float re = ga[i][m][0], im = ga[i][m][1];
              re = fmaf(h0[i].x, s0.x, re); re = fmaf(h0[i].y, s0.y, re);
              im = fmaf(h0[i].x, s0.y, im); im = fmaf(-h0[i].y, s0.x, im);
              re = fmaf(h1[i].x, s1.x, re); re = fmaf(h1[i].y, s1.y, re);
              im = fmaf(h1[i].x, s1.y, im); im = fmaf(-h1[i].y, s1.x, im);
              ga[i][m][0] = re; ga[i][m][1] = im;
            }
          }
        }
      }

      // ---------------- reduction over the eight antenna groups -------------
      {
        float* mine = red + lane * S::kRedStride;
#pragma unroll
        for (int i = 0; i < TS; ++i)
#pragma unroll
          for (int u = 0; u < UMAX; ++u) {
            mine[2 * (i * UMAX + u)] = qa[i][u][0];
            mine[2 * (i * UMAX + u) + 1] = qa[i][u][1];
          }
#pragma unroll
        for (int i = 0; i < UMAX; ++i)
#pragma unroll
          for (int m = 0; m < GC; ++m) {
            mine[2 * (TS * UMAX + i * GC + m)] = ga[i][m][0];
            mine[2 * (TS * UMAX + i * GC + m) + 1] = ga[i][m][1];
          }
      }
      __syncwarp();
      // value slot v of column group cc lives at red[(cc + 4 g) * stride + v]
      for (int f = lane; f < S::kCG * S::kVals; f += 32) {
        const int cc = f / S::kVals;
        const int v = f - cc * S::kVals;
        float acc = 0.0f;
#pragma unroll
        for (int gg = 0; gg < S::kAG; ++gg) acc += red[(cc + S::kCG * gg) * S::kRedStride + v];
        if (v < 2 * TS * UMAX) {
          // q0 of pass symbol (cc + 4 i), user u
          const int i = (v >> 1) / UMAX;
          const int u = (v >> 1) - i * UMAX;
          sq[2 * ((cc + S::kCG * i) * UMAX + u) + (v & 1)] = acc;
        } else if (first) {
          // G[i][j], j = cc + 4 m
          const int e = (v >> 1) - TS * UMAX;
          const int i = e / GC;
          const int j = cc + S::kCG * (e - i * GC);
          sg[2 * (i * UMAX + j) + (v & 1)] = acc;
        }
      }
      __syncwarp();
      if (first) {
        // ---- preprocessing (Algorithm 1): ||h_u||^2 = G_uu, d_u^-1, p_u ----
        if (lane < UMAX) {
          const float nrm = sg[2 * (lane * UMAX + lane)];
          const float den = nrm + P.alpha;
          const float dinv = (lane < U && den > 0.0f) ? 1.0f / den : 0.0f;
          spre[4 * lane] = dinv;
          spre[4 * lane + 1] = dinv * nrm;
          spre[4 * lane + 2] = nrm;
          // the diagonal of the stored G must be real
          sg[2 * (lane * UMAX + lane) + 1] = 0.0f;
        }
        __syncwarp();
      }

      // ---------------- sweeps: one lane per symbol of the pass ------------
      const int t = tb + lane;
      if (lane < S::kPass && t < T) {
        float qr[UMAX], qi[UMAX], zr[UMAX], zi[UMAX];
#pragma unroll
        for (int u = 0; u < UMAX; ++u) {
          qr[u] = sq[2 * (lane * UMAX + u)];
          qi[u] = sq[2 * (lane * UMAX + u) + 1];
          zr[u] = 0.0f;
          zi[u] = 0.0f;
        }
        for (int k = 0; k < P.K; ++k) {
#pragma unroll
          for (int u = 0; u < UMAX; ++u) {
            if (u < U) {
              const float dinv = spre[4 * u];
              const float pu = spre[4 * u + 1];
              // z_u <- proj(d_u^-1 q_u + p_u z_u)
              float wr = fmaf(dinv, qr[u], pu * zr[u]);
              float wi = fmaf(dinv, qi[u], pu * zi[u]);
              project(wr, wi, P);
              const float dr = wr - zr[u];
              const float di = wi - zi[u];
              zr[u] = wr;
              zi[u] = wi;
              // q <- q - G[:, u] dz
#pragma unroll
              for (int j = 0; j < UMAX; ++j) {
                const float2 gju = *reinterpret_cast<const float2*>(sg + 2 * (j * UMAX + u));
                qr[j] = fmaf(-gju.x, dr, fmaf(gju.y, di, qr[j]));
                qi[j] = fmaf(-gju.x, di, fmaf(-gju.y, dr, qi[j]));
              }
            }
          }
        }
#pragma unroll
        for (int u = 0; u < UMAX; ++u) {
          sz[2 * (lane * UMAX + u)] = zr[u];
          sz[2 * (lane * UMAX + u) + 1] = zi[u];
        }
      }
      __syncwarp();

      // ---------------- outputs --------------------------------------------
      const int npass = min(S::kPass, T - tb);
      for (int f = lane; f < npass * U; f += 32) {
        const int ts = f / U;
        const int u = f - ts * U;
        const float2 z = make_float2(sz[2 * (ts * UMAX + u)], sz[2 * (ts * UMAX + u) + 1]);
        const long long o = (sc * T + tb + ts) * U + u;
        if (P.xhat) P.xhat[o] = z;
        if (P.llr) user_llr(z, spre[4 * u + 2], spre[4 * u + 1], P, P.llr + o * P.Q);
      }
      __syncwarp();
    }
  }
}

}  // namespace ocd
