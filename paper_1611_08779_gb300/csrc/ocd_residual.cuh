// OCD in the residual form of Algorithm 1, FP32 on the CUDA cores.
//
// Work unit ("item"): one subcarrier w and a group of S consecutive OFDM
// symbols of it (S = 1 or 2; the last group of a subcarrier may be partial).
// A team of L lanes (L a power of two, inside one warp) owns one item.  Lane
// l holds the residual entries of the contiguous antenna block
// [2*NPP*l, 2*NPP*(l+1)) of each of the S symbols in registers for the whole
// item, so r never leaves the register file between the K sweeps.
//
// A CTA walks over chunks of `chunk` consecutive items (one per team).  The
// channel columns of every subcarrier a chunk touches are staged once into
// shared memory, user-major, together with the preprocessing of Algorithm 1
// (||h_u||^2, d_u^-1, p_u); all symbols and all K sweeps reuse that copy.  In
// a staged column, lane l's block of NPP antenna pairs starts at pair slot
// l*(NPP+1): the spare slot per block puts the L lanes of a team on distinct
// banks, and every load of the sweep is base + immediate.
//
// Per (sweep k, user u) a lane loads its block of h_u once into registers and
// uses it for the S inner products h_u^H r (lane-partial FMAs, then an
// xor-butterfly over the L lanes, which leaves a bit-identical sum on every
// lane), the scalar updates with projection (Algorithm 1 update line,
// Eq. 14) and the S rank-1 residual updates r <- r - h_u dz (Eq. 15 kept
// incrementally).  z lives in shared memory (one slot per user, symbol and
// team) so the user loop stays rolled and the sweep body stays small.
#pragma once

#include "ocd_batch.cuh"
#include "ocd_common.cuh"

namespace ocd {

// Shared-memory layout of the residual kernel (all offsets in bytes).
struct ResidualSmem {
  int col_pairs;   // pair slots per staged column: L * (NPP + 1)
  int rs;          // column stride in complex elements (even)
  int sc_stride;   // subcarrier stride in complex elements (even)
  size_t h_bytes, pre_bytes, z_bytes, total;
};

__host__ __device__ inline ResidualSmem residual_smem(int L, int npp, int S, int U, int scmax,
                                                      int teams) {
  ResidualSmem s;
  s.col_pairs = L * (npp + 1);
  int rs = 2 * s.col_pairs;
  // column stride = 4 mod 16 complex: consecutive users land 8 banks apart
  rs += ((4 - rs) % 16 + 16) % 16;
  s.rs = rs;
  s.sc_stride = U * rs + 8;
  s.h_bytes = (size_t)scmax * s.sc_stride * 8;
  s.pre_bytes = (size_t)scmax * kUserSlots * 16;  // float2 (d^-1, p) + float ||h||^2 (+pad)
  s.z_bytes = (size_t)teams * S * kUserSlots * 8;
  s.total = s.h_bytes + s.pre_bytes + s.z_bytes;
  return s;
}

// One CTA pass over chunk c of problem P: the chunk's items (one per team),
// its staged channels and preprocessing.  `rezero`: clear the staging area
// first (the layout changed since the last chunk this CTA ran).
template <int NPP, int S>
__device__ __forceinline__ void residual_chunk(const DetectParams& P, long long c,
                                               unsigned char* smem_raw, bool rezero) {
  const int teams = blockDim.x >> P.logL;
  const ResidualSmem lay = residual_smem(P.L, NPP, S, P.U, P.scmax, teams);
  float2* sH = reinterpret_cast<float2*>(smem_raw);
  float2* s_dp = reinterpret_cast<float2*>(smem_raw + lay.h_bytes);            // (d^-1, p)
  float* s_nrm = reinterpret_cast<float*>(smem_raw + lay.h_bytes) + 2 * P.scmax * kUserSlots;
  float2* s_z = reinterpret_cast<float2*>(smem_raw + lay.h_bytes + lay.pre_bytes);

  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nwarps = nt >> 5;
  const int L = P.L;
  const int lt = tid & (L - 1);
  const int team = tid >> P.logL;
  const int U = P.U;
  const int B = P.B;
  const int T = P.T;
  const int G = (T + S - 1) / S;  // symbol groups per subcarrier

  // Staging geometry: a warp copies `rows` antenna rows of U entries at a time
  // (coalesced), lane -> (row my_r, user my_u); lanes past rows*U idle.
  const int rows = 32 / U;
  const int my_r = lane / U;
  const int my_u = lane - my_r * U;
  const bool stager = my_r < rows;
  const int rstep = nwarps * rows;

  float2* zt = s_z + team * S * kUserSlots;

  {
    const long long i0 = c * P.chunk;
    const long long i1 = min(i0 + (long long)P.chunk, P.items);
    const long long sc0 = i0 / G;
    const int nsc = (int)((i1 - 1) / G - sc0 + 1);

    // ---- this team's item; its Y loads are issued before the staging barrier
    const long long it = i0 + team;
    const bool active = it < i1;  // uniform across the team
    const long long sc = active ? it / G : sc0;
    const int t0 = active ? (int)(it - sc * G) * S : 0;
    const int sl = (int)(sc - sc0);

    // r = y (Algorithm 1 initialization) for the S symbols of the group
    float4 r[S][NPP];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const bool sym_ok = active && (t0 + s < T);
      const long long yrow = (sc * T + (sym_ok ? t0 + s : 0)) * (long long)B;
      const int p0 = lt * NPP;
#pragma unroll
      for (int j = 0; j < NPP; ++j) {
        const int b0 = 2 * (p0 + j);
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (sym_ok) {
          if (P.vec_y) {
            if (b0 < B) v = load_c2(P.Y, yrow + b0, P.storage);
          } else {
            if (b0 < B) { const float2 a = load_c(P.Y, yrow + b0, P.storage); v.x = a.x; v.y = a.y; }
            if (b0 + 1 < B) {
              const float2 a = load_c(P.Y, yrow + b0 + 1, P.storage);
              v.z = a.x;
              v.w = a.y;
            }
          }
        }
        r[s][j] = v;
      }
    }

    __syncthreads();  // the previous chunk is no longer being read
    if (rezero) {
      // spare slots and antennas >= B stay zero while the layout is kept:
      // staging only ever writes the slots of antennas < B
      for (int i = tid; i < P.scmax * lay.sc_stride; i += nt) sH[i] = make_float2(0.0f, 0.0f);
      __syncthreads();
    }
    // ---- stage H[sc0 .. sc0+nsc) as user-major columns (8 loads in flight) --
    if (stager) {
      for (int s = 0; s < nsc; ++s) {
        const long long gH = (sc0 + s) * (long long)B * U + my_u;
        float2* col = sH + s * lay.sc_stride + my_u * lay.rs;
        for (int b0 = warp * rows + my_r; b0 < B; b0 += 8 * rstep) {
          float2 v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int b = b0 + q * rstep;
            if (b < B) v[q] = load_c(P.H, gH + (long long)b * U, P.storage);
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int b = b0 + q * rstep;
            if (b < B) {
              const int pp = b >> 1;
              const int slot = (pp / NPP) * (NPP + 1) + (pp & (NPP - 1));
              col[2 * slot + (b & 1)] = v[q];
            }
          }
        }
      }
    }
    __syncthreads();
    // ---- preprocessing (Algorithm 1): ||h_u||^2, d_u^-1, p_u ---------------
    for (int q = warp; q < nsc * U; q += nwarps) {
      const int s = q / U;
      const int u = q - s * U;
      const float2* col = sH + s * lay.sc_stride + u * lay.rs;
      float acc = 0.0f;
      for (int i = lane; i < 2 * lay.col_pairs; i += 32) {
        const float2 h = col[i];
        acc = fmaf(h.x, h.x, fmaf(h.y, h.y, acc));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFullMask, acc, o);
      if (lane == 0) {
        const float den = acc + P.alpha;
        const float dinv = den > 0.0f ? 1.0f / den : 0.0f;
        s_dp[s * kUserSlots + u] = make_float2(dinv, dinv * acc);
        s_nrm[s * kUserSlots + u] = acc;
      }
    }
    for (int u = lt; u < U; u += L) {
#pragma unroll
      for (int s = 0; s < S; ++s) zt[s * kUserSlots + u] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();

    const float4* hlane = reinterpret_cast<const float4*>(sH + sl * lay.sc_stride) + lt * (NPP + 1);
    const float2* dp = s_dp + sl * kUserSlots;
    const int rs4 = lay.rs >> 1;  // column stride in float4

    for (int k = 0; k < P.K; ++k) {
      const bool last_sweep = k == P.K - 1;
#pragma unroll 2
      for (int u = 0; u < U; ++u) {
        const float4* hc = hlane + u * rs4;
        const float2 dpu = dp[u];
        float4 h[NPP];
#pragma unroll
        for (int j = 0; j < NPP; ++j) h[j] = hc[j];
        float cr[S], ci[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          // eight independent chains: even/odd pairs x two antennas x (re, im)
          float ar[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          float ai[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
          for (int j = 0; j < NPP; ++j) {
            const int a = (j & 1) * 2;
            // conj(h) * r for the two antennas of the pair
            ar[a] = fmaf(h[j].x, r[s][j].x, ar[a]);
            ar[a] = fmaf(h[j].y, r[s][j].y, ar[a]);
            ai[a] = fmaf(h[j].x, r[s][j].y, ai[a]);
            ai[a] = fmaf(-h[j].y, r[s][j].x, ai[a]);
            ar[a + 1] = fmaf(h[j].z, r[s][j].z, ar[a + 1]);
            ar[a + 1] = fmaf(h[j].w, r[s][j].w, ar[a + 1]);
            ai[a + 1] = fmaf(h[j].z, r[s][j].w, ai[a + 1]);
            ai[a + 1] = fmaf(-h[j].w, r[s][j].z, ai[a + 1]);
          }
          cr[s] = (ar[0] + ar[1]) + (ar[2] + ar[3]);
          ci[s] = (ai[0] + ai[1]) + (ai[2] + ai[3]);
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          if (o >= L) break;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            cr[s] += __shfl_xor_sync(kFullMask, cr[s], o);
            ci[s] += __shfl_xor_sync(kFullMask, ci[s], o);
          }
        }
        const bool skip_update = last_sweep && u == U - 1;
#pragma unroll
        for (int s = 0; s < S; ++s) {
          // z_u <- proj(d_u^-1 h_u^H r + p_u z_u); dz = z_new - z_old
          const float2 zu = zt[s * kUserSlots + u];
          float wr = fmaf(dpu.x, cr[s], dpu.y * zu.x);
          float wi = fmaf(dpu.x, ci[s], dpu.y * zu.y);
          project(wr, wi, P);
          const float dr = wr - zu.x;
          const float di = wi - zu.y;
          zt[s * kUserSlots + u] = make_float2(wr, wi);  // every team lane stores the same value
          // r <- r - h_u dz (not needed after the last update of the last sweep)
          if (!skip_update) {
#pragma unroll
            for (int j = 0; j < NPP; ++j) {
              r[s][j].x = fmaf(-h[j].x, dr, fmaf(h[j].y, di, r[s][j].x));
              r[s][j].y = fmaf(-h[j].x, di, fmaf(-h[j].y, dr, r[s][j].y));
              r[s][j].z = fmaf(-h[j].z, dr, fmaf(h[j].w, di, r[s][j].z));
              r[s][j].w = fmaf(-h[j].z, di, fmaf(-h[j].w, dr, r[s][j].w));
            }
          }
        }
      }
    }
    __syncwarp();

    // ---- outputs: (symbol, user) pairs are spread over the team's lanes ------
    if (active) {
      const float* nrm = s_nrm + sl * kUserSlots;
      for (int q = lt; q < S * U; q += L) {
        const int s = q / U;
        const int u = q - s * U;
        const int t = t0 + s;
        if (t < T) {
          const float2 z = zt[s * kUserSlots + u];
          const long long o = (sc * T + t) * U + u;
          if (P.xhat) P.xhat[o] = z;
          if (P.llr) user_llr(z, nrm[u], dp[u].y, P, P.llr + o * P.Q);
        }
      }
    }
  }
}

// Single problem: CTA b takes chunks b, b + gridDim.x, ...
template <int NPP, int S>
__global__ void __launch_bounds__(128, 3)
ocd_residual_kernel(const __grid_constant__ DetectParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long nchunks = (P.items + P.chunk - 1) / P.chunk;
  for (long long c = blockIdx.x; c < nchunks; c += gridDim.x)
    residual_chunk<NPP, S>(P, c, smem_raw, c == blockIdx.x);
}

// Several problems in one persistent launch: each CTA draws tickets (one
// chunk of one cell each) from a device counter; tickets of cell c are
// [tick_end[c-1], tick_end[c]).  Cells of one launch share NPP, S and the
// block size; the staging layout is rebuilt when a CTA moves to a new cell.
template <int NPP, int S>
__global__ void __launch_bounds__(128, 3)
ocd_batched_residual_kernel(const __grid_constant__ BatchTable tab,
                            unsigned int* __restrict__ tickets) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned int s_ticket;
  int c = 0, last = -1;
  for (;;) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(tickets, 1u);
    __syncthreads();
    const unsigned int tk = s_ticket;
    // every thread has read s_ticket before thread 0 can overwrite it: the
    // chunk below passes further barriers, and the exit is uniform
    if (tk >= tab.total) return;
    while (tk >= tab.cell[c].tick_end) ++c;  // a CTA's tickets increase
    const long long t0 = c ? tab.cell[c - 1].tick_end : 0;
    residual_chunk<NPP, S>(tab.cell[c].P, (long long)tk - t0, smem_raw, c != last);
    last = c;
  }
}

}  // namespace ocd
